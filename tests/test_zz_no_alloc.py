"""qed_step_static -- the step for callers that cannot allocate device memory when they
step (stream capture, host applications that own all device memory) -- must give the
same particles as qed_step, call after call, and allocate nothing.

Two contexts evolve the same particles: one with qed_step, one with qed_step_static.
After a few ordinary steps (so that photons exist and pairs can be made), two calls in a
row of each are compared particle by particle, within the tolerance of the other parity
tests (1e-10 on the FP64 path, 2e-5 on the mixed path)."""
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

ALL = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN


def _workload():
    wl = workloads.c2(n=600, seed=77)
    shift = 9.0 * math.pi
    wl["e"]["z"] = wl["e"]["z"] + shift
    wl["t0"] = shift
    wl["step0"] = 900
    return wl


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _same(a, b, tol):
    assert a["next_id"] == b["next_id"]
    for sp in ("e", "pos", "ph"):
        x, y = _by_id(a[sp]), _by_id(b[sp])
        assert np.array_equal(x["id"], y["id"]), sp
        for k in ("px", "py", "pz", "s1", "s2", "s3"):
            scale = np.maximum(np.abs(y[k]), 1.0)
            assert np.all(np.abs(x[k] - y[k]) <= tol * scale), (sp, k)
        for k in ("x", "y", "z"):
            assert np.all(np.abs(x[k] - y[k]) <= tol * (np.abs(y[k]) + 1.0)), (sp, k)


@pytest.mark.parametrize("prec,tol", [(q.QED_PREC_F64, 1e-10), (q.QED_PREC_MIXED, 2e-5)])
def test_static_scratch_step_matches_qed_step(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    caps = dict(cap_e=8192, cap_p=8192, cap_ph=32768)
    ref = q.Simulation(_workload(), prec=prec, **caps)
    sta = q.Simulation(_workload(), prec=prec, **caps)
    ref.run(40, ALL)
    sta.run(40, ALL)
    torch.cuda.synchronize()
    assert sta.ph.count() > 100
    for call in range(2):
        q.qed_step(ref.ctx, ref.e.handle, ref.pos.handle, ref.ph.handle, ref.fields, ref.t, ref.dt, ref.seed,
                   ref.step_no, ALL, ref.stats.data_ptr())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        q.qed_step_static(sta.ctx, sta.e.handle, sta.pos.handle, sta.ph.handle, sta.fields, sta.t, sta.dt,
                          sta.seed, sta.step_no, ALL, sta.stats.data_ptr())
        torch.cuda.synchronize()
        if call == 1:   # the first call on a device may load the library's static array
            assert torch.cuda.mem_get_info()[0] == free_before
        for s in (ref, sta):
            s.t += s.dt
            s.step_no += 1
        _same(sta.state(), ref.state(), tol)
    assert sta.counters()["n_ncs_e"] == ref.counters()["n_ncs_e"] > 0
    assert sta.status() == 0 and ref.status() == 0
    ref.close()
    sta.close()


def test_static_scratch_step_rejects_large_sets():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    big = q.Simulation(_workload(), prec=q.QED_PREC_MIXED, cap_e=8192, cap_p=8192, cap_ph=65537)
    with pytest.raises(q.QedError, match="exceeds the limit"):
        q.qed_step_static(big.ctx, big.e.handle, big.pos.handle, big.ph.handle, big.fields, big.t, big.dt,
                          big.seed, big.step_no, ALL)
    big.close()


def _static_step(s):
    q.qed_step_static(s.ctx, s.e.handle, s.pos.handle, s.ph.handle, s.fields, s.t, s.dt, s.seed, s.step_no, ALL,
                      s.stats.data_ptr(), torch.cuda.current_stream().cuda_stream)
    s.t += s.dt
    s.step_no += 1


def _plain_step(s):
    q.qed_step(s.ctx, s.e.handle, s.pos.handle, s.ph.handle, s.fields, s.t, s.dt, s.seed, s.step_no, ALL,
               s.stats.data_ptr(), torch.cuda.current_stream().cuda_stream)
    s.t += s.dt
    s.step_no += 1


def test_static_scratch_at_its_capacity_limit():
    """Every species at the 65,536 limit, most tiles live: the whole tile-count region and the
    logs' full extent are in use; the static step equals qed_step and nothing is dropped."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    # about a quarter of the leptons emit per step at this field: 30k photons become ~61k
    wl = workloads.crossed(ne=30000, npos=30000, nph=30000, E0=60.0, seed=6)
    caps = dict(cap_e=65536, cap_p=65536, cap_ph=65536)
    ref = q.Simulation(wl, prec=q.QED_PREC_F64, **caps)
    sta = q.Simulation(wl, prec=q.QED_PREC_F64, **caps)
    for _ in range(2):
        _plain_step(ref)
        _static_step(sta)
    torch.cuda.synchronize()
    assert sta.ph.count() > 55000 and sta.e.count() > 30000
    _same(sta.state(), ref.state(), 1e-10)
    for s in (ref, sta):
        assert not s.status() & q.QED_STATUS_CAPACITY
        assert s.counters()["n_nbw"] > 0
    ref.close()
    sta.close()


def test_static_scratch_step_in_a_captured_graph():
    """A warm-up call outside capture, then two qed_step_static calls captured into a CUDA
    graph on a side stream and replayed: the particles equal two plain qed_step calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    caps = dict(cap_e=8192, cap_p=8192, cap_ph=32768)
    ref = q.Simulation(_workload(), prec=q.QED_PREC_F64, **caps)
    sta = q.Simulation(_workload(), prec=q.QED_PREC_F64, **caps)
    ref.run(30, ALL)
    sta.run(30, ALL)
    _plain_step(ref)
    _static_step(sta)                      # the first call: outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    t0, s0 = sta.t, sta.step_no
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            _static_step(sta)
            _static_step(sta)
    sta.t, sta.step_no = t0, s0            # capture ran nothing: replay does the two steps
    g.replay()
    torch.cuda.synchronize()
    _plain_step(ref)
    _plain_step(ref)
    torch.cuda.synchronize()
    _same(sta.state(), ref.state(), 1e-10)
    assert sta.status() == 0
    ref.close()
    sta.close()
