"""qed_step_host -- the step for particles held in host memory (the end-to-end entry point:
copies in, step, copies out) -- against qed_step on device-resident copies of the same
particles: identical arrays, bit for bit, over several steps in both precisions (the
copies move bytes and the kernels are the same), and the host counts follow the births
and decays."""
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

ALL = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _host_sets(sim):
    """pinned host copies of the three device sets (full capacity), as qed_soa views"""
    soas, keep = [], []
    for sp in (sim.e, sim.pos, sim.ph):
        soa = q.qed_soa()
        d = {}
        for k, v in sp.t.items():
            h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
            h.copy_(v)
            d[k] = h
            setattr(soa, k, h.data_ptr())
        soas.append(soa)
        keep.append(d)
    return soas, keep


@pytest.mark.parametrize("prec", [q.QED_PREC_MIXED, q.QED_PREC_F64])
def test_host_step_equals_device_step(ctx, prec):
    wl = workloads.c2(n=4000, seed=71)
    shift = 9.0 * math.pi
    wl["e"]["z"] = wl["e"]["z"] + shift
    wl["t0"] = shift
    wl["step0"] = 900
    caps = dict(cap_e=30000, cap_p=30000, cap_ph=300000)
    dev = q.Simulation(wl, prec=prec, ctx=ctx, **caps)
    hst = q.Simulation(wl, prec=prec, ctx=q.qed_ctx_share(ctx), **caps)
    soas, keep = _host_sets(hst)
    counts = [hst.e.count(), hst.pos.count(), hst.ph.count()]
    for _ in range(30):
        dev.run(1, ALL)
        counts = q.qed_step_host(hst.ctx, hst.e.handle, hst.pos.handle, hst.ph.handle, soas[0], soas[1], soas[2],
                                 counts, hst.fields, hst.t, hst.dt, hst.seed, hst.step_no, ALL)
        hst.t += hst.dt
        hst.step_no += 1
    ref = dev.state()
    assert counts == [len(ref["e"]["id"]), len(ref["pos"]["id"]), len(ref["ph"]["id"])]
    assert counts[1] > 0 and counts[2] > 0
    for k, sp in enumerate(("e", "pos", "ph")):
        n = counts[k]
        for name, h in keep[k].items():
            a = h[:n].numpy()
            b = ref[sp][name]
            a = a.view(np.uint64) if name == "id" else a.astype(np.float64)
            assert np.array_equal(a, b), (sp, name)
    assert q.qed_get_next_id(hst.ctx) == ref["next_id"]
    c = hst.ctx
    dev.close()
    hst.close()
    q.qed_destroy(c)
