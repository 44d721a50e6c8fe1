"""Sharded steps on the GPU (qed_step_begin / qed_step_end) through the C ABI.

Two ranks are emulated on one GPU by two contexts that step one half of a population
each; their kernels never wait on one another (each half runs to its counts, the counts
are stacked, then each half finishes).  Checked against the oracle stepping the whole
population with, before every step, its particles in the ranks' order (rank 0's, then
rank 1's): ids and the id counter exactly, FP64 values to 1e-10.  One rank alone equals
qed_step bit for bit; a rank handed counts that are not its own sets QED_STATUS_SHARD;
misuse is rejected on the host."""
import numpy as np
import pytest

import oracle
import shard_cases
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

FLAGS = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN
CAPS = {"cap_e": 8192, "cap_p": 8192, "cap_ph": 16384}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _ids(sim):
    st = sim.state()
    return {sp: st[sp]["id"] for sp in shard_cases.SPECIES}


@pytest.mark.parametrize("prec,tol", [(q.QED_PREC_F64, 1e-10)])
def test_two_shards_equal_one_population_in_rank_order(orc, ctx, prec, tol):
    wl = workloads.crossed(seed=3)
    shards = [q.Simulation(workloads.shard(wl, r, 2), prec=prec, ctx=q.qed_ctx_share(ctx), **CAPS) for r in range(2)]
    ref = oracle.Sim(orc, wl, **CAPS)
    stats = {}
    for _ in range(6):
        order = [_ids(s) for s in shards]
        ref.load(shard_cases.rank_order(ref.state(), {sp: [o[sp] for o in order] for sp in shard_cases.SPECIES}))
        for k, v in ref.run(1, FLAGS).items():
            stats[k] = stats.get(k, 0) + v
        counts = [s.step_begin(FLAGS) for s in shards]
        allc = torch.stack(counts)
        for r, s in enumerate(shards):
            s.step_end(allc, r, 2)
    torch.cuda.synchronize()
    states = [s.state() for s in shards]
    assert states[0]["next_id"] == states[1]["next_id"]
    shard_cases.assert_same(shard_cases.union(states), ref.state(), tol)
    got = [s.counters() for s in shards]
    for key in ("n_nbw", "n_ncs_e", "n_ncs_p"):
        assert got[0][key] + got[1][key] == stats[key] > 0, key
    for s in shards:
        assert s.status() == 0
        s.close()
        q.qed_destroy(s.ctx)


def test_one_rank_is_qed_step(ctx):
    wl = workloads.crossed(seed=4)
    a = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=q.qed_ctx_share(ctx), **CAPS)
    b = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=q.qed_ctx_share(ctx), **CAPS)
    a.run(5, FLAGS)
    for _ in range(5):
        c = b.step_begin(FLAGS)
        b.step_end(c.reshape(1, 3), 0, 1)
    sa, sb = a.state(), b.state()
    for sp in shard_cases.SPECIES:
        for k in sa[sp]:
            assert np.array_equal(sa[sp][k], sb[sp][k]), (sp, k)
    assert sa["next_id"] == sb["next_id"] and a.counters() == b.counters()
    for s in (a, b):
        s.close()
        q.qed_destroy(s.ctx)


def test_foreign_counts_and_misuse(ctx):
    sim = q.Simulation(workloads.crossed(seed=5, ne=64, npos=32, nph=64), prec=q.QED_PREC_F64,
                       ctx=q.qed_ctx_share(ctx), **CAPS)
    with pytest.raises(q.QedError, match="no step begun"):
        sim.step_end(torch.zeros(1, 3, dtype=torch.int64, device="cuda"), 0, 1)
    c = sim.step_begin(FLAGS)
    with pytest.raises(q.QedError, match="sharded step"):
        sim.run(1, FLAGS)                       # no plain step while one is open
    with pytest.raises(q.QedError, match="rank"):
        sim.step_end(torch.stack([c, c]), 2, 2)
    wrong = torch.stack([c, c + 1])             # rank 1's place holds counts not its own
    sim.step_end(wrong, 1, 2)
    assert sim.status() & q.QED_STATUS_SHARD
    sim.status(clear=True)
    c = sim.step_begin(FLAGS)                   # the context is usable again
    sim.step_end(c.reshape(1, 3), 0, 1)
    assert sim.status() == 0
    sim.close()
    q.qed_destroy(sim.ctx)


def test_three_shards_one_empty_mixed_equal_one_context(ctx):
    """Mixed path, three ranks, the middle one holding no particle at all: the shards' union
    equals one context stepping the whole population in the ranks' order (GPU against
    GPU, the same arithmetic: bit for bit), and the counter is every rank's."""
    wl = workloads.crossed(seed=7, ne=300, npos=150, nph=400)
    empty = {sp: {k: v[:0] for k, v in wl[sp].items()} for sp in shard_cases.SPECIES}
    parts = [workloads.shard(wl, 0, 2), dict(wl, **empty), workloads.shard(wl, 1, 2)]
    shards = [q.Simulation(p, prec=q.QED_PREC_MIXED, ctx=q.qed_ctx_share(ctx), **CAPS) for p in parts]
    ref = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=q.qed_ctx_share(ctx), **CAPS)
    for _ in range(6):
        order = [_ids(s) for s in shards]
        st = shard_cases.rank_order(ref.state(), {sp: [o[sp] for o in order] for sp in shard_cases.SPECIES})
        for sp in shard_cases.SPECIES:
            getattr(ref, sp).load(st[sp])
        ref.run(1, FLAGS)
        counts = [s.step_begin(FLAGS) for s in shards]
        allc = torch.stack(counts)
        for r, s in enumerate(shards):
            s.step_end(allc, r, 3)
    torch.cuda.synchronize()
    states = [s.state() for s in shards]
    assert len({st["next_id"] for st in states}) == 1
    want = ref.state()
    shard_cases.assert_same(shard_cases.union(states), want, 0.0)
    assert states[1]["e"]["id"].size == 0 and states[1]["ph"]["id"].size == 0
    c = [s.counters() for s in shards]
    assert sum(x["n_nbw"] for x in c) == ref.counters()["n_nbw"] > 0
    for s in shards + [ref]:
        assert s.status() == 0
        s.close()
        q.qed_destroy(s.ctx)
