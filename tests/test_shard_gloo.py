"""Two gloo ranks step one population, each its own half, and exchange only the step's
birth counts (paper_2306_11288_gb300.shard_exchange, the all-gather the GPU step uses
between qed_step_begin and qed_step_end); the oracle is the stepping engine of each rank.
At the end the photon-energy histogram is summed over the ranks
(paper_2306_11288_gb300.allreduce_hist).

Checked against one process stepping the whole population with, before every step, its
particles in the ranks' order: every particle and every id identical (bit for bit), the
same id counter, and the summed histogram equal to the whole population's."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
STEPS = 5
EDGES = np.geomspace(1.0, 1e4, 25)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _energy(ph):
    return np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path[:0] = [ROOT, HERE]
    import oracle
    import paper_2306_11288_gb300 as q
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    flags = oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN
    sim = oracle.Sim(oracle.Oracle(), workloads.shard(workloads.crossed(), rank, world))
    order = []   # per step: every rank's ids of each species before the step
    for _ in range(STEPS):
        st = sim.state()
        mine = {sp: st[sp]["id"] for sp in ("e", "pos", "ph")}
        every = [None] * world
        dist.all_gather_object(every, mine)
        order.append({sp: [every[r][sp] for r in range(world)] for sp in mine})
        cnt, _ = sim.decide(flags)
        allc = q.shard_exchange(torch.as_tensor(cnt.astype(np.int64)))
        assert tuple(allc.shape) == (world, 3)
        sim.commit(oracle.shard_bases(sim.o.next_id(), allc.numpy(), rank))
    st = sim.state()
    states = [None] * world
    dist.all_gather_object(states, st)
    h = torch.as_tensor(np.histogram(_energy(st["ph"]), EDGES)[0].astype(np.float64))
    q.allreduce_hist(h)
    if rank == 0:
        out.put((order, states, h.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process(orc):
    sys.path[:0] = [ROOT]
    import oracle
    import workloads
    import shard_cases
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    order, states, hist = qu.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flags = oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN
    ref = oracle.Sim(orc, workloads.crossed())
    stats = {}
    for k in range(STEPS):
        ref.load(shard_cases.rank_order(ref.state(), order[k]))
        for key, v in ref.run(1, flags).items():
            stats[key] = stats.get(key, 0) + v
    want = ref.state()
    assert stats["n_nbw"] > 0 and stats["n_ncs_e"] > 0 and stats["n_ncs_p"] > 0
    got = shard_cases.union(states)
    assert states[0]["next_id"] == states[1]["next_id"]
    shard_cases.assert_same(got, want)
    # the ranks' births: no id twice, and none below the start counter
    wl = workloads.crossed()
    ids = np.concatenate([got[sp]["id"] for sp in ("e", "pos", "ph")])
    assert len(np.unique(ids)) == len(ids)
    assert np.count_nonzero(ids >= wl["next_id"]) > 0
    assert np.array_equal(np.histogram(_energy(want["ph"]), EDGES)[0].astype(np.float64), hist)
