"""The oracle's step in two parts (decide, commit) and the id numbering of sharded steps.

* decide + commit with the sequential ids is or_step, bit for bit;
* the bases of or_shard_bases, written out for three ranks: each rank's pairs, e-
  emissions and e+ emissions take consecutive ids after the ranks before it, the blocks
  tile [next_id, next_id + 2 pairs + emissions) with no gap or overlap, and every rank's
  counter moves to the same place;
* one rank alone numbers its births as the sequential pass does.
The two-rank run itself is in test_shard_gloo.py."""
import numpy as np

import oracle
import workloads

FLAGS = oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN


def test_decide_commit_is_one_step(orc):
    wl = workloads.crossed(seed=2)
    a = oracle.Sim(orc, wl)
    sa = a.run(3, FLAGS)
    ref = a.state()
    b = oracle.Sim(orc, wl)
    tot = {}
    for _ in range(3):
        cnt, s1 = b.decide(FLAGS)
        s2 = b.commit()
        assert cnt[0] == s1["n_nbw"] and cnt[1] + cnt[2] == s1["n_ncs_e"] + s1["n_ncs_p"]
        for d in (s1, s2):
            for k, v in d.items():
                tot[k] = tot.get(k, 0) + v
    got = b.state()
    assert tot == sa and sa["n_nbw"] > 0 and sa["n_ncs_e"] > 0 and sa["n_ncs_p"] > 0
    for sp in ("e", "pos", "ph"):
        for k in ref[sp]:
            assert np.array_equal(got[sp][k], ref[sp][k]), (sp, k)
    assert got["next_id"] == ref["next_id"]


def test_commit_needs_a_decided_step(orc):
    sim = oracle.Sim(orc, workloads.crossed(ne=8, npos=4, nph=8))
    try:
        sim.commit()
    except RuntimeError:
        return
    raise AssertionError("commit without decide was accepted")


def test_shard_bases_three_ranks():
    allc = [[3, 5, 7], [2, 4, 6], [1, 1, 1]]   # pairs, e- emissions, e+ emissions
    b = [oracle.shard_bases(100, allc, r) for r in range(3)]
    # 6 pairs (12 ids from 100), then 10 e- emissions from 112, then 14 e+ from 122; 136 next
    assert [list(x) for x in b] == [[100, 112, 122, 136], [106, 117, 129, 136], [110, 121, 135, 136]]
    ids = []
    for r, (p, e, q) in enumerate(allc):
        ids += [b[r][0] + k for k in range(2 * p)] + [b[r][1] + k for k in range(e)] + [b[r][2] + k for k in range(q)]
    assert sorted(ids) == list(range(100, 136))


def test_one_rank_numbers_as_the_sequential_pass():
    assert list(oracle.shard_bases(7, [[4, 9, 2]], 0)) == [7, 7 + 8, 7 + 8 + 9, 7 + 8 + 9 + 2]
