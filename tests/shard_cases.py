"""Helpers of the sharding tests: a sharded run is checked against one process stepping
the whole population with, before every step, its particles in the ranks' order (rank 0's
particles, then rank 1's, ...).  Particle order is storage only -- every random number is
keyed by id -- so that reordering is a plain single-rank run; it is the order in which a
single process would number the step's births as the ranks do together."""
import numpy as np

SPECIES = ("e", "pos", "ph")


def rank_order(state, ids_by_rank):
    """``state`` (a stepping engine's state dict) with each species permuted so that its ids
    come in the order of ``ids_by_rank[sp]`` (a list of id arrays, rank 0 first)."""
    out = dict(state)
    for sp in SPECIES:
        want = np.concatenate([np.asarray(a, dtype=np.uint64) for a in ids_by_rank[sp]]) \
            if ids_by_rank[sp] else np.zeros(0, np.uint64)
        have = state[sp]["id"]
        assert len(want) == len(have) and np.array_equal(np.sort(want), np.sort(have)), sp
        o = np.argsort(have, kind="stable")
        pos = o[np.searchsorted(have[o], want)]
        out[sp] = {k: v[pos] for k, v in state[sp].items()}
    return out


def union(states):
    """The ranks' states as one population (species concatenated in rank order)."""
    out = {sp: {k: np.concatenate([s[sp][k] for s in states]) for k in states[0][sp]} for sp in SPECIES}
    out["next_id"] = states[0]["next_id"]
    return out


def by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def assert_same(a, b, tol=0.0):
    """Same particles (ids), same values (within ``tol`` relative, 0: bit-identical)."""
    for sp in SPECIES:
        x, y = by_id(a[sp]), by_id(b[sp])
        assert np.array_equal(x["id"], y["id"]), (sp, len(x["id"]), len(y["id"]))
        for k in x:
            if k == "id":
                continue
            if tol == 0.0:
                assert np.array_equal(x[k], y[k]), (sp, k)
            else:
                assert np.all(np.abs(x[k] - y[k]) <= tol * np.maximum(np.abs(y[k]), 1.0)), (sp, k)
    assert a["next_id"] == b["next_id"]
