"""The learned photon-energy sampler (qed_mlp_*) through the C ABI.

* The training target (the table sampler's mixture inverse on the FP32 tables) against the
  oracle's mixture inverse on its own tables.
* Tensor-core evaluation (tcgen05, BF16 hidden layer, FP32 accumulation in tensor memory)
  against the numpy network with the same BF16 rounding, for given parameters.
* A short training run learns the target (median and tail errors in ln u), and a step with
  QED_F_MLP (its own training run) reproduces the photon spectrum and polarisation of the
  table path and of the FP64 oracle within 3 sigma per bin (fixed seeds: the outcome is
  reproducible)."""
import math

import numpy as np
import pytest

import oracle.sampler as SM
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    return q.qed_init_tables()


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(SM.LNCHI_LO, SM.LNCHI_HI, n), rng.uniform(-1, 1, n),
                     rng.uniform(1e-6, 1 - 1e-6, n)], 1)


def test_target_matches_oracle_mixture_inverse(ctx, orc):
    rows = _rows(160, 5)
    got = q.mlp_apply(ctx, rows, "target")
    want = np.array([SM.mixture_inverse(orc, math.exp(a), b, r) for a, b, r in rows.astype(np.float32).astype(np.float64)])
    assert np.abs(got - want).max() < 2e-3 * np.maximum(np.abs(want), 1.0).max()
    assert np.median(np.abs(got - want)) < 1e-4


def test_tensor_core_eval_matches_numpy_network(ctx):
    rng = np.random.default_rng(7)
    p = np.zeros(SM.N_PARAMS, dtype=np.float32)
    p[:SM.H * 3] = rng.normal(0, 0.8, SM.H * 3)
    p[SM.H * 3:SM.H * 4] = rng.normal(0, 0.3, SM.H)
    p[SM.H * 4:SM.H * 4 + SM.H * SM.H] = rng.normal(0, 0.25, SM.H * SM.H)
    p[SM.H * 4 + SM.H * SM.H:] = rng.normal(0, 0.2, SM.N_PARAMS - SM.H * 4 - SM.H * SM.H)
    q.qed_mlp_set_params(ctx, p)
    assert np.array_equal(q.qed_mlp_get_params(ctx), p)
    rows = _rows(3 * 128 * 152 + 77, 9).astype(np.float32).astype(np.float64)   # several chunks per CTA, ragged
    got = q.mlp_apply(ctx, rows, "eval")
    want = SM.forward(p, rows[:, 0], rows[:, 1], rows[:, 2])
    d = np.abs(got - want)
    assert np.median(d) < 1e-4 and np.quantile(d, 0.999) < 2e-2 and d.max() < 0.1, (np.median(d), d.max())
    assert q.qed_read_status(ctx) == 0


TRAIN = (20_000_000, 1024)   # ~20k Adam steps, a few seconds


def test_training_learns_the_table_sampler(ctx):
    q.qed_mlp_train(ctx, *TRAIN, seed=3)
    rows = _rows(20000, 11)
    got = q.mlp_apply(ctx, rows, "eval")
    tgt = q.mlp_apply(ctx, rows, "target")
    d = np.abs(got - tgt)
    assert np.median(d) < 0.004 and np.quantile(d, 0.99) < 0.03, (np.median(d), np.quantile(d, 0.99))


def _spectrum(ph, bins):
    om = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    h, _ = np.histogram(om, bins=bins, weights=ph["w"])
    h3, _ = np.histogram(om, bins=bins, weights=ph["w"] * ph["s3"])
    return h, h3


def test_step_with_learned_sampler(ctx, orc):
    q.qed_mlp_train(ctx, *TRAIN, seed=4)
    n = 8000
    out = {}
    for name, extra in (("table", 0), ("mlp", q.QED_F_MLP)):
        wl = workloads.c1(n=n, seed=21)
        sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=q.qed_ctx_share(ctx))
        sim.run(450, q.QED_F_NCS | q.QED_F_SPIN | extra)
        assert sim.status() == 0
        out[name] = (sim.state()["ph"], sim.counters())
    (pt, ct), (pm, cm) = out["table"], out["mlp"]
    # emission decisions do not involve the sampler until the recoil changes the electrons
    assert abs(ct["n_ncs_e"] - cm["n_ncs_e"]) <= 4 * math.sqrt(ct["n_ncs_e"])
    bins = np.geomspace(1.0, 2000.0, 13)
    ht, h3t = _spectrum(pt, bins)
    hm, h3m = _spectrum(pm, bins)
    # weighted counts (weights 1 in config 1): Poisson errors of independent runs, which the
    # same-seed pair (correlated) can only undercut
    sig = np.sqrt(ht + hm + 1e-9)
    assert np.all(np.abs(ht - hm) <= 3.0 * sig), (ht, hm)
    m = (ht > 300) & (hm > 300)
    xt, xm = h3t[m] / ht[m], h3m[m] / hm[m]
    assert np.all(np.abs(xt - xm) <= 3.0 * np.sqrt(1.0 / ht[m] + 1.0 / hm[m]))
    # against the FP64 oracle (independent seed): the same bounds
    import oracle
    wl = workloads.c1(n=n, seed=22)
    osim = oracle.Sim(orc, wl)
    osim.run(450, q.QED_F_NCS | q.QED_F_SPIN)
    ho, h3o = _spectrum(osim.state()["ph"], bins)
    sig = np.sqrt(ho + hm + 1e-9)
    assert np.all(np.abs(ho - hm) <= 3.0 * sig), (ho, hm)
    m = (ho > 300) & (hm > 300)
    assert np.all(np.abs(h3o[m] / ho[m] - h3m[m] / hm[m]) <= 3.0 * np.sqrt(1.0 / ho[m] + 1.0 / hm[m]))
