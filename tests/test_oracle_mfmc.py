"""Pins of the multi-fidelity estimators: the paper's Tables 2-3 and gamma values,
and the closed-form Sobol' indices of the Ishigami function."""
import json
import os

import numpy as np
import pytest

from oracle import mfmc

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tables():
    return json.load(open(os.path.join(GOLD, "mfmc_tables.json")))


def test_allocation_reproduces_table3(tables):
    w = [1.0, tables["w2"]]
    d = tables["d"]
    for case in tables["cases"]:
        rho = [1.0, case["rho12"]]
        sig = [case["sigma1"], case["sigma2"]]
        for pkey, p in (("p36", 36), ("p72", 72)):
            ref = case[pkey]
            alpha, r, m_star = mfmc.mfmc_allocation(rho, sig, w, p / (d + 2))   # p_eff = p/(d+2)
            assert abs(alpha[1] - ref["alpha"]) < 2.5e-3                        # printed to 3 decimals
            assert int(np.floor(m_star[0])) == ref["m1"]
            # the printed m2 is not linear in p (5488/2861 != 2); the worst case deviates 5.1%
            assert abs(m_star[1] - ref["m2"]) / ref["m2"] < 0.06
            # plain MC: every evaluation on one model
            assert int(p / (d + 2)) == ref["mc_m1"]
            assert int(round(p / (d + 2) / tables["w2"])) == ref["lf_only_m"]
        assert mfmc.mfmc_precondition(rho, w)


def test_gamma_values(tables):
    for case in tables["cases"]:
        g = mfmc.gamma_two_model(case["rho12"], tables["w2"])
        assert round(g, 3) == case["gamma"]
    # limits: uncorrelated models give no reduction, a free perfect surrogate gives zero variance
    assert mfmc.gamma_two_model(0.0, 1e-3) == 1.0
    assert mfmc.gamma_two_model(1.0, 0.0) == 0.0


def test_precondition_fails_for_expensive_surrogate():
    # Fig. 7: the precondition fails for an expensive, weakly correlated low-fidelity model
    assert not mfmc.mfmc_precondition([1.0, 0.3], [1.0, 0.5])


def test_ishigami_closed_form_values():
    # published values for a = 7, b = 0.1 (e.g. Saltelli et al., Global Sensitivity Analysis, 2008)
    mean, V, s, st = mfmc.ishigami_indices()
    assert mean == 3.5
    assert V == pytest.approx(13.8446, abs=1e-4)
    assert np.allclose(s, [0.3139, 0.4424, 0.0], atol=1e-4)
    assert np.allclose(st, [0.5576, 0.4424, 0.2437], atol=1e-4)
    # against a brute-force quadrature of the variance
    g = np.linspace(-np.pi, np.pi, 81)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)
    w = np.ones(81)
    w[1:-1:2], w[2:-1:2] = 4, 2
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    Y = mfmc.ishigami(X)
    mu = np.sum(W * Y) / np.sum(W)
    var = np.sum(W * (Y - mu) ** 2) / np.sum(W)
    assert mu == pytest.approx(3.5, abs=1e-6) and var == pytest.approx(V, rel=1e-4)


def test_owen_jansen_estimate_ishigami_indices():
    _, _, s, st = mfmc.ishigami_indices()
    rng = np.random.default_rng(10)
    m = 200_000
    x = rng.uniform(-np.pi, np.pi, (m, 3))
    xp = rng.uniform(-np.pi, np.pi, (m, 3))
    Y = mfmc.ishigami(mfmc.pick_freeze_inputs(x, xp))   # [m, 5]
    s_hat, st_hat, mean, var = mfmc.mfmc_sobol([Y], [m], [1.0])
    assert np.allclose(s_hat, s, atol=0.01) and np.allclose(st_hat, st, atol=0.01)
    assert mean == pytest.approx(3.5, abs=0.03)


def test_owen_main_effect_unbiased_over_replicates():
    # Owen's estimator is unbiased for V_j: replicate mean within 3 standard errors
    _, V, s, _ = mfmc.ishigami_indices()
    rng = np.random.default_rng(11)
    reps, m = 400, 64
    est = np.zeros((reps, 3))
    for r in range(reps):
        x = rng.uniform(-np.pi, np.pi, (m, 3))
        xp = rng.uniform(-np.pi, np.pi, (m, 3))
        Y = mfmc.ishigami(mfmc.pick_freeze_inputs(x, xp))
        est[r] = [mfmc.owen_main(Y[:, 0], Y[:, 1], Y[:, 2 + j]) for j in range(3)]
    se = est.std(0) / np.sqrt(reps)
    assert np.all(np.abs(est.mean(0) - s * V) < 3 * se + 1e-12)


def test_mfmc_variance_reduction_matches_gamma():
    # two models: LF = HF + correlated noise; the MFMC mean estimator's variance over
    # replicates relative to MC at equal cost approaches gamma(rho, w2/w1).
    rng = np.random.default_rng(12)
    w = [1.0, 1e-2]
    noise = 1.5

    def hf(x):
        return mfmc.ishigami(x)

    def lf(x, e):
        return 0.8 * mfmc.ishigami(x) + noise * e

    # pilot statistics
    xs = rng.uniform(-np.pi, np.pi, (200_000, 3))
    e = rng.standard_normal(200_000)
    yh, yl = hf(xs), lf(xs, e)
    rho = np.corrcoef(yh, yl)[0, 1]
    sig = [yh.std(), yl.std()]
    p = 40.0
    alpha, r, m_star = mfmc.mfmc_allocation([1, rho], sig, w, p)
    m = [int(np.floor(m_star[0])), int(np.floor(m_star[1]))]
    reps = 3000
    est_mf, est_mc = np.zeros(reps), np.zeros(reps)
    for k in range(reps):
        x = rng.uniform(-np.pi, np.pi, (m[1], 3))
        e = rng.standard_normal(m[1])
        est_mf[k] = mfmc.mfmc_mean([hf(x[: m[0]]), lf(x, e)], m, alpha)
        est_mc[k] = mfmc.mc_mean(hf(x[: int(p)]))
    ratio = est_mf.var() / est_mc.var()
    gamma = mfmc.gamma_two_model(rho, w[1] / w[0])
    assert 0.7 * gamma < ratio < 1.3 * gamma
    assert abs(est_mf.mean() - 3.5) < 4 * est_mf.std() / np.sqrt(reps)   # unbiased


def test_dgsm_bound_linear_and_ishigami():
    # f = x on [0, 1]: s^t = 1, nu = 1, Var = 1/12 -> bound = 12/pi^2 (>= 1)
    rng = np.random.default_rng(13)
    x = rng.random((200_000, 1))
    nu, bound = mfmc.dgsm_bound(np.ones_like(x), x[:, 0], [1.0])
    assert nu[0] == 1.0 and abs(bound[0] - 12 / np.pi ** 2) < 0.01
    # Ishigami: every total index lies below its DGSM bound (Sobol'-Kucherenko inequality)
    X = rng.uniform(-np.pi, np.pi, (400_000, 3))
    nu, bound = mfmc.dgsm_bound(mfmc.ishigami_grad(X), mfmc.ishigami(X), [2 * np.pi] * 3)
    _, _, _, st = mfmc.ishigami_indices()
    assert np.all(st <= bound)
    # analytic nu_2 = E[(a sin 2 x2)^2] = a^2 / 2
    assert abs(nu[1] - 7.0 ** 2 / 2) < 0.1
