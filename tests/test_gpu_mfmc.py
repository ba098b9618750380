"""GPU parity of the MFMC / Sobol' estimators (pdq_mfmc_sobol) against the numpy oracle.

Data: the Ishigami function (closed-form indices) as the high-fidelity model and a
correlated, cheaper surrogate; pick-freeze groups with nested samples.  Estimates
agree to 1e-12 relative (the device sums in a different order than numpy);
bootstrap intervals use the same Philox resampling indices on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import mfmc  # noqa: E402


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


def _groups(n, seed, C=2):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-np.pi, np.pi, (n, 3))
    xp = rng.uniform(-np.pi, np.pi, (n, 3))
    X = mfmc.pick_freeze_inputs(x, xp)                     # [n, 5, 3]
    hf = np.stack([mfmc.ishigami(X), mfmc.ishigami(X, a=5.0, b=0.2)], -1)[..., :C]
    noise = rng.standard_normal((n, 1, C))
    lf = 0.8 * hf + 0.7 * noise                             # same noise for the whole group
    return hf, lf


def test_mc_sobol_matches_oracle_and_closed_form(pdq):
    hf, _ = _groups(40000, 1)
    out = pdq.mfmc_sobol([torch.tensor(hf, device="cuda")], [40000], [1.0])
    sm, st, mean, var = mfmc.mfmc_sobol([hf], [40000], [1.0])
    assert np.allclose(out["s_main"], sm, rtol=1e-11, atol=1e-13)
    assert np.allclose(out["s_total"], st, rtol=1e-11, atol=1e-13)
    assert np.allclose(out["mean"], mean, rtol=1e-12) and np.allclose(out["var"], var, rtol=1e-11)
    _, _, s_ref, st_ref = mfmc.ishigami_indices()
    assert np.allclose(out["s_main"][:, 0], s_ref, atol=0.03) and np.allclose(out["s_total"][:, 0], st_ref, atol=0.03)


def test_two_model_mfmc_matches_oracle(pdq):
    hf, lf = _groups(30000, 2)
    m = [500, 30000]
    rho = np.corrcoef(hf[:, 0, 0], lf[:, 0, 0])[0, 1]
    alpha = [1.0, rho * hf[:, 0, 0].std() / lf[:, 0, 0].std()]
    out = pdq.mfmc_sobol([torch.tensor(hf[:500], device="cuda"), torch.tensor(lf, device="cuda")], m, alpha)
    sm, st, mean, var = mfmc.mfmc_sobol([hf[:500], lf], m, alpha)
    assert np.allclose(out["s_main"], sm, rtol=1e-10, atol=1e-12)
    assert np.allclose(out["s_total"], st, rtol=1e-10, atol=1e-12)
    assert np.allclose(out["mean"], mean, rtol=1e-12) and np.allclose(out["var"], var, rtol=1e-11)


def test_bootstrap_intervals_match_oracle(pdq):
    hf, lf = _groups(4000, 3)
    m = [200, 4000]
    alpha = [1.0, 1.1]
    seed, B = 99, 64
    out = pdq.mfmc_sobol([torch.tensor(hf[:200], device="cuda"), torch.tensor(lf, device="cuda")], m, alpha,
                         n_boot=B, seed=seed)
    ci_m, ci_t = mfmc.bootstrap_ci([hf[:200], lf], m, alpha, lambda b: oracle.boot_indices(seed, b, m), B)
    assert np.allclose(out["s_main_ci"], ci_m, rtol=1e-10, atol=1e-12)
    assert np.allclose(out["s_total_ci"], ci_t, rtol=1e-10, atol=1e-12)
    lo, hi = out["s_main_ci"][..., 0], out["s_main_ci"][..., 1]
    assert np.all(lo <= hi)


def test_dgsm_bounds_match_oracle(pdq):
    rng = np.random.default_rng(14)
    X = rng.uniform(-np.pi, np.pi, (5000, 3))
    g = np.stack([mfmc.ishigami_grad(X), 2 * mfmc.ishigami_grad(X)], 1)     # [S, 2 outputs, 3]
    y = np.stack([mfmc.ishigami(X), 2 * mfmc.ishigami(X)], 1)
    nu, bound = pdq.dgsm_bounds(torch.tensor(g, device="cuda"), torch.tensor(y, device="cuda"), [2 * np.pi] * 3)
    nu_ref, b_ref = mfmc.dgsm_bound(g, y, [2 * np.pi] * 3)
    assert np.allclose(nu, nu_ref, rtol=1e-12) and np.allclose(bound, b_ref, rtol=1e-12)
