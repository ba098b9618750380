"""GPU parity of the 1-D Eulerian low-fidelity model (pdq_lf_fluid_variance, pdq_lf_vdep)
against the numpy oracle (oracle/lf_eulerian.py), through the C ABI.

The device marches each (sample, class) item once from the axis to the wall and
composes the flux solution on the way (P, Q); the oracle stores V and marches the
density back out from the wall.  Both are FP64 and agree to rounding: the bar is
1e-10 relative (potential differences taken from node values on one side and
from differences of the shapes on the other, expm1/exp and sqrt from different
libraries, over ~2,000 cells).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import lf_eulerian as lfo  # noqa: E402

RTOL = 1e-10
# PDQ_MIXED (FP32 march, FP64 wall condition and ratio): a float32 restatement of the march, with
# IEEE operations, stays within 3.3e-6 of the FP64 oracle (median 5e-7) on 2,000 items at 2,048
# nodes (rounding ~6e-8 per operation over ~2,000 cells); the bar leaves a factor of 6
RTOL_MIXED = 2e-5
ST5 = [0.1, 0.316, 1.0, 3.16, 10.0]


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


@pytest.fixture(scope="module")
def fields(pdq):
    out = {}
    for grid in [(64, 32, 64), (128, 64, 128)]:
        d = pdq.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2])
        f = pdq.Field(d, 0)
        of = oracle.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2])
        var_o = lfo.fluid_variance(oracle.field_grid(of, oracle.field_modes(of, 0)))
        out[grid] = (f, of, var_o)
    return out


def _params(S, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0, 0.1, S), rng.uniform(0, 1, S), rng.uniform(0, 1, S)], 1)


@pytest.mark.parametrize("grid", [(64, 32, 64), (128, 64, 128)])
def test_fluid_variance_matches_oracle(pdq, fields, grid):
    f, _, var_o = fields[grid]
    v = pdq.lf_fluid_variance(f).cpu().numpy()
    scale = var_o.max()
    assert np.all(np.abs(v - var_o) <= 1e-12 * np.abs(var_o) + 1e-15 * scale)
    # deterministic
    assert np.array_equal(v, pdq.lf_fluid_variance(f).cpu().numpy())


@pytest.mark.parametrize("n_y", [3, 4, 129, 1000, 2048, 4096])
def test_vdep_matches_oracle(pdq, fields, n_y):
    f, of, var_o = fields[(64, 32, 64)]
    S = 600 if n_y <= 2048 else 130          # 600: two full CTAs of 256 samples and a ragged one
    prm = _params(S, n_y)
    phys = pdq.phys_default()
    desc = pdq.lf_desc(n_y=n_y)
    var = pdq.lf_fluid_variance(f)
    got = pdq.lf_vdep(f, phys, desc, var, ST5, pdq.params_tensor(prm)).cpu().numpy()
    ref = lfo.lf_vdep(oracle.phys(), ST5, prm, var_o, of.r_plus, of.beta, lfo.lf_params(n_y=n_y))
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    assert np.max(np.abs(got / ref - 1)) < RTOL


@pytest.mark.parametrize("n_y", [3, 129, 2048, 4096])
def test_mixed_vdep_matches_oracle(pdq, fields, n_y):
    f, of, var_o = fields[(64, 32, 64)]
    S = 600 if n_y <= 2048 else 130
    prm = _params(S, 100 + n_y)
    prm[0] = [0.0, 0.0, 0.5]
    var = pdq.lf_fluid_variance(f)
    got = pdq.lf_vdep(f, pdq.phys_default(), pdq.lf_desc(n_y=n_y, precision=pdq.MIXED), var, ST5,
                      pdq.params_tensor(prm)).cpu().numpy()
    ref = lfo.lf_vdep(oracle.phys(), ST5, prm, var_o, of.r_plus, of.beta, lfo.lf_params(n_y=n_y))
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    assert np.max(np.abs(got / ref - 1)) < RTOL_MIXED


def test_vdep_parameters_and_class_edge_cases(pdq, fields):
    f, of, var_o = fields[(128, 64, 128)]
    phys = pdq.phys_default()
    var = pdq.lf_fluid_variance(f)
    # one class; sixteen classes (the maximum); non-default model parameters
    st16 = list(10 ** np.linspace(-1, 2, 16))
    prm = _params(70, 5)
    prm[0] = [0.0, 0.0, 0.5]                   # no charge, no vdW
    prm[1] = [0.1, 1.0, 0.5]                   # the range's top corner
    for st, kw in [([3.16], {}), (st16, {}), (ST5, dict(stretch=4.0, t_lagr=3.0, temperature=350.0,
                                                           vdw_cutoff=1e-11))]:
        desc = pdq.lf_desc(n_y=700, **kw)
        got = pdq.lf_vdep(f, phys, desc, var, st, pdq.params_tensor(prm)).cpu().numpy()
        ref = lfo.lf_vdep(oracle.phys(), st, prm, var_o, of.r_plus, of.beta, lfo.lf_params(n_y=700, **kw))
        assert got.shape == (70, len(st))
        assert np.max(np.abs(got / ref - 1)) < RTOL


def test_brownian_limit_closed_form(pdq, fields):
    # zero fluid variance, no charge, no vdW: 1/V_dep+ = sqrt(2 pi)/sigma_B + (R - d/2)/D_B
    f, _, _ = fields[(64, 32, 64)]
    phys = pdq.phys_default()
    zero = torch.zeros(64, dtype=torch.float64, device="cuda")
    st = [0.1, 1.0, 10.0]
    got = pdq.lf_vdep(f, phys, pdq.lf_desc(n_y=64), zero, st,
                      pdq.params_tensor(np.array([[0.0, 0.0, 0.3]] * 5))).cpu().numpy()
    tab = oracle.class_table(st)
    for c in range(3):
        DB, th = lfo.brownian(oracle.phys(), tab[c], 293.15)
        ref = 1 / (math.sqrt(2 * math.pi / th) + (180.0 - 0.5 * tab[c, 1]) / DB)
        assert np.all(np.abs(got[:, c] / ref - 1) < 1e-12)


def test_theta_does_not_enter_and_calls_are_deterministic(pdq, fields):
    f, _, _ = fields[(64, 32, 64)]
    phys = pdq.phys_default()
    var = pdq.lf_fluid_variance(f)
    prm = _params(50, 9)
    a = pdq.lf_vdep(f, phys, pdq.lf_desc(), var, ST5, pdq.params_tensor(prm)).cpu().numpy()
    prm2 = prm.copy()
    prm2[:, 2] = 1.0 - prm2[:, 2]
    b = pdq.lf_vdep(f, phys, pdq.lf_desc(), var, ST5, pdq.params_tensor(prm2)).cpu().numpy()
    c = pdq.lf_vdep(f, phys, pdq.lf_desc(), var, ST5, pdq.params_tensor(prm)).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_empty_and_invalid_arguments(pdq, fields):
    import ctypes as C
    f, _, _ = fields[(64, 32, 64)]
    phys = pdq.phys_default()
    var = pdq.lf_fluid_variance(f)
    L = pdq.lib()
    st = (C.c_double * 2)(0.1, 1.0)
    out = torch.full((4, 2), -7.0, dtype=torch.float64, device="cuda")
    prm = pdq.params_tensor(_params(4, 1))

    def call(desc, n_classes=2, S=4, stp=st, v=var, o=out, p=prm):
        return L.pdq_lf_vdep(f.handle, C.byref(phys), C.byref(desc), pdq._ptr(v), n_classes,
                             C.cast(stp, C.c_void_p), S, pdq._ptr(p), pdq._ptr(o), None)

    assert call(pdq.lf_desc(), S=0, p=None, o=None) == 0        # nothing to do
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)
    for bad in [dict(n_y=2), dict(n_y=4097), dict(stretch=0.0), dict(stretch=701.0), dict(t_lagr=0.0),
                dict(temperature=-1.0), dict(vdw_cutoff=0.0), dict(precision=2), dict(precision=-1)]:
        assert call(pdq.lf_desc(**bad)) == -1, bad
    assert call(pdq.lf_desc(), n_classes=0) == -1
    assert call(pdq.lf_desc(), n_classes=17) == -1
    assert call(pdq.lf_desc(), stp=(C.c_double * 2)(0.1, 0.0)) == -1
    assert call(pdq.lf_desc(), S=-1) == -1
    assert call(pdq.lf_desc(), v=None) == -1
    p2 = pdq.phys_default()
    p2.re_tau = 200.0
    assert L.pdq_lf_vdep(f.handle, C.byref(p2), C.byref(pdq.lf_desc()), pdq._ptr(var), 2, C.cast(st, C.c_void_p),
                         4, pdq._ptr(prm), pdq._ptr(out), None) == -1
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)


def test_full_size_sampled(pdq, fields):
    # the low-fidelity size of the Sobol' study: 262,144 samples x 10 classes, default nodes;
    # 48 sampled items recomputed by the oracle, every item finite and positive
    f, of, var_o = fields[(128, 64, 128)]
    S = 262144
    st10 = list(10 ** (-1 + 3 * np.arange(10) / 9))
    prm = _params(S, 77)
    phys = pdq.phys_default()
    var = pdq.lf_fluid_variance(f)
    got = pdq.lf_vdep(f, phys, pdq.lf_desc(), var, st10, pdq.params_tensor(prm)).cpu().numpy()
    assert got.shape == (S, 10) and np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.random.default_rng(3).choice(S, 48, replace=False)
    idx[0], idx[1] = 0, S - 1
    ref = lfo.lf_vdep(oracle.phys(), st10, prm[idx], var_o, of.r_plus, of.beta)
    assert np.max(np.abs(got[idx] / ref - 1)) < RTOL
    # the FP32 march on the same items: every item within the MIXED bar of the FP64 march
    mix = pdq.lf_vdep(f, phys, pdq.lf_desc(precision=pdq.MIXED), var, st10, pdq.params_tensor(prm)).cpu().numpy()
    assert np.all(np.isfinite(mix)) and np.max(np.abs(mix / got - 1)) < RTOL_MIXED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sample_blocks_walked_with_a_ragged_tail(pdq, fields, precision):
    # one wave of CTAs per class, each walking several 256-sample blocks: 40,001 samples (157
    # blocks, the last one sample) x 16 classes; the first, last and 30 random items vs the oracle
    f, of, var_o = fields[(64, 32, 64)]
    S = 40001
    st16 = list(10 ** np.linspace(-1, 2, 16))
    prm = _params(S, 31)
    prec = pdq.MIXED if precision == "mixed" else pdq.FP64
    var = pdq.lf_fluid_variance(f)
    got = pdq.lf_vdep(f, pdq.phys_default(), pdq.lf_desc(n_y=512, precision=prec), var, st16,
                      pdq.params_tensor(prm)).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.concatenate([[0, 255, 256, S - 2, S - 1], np.random.default_rng(8).choice(S, 30, replace=False)])
    ref = lfo.lf_vdep(oracle.phys(), st16, prm[idx], var_o, of.r_plus, of.beta, lfo.lf_params(n_y=512))
    assert np.max(np.abs(got[idx] / ref - 1)) < (RTOL_MIXED if precision == "mixed" else RTOL)


def test_two_model_study_with_the_eulerian_model(pdq):
    # uq.mfmc_sobol_deposition: with a given allocation its estimates equal pdq_mfmc_sobol on the two
    # tables it returns, the particle-model groups are the first m_1 of the nested groups, and the
    # low-fidelity table equals pdq_lf_vdep on the same inputs
    from paper_2205_04979_gb300 import uq
    st = (10.0,)
    r = uq.mfmc_sobol_deposition(0, 1024, 600, st_plus=st, allocation=([4, 24], [1.0, 0.7]), grid=(32, 16, 32),
                                 n_boot=0, seed=3)
    assert r["m"] == [4, 24] and r["hf"].shape == (4, 5, 1) and r["lf"].shape == (24, 5, 1)
    assert r["inputs"].shape == (24, 5, 3)
    ref = pdq.mfmc_sobol([torch.tensor(r["hf"], device="cuda"), torch.tensor(r["lf"], device="cuda")], [4, 24],
                         [1.0, 0.7])
    for q in ("mean", "var", "s_main", "s_total"):
        assert np.array_equal(r[q], ref[q]), q
    f = pdq.Field(pdq.field_desc(n_r=32, n_th=16, n_z=32), 3)
    direct = pdq.lf_vdep(f, pdq.phys_default(), pdq.lf_desc(precision=pdq.MIXED), pdq.lf_fluid_variance(f), st,
                         pdq.params_tensor(r["inputs"].reshape(-1, 3))).cpu().numpy()
    assert np.array_equal(direct.reshape(24, 5, 1), r["lf"])
    # the pilot path: an allocation with 2 <= m_1 <= m_2 and finite estimates, or one of the two
    # documented refusals (MFMC no better than MC; no variation in the pilot)
    try:
        r2 = uq.mfmc_sobol_deposition(8, 2048, 1000, st_plus=st, pilot=16, grid=(32, 16, 32), n_boot=0, seed=4)
    except pdq.PdqError as e:
        assert e.status == -6
    except ValueError as e:
        assert "no variation" in str(e)
    else:
        assert 2 <= r2["m"][0] <= r2["m"][1] and np.all(np.isfinite(r2["mean"]))
        assert -1.0 <= r2["pilot"]["rho"][0] <= 1.0 and np.all(r2["pilot"]["w_ms_per_sample"] > 0)
