"""V_dep+ over a 400-step run: GPU FP64 and batched MIXED against the FP64 oracle.

Every sample draws its own particles (a Philox stream per sample), identical on
the three sides.  Deposition decisions at the wall are discontinuous, so over a
long run a rounding difference can move a single deposition event; the FP64 bar
is therefore the tallies within 2 events (the runs share the oracle's
arithmetic up to rounding).  For MIXED the bar is the metric's validity
condition: the Monte Carlo mean of V_dep+ per class within 1e-3 relative of the
oracle's and within one Monte Carlo standard error (a class where neither run
deposits meets both with equality).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

ST = [0.1, 1.0, 10.0]
S, N, STEPS, DT = 4, 2048, 400, 0.05
WIN = workloads.window_start_step(10.0, DT)


@pytest.fixture(scope="module")
def runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as pdq
    params = workloads.sample_params(S, 77)
    grid_shape = dict(n_r=64, n_th=32, n_z=64)
    field = pdq.Field(pdq.field_desc(**grid_shape), 0)
    phys = pdq.phys_default()
    out = {}
    for name, prec, ce in (("fp64", pdq.FP64, 0), ("mixed", pdq.MIXED, 100)):
        st = pdq.State(prec, [N] * S, ST)
        prm = pdq.params_tensor(params)
        pdq.seed_particles_independent(field, phys, st, prm, 1)
        cfg = pdq.step_cfg(DT, window_start=WIN, compact_every=ce)
        tally = pdq.Tally(S, len(ST))
        pdq.step_particles(field, phys, st, prm, cfg, STEPS, tally, pdq.workspace(st, cfg))
        assert pdq.check_state(st) == 0
        out[name] = (tally.n_dep.cpu().numpy(), tally.n_alive.cpu().numpy())
    of = oracle.field_desc(**grid_shape)
    grid = oracle.field_grid(of, oracle.field_modes(of, 0))
    ost, off = oracle.seed(of, ST, [N] * S, params, 1, independent=True)
    out["oracle"] = oracle.run(of, grid, oracle.cfg(DT, window_start=WIN), ST, off, params, ost, STEPS)
    return out


def test_fp64_tallies_match_oracle(runs):
    nd, na = runs["fp64"]
    od, oa = runs["oracle"]
    assert od.sum() > 0
    assert np.abs(nd - od).sum() <= 2
    assert np.abs(na - oa).sum() <= 2 * STEPS


def test_mixed_vdep_within_mc_error(runs):
    v_m = oracle.vdep(*runs["mixed"], DT)
    v_o = oracle.vdep(*runs["oracle"], DT)
    mean_m, mean_o = v_m.mean(0), v_o.mean(0)
    se = v_o.std(0, ddof=1) / np.sqrt(S)
    assert runs["oracle"][0].sum() > 0
    for c in range(len(ST)):
        d = abs(mean_m[c] - mean_o[c])
        assert d <= 1e-3 * mean_o[c] and d <= se[c], (c, mean_m, mean_o, se)
