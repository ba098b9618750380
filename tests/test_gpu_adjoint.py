"""GPU adjoint of the smoothed deposition functional (pdq_adjoint_run) against
the oracle's forward-mode dual numbers and against central finite differences.

Two cases: A exercises the charge path (Coulomb, image; eps = 0.5), B the van
der Waals path (St+ = 10, 100 pushed to the wall by a test-only gravity vector;
eps = 0.05).  FP64: J to 1e-12 and each gradient column to 1e-8 of its largest
entry (both sides are exact derivatives of the same discrete map and differ by
rounding only).  MIXED: within 3 % (FP32 pair sums, interpolation, integrator).
theta enters only the rebound model: its derivative is exactly 0 under all-stick.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402

GRID = dict(n_r=33, n_th=16, n_z=32)
COUNTS = [300, 129]
PARAMS = np.array([[0.09, 0.7, 0.4], [0.06, 0.3, 0.8]])
SEED = 11
CASES = {
    # A: no particle reaches the vdW range (d/4), so dJ/dzeta is exactly 0 there
    "A": dict(st=[0.1, 1.0], steps=40, dt=0.05, eps=0.5, gravity=(0, 0, 1), win=5, nonzero=(0,)),
    "B": dict(st=[10.0, 100.0], steps=200, dt=0.1, eps=0.05, gravity=(1, 0, 0), win=5, nonzero=(0, 1)),
    # C: rebound mode, inputs near the sticking threshold, so theta matters (Sec. 4.3)
    "C": dict(st=[10.0, 100.0], steps=60, dt=0.1, eps=0.05, gravity=(1, 0, 0), win=5, nonzero=(0, 1, 2),
              mode=1, eps_stick=10.0, params=[[0.09, 0.9, 0.6], [0.06, 0.5, 0.7]]),
}


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


_REF = {}


def _params(case):
    return np.array(CASES[case].get("params", PARAMS), dtype=np.float64)


def ref(case):
    if case not in _REF:
        c = CASES[case]
        P = _params(case)
        of = oracle.field_desc(**GRID)
        grid = oracle.field_grid(of, oracle.field_modes(of, 0))
        st, off = oracle.seed(of, c["st"], COUNTS, np.c_[np.ones(2), P[:, 1:]], SEED)   # xi = 1: q = qhat
        cf = oracle.cfg(c["dt"], gravity=c["gravity"], smooth_eps=c["eps"], window_start=c["win"],
                        mode=c.get("mode", 0), stick_eps=c.get("eps_stick", 0.0))
        _REF[case] = oracle.smooth_run(of, grid, cf, c["st"], off, P, st.x, st.y, st.z, st.q, st.cls, c["steps"])
    return _REF[case]


def _run(pdq, case, precision, params, K=7, gbar=None):
    c = CASES[case]
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    batch = pdq.Batch(precision, COUNTS, c["st"])
    cfg = pdq.step_cfg(c["dt"], window_start=c["win"], gravity=c["gravity"], mode=c.get("mode", 0))
    return pdq.adjoint_run(field, pdq.phys_default(), batch, pdq.params_tensor(params), cfg, c["steps"], K,
                           c["eps"], SEED, gbar=gbar, eps_stick=c.get("eps_stick", 10.0))


def _onehot():
    g = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    g[0, :, 0] = 1.0
    g[1, :, 1] = 1.0
    return g


def _check_grad(got, want, rtol, nonzero):
    for k in range(3 if 2 in nonzero else 2):
        scale = np.max(np.abs(want[..., k]))
        if k in nonzero:
            assert scale > 0, "gradient column %d is identically zero" % k
        assert np.all(np.abs(got[..., k] - want[..., k]) <= rtol * scale), (k, got[..., k], want[..., k])


@pytest.mark.parametrize("case", ["A", "B", "C"])
def test_fp64_adjoint_matches_dual_numbers(pdq, case):
    J_ref, dJ_ref = ref(case)
    J, pbar = _run(pdq, case, 0, _params(case), gbar=_onehot())
    # rebound bounces amplify rounding differences near the wall: looser bar for case C
    rtol_J, rtol_g = (1e-12, 1e-8) if case != "C" else (1e-9, 1e-6)
    assert np.allclose(J.cpu().numpy(), J_ref, rtol=rtol_J, atol=1e-300)
    got = np.transpose(pbar.cpu().numpy(), (1, 0, 2))     # [sample, class, param]
    if 2 not in CASES[case]["nonzero"]:
        assert np.all(got[..., 2] == 0.0) and np.all(dJ_ref[..., 2] == 0.0)
    _check_grad(got, dJ_ref, rtol_g, CASES[case]["nonzero"])


def test_checkpoint_interval_does_not_change_gradient(pdq):
    _, p1 = _run(pdq, "A", 0, PARAMS, K=7, gbar=_onehot())
    _, p2 = _run(pdq, "A", 0, PARAMS, K=40, gbar=_onehot())
    assert torch.allclose(p1, p2, rtol=1e-13, atol=0)


def test_fp64_adjoint_matches_central_differences(pdq):
    J, pbar = _run(pdq, "B", 0, PARAMS, gbar=_onehot())
    for k, h in ((0, 1e-6), (1, 1e-5)):
        pp, pm = PARAMS.copy(), PARAMS.copy()
        pp[:, k] += h
        pm[:, k] -= h
        Jp, _ = _run(pdq, "B", 0, pp)
        Jm, _ = _run(pdq, "B", 0, pm)
        fd = ((Jp - Jm) / (2 * h)).cpu().numpy()             # [sample, class]
        adj = pbar[:, :, k].cpu().numpy().T                   # [sample, class]
        assert np.allclose(adj, fd, rtol=2e-2, atol=1e-3 * np.max(np.abs(fd)))


@pytest.mark.parametrize("case", ["A", "B", "C"])
def test_mixed_adjoint_close_to_fp64(pdq, case):
    J_ref, dJ_ref = ref(case)
    J, pbar = _run(pdq, case, 1, _params(case), gbar=_onehot())
    assert np.allclose(J.cpu().numpy(), J_ref, rtol=3e-3, atol=1e-6 * np.max(J_ref))
    got = np.transpose(pbar.cpu().numpy(), (1, 0, 2))
    _check_grad(got, dJ_ref, 3e-2, CASES[case]["nonzero"])


def test_autograd_function(pdq):
    J_ref, dJ_ref = ref("A")
    c = CASES["A"]
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    batch = pdq.Batch(0, COUNTS, c["st"])
    cfg = pdq.step_cfg(c["dt"], window_start=c["win"], gravity=c["gravity"])
    p = torch.tensor(PARAMS, dtype=torch.float64, requires_grad=True)
    J = pdq.PdqDeposition.apply(p, field, pdq.phys_default(), batch, cfg, c["steps"], 7, c["eps"], SEED, 0.0)
    w = torch.tensor([[1.0, 2.0], [0.5, -1.0]], dtype=torch.float64, device="cuda")
    (J * w).sum().backward()
    expect = np.einsum("sc,sck->sk", w.cpu().numpy(), dJ_ref)
    assert np.allclose(p.grad.numpy()[:, 0], expect[:, 0], rtol=1e-8)
    assert np.all(p.grad.numpy()[:, 2] == 0)


def test_dgsm_pipeline(pdq):
    from paper_2205_04979_gb300 import uq
    from oracle import mfmc
    r = uq.dgsm_deposition(16, 256, 40, st_plus=(10.0, 100.0), grid=(33, 16, 32), t_window=1.0, eps=0.05,
                           precision=0)
    assert r["grad"].shape == (16, 2, 3) and np.all(r["grad"][..., 2] == 0)      # theta: 0 under all-stick
    nu, bound = mfmc.dgsm_bound(r["grad"], r["J"], [0.1, 1.0, 1.0])
    assert np.allclose(r["nu"], nu, rtol=1e-12) and np.allclose(r["bound"], bound, rtol=1e-12, equal_nan=True)
    assert np.all(r["bound"][2] == 0)
