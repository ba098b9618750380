"""GPU adjoint of the smoothed deposition functional (pdq_adjoint_run, pdq_adjoint_run_seeded,
pdq_adjoint_reverse) against the oracle's forward-mode dual numbers and against central
finite differences.

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
    return pdq.adjoint_run_seeded(field, pdq.phys_default(), batch, pdq.params_tensor(params), cfg, c["steps"],
                                  K, c["eps"], SEED, gbar=gbar, eps_stick=c.get("eps_stick", 10.0))


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


# ---------------------------------------------------------------------------
# Sizes that cross the MIXED Newton-pair tiles: the forward sums take 1,536-particle i-tiles
# and the pair VJP 512-particle ones, so only samples above those sizes run the off-diagonal
# blocks, where the pair term enters the j side with the opposite sign (1,537 and 3,073: one
# particle past one and two sums tiles, and past 3 and 6 VJP tiles).  Charge active
# (case A's forces), eps+ = 0.5 and 0.02 (the widest and narrowest smoothing of the
# 256 x 16,384 adjoint workload).
# ---------------------------------------------------------------------------
TILE_COUNTS = [1537, 513, 3073, 1, 0]
TILE_PARAMS = np.array([[0.09, 0.7, 0.4], [0.06, 0.3, 0.8], [0.075, 0.5, 0.5], [0.05, 0.6, 0.3],
                        [0.07, 0.4, 0.6]])
TILE = dict(st=[0.1, 1.0], steps=24, dt=0.05, gravity=(0, 0, 1), win=5)
_TREF = {}


def _onehot_sc(S, Cn):
    g = torch.zeros((Cn, S, Cn), dtype=torch.float64, device="cuda")
    for c in range(Cn):
        g[c, :, c] = 1.0
    return g


def _rounding_bars(run, x, y, z, J, dJ):
    """FP64 bars: 10x the oracle's own response to +-4e-16 relative changes of the initial positions
    (the narrow sigmoid at eps+ = 0.02 and the stiff vdW zone amplify rounding), at least 1e-12
    for J and 1e-8 of each gradient column's largest entry."""
    rng = np.random.default_rng(7)

    def pert(a):
        return a * (1 + 4e-16 * rng.choice([-1.0, 1.0], a.shape))
    J2, dJ2 = run(pert(x), pert(y), pert(z))
    nz = np.abs(J) > 0
    rJ = np.max(np.abs(J2 - J)[nz] / np.abs(J)[nz]) if nz.any() else 0.0
    sc = np.max(np.abs(dJ), axis=(0, 1))
    rg = np.max(np.max(np.abs(dJ2 - dJ), axis=(0, 1)) / np.where(sc > 0, sc, 1.0))
    return max(1e-12, 10 * rJ), max(1e-8, 10 * rg)


def _tile_ref(eps):
    if eps not in _TREF:
        of = oracle.field_desc(**GRID)
        grid = oracle.field_grid(of, oracle.field_modes(of, 0))
        st, off = oracle.seed(of, TILE["st"], TILE_COUNTS, np.c_[np.ones(5), TILE_PARAMS[:, 1:]], SEED)
        cf = oracle.cfg(TILE["dt"], gravity=TILE["gravity"], smooth_eps=eps, window_start=TILE["win"])

        def run(x, y, z):
            return oracle.smooth_run(of, grid, cf, TILE["st"], off, TILE_PARAMS, x, y, z, st.q, st.cls,
                                     TILE["steps"])
        J, dJ = run(st.x, st.y, st.z)
        _TREF[eps] = (J, dJ) + _rounding_bars(run, st.x, st.y, st.z, J, dJ)
    return _TREF[eps]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("eps", [0.5, 0.02])
def test_adjoint_across_newton_tiles_matches_dual_numbers(pdq, precision, eps):
    J_ref, dJ_ref, bar_J, bar_g = _tile_ref(eps)
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    batch = pdq.Batch(precision, TILE_COUNTS, TILE["st"])
    cfg = pdq.step_cfg(TILE["dt"], window_start=TILE["win"], gravity=TILE["gravity"])
    J, pbar = pdq.adjoint_run_seeded(field, pdq.phys_default(), batch, pdq.params_tensor(TILE_PARAMS), cfg,
                                     TILE["steps"], 5, eps, SEED, gbar=_onehot_sc(5, 2))
    got = np.transpose(pbar.cpu().numpy(), (1, 0, 2))     # [sample, class, param]
    J = J.cpu().numpy()
    assert np.all(J[4] == 0) and np.all(got[4] == 0)      # the empty sample
    assert np.all(got[..., 1:] == 0.0) and np.all(dJ_ref[..., 1:] == 0.0)   # no particle within d/4 of the wall
    if precision == 0:
        assert np.allclose(J, J_ref, rtol=bar_J, atol=1e-300), (bar_J, np.max(np.abs(J / J_ref - 1)[J_ref > 0]))
        _check_grad(got, dJ_ref, bar_g, (0,))
    else:
        assert np.allclose(J, J_ref, rtol=3e-3, atol=1e-6 * np.max(J_ref))
        _check_grad(got, dJ_ref, 3e-2, (0,))


@pytest.mark.parametrize("eps", [0.5, 0.02])
def test_stored_pair_sums_match_dual_numbers(pdq, eps):
    # MIXED with the forward sweep's Newton-pair sums kept for the reverse sweep's recompute
    # (workspace + pdq_adjoint_stored_sums_size): the same bar against the dual numbers as the
    # recomputing path, and that path's J and gradients up to float summation order
    J_ref, dJ_ref, _, _ = _tile_ref(eps)
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    cfg = pdq.step_cfg(TILE["dt"], window_start=TILE["win"], gravity=TILE["gravity"])
    out = {}
    for store in (False, True):
        batch = pdq.Batch(1, TILE_COUNTS, TILE["st"])
        J, pbar = pdq.adjoint_run_seeded(field, pdq.phys_default(), batch, pdq.params_tensor(TILE_PARAMS), cfg,
                                         TILE["steps"], 5, eps, SEED, gbar=_onehot_sc(5, 2), store_sums=store)
        out[store] = (J.cpu().numpy(), np.transpose(pbar.cpu().numpy(), (1, 0, 2)))
    J, got = out[True]
    assert np.all(J[4] == 0) and np.all(got[4] == 0)
    assert np.allclose(J, J_ref, rtol=3e-3, atol=1e-6 * np.max(J_ref))
    _check_grad(got, dJ_ref, 3e-2, (0,))
    J0, got0 = out[False]
    assert np.allclose(J, J0, rtol=1e-5, atol=1e-9 * np.max(J0))
    sc = np.max(np.abs(got0[..., 0]))
    assert np.max(np.abs(got[..., 0] - got0[..., 0])) <= 1e-3 * sc


def test_stored_pair_sums_reverse_alone(pdq):
    # forward sweep with the sums kept, then pdq_adjoint_reverse on the same workspace, against
    # one combined call; a workspace whose forward sweep kept no sums is refused before any work
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    phys = pdq.phys_default()
    cfg = pdq.step_cfg(TILE["dt"], window_start=TILE["win"], gravity=TILE["gravity"])
    prm = pdq.params_tensor(TILE_PARAMS)
    batch = pdq.Batch(1, TILE_COUNTS, TILE["st"])
    g = _onehot_sc(5, 2)
    J1, p1 = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, TILE["steps"], 5, 0.5, SEED, gbar=g,
                                    store_sums=True)
    ws = pdq.adjoint_workspace(batch.b, TILE["steps"], 5, store_sums=True)
    J2, _ = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, TILE["steps"], 5, 0.5, SEED, ws=ws)
    p2 = pdq.adjoint_reverse(field, phys, batch.b, prm, cfg, TILE["steps"], 5, 0.5, g, ws)
    assert np.allclose(J1.cpu().numpy(), J2.cpu().numpy(), rtol=1e-5, atol=0)
    a, b = p1.cpu().numpy(), p2.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(a))
    fresh = torch.zeros_like(ws)
    with pytest.raises(pdq.PdqError, match="adjoint_reverse"):
        pdq.adjoint_reverse(field, phys, batch.b, prm, cfg, TILE["steps"], 5, 0.5, g, fresh)


# ---------------------------------------------------------------------------
# The adjoint started from a caller's state: pdq_step_particles advances a transient (with
# deposits; with and without compaction), then pdq_adjoint_run differentiates the next steps
# from that state; the oracle's dual numbers start from the same arrays (positions,
# velocities, alive flags as weights, charge per unit xi = q_eff / xi, classes from the tags).
# ---------------------------------------------------------------------------
def _state_arrays(state, params):
    pos_t, vel_t, xy_t = state.current()
    pos = pos_t.cpu().numpy().astype(np.float64)
    vel = vel_t.cpu().numpy().astype(np.float64)
    xy = None if xy_t is None else xy_t.cpu().numpy()
    tag = state.tag.cpu().numpy()
    cnt = state.count.cpu().numpy()
    off = state.offset.cpu().numpy()
    N = off[-1]
    x, y, z, qh, w = (np.zeros(N) for _ in range(5))
    v = np.zeros((N, 3))
    cls = np.zeros(N, np.int32)
    for s in range(len(cnt)):
        r = np.arange(off[s], off[s] + cnt[s])
        x[r] = xy[r, 0] if xy is not None else pos[r, 0]
        y[r] = xy[r, 1] if xy is not None else pos[r, 1]
        z[r], v[r] = pos[r, 2], vel[r, :3]
        w[r], cls[r] = vel[r, 3], tag[r, 1]
        qh[r] = pos[r, 3] / params[s, 0]
    return off, x, y, z, qh, cls, v, w


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("compact_every", [0, 5])
def test_adjoint_from_stepped_state_matches_dual_numbers(pdq, precision, compact_every):
    c = CASES["B"]
    P = _params("B")
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    phys = pdq.phys_default()
    state = pdq.State(precision, COUNTS, c["st"])
    prm = pdq.params_tensor(P)
    pdq.seed_particles(field, phys, state, prm, seed=SEED)
    # a transient under a stronger test-only gravity toward the wall, so that a few particles
    # deposit before the adjoint starts (the oracle deposits 5 of 429 in these 60 steps)
    cfg_t = pdq.step_cfg(c["dt"], gravity=(20.0, 0.0, 0.0), compact_every=compact_every)
    tally = pdq.Tally(2, 2)
    pdq.step_particles(field, phys, state, prm, cfg_t, 60, tally, pdq.workspace(state, cfg_t))
    assert int(tally.n_dep.sum()) > 0                       # deposits before the adjoint starts
    if compact_every:
        assert np.all(state.count.cpu().numpy() < np.array(COUNTS))   # empty slots after compaction
    before = [t.clone() for t in state.current() if t is not None] + [state.tag.clone(), state.count.clone()]

    # the adjoint keeps the stronger gravity, so particles reach the vdW range (zeta enters)
    cfg = pdq.step_cfg(c["dt"], window_start=c["win"], gravity=(20.0, 0.0, 0.0))
    J, pbar, _ = pdq.adjoint_run(field, phys, state, prm, cfg, 40, 7, c["eps"], gbar=_onehot())
    after = [t for t in state.current() if t is not None] + [state.tag, state.count]
    assert all(torch.equal(a, b) for a, b in zip(before, after))          # init is read only

    off, x, y, z, qh, cls, v, w = _state_arrays(state, P)
    of = oracle.field_desc(**GRID)
    grid = oracle.field_grid(of, oracle.field_modes(of, 0))
    cf = oracle.cfg(c["dt"], gravity=(20.0, 0.0, 0.0), smooth_eps=c["eps"], window_start=c["win"])

    def run(x, y, z):
        return oracle.smooth_run(of, grid, cf, c["st"], off, P, x, y, z, qh, cls, 40, v0=v, w0=w)
    J_ref, dJ_ref = run(x, y, z)
    got = np.transpose(pbar.cpu().numpy(), (1, 0, 2))
    assert np.all(got[..., 2] == 0.0) and np.all(dJ_ref[..., 2] == 0.0)
    if precision == 0:
        bar_J, bar_g = _rounding_bars(run, x, y, z, J_ref, dJ_ref)
        assert np.allclose(J.cpu().numpy(), J_ref, rtol=bar_J, atol=1e-300)
        _check_grad(got, dJ_ref, bar_g, (0, 1))
    else:
        assert np.allclose(J.cpu().numpy(), J_ref, rtol=3e-3, atol=1e-6 * np.max(J_ref))
        _check_grad(got, dJ_ref, 3e-2, (0, 1))


def test_adjoint_reverse_alone_matches_the_combined_call(pdq):
    c = CASES["A"]
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    phys = pdq.phys_default()
    batch = pdq.Batch(0, COUNTS, c["st"])
    cfg = pdq.step_cfg(c["dt"], window_start=c["win"], gravity=c["gravity"])
    prm = pdq.params_tensor(PARAMS)
    J1, p1 = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, c["steps"], 7, c["eps"], SEED, gbar=_onehot())
    ws = pdq.adjoint_workspace(batch.b, c["steps"], 7)
    J2, none = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, c["steps"], 7, c["eps"], SEED, ws=ws)
    assert none is None
    p2 = pdq.adjoint_reverse(field, phys, batch.b, prm, cfg, c["steps"], 7, c["eps"], _onehot(), ws)
    p3 = pdq.adjoint_reverse(field, phys, batch.b, prm, cfg, c["steps"], 7, c["eps"], _onehot(), ws)
    # the double atomics of the tallies and pbar may add in another order: rounding only
    assert torch.allclose(J1, J2, rtol=1e-13, atol=0)
    assert torch.allclose(p1, p2, rtol=1e-12, atol=1e-14 * float(p1.abs().max()))
    assert torch.allclose(p2, p3, rtol=1e-12, atol=1e-14 * float(p1.abs().max()))


def test_adjoint_from_state_rejects_zero_charge_scale(pdq):
    c = CASES["A"]
    field = pdq.Field(pdq.field_desc(**GRID), 0)
    phys = pdq.phys_default()
    state = pdq.State(0, COUNTS, c["st"])
    P = PARAMS.copy()
    pdq.seed_particles(field, phys, state, pdq.params_tensor(P), seed=SEED)
    P[1, 0] = 0.0                                          # charge per unit xi is undefined
    cfg = pdq.step_cfg(c["dt"], window_start=c["win"], gravity=c["gravity"])
    with pytest.raises(pdq.PdqError):
        pdq.adjoint_run(field, phys, state, pdq.params_tensor(P), cfg, 10, 5, c["eps"])
