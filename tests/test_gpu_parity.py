"""GPU-vs-oracle parity of the particle path, through the C ABI (libpdq).

Sizes span several CTA tiles with a ragged tail.  Tolerances: FP64 states
agree to 1e-12 relative after one step and 1e-9 after 50 steps (the kernels
sum the Coulomb pairs in the oracle's order; differences come from rounding
of rsqrt, FMA contraction and libm); integer data (ids, classes, tallies) are
bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


GRID = dict(n_r=33, n_th=16, n_z=32)


@pytest.fixture(scope="module")
def fields(pdq):
    f = pdq.Field(pdq.field_desc(**GRID), 0)
    of = oracle.field_desc(**GRID)
    modes = oracle.field_modes(of, 0)
    return f, of, oracle.field_grid(of, modes), modes


def test_field_parity(pdq, fields):
    f, of, grid, modes = fields
    g64, g32, m = f.grids()
    assert np.allclose(m.cpu().numpy(), modes, rtol=1e-13, atol=1e-15)
    g64 = g64.cpu().numpy()[..., :3]
    assert np.max(np.abs(g64 - grid)) < 1e-11
    g32 = g32.cpu().numpy()[..., :3]
    assert np.max(np.abs(g32 - grid)) < 1e-5 * (1 + np.max(np.abs(grid)))


def test_field_full_size_against_analytic(pdq):
    # 128 x 64 x 128 grid (2^20 nodes): sampled nodes against the oracle's analytic field
    desc = pdq.field_desc(n_r=128, n_th=64, n_z=128)
    f = pdq.Field(desc, 0)
    g64, _, _ = f.grids()
    of = oracle.field_desc(n_r=128, n_th=64, n_z=128)
    m = oracle.field_modes(of, 0)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, [128, 64, 128], size=(200, 3))
    k, j, i = idx[:, 0], idx[:, 1], idx[:, 2]
    r = 180.0 * np.tanh(2.0 * i / 127) / np.tanh(2.0)
    th = 2 * np.pi * j / 64
    P = np.stack([r * np.cos(th), r * np.sin(th), of.l_plus * k / 128], 1)
    ref = oracle.field_velocity(of, m, P)
    got = g64.cpu().numpy()[k, j, i, :3]
    assert np.max(np.abs(got - ref)) < 1e-11


def _setup(pdq, fields, precision, counts, st_plus, params, sigma=0.0, seed=1):
    f, of, grid, _ = fields
    phys = pdq.phys_default()
    st = pdq.State(precision, counts, st_plus)
    prm = pdq.params_tensor(params)
    pdq.seed_particles(f, phys, st, prm, seed, charge_sigma=sigma)
    ost, off = oracle.seed(of, st_plus, counts, params, seed, charge_sigma=sigma)
    return phys, st, prm, ost, off


def _gpu_arrays(st):
    pos, vel, _ = st.current()
    x = st.positions64().cpu().numpy()
    v = vel.double().cpu().numpy()
    q = pos[:, 3].double().cpu().numpy()
    tag = st.tag.cpu().numpy()
    return x, v, q, tag


@pytest.mark.parametrize("precision", [0, 1])
def test_seed_parity(pdq, fields, precision):
    st_plus = [0.1, 1.0, 10.0]
    counts = [1000, 333, 1]
    params = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3], [0.02, 0.9, 0.1]])
    _, st, _, ost, off = _setup(pdq, fields, precision, counts, st_plus, params, sigma=0.5)
    x, v, q, tag = _gpu_arrays(st)
    ref = np.stack([ost.x, ost.y, ost.z], 1)
    assert np.array_equal(tag[:, 0], ost.id) and np.array_equal(tag[:, 1], ost.cls)
    assert np.array_equal(st.count.cpu().numpy(), counts)
    if precision == 0:
        assert np.max(np.abs(x - ref)) < 1e-12 and np.allclose(q, ost.q, rtol=1e-13)
    else:
        assert np.max(np.abs(x[:, :2] - ref[:, :2])) < 1e-12            # FP64 wall-normal position
        assert np.max(np.abs(x[:, 2] - ref[:, 2])) < 1e-4 and np.allclose(q, ost.q, rtol=1e-6)
    assert np.all(v[:, :3] == 0) and np.all(v[:, 3] == 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_seed_independent_parity(pdq, fields, precision):
    # a Philox stream per sample (counter word 3 = s + 1), with lognormal and signed charges so
    # that all three counters are drawn; ids, classes bit-exact, positions as the shared draw
    f, of, _, _ = fields
    st_plus = [0.1, 1.0, 10.0]
    counts = [1000, 333, 1, 0]
    params = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3], [0.02, 0.9, 0.1], [0.03, 0.1, 0.1]])
    phys = pdq.phys_default()
    phys.neg_charge_frac = 0.3
    ophys = oracle.phys()
    ophys.neg_charge_frac = 0.3
    st = pdq.State(precision, counts, st_plus)
    pdq.seed_particles_independent(f, phys, st, pdq.params_tensor(params), 7, charge_sigma=0.5)
    ost, off = oracle.seed(of, st_plus, counts, params, 7, charge_sigma=0.5, p=ophys, independent=True)
    x, v, q, tag = _gpu_arrays(st)
    ref = np.stack([ost.x, ost.y, ost.z], 1)
    assert np.array_equal(tag[:, 0], ost.id) and np.array_equal(tag[:, 1], ost.cls)
    if precision == 0:
        assert np.max(np.abs(x - ref)) < 1e-12 and np.allclose(q, ost.q, rtol=1e-13)
    else:
        assert np.max(np.abs(x[:, :2] - ref[:, :2])) < 1e-12
        assert np.max(np.abs(x[:, 2] - ref[:, 2])) < 1e-4 and np.allclose(q, ost.q, rtol=1e-6)
    assert np.any(q < 0) and not np.array_equal(x[1000:1333], x[:333])     # signed; not shared


def _run_both(pdq, fields, precision, counts, st_plus, params, n_steps, cfg_kw, sigma=0.0, block=0):
    f, of, grid, _ = fields
    phys, st, prm, ost, off = _setup(pdq, fields, precision, counts, st_plus, params, sigma)
    cfg = pdq.step_cfg(0.1, block=block, **cfg_kw)
    tally = pdq.Tally(len(counts), len(st_plus))
    ws = pdq.workspace(st, cfg)
    pdq.step_particles(f, phys, st, prm, cfg, n_steps, tally, ws)
    assert pdq.check_state(st) == 0
    ocfg = oracle.cfg(0.1, **{k: v for k, v in cfg_kw.items() if k not in ("compact_every", "variant")})
    nd, na = oracle.run(of, grid, ocfg, st_plus, off, params, ost, n_steps)
    return st, tally, ost, nd, na


def _compare_by_id(st, ost, off, tol_x, tol_v, max_flip=0):
    """Match live GPU particles to oracle particles by (sample, id); compare states."""
    x, v, q, tag = _gpu_arrays(st)
    counts = st.count.cpu().numpy()
    offs = st.offset.cpu().numpy()
    ref_x = np.stack([ost.x, ost.y, ost.z], 1)
    ref_v = np.stack([ost.vx, ost.vy, ost.vz], 1)
    n_live = 0
    for s in range(len(counts)):
        sl = slice(offs[s], offs[s] + counts[s])
        ids = tag[sl, 0]
        alive = v[sl, 3] > 0.5
        gidx = off[s] + ids
        live = alive & (ost.alive[gidx] == 1)
        mism = np.sum(alive != (ost.alive[gidx] == 1))
        assert mism <= max_flip * len(ids), "deposition decisions differ for %d particles" % mism
        dx = np.abs(x[sl][live] - ref_x[gidx[live]])
        dz = dx[:, 2]
        dz = np.minimum(dz, 720.0 - dz)          # periodic z, checked against the length L = 720
        dx[:, 2] = dz
        scale = 1 + np.abs(ref_x[gidx[live]])
        scale[:, 2] = 720.0
        assert np.all(dx <= tol_x * scale), np.max(dx / scale)
        dv = np.abs(v[sl][live, :3] - ref_v[gidx[live]])
        assert np.all(dv <= tol_v * (1 + np.abs(ref_v[gidx[live]]))), np.max(dv)
        n_live += live.sum()
    return n_live


ST3 = [0.1, 1.0, 10.0]
PRM3 = np.array([[0.1, 0.5, 0.5], [0.08, 0.7, 0.2], [0.05, 0.3, 0.9]])


def test_fp64_one_step_parity(pdq, fields):
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 1, {})
    assert _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 1e-12, 1e-12) > 0
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)


@pytest.mark.parametrize("block", [32, 64, 128, 256])
def test_fp64_fifty_steps_parity(pdq, fields, block):
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 50, {"window_start": 10}, block=block)
    assert _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 1e-9, 1e-9) > 0
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)
    assert nd.sum() > 0          # particles did deposit


@pytest.mark.parametrize("block", [32, 256])
def test_fp64_single_sample_jsplit_parity(pdq, fields, block):
    # one 1,000-particle sample fills few i-tiles, so each tile's pair sum is split over
    # j-chunks (some empty at block 256) and summed by the last chunk to finish
    counts = [1000]
    prm = PRM3[:1]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, [10.0], prm, 20, {"window_start": 5}, block=block)
    assert _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 1e-10, 1e-10) > 0
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)


@pytest.mark.parametrize("variant", [0, 3])
def test_fp64_compaction_parity(pdq, fields, variant):
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 50,
                                       {"window_start": 0, "compact_every": 7, "variant": variant})
    n_live = _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 1e-9, 1e-9)
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)
    # compaction kept exactly the live particles, each once, grouped by z bin (binned at the
    # last compaction, one step before the end)
    cnt = st.count.cpu().numpy()
    assert cnt.sum() == n_live == ost.alive.sum()
    tag = st.tag.cpu().numpy()
    offs = st.offset.cpu().numpy()
    z = st.positions64().cpu().numpy()[:, 2]
    for s in range(3):
        ids = tag[offs[s]:offs[s] + cnt[s], 0]
        assert len(np.unique(ids)) == len(ids)
        b = np.floor(z[offs[s]:offs[s] + cnt[s]] * 256 / 720.0)
        assert np.mean(np.diff(b) >= -2) > 0.95


@pytest.mark.parametrize("block", [64, 128])
def test_fp64_newton_pairs_parity(pdq, fields, block):
    # pair variant 3 in FP64: each pair evaluated once, sums in double through atomics (the
    # order of the additions differs from the oracle's, within the FP64 bars)
    counts = [1000, 333, 129]
    off = np.r_[0, np.cumsum(counts)]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 1, {"variant": 3}, block=block)
    assert _compare_by_id(st, ost, off, 1e-12, 1e-12) > 0
    assert np.array_equal(tally.n_alive.cpu().numpy(), na)
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 50, {"variant": 3, "window_start": 10},
                                       block=block)
    assert _compare_by_id(st, ost, off, 1e-9, 1e-9) > 0
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)


def test_fp64_newton_pairs_chunked_single_sample(pdq, fields):
    # one 6,000-particle sample at 128 threads x 2: 24 tiles of 256, each tile's j range in 3
    # chunks of 2,048 (one work item each, the earlier chunks of late tiles empty)
    counts = [6000]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, [10.0], PRM3[:1], 10,
                                       {"variant": 3, "window_start": 2}, block=128)
    assert _compare_by_id(st, ost, np.r_[0, 6000], 1e-10, 1e-10) > 0
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)


@pytest.mark.parametrize("variant", [0, 3])
def test_fp64_rebound_parity(pdq, fields, variant):
    # Rebounding particles bounce inside the stiff vdW zone (accelerations ~1e4 wall units),
    # which amplifies rounding differences: the bound is 10x the oracle's own response to a
    # 1e-14 relative perturbation of the initial positions, floored at 1e-9.  Variant 3 sums the
    # Coulomb pairs in yet another order (Newton pairs, atomics).
    f, of, grid, _ = fields
    counts = [700, 300]
    prm = np.array([[0.1, 0.05, 0.1], [0.1, 1.0, 0.9]])   # mostly rebound / mostly stick
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, prm, 50, {"mode": 1, "variant": variant},
                                       block=128 if variant == 3 else 0)
    a, off = oracle.seed(of, ST3, counts, prm, 1)
    b = a.copy()
    b.x *= 1 + 1e-14
    oracle.run(of, grid, oracle.cfg(0.1, mode=1), ST3, off, prm, a, 50)
    oracle.run(of, grid, oracle.cfg(0.1, mode=1), ST3, off, prm, b, 50)
    sens = np.max(np.abs(a.x - b.x)[(a.alive == 1) & (b.alive == 1)])
    _compare_by_id(st, ost, off, max(1e-9, 10 * sens / 180.0), max(1e-9, 10 * sens))
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd)


def test_fp64_rebound_one_step_exact(pdq, fields):
    # constructed states just inside the wall, moving outward: every particle hits the wall in
    # this step; low zeta rebounds (CoR from Sec. 4.3), high zeta sticks
    f, of, grid, _ = fields
    phys = pdq.phys_default()
    n = 600
    rng = np.random.default_rng(3)
    cls = (np.arange(n) % 3).astype(np.int32)
    dplus = oracle.class_table(ST3)[:, 1]
    gap = rng.uniform(0.0, 0.3, n)
    r = 180.0 - 0.5 * dplus[cls] - gap
    th = rng.uniform(0, 2 * np.pi, n)
    vr = rng.uniform(4.0, 40.0, n)
    x, y, z = r * np.cos(th), r * np.sin(th), rng.uniform(0, 720.0, n)
    vx, vy, vz = vr * np.cos(th), vr * np.sin(th), rng.uniform(-5, 5, n)
    q = 0.05 * oracle.class_table(ST3)[cls, 4]
    counts = [400, 200]
    prm = np.array([[0.05, 0.02, 0.0], [0.05, 1.0, 0.95]])
    st = pdq.State(0, counts, ST3)
    pos, vel, _ = st.current()
    pos.copy_(torch.tensor(np.stack([x, y, z, q], 1)))
    vel.copy_(torch.tensor(np.stack([vx, vy, vz, np.ones(n)], 1)))
    st.tag.copy_(torch.tensor(np.stack([np.r_[np.arange(400), np.arange(200)], cls], 1), dtype=torch.int32))
    cfg = pdq.step_cfg(0.1, mode=1)
    tally = pdq.Tally(2, 3)
    pdq.step_particles(f, phys, st, pdq.params_tensor(prm), cfg, 1, tally, pdq.workspace(st, cfg))
    ost = oracle.State(n)
    ost.x, ost.y, ost.z, ost.vx, ost.vy, ost.vz, ost.q = x.copy(), y.copy(), z.copy(), vx.copy(), vy.copy(), vz.copy(), q
    ost.cls = cls.copy()
    off = np.array([0, 400, 600])
    nd, _ = oracle.run(of, grid, oracle.cfg(0.1, mode=1), ST3, off, prm, ost, 1)
    assert nd[0].sum() == 0 and nd[1].sum() > 100          # sample 0 rebounds, sample 1 mostly sticks
    _compare_by_id(st, ost, off, 1e-12, 1e-12)
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd)


def test_fp64_lognormal_charge_parity(pdq, fields):
    counts = [900]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3[:1], 20, {}, sigma=0.5)
    _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 1e-9, 1e-9)


@pytest.mark.parametrize("variant,block", [(0, 0), (3, 64), (3, 128)])
def test_mixed_parity(pdq, fields, variant, block):
    # FP32 pair sum / interpolation / velocities, FP64 wall-normal position; variant 3 evaluates
    # each pair once (Newton pairs) and sums through FP32 atomics
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 1, counts, ST3, PRM3, 20, {"variant": variant}, block=block)
    _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 2e-6, 2e-5, max_flip=0.005)


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_variant_without_coulomb(pdq, fields, precision):
    # with the Coulomb force off the Newton-pair sums are not launched; the update runs alone
    counts = [1000, 333, 129]
    forces = oracle.F_ALL & ~oracle.F_COUL
    st, tally, ost, nd, na = _run_both(pdq, fields, precision, counts, ST3, PRM3, 20,
                                       {"variant": 3, "forces": forces, "window_start": 5}, block=64)
    off = np.r_[0, np.cumsum(counts)]
    if precision == 0:
        assert _compare_by_id(st, ost, off, 1e-11, 1e-11) > 0
        assert np.array_equal(tally.n_dep.cpu().numpy(), nd)
    else:
        assert _compare_by_id(st, ost, off, 2e-6, 2e-5, max_flip=0.005) > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_contact_scale_parity(pdq, fields, precision):
    # the Coulomb clamp at the smallest class diameter (contact_scale = d_min / d_max) on both sides
    f, of, grid, _ = fields
    counts = [1000, 333, 129]
    scale = (0.1 / 10.0) ** 0.5                              # d+ grows as sqrt(St+)
    phys = pdq.phys_default()
    phys.contact_scale = scale
    ophys = oracle.phys()
    ophys.contact_scale = scale
    st = pdq.State(precision, counts, ST3)
    prm = pdq.params_tensor(PRM3)
    pdq.seed_particles(f, phys, st, prm, 1)
    ost, off = oracle.seed(of, ST3, counts, PRM3, 1, p=ophys)
    cfg = pdq.step_cfg(0.1, window_start=5, variant=3, block=64)
    tally = pdq.Tally(3, 3)
    pdq.step_particles(f, phys, st, prm, cfg, 20, tally, pdq.workspace(st, cfg))
    nd, na = oracle.run(of, grid, oracle.cfg(0.1, window_start=5), ST3, off, PRM3, ost, 20, p=ophys)
    off = np.r_[0, np.cumsum(counts)]
    if precision == 0:
        assert _compare_by_id(st, ost, off, 1e-10, 1e-10) > 0
        assert np.array_equal(tally.n_dep.cpu().numpy(), nd)
    else:
        assert _compare_by_id(st, ost, off, 2e-6, 2e-5, max_flip=0.005) > 0


def test_vdep_tally_parity(pdq, fields):
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 0, counts, ST3, PRM3, 50, {"window_start": 10})
    vdep, mean, se = pdq.deposition_tally(tally, 0.1)
    ref = oracle.vdep(nd, na, 0.1)
    assert np.allclose(vdep.cpu().numpy(), ref, rtol=1e-14, atol=0)
    assert np.allclose(mean.cpu().numpy(), ref.mean(0), rtol=1e-13)
    assert np.allclose(se.cpu().numpy(), ref.std(0, ddof=1) / np.sqrt(3), rtol=1e-12)


def test_edge_cases(pdq, fields):
    f, of, grid, _ = fields
    phys = pdq.phys_default()
    # an empty sample between non-empty ones, and a single-particle sample
    counts = [0, 5, 1, 0]
    st = pdq.State(0, counts, [1.0])
    prm = pdq.params_tensor(np.tile([0.05, 0.5, 0.5], (4, 1)))
    pdq.seed_particles(f, phys, st, prm, 1)
    cfg = pdq.step_cfg(0.1, compact_every=1)
    tally = pdq.Tally(4, 1)
    ws = pdq.workspace(st, cfg)
    pdq.step_particles(f, phys, st, prm, cfg, 0, tally, ws)        # zero steps: no-op
    pdq.step_particles(f, phys, st, prm, cfg, 3, tally, ws)
    assert pdq.check_state(st) == 0
    assert st.step_index == 3
    ost, off = oracle.seed(of, [1.0], counts, prm.cpu().numpy()[:, :3], 1)
    oracle.run(of, grid, oracle.cfg(0.1), [1.0], off, prm.cpu().numpy()[:, :3], ost, 3)
    _compare_by_id(st, ost, off, 1e-12, 1e-12)
    # workspace too small
    with pytest.raises(pdq.PdqError):
        pdq.step_particles(f, phys, st, prm, cfg, 1, tally, ws[:16])


@pytest.mark.parametrize("variant", [0, 2, 3])
def test_mixed_binned_compaction_parity(pdq, fields, variant):
    # MIXED with compaction: particles are z-binned at the start of the call and at every
    # compaction, and most tile pairs skip the per-pair minimum image (uniform shift of 0 or
    # +-L); results must still match the oracle particle by particle (4 and 8 particles per thread).
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 1, counts, ST3, PRM3, 20,
                                       {"compact_every": 5, "variant": variant})
    n_live = _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 2e-6, 2e-5, max_flip=0.005)
    cnt = st.count.cpu().numpy()
    pos, vel, _ = st.current()
    alive = vel[:, 3].cpu().numpy() > 0.5
    offs = st.offset.cpu().numpy()
    # count[s] = live particles + those deposited since the last compaction (step 15)
    assert sum(alive[offs[s]:offs[s] + cnt[s]].sum() for s in range(3)) == n_live
    # the live particles of each sample are grouped by z bin (256 bins over L)
    z = pos[:, 2].cpu().numpy()
    for s in range(3):
        zs = z[offs[s]:offs[s] + cnt[s]]
        # binned at the last compaction (step 15), then moved for 5 steps: bins stay nearly ordered
        b = np.floor(zs * 256 / 720.0)
        assert np.mean(np.diff(b) >= -2) > 0.95


def test_mixed_rebinning_between_compactions(pdq, fields):
    # compact_every = 100: the MIXED step still re-bins (and compacts) every 10 steps, so after 25
    # steps the state was last binned at step 20; parity with the oracle is unchanged
    counts = [1000, 333, 129]
    st, tally, ost, nd, na = _run_both(pdq, fields, 1, counts, ST3, PRM3, 25, {"compact_every": 100})
    n_live = _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 2e-6, 2e-5, max_flip=0.005)
    assert n_live > 0
    z = st.current()[0][:, 2].cpu().numpy()
    cnt, offs = st.count.cpu().numpy(), st.offset.cpu().numpy()
    for s in range(3):
        b = np.floor(z[offs[s]:offs[s] + cnt[s]] * 256 / 720.0)
        assert np.mean(np.diff(b) >= -2) > 0.95


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_state_reported(pdq, fields, precision):
    # failure made on the host: one particle's velocity is set to NaN; the step runs to the end,
    # the kernels set the device error word, pdq_check_state reports PDQ_ERR_NAN once and clears it
    f = fields[0]
    phys = pdq.phys_default()
    st = pdq.State(precision, [200, 100], ST3)
    prm = pdq.params_tensor(PRM3[:2])
    pdq.seed_particles(f, phys, st, prm, 1)
    _, vel, _ = st.current()
    vel[17, 0] = float("nan")
    cfg = pdq.step_cfg(0.1, compact_every=2 if precision == 1 else 0)
    tally = pdq.Tally(2, 3)
    pdq.step_particles(f, phys, st, prm, cfg, 4, tally, pdq.workspace(st, cfg))
    assert pdq.check_state(st) == -4           # PDQ_ERR_NAN
    assert pdq.check_state(st) == 0            # cleared
    # the other sample is untouched by the NaN
    _, vel, _ = st.current()
    off, cnt = st.offset.cpu().numpy(), st.count.cpu().numpy()
    assert torch.isfinite(vel[off[1]:off[1] + cnt[1]]).all()


def test_capture_efficiency(pdq, fields):
    f, of, _, _ = fields
    v = torch.tensor([[1e-3, 2e-2], [0.0, 5e-1]], dtype=torch.float64, device="cuda")
    ce = pdq.capture_efficiency(f, pdq.phys_default(), v)
    assert torch.allclose(ce.cpu(), v.cpu() * oracle.capture_factor(of), rtol=1e-14, atol=0)


@pytest.mark.parametrize("block,counts", [(128, [0, 5, 1, 0]), (128, [1536, 1537, 1535, 3073]),
                                          (64, [768, 769, 767, 1537])])
def test_mixed_newton_pairs_edge_sizes(pdq, fields, block, counts):
    # pair variant 3 at 12 particles per thread: 1,536-particle tiles at 128 threads, 768 at 64;
    # empty and one-particle samples, samples of exactly one tile, one tile +-1 and two tiles + 1
    # (the boundary between a tile's own block and the later particles), with compaction every step
    prm = np.tile(PRM3[:1], (len(counts), 1))
    st, tally, ost, nd, na = _run_both(pdq, fields, 1, counts, ST3, prm, 5, {"variant": 3, "compact_every": 1},
                                       block=block)
    _compare_by_id(st, ost, np.r_[0, np.cumsum(counts)], 2e-6, 2e-5, max_flip=0.005)
    assert np.array_equal(tally.n_alive.cpu().numpy(), na)


def test_mixed_newton_pairs_graph_replay(pdq, fields):
    # graph mode (three replays of a captured 2-step call) against direct launches: the float
    # atomics of variant 3 sum in a run-dependent order, so the bar is the MIXED one
    f, of, grid, _ = fields
    counts = [1500, 700]
    prm = PRM3[:2]
    stream = torch.cuda.Stream()
    runs = []
    for graph in (True, False):
        phys, st, p, ost, off = _setup(pdq, fields, 1, counts, ST3, prm)
        cfg = pdq.step_cfg(0.1, block=128, variant=3, use_graph=graph)
        tally = pdq.Tally(2, 3)
        ws = pdq.workspace(st, cfg)
        torch.cuda.synchronize()          # seeding and allocation ran on the default stream
        with torch.cuda.stream(stream):
            for _ in range(3):
                pdq.step_particles(f, phys, st, p, cfg, 2, tally, ws, stream)
        stream.synchronize()
        assert st.step_index == 6 and int(st.ctl[0]) == 6
        runs.append((st, tally))
    pdq.release_graphs()
    oracle.run(of, grid, oracle.cfg(0.1), ST3, off, prm, ost, 6)
    for st, tally in runs:
        _compare_by_id(st, ost, off, 2e-6, 2e-5, max_flip=0.005)
    a, b = (r[1].n_alive.cpu().numpy() for r in runs)
    assert np.abs(a - b).max() <= 2           # a deposition decision may flip on last-bit differences
