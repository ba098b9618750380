"""GPU-vs-oracle parity of the particle-particle contact forces (App. A.2:
soft-sphere collisions and Eq. vdw between particles), through the C ABI.

Constructed states put pairs of particles with charges of both signs at or
near contact (overlapping, inside the van der Waals range, approaching),
spread over several CTA tiles with a ragged tail, and step them at dt+ = 1e-4
(a few contact times).  FP64 states agree with the oracle to 1e-12 after one
step; over 30 steps the bound is the oracle's own response to last-bit changes
of the initial positions (the van der Waals force of a pair ~1e-5 wall units
apart is that sensitive), at least 1e-9.  MIXED keeps z in FP32, so its states
sit at small z (fine FP32 spacing) and are compared at FP32-level tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402

ST3 = [0.1, 1.0, 10.0]
GRID = dict(n_r=33, n_th=16, n_z=32)
DT = 1e-4      # contact time 15 dt = 1.5e-3: the soft-sphere stiffness then holds the vdW pull
               # at an overlap of ~1e-4 wall units (~10 nm), as with the stiffness the paper states


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
    f = pdq.Field(pdq.field_desc(**GRID), 0)
    of = oracle.field_desc(**GRID)
    return f, of, oracle.field_grid(of, oracle.field_modes(of, 0))


def _contact_state(counts, seed, z_range=(50.0, 600.0)):
    """Pairs of particles at surface gaps in [-2e-4, 0.3 d] (wall units), approaching, with charges of both signs."""
    rng = np.random.default_rng(seed)
    tab = oracle.class_table(ST3)
    n = int(np.sum(counts))
    cls = rng.integers(0, 3, n).astype(np.int32)
    d = tab[cls, 1]
    x, y, z = np.zeros(n), np.zeros(n), np.zeros(n)
    v = rng.normal(0.0, 0.3, (n, 3))
    for a in range(0, n - 1, 2):
        b = a + 1
        r = 150.0 * np.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * np.pi)
        c = np.array([r * np.cos(th), r * np.sin(th), rng.uniform(*z_range)])
        nv = rng.normal(size=3)
        nv /= np.linalg.norm(nv)
        sep = 0.5 * (d[a] + d[b]) + rng.uniform(-2e-4, 0.3 * min(d[a], d[b]))
        pa, pb = c - 0.5 * sep * nv, c + 0.5 * sep * nv
        x[a], y[a], z[a] = pa
        x[b], y[b], z[b] = pb
        vapp = rng.uniform(0.0, 0.1)
        v[a] += 0.5 * vapp * nv
        v[b] -= 0.5 * vapp * nv
    if n % 2:
        x[-1], y[-1], z[-1] = 0.0, 0.0, z_range[0]
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    q = 0.05 * tab[cls, 4] * sign
    ids = np.concatenate([np.arange(c) for c in counts]).astype(np.int32)
    return x, y, z, v, q, cls, ids


def _load(pdq, precision, counts, arrays):
    x, y, z, v, q, cls, ids = arrays
    n = len(x)
    st = pdq.State(precision, counts, ST3)
    pos, vel, xy = st.current()
    pos.copy_(torch.tensor(np.stack([x, y, z, q], 1)).to(pos.dtype))
    vel.copy_(torch.tensor(np.concatenate([v, np.ones((n, 1))], 1)).to(vel.dtype))
    if xy is not None:
        xy.copy_(torch.tensor(np.stack([x, y], 1)))
    st.tag.copy_(torch.tensor(np.stack([ids, cls], 1), dtype=torch.int32))
    ost = oracle.State(n)
    ost.x, ost.y, ost.z = x.copy(), y.copy(), z.copy()
    if precision == 1:      # the oracle starts from the FP32-rounded z and q the GPU holds
        ost.z = z.astype(np.float32).astype(np.float64)
        q = q.astype(np.float32).astype(np.float64)
    ost.vx, ost.vy, ost.vz = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    if precision == 1:
        ost.vx, ost.vy, ost.vz = (a.astype(np.float32).astype(np.float64) for a in (ost.vx, ost.vy, ost.vz))
    ost.q, ost.cls, ost.id = q.copy(), cls.copy(), ids.copy()
    return st, ost


def _run(pdq, fields, precision, counts, arrays, steps, forces, block=0, compact_every=0, mode=0, variant=0):
    f, of, grid = fields
    prm = np.array([[0.05, 0.8, 0.5], [0.1, 0.3, 0.2]])[:len(counts)]
    st, ost = _load(pdq, precision, counts, arrays)
    cfg = pdq.step_cfg(DT, forces=forces, block=block, compact_every=compact_every, mode=mode, variant=variant)
    tally = pdq.Tally(len(counts), 3)
    pdq.step_particles(f, pdq.phys_default(), st, pdq.params_tensor(prm), cfg, steps, tally, pdq.workspace(st, cfg))
    assert pdq.check_state(st) == 0
    off = np.r_[0, np.cumsum(counts)]
    nd, na = oracle.run(of, grid, oracle.cfg(DT, forces=forces, mode=mode), ST3, off, prm, ost, steps)
    return st, tally, ost, off, nd, na


def _compare(st, ost, off, tol_x, tol_v):
    x = st.positions64().cpu().numpy()
    _, vel, _ = st.current()
    v = vel.double().cpu().numpy()
    tag = st.tag.cpu().numpy()
    counts, offs = st.count.cpu().numpy(), st.offset.cpu().numpy()
    ref_x = np.stack([ost.x, ost.y, ost.z], 1)
    ref_v = np.stack([ost.vx, ost.vy, ost.vz], 1)
    ex = ev = 0.0
    for s in range(len(counts)):
        sl = slice(offs[s], offs[s] + counts[s])
        gidx = off[s] + tag[sl, 0]
        live = (v[sl, 3] > 0.5) & (ost.alive[gidx] == 1)
        assert np.array_equal(v[sl, 3] > 0.5, ost.alive[gidx] == 1)
        dx = np.abs(x[sl][live] - ref_x[gidx[live]])
        dx[:, 2] = np.minimum(dx[:, 2], 720.0 - dx[:, 2])
        ex = max(ex, np.max(dx / (1 + np.abs(ref_x[gidx[live]]))))
        ev = max(ev, np.max(np.abs(v[sl][live, :3] - ref_v[gidx[live]]) / (1 + np.abs(ref_v[gidx[live]]))))
    assert ex <= tol_x and ev <= tol_v, (ex, ev)
    return ex, ev


def _moved_by_contact(pdq, fields, precision, counts, arrays, steps):
    """How far the contact forces move the velocities (so that the parity test is not vacuous)."""
    _, _, ost, _, _, _ = _run(pdq, fields, precision, counts, arrays, steps, oracle.F_ALL)
    _, _, ost2, _, _, _ = _run(pdq, fields, precision, counts, arrays, steps, oracle.F_ALL | oracle.F_CONTACT)
    return np.max(np.abs(np.stack([ost.vx - ost2.vx, ost.vy - ost2.vy, ost.vz - ost2.vz])))


def _oracle_sensitivity(counts, arrays, steps, forces, z_ulp32=False, seed=0):
    """Largest relative change of the oracle's final positions and velocities when every initial
    coordinate moves by one unit in the last place (FP32 places for z when z_ulp32): the gap of a
    touching pair is ~1e-5 wall units, so the van der Waals force near delta_min turns last-bit
    differences of the absolute positions into ~1e-9 relative velocity differences within steps."""
    f, of, grid = None, oracle.field_desc(**GRID), None
    grid = oracle.field_grid(of, oracle.field_modes(of, 0))
    prm = np.array([[0.05, 0.8, 0.5], [0.1, 0.3, 0.2]])[:len(counts)]
    off = np.r_[0, np.cumsum(counts)]
    rng = np.random.default_rng(seed)
    out = []
    for k in range(2):
        x, y, z, v, q, cls, ids = (a.copy() for a in arrays)
        if z_ulp32:
            z = z.astype(np.float32).astype(np.float64)
        if k:
            x = np.nextafter(x, np.where(rng.uniform(size=len(x)) < 0.5, -np.inf, np.inf))
            y = np.nextafter(y, np.where(rng.uniform(size=len(y)) < 0.5, -np.inf, np.inf))
            if z_ulp32:
                z = np.nextafter(z.astype(np.float32), np.where(rng.uniform(size=len(z)) < 0.5, -np.inf,
                                                                np.inf).astype(np.float32)).astype(np.float64)
            else:
                z = np.nextafter(z, np.where(rng.uniform(size=len(z)) < 0.5, -np.inf, np.inf))
        st = oracle.State(len(x))
        st.x, st.y, st.z, st.q, st.cls, st.id = x, y, z, q, cls, ids
        st.vx, st.vy, st.vz = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
        oracle.run(of, grid, oracle.cfg(DT, forces=forces), ST3, off, prm, st, steps)
        out.append((np.stack([st.x, st.y, st.z], 1), np.stack([st.vx, st.vy, st.vz], 1)))
    (xa, va), (xb, vb) = out
    return (np.max(np.abs(xa - xb) / (1 + np.abs(xa))), np.max(np.abs(va - vb) / (1 + np.abs(va))))


@pytest.mark.parametrize("block", [32, 64, 256])
def test_fp64_contact_one_step_exact(pdq, fields, block):
    counts = [517, 301]
    arr = _contact_state(counts, 5)
    st, tally, ost, off, nd, na = _run(pdq, fields, 0, counts, arr, 1, oracle.F_ALL | oracle.F_CONTACT, block=block)
    _compare(st, ost, off, 1e-13, 1e-12)


@pytest.mark.parametrize("block", [32, 64, 256])
def test_fp64_contact_parity(pdq, fields, block):
    counts = [517, 301]
    arr = _contact_state(counts, 5)
    fl = oracle.F_ALL | oracle.F_CONTACT
    st, tally, ost, off, nd, na = _run(pdq, fields, 0, counts, arr, 30, fl, block=block)
    sx, sv = _oracle_sensitivity(counts, arr, 30, fl)
    _compare(st, ost, off, max(1e-9, 10 * sx), max(1e-9, 10 * sv))
    assert np.array_equal(tally.n_dep.cpu().numpy(), nd) and np.array_equal(tally.n_alive.cpu().numpy(), na)
    assert _moved_by_contact(pdq, fields, 0, counts, arr, 30) > 1e-2


@pytest.mark.parametrize("forces", ["collide", "vdw_pp"])
def test_fp64_contact_terms_separately(pdq, fields, forces):
    counts = [300]
    arr = _contact_state(counts, 9)
    fl = oracle.F_DRAG | (oracle.F_COLLIDE if forces == "collide" else oracle.F_VDWPP)
    st, _, ost, off, _, _ = _run(pdq, fields, 0, counts, arr, 20, fl, block=64)
    sx, sv = _oracle_sensitivity(counts, arr, 20, fl)
    _compare(st, ost, off, max(1e-9, 10 * sx), max(1e-9, 10 * sv))


@pytest.mark.parametrize("compact_every,variant,block", [(0, 0, 64), (5, 0, 64), (0, 3, 64), (5, 3, 64), (0, 3, 128)])
def test_mixed_contact_parity(pdq, fields, compact_every, variant, block):
    # MIXED rounds z to FP32 every step: the bound is the oracle's response to one FP32 unit of
    # z, times the number of steps.  Variant 3: Coulomb sums by Newton pairs, contact forces in
    # the contact variant that takes them; at 128 threads each sample is one 1,024-particle tile
    # whose four warp blocks are full, nearly empty (5 of 517) or empty.
    counts = [517, 301]
    arr = _contact_state(counts, 6, z_range=(2.0, 12.0))
    fl = oracle.F_ALL | oracle.F_CONTACT
    st, tally, ost, off, nd, na = _run(pdq, fields, 1, counts, arr, 30, fl, block=block,
                                       compact_every=compact_every, variant=variant)
    sx, sv = _oracle_sensitivity(counts, arr, 30, fl, z_ulp32=True)
    _compare(st, ost, off, max(2e-5, 30 * sx), max(2e-3, 30 * sv))


@pytest.mark.parametrize("precision", [0, 1])
def test_contact_variant_without_contacts_is_bit_identical(pdq, fields, precision):
    # seeded, well separated particles: no pair within the contact range, so the contact
    # variant must reproduce the plain step (MIXED bit for bit: same Coulomb sums, same update)
    f, of, grid = fields
    phys = pdq.phys_default()
    counts = [700, 333]
    prm = pdq.params_tensor(np.array([[0.05, 0.5, 0.5], [0.08, 0.2, 0.7]]))
    out = []
    for forces in (pdq.F_ALL, pdq.F_ALL | pdq.F_CONTACT):
        st = pdq.State(precision, counts, ST3)
        pdq.seed_particles(f, phys, st, prm, 3)
        cfg = pdq.step_cfg(0.05, forces=forces, block=128)
        tally = pdq.Tally(2, 3)
        pdq.step_particles(f, phys, st, prm, cfg, 10, tally, pdq.workspace(st, cfg))
        pos, vel, xy = st.current()
        out.append([t.clone() for t in (pos, vel) + ((xy,) if xy is not None else ())])
    for a, b in zip(*out):
        if precision == 1:
            assert torch.equal(a, b)
        else:   # the plain FP64 step splits these small samples' pair sums over j-chunks (other rounding)
            assert torch.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_signed_charge_seed_parity(pdq, fields):
    f, of, _ = fields
    phys = pdq.phys_default()
    phys.neg_charge_frac = 0.4
    op = oracle.phys()
    op.neg_charge_frac = 0.4
    counts = [1000, 257]
    prm = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3]])
    st = pdq.State(0, counts, ST3)
    pdq.seed_particles(f, phys, st, pdq.params_tensor(prm), 11, charge_sigma=0.5)
    ost, _ = oracle.seed(of, ST3, counts, prm, 11, charge_sigma=0.5, p=op)
    q = st.current()[0][:, 3].cpu().numpy()
    assert np.allclose(q, ost.q, rtol=1e-13, atol=0) and np.any(q < 0) and np.any(q > 0)
