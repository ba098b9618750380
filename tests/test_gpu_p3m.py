"""GPU P3M electrostatics (pdq_p3m_*) against the reference P3M of oracle/p3m.py
and against the exact periodic sum, through the C ABI.

The GPU and the reference take the same steps on the same mesh, so their sums
agree to rounding (atomics and FFT ordering: 1e-9 of the RMS sum); both sit
within the method's accuracy (RMS 1e-3 for a cloud with charges of both
signs) of the exact sum over the z images.
The P3M step is checked against the oracle stepping with the reference sums.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import p3m as ref  # noqa: E402

ST3 = [0.1, 1.0, 10.0]
GRID = dict(n_r=33, n_th=16, n_z=32)
M, NZ, AH = 32, 64, 0.5


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


@pytest.fixture(scope="module")
def setup(pdq):
    f = pdq.Field(pdq.field_desc(**GRID), 0)
    of = oracle.field_desc(**GRID)
    grid = oracle.field_grid(of, oracle.field_modes(of, 0))
    h = 2 * 180.0 / M
    alpha = AH / h
    plan = pdq.P3M(f, M=M, Nz=NZ, alpha=alpha, r_cut=3.3 / alpha, n_img=100, max_particles=2000)
    d = ref.Desc(180.0, 720.0, M, NZ, alpha, 3.3 / alpha, n_img=100)
    return f, of, grid, plan, d, ref.influence(d)


def _cloud(counts, seed):
    rng = np.random.default_rng(seed)
    n = int(np.sum(counts))
    cls = rng.integers(0, 3, n).astype(np.int32)
    dplus = oracle.class_table(ST3)[cls, 1]
    r = (180.0 - 0.5 * dplus) * np.sqrt(rng.uniform(size=n))
    th = rng.uniform(0, 2 * np.pi, n)
    x, y, z = r * np.cos(th), r * np.sin(th), rng.uniform(0, 720.0, n)
    q = 0.05 * oracle.class_table(ST3)[cls, 4] * np.where(rng.uniform(size=n) < 0.3, -1.0, 1.0)
    v = rng.normal(0, 0.5, (n, 3))
    ids = np.concatenate([np.arange(c) for c in counts]).astype(np.int32)
    return x, y, z, q, v, cls, ids


def _state(pdq, precision, counts, arr, alive=None):
    x, y, z, q, v, cls, ids = arr
    n = len(x)
    alive = np.ones(n) if alive is None else alive
    st = pdq.State(precision, counts, ST3)
    pos, vel, xy = st.current()
    pos.copy_(torch.tensor(np.stack([x, y, z, q * alive], 1)).to(pos.dtype))
    vel.copy_(torch.tensor(np.concatenate([v, alive[:, None]], 1)).to(vel.dtype))
    if xy is not None:
        xy.copy_(torch.tensor(np.stack([x, y], 1)))
    st.tag.copy_(torch.tensor(np.stack([ids, cls], 1), dtype=torch.int32))
    return st


def _ref_sums(d, Gh, counts, x, y, z, q, alive=None):
    off = np.r_[0, np.cumsum(counts)]
    out = np.zeros((len(x), 3))
    dc = oracle.class_table(ST3)[:, 1].max()
    for s in range(len(counts)):
        sl = slice(off[s], off[s + 1])
        out[sl] = ref.coulomb_sums(d, x[sl], y[sl], z[sl], q[sl], dc, Gh, None if alive is None else alive[sl])
    return out


def _rms(a):
    return np.sqrt(np.mean(np.sum(a * a, 1)))


def test_p3m_sums_match_reference_fp64(pdq, setup):
    f, of, grid, plan, d, Gh = setup
    counts = [700, 333]
    arr = _cloud(counts, 1)
    alive = (np.random.default_rng(2).uniform(size=len(arr[0])) > 0.1).astype(np.float64)
    st = _state(pdq, 0, counts, arr, alive)
    got = plan.coulomb(pdq.phys_default(), st).cpu().numpy()
    x, y, z, q = arr[:4]
    want = _ref_sums(d, Gh, counts, x, y, z, q, alive > 0.5)
    assert np.max(np.abs(got - want)) <= 1e-9 * _rms(want)
    assert np.all(got[alive < 0.5] == 0)


def test_p3m_sums_accuracy_against_exact(pdq, setup):
    f, of, grid, plan, d, Gh = setup
    counts = [900]
    arr = _cloud(counts, 3)
    st = _state(pdq, 0, counts, arr)
    got = plan.coulomb(pdq.phys_default(), st).cpu().numpy()
    x, y, z, q = arr[:4]
    dc = oracle.class_table(ST3)[:, 1].max()
    exact = oracle.coulomb_periodic(x, y, z, q, 720.0, dc, n_img=1000)
    # charges of both signs partly cancel, so the relative error is above the 1.4e-4 of a
    # like-signed cloud; it is the reference's own error on this cloud
    want = _ref_sums(d, Gh, counts, x, y, z, q)
    assert _rms(got - exact) < 1e-3 * _rms(exact)
    assert _rms(got - exact) <= 1.001 * _rms(want - exact)


def test_p3m_sums_mixed_state(pdq, setup):
    f, of, grid, plan, d, Gh = setup
    counts = [513]
    arr = _cloud(counts, 4)
    st = _state(pdq, 1, counts, arr)
    got = plan.coulomb(pdq.phys_default(), st).cpu().numpy()
    x, y, z, q = arr[:4]
    z32, q32 = z.astype(np.float32).astype(np.float64), q.astype(np.float32).astype(np.float64)
    want = _ref_sums(d, Gh, counts, x, y, z32, q32)
    assert np.max(np.abs(got - want)) <= 1e-9 * _rms(want)


@pytest.mark.parametrize("block", [64, 256])
def test_p3m_step_matches_oracle(pdq, setup, block):
    # the P3M step = the oracle's step with the reference P3M sums of each step's start state
    f, of, grid, plan, d, Gh = setup
    counts = [600, 257]
    arr = _cloud(counts, 5)
    x, y, z, q, v, cls, ids = arr
    st = _state(pdq, 0, counts, arr)
    prm = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3]])
    cfg = pdq.step_cfg(0.1, block=block, window_start=0)
    tally = pdq.Tally(2, 3)
    steps = 4
    pdq.step_particles_p3m(f, pdq.phys_default(), st, pdq.params_tensor(prm), cfg, steps, tally, plan,
                           pdq.workspace(st, cfg))
    assert pdq.check_state(st) == 0
    ost = oracle.State(len(x))
    ost.x, ost.y, ost.z, ost.q, ost.cls, ost.id = x.copy(), y.copy(), z.copy(), q.copy(), cls.copy(), ids.copy()
    ost.vx, ost.vy, ost.vz = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    off = np.r_[0, np.cumsum(counts)]
    tallies = (np.zeros((2, 3), np.int64), np.zeros((2, 3), np.int64))
    for k in range(steps):
        ext = _ref_sums(d, Gh, counts, ost.x, ost.y, ost.z, ost.q, ost.alive == 1)
        oracle.run_ext(of, grid, oracle.cfg(0.1, window_start=0), ST3, off, prm, ost, ext, step0=k, tallies=tallies)
    gx = st.positions64().cpu().numpy()
    gv = st.current()[1].double().cpu().numpy()
    tag = st.tag.cpu().numpy()
    gidx = off[np.repeat(np.arange(2), counts)] + tag[:, 0]
    live = gv[:, 3] > 0.5
    assert np.array_equal(live, ost.alive[gidx] == 1)
    rx = np.stack([ost.x, ost.y, ost.z], 1)[gidx]
    rv = np.stack([ost.vx, ost.vy, ost.vz], 1)[gidx]
    assert np.max(np.abs(gx[live] - rx[live]) / (1 + np.abs(rx[live]))) < 1e-11
    assert np.max(np.abs(gv[live, :3] - rv[live]) / (1 + np.abs(rv[live]))) < 1e-10
    assert np.array_equal(tally.n_alive.cpu().numpy(), tallies[1])
