"""pdq_step_particles_noalloc: the particle step for callers that cannot allocate.

Some callers cannot hand the step a device workspace: their device memory is
owned by another allocator or held under a hard cap, or they run a
latency-critical loop that must not call cudaMalloc (it can synchronise the
device).  The no-allocation entry point keeps the step's work queue in scratch
compiled into libpdq.  These tests call it through the C ABI two times in a row
and check every result against the workspace entry point, pdq_step_particles,
with the same configuration: the one-sided pair loop (variant 0) to 1e-12
relative with integer data exact, and the Newton-pair sums (variant 3, whose
atomics add in any order) particle by particle at the parity bars of the other
GPU tests.  The file sorts last so that a run stopping at its first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


def _snapshot(st, tally):
    pos, vel, xy = st.current()
    out = {"pos": pos.double().cpu().numpy(), "vel": vel.double().cpu().numpy(), "tag": st.tag.cpu().numpy(),
           "count": st.count.cpu().numpy(), "n_dep": tally.n_dep.cpu().numpy(),
           "n_alive": tally.n_alive.cpu().numpy()}
    if xy is not None:
        out["xy"] = xy.cpu().numpy()
    return out


def _by_id(snap, offset):
    """Rows of the live particles keyed by (sample, particle id); the step reorders rows by z."""
    out = {}
    cnt = snap["count"]
    for s in range(len(cnt)):
        for r in range(offset[s], offset[s] + cnt[s]):
            out[(s, int(snap["tag"][r, 0]))] = r
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 3])
def test_noalloc_matches_workspace_entry(pdq, precision, variant):
    st_plus = [0.1, 1.0, 10.0]
    counts = [900, 257, 40]
    params = np.array([[0.1, 0.5, 0.5], [0.07, 0.2, 0.3], [0.02, 0.9, 0.8]])
    phys = pdq.phys_default()
    field = pdq.Field(pdq.field_desc(n_r=33, n_th=16, n_z=32), 0)
    prm = pdq.params_tensor(params)
    a = pdq.State(precision, counts, st_plus)
    b = pdq.State(precision, counts, st_plus)
    pdq.seed_particles(field, phys, a, prm, 5)
    pdq.seed_particles(field, phys, b, prm, 5)
    cfg = pdq.step_cfg(0.1, compact_every=3, window_start=2, variant=variant)
    ta, tb = pdq.Tally(3, 3), pdq.Tally(3, 3)
    ws = pdq.workspace(a, cfg)
    offset = a.offset.cpu().numpy()
    for call in range(2):
        pdq.step_particles(field, phys, a, prm, cfg, 7, ta, ws)
        pdq.step_particles_noalloc(field, phys, b, prm, cfg, 7, tb)
        assert pdq.check_state(a) == 0 and pdq.check_state(b) == 0
        sa, sb = _snapshot(a, ta), _snapshot(b, tb)
        assert a.step_index == b.step_index == 7 * (call + 1)
        assert int(sa["count"].sum()) > 0
        if variant == 0:
            # one-sided sums in a fixed order: the same rows, integers exact
            for k in ("tag", "count", "n_dep", "n_alive"):
                assert np.array_equal(sa[k], sb[k]), k
            for k in ("pos", "vel", "xy"):
                if k in sa:
                    assert np.allclose(sa[k], sb[k], rtol=1e-12, atol=1e-12), k
            continue
        # Newton pairs (variant 3) add their sums through atomics in any order, in the scratch
        # as in the workspace, so the two runs differ by rounding: particles are matched by id
        # (the z-binning may order rows differently) at the parity bars of the other GPU tests,
        # FP64 1e-10 relative over 14 steps, MIXED 2e-6 for positions (z of L) and 2e-5 for
        # velocities, with at most one deposition event that rounding moved across the wall
        assert np.abs(sa["n_dep"] - sb["n_dep"]).sum() <= (0 if precision == 0 else 1)
        ia, ib = _by_id(sa, offset), _by_id(sb, offset)
        common = sorted(set(ia) & set(ib))
        assert len(common) >= len(ia) - (0 if precision == 0 else 1)
        ra, rb = np.array([ia[k] for k in common]), np.array([ib[k] for k in common])
        pa = sa["xy"][ra] if precision == 1 else sa["pos"][ra, :2]
        pb = sb["xy"][rb] if precision == 1 else sb["pos"][rb, :2]
        za, zb = sa["pos"][ra, 2], sb["pos"][rb, 2]
        va, vb = sa["vel"][ra, :3], sb["vel"][rb, :3]
        rp, rv = (1e-10, 1e-10) if precision == 0 else (2e-6, 2e-5)
        assert np.allclose(pa, pb, rtol=rp, atol=rp * 180.0)
        assert np.allclose(za, zb, rtol=0, atol=rp * 720.0)
        vs = np.abs(va).max()
        assert np.all(np.abs(va - vb) <= rv * vs)


def test_noalloc_rejects_oversize_and_graph(pdq):
    L = pdq.lib()
    # a state too large for the built-in scratch is rejected before any device work
    s = pdq.StateStruct()
    s.precision, s.n_samples, s.n_classes, s.st_plus[0] = 0, 1, 1, 1.0
    s.capacity = (1 << 31) - 1
    s.offset = s.count = s.tag = s.ctl = 16
    for h in range(2):
        s.pos[h] = s.vel[h] = 16
    cfg = pdq.step_cfg(0.1)
    t = pdq.TallyStruct(16, 16)
    phys = pdq.phys_default()
    field = pdq.Field(pdq.field_desc(n_r=5, n_th=4, n_z=4), 0)
    rc = L.pdq_step_particles_noalloc(field.handle, C.byref(phys), C.byref(s), C.c_void_p(16), C.byref(cfg), 1,
                                      C.byref(t), None)
    assert rc == -8                                   # PDQ_ERR_WORKSPACE
    cfg.use_graph = 1
    rc = L.pdq_step_particles_noalloc(field.handle, C.byref(phys), C.byref(s), C.c_void_p(16), C.byref(cfg), 1,
                                      C.byref(t), None)
    assert rc == -1                                   # PDQ_ERR_INVALID_ARG
