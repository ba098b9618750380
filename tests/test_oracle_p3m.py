"""Pins of the periodic-pipe electrostatics and of the reference P3M.

The exact sum over the z images is pinned to closed forms (the trigamma series
of charges on a line, the field of a line charge far away, Newton's third
law); the reference P3M is pinned to that exact sum within its accuracy at the
chosen splitting, to its exact invariants (no self-force, zero total force)
and to its error falling as the screening is resolved more finely.
"""
import numpy as np
import pytest
from scipy.special import polygamma

R, L = 180.0, 720.0


@pytest.fixture(scope="module")
def cloud():
    rng = np.random.default_rng(1)
    n = 300
    r = 170.0 * np.sqrt(rng.uniform(size=n))
    th = rng.uniform(0, 2 * np.pi, n)
    return r * np.cos(th), r * np.sin(th), rng.uniform(0, L, n), rng.uniform(0.5, 1.5, n)


@pytest.mark.parametrize("zz", [0.7, 3.0, 8.2])
def test_periodic_sum_on_axis_trigamma(orc, zz):
    # charges on the axis, period Lp: F_z = (psi'(z/Lp) - psi'(1 - z/Lp)) / Lp^2
    Lp = 10.0
    s = orc.coulomb_periodic(np.zeros(2), np.zeros(2), np.array([zz, 0.0]), np.array([0.0, 1.0]), Lp, 1e-9)
    ref = (polygamma(1, zz / Lp) - polygamma(1, 1 - zz / Lp)) / Lp ** 2
    assert s[0, 2] == pytest.approx(ref, rel=1e-12)
    assert abs(s[0, 0]) < 1e-15 and abs(s[0, 1]) < 1e-15


def test_periodic_sum_line_charge_limit_and_third_law(orc, cloud):
    # far from a periodic row of unit charges the field is that of a line charge 2/(Lp rho)
    s = orc.coulomb_periodic(np.array([100.0, 0.0]), np.zeros(2), np.array([3.0, 0.0]), np.array([0.0, 1.0]), 10.0,
                             1e-9)
    assert s[0, 0] == pytest.approx(2.0 / (10.0 * 100.0), rel=1e-9) and abs(s[0, 2]) < 1e-12
    x, y, z, q = cloud
    s = orc.coulomb_periodic(x, y, z, q, L, 0.29, n_img=500)
    tot = np.sum(q[:, None] * s, 0)
    assert np.all(np.abs(tot) < 1e-12 * np.sum(np.abs(q[:, None] * s), 0))


def _p3m(alpha_h, M=32, Nz=64, rc_alpha=3.3):
    from oracle import p3m
    h = 2 * R / M
    alpha = alpha_h / h
    return p3m, p3m.Desc(R, L, M, Nz, alpha, rc_alpha / alpha, n_img=100)


def _rms(s, ex):
    return np.sqrt(np.mean(np.sum((s - ex) ** 2, 1)) / np.mean(np.sum(ex ** 2, 1)))


def test_p3m_matches_the_periodic_sum(orc, cloud):
    x, y, z, q = cloud
    ex = orc.coulomb_periodic(x, y, z, q, L, 0.29, n_img=1000)
    p3m, d = _p3m(0.5)
    Gh = p3m.influence(d)
    s = p3m.coulomb_sums(d, x, y, z, q, 0.29, Gh)
    assert _rms(s, ex) < 3e-4
    rel = np.linalg.norm(s - ex, axis=1) / np.linalg.norm(ex, axis=1)
    assert np.max(rel) < 1e-2
    # the short-range part matters: the mesh alone is far off
    mesh_only = p3m.mesh_sums(d, Gh, x, y, z, q)
    assert _rms(mesh_only, ex) > 30 * _rms(s, ex)
    # zero total force (odd kernel, same weights for assignment and interpolation)
    tot = np.sum(q[:, None] * s, 0)
    assert np.all(np.abs(tot) < 1e-10 * np.sum(np.abs(q[:, None] * s), 0))


def test_p3m_error_falls_with_finer_screening(orc, cloud):
    x, y, z, q = cloud
    ex = orc.coulomb_periodic(x, y, z, q, L, 0.29, n_img=1000)
    errs = []
    for ah in (0.7, 0.5):
        p3m, d = _p3m(ah)
        errs.append(_rms(p3m.coulomb_sums(d, x, y, z, q, 0.29), ex))
    assert errs[1] < errs[0] / 2


def test_p3m_no_self_force_and_removed_particles(orc):
    p3m, d = _p3m(0.5)
    Gh = p3m.influence(d)
    for pos in [(0.0, 0.0, 0.0), (37.3, -101.2, 355.5), (-170.0, 5.0, 719.9)]:
        s = p3m.coulomb_sums(d, *(np.array([v]) for v in pos), np.array([1.0]), 0.29, Gh)
        assert np.all(np.abs(s) < 1e-12)
    # a removed particle neither feels nor exerts a force
    x, y, z, q = np.array([0.0, 5.0, 60.0]), np.zeros(3), np.array([10.0, 10.0, 30.0]), np.ones(3)
    s = p3m.coulomb_sums(d, x, y, z, q, 0.29, Gh, alive=[1, 0, 1])
    s2 = p3m.coulomb_sums(d, x[[0, 2]], y[[0, 2]], z[[0, 2]], q[[0, 2]], 0.29, Gh)
    assert np.all(s[1] == 0) and np.allclose(s[[0, 2]], s2, rtol=1e-12, atol=1e-15)
