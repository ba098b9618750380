"""Pins of the oracle's force laws: van der Waals, image charge, Coulomb, rebound.

References: closed forms and limits stated in the paper (Sec. 2.2, App. B,
Sec. 4.3), the Fig. 3 statements that follow from the printed formulas, and
mathematical identities (force = -grad energy, Newton's third law).
"""
import numpy as np
import pytest

K_E = 1 / (4 * np.pi * 8.854e-12)
USTAR, NU = 0.27, 1.5e-5
ELL = NU / USTAR
ACC = NU / USTAR ** 3


def test_vdw_limits(orc):
    A, d = 1e-18, 5e-6
    # sphere-sphere: F -> A d / (24 delta^2) for delta << d
    for dl in [1e-10, 1e-9]:
        assert abs(orc.vdw_pp(A, d, dl) / (A * d / (24 * dl ** 2)) - 1) < 5 * dl / d + 1e-12  # first-order correction is -4 delta/d
    # the bracketed form of Eq. (vdw) equals A d^6 / (6 delta^2 (2d+delta)^2 (d+delta)^3)
    for dl in [1e-9, 1e-7, 1e-6, 4e-6]:
        ref = A * d ** 6 / (6 * dl ** 2 * (2 * d + dl) ** 2 * (d + dl) ** 3)
        assert abs(orc.vdw_pp(A, d, dl) / ref - 1) < 1e-12


def test_wall_forces_match_low_fidelity_forms(orc):
    # App. B gives the particle-wall forces per unit mass:
    #   F_elec = -3 q^2 / (8 pi^2 eps0 rho_p d^3 y^2),  F_vdw = -A d / (12 m (y - d/2)^2).
    # The high-fidelity image (F_C at 2y) and wall vdW (2 F_vw) must reduce to them.
    f = orc.field_desc()
    st = [1.0]
    t = orc.class_table(st)
    dp, dplus, m = t[0, 2], t[0, 1], t[0, 3]
    qt = 0.07 * t[0, 4]                      # charge in units of 500 e
    q = qt * 500 * 1.6e-19
    yplus = 3.0                              # centre-to-wall distance, wall units
    c = orc.cfg(0.1, forces=orc.F_IMAGE)
    a = orc.wall_accel(f, c, st, np.array([f.r_plus - yplus]), np.array([0.0]), np.array([qt]),
                       np.array([0], np.int32), 0.5)
    y = yplus * ELL
    lf = 3 * q ** 2 / (8 * np.pi ** 2 * 8.854e-12 * 2650 * dp ** 3 * y ** 2)
    assert abs(a[0, 0] / (lf * ACC) - 1) < 1e-10 and a[0, 1] == 0 and a[0, 2] == 0
    # vdW at a small gap: A d / (12 m delta^2) up to O(delta/d)
    zeta = 0.8
    c = orc.cfg(0.1, forces=orc.F_VDW)
    for gap in [2e-9, 2e-8]:
        x = f.r_plus - 0.5 * dplus - gap / ELL
        a = orc.wall_accel(f, c, st, np.array([x]), np.array([0.0]), np.array([0.0]),
                           np.array([0], np.int32), zeta)
        lf = zeta * 1e-18 * dp / (12 * m * gap ** 2)
        assert abs(a[0, 0] / (lf * ACC) - 1) < 5 * gap / dp + 1e-6


def test_vdw_saturation_and_cutoff(orc):
    f = orc.field_desc()
    st = [0.1]
    t = orc.class_table(st)
    dp, dplus = t[0, 2], t[0, 1]
    c = orc.cfg(0.1, forces=orc.F_VDW)

    def acc(gap_m):
        x = f.r_plus - 0.5 * dplus - gap_m / ELL
        return orc.wall_accel(f, c, st, np.array([x]), np.array([0.0]), np.array([0.0]),
                              np.array([0], np.int32), 1.0)[0, 0]

    # saturates below delta_min = 1e-9 m (Sec. 2.2)
    assert acc(0.0) == pytest.approx(acc(1e-9), rel=1e-6)
    assert acc(-1e-8) == pytest.approx(acc(1e-9), rel=1e-6)
    # cut off beyond delta_max = d_p / 4
    assert acc(0.24 * dp) > 0 and acc(0.26 * dp) == 0.0
    # monotone decay toward the cut-off
    g = np.geomspace(1.1e-9, 0.24 * dp, 30)
    a = np.array([acc(x) for x in g])
    assert np.all(np.diff(a) < 0)


def test_fig3_statements(orc):
    # Fig. 3 / Sec. 2.2, from the printed formulas with xi = 0.1, zeta = 1:
    A = 1e-18
    for d in [1.6e-6, 5e-6, 16e-6]:
        q = 0.1 * 500 * 1.6e-19 * (d / 1e-6) ** 2
        # vdW dominates at short separation, Coulomb beyond O(1e-7..1e-6) m
        gaps = np.geomspace(1e-9, 1e-4, 400)
        diff = np.array([orc.vdw_pp(A, d, s) - orc.coulomb_pp(q, q, s + d) for s in gaps])
        cross = gaps[np.argmax(diff < 0)]
        assert diff[0] > 0 and diff[-1] < 0 and 1e-8 < cross < 1e-6
        # particle-wall vdW always exceeds particle-particle vdW at the mean spacing
        for n_p in [1e9, 1.6e10, 1e12]:
            s = n_p ** (-1 / 3)
            assert orc.wall_average(1, d, q, A) > orc.vdw_pp(A, d, s)
    # the pp Coulomb force overtakes the wall image force at n_p of order 1e11 (mid size)
    d = 5e-6
    q = 0.1 * 500 * 1.6e-19 * 25
    pw = orc.wall_average(0, d, q, A)
    n = np.geomspace(1e9, 1e13, 2000)
    pp = np.array([orc.coulomb_pp(q, q, x ** (-1 / 3)) for x in n])
    n_cross = n[np.argmax(pp > pw)]
    assert 3e10 < n_cross < 3e11
    # at the paper's n_p = 1.6e10 the wall image force dominates the pp force (d = 1.6, 5 um)
    for d in [1.6e-6, 5e-6]:
        q = 0.1 * 500 * 1.6e-19 * (d / 1e-6) ** 2
        assert orc.wall_average(0, d, q, A) > orc.coulomb_pp(q, q, 1.6e10 ** (-1 / 3))
    # larger particles: weaker vdW acceleration, stronger Coulomb acceleration at long range
    m = lambda d: 2650 * np.pi / 6 * d ** 3
    dd = [1.6e-6, 5e-6, 16e-6]
    av = [orc.vdw_pp(A, d, 1e-8) / m(d) for d in dd]
    ac = [orc.coulomb_pp(0.1 * 8e-17 * (d / 1e-6) ** 2, 0.1 * 8e-17 * (d / 1e-6) ** 2, 1e-4) / m(d) for d in dd]
    assert av[0] > av[1] > av[2] and ac[0] < ac[1] < ac[2]


def _energy(orc, f, st_plus, P, q, cls):
    # Coulomb energy per unit mass of particle i's class is not symmetric; use the
    # pair energy U = k q_i q_j / r (SI) and check m_i a_i = -grad_i U.
    n = len(q)
    U = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            d = P[i] - P[j]
            d[2] -= f.l_plus * np.rint(d[2] / f.l_plus)
            U += K_E * (q[i] * 8e-17) * (q[j] * 8e-17) / (np.linalg.norm(d) * ELL)
    return U


def test_coulomb_is_minus_grad_energy(orc):
    # brute force on 6 particles: finite-difference gradient of the pair energy
    f = orc.field_desc()
    st_plus = [1.0, 10.0]
    t = orc.class_table(st_plus)
    rng = np.random.default_rng(5)
    n = 6
    P = np.stack([rng.uniform(-60, 60, n), rng.uniform(-60, 60, n), rng.uniform(0, f.l_plus, n)], 1)
    q = rng.uniform(-3, 3, n)
    cls = (np.arange(n) % 2).astype(np.int32)
    a = orc.coulomb_accel(f, st_plus, P[:, 0], P[:, 1], P[:, 2], q, cls)
    h = 1e-4
    for i in range(n):
        for k in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            F = -(_energy(orc, f, st_plus, Pp, q, cls) - _energy(orc, f, st_plus, Pm, q, cls)) / (2 * h * ELL)
            a_si = F / t[cls[i], 3]
            assert abs(a[i, k] - a_si * ACC) < 1e-6 * np.max(np.abs(a)) + 1e-300


def test_coulomb_newton_third_law_and_permutation(orc):
    f = orc.field_desc()
    st_plus = [0.1, 1.0, 10.0]
    t = orc.class_table(st_plus)
    rng = np.random.default_rng(6)
    n = 300
    x, y = rng.uniform(-100, 100, n), rng.uniform(-100, 100, n)
    z = rng.uniform(0, f.l_plus, n)
    q = rng.uniform(0, 2, n)
    cls = rng.integers(0, 3, n).astype(np.int32)
    a = orc.coulomb_accel(f, st_plus, x, y, z, q, cls)
    ma = a * t[cls, 3][:, None]
    assert np.max(np.abs(ma.sum(0))) < 1e-12 * np.sum(np.abs(ma))
    perm = rng.permutation(n)
    ap = orc.coulomb_accel(f, st_plus, x[perm], y[perm], z[perm], q[perm], cls[perm])
    assert np.allclose(ap, a[perm], rtol=1e-12, atol=1e-14 * np.max(np.abs(a)))
    # like charges repel: two particles on the x axis push apart
    a2 = orc.coulomb_accel(f, st_plus, np.array([0.0, 10.0]), np.zeros(2), np.zeros(2), np.ones(2),
                           np.zeros(2, np.int32))
    assert a2[0, 0] < 0 < a2[1, 0]
    # dead particles neither feel nor exert force
    alive = np.ones(n, np.int32)
    alive[::3] = 0
    ad = orc.coulomb_accel(f, st_plus, x, y, z, q, cls, alive)
    keep = alive == 1
    ak = orc.coulomb_accel(f, st_plus, x[keep], y[keep], z[keep], q[keep], cls[keep])
    assert np.allclose(ad[keep], ak, rtol=1e-12) and np.all(ad[~keep] == 0)


def test_coulomb_minimum_image_and_clamp(orc):
    f = orc.field_desc()
    st_plus = [10.0]
    t = orc.class_table(st_plus)
    # two particles near z = 0 and z = L: the minimum image makes them close neighbours
    a = orc.coulomb_accel(f, st_plus, np.zeros(2), np.zeros(2), np.array([1.0, f.l_plus - 1.0]), np.ones(2),
                          np.zeros(2, np.int32))
    coef = K_E * (8e-17) ** 2 / t[0, 3] / ELL ** 2 * ACC
    assert a[0, 2] == pytest.approx(coef / 2.0 ** 2, rel=1e-12)
    # inside the contact distance the force saturates at r = d+
    dplus = t[0, 1]
    a = orc.coulomb_accel(f, st_plus, np.array([0.0, 0.3 * dplus]), np.zeros(2), np.zeros(2), np.ones(2),
                          np.zeros(2, np.int32))
    assert a[1, 0] == pytest.approx(coef * 0.3 * dplus / dplus ** 3, rel=1e-12)


def test_coulomb_clamp_scale(orc):
    # the clamp distance is contact_scale x the largest class diameter: with the smallest class's
    # diameter (scale d_min/d_max) a pair at 0.3 d_max feels the unclamped 1/r^2 force, and a pair
    # closer than d_min saturates there
    f = orc.field_desc()
    st_plus = [0.1, 10.0]
    t = orc.class_table(st_plus)
    dmin, dmax = t[0, 1], t[1, 1]
    p = orc.phys()
    p.contact_scale = dmin / dmax
    coef = K_E * (8e-17) ** 2 / t[1, 3] / ELL ** 2 * ACC     # on the St+ = 10 particle (class 1)
    cls = np.array([1, 1], np.int32)
    for r, expect in ((0.3 * dmax, 1.0 / (0.3 * dmax) ** 2), (0.5 * dmin, 0.5 * dmin / dmin ** 3)):
        a = orc.coulomb_accel(f, st_plus, np.array([0.0, r]), np.zeros(2), np.zeros(2), np.ones(2), cls, p=p)
        assert a[1, 0] == pytest.approx(coef * expect, rel=1e-12)
        a1 = orc.coulomb_accel(f, st_plus, np.array([0.0, r]), np.zeros(2), np.zeros(2), np.ones(2), cls)
        assert a1[1, 0] == pytest.approx(coef * r / dmax ** 3, rel=1e-12)     # default: clamped at d_max


def test_rebound_model(orc):
    # Sec. 4.3 / Fig. 12: CoR_n falls with zeta, theta and the impact velocity; CoR_n = 0 is sticking.
    st = 0.1
    z = np.linspace(0, 1, 11)
    v = np.geomspace(0.5, 50, 20)
    cz = np.array([[orc.cor(st, zz, 0.5, vv) for vv in v] for zz in z])
    assert np.all(np.diff(cz, axis=0) <= 1e-15) and np.all(np.diff(cz, axis=1) <= 1e-15)
    th = np.linspace(0, 1, 11)
    ct = np.array([[orc.cor(1.0, 1.0, tt, vv) for vv in v] for tt in th])
    assert np.all(np.diff(ct, axis=0) <= 1e-15)
    # threshold: stick iff sigma_y0^2 (1 - theta)^2 / (rho_p E) <= 2 A_cont gamma_c / m_p,
    # with A_cont = pi d^2/4 and gamma_c = zeta A0 / (24 pi delta_c^2)
    t = orc.class_table([st])
    d, m = t[0, 2], t[0, 3]
    elastic = (200e6 * 0.5) ** 2 / (2650 * 70e9)
    per_zeta = 2 * (np.pi * d * d / 4) * (1e-18 / (24 * np.pi * (0.165e-9) ** 2)) / m
    z_star = elastic / per_zeta
    assert orc.cor(st, z_star * 0.999, 0.5, 1.0) > 0 and orc.cor(st, z_star * 1.001, 0.5, 1.0) == 0
    # energy balance value: V_n2 = sqrt(elastic - zeta per_zeta), CoR capped at 1
    vn1 = 20.0
    assert orc.cor(st, 0.05, 0.5, vn1) == pytest.approx(np.sqrt(elastic - 0.05 * per_zeta) / vn1, rel=1e-12)
    assert orc.cor(st, 0.0, 0.0, 0.1) == 1.0


def test_capture_efficiency_factor(orc):
    # Sec. 4.3: CE = (4L/D)(u*/U_b) V_dep; for the paper's L = 10 D and U_b = 4 m/s, u* = 0.27 m/s
    f = orc.field_desc(l_over_r=20.0)
    assert orc.capture_factor(f) == pytest.approx(40 * 0.27 / 4.0, rel=1e-12)
    assert orc.capture_factor(orc.field_desc()) == pytest.approx(8 * 0.27 / 4.0, rel=1e-12)
