"""Pins of the oracle's 1-D Eulerian low-fidelity model (App. B, readings c33-c41).

Each part is checked against something other than its own formula:
  - the closures R_ratio and eps against the stationary covariance of the
    linear SDE they stand for (scipy's Lyapunov solver);
  - the kinetic wall condition against quadrature of the Gaussian one-way flux,
    and against the printed form of App. B;
  - the force potentials against the high-fidelity oracle's own wall forces
    (image charge by Coulomb's law at 2y, the wall vdW as 2 x Eq. vdw);
  - D_B against the Stokes-Einstein relation;
  - the momentum march against the exact (implicit) solution of the ODE under
    a uniform force, with its order of accuracy (first: the drag is fully implicit);
  - the continuity march against closed forms (constant V and D, V = 0 with
    D(y) = D0 + D1 y^2) and against scipy's ODE solver;
  - the whole model against the closed form of the pure-Brownian limit, and
    against the trends App. B / Sec. 2.3 state (Fig. 5).
"""
import math

import numpy as np
import pytest
from scipy import integrate, linalg

from oracle import lf_eulerian as lf


@pytest.fixture(scope="module")
def field_var(orc):
    f = orc.field_desc(n_r=64, n_th=32, n_z=64)
    g = orc.field_grid(f, orc.field_modes(f, 0))
    return f, lf.fluid_variance(g)


def test_response_ratio_and_diffusivity_from_the_sde():
    # fluid velocity u: Ornstein-Uhlenbeck with variance s2 and integral time T; particle velocity
    # v: dv/dt = (u - v)/tau.  Stationary covariance from A S + S A^T + B B^T = 0.
    for T, tau, s2 in [(10.0, 0.1, 1.0), (10.0, 10.0, 0.3), (3.0, 50.0, 2.0)]:
        A = np.array([[-1.0 / T, 0.0], [1.0 / tau, -1.0 / tau]])
        BB = np.array([[2.0 * s2 / T, 0.0], [0.0, 0.0]])
        S = linalg.solve_continuous_lyapunov(A, -BB)
        assert abs(S[0, 0] / s2 - 1) < 1e-12
        assert abs(S[1, 1] / S[0, 0] - lf.response_ratio(tau, T)) < 1e-12
        # long-time diffusivity = integral of the stationary autocovariance e^{At} S = (-A)^{-1} S
        Dlong = np.linalg.solve(-A, S)[1, 1]
        assert abs(Dlong / lf.eddy_diffusivity(s2, T) - 1) < 1e-12


@pytest.mark.parametrize("u,sigma", [(0.0, 1.0), (0.3, 1.0), (2.0, 0.5), (-0.4, 0.7), (5.0, 0.01)])
def test_wall_flux_is_the_gaussian_one_way_flux(u, sigma):
    # wall-ward speed s ~ N(u, sigma^2): flux into an absorbing wall = int_0^inf s pdf(s) ds
    pdf = lambda s: math.exp(-0.5 * ((s - u) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
    ref, _ = integrate.quad(lambda s: s * pdf(s), 0.0, max(u, 0.0) + 40 * sigma, epsabs=0, epsrel=1e-13,
                            limit=400, points=[max(u, 0.0)])
    K = lf.wall_flux_factor(-u, sigma)
    assert abs(-K / ref - 1) < 1e-10


@pytest.mark.parametrize("u,sigma", [(0.3, 1.0), (2.0, 0.5), (0.05, 0.2)])
def test_wall_flux_matches_the_printed_condition(u, sigma):
    # App. B: -(D_B + eps) drho/dy = rho_w V (exp(-M^2)/(2 sqrt(pi) M) - (1 - erf M)/2) with
    # J = -(D_B + eps) drho/dy + rho V: J/rho_w - V is the printed bracket times V.
    V = -u
    M = u / (math.sqrt(2) * sigma)
    printed = V * (math.exp(-M * M) / (2 * math.sqrt(math.pi) * M) - 0.5 * (1 - math.erf(M)))
    K = lf.wall_flux_factor(V, sigma)
    assert abs(K - (V + printed)) < 1e-14 * abs(V) and abs(K / (V + printed) - 1) < 1e-14


def test_potentials_reproduce_the_high_fidelity_wall_forces(orc):
    # -dPhi/dy of the low-fidelity potentials against the oracle's own high-fidelity wall
    # accelerations: image charge (Coulomb's law with the image at 2y) and wall vdW (2 x Eq. vdw,
    # whose small-gap limit App. B prints); compared where neither model clamps.
    p = orc.phys()
    f = orc.field_desc()
    st = [0.1, 1.0, 10.0]
    tab = orc.class_table(st, p)
    _, ell, _ = lf.units(p)
    for c in range(len(st)):
        ce, cv = lf.potential_constants(p, tab[c])
        dplus, dp = tab[c, 1], tab[c, 2]
        xi, zeta = 0.07, 0.6
        for y in [0.8 * dplus + 0.5, 2.0, 9.0]:
            a = orc.wall_accel(f, orc.cfg(0.1, forces=orc.F_IMAGE), [st[c]], np.array([f.r_plus - y]),
                               np.array([0.0]), np.array([xi * tab[c, 4]]), np.array([0], np.int32), zeta, p)
            h = 1e-4 * y
            dphi = (-ce * xi * xi / (y + h) - (-ce * xi * xi / (y - h))) / (2 * h)
            # HF: +x acceleration toward the wall at (R - y, 0); LF: force -dPhi/dy along -y
            assert abs(a[0, 0] / dphi - 1) < 1e-7
        cut = 1e-12 / ell
        for gap in [3e-9, 3e-8, 0.1 * dp]:
            y = 0.5 * dplus + gap / ell
            a = orc.wall_accel(f, orc.cfg(0.1, forces=orc.F_VDW), [st[c]], np.array([f.r_plus - y]),
                               np.array([0.0]), np.array([0.0]), np.array([0], np.int32), zeta, p)
            g = gap / ell
            h = 1e-6 * g
            dphi = -cv * zeta * (lf.vdw_shape(g + h, cut) - lf.vdw_shape(g - h, cut)) / (2 * h)
            assert abs(a[0, 0] / dphi - 1) < 5 * gap / dp + 1e-6


def test_vdw_shape_is_continuous_at_the_cutoff():
    cut = 1e-8
    h = 1e-4 * cut
    # force -dpsi/dg: 1/cut^2 inside the cutoff, 1/g^2 beyond it
    for g in [0.5 * h, 0.5 * cut, 0.9 * cut, 1.5 * cut, 4.0 * cut]:
        slope = -(lf.vdw_shape(g + h / 2, cut) - lf.vdw_shape(g - h / 2, cut)) / h
        assert abs(slope * max(g, cut) ** 2 - 1) < 1e-6
    assert abs(lf.vdw_shape(cut, cut) * cut - 1) < 1e-15
    assert abs(lf.vdw_shape(cut * (1 - 1e-9), cut) * cut - 1) < 1e-8


def test_brownian_diffusivity_is_stokes_einstein(orc):
    p = orc.phys()
    tab = orc.class_table([0.1, 1.0, 10.0], p)
    ustar, _, _ = lf.units(p)
    mu = p.rho_f * p.nu
    for row in tab:
        DB, th = lf.brownian(p, row, 293.15)
        se = lf.KB * 293.15 / (3 * math.pi * mu * row[2])          # Stokes-Einstein, m^2/s
        assert abs(DB * p.nu / se - 1) < 1e-12
        m = 2650.0 * math.pi / 6 * row[2] ** 3
        assert abs(th * ustar ** 2 / (lf.KB * 293.15 / m) - 1) < 1e-12


def test_nodes_span_contact_to_axis():
    y = lf.nodes(0.05, 180.0, 1000, 10.0)
    assert y[0] == 0.05 and abs(y[-1] - 180.0) < 1e-12
    assert np.all(np.diff(y) > 0) and np.diff(y)[0] < 1e-3 * np.diff(y)[-1]


def test_variance_of_an_analytic_grid():
    # u_r = A(r) cos(k z) (+ a swirl and an axial mean that carry no radial part): variance A^2/2
    n_z, n_th, n_r = 16, 12, 5
    th = 2 * np.pi * np.arange(n_th) / n_th
    z = np.arange(n_z) / n_z
    A = np.array([0.0, 0.3, 1.1, 0.7, 2.0])
    g = np.zeros((n_z, n_th, n_r, 3))
    ur = A[None, None, :] * np.cos(2 * np.pi * 3 * z)[:, None, None]
    ut = 0.9
    g[..., 0] = np.cos(th)[None, :, None] * ur - np.sin(th)[None, :, None] * ut
    g[..., 1] = np.sin(th)[None, :, None] * ur + np.cos(th)[None, :, None] * ut
    g[..., 2] = 5.0
    assert np.allclose(lf.fluid_variance(g), A ** 2 / 2, rtol=1e-13, atol=1e-15)
    # the interpolation returns the node values at the node radii
    R, beta = 180.0, 2.0
    r = R * np.tanh(beta * np.arange(n_r) / (n_r - 1)) / np.tanh(beta)
    v = lf.variance_at(A ** 2 / 2, R, beta, R - r)
    assert np.allclose(v, A ** 2 / 2, rtol=1e-12, atol=1e-14)


def test_synthetic_field_variance_vanishes_at_the_wall(field_var):
    f, var = field_var
    assert var[-1] < 1e-30 * var[0] and np.all(var[:-1] > 0) and np.all(np.diff(var) <= 0)


def test_momentum_uniform_force_reaches_the_exact_terminal_drift():
    # V V' + V/tau = S with S uniform: V relaxes from V(axis) = 0 to tau S; with the drag implicit,
    # tau S is an exact fixed point of the march, so it is reached to rounding in the stiff case
    S, yc, tau = -0.02, 20.0, 0.5
    y = lf.nodes(0.1, yc, 300, 3.0)
    V = lf.momentum(y, np.zeros(300), -S * y, tau)
    far = y < 0.5 * yc
    assert np.max(np.abs(V[far] / (tau * S) - 1)) < 1e-13
    # forces through w or through phi are the same potential
    assert np.array_equal(V, lf.momentum(y, -S * y, np.zeros(300), tau))


@pytest.mark.parametrize("tau", [0.5, 5.0])
def test_momentum_march_converges_to_the_ode_solution(tau):
    # S(y) = -S1 (yc - y): smooth solution V = -alpha x near the axis (x = yc - y) with
    # alpha^2 + alpha/tau - S1 = 0; scipy's Radau integrates V dV/dx = -(S - V/tau) from there
    S1, yc = 0.004, 20.0
    alpha = 0.5 * (-1 / tau + math.sqrt(1 / tau ** 2 + 4 * S1))
    x0 = 1e-7
    sol = integrate.solve_ivp(lambda x, v: [-(-S1 * x - v[0] / tau) / v[0]], (x0, yc - 0.1), [-alpha * x0],
                              method="Radau", rtol=1e-12, atol=1e-15, dense_output=True)
    errs = []
    for n in (400, 800):
        y = lf.nodes(0.1, yc, n, 3.0)
        phi = S1 * (yc * y - 0.5 * y * y)            # -dphi/dy = -S1 (yc - y)
        V = lf.momentum(y, np.zeros(n), phi, tau)
        ref = np.array([sol.sol(yc - yy)[0] if yc - yy > x0 else 0.0 for yy in y])
        errs.append(np.max(np.abs(V - ref)) / np.max(np.abs(ref)))
    assert errs[0] < 2e-2
    assert 1.6 < errs[0] / errs[1] < 2.4          # first order: the drag is fully implicit


def test_momentum_no_outward_drift():
    y = lf.nodes(0.1, 10.0, 50, 2.0)
    V = lf.momentum(y, np.zeros(50), 0.01 * (10.0 - y), 1.0)    # -dphi/dy = +0.01: away from the wall
    assert np.all(V == 0.0)


def test_continuity_closed_forms():
    y = lf.nodes(0.2, 50.0, 300, 6.0)
    L = y[-1] - y[0]
    # V = 0, D constant: resistances in series 1/V_dep = 1/|K| + L/D
    K, D = -0.03, 0.7
    v = lf.continuity(y, np.zeros(300), np.full(300, D), K)
    assert abs(v / (1 / (1 / abs(K) + L / D)) - 1) < 1e-12
    # constant V < 0, D constant: rho = J/V + (rho_w - J/V) e^{V (y - y_w)/D}, J = K rho_w, rho_c = 1
    V0 = -0.05
    e = math.exp(V0 * L / D)
    ref = -K / (e + K / V0 * (1 - e))
    v = lf.continuity(y, np.full(300, V0), np.full(300, D), K)
    assert abs(v / ref - 1) < 1e-12
    # V = 0, D = D0 + D1 y^2: 1/V_dep = 1/|K| + int dy/D, second order in the cell means
    D0, D1 = 0.01, 0.2
    I = (math.atan(y[-1] * math.sqrt(D1 / D0)) - math.atan(y[0] * math.sqrt(D1 / D0))) / math.sqrt(D0 * D1)
    errs = []
    for n in (400, 800):
        yy = lf.nodes(0.2, 50.0, n, 6.0)
        v = lf.continuity(yy, np.zeros(n), D0 + D1 * yy ** 2, K)
        errs.append(abs(v * (1 / abs(K) + I) - 1))
    assert errs[0] < 1e-3 and 3.0 < errs[0] / errs[1] < 5.0


def test_continuity_against_an_ode_solver():
    yw, yc, K = 0.1, 30.0, -0.02
    Vf = lambda y: -0.4 * (1 - y / yc) ** 2
    Df = lambda y: 1e-3 + 0.05 * y * y / (1 + 0.01 * y * y)
    sol = integrate.solve_ivp(lambda y, r: [(r[0] * Vf(y) - K) / Df(y)], (yw, yc), [1.0], method="Radau",
                              rtol=1e-12, atol=1e-14)
    ref = -K / sol.y[0, -1]
    errs = []
    for n in (1000, 2000):
        y = lf.nodes(yw, yc, n, 6.0)
        errs.append(abs(lf.continuity(y, Vf(y), Df(y), K) / ref - 1))
    assert errs[0] < 1e-4 and 3.0 < errs[0] / errs[1] < 5.0


def test_brownian_limit_of_the_model(orc):
    # no turbulence (v_f'^2 = 0), no charge, no vdW: V = 0, D = D_B, sigma^2 = k_B T/m, so
    # 1/V_dep = sqrt(2 pi)/sigma + (R - d/2)/D_B
    p = orc.phys()
    st = [0.1, 1.0, 10.0]
    tab = orc.class_table(st, p)
    v = lf.lf_vdep(p, st, np.array([[0.0, 0.0, 0.5]]), np.zeros(64), 180.0, 2.0, lf.lf_params(n_y=200))
    for c in range(3):
        DB, th = lf.brownian(p, tab[c], 293.15)
        ref = 1 / (math.sqrt(2 * math.pi / th) + (180.0 - 0.5 * tab[c, 1]) / DB)
        assert abs(v[0, c] / ref - 1) < 1e-12


def test_model_trends(orc, field_var):
    # Sec. 2.3 / Fig. 5: V_dep+ grows with the charge (xi) and the Hamaker constant (zeta); the
    # electrostatic effect exceeds the vdW one over the ranges, and the vdW effect fades with size.
    # theta does not enter the model (STICK, isothermal gas).
    f, var = field_var
    p = orc.phys()
    st = [0.1, 1.0, 10.0]
    xs = np.linspace(0, 0.1, 5)
    zs = np.linspace(0, 1, 5)
    prm = np.array([[x, 0.5, 0.5] for x in xs] + [[0.05, z, 0.5] for z in zs] + [[0.05, 0.5, 0.1],
                                                                                [0.05, 0.5, 0.9]])
    v = lf.lf_vdep(p, st, prm, var, f.r_plus, f.beta, lf.lf_params(n_y=512))
    vx, vz = v[:5], v[5:10]
    assert np.all(np.diff(vx, axis=0) > 0) and np.all(np.diff(vz, axis=0) >= 0)
    ex = vx[-1] / vx[0] - 1
    ez = vz[-1] / vz[0] - 1
    assert np.all(ex > ez) and ez[0] > ez[1] > ez[2]
    assert np.array_equal(v[10], v[11])


def test_grid_convergence(orc, field_var):
    # first order in the node spacing (the implicit drag); about 1 % at the default 2,048 nodes
    f, var = field_var
    p = orc.phys()
    st = [0.1, 1.0, 10.0]
    prm = np.array([[0.05, 0.5, 0.5], [0.1, 1.0, 0.5]])
    v = {n: lf.lf_vdep(p, st, prm, var, f.r_plus, f.beta, lf.lf_params(n_y=n)) for n in (1024, 2048, 8192)}
    assert np.max(np.abs(v[2048] / v[8192] - 1)) < 0.015
    r = (v[1024] - v[8192]) / (v[2048] - v[8192])
    assert np.all((r > 1.8) & (r < 2.7))
