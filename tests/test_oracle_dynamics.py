"""Pins of the oracle's time integration, wall contact, tallies and derivatives.

References: an independent high-order ODE solver (scipy) for the drag law, the
scalar root of the Schiller-Naumann settling balance, closed-form ballistic
trajectories for deposition counts, energy conservation of two charges, the SI
definition of V_dep+ (Sec. 2.1), and finite differences for the dual numbers.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

USTAR, NU, R_SI = 0.27, 1.5e-5, 0.01
ELL = NU / USTAR
G_PLUS = 9.81 * NU / USTAR ** 3


def _grid(f, u=(0.0, 0.0, 0.0)):
    g = np.zeros((f.n_z, f.n_th, f.n_r, 3))
    g[...] = u
    return g


def _one(orc, f, st_plus, pos, vel=(0, 0, 0), q=0.0, cls=0):
    st = orc.State(1)
    st.x[0], st.y[0], st.z[0] = pos
    st.vx[0], st.vy[0], st.vz[0] = vel
    st.q[0], st.cls[0] = q, cls
    return st, np.array([0, 1], np.int64)


@pytest.mark.parametrize("st_plus", [0.1, 1.0, 10.0])
def test_drag_relaxation_matches_ode_solution(orc, st_plus):
    # uniform axial flow U: w = U - v obeys dw/dt = -(1 + 0.15 (w d+)^0.687) w / tau+ (Eq. part_source)
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    U = 15.0
    g = _grid(f, (0.0, 0.0, U))
    tau, dplus = orc.class_table([st_plus])[0, :2]
    T = 2.0 * st_plus
    sol = solve_ivp(lambda t, y: [-(1 + 0.15 * (y[0] * dplus) ** 0.687) * y[0] / tau, U - y[0]],
                    (0, T), [U, 0.0], method="DOP853", rtol=1e-13, atol=1e-13)
    w_ref, z_ref = sol.y[0, -1], sol.y[1, -1]
    errs = []
    for n in (40, 80, 160):
        st, off = _one(orc, f, [st_plus], (10.0, 0.0, 5.0))
        c = orc.cfg(T / n, forces=orc.F_DRAG)
        orc.run(f, g, c, [st_plus], off, np.array([[0, 0, 0.0]]), st, n)
        errs.append(abs((U - st.vz[0]) - w_ref) / U)
        dz = (st.z[0] - 5.0) % f.l_plus
        assert abs(dz - z_ref) < 50 * errs[-1] * U * T + 1e-9
        assert st.x[0] == 10.0 and st.vx[0] == 0.0
    # first order in dt (drag factor frozen over the step), and small
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4
    assert errs[2] < 2e-3


@pytest.mark.parametrize("st_plus", [1.0, 10.0, 100.0])
def test_stokes_settling_terminal_velocity(orc, st_plus):
    # quiescent fluid, gravity + drag: v (1 + 0.15 (v d+)^0.687) = g+ tau+
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    tau, dplus = orc.class_table([st_plus])[0, :2]
    vt = brentq(lambda v: v * (1 + 0.15 * (v * dplus) ** 0.687) - G_PLUS * tau, 0, 10)
    st, off = _one(orc, f, [st_plus], (0.0, 0.0, 1.0))
    dt = 0.05 * tau
    c = orc.cfg(dt, forces=orc.F_DRAG | orc.F_GRAV, gravity=(0, 0, 1))
    orc.run(f, _grid(f), c, [st_plus], off, np.array([[0, 0, 0.0]]), st, int(40 * tau / dt))
    assert st.vz[0] == pytest.approx(vt, rel=1e-9)


def test_free_fall_exact_and_ballistic_deposition(orc):
    # gravity only (drag off): x = x0 + g t^2 / 2 exactly; particles deposit at the first
    # step end with gap <= 0; tallies count steps from window_start on.
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    st_plus = [1.0, 10.0]
    t = orc.class_table(st_plus)
    rng = np.random.default_rng(8)
    n = 400
    st = orc.State(n)
    r = 170 * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    st.x, st.y, st.z = r * np.cos(th), r * np.sin(th), rng.uniform(0, f.l_plus, n)
    st.cls = (np.arange(n) % 2).astype(np.int32)
    st.q[:] = 1.0
    off = np.array([0, n], np.int64)
    dt, n_steps, w0 = 2.0, 120, 30
    c = orc.cfg(dt, forces=orc.F_GRAV, gravity=(1, 0, 0), window_start=w0)
    x0, y0 = st.x.copy(), st.y.copy()
    ndep, nal = orc.run(f, _grid(f), c, st_plus, off, np.array([[0.1, 0.5, 0.5]]), st, n_steps)
    # closed form: first step index k with |(x0 + g t_{k+1}^2/2, y0)| >= R - d/2
    tk = dt * np.arange(1, n_steps + 1)
    xs = x0[:, None] + 0.5 * G_PLUS * tk[None, :] ** 2
    gap = f.r_plus - np.hypot(xs, y0[:, None]) - 0.5 * t[st.cls, 1][:, None]
    assert np.min(np.abs(gap)) > 1e-9               # no ties in this draw
    hit = gap <= 0
    first = np.where(hit.any(1), hit.argmax(1), n_steps)
    for c_ in range(2):
        m = st.cls == c_
        assert ndep[0, c_] == np.sum((first[m] >= w0) & (first[m] < n_steps))
        alive_steps = sum(np.sum(first[m] >= k) for k in range(w0, n_steps))
        assert nal[0, c_] == alive_steps
    dead = first < n_steps
    assert np.array_equal(st.alive == 0, dead)
    live = ~dead
    assert np.allclose(st.x[live], x0[live] + 0.5 * G_PLUS * (dt * n_steps) ** 2, rtol=1e-12)
    assert np.allclose(st.vx[live], G_PLUS * dt * n_steps, rtol=1e-12)


def test_vdep_matches_si_definition(orc):
    # V_dep+ = J_w / (rho_pm u*) with J_w = (dN/dt) m_p / (2 pi R L) and rho_pm = N m_p / (pi R^2 L)
    ndep = np.array([[37, 5]], np.int64)
    nal = np.array([[91234, 17000]], np.int64)
    dt_plus = 0.05
    v = orc.vdep(ndep, nal, dt_plus)
    tauf = NU / USTAR ** 2
    m_p, L = 1e-12, 0.04
    for k in range(2):
        T = nal[0, k] * dt_plus * tauf             # time-integral of N (s) -> mean N over the window
        Jw = ndep[0, k] * m_p / (2 * np.pi * R_SI * L)   # mass per area
        rho_pm_T = m_p / (np.pi * R_SI ** 2 * L) * T      # density x time
        assert v[0, k] == pytest.approx(Jw / rho_pm_T / USTAR, rel=1e-12)


def test_two_charge_energy_conservation(orc):
    # drag and gravity off: E = (v1^2 + v2^2)/2 + kappa q1 q2 / r is conserved (equal masses);
    # the integrator is first order, so the drift halves with dt.
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    st_plus = [10.0]
    m = orc.class_table(st_plus)[0, 3]
    kappa = (8e-17) ** 2 / (4 * np.pi * 8.854e-12) / m / ELL ** 2 * (NU / USTAR ** 3)
    q = 50.0
    drifts = []
    for n in (100, 200, 400):
        st = orc.State(2)
        st.x[:] = [0.0, 0.0]
        st.y[:] = [-1.0, 1.0]
        st.z[:] = [360.0, 360.3]
        st.q[:] = q
        st.cls[:] = 0
        off = np.array([0, 2], np.int64)

        def energy():
            d = np.array([st.x[0] - st.x[1], st.y[0] - st.y[1], st.z[0] - st.z[1]])
            v2 = st.vx ** 2 + st.vy ** 2 + st.vz ** 2
            return 0.5 * v2.sum() + kappa * q * q / np.linalg.norm(d)

        E0 = energy()
        c = orc.cfg(60.0 / n, forces=orc.F_COUL)
        orc.run(f, _grid(f), c, st_plus, off, np.array([[0.1, 0.5, 0.5]]), st, n)
        assert np.hypot(st.y[1] - st.y[0], st.z[1] - st.z[0]) > 4.0   # they repelled substantially
        drifts.append(abs(energy() - E0) / E0)
    assert drifts[2] < 5e-3 and 1.6 < drifts[0] / drifts[1] < 2.4 and 1.6 < drifts[1] / drifts[2] < 2.4
    # momentum (equal masses) is conserved exactly up to rounding
    assert abs(st.vy.sum()) < 1e-12 and abs(st.vz.sum()) < 1e-12


def test_zero_charge_zero_hamaker_invariance(orc):
    # xi = zeta = 0: Coulomb, image and vdW vanish, so the run equals drag + gravity only
    f = orc.field_desc(n_r=17, n_th=16, n_z=16)
    g = orc.field_grid(f, orc.field_modes(f, 0))
    st_plus = [0.1, 10.0]
    prm = np.array([[0.0, 0.0, 0.5]])
    a, off = orc.seed(f, st_plus, [300], prm, 4)
    b = a.copy()
    t1 = orc.run(f, g, orc.cfg(0.1), st_plus, off, prm, a, 60)
    t2 = orc.run(f, g, orc.cfg(0.1, forces=orc.F_DRAG | orc.F_GRAV), st_plus, off, prm, b, 60)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.vz, b.vz) and np.array_equal(a.alive, b.alive)
    assert np.array_equal(t1[0], t2[0])


def test_rebound_mode_reflects_and_sticks(orc):
    # a particle driven into the wall: theta = 0, zeta = 0 rebounds elastically; zeta = 1 at
    # theta = 0.5 sticks (110.3 zeta > 215.6 (1 - theta)^2 m^2/s^2 for d = 5 um)
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    st_plus = [1.0]
    dplus = orc.class_table(st_plus)[0, 1]
    for zeta, theta, stick in [(0.0, 0.0, False), (1.0, 0.5, True)]:
        st, off = _one(orc, f, st_plus, (f.r_plus - 0.5 * dplus - 0.05, 0.0, 1.0), vel=(1.0, 0.0, 0.0))
        c = orc.cfg(0.1, forces=0, mode=orc.REBOUND)
        ndep, _ = orc.run(f, _grid(f), c, st_plus, off, np.array([[0.0, zeta, theta]]), st, 1)
        if stick:
            assert ndep[0, 0] == 1 and st.alive[0] == 0
        else:
            # free flight overshoots by 0.05 wall units; mirrored back, velocity reversed (CoR = 1)
            assert ndep[0, 0] == 0 and st.alive[0] == 1
            assert st.vx[0] == pytest.approx(-1.0) and st.x[0] == pytest.approx(f.r_plus - 0.5 * dplus - 0.05)


@pytest.fixture(scope="module")
def smooth_case(orc):
    f = orc.field_desc(n_r=33, n_th=16, n_z=32)
    g = orc.field_grid(f, orc.field_modes(f, 0))
    st_plus = [0.1, 1.0]
    n = 48
    rng = np.random.default_rng(9)
    r = f.r_plus - rng.uniform(0.05, 3.0, n)
    th = 2 * np.pi * rng.random(n)
    x0, y0, z0 = r * np.cos(th), r * np.sin(th), rng.uniform(0, f.l_plus, n)
    cls = (np.arange(n) % 2).astype(np.int32)
    qhat = orc.class_table(st_plus)[cls, 4] * 40.0          # strong charge so xi matters
    off = np.array([0, n], np.int64)
    return f, g, st_plus, off, x0, y0, z0, qhat, cls


def test_dual_numbers_match_finite_differences(orc, smooth_case):
    f, g, st_plus, off, x0, y0, z0, qhat, cls = smooth_case
    c = orc.cfg(0.05, forces=orc.F_ALL, gravity=(0, 0, 1), smooth_eps=0.5, window_start=5)
    p0 = np.array([0.06, 0.7, 0.4])
    J, dJ = orc.smooth_run(f, g, c, st_plus, off, p0[None], x0, y0, z0, qhat, cls, 40)
    assert np.all(J > 0)
    for k, h in [(0, 1e-6), (1, 1e-5)]:
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        Jp, _ = orc.smooth_run(f, g, c, st_plus, off, pp[None], x0, y0, z0, qhat, cls, 40, want_grad=False)
        Jm, _ = orc.smooth_run(f, g, c, st_plus, off, pm[None], x0, y0, z0, qhat, cls, 40, want_grad=False)
        fd = (Jp - Jm) / (2 * h)
        assert np.all(np.abs(fd) > 0)
        assert np.allclose(dJ[0, :, k], fd[0], rtol=2e-4, atol=1e-9 * np.max(np.abs(J)))
    # temperature only enters the rebound model: dJ/dtheta = 0 under all-stick
    assert np.all(dJ[..., 2] == 0)
    # the smoothed functional approaches the all-stick V_dep as eps -> 0 (same sign, same order)
    st = orc.State(len(x0))
    st.x, st.y, st.z, st.q, st.cls = x0.copy(), y0.copy(), z0.copy(), p0[0] * qhat, cls.copy()
    cs = orc.cfg(0.05, forces=orc.F_ALL, gravity=(0, 0, 1), window_start=5)
    nd, na = orc.run(f, g, cs, st_plus, off, p0[None], st, 40)
    v = orc.vdep(nd, na, 0.05)
    Js, _ = orc.smooth_run(f, g, orc.cfg(0.05, forces=orc.F_ALL, gravity=(0, 0, 1), smooth_eps=1e-4,
                                         window_start=5), st_plus, off, p0[None], x0, y0, z0, qhat, cls, 40,
                           want_grad=False)
    assert np.allclose(Js, v, rtol=0.15)


def test_smoothed_rebound_dual_numbers(orc):
    # rebound mode of the smoothed functional: the weight loss carries the smoothed sticking
    # probability sigma(-arg/eps_s) of the Bons model (Sec. 4.3), so theta now matters
    f = orc.field_desc(n_r=33, n_th=16, n_z=32)
    g = orc.field_grid(f, orc.field_modes(f, 0))
    st_plus = [10.0, 100.0]
    p0 = np.array([[0.09, 0.9, 0.6], [0.06, 0.5, 0.7]])
    st, off = orc.seed(f, st_plus, [300, 129], np.c_[np.ones(2), p0[:, 1:]], 11)
    c = orc.cfg(0.1, mode=orc.REBOUND, gravity=(1, 0, 0), smooth_eps=0.05, stick_eps=10.0, window_start=5)
    J, dJ = orc.smooth_run(f, g, c, st_plus, off, p0, st.x, st.y, st.z, st.q, st.cls, 60)
    assert np.all(np.abs(dJ[:, 1, 2]) > 0)          # theta derivative of the large class
    for k in range(3):
        pp, pm = p0.copy(), p0.copy()
        pp[:, k] += 1e-6
        pm[:, k] -= 1e-6
        Jp, _ = orc.smooth_run(f, g, c, st_plus, off, pp, st.x, st.y, st.z, st.q, st.cls, 60, want_grad=False)
        Jm, _ = orc.smooth_run(f, g, c, st_plus, off, pm, st.x, st.y, st.z, st.q, st.cls, 60, want_grad=False)
        fd = (Jp - Jm) / 2e-6
        assert np.allclose(dJ[..., k], fd, rtol=1e-4, atol=1e-6 * np.max(np.abs(fd)))
