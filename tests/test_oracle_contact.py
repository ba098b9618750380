"""Pins of the oracle's particle-particle contact forces (App. A.2 collision and
van der Waals forces) and of the signed-charge seeding.

References: the damped linear oscillator (a soft-sphere contact must last
tau_col and return e times the approach speed), conservation of momentum for
unequal masses, the Derjaguin limit F -> A R_eff / (6 g^2) of two spheres
(R_eff = R_1 R_2 / (R_1 + R_2)), the saturation and cut-off stated with
Eq. (vdw) (Sec. 2.2), and binomial bounds for the charge signs.
"""
import numpy as np
import pytest

USTAR, NU = 0.27, 1.5e-5
ELL = NU / USTAR
ACC = NU / USTAR ** 3          # SI acceleration -> wall units


def _grid(f):
    return np.zeros((f.n_z, f.n_th, f.n_r, 3))


def _pair(orc, pos, vel, cls):
    st = orc.State(2)
    for k in range(2):
        st.x[k], st.y[k], st.z[k] = pos[k]
        st.vx[k], st.vy[k], st.vz[k] = vel[k]
        st.cls[k] = cls[k]
    return st, np.array([0, 2], np.int64)


def _collide(orc, st_plus, steps_per_contact, v0=0.5, tau_col=0.1, offset=0.0, forces=None, zeta=0.0):
    """Head-on (or offset) approach of two particles on the axis; returns the per-step history."""
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    p = orc.phys()
    p.tau_col_steps = steps_per_contact
    dt = tau_col / steps_per_contact
    tab = orc.class_table(st_plus)
    d = tab[:, 1]
    contact = 0.5 * (d[0] + d[-1])
    z0 = 100.0
    gap0 = 0.2 * v0 * tau_col
    st, off = _pair(orc, [(0.0, 0.0, z0), (offset, 0.0, z0 + np.sqrt(contact ** 2 - offset ** 2) + gap0)],
                    [(0, 0, 0.5 * v0), (0, 0, -0.5 * v0)], [0, len(st_plus) - 1])
    c = orc.cfg(dt, forces=orc.F_COLLIDE if forces is None else forces)
    hist = []
    for _ in range(int(round((0.4 + 1.6) * tau_col / dt))):
        orc.run(f, _grid(f), c, list(st_plus), off, np.array([[0.0, zeta, 0.0]]), st, 1, p=p)
        r = np.sqrt((st.x[1] - st.x[0]) ** 2 + (st.y[1] - st.y[0]) ** 2 + (st.z[1] - st.z[0]) ** 2)
        hist.append((r, st.vx.copy(), st.vy.copy(), st.vz.copy()))
    return hist, contact, dt, tab


def test_head_on_collision_restitution_and_contact_time(orc):
    # K = (pi^2 + ln^2 e)/tau^2, H = -2 ln e / tau: the overlap obeys delta'' + H delta' + K delta = 0,
    # a half period of the damped oscillation lasts tau_col and ends at e times the approach speed
    v0, tau = 0.5, 0.1
    errs = []
    for n in (50, 400):
        hist, contact, dt, _ = _collide(orc, [10.0], n, v0=v0, tau_col=tau)
        vrel = hist[-1][3][1] - hist[-1][3][0]
        assert vrel > 0
        errs.append(abs(vrel / v0 - 0.9))
        t_contact = dt * sum(1 for h in hist if h[0] < contact)
        assert abs(t_contact - tau) <= 2 * dt
    assert errs[1] < 1e-4 and errs[1] < errs[0] / 4
    # the paper's resolution (tau_col = 15 dt): the mid-step contact evaluation keeps e
    hist15, _, _, _ = _collide(orc, [10.0], 15, v0=v0, tau_col=tau)
    vrel15 = hist15[-1][3][1] - hist15[-1][3][0]
    assert abs(vrel15 / v0 - 0.9) < 3e-3


def test_restitution_is_a_parameter(orc):
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    p = orc.phys()
    assert p.restitution == 0.9 and p.tau_col_steps == 15.0 and p.neg_charge_frac == 0.0
    # e = 0.5 is recovered too (the formula, not a constant, fixes the rebound)
    p.restitution, p.tau_col_steps = 0.5, 400
    st, off = _pair(orc, [(0, 0, 100.0), (0, 0, 100.0 + 0.2855 + 0.01)], [(0, 0, 0.25), (0, 0, -0.25)], [0, 0])
    c = orc.cfg(0.1 / 400, forces=orc.F_COLLIDE)
    orc.run(f, _grid(f), c, [10.0], off, np.array([[0.0, 0.0, 0.0]]), st, 1000, p=p)
    assert abs((st.vz[1] - st.vz[0]) / 0.5 - 0.5) < 5e-3


@pytest.mark.parametrize("forces", ["collide", "both"])
def test_momentum_conserved_unequal_masses(orc, forces):
    # oblique contact of a St+ = 1 and a St+ = 10 particle: the contact forces are equal and
    # opposite, so m1 v1 + m2 v2 stays put (a wrong effective-mass share breaks this)
    fl = orc.F_COLLIDE if forces == "collide" else orc.F_CONTACT
    hist, contact, dt, tab = _collide(orc, [1.0, 10.0], 60, v0=0.5, tau_col=0.1, offset=0.08, forces=fl, zeta=1.0)
    m = tab[:, 3]
    p0 = m[0] * np.array([0, 0, 0.25]) + m[1] * np.array([0, 0, -0.25])
    touched = False
    for r, vx, vy, vz in hist:
        P = m[0] * np.array([vx[0], vy[0], vz[0]]) + m[1] * np.array([vx[1], vy[1], vz[1]])
        assert np.all(np.abs(P - p0) <= 1e-12 * np.abs(p0).max())
        touched |= r < contact
    assert touched
    # the lighter particle is deflected sideways (oblique normal)
    assert abs(hist[-1][1][0]) > 1e-3


def _vdw_accel(orc, st_plus, gap_m, zeta=1.0):
    """Accelerations (wall units) of two particles at rest whose surfaces are gap_m apart."""
    f = orc.field_desc(n_r=5, n_th=4, n_z=4)
    tab = orc.class_table(st_plus)
    d = tab[:, 1]
    r = 0.5 * (d[0] + d[-1]) + gap_m / ELL
    st, off = _pair(orc, [(-0.5 * r, 0.0, 100.0), (0.5 * r, 0.0, 100.0)], [(0, 0, 0), (0, 0, 0)],
                    [0, len(st_plus) - 1])
    h = 1e-6
    orc.run(f, _grid(f), orc.cfg(h, forces=orc.F_VDWPP), list(st_plus), off, np.array([[0.0, zeta, 0.0]]), st, 1)
    return st.vx / h, tab      # v = a h exactly without drag (phi1(0) = 1)


@pytest.mark.parametrize("st_plus", [[1.0], [10.0], [1.0, 10.0]])
def test_vdw_pp_derjaguin_limit_and_third_law(orc, st_plus):
    g = 3e-9
    a, tab = _vdw_accel(orc, st_plus, g)
    m = tab[:, 3][[0, -1]]
    R1, R2 = 0.5 * tab[0, 2], 0.5 * tab[-1, 2]
    F_derj = 1e-18 * (R1 * R2 / (R1 + R2)) / (6 * g * g)
    assert a[0] > 0 and a[1] < 0                               # attraction along the line of centres
    assert abs(a[0] * m[0] / ACC / F_derj - 1) < 5e-3         # O(g/d) from the Derjaguin form
    assert abs(a[0] * m[0] + a[1] * m[1]) <= 1e-12 * abs(a[0] * m[0])


def test_vdw_pp_saturation_and_cutoff(orc):
    a_min, tab = _vdw_accel(orc, [5.0], 1e-9)
    a_in, _ = _vdw_accel(orc, [5.0], 0.3e-9)
    a_ov, _ = _vdw_accel(orc, [5.0], -2e-9)                    # overlapping surfaces
    assert a_in[0] == pytest.approx(a_min[0], rel=1e-12) and a_ov[0] == pytest.approx(a_min[0], rel=1e-12)
    d = tab[0, 2]
    a_in_cut, _ = _vdw_accel(orc, [5.0], 0.249 * d)
    a_out_cut, _ = _vdw_accel(orc, [5.0], 0.251 * d)
    assert a_in_cut[0] > 0 and a_out_cut[0] == 0.0
    # proportional to zeta (A = zeta A0)
    a_half, _ = _vdw_accel(orc, [5.0], 1e-9, zeta=0.5)
    assert a_half[0] == pytest.approx(0.5 * a_min[0], rel=1e-12)


def test_signed_charge_seeding(orc):
    f = orc.field_desc()
    counts = [4000]
    prm = np.array([[0.05, 0.5, 0.5]])
    base, _ = orc.seed(f, [0.1, 1.0, 10.0], counts, prm, 7)
    p = orc.phys()
    p.neg_charge_frac = 0.3
    bip, _ = orc.seed(f, [0.1, 1.0, 10.0], counts, prm, 7, p=p)
    assert np.array_equal(np.abs(bip.q), base.q) and np.array_equal(bip.x, base.x)
    frac = np.mean(bip.q < 0)
    assert abs(frac - 0.3) < 4 * np.sqrt(0.3 * 0.7 / 4000)
    assert np.all(base.q > 0)
