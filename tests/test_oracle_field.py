"""Pins of the oracle's RNG, units, synthetic carrier field, interpolation and seeding.

Each test checks the oracle against something other than itself: published
known-answer vectors, values printed in the paper, closed forms, or
mathematical identities evaluated numerically.
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(orc):
    kat = json.load(open(os.path.join(GOLD, "philox_kat.json")))
    for v in kat["vectors"]:
        c = np.array([int(x, 16) for x in v["ctr"]], np.uint32)
        k = np.array([int(x, 16) for x in v["key"]], np.uint32)
        assert [int(x) for x in orc.philox(c, k)] == [int(x, 16) for x in v["out"]]


def test_class_sizes_match_paper(orc):
    # Sec. 2.1: tau_p+ = 0.1, 1, 10 correspond to d_p = 1.6, 5, 16 um (rho_p = 2650,
    # Re_tau = 180, D = 20 mm, nu = 1.5e-5; rho_f = 1.2 is the reading).
    t = orc.class_table([0.1, 1.0, 10.0])
    d_um = t[:, 2] * 1e6
    assert np.allclose(d_um, [1.6, 5.0, 16.0], rtol=0.02)
    # d+ = d u*/nu with u* = Re_tau nu / R = 0.27 m/s
    assert np.allclose(t[:, 1], t[:, 2] * 0.27 / 1.5e-5, rtol=1e-12)
    # mass of a sphere
    assert np.allclose(t[:, 3], 2650 * np.pi / 6 * t[:, 2] ** 3, rtol=1e-12)


def test_mean_profile_law_of_the_wall(orc):
    yc = orc.ycross()
    assert 10.5 < yc < 11.8                      # conventional sublayer / log-law crossing
    assert orc.mean_profile(5.0) == 5.0           # viscous sublayer U+ = y+
    assert abs(orc.mean_profile(100.0) - (np.log(100.0) / 0.41 + 5.2)) < 1e-12
    # continuity at the crossing
    assert abs(orc.mean_profile(yc * (1 - 1e-9)) - orc.mean_profile(yc * (1 + 1e-9))) < 1e-6


@pytest.fixture(scope="module")
def fld(orc):
    f = orc.field_desc()
    return f, orc.field_modes(f, 0)


def test_modes_divergence_free_structure(orc, fld):
    f, m = fld
    k, b = m[:, :3], m[:, 3:6]
    # b_n is perpendicular to k_n; k_z sits on the periodic lattice 2 pi n / L
    assert np.max(np.abs(np.sum(k * b, axis=1)) / (np.linalg.norm(k, axis=1) * np.linalg.norm(b, axis=1))) < 1e-12
    nz = k[:, 2] * f.l_plus / (2 * np.pi)
    assert np.allclose(nz, np.round(nz), atol=1e-9)


def _rand_points(n, R, L, rng, rmax=0.95):
    r = R * rmax * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th), L * rng.random(n)], 1)


def test_field_is_divergence_free(orc, fld):
    f, m = fld
    rng = np.random.default_rng(1)
    P = _rand_points(50, f.r_plus, f.l_plus, rng)
    h = 1e-3
    div = np.zeros(len(P))
    gnorm = np.zeros(len(P))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        up = orc.field_velocity(f, m, P + e)
        um = orc.field_velocity(f, m, P - e)
        div += (up[:, a] - um[:, a]) / (2 * h)
        gnorm += np.sum(((up - um) / (2 * h)) ** 2, axis=1)
    assert np.max(np.abs(div) / np.sqrt(gnorm)) < 1e-6


def test_field_is_curl_of_vector_potential(orc, fld):
    # u' = curl(f(r) sum_n b_n cos(k_n.x + phi_n)), f = (1 - r^2/R^2)^2: the analytic
    # curl must match a numerical curl of the potential (mean flow removed).
    f, m = fld
    R = f.r_plus

    def potential(P):
        r2 = P[:, 0] ** 2 + P[:, 1] ** 2
        fr = (1 - r2 / R ** 2) ** 2
        arg = P @ m[:, :3].T + m[:, 6]
        return fr[:, None] * (np.cos(arg) @ m[:, 3:6])

    rng = np.random.default_rng(2)
    P = _rand_points(40, R, f.l_plus, rng)
    h = 1e-4
    J = np.zeros((len(P), 3, 3))  # J[:, i, a] = dA_i/dx_a
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        J[:, :, a] = (potential(P + e) - potential(P - e)) / (2 * h)
    curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], 1)
    u = orc.field_velocity(f, m, P)
    yp = R - np.hypot(P[:, 0], P[:, 1])
    u[:, 2] -= np.array([orc.mean_profile(y) for y in yp])
    assert np.max(np.abs(u - curl)) < 1e-6 * max(1.0, np.max(np.abs(u)))


def test_field_no_slip_and_periodic(orc, fld):
    f, m = fld
    th = np.linspace(0, 2 * np.pi, 17)
    z = np.linspace(0, f.l_plus, 17)
    P = np.stack([f.r_plus * np.cos(th), f.r_plus * np.sin(th), z], 1)
    assert np.max(np.abs(orc.field_velocity(f, m, P))) < 1e-12
    rng = np.random.default_rng(3)
    P = _rand_points(20, f.r_plus, f.l_plus, rng)
    Q = P.copy()
    Q[:, 2] += f.l_plus
    assert np.allclose(orc.field_velocity(f, m, P), orc.field_velocity(f, m, Q), atol=1e-9)


def test_field_axis_rms(orc, fld):
    # amplitude normalisation: per-component rms of u' on the axis ~ u_rms (64 random modes)
    f, m = fld
    z = np.linspace(0, f.l_plus, 4001)[:-1]
    P = np.stack([np.zeros_like(z), np.zeros_like(z), z], 1)
    u = orc.field_velocity(f, m, P)
    u[:, 2] -= orc.mean_profile(f.r_plus)
    rms = np.sqrt(np.mean(u ** 2))
    assert 0.5 * f.u_rms < rms < 1.5 * f.u_rms


def test_grid_nodes_and_interpolation(orc):
    f = orc.field_desc(n_r=17, n_th=16, n_z=16)
    m = orc.field_modes(f, 7)
    g = orc.field_grid(f, m)
    # nodes: r_i = R tanh(beta s_i)/tanh(beta), theta_j = 2 pi j / n_th, z_k = L k / n_z
    i, j, k = 5, 3, 9
    r = f.r_plus * np.tanh(f.beta * i / (f.n_r - 1)) / np.tanh(f.beta)
    th = 2 * np.pi * j / f.n_th
    P = np.array([[r * np.cos(th), r * np.sin(th), f.l_plus * k / f.n_z]])
    assert np.allclose(g[k, j, i], orc.field_velocity(f, m, P)[0], atol=1e-12)
    # interpolation reproduces node values exactly (weights 0/1)
    assert np.allclose(orc.interp(f, g, P)[0], g[k, j, i], atol=1e-9)
    # periodic wrap in z and theta
    Q = P.copy()
    Q[0, 2] += f.l_plus
    assert np.allclose(orc.interp(f, g, Q), orc.interp(f, g, P), atol=1e-9)


def test_interpolation_second_order(orc):
    # trilinear interpolation error falls ~4x when the grid spacing halves
    rng = np.random.default_rng(4)
    errs = []
    for (nr, nt, nz) in [(33, 32, 32), (65, 64, 64)]:
        f = orc.field_desc(n_r=nr, n_th=nt, n_z=nz, lam_min=80.0)
        m = orc.field_modes(f, 11)
        g = orc.field_grid(f, m)
        P = _rand_points(400, f.r_plus, f.l_plus, rng, rmax=0.8)
        errs.append(np.sqrt(np.mean((orc.interp(f, g, P) - orc.field_velocity(f, m, P)) ** 2)))
    assert errs[1] < errs[0] / 2.8


def test_seed_layout_and_statistics(orc):
    f = orc.field_desc()
    st_plus = [0.1, 1.0, 10.0]
    params = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3]])
    st, off = orc.seed(f, st_plus, [3000, 2000], params, seed_value=1)
    t = orc.class_table(st_plus)
    n = len(st.x)
    assert list(off) == [0, 3000, 5000]
    j = np.concatenate([np.arange(3000), np.arange(2000)])
    assert np.array_equal(st.id, j) and np.array_equal(st.cls, j % 3)
    s = np.repeat([0, 1], [3000, 2000])
    assert np.allclose(st.q, params[s, 0] * t[st.cls, 4], rtol=1e-14)
    r = np.hypot(st.x, st.y)
    rmax = f.r_plus - 0.5 * t[st.cls, 1]
    assert np.all(r < rmax) and np.all(st.z >= 0) and np.all(st.z < f.l_plus)
    # uniform in the cross-section: E[(r/rmax)^2] = 1/2; uniform z: E[z] = L/2
    se = np.sqrt(1 / 12 / n)
    assert abs(np.mean((r / rmax) ** 2) - 0.5) < 4 * se
    assert abs(np.mean(st.z / f.l_plus) - 0.5) < 4 * se
    # common random numbers: sample 1 repeats sample 0's first particles
    assert np.array_equal(st.x[3000:], st.x[:2000]) and np.array_equal(st.z[3000:], st.z[:2000])
    assert np.all(st.vx == 0) and np.all(st.alive == 1)


def test_seed_lognormal_charge(orc):
    f = orc.field_desc()
    st, _ = orc.seed(f, [1.0], [20000], [[0.05, 0.5, 0.5]], seed_value=3, charge_sigma=0.5)
    t = orc.class_table([1.0])
    lam = st.q / (0.05 * t[0, 4])
    ln = np.log(lam)
    assert abs(np.mean(ln)) < 4 * 0.5 / np.sqrt(len(ln))          # median 1
    assert abs(np.std(ln) - 0.5) < 0.02


def test_seed_independent_streams(orc):
    # a stream per sample: the samples no longer share particles, each is still uniform in the
    # pipe, and the draw of sample s equals the common-random-numbers draw only when s + 1 = 0
    f = orc.field_desc()
    st_plus = [0.1, 1.0, 10.0]
    params = np.array([[0.05, 0.5, 0.5], [0.1, 0.2, 0.3], [0.07, 0.4, 0.6]])
    st, off = orc.seed(f, st_plus, [4000, 4000, 4000], params, seed_value=1, independent=True)
    crn, _ = orc.seed(f, st_plus, [4000, 4000, 4000], params, seed_value=1)
    t = orc.class_table(st_plus)
    for s in range(3):
        sl = slice(off[s], off[s + 1])
        assert np.array_equal(st.id[sl], np.arange(4000)) and np.array_equal(st.cls[sl], np.arange(4000) % 3)
        r = np.hypot(st.x[sl], st.y[sl])
        rmax = f.r_plus - 0.5 * t[st.cls[sl], 1]
        se = np.sqrt(1 / 12 / 4000)
        assert np.all(r < rmax) and abs(np.mean((r / rmax) ** 2) - 0.5) < 4 * se
        assert abs(np.mean(st.z[sl] / f.l_plus) - 0.5) < 4 * se
        # independent of the shared draw and of the other samples: correlations near 0
        assert abs(np.corrcoef(st.z[sl], crn.z[sl])[0, 1]) < 4 / np.sqrt(4000)
    assert abs(np.corrcoef(st.x[off[0]:off[1]], st.x[off[1]:off[2]])[0, 1]) < 4 / np.sqrt(4000)
    assert not np.any(st.x[off[0]:off[1]] == st.x[off[1]:off[2]])
