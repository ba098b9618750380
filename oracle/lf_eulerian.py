"""FP64 oracle of the 1-D Eulerian low-fidelity deposition model (App. B) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this module.  It shares no code with the CUDA library
and imports nothing from it.  Plain numpy in FP64: a Python loop over the
wall-normal nodes, vectorised over the (sample, class) items.

The model (App. B, Eqs. momentum/mom_modified, continuity and the kinetic wall
condition) in wall units, y = wall distance of the particle centre, V = mean
wall-normal particle velocity (negative toward the wall), rho = particle density
over its centreline value:

  V dV/dy + V/tau_1 = -d/dy(R_ratio v_f'^2) + F_elec+ + F_vdw+            (momentum)
  J = -(D_B + eps) drho/dy - rho D_T dlnT/dy + rho V = const,  V_dep+ = -J  (continuity)
  -(D_B + eps) drho/dy = rho_w V_w (exp(-M^2)/(2 sqrt(pi) M) - (1 - erf M)/2) (wall, y = d/2)

App. B cites its closures (R_ratio, v_f'^2, D_B, D_T, eps, M_r) to other papers
and prints none of them; the readings this module takes, each one a line of the
design notes (readings c33-c41):

  v_f'^2(y)  the (theta, z) variance of the radial velocity of the synthetic
             carrier field at radius R - y (the high-fidelity model's own flow),
             linear in the field's stretched radial coordinate s between nodes;
  R_ratio    T_L / (T_L + tau_p): stationary response of a first-order particle
             to a fluid velocity with exponential autocorrelation of time T_L;
  eps        v_f'^2 T_L: Taylor's long-time diffusivity of that velocity;
  tau_1      tau_p+ (Stokes relaxation, as the paper defines tau_p+);
  D_B        Einstein: k_B T tau_p / m_p (Stokes-Einstein with the same tau_p);
  D_T        0 (isothermal gas: dlnT/dy = 0);
  M_r        u / (sqrt 2 sigma), u = -V_w, sigma^2 = R_ratio v_f'^2 + k_B T/m_p at
             the wall: the kinetic condition is then exactly the one-way flux of a
             Gaussian wall-normal velocity (mean V_w, variance sigma^2) into an
             absorbing wall;
  F_elec+, F_vdw+  the printed forms per unit mass, q = xi q_max, A = zeta A0,
             the vdW gap cut at vdw_cutoff (1e-12 m, App. B).

Pins (tests/test_oracle_lf.py): every closure, the wall condition, the force
potentials and both marches against independent references (Lyapunov
covariances, quadrature, the high-fidelity oracle's wall forces, exact ODE
solutions, scipy's solvers), the Brownian closed form and the Fig. 5 trends.
The model's V_dep+ values against the paper's Fig. 5: parity unpinned, because
the closures are readings, not the cited papers' fits.

Discretisation (App. B: refined near the wall, drag implicit):
  nodes y_k = y_w + (R - y_w) expm1(gamma s_k)/expm1(gamma), s_k = k/(n-1),
  y_w = d+/2 (contact), y_{n-1} = R+ (axis), V_{n-1} = 0;
  momentum in energy form d/dy(V^2/2 + w + Phi) = -V/tau_1 (w = R_ratio v_f'^2,
  Phi the force potentials), the drag fully implicit (taken at the new node, so
  the march stays stable where a cell is longer than the relaxation length),
  marched from the axis to the wall: V_k^2/2 - a V_k = c with a = dy/tau_1,
  c = V_{k+1}^2/2 + dw + dPhi; V_k is the root <= 0, and 0 where c < 0 (no
  outward mean drift);
  continuity with the flux J constant: exact solution of J = -D rho' + V rho
  over each cell with V, D at their cell means (exponential fitting), marched
  from the wall (rho_w = 1, J = rho_w K from the wall condition) and rescaled so
  that rho = 1 on the axis.
"""
import math

import numpy as np
from scipy.special import erf

KB = 1.380649e-23          # Boltzmann constant, J/K (SI exact)


def lf_params(n_y=2048, stretch=8.0, t_lagr=10.0, temperature=293.15, vdw_cutoff=1e-12):
    """Parameters of the low-fidelity model (readings c33-c41): nodes, wall stretching gamma,
    T_L+ (wall units), gas temperature (K), vdW gap cutoff (m, App. B)."""
    return dict(n_y=int(n_y), stretch=float(stretch), t_lagr=float(t_lagr), temperature=float(temperature),
                vdw_cutoff=float(vdw_cutoff))


def units(p):
    """u* (m/s), wall unit (m) and the factor from SI acceleration to wall units."""
    ustar = p.re_tau * p.nu / p.radius
    return ustar, p.nu / ustar, p.nu / ustar ** 3


# ---------------------------------------------------------------------------
# Fluid wall-normal variance from the synthetic field
# ---------------------------------------------------------------------------
def fluid_variance(grid):
    """Population variance over (theta, z) of u_r = cos(theta) u_x + sin(theta) u_y at each radial
    node; grid [n_z][n_th][n_r][3] Cartesian velocity at theta_j = 2 pi j / n_th.  The v_f'^2 of
    Eq. momentum (App. B), reading c33."""
    n_th = grid.shape[1]
    th = 2.0 * np.pi * np.arange(n_th) / n_th
    ur = np.cos(th)[None, :, None] * grid[..., 0] + np.sin(th)[None, :, None] * grid[..., 1]
    mean = ur.mean(axis=(0, 1))
    return ((ur - mean) ** 2).mean(axis=(0, 1))


def variance_at(var_r, r_plus, beta, y):
    """v_f'^2 at wall distance y: linear in s = atanh(r tanh(beta)/R)/beta between the field's
    radial nodes r_i = R tanh(beta i/(n_r-1))/tanh(beta)."""
    n_r = len(var_r)
    r = r_plus - np.asarray(y, np.float64)
    s = np.arctanh(r * math.tanh(beta) / r_plus) / beta
    t = s * (n_r - 1)
    i = np.minimum(np.floor(t).astype(np.int64), n_r - 2)
    i = np.maximum(i, 0)
    f = t - i
    return (1.0 - f) * var_r[i] + f * var_r[i + 1]


# ---------------------------------------------------------------------------
# Closures and force potentials (App. B; readings c33-c41)
# ---------------------------------------------------------------------------
def response_ratio(tau_p, t_lagr):
    """R_ratio of Eq. momentum (App. B) = <v_p'^2>/<v_f'^2> = T_L/(T_L + tau_p) (reading c34)."""
    return t_lagr / (t_lagr + tau_p)


def eddy_diffusivity(var_f, t_lagr):
    """eps/nu of Eq. continuity (App. B) = v_f'^2 T_L, wall units (reading c35)."""
    return var_f * t_lagr


def brownian(p, cls_row, temperature):
    """(D_B/nu, k_B T/(m u*^2)): D_B of Eq. continuity (App. B) by Einstein, k_B T tau_p/m_p (reading
    c37), and the thermal velocity variance of the wall condition (reading c39)."""
    ustar, ell, _ = units(p)
    tau_p = cls_row[0] * p.nu / ustar ** 2          # s
    m = cls_row[3]
    return KB * temperature * tau_p / m / p.nu, KB * temperature / m / ustar ** 2


def potential_constants(p, cls_row):
    """(C_e, C_v): Phi_elec+ = -C_e xi^2 / y+ and Phi_vdw+ = -C_v zeta psi(gap+), from
    F_elec = -3 q^2/(8 pi^2 eps0 rho_p d^3 y^2) with q = xi q_max and
    F_vdw = -A d/(12 m (y - d/2)^2) with A = zeta A0, per unit mass, in wall units."""
    ustar, ell, acc = units(p)
    d, m, qfac = cls_row[2], cls_row[3], cls_row[4]
    q1 = p.qmax_coef * qfac                             # q_max of the class, C
    ce = 3.0 * q1 * q1 / (8.0 * np.pi ** 2 * p.eps0 * p.rho_p * d ** 3) * acc / ell ** 2
    cv = p.hamaker0 * d / (12.0 * m) * acc / ell ** 2
    return ce, cv


def vdw_shape(gap, cut):
    """psi with -dpsi/dgap = 1/max(gap, cut)^2 and psi = 1/gap beyond the cutoff (linear inside):
    the shape of F_vdw's potential with App. B's gap cutoff (reading c41)."""
    gap = np.asarray(gap, np.float64)
    return np.where(gap >= cut, 1.0 / np.maximum(gap, cut), 2.0 / cut - gap / (cut * cut))


def wall_flux_factor(v_w, sigma):
    """K = J/rho_w from the kinetic wall condition: the net wall-normal flux per unit wall density
    of a Gaussian velocity with mean v_w (<= 0 toward the wall) and standard deviation sigma into
    an absorbing wall, -(u (1 + erf M)/2 + sigma exp(-M^2)/sqrt(2 pi)) with u = -v_w and
    M = u/(sqrt(2) sigma); equals v_w + v_w (exp(-M^2)/(2 sqrt(pi) M) - (1 - erf M)/2)."""
    u = -np.asarray(v_w, np.float64)
    sigma = np.asarray(sigma, np.float64)
    M = u / (np.sqrt(2.0) * sigma)
    return -(0.5 * u * (1.0 + erf(M)) + sigma * np.exp(-M * M) / np.sqrt(2.0 * np.pi))


def nodes(y_w, r_plus, n_y, stretch):
    """Wall-normal nodes refined near the wall (App. B; reading c40), contact y_w to the axis."""
    s = np.arange(n_y) / (n_y - 1)
    return y_w + (r_plus - y_w) * np.expm1(stretch * s) / np.expm1(stretch)


# ---------------------------------------------------------------------------
# The two marches on given node tables
# ---------------------------------------------------------------------------
def momentum(y, w, phi, tau):
    """V at the nodes: Eq. mom_modified (App. B) in energy form with the force potentials phi and
    the drag implicit (reading c40), marched from the axis: y [n], w and phi [..., n] (broadcast
    over items), tau scalar or [...]."""
    n = y.shape[-1]
    shape = np.broadcast(w[..., 0], phi[..., 0], np.asarray(tau)).shape
    V = np.zeros(shape + (n,))
    for k in range(n - 2, -1, -1):
        dy = y[..., k + 1] - y[..., k]
        a = dy / tau
        vn = V[..., k + 1]
        c = 0.5 * vn * vn + (w[..., k + 1] - w[..., k]) + (phi[..., k + 1] - phi[..., k])
        root = -2.0 * c / (a + np.sqrt(a * a + 2.0 * np.maximum(c, 0.0)))
        V[..., k] = np.where(c > 0.0, root, 0.0)
    return V


def continuity(y, V, D, K):
    """V_dep+ = -J for the flux J = -D rho' + V rho of Eq. continuity (App. B, D_T term zero), J =
    rho_w K at the wall (the kinetic condition), rho = 1 on the axis: cell-wise exact solution with
    V, D at their cell means, marched from rho_w = 1 outward (reading c40)."""
    n = V.shape[-1]
    rho = np.ones(V.shape[:-1])
    J = K * rho
    for k in range(n - 1):
        dy = y[..., k + 1] - y[..., k]
        vm = 0.5 * (V[..., k] + V[..., k + 1])
        h = dy / (0.5 * (D[..., k] + D[..., k + 1]))
        a = vm * h
        safe = np.where(a != 0.0, a, 1.0)
        G = np.where(a != 0.0, h * np.expm1(a) / safe, h)
        rho = np.exp(a) * rho - J * G
    return -J / rho


# ---------------------------------------------------------------------------
# The model
# ---------------------------------------------------------------------------
def lf_vdep(p, st_plus, params, var_r, r_plus, beta, lf=None, cls=None):
    """V_dep+ [S, C] of the low-fidelity model for params [S, 3] = (xi, zeta, theta) per sample
    and classes st_plus [C]; var_r [n_r] the field's radial-velocity variance at its radial nodes.
    cls: the class table rows [tau+, d+, d, m, (d/1um)^2] (oracle.class_table)."""
    lf = lf or lf_params()
    params = np.asarray(params, np.float64).reshape(-1, 3)
    if cls is None:
        from . import class_table
        cls = class_table(st_plus, p)
    S, C = len(params), len(st_plus)
    out = np.zeros((S, C))
    _, ell, _ = units(p)
    cut = lf["vdw_cutoff"] / ell
    TL = lf["t_lagr"]
    for c in range(C):
        tau, dp = cls[c, 0], cls[c, 1]
        y = nodes(0.5 * dp, r_plus, lf["n_y"], lf["stretch"])
        var = variance_at(var_r, r_plus, beta, y)
        Rr = response_ratio(tau, TL)
        w = Rr * var
        DB, thermal = brownian(p, cls[c], lf["temperature"])
        D = DB + eddy_diffusivity(var, TL)
        ce, cv = potential_constants(p, cls[c])
        xi, zeta = params[:, 0:1], params[:, 1:2]
        phi = -ce * xi * xi / y[None, :] - cv * zeta * vdw_shape(y - 0.5 * dp, cut)[None, :]
        V = momentum(y, w[None, :], phi, tau)
        K = wall_flux_factor(V[:, 0], np.sqrt(Rr * var[0] + thermal))
        out[:, c] = continuity(y, V, D[None, :], K)
    return out
