"""Multi-fidelity Monte Carlo and Sobol' estimators in plain numpy -- TEST INFRASTRUCTURE.

Oracle for the estimator half of the hot path (Sec. 3 of the paper).  Only the
test-suite and the benchmark's CPU baseline may import it.  Each function
follows one equation; no blocking, fusion or reordering beyond it.

Readings where the printed text is ambiguous:
* Precondition (Eq. mf-precond): rho_{1,k+1} is read as 0 (printed as 1,
  which makes the right-hand side's denominator negative for i = k).
* Owen's main-effect estimator (Eq. owen): z_i^(j) takes coordinate j from
  x_i and the others from x'_i; E-hat and V-hat come from f(x), E-hat' and
  V-hat' from f(x'); sample variances use the divisor m - 1.
* Var(Y) in the Sobol' ratios: the MFMC variance estimator with the same
  alpha and nested samples, applied to f(x).
* Sample nesting (Eq. MFMC_mean): model i uses the first m_i samples, and its
  m_{i-1} estimator the first m_{i-1} of those.
"""
import numpy as np


def mc_mean(y):
    """Plain MC estimator: mean of m i.i.d. evaluations (Sec. 3.1)."""
    y = np.asarray(y, np.float64)
    return y.sum(axis=0) / y.shape[0]


def mfmc_allocation(rho, sigma, w, p):
    """Optimal alpha_i, r_i, m_i of Eqs. (opt1)-(opt3) for k models sorted by fidelity.

    rho[0] = 1 (the high-fidelity model); rho_{1,k+1} read as 0.
    Returns alpha [k] (alpha[0] = 1), r [k] (r[0] = 1), m_star [k] (real) and m1
    floored to an integer count as Table 3 tabulates it.
    """
    rho = np.asarray(rho, np.float64)
    sigma = np.asarray(sigma, np.float64)
    w = np.asarray(w, np.float64)
    k = len(rho)
    rho_ext = np.append(rho, 0.0)
    alpha = np.ones(k)
    r = np.ones(k)
    for i in range(1, k):
        alpha[i] = rho[i] * sigma[0] / sigma[i]
    for i in range(k):
        r[i] = np.sqrt(w[0] * (rho_ext[i] ** 2 - rho_ext[i + 1] ** 2) / (w[i] * (1.0 - rho_ext[1] ** 2)))
    m1 = p / np.dot(w, r)
    m_star = m1 * r
    return alpha, r, m_star


def mfmc_precondition(rho, w):
    """Eq. (mf-precond): w_{i-1}/w_i > (rho_{i-1}^2 - rho_i^2)/(rho_i^2 - rho_{i+1}^2), i = 2..k."""
    rho_ext = np.append(np.asarray(rho, np.float64), 0.0)
    w = np.asarray(w, np.float64)
    ok = True
    for i in range(1, len(w)):
        lhs = w[i - 1] / w[i]
        rhs = (rho_ext[i - 1] ** 2 - rho_ext[i] ** 2) / (rho_ext[i] ** 2 - rho_ext[i + 1] ** 2)
        ok = ok and lhs > rhs
    return ok


def gamma_two_model(rho12, w_ratio):
    """Variance-reduction ratio of the two-model MFMC estimator (Sec. 4.1)."""
    return (np.sqrt(1.0 - rho12 ** 2) + rho12 * np.sqrt(w_ratio)) ** 2


def mfmc_mean(ys, m, alpha):
    """Eq. (MFMC_mean): ys[i] holds >= m[i] evaluations of model i on the shared sample sequence."""
    S = mc_mean(np.asarray(ys[0])[: m[0]])
    for i in range(1, len(ys)):
        yi = np.asarray(ys[i])
        S = S + alpha[i] * (mc_mean(yi[: m[i]]) - mc_mean(yi[: m[i - 1]]))
    return S


def _var(y):
    y = np.asarray(y, np.float64)
    mu = y.sum(axis=0) / y.shape[0]
    return ((y - mu) ** 2).sum(axis=0) / (y.shape[0] - 1)


def mfmc_variance(ys, m, alpha):
    """Variance of Y by the control-variate form of Eq. (MFMC_mean) applied to sample variances."""
    V = _var(np.asarray(ys[0])[: m[0]])
    for i in range(1, len(ys)):
        yi = np.asarray(ys[i])
        V = V + alpha[i] * (_var(yi[: m[i]]) - _var(yi[: m[i - 1]]))
    return V


def owen_main(fx, fxp, fz):
    """Owen's main-effect estimator V-hat_j (Eq. owen) from m pick-freeze groups.

    fx = f(x_i), fxp = f(x'_i), fz = f(z_i^(j)) with z_i^(j) = x'_i except coordinate j from x_i.
    """
    fx, fxp, fz = (np.asarray(a, np.float64) for a in (fx, fxp, fz))
    m = fx.shape[0]
    E, Ep = fx.sum(axis=0) / m, fxp.sum(axis=0) / m
    V, Vp = _var(fx), _var(fxp)
    return 2.0 * m / (2.0 * m - 1.0) * ((fx * fz).sum(axis=0) / m - ((E + Ep) / 2.0) ** 2 + (V + Vp) / (4.0 * m))


def jansen_total(fxp, fz):
    """Jansen's total-effect estimator T-hat_j (Eq. jansen): (1/2m) sum (f(x') - f(z^(j)))^2."""
    fxp, fz = np.asarray(fxp, np.float64), np.asarray(fz, np.float64)
    m = fxp.shape[0]
    return ((fxp - fz) ** 2).sum(axis=0) / (2.0 * m)


def mfmc_sobol(groups, m, alpha):
    """MFMC main and total Sobol' indices (Eqs. V_mf, T_mf) of d inputs.

    groups[i] is an array [n_i, d+2, ...] of model i's evaluations per
    pick-freeze group: column 0 = f(x), 1 = f(x'), 2+j = f(z^(j)).  Returns
    (s_main [d, ...], s_total [d, ...], mean, variance).
    """
    d = np.asarray(groups[0]).shape[1] - 2
    k = len(groups)

    def V_j(g, mm, j):
        g = np.asarray(g)[:mm]
        return owen_main(g[:, 0], g[:, 1], g[:, 2 + j])

    def T_j(g, mm, j):
        g = np.asarray(g)[:mm]
        return jansen_total(g[:, 1], g[:, 2 + j])

    s_main, s_tot = [], []
    var_y = mfmc_variance([np.asarray(g)[:, 0] for g in groups], m, alpha)
    mean_y = mfmc_mean([np.asarray(g)[:, 0] for g in groups], m, alpha)
    for j in range(d):
        Vmf = V_j(groups[0], m[0], j)
        Tmf = T_j(groups[0], m[0], j)
        for i in range(1, k):
            Vmf = Vmf + alpha[i] * (V_j(groups[i], m[i], j) - V_j(groups[i], m[i - 1], j))
            Tmf = Tmf + alpha[i] * (T_j(groups[i], m[i], j) - T_j(groups[i], m[i - 1], j))
        s_main.append(Vmf / var_y)
        s_tot.append(Tmf / var_y)
    return np.array(s_main), np.array(s_tot), mean_y, var_y


# ---------------------------------------------------------------------------
# Ishigami test function (Ishigami & Homma 1990) and its closed-form indices.
# ---------------------------------------------------------------------------
def ishigami(x, a=7.0, b=0.1):
    x = np.asarray(x, np.float64)
    return np.sin(x[..., 0]) + a * np.sin(x[..., 1]) ** 2 + b * x[..., 2] ** 4 * np.sin(x[..., 0])


def ishigami_indices(a=7.0, b=0.1):
    """Exact (mean, variance, first-order [3], total [3]) on U[-pi, pi]^3."""
    pi = np.pi
    V1 = 0.5 * (1 + b * pi ** 4 / 5) ** 2
    V2 = a ** 2 / 8
    V13 = b ** 2 * pi ** 8 * (1 / 18 - 1 / 50)
    V = V1 + V2 + V13
    s = np.array([V1, V2, 0.0]) / V
    st = np.array([V1 + V13, V2, V13]) / V
    return a / 2.0, V, s, st


def pick_freeze_inputs(x, xp):
    """[m, d+2, d] inputs of the pick-freeze groups: x, x', z^(1..d)."""
    x, xp = np.asarray(x), np.asarray(xp)
    m, d = x.shape
    out = np.empty((m, d + 2, d))
    out[:, 0] = x
    out[:, 1] = xp
    for j in range(d):
        z = xp.copy()
        z[:, j] = x[:, j]
        out[:, 2 + j] = z
    return out


def bootstrap_ci(groups, m, alpha, boot_index, n_boot):
    """Percentile intervals (ranks round(0.025 (B-1)), round(0.975 (B-1))) of the MFMC Sobol' indices.

    boot_index(b) gives the resampled group indices (length m[-1]) of replicate b, drawn within
    the nesting blocks [m[i-1], m[i]); model i uses the first m[i] of them.
    """
    reps_m, reps_t = [], []
    for b in range(1, n_boot + 1):
        idx = boot_index(b)
        g = [np.asarray(gr)[idx[: m[i]]] for i, gr in enumerate(groups)]
        sm, st, _, _ = mfmc_sobol(g, m, alpha)
        reps_m.append(sm)
        reps_t.append(st)
    reps_m, reps_t = np.sort(np.array(reps_m), axis=0), np.sort(np.array(reps_t), axis=0)
    lo, hi = int(round(0.025 * (n_boot - 1))), int(round(0.975 * (n_boot - 1)))
    return np.stack([reps_m[lo], reps_m[hi]], -1), np.stack([reps_t[lo], reps_t[hi]], -1)


def dgsm_bound(grad, y, width):
    """Sobol'-Kucherenko bound s_j^t <= (b_j - a_j)^2 E[(df/dx_j)^2] / (pi^2 Var f), inputs uniform.

    grad [S, ..., d], y [S, ...]; returns (nu [d, ...], bound [d, ...]).
    """
    grad, y = np.asarray(grad, np.float64), np.asarray(y, np.float64)
    S = y.shape[0]
    nu = np.moveaxis((grad ** 2).sum(axis=0) / S, -1, 0)
    var = ((y - y.sum(axis=0) / S) ** 2).sum(axis=0) / (S - 1)
    w = np.asarray(width, np.float64).reshape((-1,) + (1,) * (nu.ndim - 1))
    return nu, w ** 2 * nu / (np.pi ** 2 * var)


def ishigami_grad(x, a=7.0, b=0.1):
    x = np.asarray(x, np.float64)
    g = np.empty_like(x)
    g[..., 0] = np.cos(x[..., 0]) * (1 + b * x[..., 2] ** 4)
    g[..., 1] = 2 * a * np.sin(x[..., 1]) * np.cos(x[..., 1])
    g[..., 2] = 4 * b * x[..., 2] ** 3 * np.sin(x[..., 0])
    return g
