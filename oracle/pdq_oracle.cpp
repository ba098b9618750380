// pdq_oracle.cpp -- FP64 CPU oracle of the Lagrangian particle-deposition step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA library is checked against.  Only the test-suite, the smoke check and
// the benchmark's CPU-baseline / reference arm may load it; the product path
// never does.  It shares no code, header, table or constant generator with the
// CUDA library: every formula below is written out again from the paper
// (Yao, Huan & Capecelatro, "Multi-fidelity uncertainty quantification of
// particle deposition in turbulent pipe flow").
//
// Loops run in natural order: samples, then particles i, then all particles j
// of the same sample.  OpenMP parallelises only the loop over i; each i keeps
// its own sequential sum, so results do not depend on the thread count.
//
// Everything is in wall units (+): length nu/u*, velocity u*, time nu/u*^2.
// Parameter derivatives for the dual-number reference use the same templated
// code with T = Dual (forward mode, three tangents: xi, zeta, theta).
//
// Pinned by tests/test_oracle_*.py; functions without a pin say so below.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random numbers:
// as easy as 1, 2, 3").  Used to draw the synthetic-field modes and the
// particle seeds; the CUDA library carries its own implementation.
// ---------------------------------------------------------------------------
static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// 32-bit word -> double strictly inside (0, 1): (x + 1/2) / 2^32, exact.
static inline double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// ---------------------------------------------------------------------------
// Dual numbers (value + 3 tangents) for the forward-mode derivative reference.
// ---------------------------------------------------------------------------
struct Dual {
    double v; double d[3];
    Dual() : v(0) { d[0] = d[1] = d[2] = 0; }
    Dual(double x) : v(x) { d[0] = d[1] = d[2] = 0; }
};
static inline double val(double x) { return x; }
static inline double val(const Dual& x) { return x.v; }
static inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
static inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
static inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < 3; ++i) r.d[i] = -a.d[i]; return r; }
static inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
static inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < 3; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
static inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
static inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
static inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
static inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
static inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * b; return r; }
static inline Dual operator*(double a, const Dual& b) { return b * a; }
static inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
static inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
static inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
static inline Dual chain(const Dual& a, double f, double df) { Dual r(f); for (int i = 0; i < 3; ++i) r.d[i] = df * a.d[i]; return r; }
static inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, s > 0 ? 0.5 / s : 0.0); }
static inline Dual exp(const Dual& a) { double e = std::exp(a.v); return chain(a, e, e); }
static inline Dual expm1(const Dual& a) { return chain(a, std::expm1(a.v), std::exp(a.v)); }
static inline Dual log(const Dual& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
static inline Dual pow(const Dual& a, double p) { double f = std::pow(a.v, p); return chain(a, f, a.v > 0 ? p * f / a.v : 0.0); }
static inline Dual atanh(const Dual& a) { return chain(a, std::atanh(a.v), 1.0 / (1.0 - a.v * a.v)); }
static inline Dual atan2(const Dual& y, const Dual& x) {
    Dual r(std::atan2(y.v, x.v));
    double q = x.v * x.v + y.v * y.v;
    for (int i = 0; i < 3; ++i) r.d[i] = q > 0 ? (x.v * y.d[i] - y.v * x.d[i]) / q : 0.0;
    return r;
}
static inline Dual sin(const Dual& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
static inline Dual cos(const Dual& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
using std::sqrt; using std::exp; using std::expm1; using std::log; using std::pow; using std::atanh; using std::atan2;
using std::sin; using std::cos;
// max/min choose by value (the derivative of the selected branch).
template <class T> static inline T vmax(const T& a, const T& b) { return val(a) >= val(b) ? a : b; }
template <class T> static inline T vmin(const T& a, const T& b) { return val(a) <= val(b) ? a : b; }

// ---------------------------------------------------------------------------
// Physical constants and derived wall units.
// Values: pipe D = 20 mm, nu = 1.5e-5 m^2/s, Re_tau = 180, U_b = 4 m/s,
// rho_p = 2650 kg/m^3 (Sec. 2.1); rho_f = 1.2 kg/m^3 (not printed; this value
// reproduces the printed tau_p+ = 0.1, 1, 10 for d_p = 1.6, 5, 16 um);
// eps0 = 8.854e-12 (Eq. coulomb); q_max = 500 e (d_p/1um)^2 (Eq. q_max);
// A0 = 1e-18 J (Sec. 2.1); delta_min = 1e-9 m (Sec. 2.2);
// E = 70 GPa, delta_c = 0.165 nm, sigma_y0 = 200 MPa (Sec. 4.3);
// restitution e = 0.9 and contact time tau_col = 15 dt of the soft-sphere
// collisions (App. A.2, collision force); neg_charge_frac = share of particles
// seeded with a negative charge (0: the paper's like-signed charges).
// ---------------------------------------------------------------------------
extern "C" {

struct OrcPhys {
    double nu, radius, re_tau, u_bulk, rho_p, rho_f, eps0, qmax_coef,
           hamaker0, delta_min, young, delta_c, sigma_y0, g,
           restitution, tau_col_steps, neg_charge_frac,
           contact_scale;   // Coulomb distance clamp = contact_scale x the largest class diameter
};

struct OrcField {
    double r_plus;      // pipe radius in wall units (= Re_tau)
    double l_plus;      // periodic length in wall units
    int32_t n_r, n_th, n_z, n_modes;
    double u_rms;       // per-component rms of the fluctuation at the axis
    double beta;        // radial stretching: r = R tanh(beta s)/tanh(beta)
    double kappa, b_log;// log-law constants
    double k_min, k_max;// wavenumber shell of the random modes
};

// Step configuration (mirrors the CUDA library's meaning, not its layout).
struct OrcCfg {
    double dt;                 // time step, wall units
    double gravity[3];         // gravity direction (unit vector or zero)
    int32_t mode;              // 0 = all-stick, 1 = rebound (Bons et al.)
    int32_t forces;            // bit mask: 1 drag, 2 gravity, 4 coulomb, 8 image, 16 vdw (wall),
                               // 32 soft-sphere collisions, 64 particle-particle vdw
    int64_t window_start;      // first step index counted in the tallies
    double smooth_eps;         // > 0: smoothed wall indicator of this width (no removal)
    double stick_eps;          // smoothed rebound: width (m^2/s^2) of the sticking probability
};

void orc_phys_default(OrcPhys* p) {
    p->nu = 1.5e-5; p->radius = 0.01; p->re_tau = 180.0; p->u_bulk = 4.0;
    p->rho_p = 2650.0; p->rho_f = 1.2; p->eps0 = 8.854e-12; p->qmax_coef = 500.0 * 1.6e-19;
    p->hamaker0 = 1e-18; p->delta_min = 1e-9; p->young = 70e9; p->delta_c = 0.165e-9;
    p->sigma_y0 = 200e6; p->g = 9.81;
    p->restitution = 0.9; p->tau_col_steps = 15.0; p->neg_charge_frac = 0.0;
    p->contact_scale = 1.0;
}

}  // extern "C"

struct Units {
    double ustar, ell, tauf, acc;  // u*, nu/u*, nu/u*^2, SI acceleration -> wall units factor
};
static Units units(const OrcPhys& p) {
    Units u;
    u.ustar = p.re_tau * p.nu / p.radius;
    u.ell = p.nu / u.ustar;
    u.tauf = p.nu / (u.ustar * u.ustar);
    u.acc = p.nu / (u.ustar * u.ustar * u.ustar);
    return u;
}

// One size class, from its Stokes number tau_p+ = tau_p / tau_f with
// tau_p = rho_p d^2 / (18 rho_f nu) (Sec. 2.1).
struct ClassProps {
    double tau_plus, d_plus, d, mass, qfac;  // qfac = (d / 1 um)^2
};
static ClassProps class_props(const OrcPhys& p, double st_plus) {
    Units u = units(p);
    ClassProps c;
    c.tau_plus = st_plus;
    double tau_p = st_plus * u.tauf;
    c.d = std::sqrt(tau_p * 18.0 * p.rho_f * p.nu / p.rho_p);
    c.d_plus = c.d / u.ell;
    c.mass = p.rho_p * M_PI * c.d * c.d * c.d / 6.0;
    c.qfac = (c.d / 1e-6) * (c.d / 1e-6);
    return c;
}

extern "C" {

// Per-class table row: [tau+, d+, d (m), mass (kg), (d/1um)^2].
void orc_class_table(const OrcPhys* p, int n, const double* st_plus, double* out) {
    for (int c = 0; c < n; ++c) {
        ClassProps k = class_props(*p, st_plus[c]);
        out[5 * c + 0] = k.tau_plus; out[5 * c + 1] = k.d_plus; out[5 * c + 2] = k.d;
        out[5 * c + 3] = k.mass; out[5 * c + 4] = k.qfac;
    }
}

// ---------------------------------------------------------------------------
// Force laws in SI (Sec. 2.2).  These are the printed forms.
// ---------------------------------------------------------------------------

// Eq. (vdw): van der Waals force magnitude between two equal spheres of
// diameter d whose surfaces are delta apart.
double orc_vdw_pp(double A, double d, double delta) {
    double a = A / 6.0 * d * d * (d + delta) / (delta * delta * (2 * d + delta) * (2 * d + delta));
    double br = delta * (2 * d + delta) / ((d + delta) * (d + delta)) - 1.0;
    return a * br * br;
}

// Eq. (coulomb), read with the centre distance r (the 1/delta form is
// dimensionally inconsistent).  Positive = repulsive.
double orc_coulomb_pp(double q1, double q2, double r, double eps0) {
    return q1 * q2 / (4.0 * M_PI * eps0) / (r * r);
}

// Domain-averaged particle-wall force of Sec. 2.2 (the radial integral with
// weight 8 delta / D^2), by composite Simpson on a graded grid.  kind 0:
// electrostatic image, F_wall(s) = F_C(2s), cut-off d/2; kind 1: van der
// Waals, F_wall(s) = 2 F_vw(s), cut-off delta_min.
double orc_wall_average(int kind, double D, double d, double q, double A, double eps0, double delta_min) {
    double R = 0.5 * D;
    double cut = kind == 0 ? 0.5 * d : delta_min;
    // integrate over s = distance to the wall in [cut, R]; radial coordinate = R - s
    // substitution s = cut * exp(t), t in [0, ln(R/cut)] resolves the 1/s^2 end.
    int n = 200000;
    double T = std::log(R / cut);
    double h = T / n, sum = 0.0;
    for (int k = 0; k <= n; ++k) {
        double t = k * h, s = cut * std::exp(t);
        double F = kind == 0 ? orc_coulomb_pp(q, q, 2.0 * s, eps0) : 2.0 * orc_vdw_pp(A, d, s);
        double w = (k == 0 || k == n) ? 1.0 : (k % 2 ? 4.0 : 2.0);
        sum += w * F * (8.0 * (R - s) / (D * D)) * s;  // ds = s dt
    }
    return sum * h / 3.0;
}

// ---------------------------------------------------------------------------
// Synthetic carrier field (the paper's DNS field is not available).
// Mean: U+(y+) = y+ below the crossing y_c, (1/kappa) ln y+ + B above.
// Fluctuation: u' = curl( f(r) sum_n b_n cos(k_n . x + phi_n) ),
// f = (1 - r^2/R^2)^2, so div u' = 0 and u' = 0 at the wall.
// ---------------------------------------------------------------------------

// Crossing of the viscous sublayer and the log law, by bisection.
double orc_ycross(double kappa, double B) {
    double lo = 1.0 / kappa, hi = 1000.0;   // g(y) = y - ln(y)/kappa - B increases for y > 1/kappa
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double g = mid - std::log(mid) / kappa - B;
        if (g > 0) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

double orc_mean_profile(double yplus, double kappa, double B, double yc) {
    if (yplus <= yc) return yplus;
    return std::log(yplus) / kappa + B;
}

// Mode table [n_modes][7] = (kx, ky, kz, bx, by, bz, phi).
void orc_field_modes(const OrcField* f, uint64_t seed, double* modes) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double amp = f->u_rms * std::sqrt(6.0 / f->n_modes);
    double dkz = 2.0 * M_PI / f->l_plus;
    for (int n = 0; n < f->n_modes; ++n) {
        uint32_t c0[4] = {(uint32_t)n, 0u, 0u, 1u}, c1[4] = {(uint32_t)n, 1u, 0u, 1u};
        uint32_t a[4], b[4];
        philox4x32_10(c0, key, a);
        philox4x32_10(c1, key, b);
        double kmag = f->k_min * std::pow(f->k_max / f->k_min, u01(a[0]));
        double ct = 2.0 * u01(a[1]) - 1.0;
        double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
        double ph = 2.0 * M_PI * u01(a[2]);
        double kx = kmag * st * std::cos(ph), ky = kmag * st * std::sin(ph), kz = kmag * ct;
        kz = dkz * std::rint(kz / dkz);  // periodic in z
        double kn = std::sqrt(kx * kx + ky * ky + kz * kz);
        double e1[3], e2[3];
        double kp = std::sqrt(kx * kx + ky * ky);
        if (kp > 0) { e1[0] = ky / kp; e1[1] = -kx / kp; e1[2] = 0.0; }
        else { e1[0] = 1.0; e1[1] = 0.0; e1[2] = 0.0; }
        double kh[3] = {kx / kn, ky / kn, kz / kn};
        e2[0] = kh[1] * e1[2] - kh[2] * e1[1];
        e2[1] = kh[2] * e1[0] - kh[0] * e1[2];
        e2[2] = kh[0] * e1[1] - kh[1] * e1[0];
        double psi = 2.0 * M_PI * u01(a[3]);
        double bm = amp / kn;
        double* m = modes + 7 * n;
        m[0] = kx; m[1] = ky; m[2] = kz;
        for (int i = 0; i < 3; ++i) m[3 + i] = bm * (std::cos(psi) * e1[i] + std::sin(psi) * e2[i]);
        m[6] = 2.0 * M_PI * u01(b[0]);
    }
}

// Analytic velocity at n Cartesian points xyz[n][3] -> u[n][3].
void orc_field_velocity(const OrcField* f, const double* modes, int n, const double* xyz, double* out) {
    const double R = f->r_plus;
    const double yc = orc_ycross(f->kappa, f->b_log);
    for (int p = 0; p < n; ++p) {
        double x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
        double r2 = x * x + y * y, r = std::sqrt(r2);
        double g = 1.0 - r2 / (R * R);
        double fr = 0.0, gf[3] = {0, 0, 0};
        if (r < R) { fr = g * g; gf[0] = -4.0 / (R * R) * g * x; gf[1] = -4.0 / (R * R) * g * y; }
        double S[3] = {0, 0, 0}, Tv[3] = {0, 0, 0};
        for (int k = 0; k < f->n_modes; ++k) {
            const double* m = modes + 7 * k;
            double arg = m[0] * x + m[1] * y + m[2] * z + m[6];
            double c = std::cos(arg), s = std::sin(arg);
            // k x b
            double kb[3] = {m[1] * m[5] - m[2] * m[4], m[2] * m[3] - m[0] * m[5], m[0] * m[4] - m[1] * m[3]};
            for (int i = 0; i < 3; ++i) { S[i] += m[3 + i] * c; Tv[i] += s * kb[i]; }
        }
        // curl(f b cos) = cos (grad f x b) - f sin (k x b)
        double u[3];
        u[0] = gf[1] * S[2] - gf[2] * S[1] - fr * Tv[0];
        u[1] = gf[2] * S[0] - gf[0] * S[2] - fr * Tv[1];
        u[2] = gf[0] * S[1] - gf[1] * S[0] - fr * Tv[2];
        double yp = R - r;
        if (yp < 0) yp = 0;
        u[2] += orc_mean_profile(yp, f->kappa, f->b_log, yc);
        out[3 * p] = u[0]; out[3 * p + 1] = u[1]; out[3 * p + 2] = u[2];
    }
}

// Node position of grid point (i, j, k): r_i = R tanh(beta s_i)/tanh(beta),
// s_i = i/(n_r-1), theta_j = 2 pi j / n_th, z_k = L k / n_z.
static void node_xyz(const OrcField* f, int i, int j, int k, double* xyz) {
    double s = (double)i / (f->n_r - 1);
    double r = f->r_plus * std::tanh(f->beta * s) / std::tanh(f->beta);
    double th = 2.0 * M_PI * j / f->n_th;
    xyz[0] = r * std::cos(th); xyz[1] = r * std::sin(th); xyz[2] = f->l_plus * k / f->n_z;
}

// Gridded field [n_z][n_th][n_r][3] (Cartesian components at the nodes).
void orc_field_grid(const OrcField* f, const double* modes, double* grid) {
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < f->n_z; ++k)
        for (int j = 0; j < f->n_th; ++j)
            for (int i = 0; i < f->n_r; ++i) {
                double xyz[3];
                node_xyz(f, i, j, k, xyz);
                orc_field_velocity(f, modes, 1, xyz, grid + 3 * (((size_t)k * f->n_th + j) * f->n_r + i));
            }
}

}  // extern "C"

// Trilinear interpolation in (s, theta, z) index space; periodic theta, z;
// s clamped to [0, 1].
template <class T>
static void interp(const OrcField* f, const double* grid, const T& x, const T& y, const T& z, T u[3]) {
    const double R = f->r_plus, L = f->l_plus;
    T r = sqrt(x * x + y * y);
    T rho = vmin(r / R, T(1.0));
    T s = atanh(rho * std::tanh(f->beta)) / f->beta;
    T fi = s * (double)(f->n_r - 1);
    int i0 = (int)std::floor(val(fi));
    if (i0 > f->n_r - 2) i0 = f->n_r - 2;
    if (i0 < 0) i0 = 0;
    T tr = fi - (double)i0;
    T th = atan2(y, x);
    T fj = th * (f->n_th / (2.0 * M_PI));
    if (val(fj) < 0) fj = fj + (double)f->n_th;
    int j0 = (int)std::floor(val(fj));
    T tt = fj - (double)j0;
    j0 %= f->n_th;
    int j1 = (j0 + 1) % f->n_th;
    T zz = z - L * std::floor(val(z) / L);
    T fk = zz * (f->n_z / L);
    int k0 = (int)std::floor(val(fk));
    T tz = fk - (double)k0;
    k0 %= f->n_z;
    int k1 = (k0 + 1) % f->n_z;
    for (int c = 0; c < 3; ++c) u[c] = T(0.0);
    const int js[2] = {j0, j1}, ks[2] = {k0, k1};
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                T w = (di ? tr : 1.0 - tr) * (dj ? tt : 1.0 - tt) * (dk ? tz : 1.0 - tz);
                const double* g = grid + 3 * (((size_t)ks[dk] * f->n_th + js[dj]) * f->n_r + (i0 + di));
                for (int c = 0; c < 3; ++c) u[c] += w * g[c];
            }
}

extern "C" void orc_interp(const OrcField* f, const double* grid, int n, const double* xyz, double* out) {
    for (int p = 0; p < n; ++p) {
        double u[3];
        interp<double>(f, grid, xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], u);
        for (int c = 0; c < 3; ++c) out[3 * p + c] = u[c];
    }
}

// ---------------------------------------------------------------------------
// Seeding (Sec. 2.1: particles randomly distributed in the pipe, q_p = xi
// q_max).  Particle j of every sample uses Philox counter (j, 0, 0, w3) (and
// (j, 1, 0, w3) for the charge factor, (j, 2, 0, w3) for its sign), with
// w3 = 0, so all samples share their first particles (common random numbers),
// or, when `independent`, w3 = s + 1: a stream per sample.  Class = j mod C.
// ---------------------------------------------------------------------------
extern "C" int orc_seed(const OrcPhys* p, const OrcField* f, int n_classes, const double* st_plus,
                        double charge_sigma, uint64_t seed, int n_samples, const int64_t* offset,
                        const double* params /*[S][3]: xi, zeta, theta*/,
                        double* x, double* y, double* z, double* vx, double* vy, double* vz,
                        double* q, int32_t* alive, int32_t* cls, int32_t* id, int independent) {
    std::vector<ClassProps> cp(n_classes);
    for (int c = 0; c < n_classes; ++c) cp[c] = class_props(*p, st_plus[c]);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int s = 0; s < n_samples; ++s) {
        double xi = params[3 * s];
        const uint32_t w3 = independent ? (uint32_t)(s + 1) : 0u;
        for (int64_t g = offset[s]; g < offset[s + 1]; ++g) {
            uint32_t j = (uint32_t)(g - offset[s]);
            uint32_t c0[4] = {j, 0u, 0u, w3}, a[4];
            philox4x32_10(c0, key, a);
            int c = (int)(j % (uint32_t)n_classes);
            double lam = 1.0;
            if (p->neg_charge_frac > 0) {
                // sign of the charge: negative with probability neg_charge_frac (counter word 2)
                uint32_t c2[4] = {j, 2u, 0u, w3}, b[4];
                philox4x32_10(c2, key, b);
                if (u01(b[0]) < p->neg_charge_frac) lam = -1.0;
            }
            if (charge_sigma > 0) {
                uint32_t c1[4] = {j, 1u, 0u, w3}, b[4];
                philox4x32_10(c1, key, b);
                double nrm = std::sqrt(-2.0 * std::log(u01(b[0]))) * std::cos(2.0 * M_PI * u01(b[1]));
                lam *= std::exp(charge_sigma * nrm);
            }
            double rr = (f->r_plus - 0.5 * cp[c].d_plus) * std::sqrt(u01(a[0]));
            double th = 2.0 * M_PI * u01(a[1]);
            x[g] = rr * std::cos(th); y[g] = rr * std::sin(th); z[g] = f->l_plus * u01(a[2]);
            vx[g] = vy[g] = vz[g] = 0.0;
            q[g] = xi * cp[c].qfac * lam;
            alive[g] = 1; cls[g] = c; id[g] = (int32_t)j;
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Particle step (App. A.2, Eq. newtonlaw with Eq. part_source), plus gravity,
// image charge and van der Waals wall cohesion, wall contact and the V_dep
// tally.  Time integration: exponential integrator with the fluid velocity,
// the drag factor and the non-drag acceleration frozen over the step:
//   v' = v e + (lam u + a) h phi1(-lam h),  x' = x + v h phi1 + (lam u + a) h^2 phi2,
//   e = exp(-lam h), lam = f / tau_p+, phi1(z) = (e^z-1)/z, phi2(z) = (e^z-1-z)/z^2.
// ---------------------------------------------------------------------------
template <class T> static T phi1(const T& zz) {
    if (std::fabs(val(zz)) < 1e-2) {
        T z2 = zz * zz;
        return 1.0 + zz / 2.0 + z2 / 6.0 + z2 * zz / 24.0 + z2 * z2 / 120.0 + z2 * z2 * zz / 720.0;
    }
    return expm1(zz) / zz;
}
template <class T> static T phi2(const T& zz) {
    if (std::fabs(val(zz)) < 1e-2) {
        T z2 = zz * zz;
        return 0.5 + zz / 6.0 + z2 / 24.0 + z2 * zz / 120.0 + z2 * z2 / 720.0 + z2 * z2 * zz / 5040.0;
    }
    return (expm1(zz) - zz) / (zz * zz);
}

// logistic(a) = 1 / (1 + e^-a), evaluated without overflow for either sign of a
template <class T> static T logistic(const T& a) {
    if (val(a) >= 0) return 1.0 / (1.0 + exp(-a));
    T e = exp(a);
    return e / (1.0 + e);
}

enum { F_DRAG = 1, F_GRAV = 2, F_COUL = 4, F_IMAGE = 8, F_VDW = 16, F_COLLIDE = 32, F_VDWPP = 64 };

struct SampleParams { double xi, zeta, theta; };

template <class T>
struct Run {
    const OrcPhys* p; const OrcField* f; const double* grid; const OrcCfg* cfg;
    Units un; std::vector<ClassProps> cp; double contact;  // Coulomb clamp distance (wall units)
    const double* ext = nullptr;   // given Coulomb sums [n][3] of this sample (replace the pair loop)
};

// Non-drag acceleration of particle i (wall units) without the Coulomb sum.
template <class T>
static void wall_and_body(const Run<T>& rn, const ClassProps& c, const T& x, const T& y, const T& qi,
                          const T& zeta, T a[3]) {
    const OrcPhys& p = *rn.p;
    const double R = rn.f->r_plus;
    a[0] = a[1] = a[2] = T(0.0);
    if (rn.cfg->forces & F_GRAV) {
        double gp = p.g * rn.un.acc;
        for (int k = 0; k < 3; ++k) a[k] = a[k] + gp * rn.cfg->gravity[k];
    }
    T r = sqrt(x * x + y * y);
    if (val(r) <= 0) return;  // radial direction undefined at the axis; both wall forces are negligible there
    T nx = x / r, ny = y / r;  // outward unit normal
    if (rn.cfg->forces & F_IMAGE) {
        // image charge of opposite sign mirrored across the wall (Sec. 2.2):
        // F = q^2 / (4 pi eps0 (2 y)^2), toward the wall; y >= d/2.
        T yw = vmax(R - r, T(0.5 * c.d_plus)) * rn.un.ell;  // SI
        T qq = qi * p.qmax_coef;
        T F = qq * qq / (4.0 * M_PI * p.eps0) / (4.0 * yw * yw);
        T acc = F / c.mass * rn.un.acc;
        a[0] = a[0] + acc * nx; a[1] = a[1] + acc * ny;
    }
    if (rn.cfg->forces & F_VDW) {
        // F_wall = 2 F_vw(delta) (Sec. 2.2), delta = surface-wall gap, saturated
        // at delta_min and cut off beyond d/4.
        T gap = (R - r - 0.5 * c.d_plus) * rn.un.ell;
        if (val(gap) <= 0.25 * c.d) {
            T dl = vmax(gap, T(p.delta_min));
            T A = zeta * p.hamaker0;
            T d = T(c.d);
            T F = 2.0 * (A / 6.0 * d * d * (d + dl) / (dl * dl * (2.0 * d + dl) * (2.0 * d + dl)));
            T br = dl * (2.0 * d + dl) / ((d + dl) * (d + dl)) - 1.0;
            F = F * br * br;
            T acc = F / c.mass * rn.un.acc;
            a[0] = a[0] + acc * nx; a[1] = a[1] + acc * ny;
        }
    }
}

// Contact accelerations (wall units) added to a*[i].
//  Collision: a linear spring-dashpot between the two surfaces (normal direction only: the
//  paper names tangential collisions but prints no friction coefficient).  For a pair with
//  effective mass m_ij = m_i m_j / (m_i + m_j) the relative normal motion obeys
//  delta'' + H delta' + K delta = 0 while the spheres overlap by delta; choosing
//  K = (pi^2 + ln^2 e) / tau_col^2 and H = -2 ln e / tau_col makes a contact last exactly
//  tau_col and return the approach speed times e (the damped-oscillator solution).  Particle
//  i receives m_ij / m_i of that relative acceleration, along n = (x_i - x_j) / r.
//  Van der Waals: Eq. (vdw) for equal spheres, evaluated with the effective diameter
//  2 d_i d_j / (d_i + d_j) (so that its contact limit is the Derjaguin force of the two
//  unequal spheres), surface gap saturated at delta_min, zero beyond a quarter of that
//  diameter (Sec. 2.2); attractive, along -n.  Overlapping spheres keep the saturated value
//  (the modified cohesion model the paper cites is not printed).
template <class T>
static void contact_forces(const Run<T>& rn, int n, const T* x, const T* y, const T* z, const T* vx,
                           const T* vy, const T* vz, const int32_t* alive, const int32_t* cls, const T& zeta,
                           T* ax, T* ay, T* az) {
    const OrcCfg& cfg = *rn.cfg;
    const OrcPhys& p = *rn.p;
    const double L = rn.f->l_plus, h = cfg.dt;
    const double tc = p.tau_col_steps * cfg.dt;
    const double le = std::log(p.restitution);
    const double Kc = (M_PI * M_PI + le * le) / (tc * tc);
    const double Hc = -2.0 * le / tc;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        if (!alive[i]) continue;
        const ClassProps& ci = rn.cp[cls[i]];
        for (int j = 0; j < n; ++j) {
            if (j == i || !alive[j]) continue;
            const ClassProps& cj = rn.cp[cls[j]];
            // separation at the mid-step predicted positions x + v dt/2
            T dx = x[i] - x[j] + 0.5 * h * (vx[i] - vx[j]);
            T dy = y[i] - y[j] + 0.5 * h * (vy[i] - vy[j]);
            T dz = z[i] - z[j] + 0.5 * h * (vz[i] - vz[j]);
            dz = dz - L * std::rint(val(dz) / L);
            T r = sqrt(dx * dx + dy * dy + dz * dz);
            if (val(r) <= 0) continue;
            T nx = dx / r, ny = dy / r, nz = dz / r;
            const double contact = 0.5 * (ci.d_plus + cj.d_plus);
            if ((cfg.forces & F_COLLIDE) && val(r) < contact) {
                T overlap = contact - r;
                T vn = (vx[i] - vx[j]) * nx + (vy[i] - vy[j]) * ny + (vz[i] - vz[j]) * nz;
                double mu = cj.mass / (ci.mass + cj.mass);   // m_ij / m_i
                T a = mu * (Kc * overlap - Hc * vn);
                ax[i] += a * nx; ay[i] += a * ny; az[i] += a * nz;
            }
            if (cfg.forces & F_VDWPP) {
                double deff = 2.0 * ci.d * cj.d / (ci.d + cj.d);   // m
                T gap = (r - contact) * rn.un.ell;                 // surface gap, m
                if (val(gap) <= 0.25 * deff) {
                    double g = std::max(val(gap), p.delta_min);
                    double F = orc_vdw_pp(val(zeta) * p.hamaker0, deff, g);
                    T a = T(F / ci.mass * rn.un.acc);
                    ax[i] -= a * nx; ay[i] -= a * ny; az[i] -= a * nz;
                }
            }
        }
    }
}

// Advance one sample by one step.  State arrays are this sample's slice.
// Returns per-class deposited count and alive-at-start count (STICK/REBOUND),
// or the smoothed sums (smooth mode) through num/den.
template <class T>
static void step_sample(const Run<T>& rn, int n, T* x, T* y, T* z, T* vx, T* vy, T* vz, const T* q,
                        T* w, int32_t* alive, const int32_t* cls,
                        const T& zeta, const T& theta, bool counted, int64_t* ndep, int64_t* nalive,
                        T* num, T* den) {
    const OrcCfg& cfg = *rn.cfg;
    const double R = rn.f->r_plus, L = rn.f->l_plus, h = cfg.dt;
    const bool smooth = cfg.smooth_eps > 0;
    std::vector<T> ax(n), ay(n), az(n);
    // 1) Coulomb all-pairs (Eq. coulomb, App. A.2: F_i = sum_{j != i} F_ij n_ij),
    //    minimum image in z, centre distance clamped at the contact distance (or given sums).
    if (cfg.forces & F_COUL) {
        if (rn.ext) {
            for (int i = 0; i < n; ++i) {
                ax[i] = T(rn.ext[3 * i]); ay[i] = T(rn.ext[3 * i + 1]); az[i] = T(rn.ext[3 * i + 2]);
            }
        } else {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            T sx(0.0), sy(0.0), sz(0.0);
            if (smooth || alive[i]) {
                for (int j = 0; j < n; ++j) {
                    if (j == i) continue;
                    if (!smooth && !alive[j]) continue;
                    T dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
                    dz = dz - L * std::rint(val(dz) / L);
                    T r2 = dx * dx + dy * dy + dz * dz;
                    T rr = vmax(sqrt(r2), T(rn.contact));
                    T qj = smooth ? q[j] * w[j] : q[j];
                    T s = qj / (rr * rr * rr);
                    sx += s * dx; sy += s * dy; sz += s * dz;
                }
            }
            ax[i] = sx; ay[i] = sy; az[i] = sz;
        }
        }
        // coefficient q_i (q_ref^2 / (4 pi eps0 m_i)) in wall units
        for (int i = 0; i < n; ++i) {
            const ClassProps& c = rn.cp[cls[i]];
            double coef = rn.p->qmax_coef * rn.p->qmax_coef / (4.0 * M_PI * rn.p->eps0) / c.mass
                          / (rn.un.ell * rn.un.ell) * rn.un.acc;
            T k = q[i] * coef;
            ax[i] = k * ax[i]; ay[i] = k * ay[i]; az[i] = k * az[i];
        }
    } else {
        for (int i = 0; i < n; ++i) ax[i] = ay[i] = az[i] = T(0.0);
    }
    // 1b) particle-particle contact (App. A.2): soft-sphere normal collisions and the van der
    //     Waals attraction of Eq. (vdw), pair by pair over the live particles of the sample.
    if (!smooth && (cfg.forces & (F_COLLIDE | F_VDWPP))) contact_forces(rn, n, x, y, z, vx, vy, vz, alive, cls,
                                                                         zeta, ax.data(), ay.data(), az.data());
    // 2) local forces, integration, wall contact, tallies.
    for (int i = 0; i < n; ++i) {
        if (!smooth && !alive[i]) continue;
        const int ci = cls[i];
        const ClassProps& c = rn.cp[ci];
        T a[3];
        wall_and_body(rn, c, x[i], y[i], q[i], zeta, a);
        a[0] = a[0] + ax[i]; a[1] = a[1] + ay[i]; a[2] = a[2] + az[i];
        T u[3];
        interp(rn.f, rn.grid, x[i], y[i], z[i], u);
        T lam(0.0);
        if (cfg.forces & F_DRAG) {
            T rx = u[0] - vx[i], ry = u[1] - vy[i], rz = u[2] - vz[i];
            T rep = sqrt(rx * rx + ry * ry + rz * rz) * c.d_plus;   // Re_p = |u - v| d_p / nu
            T fd = 1.0 + 0.15 * pow(rep, 0.687);                   // Schiller-Naumann
            lam = fd / c.tau_plus;
        } else {
            u[0] = u[1] = u[2] = T(0.0);
        }
        T zz = -(lam * h);
        T p1 = phi1(zz), p2 = phi2(zz);
        T e = exp(zz);
        T v[3] = {vx[i], vy[i], vz[i]};
        T pos[3] = {x[i], y[i], z[i]};
        for (int k = 0; k < 3; ++k) {
            T forcing = lam * u[k] + a[k];
            T vn = v[k] * e + forcing * h * p1;
            pos[k] = pos[k] + v[k] * h * p1 + forcing * (h * h) * p2;
            v[k] = vn;
        }
        pos[2] = pos[2] - L * std::floor(val(pos[2]) / L);
        T rnew = sqrt(pos[0] * pos[0] + pos[1] * pos[1]);
        T gap = R - rnew - 0.5 * c.d_plus;
        if (smooth) {
            // smoothed removal: the weight drops by the contact indicator sigma(-gap/eps), times,
            // in rebound mode, the sticking probability sigma(-arg/eps_s) of the Bons model; the
            // weight that does not stick rebounds with CoR_n (Sec. 4.3; CoR_n = 0 when arg <= 0)
            T pstick(1.0);
            if (cfg.mode == 1) {
                const OrcPhys& p = *rn.p;
                T sy = p.sigma_y0 * (1.0 - theta);
                T gc = zeta * p.hamaker0 / (24.0 * M_PI * p.delta_c * p.delta_c);
                double acont = M_PI * c.d * c.d / 4.0;
                T arg = sy * sy / (p.rho_p * p.young) - 2.0 * acont * gc / c.mass;
                pstick = logistic(-arg / cfg.stick_eps);
                if (val(gap) <= 0) {
                    T nx = pos[0] / rnew, ny = pos[1] / rnew;
                    T vn1 = v[0] * nx + v[1] * ny;
                    T vn1_si = vn1 * rn.un.ustar;
                    T cor(0.0);
                    if (val(arg) > 0) {
                        cor = T(1.0);
                        if (val(vn1_si) > 0) cor = vmin(T(1.0), sqrt(arg) / vn1_si);
                    }
                    T vabs = val(vn1) >= 0 ? vn1 : -vn1;
                    T dv = -cor * vabs - vn1;
                    v[0] = v[0] + dv * nx; v[1] = v[1] + dv * ny;
                    T rc = R - 0.5 * c.d_plus;
                    T rref = 2.0 * rc - rnew;
                    pos[0] = nx * rref; pos[1] = ny * rref;
                }
            }
            T wn = w[i] * (1.0 - logistic(-gap / cfg.smooth_eps) * pstick);
            if (counted) { num[ci] = num[ci] + (w[i] - wn); den[ci] = den[ci] + w[i]; }
            w[i] = wn;
        } else {
            if (counted) nalive[ci] += 1;
            if (val(gap) <= 0) {
                bool stick = true;
                if (cfg.mode == 1) {
                    // Bons et al. rebound (Sec. 4.3): CoR_n = sqrt(sy^2/(rho_p E) - 2 A_cont gc / m) / V_n1,
                    // sy = sigma_y0 (1 - theta), gc = A / (24 pi delta_c^2), A_cont = pi d^2 / 4.
                    const OrcPhys& p = *rn.p;
                    T sy = p.sigma_y0 * (1.0 - theta);
                    T gc = zeta * p.hamaker0 / (24.0 * M_PI * p.delta_c * p.delta_c);
                    double acont = M_PI * c.d * c.d / 4.0;
                    T arg = sy * sy / (p.rho_p * p.young) - 2.0 * acont * gc / c.mass;
                    if (val(arg) > 0) {
                        stick = false;
                        T nx = pos[0] / rnew, ny = pos[1] / rnew;
                        T vn1 = v[0] * nx + v[1] * ny;               // outward normal velocity (wall units)
                        T vn1_si = vn1 * rn.un.ustar;
                        T cor(1.0);
                        if (val(vn1_si) > 0) cor = vmin(T(1.0), sqrt(arg) / vn1_si);
                        T vabs = val(vn1) >= 0 ? vn1 : -vn1;
                        T dv = -cor * vabs - vn1;                    // new normal velocity minus old
                        v[0] = v[0] + dv * nx; v[1] = v[1] + dv * ny;
                        T rc = R - 0.5 * c.d_plus;
                        T rref = 2.0 * rc - rnew;                    // mirror into the pipe
                        pos[0] = nx * rref; pos[1] = ny * rref;
                    }
                }
                if (stick) { alive[i] = 0; if (counted) ndep[ci] += 1; }
            }
        }
        x[i] = pos[0]; y[i] = pos[1]; z[i] = pos[2];
        vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
    }
}

// Coulomb contact distance (reading c1): contact_scale x the largest class diameter.
static double contact_distance(const OrcPhys& p, const std::vector<ClassProps>& cp) {
    double m = 0;
    for (auto& c : cp) m = std::max(m, c.d_plus);
    return p.contact_scale * m;
}

extern "C" {

// Advance every sample n_steps steps from global step index step0, in place.
// Tallies (per sample and class, [S][C]) are accumulated, not overwritten.
int orc_run(const OrcPhys* p, const OrcField* f, const double* grid, const OrcCfg* cfg,
            int n_classes, const double* st_plus, int n_samples, const int64_t* offset,
            const double* params, int64_t step0, int64_t n_steps,
            double* x, double* y, double* z, double* vx, double* vy, double* vz, const double* q,
            int32_t* alive, const int32_t* cls, int64_t* ndep, int64_t* nalive) {
    if (cfg->smooth_eps > 0) return -1;
    Run<double> rn;
    rn.p = p; rn.f = f; rn.grid = grid; rn.cfg = cfg; rn.un = units(*p);
    for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
    rn.contact = contact_distance(*rn.p, rn.cp);
    for (int s = 0; s < n_samples; ++s) {
        int64_t o = offset[s];
        int n = (int)(offset[s + 1] - o);
        SampleParams sp{params[3 * s], params[3 * s + 1], params[3 * s + 2]};
        for (int64_t st = step0; st < step0 + n_steps; ++st) {
            bool counted = st >= cfg->window_start;
            step_sample<double>(rn, n, x + o, y + o, z + o, vx + o, vy + o, vz + o, q + o, nullptr,
                                alive + o, cls + o, sp.zeta, sp.theta, counted,
                                ndep + (size_t)s * n_classes, nalive + (size_t)s * n_classes, nullptr, nullptr);
        }
    }
    return 0;
}

// V_dep+ = (R+/2) N_dep / integral of N_alive dt+ (Sec. 2.1 definition with
// J_w = dN_dep/dt m_p / (2 pi R L) and rho_pm = N m_p / (pi R^2 L)).
void orc_vdep(int n, const int64_t* ndep, const int64_t* nalive, double dt, double r_plus, double* out) {
    for (int k = 0; k < n; ++k)
        out[k] = nalive[k] > 0 ? 0.5 * r_plus * (double)ndep[k] / ((double)nalive[k] * dt) : 0.0;
}

// Smoothed deposition functional of one or more samples (no removal):
// w^{n+1} = w^n (1 - logistic(-gap^{n+1}/eps)),
// J_eps = (R+/2) sum_n sum_p (w^n - w^{n+1}) / (dt sum_n sum_p w^n), per class.
// With want_grad, the forward-mode dual numbers give dJ/d(xi, zeta, theta).
// Rebound mode (mode 1) multiplies the weight loss by the smoothed sticking
// probability sigma(-arg/stick_eps) and reflects the rest of the particle.
int orc_smooth_run(const OrcPhys* p, const OrcField* f, const double* grid, const OrcCfg* cfg,
                   int n_classes, const double* st_plus, int n_samples, const int64_t* offset,
                   const double* params, int64_t n_steps,
                   const double* x0, const double* y0, const double* z0, const double* qhat /*charge per unit xi*/,
                   const int32_t* cls, const double* v0 /*[N][3] or NULL: at rest*/,
                   const double* w0 /*[N] or NULL: all 1*/, int want_grad, double* J /*[S][C]*/,
                   double* dJ /*[S][C][3]*/) {
    if (cfg->smooth_eps <= 0 || (cfg->mode == 1 && !(cfg->stick_eps > 0))) return -1;
    if (cfg->forces & (F_COLLIDE | F_VDWPP)) return -1;     // contact forces: plain runs only
    for (int s = 0; s < n_samples; ++s) {
        int64_t o = offset[s];
        int n = (int)(offset[s + 1] - o);
        SampleParams sp{params[3 * s], params[3 * s + 1], params[3 * s + 2]};
        if (want_grad) {
            Run<Dual> rn;
            rn.p = p; rn.f = f; rn.grid = grid; rn.cfg = cfg; rn.un = units(*p);
            for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
            rn.contact = contact_distance(*rn.p, rn.cp);
            std::vector<Dual> x(n), y(n), z(n), vx(n), vy(n), vz(n), q(n), w(n);
            std::vector<int32_t> alive(n, 1);
            Dual xi(sp.xi), zeta(sp.zeta), theta(sp.theta);
            xi.d[0] = 1; zeta.d[1] = 1; theta.d[2] = 1;
            for (int i = 0; i < n; ++i) {
                x[i] = Dual(x0[o + i]); y[i] = Dual(y0[o + i]); z[i] = Dual(z0[o + i]);
                vx[i] = Dual(v0 ? v0[3 * (o + i)] : 0.0);
                vy[i] = Dual(v0 ? v0[3 * (o + i) + 1] : 0.0);
                vz[i] = Dual(v0 ? v0[3 * (o + i) + 2] : 0.0);
                q[i] = xi * qhat[o + i]; w[i] = Dual(w0 ? w0[o + i] : 1.0);
            }
            std::vector<Dual> num(n_classes, Dual(0.0)), den(n_classes, Dual(0.0));
            for (int64_t st = 0; st < n_steps; ++st)
                step_sample<Dual>(rn, n, x.data(), y.data(), z.data(), vx.data(), vy.data(), vz.data(), q.data(),
                                  w.data(), alive.data(), cls + o, zeta, theta, st >= cfg->window_start,
                                  nullptr, nullptr, num.data(), den.data());
            for (int c = 0; c < n_classes; ++c) {
                Dual j = den[c].v > 0 ? 0.5 * f->r_plus * num[c] / (den[c] * cfg->dt) : Dual(0.0);
                J[(size_t)s * n_classes + c] = j.v;
                for (int k = 0; k < 3; ++k) dJ[((size_t)s * n_classes + c) * 3 + k] = j.d[k];
            }
        } else {
            Run<double> rn;
            rn.p = p; rn.f = f; rn.grid = grid; rn.cfg = cfg; rn.un = units(*p);
            for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
            rn.contact = contact_distance(*rn.p, rn.cp);
            std::vector<double> x(x0 + o, x0 + o + n), y(y0 + o, y0 + o + n), z(z0 + o, z0 + o + n);
            std::vector<double> vx(n, 0.0), vy(n, 0.0), vz(n, 0.0), q(n), w(n, 1.0);
            std::vector<int32_t> alive(n, 1);
            for (int i = 0; i < n; ++i) {
                q[i] = sp.xi * qhat[o + i];
                if (v0) { vx[i] = v0[3 * (o + i)]; vy[i] = v0[3 * (o + i) + 1]; vz[i] = v0[3 * (o + i) + 2]; }
                if (w0) w[i] = w0[o + i];
            }
            std::vector<double> num(n_classes, 0.0), den(n_classes, 0.0);
            for (int64_t st = 0; st < n_steps; ++st)
                step_sample<double>(rn, n, x.data(), y.data(), z.data(), vx.data(), vy.data(), vz.data(), q.data(),
                                    w.data(), alive.data(), cls + o, sp.zeta, sp.theta, st >= cfg->window_start,
                                    nullptr, nullptr, num.data(), den.data());
            for (int c = 0; c < n_classes; ++c)
                J[(size_t)s * n_classes + c] = den[c] > 0 ? 0.5 * f->r_plus * num[c] / (den[c] * cfg->dt) : 0.0;
        }
    }
    return 0;
}

// Coulomb acceleration only (wall units), for brute-force and invariance pins.
void orc_coulomb_accel(const OrcPhys* p, const OrcField* f, int n_classes, const double* st_plus, int n,
                       const double* x, const double* y, const double* z, const double* q, const int32_t* cls,
                       const int32_t* alive, double* a /*[n][3]*/) {
    OrcCfg cfg; std::memset(&cfg, 0, sizeof(cfg)); cfg.forces = F_COUL; cfg.dt = 0.0;
    Run<double> rn;
    rn.p = p; rn.f = f; rn.grid = nullptr; rn.cfg = &cfg; rn.un = units(*p);
    for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
    rn.contact = contact_distance(*rn.p, rn.cp);
    const double L = f->l_plus;
    for (int i = 0; i < n; ++i) {
        double s[3] = {0, 0, 0};
        if (alive[i]) {
            for (int j = 0; j < n; ++j) {
                if (j == i || !alive[j]) continue;
                double d[3] = {x[i] - x[j], y[i] - y[j], z[i] - z[j]};
                d[2] -= L * std::rint(d[2] / L);
                double rr = std::max(std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), rn.contact);
                for (int k = 0; k < 3; ++k) s[k] += q[j] * d[k] / (rr * rr * rr);
            }
        }
        const ClassProps& c = rn.cp[cls[i]];
        double coef = p->qmax_coef * p->qmax_coef / (4.0 * M_PI * p->eps0) / c.mass / (rn.un.ell * rn.un.ell) * rn.un.acc;
        for (int k = 0; k < 3; ++k) a[3 * i + k] = q[i] * coef * s[k];
    }
}

// Coulomb sums s_i = sum_j q_j d / max(|d|, contact)^3 over every periodic image of particle j
// along z (d = x_i - x_j - k L e_z, |k| <= n_img), j != i, live particles: the electrostatics the
// paper's P3M approximates (periodic pipe, no images across the wall).  The images beyond n_img
// are added in their far-field form: pairs (k, -k) contribute 2 d_xy / (kL)^3 across and
// -4 d_z / (kL)^3 along the axis, summed with sum_{k > K} k^-3 ~ 1 / (2 (K + 1/2)^2).
void orc_coulomb_periodic(int n, const double* x, const double* y, const double* z, const double* q,
                          const int32_t* alive, double L, double contact, int n_img, double* s /*[n][3]*/) {
    const double tail = 1.0 / (2.0 * (n_img + 0.5) * (n_img + 0.5)) / (L * L * L);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
        double acc[3] = {0, 0, 0};
        if (alive[i]) {
            for (int j = 0; j < n; ++j) {
                if (j == i || !alive[j]) continue;
                const double dx = x[i] - x[j], dy = y[i] - y[j];
                const double dz0 = z[i] - z[j];
                double px = 0, py = 0, pz = 0;
                for (int k = -n_img; k <= n_img; ++k) {
                    const double dz = dz0 - k * L;
                    const double r = std::max(std::sqrt(dx * dx + dy * dy + dz * dz), contact);
                    const double w = 1.0 / (r * r * r);
                    px += w * dx; py += w * dy; pz += w * dz;
                }
                px += 2.0 * dx * tail; py += 2.0 * dy * tail; pz += -4.0 * dz0 * tail;
                acc[0] += q[j] * px; acc[1] += q[j] * py; acc[2] += q[j] * pz;
            }
        }
        for (int k = 0; k < 3; ++k) s[3 * i + k] = acc[k];
    }
}

// One step of every sample with the Coulomb sums given (ext [N][3], e.g. from a P3M solve of
// the current state) instead of the all-pairs loop; otherwise as orc_run.
int orc_run_ext(const OrcPhys* p, const OrcField* f, const double* grid, const OrcCfg* cfg,
                int n_classes, const double* st_plus, int n_samples, const int64_t* offset,
                const double* params, int64_t step0, const double* ext,
                double* x, double* y, double* z, double* vx, double* vy, double* vz, const double* q,
                int32_t* alive, const int32_t* cls, int64_t* ndep, int64_t* nalive) {
    if (cfg->smooth_eps > 0) return -1;
    Run<double> rn;
    rn.p = p; rn.f = f; rn.grid = grid; rn.cfg = cfg; rn.un = units(*p);
    for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
    rn.contact = contact_distance(*rn.p, rn.cp);
    for (int s = 0; s < n_samples; ++s) {
        int64_t o = offset[s];
        int n = (int)(offset[s + 1] - o);
        SampleParams sp{params[3 * s], params[3 * s + 1], params[3 * s + 2]};
        rn.ext = ext + 3 * o;
        step_sample<double>(rn, n, x + o, y + o, z + o, vx + o, vy + o, vz + o, q + o, nullptr,
                            alive + o, cls + o, sp.zeta, sp.theta, step0 >= cfg->window_start,
                            ndep + (size_t)s * n_classes, nalive + (size_t)s * n_classes, nullptr, nullptr);
    }
    return 0;
}

// Non-Coulomb, non-drag acceleration (gravity + image + vdW) at given points.
void orc_wall_accel(const OrcPhys* p, const OrcField* f, const OrcCfg* cfg, int n_classes, const double* st_plus,
                    int n, const double* x, const double* y, const double* q, const int32_t* cls, double zeta,
                    double* a) {
    Run<double> rn;
    rn.p = p; rn.f = f; rn.grid = nullptr; rn.cfg = cfg; rn.un = units(*p);
    for (int c = 0; c < n_classes; ++c) rn.cp.push_back(class_props(*p, st_plus[c]));
    rn.contact = contact_distance(*rn.p, rn.cp);
    for (int i = 0; i < n; ++i) {
        double acc[3];
        wall_and_body<double>(rn, rn.cp[cls[i]], x[i], y[i], q[i], zeta, acc);
        for (int k = 0; k < 3; ++k) a[3 * i + k] = acc[k];
    }
}

// Normal coefficient of restitution of the rebound model (Sec. 4.3), for
// given zeta, theta and impact velocity (m/s).  Returns 0 for sticking.
double orc_cor(const OrcPhys* p, double st_plus, double zeta, double theta, double vn1) {
    ClassProps c = class_props(*p, st_plus);
    double sy = p->sigma_y0 * (1.0 - theta);
    double gc = zeta * p->hamaker0 / (24.0 * M_PI * p->delta_c * p->delta_c);
    double arg = sy * sy / (p->rho_p * p->young) - 2.0 * (M_PI * c.d * c.d / 4.0) * gc / c.mass;
    if (arg <= 0) return 0.0;
    if (vn1 <= 0) return 1.0;
    return std::min(1.0, std::sqrt(arg) / vn1);
}

// Bootstrap resampling of group position t in replicate b: Philox4x32-10 counter
// (t, b, 0, 2), key = seed; position t in the nesting block [m_{l-1}, m_l)
// draws m_{l-1} + (word0 (m_l - m_{l-1})) >> 32.
void orc_boot_indices(uint64_t seed, uint32_t b, int k, const int64_t* m, int64_t* out) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t t = 0; t < m[k - 1]; ++t) {
        int l = 0;
        while (t >= m[l]) ++l;
        int64_t lo = l > 0 ? m[l - 1] : 0;
        uint32_t c[4] = {(uint32_t)t, b, 0u, 2u}, w[4];
        philox4x32_10(c, key, w);
        out[t] = lo + (int64_t)(((uint64_t)w[0] * (uint64_t)(m[l] - lo)) >> 32);
    }
}

// Capture efficiency factor of Sec. 4.3: CE = (4 L / D) (u* / U_b) V_dep+|stick.
double orc_capture_factor(const OrcPhys* p, const OrcField* f) {
    Units u = units(*p);
    return 4.0 * (f->l_plus / (2.0 * f->r_plus)) * (u.ustar / p->u_bulk);
}

// Philox known-answer access for the pin test.
void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
