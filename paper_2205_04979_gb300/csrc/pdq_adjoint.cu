// pdq_adjoint.cu -- hand-written reverse-mode adjoint of the particle step.
//
// Functional (a smoothed form of V_dep+, Sec. 2.1): particles are never
// removed; each carries a weight w, updated after the step as
//   w' = w (1 - sigma(-gap'/eps)),  sigma(a) = 1 / (1 + exp(-a)),
// with gap' = R - r' - d/2 the wall gap after the step.  Over the counted
// steps, per (sample, class):
//   num = sum_n sum_p (w_n - w_{n+1}),  den = sum_n sum_p w_n,
//   J = (R+/2) num / (dt+ den),
// which tends to the all-stick V_dep+ as eps -> 0.  The Coulomb sum uses the
// weighted charges w_j q_j.  Gradients are taken with respect to the
// per-sample inputs (xi, zeta, theta); theta only enters the rebound model, so
// under all-stick its derivative is exactly zero.
//
// Schedule: one forward sweep stores a checkpoint every K steps and the
// functional; every backward sweep (one per cotangent vector) recomputes each
// segment of K steps from its checkpoint, storing each state and its raw
// Coulomb sum S_i = sum_j w_j q_j G(x_i - x_j), then walks the segment
// backwards with two kernels per step: the local adjoint (weights, wall
// sigmoid, exponential integrator, drag, interpolation gradient, image charge,
// van der Waals) and the all-pairs adjoint of the Coulomb sum.
//
// Storage is FP64 in both precisions; PDQ_MIXED computes the pair sums, the
// interpolation, drag and integrator in FP32 like the forward step, the
// wall-normal position, wall forces and weights in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "pdq_common.cuh"
#include "pdq_device.cuh"
#include "pdq_newton.cuh"

namespace pdq {

struct Slot {   // one time level, SoA (FP64)
    double *x, *y, *z, *vx, *vy, *vz, *w, *sx, *sy, *sz;
};

struct AdjArgs {
    StepConst K;
    const int64_t* offset;
    int32_t S, C;
    const int32_t* cls;
    const double* qhat;                 // charge per unit xi
    const pdq_sample_params* params;
    double eps;                         // width of the smoothed wall indicator (wall units)
    double eps_stick;                   // width of the smoothed sticking probability (m^2/s^2)
    int32_t mode;                       // PDQ_STICK or PDQ_REBOUND
    Slot in, out;                       // state n (S_n written here) and state n+1
    int64_t step;
    int32_t tally;
    double *num, *den;                  // [S][C]
    double *xb, *yb, *zb, *vxb, *vyb, *vzb, *wb, *qb;   // cotangents [N]
    double *cx, *cy, *cz;               // c = coul q abar [N]
    const double *nbar, *dbar;          // cotangents of num and den [S][C]
    double* pbar;                       // [S][3]
    float4* acc4;                       // MIXED Newton-pair sums [N]: forward Coulomb sums (x, y, z),
                                        // reverse pair-VJP sums (x-bar x, y, z; charge term w)
    // seeding
    uint2 key;
    double sigma, neg_frac;
};

__device__ __forceinline__ double logistic(double a) {
    if (a >= 0.0) return 1.0 / (1.0 + exp(-a));
    const double e = exp(a);   // no overflow for large -a
    return e / (1.0 + e);
}

// Everything the local part of a step computes from (x, v, w) and the Coulomb
// sum S, in the forward step's precisions; GRAD adds the interpolation Jacobian
// and the derivatives the adjoint needs.
template <class T>
struct Local {
    double x, y, r, nx, ny;
    T z, v[3];
    double w, q;
    // wall: a_wall = A (nx, ny), A = A_img + A_vdw; dA/dr and the vdW factor per unit zeta
    double A, dAdr, img_q, vdw_z;
    T a[3];
    T u[3], du[3][3];   // du[k][m] = d u_k / d x_m
    T rel[3], relm, Re, lam;
    T zz, e, p1, p2, dp1, dp2;
    T F[3];
    double xn, yn;                      // after integration (before a rebound)
    T zn, vn[3];
    double rn, gap, Sg, wn;
    // smoothed rebound: sticking probability, and the reflection of the rest
    double arg, pst, dv, nxa, nya, vnrm;
    int rcase;                          // 0 CoR = 0, 1 inward (no change), 2 CoR capped at 1, 3 CoR < 1
    bool reflect;
    double xr, yr, vr[3];               // final state (after a rebound)
};

template <class T, class T4, bool GRAD>
__device__ __forceinline__ void interp_jac(const StepConst& K, double r, double x, double y, T z, T u[3], T du[3][3]) {
    // value: the same routine as the forward step
    interp<T, T4>(K, (T)r, (T)x, (T)y, z, u);
    if (!GRAD) return;
    if (!(isfinite(r) && isfinite(x) && isfinite(y) && isfinite((double)z))) {
        for (int k = 0; k < 3; ++k) du[k][0] = du[k][1] = du[k][2] = (T)NAN;
        return;
    }
    // derivatives of the trilinear weights in (s(r), theta, z) chained to (x, y, z)
    const GridT<T> G(K);
    const T R = G.R;
    const T rho = fmin((T)r / R, (T)1);
    const T s = atanh_(rho * G.tanh_b) * G.inv_b;
    const T fi = s * (T)(K.n_r - 1);
    int i0 = (int)floor_(fi);
    i0 = i0 < 0 ? 0 : (i0 > K.n_r - 2 ? K.n_r - 2 : i0);
    const T tr = fi - (T)i0;
    T fj = atan2_((T)y, (T)x) * G.th_scale;
    if (fj < (T)0) fj += (T)K.n_th;
    int j0 = (int)floor_(fj);
    const T tt = fj - (T)j0;
    j0 %= K.n_th;
    if (j0 < 0) j0 += K.n_th;
    const int j1 = (j0 + 1 == K.n_th) ? 0 : j0 + 1;
    const T fk = z * G.z_scale;
    int k0 = (int)floor_(fk);
    const T tz = fk - (T)k0;
    k0 %= K.n_z;
    if (k0 < 0) k0 += K.n_z;
    const int k1 = (k0 + 1 == K.n_z) ? 0 : k0 + 1;
    const int64_t nr = K.n_r, plane = (int64_t)K.n_r * K.n_th;
    const int64_t b00 = k0 * plane + j0 * nr + i0, b01 = k0 * plane + j1 * nr + i0;
    const int64_t b10 = k1 * plane + j0 * nr + i0, b11 = k1 * plane + j1 * nr + i0;
    const T4* tag = nullptr;
    const T4 g[8] = {grid_at(K, tag, b00), grid_at(K, tag, b00 + 1), grid_at(K, tag, b01), grid_at(K, tag, b01 + 1),
                     grid_at(K, tag, b10), grid_at(K, tag, b10 + 1), grid_at(K, tag, b11), grid_at(K, tag, b11 + 1)};
    // corner c = (dk, dj, di) with index 4 dk + 2 dj + di
    T dtr[3] = {0, 0, 0}, dtt[3] = {0, 0, 0}, dtz[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = c >> 2;
        const T wr = di ? tr : (T)1 - tr, wt = dj ? tt : (T)1 - tt, wz = dk ? tz : (T)1 - tz;
        const T sr = di ? (T)1 : (T)-1, st = dj ? (T)1 : (T)-1, sz = dk ? (T)1 : (T)-1;
        const T gv[3] = {g[c].x, g[c].y, g[c].z};
        for (int k = 0; k < 3; ++k) {
            dtr[k] += sr * wt * wz * gv[k];
            dtt[k] += wr * st * wz * gv[k];
            dtz[k] += wr * wt * sz * gv[k];
        }
    }
    // d tr / d r, d tt / d(x, y), d tz / dz
    T dsdr = (T)0;
    if ((T)r < R) {
        const T a = rho * G.tanh_b;
        dsdr = G.tanh_b * G.inv_b / (R * ((T)1 - a * a));
    }
    const T dtr_dr = dsdr * (T)(K.n_r - 1);
    T drdx = 0, drdy = 0, dthdx = 0, dthdy = 0;
    if (r > 1e-12) {
        drdx = (T)(x / r);
        drdy = (T)(y / r);
        const T k2 = G.th_scale / (T)(r * r);
        dthdx = -(T)y * k2;
        dthdy = (T)x * k2;
    }
    const T dtz_dz = G.z_scale;
    for (int k = 0; k < 3; ++k) {
        du[k][0] = dtr[k] * dtr_dr * drdx + dtt[k] * dthdx;
        du[k][1] = dtr[k] * dtr_dr * drdy + dtt[k] * dthdy;
        du[k][2] = dtz[k] * dtz_dz;
    }
}

// phi1' = sum_k (k+1) z^k/(k+2)!, phi2' = sum_k (k+1) z^k/(k+3)! near 0; closed forms elsewhere.
__device__ __forceinline__ void dphi12(double z, double p1, double p2, double e, double& d1, double& d2) {
    if (fabs(z) < 0.05) {
        double a = 0.0, b = 0.0, f2 = 1.0;   // f2 tracks (k+2)! as k rises
        double zk = 1.0;
        for (int k = 0; k <= 10; ++k) {
            f2 *= (k + 2);                    // (k+2)!
            a += (k + 1) * zk / f2;
            b += (k + 1) * zk / (f2 * (k + 3));
            zk *= z;
        }
        d1 = a;
        d2 = b;
        return;
    }
    d1 = (e - p1) / z;
    d2 = (p1 - 2.0 * p2) / z;
}
__device__ __forceinline__ void dphi12(float z, float p1, float p2, float e, float& d1, float& d2) {
    if (fabsf(z) < 0.1f) {
        float a = 0.f, b = 0.f, f2 = 1.f, zk = 1.f;
        for (int k = 0; k <= 8; ++k) {
            f2 *= (float)(k + 2);
            a += (float)(k + 1) * zk / f2;
            b += (float)(k + 1) * zk / (f2 * (float)(k + 3));
            zk *= z;
        }
        d1 = a;
        d2 = b;
        return;
    }
    d1 = (e - p1) / z;
    d2 = (p1 - 2.f * p2) / z;
}

template <int P, bool GRAD>
__device__ __forceinline__ void local_step(const AdjArgs& A, const ClassK& c, const pdq_sample_params& sp,
                                           Local<typename Real<P>::T>& L, typename Real<P>::T sx,
                                           typename Real<P>::T sy, typename Real<P>::T sz) {
    typedef typename Real<P>::T T;
    typedef typename Real<P>::T4 T4;
    const StepConst& K = A.K;
    for (int k = 0; k < 3; ++k) L.a[k] = (T)0;
    if (K.forces & PDQ_F_COULOMB) {
        const T kq = (P == PDQ_FP64 ? (T)c.coul : (T)c.coul_f) * (T)L.q;
        L.a[0] = kq * sx; L.a[1] = kq * sy; L.a[2] = kq * sz;
    }
    if (K.forces & PDQ_F_GRAVITY) {
        if constexpr (P == PDQ_FP64) { L.a[0] += K.grav[0]; L.a[1] += K.grav[1]; L.a[2] += K.grav[2]; }
        else { L.a[0] += K.gravf[0]; L.a[1] += K.gravf[1]; L.a[2] += K.gravf[2]; }
    }
    L.r = sqrt(L.x * L.x + L.y * L.y);
    L.A = 0.0; L.dAdr = 0.0; L.img_q = 0.0; L.vdw_z = 0.0;
    L.nx = 0.0; L.ny = 0.0;
    if (L.r > 0.0 && (K.forces & (PDQ_F_IMAGE | PDQ_F_VDW))) {
        L.nx = L.x / L.r;
        L.ny = L.y / L.r;
        if (K.forces & PDQ_F_IMAGE) {
            const double yw = fmax(K.R - L.r, c.half_d);
            const double ai = 0.25 * c.coul * L.q * L.q / (yw * yw);
            L.A += ai;
            L.img_q = 0.5 * c.coul * L.q / (yw * yw);                 // d A_img / d q
            if (K.R - L.r > c.half_d) L.dAdr += 2.0 * ai / yw;         // d/dr of 1/(R-r)^2
        }
        if (K.forces & PDQ_F_VDW) {
            const double gap = (K.R - L.r - c.half_d) * K.ell;
            if (gap <= 0.25 * c.d_m) {
                const double dl = fmax(gap, K.delta_min);
                const double d = c.d_m, d2 = d * d, d6 = d2 * d2 * d2;
                const double e1 = 2.0 * d + dl, e2 = d + dl;
                const double F = d6 / (dl * dl * e1 * e1 * e2 * e2 * e2);
                L.vdw_z = c.vdw * F;
                L.A += sp.zeta * L.vdw_z;
                if (gap > K.delta_min) {
                    const double dlogF = -2.0 / dl - 2.0 / e1 - 3.0 / e2;   // d ln F / d delta
                    L.dAdr += sp.zeta * L.vdw_z * dlogF * (-K.ell);
                }
            }
        }
        L.a[0] += (T)(L.A * L.nx);
        L.a[1] += (T)(L.A * L.ny);
    }
    for (int k = 0; k < 3; ++k) L.u[k] = (T)0;
    L.lam = (T)0;
    L.Re = (T)0;
    L.relm = (T)0;
    if (K.forces & PDQ_F_DRAG) {
        interp_jac<T, T4, GRAD>(K, L.r, L.x, L.y, L.z, L.u, L.du);
        for (int k = 0; k < 3; ++k) L.rel[k] = L.u[k] - L.v[k];
        L.relm = sqrt_(L.rel[0] * L.rel[0] + L.rel[1] * L.rel[1] + L.rel[2] * L.rel[2]);
        L.Re = L.relm * (P == PDQ_FP64 ? (T)c.d_plus : (T)c.d_plus_f);
        const T fd = (T)1 + (T)0.15 * (L.Re > (T)0 ? pow_(L.Re, (T)0.687) : (T)0);
        L.lam = fd * (P == PDQ_FP64 ? (T)(1.0 / c.tau) : (T)c.inv_tau_f);
    }
    const T h = P == PDQ_FP64 ? (T)K.dt : (T)K.dtf;
    L.zz = -L.lam * h;
    phi12(L.zz, L.p1, L.p2);
    L.e = exp_(L.zz);
    if (GRAD) dphi12(L.zz, L.p1, L.p2, L.e, L.dp1, L.dp2);
    T dxv[3];
    for (int k = 0; k < 3; ++k) {
        L.F[k] = L.lam * L.u[k] + L.a[k];
        dxv[k] = L.v[k] * h * L.p1 + L.F[k] * (h * h) * L.p2;
        L.vn[k] = L.v[k] * L.e + L.F[k] * h * L.p1;
    }
    L.xn = L.x + (double)dxv[0];
    L.yn = L.y + (double)dxv[1];
    T zn = L.z + dxv[2];
    const T Lz = P == PDQ_FP64 ? (T)K.L : (T)K.Lf, invLz = P == PDQ_FP64 ? (T)K.invL : (T)K.invLf;
    zn -= Lz * floor_(zn * invLz);
    if (zn >= Lz) zn -= Lz;
    if (zn < (T)0) zn = (T)0;
    L.zn = zn;
    L.rn = sqrt(L.xn * L.xn + L.yn * L.yn);
    L.gap = K.R - L.rn - c.half_d;
    L.Sg = logistic(-L.gap / A.eps);
    L.pst = 1.0;
    L.reflect = false;
    L.rcase = 0;
    L.dv = 0.0;
    L.xr = L.xn; L.yr = L.yn;
    for (int k = 0; k < 3; ++k) L.vr[k] = (double)L.vn[k];
    if (A.mode == PDQ_REBOUND) {
        // Bons et al. (Sec. 4.3): sticking probability sigma(-arg/eps_s) with
        // arg = sigma_y0^2 (1 - theta)^2 / (rho_p E) - 2 A_cont gamma_c / m; the rest rebounds
        const double one_m = 1.0 - sp.theta;
        L.arg = K.elastic0 * one_m * one_m - sp.zeta * c.stick;
        L.pst = logistic(-L.arg / A.eps_stick);
        if (L.gap <= 0.0 && L.rn > 0.0) {
            L.reflect = true;
            L.nxa = L.xn / L.rn;
            L.nya = L.yn / L.rn;
            L.vnrm = (double)L.vn[0] * L.nxa + (double)L.vn[1] * L.nya;
            double cor = 0.0;
            L.rcase = 0;
            if (L.arg > 0.0) {
                cor = 1.0;
                L.rcase = 1;
                const double vsi = L.vnrm * K.ustar;
                if (vsi > 0.0) {
                    const double ratio = sqrt(L.arg) / vsi;
                    if (ratio >= 1.0) { L.rcase = 2; } else { cor = ratio; L.rcase = 3; }
                }
            }
            L.dv = -cor * fabs(L.vnrm) - L.vnrm;
            L.vr[0] = (double)L.vn[0] + L.dv * L.nxa;
            L.vr[1] = (double)L.vn[1] + L.dv * L.nya;
            const double rref = 2.0 * (K.R - c.half_d) - L.rn;
            L.xr = L.nxa * rref;
            L.yr = L.nya * rref;
        }
    }
    L.wn = L.w * (1.0 - L.Sg * L.pst);
}

// Sum over a warp of v for the lanes whose class is c, for every class; lane 0 adds to dst[c].
__device__ __forceinline__ void warp_class_add(double v, int cls, int C, double* dst) {
    for (int c = 0; c < C; ++c) {
        double t = cls == c ? v : 0.0;
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(dst + c, t);
    }
}
__device__ __forceinline__ void warp_add(double v, double* dst) {
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

// ---------------------------------------------------------------------------
// Kernels.  Grid (tiles, samples), NT threads, one particle per thread.
// ---------------------------------------------------------------------------
__global__ void k_adj_seed(const AdjArgs A) {
    const int s = blockIdx.y;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = o + i;
    const int c = (int)((uint32_t)i % (uint32_t)A.C);
    double x, y, z, qh;
    seed_particle(A.key, (uint32_t)i, A.sigma, A.neg_frac, A.K.R, A.K.L, A.K.cls[c].half_d, A.K.cls[c].qfac, x, y,
                  z, qh);
    A.out.x[g] = x; A.out.y[g] = y; A.out.z[g] = z;
    A.out.vx[g] = 0.0; A.out.vy[g] = 0.0; A.out.vz[g] = 0.0; A.out.w[g] = 1.0;
    ((int32_t*)A.cls)[g] = c;
    ((double*)A.qhat)[g] = qh;
}

// Initial smoothed state from a caller's particle state (its current half): positions and
// velocities, weight = the alive flag (a deposited particle keeps weight 0), charge per unit xi
// = q_eff / xi_s (the host has checked xi_s != 0), class from the tag.  Slots past count[s]
// become weightless, uncharged particles at rest on the axis; they add nothing to J or to any
// Coulomb sum.
template <int P>
__global__ void k_adj_load(const AdjArgs A, const int32_t* __restrict__ count, const void* __restrict__ pos,
                           const void* __restrict__ vel, const double2* __restrict__ xy,
                           const int2* __restrict__ tag) {
    const int s = blockIdx.y;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = o + i;
    double x = 0.0, y = 0.0, z = 0.0, vx = 0.0, vy = 0.0, vz = 0.0, w = 0.0, qe = 0.0;
    int c = 0;
    if (i < count[s]) {
        if constexpr (P == PDQ_FP64) {
            const double4_32a pp = ((const double4_32a*)pos)[g], vv = ((const double4_32a*)vel)[g];
            x = pp.x; y = pp.y; z = pp.z; qe = pp.w;
            vx = vv.x; vy = vv.y; vz = vv.z; w = vv.w;
        } else {
            const double2 q2 = xy[g];
            const float4 pp = ((const float4*)pos)[g], vv = ((const float4*)vel)[g];
            x = q2.x; y = q2.y; z = (double)pp.z; qe = (double)pp.w;
            vx = (double)vv.x; vy = (double)vv.y; vz = (double)vv.z; w = (double)vv.w;
        }
        c = min(max(tag[g].y, 0), A.C - 1);   // the class table has C entries
    }
    A.out.x[g] = x; A.out.y[g] = y; A.out.z[g] = z;
    A.out.vx[g] = vx; A.out.vy[g] = vy; A.out.vz[g] = vz; A.out.w[g] = w;
    ((int32_t*)A.cls)[g] = c;
    ((double*)A.qhat)[g] = qe / A.params[s].xi;
}

// z-binning of the adjoint state at a checkpoint: one CTA per sample copies the state slot
// `src` (and the per-particle qhat, class) into `dst` grouped by 256 bins of z, stable inside
// a bin (histogram, bin bases, chunks ranked with __match_any_sync), and records
// perm[new] = old index within the sample.  No particle is removed in the smoothed
// functional, so this is a permutation; the reverse sweep undoes it on the cotangents.
constexpr int kAdjBins = 256;
__global__ void __launch_bounds__(1024) k_adj_sort(const int64_t* __restrict__ offset, Slot src,
                                                   const double* __restrict__ qh_in, const int32_t* __restrict__ cl_in,
                                                   Slot dst, double* __restrict__ qh_out, int32_t* __restrict__ cl_out,
                                                   int32_t* __restrict__ perm, float bins_per_length) {
    __shared__ int base[kAdjBins];
    __shared__ int running[kAdjBins];
    __shared__ int wcnt[32][kAdjBins];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = offset[s];
    const int n = (int)(offset[s + 1] - o);
    auto bin_of = [&](double z) -> int {
        const float zb = (float)z * bins_per_length;
        return isfinite(zb) ? min(kAdjBins - 1, max(0, (int)zb)) : 0;
    };
    for (int b = tid; b < kAdjBins; b += blockDim.x) { base[b] = 0; running[b] = 0; }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) atomicAdd(&base[bin_of(src.z[o + i])], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int b = 0; b < kAdjBins; ++b) { const int h = base[b]; base[b] = acc; acc += h; }
    }
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        for (int q = tid; q < 32 * kAdjBins; q += blockDim.x) (&wcnt[0][0])[q] = 0;
        const int i = c0 + tid;
        const int b = i < n ? bin_of(src.z[o + i]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        __syncthreads();
        if (b >= 0 && rank == 0) wcnt[warp][b] = __popc(peers);
        __syncthreads();
        if (tid < kAdjBins) {
            int acc = running[tid];
            for (int q = 0; q < 32; ++q) { const int cc = wcnt[q][tid]; wcnt[q][tid] = acc; acc += cc; }
            running[tid] = acc;
        }
        __syncthreads();
        if (b >= 0) {
            const int64_t g = o + i, d = o + base[b] + wcnt[warp][b] + rank;
            dst.x[d] = src.x[g]; dst.y[d] = src.y[g]; dst.z[d] = src.z[g];
            dst.vx[d] = src.vx[g]; dst.vy[d] = src.vy[g]; dst.vz[d] = src.vz[g]; dst.w[d] = src.w[g];
            qh_out[d] = qh_in[g];
            cl_out[d] = cl_in[g];
            perm[d] = i;
        }
        __syncthreads();
    }
}

// Cotangents of a binned state back to the order before the binning: out[o + perm[i]] = in[o + i].
__global__ void k_adj_unperm(const int64_t* __restrict__ offset, const int32_t* __restrict__ perm,
                             const double* __restrict__ in, double* __restrict__ out) {
    const int s = blockIdx.y;
    const int64_t o = offset[s], n = offset[s + 1] - o;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[o + perm[o + i]] = in[o + i];
}

// z range (min, max) over a warp.
__device__ __forceinline__ float2 warp_range(float lo, float hi) {
    for (int d = 16; d > 0; d >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    return make_float2(lo, hi);
}

// Particles per thread of k_adj_forward and k_adj_pairs: MIXED 4 (their local parts only: its
// pair sums and pair VJP are the Newton-pair kernels below), FP64 2 for ILP in the pair loops.
template <int P> __host__ __device__ constexpr int adj_ilp() { return P == PDQ_MIXED ? 4 : 2; }

// SUMS: the Coulomb sums come from A.acc4 (the Newton-pair kernel k_adj_sums_sym) instead of the
// pair loop below.
template <int P, int NT, bool SUMS = false>
__global__ void __launch_bounds__(NT) k_adj_forward(const AdjArgs A) {
    typedef typename Real<P>::T T;
    typedef typename Real<P>::T4 T4;
    constexpr int U = adj_ilp<P>();          // particles per thread (ILP over the shared j-tile)
    __shared__ __align__(32) unsigned char smem_raw[NT * 32];
    T4* sj = reinterpret_cast<T4*>(smem_raw);
    const int s = blockIdx.y, tid = threadIdx.x;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    if ((int64_t)blockIdx.x * NT * U >= n) return;
    const pdq_sample_params sp = A.params[s];
    const StepConst& K = A.K;
    T xi[U], yi[U], zi[U], ax[U], ay[U], az[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
        const bool valid = i < n;
        const int64_t g = o + (valid ? i : 0);
        xi[u] = valid ? (T)A.in.x[g] : (T)0;
        yi[u] = valid ? (T)A.in.y[g] : (T)0;
        zi[u] = valid ? (T)A.in.z[g] : (T)0;
        ax[u] = ay[u] = az[u] = (T)0;
    }
    if constexpr (SUMS) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
            if (i < n) {
                const float4 a = A.acc4[o + i];
                ax[u] = (T)a.x; ay[u] = (T)a.y; az[u] = (T)a.z;
            }
        }
    } else if (P == PDQ_FP64 && (K.forces & PDQ_F_COULOMB)) {
        // (MIXED takes the Coulomb sums from k_adj_sums_sym: SUMS)
        const T L = (T)K.L, invL = (T)K.invL;
        const T c2 = P == PDQ_FP64 ? (T)K.contact2 : (T)K.contact2f;
        for (int64_t j0 = 0; j0 < n; j0 += NT) {
            const int64_t j = j0 + tid;
            T4 p;
            if (j < n) {
                const int64_t gj = o + j;
                p.x = (T)A.in.x[gj]; p.y = (T)A.in.y[gj]; p.z = (T)A.in.z[gj];
                p.w = (T)(A.in.w[gj] * sp.xi * A.qhat[gj]);
            } else {
                p.x = (T)0; p.y = (T)0; p.z = (T)0; p.w = (T)0;
            }
            sj[tid] = p;
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < NT; ++k) {
                const T4 q = sj[k];
#pragma unroll
                for (int u = 0; u < U; ++u) coulomb_pair(xi[u], yi[u], zi[u], q, L, invL, c2, ax[u], ay[u], az[u]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
        const bool valid = i < n;
        int cls = -1;
        double dnum = 0.0, dden = 0.0;
        if (valid) {
            const int64_t g = o + i;
            cls = A.cls[g];
            Local<T> Lc;
            Lc.x = A.in.x[g]; Lc.y = A.in.y[g]; Lc.z = (T)A.in.z[g];
            Lc.v[0] = (T)A.in.vx[g]; Lc.v[1] = (T)A.in.vy[g]; Lc.v[2] = (T)A.in.vz[g];
            Lc.w = A.in.w[g];
            Lc.q = sp.xi * A.qhat[g];
            local_step<P, false>(A, K.cls[cls], sp, Lc, ax[u], ay[u], az[u]);
            A.in.sx[g] = (double)ax[u]; A.in.sy[g] = (double)ay[u]; A.in.sz[g] = (double)az[u];
            A.out.x[g] = Lc.xr; A.out.y[g] = Lc.yr; A.out.z[g] = (double)Lc.zn;
            A.out.vx[g] = (double)(T)Lc.vr[0]; A.out.vy[g] = (double)(T)Lc.vr[1]; A.out.vz[g] = (double)Lc.vn[2];
            A.out.w[g] = Lc.wn;
            dnum = Lc.w - Lc.wn;
            dden = Lc.w;
        }
        if (A.tally && A.step >= K.window_start) {
            warp_class_add(dnum, cls, A.C, A.num + (int64_t)s * A.C);
            warp_class_add(dden, cls, A.C, A.den + (int64_t)s * A.C);
        }
    }
}

// Local adjoint of step n: cotangents of state n+1 (in xb..wb) -> cotangents of
// state n (partial: the Coulomb pair terms follow), c = coul q abar, qbar, zeta-bar.
template <int P>
__global__ void __launch_bounds__(128) k_adj_local(const AdjArgs A) {
    typedef typename Real<P>::T T;
    const int s = blockIdx.y;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    if ((int64_t)blockIdx.x * blockDim.x >= n) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const pdq_sample_params sp = A.params[s];
    const StepConst& K = A.K;
    double zeta_bar = 0.0, theta_bar = 0.0;
    if (valid) {
        const int64_t g = o + i;
        const int cls = A.cls[g];
        const ClassK& c = K.cls[cls];
        Local<T> L;
        L.x = A.in.x[g]; L.y = A.in.y[g]; L.z = (T)A.in.z[g];
        L.v[0] = (T)A.in.vx[g]; L.v[1] = (T)A.in.vy[g]; L.v[2] = (T)A.in.vz[g];
        L.w = A.in.w[g];
        L.q = sp.xi * A.qhat[g];
        const T S3[3] = {(T)A.in.sx[g], (T)A.in.sy[g], (T)A.in.sz[g]};
        local_step<P, true>(A, c, sp, L, S3[0], S3[1], S3[2]);
        const double h = K.dt;
        double xb[3] = {A.xb[g], A.yb[g], A.zb[g]};
        double vb[3] = {A.vxb[g], A.vyb[g], A.vzb[g]};
        double wb_next = A.wb[g];
        // tally of step n: num += w_n - w_{n+1}, den += w_n
        double wbar = 0.0;
        if (A.step >= K.window_start) {
            const double nb = A.nbar[(int64_t)s * A.C + cls], db = A.dbar[(int64_t)s * A.C + cls];
            wbar += nb + db;
            wb_next -= nb;
        }
        // weight update w' = w (1 - Sg pst), Sg = sigma(-gap'/eps), pst = sigma(-arg/eps_s) (1 under all-stick)
        wbar += wb_next * (1.0 - L.Sg * L.pst);
        const double gapbar = wb_next * L.w * L.pst * L.Sg * (1.0 - L.Sg) / A.eps;
        double argbar = 0.0;
        if (A.mode == PDQ_REBOUND) argbar += wb_next * L.w * L.Sg * L.pst * (1.0 - L.pst) / A.eps_stick;
        if (L.reflect) {
            // rebound: x'' = x' (2 rc / r' - 1), v'' = v' + dv n, n = x'/r', dv = f(v'.n, arg)
            const double nx = L.nxa, ny = L.nya, rp = L.rn, rc = K.R - c.half_d;
            const double dvbar = vb[0] * nx + vb[1] * ny;
            double nbx = L.dv * vb[0], nby = L.dv * vb[1];
            double vnbar = 0.0;
            if (L.rcase == 0) vnbar = -dvbar;                            // dv = -v_n
            else if (L.rcase == 2) vnbar = -2.0 * dvbar;                 // dv = -2 v_n
            else if (L.rcase == 3) {                                     // dv = -v_n - sqrt(arg)/u*
                vnbar = -dvbar;
                argbar += dvbar * (-0.5 / (K.ustar * sqrt(L.arg)));
            }
            vb[0] += vnbar * nx;
            vb[1] += vnbar * ny;
            nbx += vnbar * (double)L.vn[0];
            nby += vnbar * (double)L.vn[1];
            const double gm = 2.0 * rc / rp - 1.0;
            const double gbar = xb[0] * L.xn + xb[1] * L.yn;
            double xbx = gm * xb[0], xby = gm * xb[1];
            const double rbar = gbar * (-2.0 * rc / (rp * rp));
            const double nn = nbx * nx + nby * ny;
            xbx += (nbx - nn * nx) / rp + rbar * nx;
            xby += (nby - nn * ny) / rp + rbar * ny;
            xb[0] = xbx;
            xb[1] = xby;
        }
        if (L.rn > 0.0) {   // gap' = R - r' - d/2
            xb[0] += -gapbar * L.xn / L.rn;
            xb[1] += -gapbar * L.yn / L.rn;
        }
        // exponential integrator: x' = x + v h phi1 + F h^2 phi2, v' = v e + F h phi1
        double vbar[3], Fbar[3], lambar = 0.0;
        const double p1 = (double)L.p1, p2 = (double)L.p2, e = (double)L.e;
        const double p1l = -h * (double)L.dp1, p2l = -h * (double)L.dp2, el = -h * e;   // d/d lambda
        for (int k = 0; k < 3; ++k) {
            const double v = (double)L.v[k], F = (double)L.F[k];
            vbar[k] = xb[k] * h * p1 + vb[k] * e;
            Fbar[k] = xb[k] * h * h * p2 + vb[k] * h * p1;
            lambar += xb[k] * (v * h * p1l + F * h * h * p2l) + vb[k] * (v * el + F * h * p1l);
            lambar += Fbar[k] * (double)L.u[k];
        }
        double ubar[3] = {Fbar[0] * (double)L.lam, Fbar[1] * (double)L.lam, Fbar[2] * (double)L.lam};
        const double abar[3] = {Fbar[0], Fbar[1], Fbar[2]};
        double xbn[3] = {xb[0], xb[1], xb[2]};   // dx'/dx = I
        if (K.forces & PDQ_F_DRAG) {
            // lambda = f / tau, f = 1 + 0.15 Re^0.687, Re = |u - v| d+
            const double fbar = lambar / c.tau;
            const double Re = (double)L.Re;
            const double rebar = Re > 0.0 ? fbar * 0.15 * 0.687 * pow(Re, -0.313) : 0.0;
            const double relm = (double)L.relm;
            if (relm > 0.0) {
                const double mbar = rebar * c.d_plus;
                for (int k = 0; k < 3; ++k) {
                    const double rb = mbar * (double)L.rel[k] / relm;
                    ubar[k] += rb;
                    vbar[k] -= rb;
                }
            }
            for (int m = 0; m < 3; ++m)
                for (int k = 0; k < 3; ++k) xbn[m] += ubar[k] * (double)L.du[k][m];
        }
        // wall forces a_wall = A(r) n, n = (x, y)/r
        double qbar = 0.0;
        if (L.r > 0.0 && (K.forces & (PDQ_F_IMAGE | PDQ_F_VDW))) {
            const double Abar = abar[0] * L.nx + abar[1] * L.ny;
            xbn[0] += L.dAdr * Abar * L.nx + L.A * (abar[0] - Abar * L.nx) / L.r;
            xbn[1] += L.dAdr * Abar * L.ny + L.A * (abar[1] - Abar * L.ny) / L.r;
            qbar += Abar * L.img_q;
            zeta_bar += Abar * L.vdw_z;
        }
        // Coulomb a_C = coul q S: qbar += coul abar . S; c = coul q abar for the pair adjoint
        double cx = 0.0, cy = 0.0, cz = 0.0;
        if (K.forces & PDQ_F_COULOMB) {
            qbar += c.coul * (abar[0] * (double)S3[0] + abar[1] * (double)S3[1] + abar[2] * (double)S3[2]);
            cx = c.coul * L.q * abar[0];
            cy = c.coul * L.q * abar[1];
            cz = c.coul * L.q * abar[2];
        }
        if (A.mode == PDQ_REBOUND) {
            // arg = elastic0 (1 - theta)^2 - zeta stick
            zeta_bar += argbar * (-c.stick);
            theta_bar = argbar * (-2.0 * K.elastic0 * (1.0 - sp.theta));
        }
        A.xb[g] = xbn[0]; A.yb[g] = xbn[1]; A.zb[g] = xbn[2];
        A.vxb[g] = vbar[0]; A.vyb[g] = vbar[1]; A.vzb[g] = vbar[2];
        A.wb[g] = wbar;
        A.qb[g] = qbar;
        A.cx[g] = cx; A.cy[g] = cy; A.cz[g] = cz;
    }
    warp_add(zeta_bar, A.pbar + (int64_t)s * 3 + 1);
    if (A.mode == PDQ_REBOUND) warp_add(theta_bar, A.pbar + (int64_t)s * 3 + 2);
}

// All-pairs adjoint of S_m = sum_j Q_j G(x_m - x_j), Q = w q, G(d) = d / max(|d|, d_c)^3:
//   xbar_m += sum_j J(d_mj) (Q_j c_m - Q_m c_j),  J = (I - 3 d d^T / |d|^2) / |d|^3 (|d| > d_c) or I / d_c^3,
//   Qbar_m  = -sum_j c_j . G(d_mj);  then qbar_m += w_m Qbar_m, wbar_m += q_m Qbar_m, xi-bar += qbar_m qhat_m.
// A j-particle of the packed pair VJP, each value duplicated in both halves: position, Q, c.
struct VjpJ { f2 x, y, z, Q, cx, cy, cz; };

template <int P, int NT>
__global__ void __launch_bounds__(NT) k_adj_pairs(const AdjArgs A) {
    typedef typename Real<P>::T T;
    constexpr int U = adj_ilp<P>();          // particles m per thread
    __shared__ __align__(16) unsigned char smem_raw[P == PDQ_MIXED ? NT * 64 : 7 * NT * sizeof(T)];
    T (*sj)[NT] = reinterpret_cast<T (*)[NT]>(smem_raw);
    const int s = blockIdx.y, tid = threadIdx.x;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    if ((int64_t)blockIdx.x * NT * U >= n) return;
    const pdq_sample_params sp = A.params[s];
    const StepConst& K = A.K;
    double xi_bar[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xi_bar[u] = 0.0;
    // (MIXED with Coulomb forces runs the Newton-pair VJP, k_adj_pairs_sym, instead)
    if (P == PDQ_FP64 && (K.forces & PDQ_F_COULOMB)) {
        T xm[U], ym[U], zm[U], Qm[U], cmx[U], cmy[U], cmz[U];
        // per m: A1 = sum_j Q_j / r^3, A2 = sum_j c_j / r^3, A3 = sum_j k_mj d (J's outer-product term),
        // Qb = -sum_j c_j . d / r^3; then xbar_m = c_m A1 - Q_m A2 + A3
        T A1[U], A2x[U], A2y[U], A2z[U], A3x[U], A3y[U], A3z[U], Qb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
            const bool valid = i < n;
            const int64_t g = o + (valid ? i : 0);
            xm[u] = valid ? (T)A.in.x[g] : (T)0;
            ym[u] = valid ? (T)A.in.y[g] : (T)0;
            zm[u] = valid ? (T)A.in.z[g] : (T)0;
            Qm[u] = valid ? (T)(A.in.w[g] * sp.xi * A.qhat[g]) : (T)0;
            cmx[u] = valid ? (T)A.cx[g] : (T)0;
            cmy[u] = valid ? (T)A.cy[g] : (T)0;
            cmz[u] = valid ? (T)A.cz[g] : (T)0;
            A1[u] = A2x[u] = A2y[u] = A2z[u] = A3x[u] = A3y[u] = A3z[u] = Qb[u] = (T)0;
        }
        const T L = (T)K.L, invL = (T)K.invL;
        const T c2 = P == PDQ_FP64 ? (T)K.contact2 : (T)K.contact2f;
        const T M = P == PDQ_FP64 ? (T)6755399441055744.0 : (T)12582912.0f;   // 1.5 * 2^52 / 1.5 * 2^23
        for (int64_t j0 = 0; j0 < n; j0 += NT) {
            const int64_t j = j0 + tid;
            if (j < n) {
                const int64_t gj = o + j;
                sj[0][tid] = (T)A.in.x[gj]; sj[1][tid] = (T)A.in.y[gj]; sj[2][tid] = (T)A.in.z[gj];
                sj[3][tid] = (T)(A.in.w[gj] * sp.xi * A.qhat[gj]);
                sj[4][tid] = (T)A.cx[gj]; sj[5][tid] = (T)A.cy[gj]; sj[6][tid] = (T)A.cz[gj];
            } else {
                for (int q = 0; q < 7; ++q) sj[q][tid] = (T)0;
            }
            __syncthreads();
#pragma unroll 2
            for (int k = 0; k < NT; ++k) {
                const T xj = sj[0][k], yj = sj[1][k], zj = sj[2][k], Qj = sj[3][k];
                const T cjx = sj[4][k], cjy = sj[5][k], cjz = sj[6][k];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const T dx = xm[u] - xj, dy = ym[u] - yj;
                    T dz = zm[u] - zj;
                    const T t = (dz * invL + M) - M;                 // rint(dz / L)
                    dz -= L * t;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    const T ri = rsqrt_ftz(r2 > c2 ? r2 : c2);
                    const T ri2 = ri * ri, ri3 = ri2 * ri;
                    const T dcj = dx * cjx + dy * cjy + dz * cjz;      // d . c_j
                    const T dcm = dx * cmx[u] + dy * cmy[u] + dz * cmz[u];
                    A1[u] += Qj * ri3;
                    A2x[u] += ri3 * cjx; A2y[u] += ri3 * cjy; A2z[u] += ri3 * cjz;
                    // J v with v = Q_j c_m - Q_m c_j: the -3 d (d . v) / r^5 part, zero inside the contact clamp
                    const T kk = r2 > c2 ? (T)-3 * ri3 * ri2 * (Qj * dcm - Qm[u] * dcj) : (T)0;
                    A3x[u] += kk * dx; A3y[u] += kk * dy; A3z[u] += kk * dz;
                    Qb[u] -= ri3 * dcj;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
            if (i < n) {
                const int64_t g = o + i;
                A.xb[g] += (double)(cmx[u] * A1[u] - Qm[u] * A2x[u] + A3x[u]);
                A.yb[g] += (double)(cmy[u] * A1[u] - Qm[u] * A2y[u] + A3y[u]);
                A.zb[g] += (double)(cmz[u] * A1[u] - Qm[u] * A2z[u] + A3z[u]);
                const double qm = sp.xi * A.qhat[g];
                const double w = A.in.w[g];
                A.wb[g] += (double)Qb[u] * qm;
                xi_bar[u] = (A.qb[g] + (double)Qb[u] * w) * A.qhat[g];
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = (int64_t)blockIdx.x * NT * U + u * NT + tid;
            if (i < n) xi_bar[u] = A.qb[o + i] * A.qhat[o + i];
        }
    }
    double xs = 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) xs += xi_bar[u];
    warp_add(xs, A.pbar + (int64_t)s * 3 + 0);
}

// ---------------------------------------------------------------------------
// Newton pairs (MIXED): each unordered pair evaluated once for both particles.
// ---------------------------------------------------------------------------
// Forward Coulomb sums S_i = sum_j Q_j G(x_i - x_j), Q = w xi qhat, into A.acc4 (zeroed before
// the launch) with the step's newton_tile; grid (samples, i-tiles of NT*U): CTAs go out in
// tile order, so the first tiles of every sample (the most later particles) start first.
// k_adj_forward with SUMS then does the local part.
template <int NT, int U>
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 6) k_adj_sums_sym(const AdjArgs A) {
    const int s = blockIdx.x;
    const int64_t o = A.offset[s], end = A.offset[s + 1];
    const int64_t base = o + (int64_t)blockIdx.y * NT * U;
    if (base >= end) return;
    const double xi = A.params[s].xi;
    const auto load = [&](int64_t g) {
        return make_float4((float)A.in.x[g], (float)A.in.y[g], (float)A.in.z[g], (float)(A.in.w[g] * xi * A.qhat[g]));
    };
    newton_tile<NT, U>(load, base, end, (float)A.K.L, (float)A.K.invL, (float)A.K.contact2f, A.acc4);
}

// Pair-VJP term of pair (m, j) in x-bar_m, d = x_m - x_j:
//   T = J(d)(Q_j c_m - Q_m c_j) = u / r^3 - 3 d (d.u) / r^5,  u = Q_j c_m - Q_m c_j
// (u / d_c^3 inside the clamp).  J is even in d and u odd under m <-> j, so T enters x-bar_j
// with the opposite sign.  The charge term Qp_m = sum_j (d.c_j)/r^3 (Q-bar_m = -Qp_m) gets
// -(d.c_m)/r^3 for j.  One j against two m-particles, packed: T is added to (tx, ty, tz) and
// (jx, jy, jz), (d.c_j)/r^3 to qp and (d.c_m)/r^3 to jq; the caller negates the j sums.
// 38 packed operations (d.u taken from d.c_m and d.c_j, T from c_m and c_j scaled by Q/r^3).
// nQm = -Q_m; MINIMG / CLAMP as in vjp_pair_x2.
template <bool MINIMG, bool CLAMP>
__device__ __forceinline__ void vjp_pair_x2_sym(f2 xm, f2 ym, f2 zm, f2 nQm, f2 cmx, f2 cmy, f2 cmz, const VjpJ& J,
                                                f2 invL2, f2 M2, f2 nM2, f2 nL2, float c2, f2& tx, f2& ty, f2& tz,
                                                f2& qp, f2& jx, f2& jy, f2& jz, f2& jq) {
    const f2 dx = f2_sub(xm, J.x), dy = f2_sub(ym, J.y);
    f2 dz = f2_sub(zm, J.z);
    if constexpr (MINIMG) {
        const f2 t = f2_add(f2_fma(dz, invL2, M2), nM2);
        dz = f2_fma(nL2, t, dz);
    }
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    f2 ri, mask3;
    if constexpr (CLAMP) {
        ri = f2_pack(rsqrt_ftz(fmaxf(ra, c2)), rsqrt_ftz(fmaxf(rb, c2)));
        mask3 = f2_pack(ra > c2 ? -3.f : 0.f, rb > c2 ? -3.f : 0.f);
    } else {
        ri = f2_pack(rsqrt_ftz(ra), rsqrt_ftz(rb));
        mask3 = f2_pack(-3.f, -3.f);
    }
    const f2 ri2 = f2_mul(ri, ri), ri3 = f2_mul(ri2, ri);
    const f2 dcj = f2_fma(dx, J.cx, f2_fma(dy, J.cy, f2_mul(dz, J.cz)));
    const f2 dcm = f2_fma(dx, cmx, f2_fma(dy, cmy, f2_mul(dz, cmz)));
    // d.u = Q_j (d.c_m) - Q_m (d.c_j), from the products the charge terms need anyway
    const f2 du = f2_fma(J.Q, dcm, f2_mul(nQm, dcj));
    const f2 kk = f2_mul(f2_mul(f2_mul(ri3, ri2), mask3), du);
    // T = (Q_j / r^3) c_m - (Q_m / r^3) c_j + kk d
    const f2 a = f2_mul(ri3, J.Q), b = f2_mul(ri3, nQm);
    const f2 Tx = f2_fma(a, cmx, f2_fma(b, J.cx, f2_mul(kk, dx)));
    const f2 Ty = f2_fma(a, cmy, f2_fma(b, J.cy, f2_mul(kk, dy)));
    const f2 Tz = f2_fma(a, cmz, f2_fma(b, J.cz, f2_mul(kk, dz)));
    tx = f2_add(tx, Tx);
    ty = f2_add(ty, Ty);
    tz = f2_add(tz, Tz);
    jx = f2_add(jx, Tx);
    jy = f2_add(jy, Ty);
    jz = f2_add(jz, Tz);
    qp = f2_fma(ri3, dcj, qp);
    jq = f2_fma(ri3, dcm, jq);
}

// Pair VJP with Newton pairs (MIXED), the scheme of newton_tile: grid (samples, m-tiles of
// NT*U), heavy first tiles first; warp w holds the m-particles [32 U w, 32 U (w + 1)) of the
// tile, a contiguous run of the z-binned checkpoint (narrow z range: fewer clamped groups); the
// tile's own block one-sided (the j sums of vjp_pair_x2_sym left unused), every
// later particle of the sample as a Newton pair with 32-j groups walked by skewed lanes.  Sums
// (x-bar x, y, z, Qp) go to A.acc4 by float4 atomics; k_adj_pairs_finish applies them.
template <int NT, int U>
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 6) k_adj_pairs_sym(const AdjArgs A) {
    constexpr int W = NT / 32, H = U / 2;
    static_assert(U % 2 == 0 && NT % 32 == 0, "packed pairs over whole warps");
    // staged j: (x,x,y,y), (z,z,Q,Q), (cx,cx,cy,cy), (cz,cz,-,-), each array at a 16-byte stride;
    // j = 32 g + t of group g at entries 64 g + t and 64 g + 32 + t, so that lane l reads entry
    // l + k at step k without wrapping
    __shared__ __align__(16) ulonglong2 sA[2 * NT], sB[2 * NT], sC[2 * NT], sD[2 * NT];
    __shared__ float s_jacc[W][4][NT];
    __shared__ float2 s_zr[W];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = A.offset[s], end = A.offset[s + 1];
    const int64_t base = o + (int64_t)blockIdx.y * NT * U;
    if (base >= end) return;
    const int64_t dend = base + NT * U < end ? base + NT * U : end;
    const double xi = A.params[s].xi;
    const StepConst& K = A.K;
    const float L = (float)K.L, M = 12582912.0f;
    const f2 invL2 = f2_pack((float)K.invL, (float)K.invL), M2 = f2_pack(M, M), nM2 = f2_pack(-M, -M);
    const f2 nL2 = f2_pack(-L, -L);
    const float c2 = (float)K.contact2f;
    const float dcz = sqrtf(c2) + 1e-3f;
    f2 X[H], Y[H], Z[H], NQ[H], CX[H], CY[H], CZ[H], TX[H], TY[H], TZ[H], QP[H];
    float ilo = INFINITY, ihi = -INFINITY;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float v[2][7];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t g = base + warp * (32 * U) + (2 * h + e) * 32 + lane;   // contiguous per warp
            if (g < end) {
                v[e][0] = (float)A.in.x[g]; v[e][1] = (float)A.in.y[g]; v[e][2] = (float)A.in.z[g];
                v[e][3] = (float)(A.in.w[g] * xi * A.qhat[g]);
                v[e][4] = (float)A.cx[g]; v[e][5] = (float)A.cy[g]; v[e][6] = (float)A.cz[g];
                ilo = fminf(ilo, v[e][2]);
                ihi = fmaxf(ihi, v[e][2]);
            } else {     // padding: far off the axis, no charge, no cotangent
                v[e][0] = 1e15f;
#pragma unroll
                for (int q = 1; q < 7; ++q) v[e][q] = 0.f;
            }
        }
        X[h] = f2_pack(v[0][0], v[1][0]); Y[h] = f2_pack(v[0][1], v[1][1]); Z[h] = f2_pack(v[0][2], v[1][2]);
        NQ[h] = f2_pack(-v[0][3], -v[1][3]);
        CX[h] = f2_pack(v[0][4], v[1][4]); CY[h] = f2_pack(v[0][5], v[1][5]); CZ[h] = f2_pack(v[0][6], v[1][6]);
        TX[h] = TY[h] = TZ[h] = QP[h] = 0ull;
    }
    for (int d = 16; d > 0; d >>= 1) {
        ilo = fminf(ilo, __shfl_xor_sync(0xffffffffu, ilo, d));
        ihi = fmaxf(ihi, __shfl_xor_sync(0xffffffffu, ihi, d));
    }
    for (int64_t j0 = base; j0 < end; j0 += NT) {
        const bool diag = j0 < dend;
        const int64_t jlim = diag ? dend : end;
        const int64_t j = j0 + tid;
        float v[7] = {-1e15f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (j < jlim) {
            v[0] = (float)A.in.x[j]; v[1] = (float)A.in.y[j]; v[2] = (float)A.in.z[j];
            v[3] = (float)(A.in.w[j] * xi * A.qhat[j]);
            v[4] = (float)A.cx[j]; v[5] = (float)A.cy[j]; v[6] = (float)A.cz[j];
        }
        const float2 r = warp_range(j < jlim ? v[2] : INFINITY, j < jlim ? v[2] : -INFINITY);
        if (lane == 0) s_zr[warp] = r;
        {
            const int e = warp * 64 + lane;
            sA[e] = sA[e + 32] = make_ulonglong2(f2_pack(v[0], v[0]), f2_pack(v[1], v[1]));
            sB[e] = sB[e + 32] = make_ulonglong2(f2_pack(v[2], v[2]), f2_pack(v[3], v[3]));
            sC[e] = sC[e + 32] = make_ulonglong2(f2_pack(v[4], v[4]), f2_pack(v[5], v[5]));
            sD[e] = sD[e + 32] = make_ulonglong2(f2_pack(v[6], v[6]), 0ull);
        }
        __syncthreads();
        if (diag) {      // one-sided over the tile's own particles (self pair: d = 0, u = 0)
            float blo = INFINITY, bhi = -INFINITY;
#pragma unroll
            for (int w = 0; w < W; ++w) { blo = fminf(blo, s_zr[w].x); bhi = fmaxf(bhi, s_zr[w].y); }
            const ZClass zc = zclass(ilo, ihi, blo, bhi, L, dcz);
            auto block = [&](auto minimg, const f2* Zt) {
#pragma unroll 2
                for (int k = 0; k < NT; ++k) {
                    const int e = 64 * (k >> 5) + (k & 31);
                    const ulonglong2 a = sA[e], b = sB[e], cc = sC[e], dd = sD[e];
                    const VjpJ J{a.x, a.y, b.x, b.y, cc.x, cc.y, dd.x};
                    f2 ux = 0ull, uy = 0ull, uz = 0ull, uq = 0ull;      // j sums: not used
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        vjp_pair_x2_sym<decltype(minimg)::value, true>(X[h], Y[h], Zt[h], NQ[h], CX[h], CY[h], CZ[h],
                                                                        J, invL2, M2, nM2, nL2, c2, TX[h], TY[h],
                                                                        TZ[h], QP[h], ux, uy, uz, uq);
                }
            };
            if (zc.direct) {
                const f2 sh = f2_pack(zc.shift, zc.shift);
                f2 Zs[H];
#pragma unroll
                for (int h = 0; h < H; ++h) Zs[h] = f2_sub(Z[h], sh);
                block(std::false_type{}, Zs);
            } else {
                block(std::true_type{}, Z);
            }
            __syncthreads();
            continue;
        }
#pragma unroll 1
        for (int g = 0; g < W; ++g) {
            const float2 zr = s_zr[g];
            const ZClass zc = zclass(ilo, ihi, zr.x, zr.y, L, dcz);
            // the j sums stay packed (one half per i-half) and rotate as 64-bit shuffles; the
            // halves are added once, back at home after 32 steps
            f2 JX = 0ull, JY = 0ull, JZ = 0ull, JQ = 0ull;
            const int from = (lane + 1) & 31;
            const ulonglong2 *pA = sA + 64 * g + lane, *pB = sB + 64 * g + lane, *pC = sC + 64 * g + lane,
                             *pD = sD + 64 * g + lane;
            auto group = [&](auto minimg, auto clamp, const f2* Zt) {
#pragma unroll 4
                for (int k = 0; k < 32; ++k) {
                    const ulonglong2 a = pA[k], b = pB[k], cc = pC[k], dd = pD[k];
                    const VjpJ J{a.x, a.y, b.x, b.y, cc.x, cc.y, dd.x};
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        vjp_pair_x2_sym<decltype(minimg)::value, decltype(clamp)::value>(
                            X[h], Y[h], Zt[h], NQ[h], CX[h], CY[h], CZ[h], J, invL2, M2, nM2, nL2, c2, TX[h], TY[h],
                            TZ[h], QP[h], JX, JY, JZ, JQ);
                    JX = __shfl_sync(0xffffffffu, JX, from);
                    JY = __shfl_sync(0xffffffffu, JY, from);
                    JZ = __shfl_sync(0xffffffffu, JZ, from);
                    JQ = __shfl_sync(0xffffffffu, JQ, from);
                }
            };
            if (zc.direct) {
                const f2 sh = f2_pack(zc.shift, zc.shift);
                f2 Zs[H];
#pragma unroll
                for (int h = 0; h < H; ++h) Zs[h] = f2_sub(Z[h], sh);
                if (zc.apart) group(std::false_type{}, std::false_type{}, Zs);
                else group(std::false_type{}, std::true_type{}, Zs);
            } else {
                group(std::true_type{}, std::true_type{}, Z);
            }
            float l0, l1;
            f2_unpack(JX, l0, l1); s_jacc[warp][0][g * 32 + lane] = l0 + l1;
            f2_unpack(JY, l0, l1); s_jacc[warp][1][g * 32 + lane] = l0 + l1;
            f2_unpack(JZ, l0, l1); s_jacc[warp][2][g * 32 + lane] = l0 + l1;
            f2_unpack(JQ, l0, l1); s_jacc[warp][3][g * 32 + lane] = l0 + l1;
        }
        __syncthreads();
        if (j < end) {     // j's terms carry the opposite sign
            float sx = 0.f, sy = 0.f, sz = 0.f, sq = 0.f;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                sx += s_jacc[w][0][tid]; sy += s_jacc[w][1][tid]; sz += s_jacc[w][2][tid]; sq += s_jacc[w][3][tid];
            }
            atomicAdd(&A.acc4[j], make_float4(-sx, -sy, -sz, -sq));
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float t0[4], t1[4];
        f2_unpack(TX[h], t0[0], t1[0]);
        f2_unpack(TY[h], t0[1], t1[1]);
        f2_unpack(TZ[h], t0[2], t1[2]);
        f2_unpack(QP[h], t0[3], t1[3]);
        const int64_t g0 = base + warp * (32 * U) + (2 * h) * 32 + lane, g1 = g0 + 32;
        if (g0 < end) atomicAdd(&A.acc4[g0], make_float4(t0[0], t0[1], t0[2], t0[3]));
        if (g1 < end) atomicAdd(&A.acc4[g1], make_float4(t1[0], t1[1], t1[2], t1[3]));
    }
}

// Applies the Newton-pair VJP sums: x-bar += (x, y, z), w-bar += -Qp xi qhat, and the xi
// cotangent (q-bar - Qp w) qhat summed per sample.  Grid (particles / 256, samples).
__global__ void k_adj_pairs_finish(const AdjArgs A) {
    const int s = blockIdx.y;
    const int64_t o = A.offset[s], n = A.offset[s + 1] - o;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double xs = 0.0;
    if (i < n) {
        const int64_t g = o + i;
        const float4 t = A.acc4[g];
        A.xb[g] += (double)t.x;
        A.yb[g] += (double)t.y;
        A.zb[g] += (double)t.z;
        const double qm = A.params[s].xi * A.qhat[g];
        A.wb[g] += (double)(-t.w) * qm;
        xs = (A.qb[g] + (double)(-t.w) * A.in.w[g]) * A.qhat[g];
    }
    warp_add(xs, A.pbar + (int64_t)s * 3 + 0);
}

// J = (R+/2) num / (dt den) and the cotangents of num and den for one vector gbar.
__global__ void k_adj_finish(const double* num, const double* den, const double* gbar, int n, double R, double dt,
                             double* J, double* nbar, double* dbar) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double d = den[k];
    const double f = d > 0.0 ? 0.5 * R / dt : 0.0;
    if (J) J[k] = d > 0.0 ? f * num[k] / d : 0.0;
    if (gbar) {
        nbar[k] = d > 0.0 ? gbar[k] * f / d : 0.0;
        dbar[k] = d > 0.0 ? -gbar[k] * f * num[k] / (d * d) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host.
// ---------------------------------------------------------------------------
struct AdjLayout {
    int64_t N;
    int64_t n_ck;       // checkpoints (states at 0, K, 2K, ...)
    int32_t K;
    size_t bytes;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static AdjLayout adj_layout(int64_t N, int32_t S, int32_t C, int64_t n_steps, int32_t K) {
    AdjLayout L;
    L.N = N;
    L.K = K;
    L.n_ck = (n_steps + K - 1) / K;
    if (L.n_ck < 1) L.n_ck = 1;
    const size_t vec = a256(sizeof(double) * (size_t)(N > 0 ? N : 1));
    size_t b = 0;
    b += vec * 7 * (size_t)L.n_ck;                 // checkpoints
    b += vec * 10 * (size_t)(K + 1);               // segment slots
    b += vec * 11;                                 // cotangents, c
    b += vec;                                      // qhat
    b += a256(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));   // classes
    // per checkpoint, the z-binned order's qhat, classes and permutation; 7 scratch cotangents
    b += (vec + 2 * a256(sizeof(int32_t) * (size_t)(N > 0 ? N : 1))) * (size_t)L.n_ck;
    b += vec * 7;
    b += a256(sizeof(float) * 4 * (size_t)(N > 0 ? N : 1));   // MIXED Newton-pair sums
    b += a256(sizeof(double) * (size_t)S * C) * 4; // num, den, nbar, dbar
    L.bytes = b;
    return L;
}

// Stored Newton-pair sums, past the layout: a 256-byte marker, then one float4 [capacity] array
// per step.
static size_t adj_sums_bytes(int64_t N, int64_t n_steps) {
    return 256 + a256(sizeof(float) * 4 * (size_t)(N > 0 ? N : 1)) * (size_t)n_steps;
}

}  // namespace pdq

using namespace pdq;

extern "C" int pdq_adjoint_stored_sums_size(int64_t capacity, int64_t n_steps, size_t* bytes) {
    if (!bytes || capacity < 0 || n_steps < 1) return PDQ_ERR_INVALID_ARG;
    *bytes = adj_sums_bytes(capacity, n_steps);
    return PDQ_OK;
}

extern "C" int pdq_adjoint_workspace_size(const pdq_batch* batch, int64_t n_steps, int32_t K, size_t* bytes) {
    if (!batch || !bytes || batch->n_samples < 1 || batch->n_classes < 1 || batch->n_classes > PDQ_MAX_CLASSES ||
        batch->capacity < 0 || n_steps < 1 || K < 1)
        return PDQ_ERR_INVALID_ARG;
    *bytes = adj_layout(batch->capacity, batch->n_samples, batch->n_classes, n_steps, K).bytes;
    return PDQ_OK;
}

namespace pdq {

// Where the adjoint's initial state comes from.
enum AdjInit { ADJ_SEED = 0, ADJ_STATE = 1, ADJ_REVERSE_ONLY = 2 };

// The three entry points below share this routine.  ADJ_SEED seeds the particles as
// pdq_seed_particles would; ADJ_STATE loads them from `init`; ADJ_REVERSE_ONLY skips the forward
// sweep and runs the reverse sweeps on the checkpoints and sums a forward sweep left in the
// workspace (the workspace layout depends only on the batch, n_steps and K).
static int adjoint_impl(const pdq_field* field, const pdq_phys* phys, const pdq_batch* batch,
                        const pdq_sample_params* params, AdjInit init_kind, const pdq_state* init,
                        double charge_sigma, uint64_t seed, const pdq_step_cfg* cfg, int64_t n_steps, int32_t K,
                        double eps, double eps_stick, int32_t n_vec, const double* gbar, double* J, double* pbar,
                        void* workspace, size_t workspace_bytes, pdq_stream_t stream) {
    const bool forward = init_kind != ADJ_REVERSE_ONLY;
    if (!field || !phys || !batch || !params || !cfg || (forward && !J) || n_steps < 1 || K < 1 || !(eps > 0) ||
        n_vec < 0 || (n_vec > 0 && (!gbar || !pbar)) || (!forward && n_vec < 1) || !(charge_sigma >= 0))
        return PDQ_ERR_INVALID_ARG;
    if (cfg->mode != PDQ_STICK && cfg->mode != PDQ_REBOUND) return PDQ_ERR_INVALID_ARG;
    if (cfg->mode == PDQ_REBOUND && !(eps_stick > 0)) return PDQ_ERR_INVALID_ARG;
    if (!(cfg->dt > 0) || (cfg->forces & ~PDQ_F_ALL)) return PDQ_ERR_INVALID_ARG;
    if (batch->precision != PDQ_FP64 && batch->precision != PDQ_MIXED) return PDQ_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = pdq_adjoint_workspace_size(batch, n_steps, K, &need);
    if (rc) return rc;
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return PDQ_ERR_WORKSPACE;
    if (batch->capacity > ((int64_t)1 << 31) - 1) return PDQ_ERR_INVALID_ARG;
    pdq_state st;   // only the class description is read by make_step_const
    memset(&st, 0, sizeof(st));
    st.n_classes = batch->n_classes;
    st.n_samples = batch->n_samples;
    for (int c = 0; c < batch->n_classes; ++c) st.st_plus[c] = batch->st_plus[c];
    AdjArgs A;
    memset(&A, 0, sizeof(A));
    rc = make_step_const(field, phys, &st, &A.K);
    if (rc) return rc;
    A.K.dt = cfg->dt;
    A.K.dtf = (float)cfg->dt;
    A.K.forces = cfg->forces;
    A.K.mode = cfg->mode;
    A.K.window_start = cfg->window_start;
    const double gplus = phys->g * phys->nu / pow(phys->re_tau * phys->nu / phys->radius, 3);
    for (int k = 0; k < 3; ++k) { A.K.grav[k] = gplus * cfg->gravity[k]; A.K.gravf[k] = (float)A.K.grav[k]; }
    A.offset = batch->offset;
    A.S = batch->n_samples;
    A.C = batch->n_classes;
    A.params = params;
    A.eps = eps;
    A.eps_stick = eps_stick;
    A.mode = cfg->mode;
    A.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    A.sigma = charge_sigma;
    A.neg_frac = phys->neg_charge_frac;

    const AdjLayout Ly = adj_layout(batch->capacity, A.S, A.C, n_steps, K);
    const int64_t N = Ly.N;
    const size_t vec = a256(sizeof(double) * (size_t)(N > 0 ? N : 1));
    char* p = (char*)workspace;
    auto take = [&](size_t n) { char* r = p; p += n; return r; };
    std::vector<Slot> ck(Ly.n_ck), seg(K + 1);
    for (auto& s : ck) {
        s.x = (double*)take(vec); s.y = (double*)take(vec); s.z = (double*)take(vec);
        s.vx = (double*)take(vec); s.vy = (double*)take(vec); s.vz = (double*)take(vec); s.w = (double*)take(vec);
        s.sx = s.sy = s.sz = nullptr;
    }
    for (auto& s : seg) {
        s.x = (double*)take(vec); s.y = (double*)take(vec); s.z = (double*)take(vec);
        s.vx = (double*)take(vec); s.vy = (double*)take(vec); s.vz = (double*)take(vec); s.w = (double*)take(vec);
        s.sx = (double*)take(vec); s.sy = (double*)take(vec); s.sz = (double*)take(vec);
    }
    A.xb = (double*)take(vec); A.yb = (double*)take(vec); A.zb = (double*)take(vec);
    A.vxb = (double*)take(vec); A.vyb = (double*)take(vec); A.vzb = (double*)take(vec);
    A.wb = (double*)take(vec); A.qb = (double*)take(vec);
    A.cx = (double*)take(vec); A.cy = (double*)take(vec); A.cz = (double*)take(vec);
    A.qhat = (double*)take(vec);
    const size_t ivec = a256(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    A.cls = (int32_t*)take(ivec);
    // z-binned order of each checkpoint: its qhat, classes and permutation; scratch cotangents
    std::vector<double*> ck_qh(Ly.n_ck);
    std::vector<int32_t*> ck_cl(Ly.n_ck), ck_perm(Ly.n_ck);
    for (int64_t k = 0; k < Ly.n_ck; ++k) {
        ck_qh[k] = (double*)take(vec);
        ck_cl[k] = (int32_t*)take(ivec);
        ck_perm[k] = (int32_t*)take(ivec);
    }
    double* scratch[7];
    for (auto& q : scratch) q = (double*)take(vec);
    A.acc4 = (float4*)take(a256(sizeof(float) * 4 * (size_t)(N > 0 ? N : 1)));
    const size_t acc_bytes = sizeof(float4) * (size_t)(N > 0 ? N : 1);
    const size_t sc = a256(sizeof(double) * (size_t)A.S * A.C);
    A.num = (double*)take(sc); A.den = (double*)take(sc);
    double* nbar = (double*)take(sc);
    double* dbar = (double*)take(sc);
    A.nbar = nbar; A.dbar = dbar;
    // MIXED with Coulomb forces and room past the layout: every step's Newton-pair sums are kept
    // (the forward sweep accumulates them in place), so the reverse sweep's segment recompute
    // reruns only the local part; the marker ties them to the forward sweep that wrote them
    const bool newton_sums = batch->precision == PDQ_MIXED && (A.K.forces & PDQ_F_COULOMB);
    const bool store = newton_sums && workspace_bytes >= need + adj_sums_bytes(N, n_steps);
    int64_t* const marker = store ? (int64_t*)take(256) : nullptr;
    const size_t sums_stride = a256(sizeof(float) * 4 * (size_t)(N > 0 ? N : 1));
    char* const sums_base = store ? p : nullptr;
    float4* const acc_scratch = A.acc4;
    const int64_t mark[4] = {0x70647153756d7331LL, n_steps, K, N};

    // largest sample -> tiles per grid row
    std::vector<int64_t> off(A.S + 1);
    cudaStream_t s = (cudaStream_t)stream;
    PDQ_CUDA(cudaMemcpyAsync(off.data(), batch->offset, sizeof(int64_t) * (A.S + 1), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    int64_t nmax = 0;
    for (int k = 0; k < A.S; ++k) nmax = std::max(nmax, off[k + 1] - off[k]);
    if (off[A.S] != N) return PDQ_ERR_INVALID_ARG;
    if (nmax == 0) nmax = 1;
    const int NT = 128;
    const bool mixed = batch->precision == PDQ_MIXED;
    const int ilp = mixed ? adj_ilp<PDQ_MIXED>() : adj_ilp<PDQ_FP64>();             // particles per thread
    const dim3 grid((unsigned)((nmax + ilp * NT - 1) / (ilp * NT)), (unsigned)A.S);

    // MIXED with Coulomb forces: the pair sums (forward) and the pair VJP (reverse) take Newton
    // pairs, each unordered pair once, through A.acc4
    const bool newton = mixed && (A.K.forces & PDQ_F_COULOMB);
    const int NTN = 128;
    // grid y counts the tiles of the largest sample (at most 65,535: 33.5 M particles per sample)
    if (newton && (nmax + 4 * NTN - 1) / (4 * NTN) > 65535) return PDQ_ERR_UNSUPPORTED;
    constexpr int US = 12;   // forward sums: 12 particles per thread (as the step's Newton kernel)
    const dim3 grid_sums((unsigned)A.S, (unsigned)((nmax + US * NTN - 1) / (US * NTN)));
    const dim3 grid_vjp((unsigned)A.S, (unsigned)((nmax + 4 * NTN - 1) / (4 * NTN)));
    // one forward step; `recompute`: a step of the reverse sweep's segment recompute, which takes
    // the stored sums when there are any
    auto fwd = [&](const Slot& in, const Slot& out, int64_t step, int tally, bool recompute) -> cudaError_t {
        A.in = in; A.out = out; A.step = step; A.tally = tally;
        if (newton) {
            A.acc4 = store ? (float4*)(sums_base + sums_stride * (size_t)step) : acc_scratch;
            if (!(store && recompute)) {
                const cudaError_t e = cudaMemsetAsync(A.acc4, 0, acc_bytes, s);
                if (e != cudaSuccess) return e;
                k_adj_sums_sym<NTN, US><<<grid_sums, NTN, 0, s>>>(A);
            }
            k_adj_forward<PDQ_MIXED, NT, true><<<grid, NT, 0, s>>>(A);
            A.acc4 = acc_scratch;
        } else if (mixed) {
            k_adj_forward<PDQ_MIXED, NT><<<grid, NT, 0, s>>>(A);
        } else {
            k_adj_forward<PDQ_FP64, NT><<<grid, NT, 0, s>>>(A);
        }
        return cudaSuccess;
    };
    auto copy_state = [&](const Slot& dst, const Slot& src) -> cudaError_t {
        const size_t nb = sizeof(double) * (size_t)N;
        double* const d[7] = {dst.x, dst.y, dst.z, dst.vx, dst.vy, dst.vz, dst.w};
        double* const r[7] = {src.x, src.y, src.z, src.vx, src.vy, src.vz, src.w};
        for (int q = 0; q < 7; ++q) {
            cudaError_t e = cudaMemcpyAsync(d[q], r[q], nb, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };

    // Checkpoint k holds the state z-binned (the pair loops then see tiles of nearby z, see
    // k_adj_forward); the steps of segment k run in that order with its qhat and classes.
    const float bpl = (float)(kAdjBins / A.K.L);
    const double* qh_cur = A.qhat;
    const int32_t* cl_cur = A.cls;
    auto checkpoint = [&](int64_t k, const Slot& from) -> cudaError_t {
        k_adj_sort<<<(unsigned)A.S, 1024, 0, s>>>(batch->offset, from, qh_cur, cl_cur, ck[k], ck_qh[k], ck_cl[k],
                                                  ck_perm[k], bpl);
        qh_cur = ck_qh[k];
        cl_cur = ck_cl[k];
        A.qhat = ck_qh[k];
        A.cls = ck_cl[k];
        return copy_state(from, ck[k]);
    };
    const int nsc = A.S * A.C;
    if (forward) {
        // seed (or load) into segment slot 0, save as checkpoint 0
        A.out = seg[0];
        const dim3 g1((unsigned)((nmax + NT - 1) / NT), (unsigned)A.S);
        if (init_kind == ADJ_SEED) {
            k_adj_seed<<<g1, NT, 0, s>>>(A);
        } else if (init->precision == PDQ_FP64) {
            k_adj_load<PDQ_FP64><<<g1, NT, 0, s>>>(A, init->count, init->pos[init->cur], init->vel[init->cur],
                                                  nullptr, (const int2*)init->tag);
        } else {
            k_adj_load<PDQ_MIXED><<<g1, NT, 0, s>>>(A, init->count, init->pos[init->cur], init->vel[init->cur],
                                                   (const double2*)init->xy[init->cur], (const int2*)init->tag);
        }
        PDQ_CUDA(cudaMemsetAsync(A.num, 0, sc, s));
        PDQ_CUDA(cudaMemsetAsync(A.den, 0, sc, s));
        PDQ_CUDA(checkpoint(0, seg[0]));
        // forward sweep: ping-pong between segment slots 0 and 1, checkpoint every K steps
        if (store) PDQ_CUDA(cudaMemcpyAsync(marker, mark, sizeof(mark), cudaMemcpyHostToDevice, s));
        for (int64_t n = 0; n < n_steps; ++n) {
            PDQ_CUDA(fwd(seg[n & 1], seg[(n + 1) & 1], n, 1, false));
            if ((n + 1) % K == 0 && (n + 1) < n_steps) PDQ_CUDA(checkpoint((n + 1) / K, seg[(n + 1) & 1]));
        }
        k_adj_finish<<<(nsc + 255) / 256, 256, 0, s>>>(A.num, A.den, nullptr, nsc, A.K.R, A.K.dt, J, nullptr,
                                                       nullptr);
        PDQ_CUDA(cudaGetLastError());
    }

    if (store && !forward) {   // the stored sums must come from a forward sweep of this layout
        int64_t got[4];
        PDQ_CUDA(cudaMemcpyAsync(got, marker, sizeof(got), cudaMemcpyDeviceToHost, s));
        PDQ_CUDA(cudaStreamSynchronize(s));
        if (memcmp(got, mark, sizeof(got)) != 0) return PDQ_ERR_INVALID_ARG;
    }
    // backward sweeps, one per cotangent vector
    for (int v = 0; v < n_vec; ++v) {
        k_adj_finish<<<(nsc + 255) / 256, 256, 0, s>>>(A.num, A.den, gbar + (size_t)v * nsc, nsc, A.K.R, A.K.dt,
                                                       nullptr, nbar, dbar);
        A.pbar = pbar + (size_t)v * A.S * 3;
        PDQ_CUDA(cudaMemsetAsync(A.pbar, 0, sizeof(double) * A.S * 3, s));
        for (double* q : {A.xb, A.yb, A.zb, A.vxb, A.vyb, A.vzb, A.wb}) PDQ_CUDA(cudaMemsetAsync(q, 0, vec, s));
        for (int64_t kseg = Ly.n_ck - 1; kseg >= 0; --kseg) {
            const int64_t n0 = kseg * K;
            const int64_t len = std::min<int64_t>(K, n_steps - n0);
            A.qhat = ck_qh[kseg];
            A.cls = ck_cl[kseg];
            PDQ_CUDA(copy_state(seg[0], ck[kseg]));
            for (int64_t t = 0; t < len; ++t) PDQ_CUDA(fwd(seg[t], seg[t + 1], n0 + t, 0, true));
            for (int64_t t = len - 1; t >= 0; --t) {
                A.in = seg[t];
                A.step = n0 + t;
                if (newton) {
                    PDQ_CUDA(cudaMemsetAsync(A.acc4, 0, acc_bytes, s));
                    k_adj_local<PDQ_MIXED><<<dim3((unsigned)((nmax + 127) / 128), (unsigned)A.S), 128, 0, s>>>(A);
                    k_adj_pairs_sym<NTN, 4><<<grid_vjp, NTN, 0, s>>>(A);
                    k_adj_pairs_finish<<<dim3((unsigned)((nmax + 255) / 256), (unsigned)A.S), 256, 0, s>>>(A);
                } else if (mixed) {
                    k_adj_local<PDQ_MIXED><<<dim3((unsigned)((nmax + 127) / 128), (unsigned)A.S), 128, 0, s>>>(A);
                    k_adj_pairs<PDQ_MIXED, NT><<<grid, NT, 0, s>>>(A);
                } else {
                    k_adj_local<PDQ_FP64><<<dim3((unsigned)((nmax + 127) / 128), (unsigned)A.S), 128, 0, s>>>(A);
                    k_adj_pairs<PDQ_FP64, NT><<<grid, NT, 0, s>>>(A);
                }
            }
            if (kseg > 0) {
                // cotangents of checkpoint kseg's binned state -> the order segment kseg-1 ends in
                double** bars[7] = {&A.xb, &A.yb, &A.zb, &A.vxb, &A.vyb, &A.vzb, &A.wb};
                for (int q = 0; q < 7; ++q) {
                    k_adj_unperm<<<dim3((unsigned)((nmax + 255) / 256), (unsigned)A.S), 256, 0, s>>>(
                        batch->offset, ck_perm[kseg], *bars[q], scratch[q]);
                    std::swap(*bars[q], scratch[q]);
                }
            }
            PDQ_CUDA(cudaGetLastError());
        }
    }
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

// The pdq_batch a state's adjoint is laid out by.
static void batch_of_state(const pdq_state* st, pdq_batch* b) {
    memset(b, 0, sizeof(*b));
    b->precision = st->precision;
    b->n_samples = st->n_samples;
    b->n_classes = st->n_classes;
    for (int c = 0; c < st->n_classes && c < PDQ_MAX_CLASSES; ++c) b->st_plus[c] = st->st_plus[c];
    b->capacity = st->capacity;
    b->offset = st->offset;
}

}  // namespace pdq

extern "C" int pdq_adjoint_state_workspace_size(const pdq_state* init, int64_t n_steps, int32_t K, size_t* bytes) {
    if (!init) return PDQ_ERR_INVALID_ARG;
    pdq_batch b;
    batch_of_state(init, &b);
    return pdq_adjoint_workspace_size(&b, n_steps, K, bytes);
}

extern "C" int pdq_adjoint_run(const pdq_field* field, const pdq_phys* phys, const pdq_state* init,
                               const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps, int32_t K,
                               double eps, double eps_stick, int32_t n_vec, const double* gbar, double* J,
                               double* pbar, void* workspace, size_t workspace_bytes, pdq_stream_t stream) {
    if (!init || !params || !init->offset || !init->count || !init->tag || (init->cur != 0 && init->cur != 1) ||
        !init->pos[init->cur] || !init->vel[init->cur] || (init->precision == PDQ_MIXED && !init->xy[init->cur]))
        return PDQ_ERR_INVALID_ARG;
    if (init->n_samples < 1 || init->n_samples > (1 << 20)) return PDQ_ERR_INVALID_ARG;
    // charge per unit xi = q_eff / xi: every sample needs xi != 0
    std::vector<pdq_sample_params> hp((size_t)init->n_samples);
    cudaStream_t s = (cudaStream_t)stream;
    PDQ_CUDA(cudaMemcpyAsync(hp.data(), params, sizeof(pdq_sample_params) * hp.size(), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    for (const auto& q : hp)
        if (!(q.xi != 0.0) || !std::isfinite(q.xi)) return PDQ_ERR_INVALID_ARG;
    pdq_batch b;
    batch_of_state(init, &b);
    return adjoint_impl(field, phys, &b, params, ADJ_STATE, init, 0.0, 0, cfg, n_steps, K, eps, eps_stick, n_vec,
                        gbar, J, pbar, workspace, workspace_bytes, stream);
}

extern "C" int pdq_adjoint_run_seeded(const pdq_field* field, const pdq_phys* phys, const pdq_batch* batch,
                                      const pdq_sample_params* params, double charge_sigma, uint64_t seed,
                                      const pdq_step_cfg* cfg, int64_t n_steps, int32_t K, double eps,
                                      double eps_stick, int32_t n_vec, const double* gbar, double* J, double* pbar,
                                      void* workspace, size_t workspace_bytes, pdq_stream_t stream) {
    return adjoint_impl(field, phys, batch, params, ADJ_SEED, nullptr, charge_sigma, seed, cfg, n_steps, K, eps,
                        eps_stick, n_vec, gbar, J, pbar, workspace, workspace_bytes, stream);
}

extern "C" int pdq_adjoint_reverse(const pdq_field* field, const pdq_phys* phys, const pdq_batch* batch,
                                   const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                                   int32_t K, double eps, double eps_stick, int32_t n_vec, const double* gbar,
                                   double* pbar, void* workspace, size_t workspace_bytes, pdq_stream_t stream) {
    return adjoint_impl(field, phys, batch, params, ADJ_REVERSE_ONLY, nullptr, 0.0, 0, cfg, n_steps, K, eps,
                        eps_stick, n_vec, gbar, nullptr, pbar, workspace, workspace_bytes, stream);
}
