// pdq_particles.cu -- seeding, the fused particle step, compaction and the
// deposition tally of libpdq.
//
// Step kernel layout: a persistent grid pulls work items (sample s, i-tile t)
// from a device queue ordered largest sample first.  A CTA of NT threads owns
// NT*U particles of one sample (U per thread), streams every j-tile of that
// sample through shared memory for the all-pairs Coulomb sum (Eq. coulomb,
// App. A.2), then runs the local physics of its particles (interpolation,
// drag, gravity, image charge, vdW, exponential integrator, wall contact) and
// writes the new state into the other half of the double buffer.  Tallies are
// reduced with warp ballots, then one shared-memory and one global atomic per
// class.  The last CTA to finish advances the device step counter and resets
// the queue, so consecutive launches need no host round trip.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "pdq_common.cuh"
#include "pdq_device.cuh"
#include "pdq_newton.cuh"

namespace pdq {

// CTL_QUEUE2 / CTL_DONE2: work queue and done counter of the Newton-pair sum kernel (pair variant 3)
enum { CTL_STEP = 0, CTL_QUEUE = 1, CTL_DONE = 2, CTL_ERROR = 3, CTL_NITEMS = 4, CTL_QUEUE2 = 5, CTL_DONE2 = 6 };
enum { ERR_NONFINITE = 1 };


// ---------------------------------------------------------------------------
// Host: per-class constants from the physical constants (all SI -> wall units).
// ---------------------------------------------------------------------------
// The Coulomb contact distance of a state, wall units: contact_scale x the largest class diameter.
double contact_distance(const pdq_phys* p, const pdq_state* st) {
    const double ustar = p->re_tau * p->nu / p->radius;
    const double ell = p->nu / ustar, tauf = p->nu / (ustar * ustar);
    double dmax = 0.0;
    for (int c = 0; c < st->n_classes; ++c)
        dmax = fmax(dmax, sqrt(18.0 * p->rho_f * p->nu * st->st_plus[c] * tauf / p->rho_p) / ell);
    return p->contact_scale * dmax;
}

int make_step_const(const pdq_field* f, const pdq_phys* p, const pdq_state* st, StepConst* K) {
    memset(K, 0, sizeof(*K));
    const double ustar = p->re_tau * p->nu / p->radius;   // u* = Re_tau nu / R
    const double ell = p->nu / ustar;                       // m per wall unit
    const double tauf = p->nu / (ustar * ustar);
    const double acc = p->nu / (ustar * ustar * ustar);     // SI acceleration -> wall units
    const double ke = 1.0 / (4.0 * kPi * p->eps0);
    if (fabs(f->desc.r_plus - p->re_tau) > 1e-9 * p->re_tau) return PDQ_ERR_INVALID_ARG;
    if (!(p->contact_scale > 0.0) || !(p->contact_scale <= 1e6)) return PDQ_ERR_INVALID_ARG;
    double dmax = 0.0;
    K->n_classes = st->n_classes;
    for (int c = 0; c < st->n_classes; ++c) {
        ClassK& k = K->cls[c];
        const double tau = st->st_plus[c];
        if (!(tau > 0)) return PDQ_ERR_INVALID_ARG;
        // tau_p = rho_p d^2 / (18 rho_f nu) and tau_p+ = tau_p / tau_f  (Sec. 2.1)
        k.tau = tau;
        k.d_m = sqrt(18.0 * p->rho_f * p->nu * tau * tauf / p->rho_p);
        k.d_plus = k.d_m / ell;
        k.half_d = 0.5 * k.d_plus;
        k.mass = p->rho_p * kPi * k.d_m * k.d_m * k.d_m / 6.0;
        k.qfac = (k.d_m * 1e6) * (k.d_m * 1e6);
        k.coul = ke * p->q_unit * p->q_unit / (k.mass * ell * ell) * acc;
        k.vdw = p->hamaker0 / (3.0 * k.mass) * acc;          // 2 x (A0/6) / m
        k.stick = 2.0 * (0.25 * kPi * k.d_m * k.d_m) * p->hamaker0 / (24.0 * kPi * p->delta_c * p->delta_c) / k.mass;
        k.d3 = k.d_plus * k.d_plus * k.d_plus;
        k.vdw_pp = p->hamaker0 / (6.0 * k.mass) * acc;
        k.tau_f = (float)tau;
        k.inv_tau_f = (float)(1.0 / tau);
        k.d_plus_f = (float)k.d_plus;
        k.half_d_f = (float)k.half_d;
        k.coul_f = (float)k.coul;
        k.img_f = (float)(0.25 * k.coul);                     // image at distance 2y: coul / 4 / y^2
        k.wall2 = (f->desc.r_plus - k.half_d) * (f->desc.r_plus - k.half_d);
        k.vdw_reach_f = (float)(0.75 * k.d_plus * 1.001 + 1e-6);   // gap + d/2 <= d/4 + d/2, widened
        if (k.d_plus > dmax) dmax = k.d_plus;
    }
    K->R = f->desc.r_plus;
    K->L = f->desc.l_plus;
    K->invL = 1.0 / K->L;
    K->ell = ell;
    K->delta_min = p->delta_min;
    K->ustar = ustar;
    K->elastic0 = p->sigma_y0 * p->sigma_y0 / (p->rho_p * p->young);
    K->contact2 = (p->contact_scale * dmax) * (p->contact_scale * dmax);
    K->near = 1.25 * dmax;      // (d_i + d_j)/2 + d_eff/4 <= 1.25 d_max
    K->inv_beta = 1.0 / f->desc.beta;
    K->tanh_beta = tanh(f->desc.beta);
    K->n_r = f->desc.n_r; K->n_th = f->desc.n_th; K->n_z = f->desc.n_z;
    K->R2 = K->R * K->R;
    K->th_scale_f = (float)(K->n_th / (2.0 * kPi));
    K->z_scale_f = (float)(K->n_z * K->invL);
    K->Rf = (float)K->R; K->Lf = (float)K->L; K->invLf = (float)K->invL;
    K->contact2f = (float)K->contact2;
    K->inv_beta_f = (float)K->inv_beta; K->tanh_beta_f = (float)K->tanh_beta;
    K->grid64 = f->grid64;
    K->grid32 = f->grid32;
    return PDQ_OK;
}

// ---------------------------------------------------------------------------
// Seeding.
// ---------------------------------------------------------------------------
struct SeedArgs {
    const int64_t* offset; int32_t* count; int64_t* ctl;
    const pdq_sample_params* params;
    void* pos; void* vel; double2* xy; int2* tag;
    int64_t capacity; int32_t S, C; double sigma, neg_frac; uint2 key;
    int32_t independent;   // 1: sample s draws with Philox counter word 3 = s + 1
    double R, L; double half_d[PDQ_MAX_CLASSES]; double qfac[PDQ_MAX_CLASSES];
};

template <int P>
__global__ void k_seed(const SeedArgs A) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < A.S) A.count[g] = (int32_t)(A.offset[g + 1] - A.offset[g]);
    if (g < 8) A.ctl[g] = 0;
    if (g >= A.capacity) return;
    int lo = 0, hi = A.S;                       // offset[lo] <= g < offset[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.offset[mid] <= g) lo = mid; else hi = mid;
    }
    const int s = lo;
    const uint32_t j = (uint32_t)(g - A.offset[s]);
    const int c = (int)(j % (uint32_t)A.C);
    double x, y, z, qhat;
    seed_particle(A.key, j, A.sigma, A.neg_frac, A.R, A.L, A.half_d[c], A.qfac[c], x, y, z, qhat,
                  A.independent ? (uint32_t)(s + 1) : 0u);
    const double q = A.params[s].xi * qhat;
    if (P == PDQ_FP64) {
        ((double4_32a*)A.pos)[g] = make_double4_32a(x, y, z, q);
        ((double4_32a*)A.vel)[g] = make_double4_32a(0.0, 0.0, 0.0, 1.0);
    } else {
        A.xy[g] = make_double2(x, y);
        ((float4*)A.pos)[g] = make_float4((float)x, (float)y, (float)z, (float)q);
        ((float4*)A.vel)[g] = make_float4(0.f, 0.f, 0.f, 1.f);
    }
    A.tag[g] = make_int2((int)j, c);
}

// ---------------------------------------------------------------------------
// Packed FP32 pair math (sm_100+ f32x2 instructions): one 64-bit register holds
// the same quantity for two i-particles, so each FMA-pipe instruction serves
// two pairs.  rsqrt is the flush-to-zero hardware approximation (no denormal
// fix-up path; pair distances are clamped at the contact distance anyway).
// ---------------------------------------------------------------------------
// Same pairs, with the three accumulations issued as scalar FFMA (two per
// component) so that they can run on the FMA-lite pipe beside the packed work.
__device__ __forceinline__ void coulomb_pair_x2s(f2 xi, f2 yi, f2 zi, f2 xj, f2 yj, f2 zj, f2 qj, f2 invL2, f2 M2,
                                                 f2 nM2, f2 nL2, float c2, float (&ax)[2], float (&ay)[2],
                                                 float (&az)[2]) {
    const f2 dx = f2_sub(xi, xj), dy = f2_sub(yi, yj);
    f2 dz = f2_sub(zi, zj);
    const f2 t = f2_add(f2_fma(dz, invL2, M2), nM2);
    dz = f2_fma(nL2, t, dz);
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    const f2 ri = f2_pack(rsqrt_ftz(fmaxf(ra, c2)), rsqrt_ftz(fmaxf(rb, c2)));
    const f2 s = f2_mul(f2_mul(ri, qj), f2_mul(ri, ri));
    float s0, s1, x0, x1, y0, y1, z0, z1;
    f2_unpack(s, s0, s1);
    f2_unpack(dx, x0, x1);
    f2_unpack(dy, y0, y1);
    f2_unpack(dz, z0, z1);
    ax[0] = __fmaf_rn(s0, x0, ax[0]); ax[1] = __fmaf_rn(s1, x1, ax[1]);
    ay[0] = __fmaf_rn(s0, y0, ay[0]); ay[1] = __fmaf_rn(s1, y1, ay[1]);
    az[0] = __fmaf_rn(s0, z0, az[0]); az[1] = __fmaf_rn(s1, z1, az[1]);
}

struct StepArgs {
    StepConst K;
    const void* pos_in; const void* vel_in; const double2* xy_in;
    void* pos_out; void* vel_out; double2* xy_out;
    const int2* tag; const int64_t* offset; const int32_t* count;
    const pdq_sample_params* params;
    const int2* items; int64_t* ctl;
    unsigned long long* n_dep; unsigned long long* n_alive;
    // j-split (FP64 only; 1 otherwise): each i-tile's pair sum is cut into jsplit
    // chunks, one work item each; partial sums go to part[(chunk*3 + k)*cap + g] and
    // the last chunk to finish (tile_cnt) adds them in chunk order and does the update.
    int jsplit; int64_t cap; double* part; int* tile_cnt;
    // Coulomb sums given per particle ([cap][3], e.g. from P3M): replace the pair loop when set
    const double* ext;
    // pair variant 3: FP32 Coulomb sums [cap] (x, y, z, unused) accumulated by k_pairs_sym; the
    // given-sums step (V = 5) reads them instead of ext when set.  FP64: acc64 [cap][3], summed by
    // k_pairs_sym64 and passed to the given-sums step as ext
    float4* acc4;
    double* acc64;
    // host only: upper bound on the work items of a launch (the persistent grid is capped by it,
    // so that few items spread one per CTA over the SMs instead of piling onto the first CTAs)
    int64_t max_items;
};

// Local physics of one particle; returns its class, whether it was alive at the
// start of the step, and whether it deposited.
template <int P, bool CT = false>
__device__ __forceinline__ void local_update(const StepArgs& A, int64_t g, typename Real<P>::T acx,
                                             typename Real<P>::T acy, typename Real<P>::T acz,
                                             const pdq_sample_params& sp, int& cls, bool& was_alive, bool& dep,
                                             double cx = 0.0, double cy = 0.0, double cz = 0.0) {
    typedef typename Real<P>::T T;
    typedef typename Real<P>::T4 T4;
    const StepConst& K = A.K;
    const T4 p4 = ((const T4*)A.pos_in)[g];
    const T4 v4 = ((const T4*)A.vel_in)[g];
    double x, y;
    if (P == PDQ_FP64) { x = (double)p4.x; y = (double)p4.y; }
    else { const double2 xy = A.xy_in[g]; x = xy.x; y = xy.y; }
    T z = p4.z;
    const T q = p4.w;
    cls = A.tag[g].y;
    dep = false;
    was_alive = v4.w > (T)0.5;
    if (!was_alive) {
        ((T4*)A.pos_out)[g] = p4;
        ((T4*)A.vel_out)[g] = v4;
        if (P == PDQ_MIXED) A.xy_out[g] = make_double2(x, y);
        return;
    }
    const ClassK& c = K.cls[cls];
    T a[3] = {(T)0, (T)0, (T)0};
    if (K.forces & PDQ_F_COULOMB) {
        const T kq = (P == PDQ_FP64 ? (T)c.coul : (T)c.coul_f) * q;
        a[0] = kq * acx; a[1] = kq * acy; a[2] = kq * acz;
    }
    if (K.forces & PDQ_F_GRAVITY) {
        if constexpr (P == PDQ_FP64) { a[0] += K.grav[0]; a[1] += K.grav[1]; a[2] += K.grav[2]; }
        else { a[0] += K.gravf[0]; a[1] += K.gravf[1]; a[2] += K.gravf[2]; }
    }
    if constexpr (CT) { a[0] += (T)cx; a[1] += (T)cy; a[2] += (T)cz; }
    // 2 F_vw(delta) at the gap delta (m): Eq. (vdw) written as A d^6 / (6 delta^2 (2d+delta)^2 (d+delta)^3),
    // zero beyond d/4 and saturated at delta_min
    auto vdw_wall = [&](double gap) {
        if (!(gap <= 0.25 * c.d_m)) return 0.0;
        const double dl = fmax(gap, K.delta_min);
        const double d = c.d_m;
        const double d2 = d * d, d6 = d2 * d2 * d2;
        const double e1 = 2.0 * d + dl, e2 = d + dl;
        return sp.zeta * c.vdw * d6 / (dl * dl * e1 * e1 * e2 * e2 * e2);
    };
    const double r2 = x * x + y * y;
    T rT;                  // radius for the field interpolation
    if constexpr (P == PDQ_FP64) {
        const double r = sqrt(r2);
        rT = r;
        if (r > 0.0 && (K.forces & (PDQ_F_IMAGE | PDQ_F_VDW))) {
            double aw = 0.0;   // toward the wall
            if (K.forces & PDQ_F_IMAGE) {
                // image of opposite sign mirrored across the wall: q^2 / (4 pi eps0 (2y)^2 m), y >= d/2
                const double yw = fmax(K.R - r, c.half_d);
                aw += 0.25 * c.coul * (double)q * (double)q / (yw * yw);
            }
            if (K.forces & PDQ_F_VDW) aw += vdw_wall((K.R - r - c.half_d) * K.ell);
            const double inv_r = 1.0 / r;
            a[0] += (T)(aw * x * inv_r);
            a[1] += (T)(aw * y * inv_r);
        }
    } else {
        // The wall distance R - r = (R^2 - r^2) / (R + r): the difference in FP64 (no cancellation
        // near the wall), the quotient and the force direction in FP32 (the forces are FP32); the
        // vdW gap in FP64 from the FP64 radius, taken only near the wall.
        rT = sqrtf((float)r2);
        if (r2 > 0.0 && (K.forces & (PDQ_F_IMAGE | PDQ_F_VDW))) {
            const float yw0 = (float)(K.R2 - r2) / (K.Rf + rT);
            float aw = 0.f;    // toward the wall
            if (K.forces & PDQ_F_IMAGE) {
                const float yw = fmaxf(yw0, c.half_d_f);
                aw = c.img_f * (float)q * (float)q / (yw * yw);
            }
            if ((K.forces & PDQ_F_VDW) && yw0 <= c.vdw_reach_f)
                aw = (float)((double)aw + vdw_wall((K.R - sqrt(r2) - c.half_d) * K.ell));
            const float ir = 1.0f / rT;
            a[0] += aw * (p4.x * ir);
            a[1] += aw * (p4.y * ir);
        }
    }
    T v[3] = {v4.x, v4.y, v4.z};
    T u[3] = {(T)0, (T)0, (T)0};
    T lam = (T)0;
    if (K.forces & PDQ_F_DRAG) {
        if constexpr (P == PDQ_FP64) interp<T, T4>(K, rT, (T)x, (T)y, z, u);
        else interp<T, T4>(K, rT, p4.x, p4.y, z, u);       // p4.x, p4.y: x, y rounded to FP32
        const T rx = u[0] - v[0], ry = u[1] - v[1], rz = u[2] - v[2];
        const T re = sqrt_(rx * rx + ry * ry + rz * rz) * (P == PDQ_FP64 ? (T)c.d_plus : (T)c.d_plus_f);
        const T fd = (T)1 + (T)0.15 * (re > (T)0 ? pow_(re, (T)0.687) : (T)0);   // Schiller-Naumann
        lam = fd * (P == PDQ_FP64 ? (T)(1.0 / c.tau) : (T)c.inv_tau_f);
    }
    const T h = P == PDQ_FP64 ? (T)K.dt : (T)K.dtf;
    const T zz = -lam * h;
    T p1, p2;
    phi12(zz, p1, p2);
    const T e = exp_(zz);
    T dxv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T F = lam * u[k] + a[k];
        dxv[k] = v[k] * h * p1 + F * (h * h) * p2;
        v[k] = v[k] * e + F * h * p1;
    }
    double xn = x + (double)dxv[0];
    double yn = y + (double)dxv[1];
    T zn = z + dxv[2];
    const T Lz = P == PDQ_FP64 ? (T)K.L : (T)K.Lf, invLz = P == PDQ_FP64 ? (T)K.invL : (T)K.invLf;
    zn -= Lz * floor_(zn * invLz);
    if (zn >= Lz) zn -= Lz;
    if (zn < (T)0) zn = (T)0;
    // wall contact: gap R - r - d/2 <= 0 (App. A: removal on impact); MIXED compares r^2 with
    // (R - d/2)^2 in FP64 and takes the square root only on contact
    double rn;
    bool contact;
    if constexpr (P == PDQ_FP64) {
        rn = sqrt(xn * xn + yn * yn);
        contact = K.R - rn - c.half_d <= 0.0;
    } else {
        const double rn2 = xn * xn + yn * yn;
        contact = rn2 >= c.wall2;
        rn = contact ? sqrt(rn2) : 0.0;
    }
    bool alive = true;
    if (contact) {
        bool stick = true;
        if (K.mode == PDQ_REBOUND) {
            // Bons et al. (Sec. 4.3): CoR_n = sqrt(sigma_y^2/(rho_p E) - 2 A_cont gamma_c / m) / V_n1
            const double one_m = 1.0 - sp.theta;
            const double arg = K.elastic0 * one_m * one_m - sp.zeta * c.stick;
            if (arg > 0.0) {
                stick = false;
                const double nx = xn / rn, ny = yn / rn;
                const double vn = (double)v[0] * nx + (double)v[1] * ny;     // outward, wall units
                const double vn_si = vn * K.ustar;
                const double cor = vn_si > 0.0 ? fmin(1.0, sqrt(arg) / vn_si) : 1.0;
                const double dv = -cor * fabs(vn) - vn;
                v[0] = (T)((double)v[0] + dv * nx);
                v[1] = (T)((double)v[1] + dv * ny);
                const double rref = 2.0 * (K.R - c.half_d) - rn;
                xn = nx * rref;
                yn = ny * rref;
            }
        }
        if (stick) { alive = false; dep = true; }
    }
    if (!(isfinite(xn) && isfinite(yn) && isfinite(zn) && isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2])))
        atomicOr((unsigned long long*)&A.ctl[CTL_ERROR], (unsigned long long)ERR_NONFINITE);
    if (P == PDQ_FP64) {
        ((double4_32a*)A.pos_out)[g] = make_double4_32a(xn, yn, (double)zn, alive ? (double)q : 0.0);
        ((double4_32a*)A.vel_out)[g] = make_double4_32a((double)v[0], (double)v[1], (double)v[2], alive ? 1.0 : 0.0);
    } else {
        A.xy_out[g] = make_double2(xn, yn);
        ((float4*)A.pos_out)[g] = make_float4((float)xn, (float)yn, (float)zn, alive ? (float)q : 0.f);
        ((float4*)A.vel_out)[g] = make_float4((float)v[0], (float)v[1], (float)v[2], alive ? 1.f : 0.f);
    }
}

// ---------------------------------------------------------------------------
// Particle-particle contact (App. A.2 collision force and Eq. vdw between
// particles) of particle gi with the particles [jb, je) of its sample, in FP64,
// at the mid-step predicted positions x + v dt/2; accumulated into c[3].
//  collision (overlap o = (d_i + d_j)/2 - r > 0): m_ij/m_i (K o - H v_n) n,
//    K = (pi^2 + ln^2 e)/tau_col^2, H = -2 ln e/tau_col, v_n = (v_i - v_j).n,
//    n = (x_i - x_j)/r, m_ij/m_i = d_j^3/(d_i^3 + d_j^3);
//  vdW: -zeta A0 d^6 / (6 m_i g^2 (2d+g)^2 (d+g)^3) n with d = 2 d_i d_j/(d_i + d_j),
//    g = max(surface gap, delta_min), zero when the gap exceeds d/4.
// Rare: reached only for a thread whose tile pair holds a pair inside the
// contact range, so it reads the j data straight from global memory.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ void contact_tile(const StepArgs& A, int64_t gi, int64_t jb, int64_t je, double zeta,
                                          double c[3]) {
    typedef typename Real<P>::T4 T4;
    const StepConst& K = A.K;
    const T4* pos = (const T4*)A.pos_in;
    const T4* vel = (const T4*)A.vel_in;
    const T4 vi = vel[gi];
    if (!((double)vi.w > 0.5)) return;
    const double h2 = 0.5 * K.dt;
    const T4 pi4 = pos[gi];
    double xi, yi;
    if (P == PDQ_FP64) { xi = (double)pi4.x; yi = (double)pi4.y; }
    else { const double2 xy = A.xy_in[gi]; xi = xy.x; yi = xy.y; }
    const double zi = (double)pi4.z;
    const ClassK& ci = K.cls[A.tag[gi].y];
    const double near2 = K.near * K.near;
    // MIXED: an FP32 screen on the FP32 snapshot first.  Its separation differs from the FP64
    // one by ~3e-5 at most (the snapshot's rounding at |x| <= R, |z| <= L; z itself is FP32 in
    // MIXED), so with a 0.05 margin it only drops pairs that the FP64 test drops as well, and
    // results are unchanged; it keeps most candidate pairs off the narrow FP64 pipe.
    const float h2f = 0.5f * K.dtf, Lf = (float)K.L, invLf = (float)K.invL;
    const float scr = (float)K.near + 0.05f, scr2 = scr * scr;
    for (int64_t j = jb; j < je; ++j) {
        if (j == gi) continue;
        const T4 vj = vel[j];
        if (!((double)vj.w > 0.5)) continue;
        const T4 pj = pos[j];
        if constexpr (P == PDQ_MIXED) {
            const float fx = (pi4.x - pj.x) + h2f * (vi.x - vj.x);
            const float fy = (pi4.y - pj.y) + h2f * (vi.y - vj.y);
            float fz = (pi4.z - pj.z) + h2f * (vi.z - vj.z);
            fz -= Lf * rintf(fz * invLf);
            if (!(fx * fx + fy * fy + fz * fz < scr2)) continue;
        }
        double xj, yj;
        if (P == PDQ_FP64) { xj = (double)pj.x; yj = (double)pj.y; }
        else { const double2 xy = A.xy_in[j]; xj = xy.x; yj = xy.y; }
        // separation of nearby particles first (exact by Sterbenz's lemma), then the drift
        const double dx = (xi - xj) + h2 * ((double)vi.x - (double)vj.x);
        const double dy = (yi - yj) + h2 * ((double)vi.y - (double)vj.y);
        double dz = (zi - (double)pj.z) + h2 * ((double)vi.z - (double)vj.z);
        dz -= K.L * rint(dz * K.invL);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < near2) || !(r2 > 0.0)) continue;
        const double r = sqrt(r2), inv_r = 1.0 / r;
        const double nx = dx * inv_r, ny = dy * inv_r, nz = dz * inv_r;
        const ClassK& cj = K.cls[A.tag[j].y];
        const double contact = ci.half_d + cj.half_d;
        double a = 0.0;
        if ((K.forces & PDQ_F_COLLIDE) && r < contact) {
            const double vn = ((double)vi.x - (double)vj.x) * nx + ((double)vi.y - (double)vj.y) * ny +
                              ((double)vi.z - (double)vj.z) * nz;
            a += cj.d3 / (ci.d3 + cj.d3) * (K.col_k * (contact - r) - K.col_h * vn);
        }
        if (K.forces & PDQ_F_VDW_PP) {
            const double d = 2.0 * ci.d_m * cj.d_m / (ci.d_m + cj.d_m);
            const double gap = (r - contact) * K.ell;
            if (gap <= 0.25 * d) {
                const double gs = fmax(gap, K.delta_min);
                const double d2 = d * d, e1 = 2.0 * d + gs, e2 = d + gs;
                a -= zeta * ci.vdw_pp * d2 * d2 * d2 / (gs * gs * e1 * e1 * e2 * e2 * e2);
            }
        }
        c[0] += a * nx; c[1] += a * ny; c[2] += a * nz;
    }
}

// Largest speed of the staged j-tile, per warp (0 for padding and removed particles).
template <int P>
__device__ __forceinline__ void stage_speed(const StepArgs& A, int64_t j, int64_t end, int lane, int tid, float* s_v) {
    typedef typename Real<P>::T4 T4;
    float v = 0.f;
    if (j < end) {
        const T4 w = ((const T4*)A.vel_in)[j];
        if ((double)w.w > 0.5)
            v = (float)sqrt((double)w.x * (double)w.x + (double)w.y * (double)w.y + (double)w.z * (double)w.z);
    }
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
    if (lane == 0) s_v[tid >> 5] = v;
}

// Start-of-step separation beyond which no pair of the tile pair can come within the contact
// range by mid-step: range + (largest i speed + largest j speed) dt/2, with margins for the
// FP32 speeds and positions.
__device__ __forceinline__ float near_bound(const StepConst& K, const float* s_vi, const float* s_vj, int nw) {
    float vi = 0.f, vj = 0.f;
    for (int w = 0; w < nw; ++w) { vi = fmaxf(vi, s_vi[w]); vj = fmaxf(vj, s_vj[w]); }
    return (float)K.near + 0.5f * (float)K.dt * (vi + vj) * 1.001f + 1e-3f;
}

// Contact accelerations of this thread's particles from the j-tile starting at j0, added to
// its own slots of s_ct[3][U][NT].
template <int P, int NT, int U>
__device__ __forceinline__ void contact_rows(const StepArgs& A, int64_t base, int64_t end, int64_t j0, double zeta,
                                             double* s_ct) {
    const int tid = threadIdx.x;
    const int64_t je = j0 + NT < end ? j0 + NT : end;
    for (int u = 0; u < U; ++u) {
        const int64_t g = base + u * NT + tid;
        if (g >= end) continue;
        double c3[3] = {0.0, 0.0, 0.0};
        contact_tile<P>(A, g, j0, je, zeta, c3);
        s_ct[(0 * U + u) * NT + tid] += c3[0];
        s_ct[(1 * U + u) * NT + tid] += c3[1];
        s_ct[(2 * U + u) * NT + tid] += c3[2];
    }
}

// End of a j-tile in the contact variant: the closing barrier also ORs the threads' near-pair
// flags; a flagged tile is appended to the CTA's list (contact_rows runs when the list is full).
template <int P, int NT, int U, int NF>
__device__ __forceinline__ void flag_tile(const StepArgs& A, bool near, int64_t j0, int& nflag, long long* s_flag,
                                          int64_t base, int64_t end, double zeta, double* s_ct) {
    if (!__syncthreads_or(near)) return;
    if (nflag == NF) {
        for (int f = 0; f < NF; ++f) contact_rows<P, NT, U>(A, base, end, s_flag[f], zeta, s_ct);
        nflag = 0;
        __syncthreads();           // every thread has read the list before it is overwritten
    }
    if (threadIdx.x == 0) s_flag[nflag] = j0;
    ++nflag;
}

// Contact accelerations from every flagged j-tile of the item.
template <int P, int NT, int U>
__device__ __forceinline__ void flush_flags(const StepArgs& A, int nflag, const long long* s_flag, int64_t base,
                                            int64_t end, double zeta, double* s_ct) {
    if (!nflag) return;
    __syncthreads();               // the last entry is visible
    for (int f = 0; f < nflag; ++f) contact_rows<P, NT, U>(A, base, end, s_flag[f], zeta, s_ct);
    __syncthreads();               // the list is free for the next item
}

// FP64 pair of a tile pair that needs no periodic image (the shift is folded into zi); without
// CLAMP every |dz| of the tile pair exceeds the contact distance, so r^2 > c2 (self pair excluded).
template <bool CLAMP>
__device__ __forceinline__ void coulomb_pair_direct64(double xi, double yi, double zi, const double4_32a pj,
                                                      double c2, double& ax, double& ay, double& az) {
    const double dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
    double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, dz * dz));
    if constexpr (CLAMP) r2 = fmax(r2, c2);
    const double ri = rsqrt(r2);
    const double s = pj.w * ri * (ri * ri);
    ax = __fma_rn(s, dx, ax);
    ay = __fma_rn(s, dy, ay);
    az = __fma_rn(s, dz, az);
}

// FP64 pair of the contact-force variant: the Coulomb pair plus the smallest high word of r^2
// seen (for r^2 >= 0 the high word orders like the value; integer ALU work, off the narrow
// FP64 pipe; the self pair gives 0 and flags its own tile).
__device__ __forceinline__ void coulomb_pair_track(double xi, double yi, double zi, const double4_32a pj, double L,
                                                   double invL, double c2, double& ax, double& ay, double& az,
                                                   int& mnh) {
    const double dx = xi - pj.x, dy = yi - pj.y;
    double dz = zi - pj.z;
    const double t = __dadd_rn(__fma_rn(dz, invL, 6755399441055744.0), -6755399441055744.0);
    dz = __fma_rn(-L, t, dz);
    const double r2u = __fma_rn(dx, dx, __fma_rn(dy, dy, dz * dz));
    mnh = min(mnh, __double2hiint(r2u));
    const double r2 = fmax(r2u, c2);
    const double ri = rsqrt(r2);
    const double s = pj.w * ri * (ri * ri);
    ax = __fma_rn(s, dx, ax);
    ay = __fma_rn(s, dy, ay);
    az = __fma_rn(s, dz, az);
}

// Smallest nonzero r^2 of two i-particles against one j (the near-pair test of the contact
// variant whose Coulomb sums come from the Newton-pair kernel, V = 6; the self pair, r = 0, is
// left out).  MINIMG folds dz to the minimum image, else zi carries the tile pair's shift.
template <bool MINIMG>
__device__ __forceinline__ void near_pair_x2(f2 xi, f2 yi, f2 zi, f2 xj, f2 yj, f2 zj, f2 invL2, f2 M2, f2 nM2,
                                             f2 nL2, float& mn) {
    const f2 dx = f2_sub(xi, xj), dy = f2_sub(yi, yj);
    f2 dz = f2_sub(zi, zj);
    if constexpr (MINIMG) {
        const f2 t = f2_add(f2_fma(dz, invL2, M2), nM2);
        dz = f2_fma(nL2, t, dz);
    }
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    mn = fminf(mn, fminf(ra > 0.f ? ra : INFINITY, rb > 0.f ? rb : INFINITY));
}

// The MIXED contact variant is held to 96 registers (its rare FP64 contact path would
// otherwise set the register count, and the occupancy, of the whole pair loop).
template <int P, int NT, int U, int V>
__global__ void __launch_bounds__(NT, ((V == 4 || V == 6) && P == PDQ_MIXED) ? 65536 / (NT * 96) : 0)
    k_step(const StepArgs A) {
    typedef typename Real<P>::T T;
    typedef typename Real<P>::T4 T4;
    // j-tile: FP64 holds double4 (x, y, z, q); MIXED holds each value twice,
    // (x, x, y, y), (z, z, q, q), so packed f32x2 operands load without moves.
    __shared__ __align__(32) unsigned char smem_raw[NT * 32];
    __shared__ float2 s_zr[NT / 32];      // per-warp z range of the staged j-tile
    __shared__ float2 s_zi[NT / 32];      // per-warp z range of this CTA's i-particles
    __shared__ double2 s_z64[P == PDQ_FP64 ? 2 * (NT / 32) : 1];   // FP64: i ranges, then j ranges
    __shared__ int s_item, s_last;
    __shared__ unsigned int s_alive[PDQ_MAX_CLASSES], s_dep[PDQ_MAX_CLASSES];
    // contact-force variants (V == 4; V == 6 with the Coulomb sums of the Newton-pair kernel in
    // A.acc4): per-particle contact accelerations of the item, and the per-warp largest speeds of
    // the i-particles and of the staged j-tile (near-pair bound)
    constexpr bool CT = V == 4 || V == 6;
    __shared__ double s_ct[CT ? 3 * NT * U : 1];
    __shared__ float s_vi[NT / 32], s_vj[NT / 32];
    // j-tiles (first index) flagged as holding a near pair of this item; evaluated after the pair
    // loop so that the rare contact path stays out of the hot loop (flushed when full)
    constexpr int kFlags = 64;
    __shared__ long long s_flag[CT ? kFlags : 1];
    const StepConst& K = A.K;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t step = A.ctl[CTL_STEP];
    const bool counted = step >= K.window_start;
    const int64_t n_items = A.ctl[CTL_NITEMS];
    const T4* __restrict__ pos_in = (const T4*)A.pos_in;
    const T L = (T)K.L, invL = (T)K.invL;
    const T c2 = P == PDQ_FP64 ? (T)K.contact2 : (T)K.contact2f;
    const int C = K.n_classes;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd((unsigned long long*)&A.ctl[CTL_QUEUE], 1ull);
        if (tid < PDQ_MAX_CLASSES) { s_alive[tid] = 0u; s_dep[tid] = 0u; }
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int2 it = A.items[item];
        const int s = it.x;
        const int64_t o = A.offset[s];
        const int64_t end = o + A.count[s];
        const int JS = P == PDQ_FP64 ? A.jsplit : 1;
        const int tile = it.y / JS, jc = it.y - tile * JS;
        const int64_t base = o + (int64_t)tile * (NT * U);
        if constexpr (V == 5) {      // FP64 Newton pairs: one update per tile, from its chunk-0 item
            if (jc != 0) {
                __syncthreads();
                continue;
            }
        }
        T xi[U], yi[U], zi[U], ax[U], ay[U], az[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * NT + tid;
            if (g < end) { const T4 p = pos_in[g]; xi[u] = p.x; yi[u] = p.y; zi[u] = p.z; }
            else { xi[u] = (T)0; yi[u] = (T)0; zi[u] = (T)0; }
            ax[u] = ay[u] = az[u] = (T)0;
        }
        double zeta = 0.0;
        int nflag = 0;              // flagged j-tiles (uniform across the CTA)
        if constexpr (CT) {
            zeta = A.params[s].zeta;
            float vmax = 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * NT + tid;
                s_ct[(0 * U + u) * NT + tid] = 0.0;
                s_ct[(1 * U + u) * NT + tid] = 0.0;
                s_ct[(2 * U + u) * NT + tid] = 0.0;
                if (g < end) {
                    const T4 v = ((const T4*)A.vel_in)[g];
                    if ((float)v.w > 0.5f)
                        vmax = fmaxf(vmax, (float)sqrt((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z));
                }
            }
            for (int d = 16; d > 0; d >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, d));
            if (lane == 0) s_vi[tid >> 5] = vmax;
        }
        if constexpr (V == 5) {      // Coulomb sums given (P3M, or the Newton-pair kernel): no pair loop
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = base + u * NT + tid;
                if (g < end) {
                    if (A.acc4) { const float4 a = A.acc4[g]; ax[u] = (T)a.x; ay[u] = (T)a.y; az[u] = (T)a.z; }
                    else { ax[u] = (T)A.ext[3 * g]; ay[u] = (T)A.ext[3 * g + 1]; az[u] = (T)A.ext[3 * g + 2]; }
                }
            }
        } else if ((K.forces & PDQ_F_COULOMB) || CT) {
            if constexpr (P == PDQ_MIXED) {
                static_assert(U % 2 == 0, "packed pairs need an even number of i-particles per thread");
                constexpr int H = U / 2;
                ulonglong2* sj2 = reinterpret_cast<ulonglong2*>(smem_raw);
                const float M = 12582912.0f;
                const f2 invL2 = f2_pack((float)invL, (float)invL), M2 = f2_pack(M, M), nM2 = f2_pack(-M, -M);
                const f2 nL2 = f2_pack(-(float)L, -(float)L);
                f2 X[H], Y[H], Z[H], AX[H], AY[H], AZ[H];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    X[h] = f2_pack(xi[2 * h], xi[2 * h + 1]);
                    Y[h] = f2_pack(yi[2 * h], yi[2 * h + 1]);
                    Z[h] = f2_pack(zi[2 * h], zi[2 * h + 1]);
                    AX[h] = AY[h] = AZ[h] = 0ull;
                }
                // z range of this CTA's i-particles (the tiles of a z-binned sample are narrow)
                float ilo = INFINITY, ihi = -INFINITY;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (base + u * NT + tid < end) { ilo = fminf(ilo, (float)zi[u]); ihi = fmaxf(ihi, (float)zi[u]); }
                for (int d = 16; d > 0; d >>= 1) {
                    ilo = fminf(ilo, __shfl_xor_sync(0xffffffffu, ilo, d));
                    ihi = fmaxf(ihi, __shfl_xor_sync(0xffffffffu, ihi, d));
                }
                if (lane == 0) s_zi[tid >> 5] = make_float2(ilo, ihi);
                const float Lf = (float)L, halfL = 0.5f * Lf;
                const float dcz = sqrtf((float)c2) + 1e-3f;     // contact distance + rounding margin
                for (int64_t j0 = o; j0 < end; j0 += NT) {
                    const int64_t j = j0 + tid;
                    const float4 pj = j < end ? ((const float4*)pos_in)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    float jlo = j < end ? pj.z : INFINITY, jhi = j < end ? pj.z : -INFINITY;
                    for (int d = 16; d > 0; d >>= 1) {
                        jlo = fminf(jlo, __shfl_xor_sync(0xffffffffu, jlo, d));
                        jhi = fmaxf(jhi, __shfl_xor_sync(0xffffffffu, jhi, d));
                    }
                    if (lane == 0) s_zr[tid >> 5] = make_float2(jlo, jhi);
                    if constexpr (CT) stage_speed<P>(A, j, end, lane, tid, s_vj);
                    sj2[2 * tid] = make_ulonglong2(f2_pack(pj.x, pj.x), f2_pack(pj.y, pj.y));
                    sj2[2 * tid + 1] = make_ulonglong2(f2_pack(pj.z, pj.z), f2_pack(pj.w, pj.w));
                    __syncthreads();
                    // dz = z_i - z_j over the tile pair lies in [a_lo - b_hi, a_hi - b_lo]; when that
                    // interval sits strictly inside one period window, the minimum image is a
                    // uniform shift of 0 or +-L and the per-pair rounding step is skipped.
                    float alo = INFINITY, ahi = -INFINITY, blo = INFINITY, bhi = -INFINITY;
#pragma unroll
                    for (int w = 0; w < NT / 32; ++w) {
                        alo = fminf(alo, s_zi[w].x); ahi = fmaxf(ahi, s_zi[w].y);
                        blo = fminf(blo, s_zr[w].x); bhi = fmaxf(bhi, s_zr[w].y);
                    }
                    const float dlo = alo - bhi, dhi = ahi - blo;
                    // contact variant: pairs farther apart than thr cannot reach the contact range by
                    // mid-step (thr adds the largest relative drift over half a step)
                    float thr = dcz;
                    if constexpr (CT) thr = fmaxf(dcz, near_bound(K, s_vi, s_vj, NT / 32));
                    float mn = INFINITY;
                    float shift = 0.f;
                    bool direct = V == 0 || V == 4 || V == 6;
                    if (dlo > -halfL && dhi < halfL) shift = 0.f;
                    else if (dlo > halfL && dhi < 3.f * halfL) shift = Lf;
                    else if (dhi < -halfL && dlo > -3.f * halfL) shift = -Lf;
                    else direct = false;
                    if constexpr (V == 6) {
                        // Coulomb sums from A.acc4: a tile pair is visited only when it may hold a
                        // pair within reach of the contact range, and only for the nearest r^2
                        const bool far = direct && ((dlo - shift > thr) || (dhi - shift < -thr));
                        if (!far) {
                            if (direct) {
                                const f2 sh = f2_pack(shift, shift);
                                f2 Zs[H];
#pragma unroll
                                for (int h = 0; h < H; ++h) Zs[h] = f2_sub(Z[h], sh);
#pragma unroll 4
                                for (int k = 0; k < NT; ++k) {
                                    const ulonglong2 a = sj2[2 * k], b = sj2[2 * k + 1];
#pragma unroll
                                    for (int h = 0; h < H; ++h)
                                        near_pair_x2<false>(X[h], Y[h], Zs[h], a.x, a.y, b.x, invL2, M2, nM2, nL2,
                                                            mn);
                                }
                            } else {
#pragma unroll 4
                                for (int k = 0; k < NT; ++k) {
                                    const ulonglong2 a = sj2[2 * k], b = sj2[2 * k + 1];
#pragma unroll
                                    for (int h = 0; h < H; ++h)
                                        near_pair_x2<true>(X[h], Y[h], Z[h], a.x, a.y, b.x, invL2, M2, nM2, nL2, mn);
                                }
                            }
                        }
                    } else if (direct) {
                        const f2 sh = f2_pack(shift, shift);
                        f2 Zs[H];
#pragma unroll
                        for (int h = 0; h < H; ++h) Zs[h] = f2_sub(Z[h], sh);
                        // z-separated tiles: every |dz| clears the contact distance by a margin far
                        // above the rounding of dz, so the r^2 clamp is dropped for this tile pair
                        const bool apart = (dlo - shift > thr) || (dhi - shift < -thr);
                        if (apart) {
#pragma unroll 4
                            for (int k = 0; k < NT; ++k) {
                                const ulonglong2 a = sj2[2 * k], b = sj2[2 * k + 1];
#pragma unroll
                                for (int h = 0; h < H; ++h)
                                    coulomb_pair_x2_direct<false>(X[h], Y[h], Zs[h], a.x, a.y, b.x, b.y, (float)c2,
                                                                  AX[h], AY[h], AZ[h], mn);
                            }
                        } else {
#pragma unroll 4
                            for (int k = 0; k < NT; ++k) {
                                const ulonglong2 a = sj2[2 * k], b = sj2[2 * k + 1];
#pragma unroll
                                for (int h = 0; h < H; ++h)
                                    coulomb_pair_x2_direct<true, CT>(X[h], Y[h], Zs[h], a.x, a.y, b.x, b.y,
                                                                     (float)c2, AX[h], AY[h], AZ[h], mn);
                            }
                        }
                    } else {
#pragma unroll 4
                        for (int k = 0; k < NT; ++k) {
                            const ulonglong2 a = sj2[2 * k], b = sj2[2 * k + 1];
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                if constexpr (V == 1) {
                                    float(&sx)[2] = *reinterpret_cast<float(*)[2]>(&ax[2 * h]);
                                    float(&sy)[2] = *reinterpret_cast<float(*)[2]>(&ay[2 * h]);
                                    float(&sz)[2] = *reinterpret_cast<float(*)[2]>(&az[2 * h]);
                                    coulomb_pair_x2s(X[h], Y[h], Z[h], a.x, a.y, b.x, b.y, invL2, M2, nM2, nL2,
                                                     (float)c2, sx, sy, sz);
                                } else {
                                    coulomb_pair_x2<CT>(X[h], Y[h], Z[h], a.x, a.y, b.x, b.y, invL2, M2, nM2, nL2,
                                                        (float)c2, AX[h], AY[h], AZ[h], mn);
                                }
                            }
                        }
                    }
                    if constexpr (CT)
                        flag_tile<P, NT, U, kFlags>(A, mn < thr * thr, j0, nflag, s_flag, base, end, zeta, s_ct);
                    else
                        __syncthreads();
                }
                if constexpr (CT) flush_flags<P, NT, U>(A, nflag, s_flag, base, end, zeta, s_ct);
                if constexpr (V == 6) {       // the Coulomb sums of the Newton-pair kernel
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t g = base + u * NT + tid;
                        if (g < end) { const float4 a = A.acc4[g]; ax[u] = a.x; ay[u] = a.y; az[u] = a.z; }
                    }
                } else if constexpr (V != 1) {
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        float a0, a1;
                        f2_unpack(AX[h], a0, a1); ax[2 * h] = a0; ax[2 * h + 1] = a1;
                        f2_unpack(AY[h], a0, a1); ay[2 * h] = a0; ay[2 * h + 1] = a1;
                        f2_unpack(AZ[h], a0, a1); az[2 * h] = a0; az[2 * h + 1] = a1;
                    }
                }
            } else {
                T4* sj = reinterpret_cast<T4*>(smem_raw);
                // z range of this CTA's i-particles, in FP64 (the tiles of a z-binned sample are narrow)
                {
                    double lo = INFINITY, hi = -INFINITY;
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (base + u * NT + tid < end) { lo = fmin(lo, (double)zi[u]); hi = fmax(hi, (double)zi[u]); }
                    for (int d = 16; d > 0; d >>= 1) {
                        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, d));
                        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, d));
                    }
                    if (lane == 0) s_z64[tid >> 5] = make_double2(lo, hi);
                }
                const double dcz64 = sqrt((double)c2) + 1e-9;    // contact distance + rounding margin
                int64_t jb = o, je = end;
                if (JS > 1) {      // chunk jc of the sample's j range, a whole number of j-tiles long
                    const int64_t ch = ((end - o + JS - 1) / JS + NT - 1) / NT * NT;
                    jb = o + jc * ch;
                    je = jb + ch < end ? jb + ch : end;
                }
                for (int64_t j0 = jb; j0 < je; j0 += NT) {
                    const int64_t j = j0 + tid;
                    T4 pj;
                    if (j < je) pj = pos_in[j];
                    else { pj.x = (T)0; pj.y = (T)0; pj.z = (T)0; pj.w = (T)0; }
                    sj[tid] = pj;
                    if constexpr (CT) stage_speed<P>(A, j, je, lane, tid, s_vj);
                    if constexpr (!CT) {
                        double lo = j < je ? (double)pj.z : INFINITY, hi = j < je ? (double)pj.z : -INFINITY;
                        for (int d = 16; d > 0; d >>= 1) {
                            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, d));
                            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, d));
                        }
                        if (lane == 0) s_z64[NT / 32 + (tid >> 5)] = make_double2(lo, hi);
                    }
                    __syncthreads();
                    if constexpr (CT) {
                        const double thr = (double)near_bound(K, s_vi, s_vj, NT / 32);
                        int mnh = 0x7fffffff;
#pragma unroll 8
                        for (int k = 0; k < NT; ++k) {
                            const T4 p = sj[k];
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                coulomb_pair_track(xi[u], yi[u], zi[u], p, L, invL, c2, ax[u], ay[u], az[u], mnh);
                        }
                        flag_tile<P, NT, U, kFlags>(A, mnh <= __double2hiint(thr * thr), j0, nflag, s_flag, base, end,
                                                    zeta, s_ct);
                    } else {
                        // as the MIXED path: a tile pair inside one period window takes a uniform
                        // shift instead of the per-pair minimum image, and z-separated tile pairs
                        // (every |dz| beyond the contact distance) skip the clamp
                        double alo = INFINITY, ahi = -INFINITY, blo = INFINITY, bhi = -INFINITY;
#pragma unroll
                        for (int w = 0; w < NT / 32; ++w) {
                            alo = fmin(alo, s_z64[w].x); ahi = fmax(ahi, s_z64[w].y);
                            blo = fmin(blo, s_z64[NT / 32 + w].x); bhi = fmax(bhi, s_z64[NT / 32 + w].y);
                        }
                        const double dlo = alo - bhi, dhi = ahi - blo, halfL = 0.5 * (double)L;
                        double shift = 0.0;
                        bool direct = true;
                        if (dlo > -halfL && dhi < halfL) shift = 0.0;
                        else if (dlo > halfL && dhi < 3.0 * halfL) shift = (double)L;
                        else if (dhi < -halfL && dlo > -3.0 * halfL) shift = -(double)L;
                        else direct = false;
                        if (direct) {
                            T zs[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) zs[u] = zi[u] - (T)shift;
                            if ((dlo - shift > dcz64) || (dhi - shift < -dcz64)) {
#pragma unroll 8
                                for (int k = 0; k < NT; ++k) {
                                    const T4 p = sj[k];
#pragma unroll
                                    for (int u = 0; u < U; ++u)
                                        coulomb_pair_direct64<false>(xi[u], yi[u], zs[u], p, c2, ax[u], ay[u], az[u]);
                                }
                            } else {
#pragma unroll 8
                                for (int k = 0; k < NT; ++k) {
                                    const T4 p = sj[k];
#pragma unroll
                                    for (int u = 0; u < U; ++u)
                                        coulomb_pair_direct64<true>(xi[u], yi[u], zs[u], p, c2, ax[u], ay[u], az[u]);
                                }
                            }
                        } else {
#pragma unroll 8
                            for (int k = 0; k < NT; ++k) {
                                const T4 p = sj[k];
#pragma unroll
                                for (int u = 0; u < U; ++u)
                                    coulomb_pair(xi[u], yi[u], zi[u], p, L, invL, c2, ax[u], ay[u], az[u]);
                            }
                        }
                        __syncthreads();
                    }
                }
                if constexpr (CT) flush_flags<P, NT, U>(A, nflag, s_flag, base, end, zeta, s_ct);
            }
        }
        if constexpr (P == PDQ_FP64 && V != 5) {
            if (JS > 1) {
                double* part = A.part;
                const int64_t cap = A.cap;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t g = base + u * NT + tid;
                    if (g < end) {
                        part[(jc * 3 + 0) * cap + g] = ax[u];
                        part[(jc * 3 + 1) * cap + g] = ay[u];
                        part[(jc * 3 + 2) * cap + g] = az[u];
                    }
                }
                __threadfence();
                __syncthreads();
                if (tid == 0) s_last = atomicAdd(&A.tile_cnt[item / JS], 1) == JS - 1;
                __syncthreads();
                if (!s_last) continue;          // another chunk of this tile finishes it
                __threadfence();
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t g = base + u * NT + tid;
                    if (g < end) {
                        double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll 4
                        for (int c = 0; c < JS; ++c) {
                            sx += __ldcg(&part[(c * 3 + 0) * cap + g]);
                            sy += __ldcg(&part[(c * 3 + 1) * cap + g]);
                            sz += __ldcg(&part[(c * 3 + 2) * cap + g]);
                        }
                        ax[u] = sx; ay[u] = sy; az[u] = sz;
                    }
                }
                if (tid == 0) A.tile_cnt[item / JS] = 0;
            }
        }
        const pdq_sample_params sp = A.params[s];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * NT + tid;
            int cls = -1;
            bool was_alive = false, dep = false;
            if (g < end) {
                if constexpr (CT)
                    local_update<P, true>(A, g, ax[u], ay[u], az[u], sp, cls, was_alive, dep, s_ct[(0 * U + u) * NT + tid],
                                    s_ct[(1 * U + u) * NT + tid], s_ct[(2 * U + u) * NT + tid]);
                else
                    local_update<P>(A, g, ax[u], ay[u], az[u], sp, cls, was_alive, dep);
            }
            if (counted) {
                const unsigned live = __ballot_sync(0xffffffffu, was_alive);
                if (live) {
                    const unsigned dm = __ballot_sync(0xffffffffu, dep);
                    for (int c = 0; c < C; ++c) {
                        const unsigned m = __ballot_sync(0xffffffffu, cls == c);
                        const unsigned na = __popc(m & live), nd = __popc(m & dm);
                        if (lane == 0) {
                            if (na) atomicAdd(&s_alive[c], na);
                            if (nd) atomicAdd(&s_dep[c], nd);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (counted && tid < C) {
            if (s_alive[tid]) atomicAdd(&A.n_alive[(int64_t)s * C + tid], (unsigned long long)s_alive[tid]);
            if (s_dep[tid]) atomicAdd(&A.n_dep[(int64_t)s * C + tid], (unsigned long long)s_dep[tid]);
        }
    }
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd((unsigned long long*)&A.ctl[CTL_DONE], 1ull);
        if (prev == gridDim.x - 1) {   // last CTA: advance the step, reset the queue
            A.ctl[CTL_QUEUE] = 0;
            A.ctl[CTL_DONE] = 0;
            A.ctl[CTL_STEP] = step + 1;
            __threadfence();
        }
    }
}

// Coulomb sums of pair variant 3 into A.acc4 (zeroed before the launch); the given-sums step
// then does the local update.  One CTA per (sample, i-tile) item of the table k_build_items
// sorted heaviest first; the grid covers the host's bound on the item count and CTAs past the
// device count return at once.  The hardware hands out CTAs in index order as SMs free up,
// which balances the triangular per-tile work like a queue would: a persistent CTA looping
// over a queue measured ~5 more register moves per packed pair evaluation in the hot loop.
// Each CTA sums its tile's pairs with newton_tile (Newton pairs between the warps' blocks of the
// tile and with every later particle of the sample; one-sided only within a warp's block).
// Register budget: 3 CTAs of 128 threads per SM (168 registers) for 12 particles per thread (8 per
// thread ran 1 % faster at 4 CTAs and 128 registers than at 3), 6 CTAs of 64.
template <int NT, int U>
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 6) k_pairs_sym(const StepArgs A) {
    const int item = blockIdx.x;
    if (item >= A.ctl[CTL_NITEMS]) return;
    const float4* __restrict__ pos_in = (const float4*)A.pos_in;
    const auto load = [&](int64_t g) { return pos_in[g]; };
    const int2 it = A.items[item];
    const int64_t o = A.offset[it.x];
    const int64_t end = o + A.count[it.x];
    const int64_t base = o + (int64_t)it.y * (NT * U);
    newton_tile<NT, U>(load, base, end, (float)A.K.L, (float)A.K.invL, (float)A.K.contact2f, A.acc4);
}

// FP64 Newton pair: coulomb_pair_x2_sym for one i-particle in double (minimum image by the
// 1.5 * 2^52 rounding constant, as the one-sided FP64 pair).
template <bool MINIMG, bool CLAMP>
__device__ __forceinline__ void coulomb_pair_sym64(double xi, double yi, double zi, double nqi, double2 xyj,
                                                   double2 zqj, double L, double invL, double c2, double& ax,
                                                   double& ay, double& az, double& jx, double& jy, double& jz) {
    const double dx = xi - xyj.x, dy = yi - xyj.y;
    double dz = zi - zqj.x;
    if constexpr (MINIMG) {
        const double t = __dadd_rn(__fma_rn(dz, invL, 6755399441055744.0), -6755399441055744.0);
        dz = __fma_rn(-L, t, dz);
    }
    double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, dz * dz));
    if constexpr (CLAMP) r2 = fmax(r2, c2);
    const double ri = rsqrt(r2);
    const double ri3 = ri * (ri * ri);
    const double si = zqj.y * ri3, sj = nqi * ri3;
    ax = __fma_rn(si, dx, ax);
    ay = __fma_rn(si, dy, ay);
    az = __fma_rn(si, dz, az);
    jx = __fma_rn(sj, dx, jx);
    jy = __fma_rn(sj, dy, jy);
    jz = __fma_rn(sj, dz, jz);
}

// Pair variant 3 in FP64: k_pairs_sym's scheme with U particles per thread (no packing) and the
// sums in double through atomics into A.acc64 [cap][3] (zeroed before the launch).  A single
// large sample gives few i-tiles with triangular work, so each tile's j range is cut into
// A.jsplit chunks of whole j-tiles, one work item each (item.y = tile * JS + chunk; chunks that
// end before the tile are empty items).
template <int NT, int U>
__global__ void __launch_bounds__(NT) k_pairs_sym64(const StepArgs A) {
    constexpr int W = NT / 32;
    static_assert(NT % 32 == 0, "whole warps");
    __shared__ __align__(16) double2 s_xy[NT];     // staged j: (x, y) and (z, q) apart, 16-byte strides
    __shared__ __align__(16) double2 s_zq[NT];
    __shared__ double s_jacc[W][3][NT];
    __shared__ double2 s_zr[W];
    __shared__ int s_item;
    const StepConst& K = A.K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_items = A.ctl[CTL_NITEMS];
    const double4_32a* __restrict__ pos_in = (const double4_32a*)A.pos_in;
    const double L = K.L, invL = K.invL, c2 = K.contact2;
    const double dcz = sqrt(c2) + 1e-9;        // contact distance + rounding margin
    const int JS = A.jsplit;
    double* __restrict__ acc = A.acc64;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd((unsigned long long*)&A.ctl[CTL_QUEUE2], 1ull);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int2 it = A.items[item];
        const int64_t o = A.offset[it.x];
        const int64_t end = o + A.count[it.x];
        const int tile = it.y / JS, jc = it.y - tile * JS;
        const int64_t base = o + (int64_t)tile * (NT * U);
        const int64_t dend = base + NT * U < end ? base + NT * U : end;
        int64_t jb = base, je = end;
        if (JS > 1) {      // chunk jc of the sample, a whole number of j-tiles long, from this tile on
            const int64_t ch = ((end - o + JS - 1) / JS + NT - 1) / NT * NT;
            const int64_t cb = o + jc * ch, ce = cb + ch < end ? cb + ch : end;
            jb = cb > base ? cb : base;
            je = ce;
        }
        if (jb >= je) {    // the chunk lies before this tile (uniform across the CTA)
            __syncthreads();
            continue;
        }
        double xi[U], yi[U], zi[U], nq[U], ax[U], ay[U], az[U];
        double ilo = INFINITY, ihi = -INFINITY;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * NT + tid;
            if (g < end) {
                const double4_32a p = pos_in[g];
                xi[u] = p.x; yi[u] = p.y; zi[u] = p.z; nq[u] = -p.w;
                ilo = fmin(ilo, p.z);
                ihi = fmax(ihi, p.z);
            } else {
                xi[u] = 1e15; yi[u] = 0.0; zi[u] = 0.0; nq[u] = 0.0;
            }
            ax[u] = ay[u] = az[u] = 0.0;
        }
        for (int d = 16; d > 0; d >>= 1) {
            ilo = fmin(ilo, __shfl_xor_sync(0xffffffffu, ilo, d));
            ihi = fmax(ihi, __shfl_xor_sync(0xffffffffu, ihi, d));
        }
        for (int64_t j0 = jb; j0 < je; j0 += NT) {
            const bool diag = j0 < dend;
            const int64_t jlim = diag ? (dend < je ? dend : je) : je;
            const int64_t j = j0 + tid;
            double2 xy = make_double2(-1e15, 0.0), zq = make_double2(0.0, 0.0);
            if (j < jlim) {
                const double4_32a p = pos_in[j];
                xy = make_double2(p.x, p.y);
                zq = make_double2(p.z, p.w);
            }
            double jlo = j < jlim ? zq.x : INFINITY, jhi = j < jlim ? zq.x : -INFINITY;
            for (int d = 16; d > 0; d >>= 1) {
                jlo = fmin(jlo, __shfl_xor_sync(0xffffffffu, jlo, d));
                jhi = fmax(jhi, __shfl_xor_sync(0xffffffffu, jhi, d));
            }
            if (lane == 0) s_zr[warp] = make_double2(jlo, jhi);
            s_xy[tid] = xy;
            s_zq[tid] = zq;
            __syncthreads();
            const double halfL = 0.5 * L;
            auto classify = [&](double blo, double bhi, bool& direct, bool& apart, double& shift) {
                const double dlo = ilo - bhi, dhi = ihi - blo;
                direct = true;
                shift = 0.0;
                if (dlo > -halfL && dhi < halfL) shift = 0.0;
                else if (dlo > halfL && dhi < 3.0 * halfL) shift = L;
                else if (dhi < -halfL && dlo > -3.0 * halfL) shift = -L;
                else direct = false;
                apart = direct && ((dlo - shift > dcz) || (dhi - shift < -dcz));
            };
            if (diag) {
                // one-sided over the tile's own particles (self pair: d = 0 adds nothing)
                double blo = INFINITY, bhi = -INFINITY;
#pragma unroll
                for (int w = 0; w < W; ++w) { blo = fmin(blo, s_zr[w].x); bhi = fmax(bhi, s_zr[w].y); }
                bool direct, apart;
                double shift;
                classify(blo, bhi, direct, apart, shift);
                if (direct) {
                    double zs[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) zs[u] = zi[u] - shift;
#pragma unroll 4
                    for (int k = 0; k < NT; ++k) {
                        const double2 a = s_xy[k], b = s_zq[k];
                        const double4_32a pj = make_double4_32a(a.x, a.y, b.x, b.y);
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            coulomb_pair_direct64<true>(xi[u], yi[u], zs[u], pj, c2, ax[u], ay[u], az[u]);
                    }
                } else {
#pragma unroll 4
                    for (int k = 0; k < NT; ++k) {
                        const double2 a = s_xy[k], b = s_zq[k];
                        const double4_32a pj = make_double4_32a(a.x, a.y, b.x, b.y);
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            coulomb_pair(xi[u], yi[u], zi[u], pj, L, invL, c2, ax[u], ay[u], az[u]);
                    }
                }
                __syncthreads();
                continue;
            }
#pragma unroll 1
            for (int g = 0; g < W; ++g) {
                bool direct, apart;
                double shift;
                classify(s_zr[g].x, s_zr[g].y, direct, apart, shift);
                double jx = 0.0, jy = 0.0, jz = 0.0;
                auto group = [&](auto minimg, auto clamp, const double* zt) {
#pragma unroll 2
                    for (int k = 0; k < 32; ++k) {
                        const int jj = g * 32 + ((lane + k) & 31);
                        const double2 a = s_xy[jj], b = s_zq[jj];
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            coulomb_pair_sym64<decltype(minimg)::value, decltype(clamp)::value>(
                                xi[u], yi[u], zt[u], nq[u], a, b, L, invL, c2, ax[u], ay[u], az[u], jx, jy, jz);
                        jx = __shfl_sync(0xffffffffu, jx, (lane + 1) & 31);
                        jy = __shfl_sync(0xffffffffu, jy, (lane + 1) & 31);
                        jz = __shfl_sync(0xffffffffu, jz, (lane + 1) & 31);
                    }
                };
                if (direct) {
                    double zs[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) zs[u] = zi[u] - shift;
                    if (apart) group(std::false_type{}, std::false_type{}, zs);
                    else group(std::false_type{}, std::true_type{}, zs);
                } else {
                    group(std::true_type{}, std::true_type{}, zi);
                }
                s_jacc[warp][0][g * 32 + lane] = jx;
                s_jacc[warp][1][g * 32 + lane] = jy;
                s_jacc[warp][2][g * 32 + lane] = jz;
            }
            __syncthreads();
            if (j < je) {
                double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
                for (int w = 0; w < W; ++w) { sx += s_jacc[w][0][tid]; sy += s_jacc[w][1][tid]; sz += s_jacc[w][2][tid]; }
                atomicAdd(&acc[3 * j], sx);
                atomicAdd(&acc[3 * j + 1], sy);
                atomicAdd(&acc[3 * j + 2], sz);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = base + u * NT + tid;
            if (g < end) {
                atomicAdd(&acc[3 * g], ax[u]);
                atomicAdd(&acc[3 * g + 1], ay[u]);
                atomicAdd(&acc[3 * g + 2], az[u]);
            }
        }
    }
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd((unsigned long long*)&A.ctl[CTL_DONE2], 1ull);
        if (prev == gridDim.x - 1) {
            A.ctl[CTL_QUEUE2] = 0;
            A.ctl[CTL_DONE2] = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Work items: samples ordered by live count (largest first), JS items per i-tile
// (one per j-chunk; JS = 1 unless the FP64 j-split is on), item.y = tile * JS + chunk.
// Single CTA of 1024 threads; order[] and items[] live in the caller workspace.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_buf, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_buf[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? warp_buf[lane] : 0;
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += t;
        }
        if (lane < nw) warp_buf[lane] = wi - w;
        if (lane == 31) warp_buf[32] = wi;
    }
    __syncthreads();
    const int ex = warp_buf[warp] + incl - v;
    total = warp_buf[32];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(1024) k_build_items(const int32_t* __restrict__ count, int S, int TI, int JS,
                                                      int32_t* __restrict__ order, int2* __restrict__ items,
                                                      int64_t* __restrict__ ctl) {
    __shared__ int warp_buf[33];
    const int tid = threadIdx.x;
    for (int s = tid; s < S; s += blockDim.x) {
        if (S <= 8192) {
            const int cs = count[s];
            int rank = 0;
            for (int t = 0; t < S; ++t) {
                const int ct = count[t];
                rank += (ct > cs) || (ct == cs && t < s);
            }
            order[rank] = s;
        } else {
            order[s] = s;
        }
    }
    __syncthreads();
    int64_t running = 0;
    for (int k0 = 0; k0 < S; k0 += blockDim.x) {
        const int k = k0 + tid;
        const int sidx = k < S ? order[k] : 0;
        const int nt = k < S ? (count[sidx] + TI - 1) / TI * JS : 0;
        int total;
        const int pre = block_exclusive_scan(nt, warp_buf, total);
        for (int t = 0; t < nt; ++t) items[running + pre + t] = make_int2(sidx, t);
        running += total;
    }
    if (tid == 0) {
        ctl[CTL_NITEMS] = running;
        ctl[CTL_QUEUE] = 0;
        ctl[CTL_DONE] = 0;
        ctl[CTL_QUEUE2] = 0;
        ctl[CTL_DONE2] = 0;
    }
}

// ---------------------------------------------------------------------------
// Compaction: one CTA per sample, chunks of blockDim particles in order; all
// loads of a chunk precede its writes, and writes land at or before the read
// position, so the in-place pass is stable and race-free.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(1024) k_compact(void* pos, void* vel, double2* xy, int2* tag,
                                                  const int64_t* __restrict__ offset, int32_t* __restrict__ count) {
    typedef typename Real<P>::T4 T4;
    __shared__ int warp_buf[33];
    const int s = blockIdx.x;
    const int64_t o = offset[s];
    const int n = count[s];
    int out = 0;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        T4 p = {}, v = {};
        double2 w = make_double2(0.0, 0.0);
        int2 tg = make_int2(0, 0);
        bool alive = false;
        if (i < n) {
            p = ((T4*)pos)[o + i];
            v = ((T4*)vel)[o + i];
            if (P == PDQ_MIXED) w = xy[o + i];
            tg = tag[o + i];
            alive = v.w > 0.5;
        }
        int total;
        const int pre = block_exclusive_scan(alive ? 1 : 0, warp_buf, total);
        if (alive) {
            const int64_t d = o + out + pre;
            ((T4*)pos)[d] = p;
            ((T4*)vel)[d] = v;
            if (P == PDQ_MIXED) xy[d] = w;
            tag[d] = tg;
        }
        out += total;
    }
    if (threadIdx.x == 0) count[s] = out;
}

// ---------------------------------------------------------------------------
// z-binning: one CTA per sample copies the particles of the current half into
// the other half, grouped by 256 bins of z and in their previous order inside a
// bin (a stable counting sort: histogram, bin bases, then chunks in order with
// ranks from __match_any_sync).  With `compact` the removed particles are left
// out (a compaction); without, they are binned like the others and the count is
// unchanged.  Tiles of a binned sample cover short z-intervals, which lets the
// step skip the per-pair minimum image for most tile pairs.  Tags go to
// `tag_out` (scratch).
// ---------------------------------------------------------------------------
constexpr int kZBins = 256;

template <int P>
__global__ void __launch_bounds__(1024) k_sort_compact(const void* __restrict__ pos_in_, const void* __restrict__ vel_in_,
                                                       const double2* __restrict__ xy_in, const int2* __restrict__ tag_in,
                                                       void* __restrict__ pos_out_, void* __restrict__ vel_out_,
                                                       double2* __restrict__ xy_out, int2* __restrict__ tag_out,
                                                       const int64_t* __restrict__ offset, int32_t* __restrict__ count,
                                                       float bins_per_length, int compact) {
    typedef typename Real<P>::T4 T4;
    const T4* pos_in = (const T4*)pos_in_;
    const T4* vel_in = (const T4*)vel_in_;
    T4* pos_out = (T4*)pos_out_;
    T4* vel_out = (T4*)vel_out_;
    __shared__ int base[kZBins];
    __shared__ int running[kZBins];
    __shared__ int wcnt[32][kZBins];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = offset[s];
    const int n = count[s];
    auto bin_of = [&](const T4& p, const T4& v) -> int {
        if (compact && !((double)v.w > 0.5)) return -1;
        const float zb = (float)p.z * bins_per_length;
        return isfinite(zb) ? min(kZBins - 1, max(0, (int)zb)) : 0;
    };
    for (int b = tid; b < kZBins; b += blockDim.x) { base[b] = 0; running[b] = 0; }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        const int b = bin_of(pos_in[o + i], vel_in[o + i]);
        if (b >= 0) atomicAdd(&base[b], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int b = 0; b < kZBins; ++b) { const int h = base[b]; base[b] = acc; acc += h; }
        count[s] = acc;
    }
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        for (int q = tid; q < 32 * kZBins; q += blockDim.x) (&wcnt[0][0])[q] = 0;
        const int i = c0 + tid;
        T4 p = {}, v = {};
        double2 w = make_double2(0.0, 0.0);
        int2 tg = make_int2(0, 0);
        int b = -1;
        if (i < n) {
            p = pos_in[o + i];
            v = vel_in[o + i];
            if (P == PDQ_MIXED) w = xy_in[o + i];
            tg = tag_in[o + i];
            b = bin_of(p, v);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        __syncthreads();                                   // wcnt cleared
        if (b >= 0 && rank == 0) wcnt[warp][b] = __popc(peers);
        __syncthreads();
        if (tid < kZBins) {                                // per bin: offsets of the warps, in warp order
            int acc = running[tid];
            for (int q = 0; q < 32; ++q) { const int c = wcnt[q][tid]; wcnt[q][tid] = acc; acc += c; }
            running[tid] = acc;
        }
        __syncthreads();
        if (b >= 0) {
            const int64_t d = o + base[b] + wcnt[warp][b] + rank;
            pos_out[d] = p;
            vel_out[d] = v;
            if (P == PDQ_MIXED) xy_out[d] = w;
            tag_out[d] = tg;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Deposition velocity per (sample, class) and the Monte Carlo mean / SE.
// ---------------------------------------------------------------------------
__global__ void k_vdep(const int64_t* __restrict__ nd, const int64_t* __restrict__ na, int n, double scale,
                       double* __restrict__ vdep) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) vdep[k] = na[k] > 0 ? scale * (double)nd[k] / (double)na[k] : 0.0;
}

// One warp per class: lane-strided FP64 sums, then a fixed shuffle tree (deterministic).
__global__ void k_vdep_stats(const double* __restrict__ vdep, int S, int C, double* mean, double* se) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double s1 = 0.0;
    for (int s = lane; s < S; s += 32) s1 += vdep[(int64_t)s * C + c];
    for (int d = 16; d > 0; d >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, d);
    const double mu = s1 / S;
    double s2 = 0.0;
    for (int s = lane; s < S; s += 32) {
        const double e = vdep[(int64_t)s * C + c] - mu;
        s2 += e * e;
    }
    for (int d = 16; d > 0; d >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, d);
    if (lane == 0) {
        if (mean) mean[c] = mu;
        if (se) se[c] = S > 1 ? sqrt(s2 / (S - 1) / S) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host helpers.
// ---------------------------------------------------------------------------
static int validate_state(const pdq_state* st) {
    if (!st || st->n_samples < 1 || st->n_classes < 1 || st->n_classes > PDQ_MAX_CLASSES || st->capacity < 0 ||
        st->capacity > ((int64_t)1 << 31) - 1 || !st->offset || !st->count || !st->tag || !st->ctl ||
        (st->cur != 0 && st->cur != 1))
        return PDQ_ERR_INVALID_ARG;
    if (st->precision != PDQ_FP64 && st->precision != PDQ_MIXED) return PDQ_ERR_INVALID_ARG;
    for (int h = 0; h < 2; ++h) {
        if (!st->pos[h] || !st->vel[h]) return PDQ_ERR_INVALID_ARG;
        if (st->precision == PDQ_MIXED && !st->xy[h]) return PDQ_ERR_INVALID_ARG;
    }
    return PDQ_OK;
}

static int tile_threads(const pdq_state* st, const pdq_step_cfg* cfg) {
    if (cfg && cfg->block) return cfg->block;
    return st->precision == PDQ_FP64 ? 128 : 128;
}
// Pair variant 3 (Newton pairs): both precisions; with contact forces MIXED only (its contact
// forces stay in the contact variant of k_step, V = 6).
static bool newton_pairs(const pdq_state* st, const pdq_step_cfg* cfg) {
    return cfg && cfg->variant == 3 && (!(cfg->forces & PDQ_F_CONTACT) || st->precision == PDQ_MIXED);
}
// particles per thread: FP64 1 (2 for its Newton-pair kernel); MIXED 4 (two packed pairs), 8 for
// pair variant 2, 12 for pair variant 3 (8 with contact forces: their update runs 4 per thread
// over 2 NT threads); 12 gave 1.2 % over 8 (six packed calls share each step's shared loads and
// shuffles) at 3 CTAs of 128 threads per SM
static int tile_ilp(const pdq_state* st, const pdq_step_cfg* cfg = nullptr) {
    if (st->precision == PDQ_FP64) return newton_pairs(st, cfg) ? 2 : 1;
    if (newton_pairs(st, cfg)) return (cfg->forces & PDQ_F_CONTACT) ? 8 : 12;
    if (cfg && (cfg->forces & PDQ_F_CONTACT)) return 4;      // contact runs: variant 0 layout
    return (cfg && cfg->variant == 2) ? 8 : 4;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int P, int NT, int U, int V>
static int launch_step(const StepArgs& A, cudaStream_t s) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<P, NT, U, V>, NT, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    const int64_t full = (int64_t)sm_count() * per_sm;
    k_step<P, NT, U, V><<<(unsigned)std::max<int64_t>(1, std::min(full, A.max_items > 0 ? A.max_items : full)), NT, 0,
                          s>>>(A);
    return PDQ_OK;
}

// Pair variant 3: the Newton-pair sums (NT threads, 12 particles per thread) into A.acc4, then
// the given-sums step over the same tiles (2 NT threads, 6 particles per thread; with contact forces
// the sums take 8 per thread and the contact variant 4 per thread over 2 NT threads).
template <int NT>
static int launch_newton64(const StepArgs& A, cudaStream_t s) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_sym64<NT, 2>, NT, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    const int64_t full = (int64_t)sm_count() * per_sm;
    PDQ_CUDA(cudaMemsetAsync(A.acc64, 0, 3 * sizeof(double) * (size_t)(A.cap > 0 ? A.cap : 1), s));
    if (A.K.forces & PDQ_F_COULOMB) {    // the sums enter the update only with the Coulomb force on
        k_pairs_sym64<NT, 2><<<(unsigned)std::max<int64_t>(1, std::min(full, A.max_items > 0 ? A.max_items : full)),
                               NT, 0, s>>>(A);
    }
    StepArgs B = A;
    B.ext = A.acc64;
    return launch_step<PDQ_FP64, 2 * NT, 1, 5>(B, s);
}
// MIXED contact runs under pair variant 3: the Newton-pair sums, then the contact variant of the
// step that takes them from A.acc4 (V = 6) over the same tiles.
template <int NT>
static int launch_newton_contact(const StepArgs& A, cudaStream_t s) {
    PDQ_CUDA(cudaMemsetAsync(A.acc4, 0, sizeof(float4) * (size_t)(A.cap > 0 ? A.cap : 1), s));
    if (A.K.forces & PDQ_F_COULOMB)      // the sums enter the update only with the Coulomb force on
        k_pairs_sym<NT, 8><<<(unsigned)std::max<int64_t>(1, A.max_items), NT, 0, s>>>(A);
    return launch_step<PDQ_MIXED, 2 * NT, 4, 6>(A, s);
}
template <int NT>
static int launch_newton(const StepArgs& A, cudaStream_t s) {
    PDQ_CUDA(cudaMemsetAsync(A.acc4, 0, sizeof(float4) * (size_t)(A.cap > 0 ? A.cap : 1), s));
    if (A.K.forces & PDQ_F_COULOMB)      // the sums enter the update only with the Coulomb force on
        k_pairs_sym<NT, 12><<<(unsigned)std::max<int64_t>(1, A.max_items), NT, 0, s>>>(A);
    return launch_step<PDQ_MIXED, 2 * NT, 6, 5>(A, s);
}

// variant: MIXED pair math, 0 = all packed f32x2, 1 = packed with scalar accumulation,
// 2 = as 0 with 8 particles per thread, 3 = Newton pairs (A.acc4 set: k_pairs_sym, then the
// given-sums step, or with contact the contact variant that takes the sums).
// contact: the particle-particle contact variant (V = 4), whatever the variant; given
// Coulomb sums (A.ext, P3M): V = 5, no pair loop.
static int dispatch_step(int prec, int NT, int variant, bool contact, const StepArgs& A, cudaStream_t s) {
    if (A.acc4) {
        if (NT == 64) return contact ? launch_newton_contact<64>(A, s) : launch_newton<64>(A, s);
        if (NT == 128) return contact ? launch_newton_contact<128>(A, s) : launch_newton<128>(A, s);
        return PDQ_ERR_INVALID_ARG;
    }
    if (A.acc64) {
        if (NT == 64) return launch_newton64<64>(A, s);
        if (NT == 128) return launch_newton64<128>(A, s);
        return PDQ_ERR_INVALID_ARG;
    }
    if (A.ext) {
        if (prec == PDQ_FP64) {
            if (NT == 32) return launch_step<PDQ_FP64, 32, 1, 5>(A, s);
            if (NT == 64) return launch_step<PDQ_FP64, 64, 1, 5>(A, s);
            if (NT == 128) return launch_step<PDQ_FP64, 128, 1, 5>(A, s);
            if (NT == 256) return launch_step<PDQ_FP64, 256, 1, 5>(A, s);
        } else {
            if (NT == 64) return launch_step<PDQ_MIXED, 64, 4, 5>(A, s);
            if (NT == 128) return launch_step<PDQ_MIXED, 128, 4, 5>(A, s);
            if (NT == 256) return launch_step<PDQ_MIXED, 256, 4, 5>(A, s);
        }
        return PDQ_ERR_INVALID_ARG;
    }
    if (contact) {
        if (prec == PDQ_FP64) {
            if (NT == 32) return launch_step<PDQ_FP64, 32, 1, 4>(A, s);
            if (NT == 64) return launch_step<PDQ_FP64, 64, 1, 4>(A, s);
            if (NT == 128) return launch_step<PDQ_FP64, 128, 1, 4>(A, s);
            if (NT == 256) return launch_step<PDQ_FP64, 256, 1, 4>(A, s);
        } else {
            if (NT == 64) return launch_step<PDQ_MIXED, 64, 4, 4>(A, s);
            if (NT == 128) return launch_step<PDQ_MIXED, 128, 4, 4>(A, s);
            if (NT == 256) return launch_step<PDQ_MIXED, 256, 4, 4>(A, s);
        }
        return PDQ_ERR_INVALID_ARG;
    }
    if (prec == PDQ_FP64) {
        if (NT == 32) return launch_step<PDQ_FP64, 32, 1, 0>(A, s);
        if (NT == 64) return launch_step<PDQ_FP64, 64, 1, 0>(A, s);
        if (NT == 128) return launch_step<PDQ_FP64, 128, 1, 0>(A, s);
        if (NT == 256) return launch_step<PDQ_FP64, 256, 1, 0>(A, s);
    } else if (variant == 1) {
        if (NT == 64) return launch_step<PDQ_MIXED, 64, 4, 1>(A, s);
        if (NT == 128) return launch_step<PDQ_MIXED, 128, 4, 1>(A, s);
        if (NT == 256) return launch_step<PDQ_MIXED, 256, 4, 1>(A, s);
    } else if (variant == 2) {          // packed pairs, 8 particles per thread
        if (NT == 64) return launch_step<PDQ_MIXED, 64, 8, 0>(A, s);
        if (NT == 128) return launch_step<PDQ_MIXED, 128, 8, 0>(A, s);
        if (NT == 256) return launch_step<PDQ_MIXED, 256, 8, 0>(A, s);
    } else {
        if (NT == 64) return launch_step<PDQ_MIXED, 64, 4, 0>(A, s);
        if (NT == 128) return launch_step<PDQ_MIXED, 128, 4, 0>(A, s);
        if (NT == 256) return launch_step<PDQ_MIXED, 256, 4, 0>(A, s);
    }
    return PDQ_ERR_INVALID_ARG;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// FP64 j-split factor.  The FP64 pipe is narrow and split over the four schedulers
// of an SM, so the step wants about 1024 busy warps (~7 per SM) however few
// particles there are; when the i-tiles alone give fewer, each tile's pair sum is
// spread over JS work items (j-chunks of at least one j-tile).  MIXED never splits
// (its batches have thousands of tiles); neither do contact runs.
static int j_split(const pdq_state* st, int TI, bool contact = false) {
    if (st->precision != PDQ_FP64 || contact) return 1;
    const int64_t cap = st->capacity > 0 ? st->capacity : 1;
    const int64_t tile_warps = (cap + TI - 1) / TI * ((TI + 31) / 32);
    int64_t js = (1024 + tile_warps - 1) / tile_warps;
    const int64_t max_js = (cap + TI - 1) / TI;       // chunks are whole j-tiles of TI particles
    if (js > max_js) js = max_js;
    if (js > 64) js = 64;
    return js < 1 ? 1 : (int)js;
}

// FP64 Newton pairs: j-chunks per tile so that the triangular work of few large samples spreads
// evenly (about 8 i-tiles of j per chunk, at most 64 chunks).
static int newton_chunks(const pdq_state* st, int TI) {
    if (st->precision != PDQ_FP64) return 1;
    const int64_t cap = st->capacity > 0 ? st->capacity : 1;
    int64_t js = (cap + 8 * (int64_t)TI - 1) / (8 * (int64_t)TI);
    if (js > 64) js = 64;
    return js < 1 ? 1 : (int)js;
}

// Workspace: items | order | tag scratch of the z-binning sort;
// FP64 with JS > 1 (one-sided): tile counters | partial sums [JS][3][capacity];
// pair variant 3: the sums, float4 [capacity] (MIXED) or double [capacity][3] (FP64).
static void workspace_layout(const pdq_state* st, int TI, size_t* items_bytes, size_t* total,
                             size_t* cnt_off = nullptr, size_t* part_off = nullptr, bool contact = false,
                             size_t* acc_off = nullptr, bool newton = false) {
    const int JS = newton ? newton_chunks(st, TI) : j_split(st, TI, contact);
    const int64_t max_tiles = st->capacity / TI + st->n_samples + 1;
    *items_bytes = align256(sizeof(int2) * (size_t)max_tiles * JS);
    *total = *items_bytes + align256(sizeof(int32_t) * (size_t)st->n_samples);
    *total += align256(sizeof(int2) * (size_t)(st->capacity > 0 ? st->capacity : 1));   // tag scratch of the z-binning
    if (newton) {
        if (acc_off) *acc_off = *total;
        const size_t per = st->precision == PDQ_FP64 ? 3 * sizeof(double) : sizeof(float4);
        *total += align256(per * (size_t)(st->capacity > 0 ? st->capacity : 1));
    }
    if (JS > 1 && !newton) {
        if (cnt_off) *cnt_off = *total;
        *total += align256(sizeof(int) * (size_t)max_tiles);
        if (part_off) *part_off = *total;
        *total += align256(sizeof(double) * 3 * (size_t)JS * (size_t)st->capacity);
    }
}

// z-binning (with or without compaction) from the current half into the other half, tags
// through the workspace scratch, then flip the current half.
static int enqueue_sort_compact(pdq_state* st, int2* tag_scratch, float bins_per_length, bool compact,
                                cudaStream_t s) {
    const int h = st->cur;
    if (st->precision == PDQ_FP64)
        k_sort_compact<PDQ_FP64><<<st->n_samples, 1024, 0, s>>>(st->pos[h], st->vel[h], nullptr, (const int2*)st->tag,
                                                                st->pos[h ^ 1], st->vel[h ^ 1], nullptr, tag_scratch,
                                                                st->offset, st->count, bins_per_length, (int)compact);
    else
        k_sort_compact<PDQ_MIXED><<<st->n_samples, 1024, 0, s>>>(
            st->pos[h], st->vel[h], (const double2*)st->xy[h], (const int2*)st->tag, st->pos[h ^ 1], st->vel[h ^ 1],
            (double2*)st->xy[h ^ 1], tag_scratch, st->offset, st->count, bins_per_length, (int)compact);
    PDQ_CUDA(cudaMemcpyAsync(st->tag, tag_scratch, sizeof(int2) * (size_t)st->capacity, cudaMemcpyDeviceToDevice, s));
    st->cur = h ^ 1;
    return PDQ_OK;
}

static int enqueue_compact(pdq_state* st, cudaStream_t s) {
    const int h = st->cur;
    if (st->precision == PDQ_FP64)
        k_compact<PDQ_FP64><<<st->n_samples, 1024, 0, s>>>(st->pos[h], st->vel[h], nullptr, (int2*)st->tag,
                                                          st->offset, st->count);
    else
        k_compact<PDQ_MIXED><<<st->n_samples, 1024, 0, s>>>(st->pos[h], st->vel[h], (double2*)st->xy[h],
                                                           (int2*)st->tag, st->offset, st->count);
    return PDQ_OK;
}

// Cache of instantiated step graphs, keyed by every argument that the captured
// launches bake in (pointers, configuration, buffer parity, step phase of the
// compaction schedule).
struct GraphEntry {
    cudaGraphExec_t exec;
    int cur_after;
};
static std::mutex g_graph_mu;
static std::map<std::string, GraphEntry> g_graphs;

// z-binning schedule of the step: the state is binned by z at the start of a call and
// re-binned every rebin_interval steps, compacting at the same time when compaction is on
// (compact_every > 0; then at most every compact_every steps).  The bins widen as particles
// stream along z: over a 100-step cycle of the batched workload the step averaged 180.8 ms
// re-binned every 100 steps and 173.0 ms every 10; each pass costs ~0.6 ms there.
constexpr int kRebinSteps = 10;
static int64_t rebin_interval(const pdq_step_cfg* cfg) {
    return cfg->compact_every > 0 ? std::min<int64_t>(cfg->compact_every, kRebinSteps) : kRebinSteps;
}

static std::string graph_key(const pdq_field* field, const pdq_phys* phys, const pdq_state* st,
                             const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                             const pdq_tally* tally, const void* ws, size_t ws_bytes, cudaStream_t s) {
    pdq_state k = *st;
    k.step = st->step % rebin_interval(cfg);
    std::string key;
    auto put = [&](const void* p, size_t n) { key.append((const char*)p, n); };
    put(&field, sizeof(field)); put(phys, sizeof(*phys)); put(&k, sizeof(k)); put(&params, sizeof(params));
    put(cfg, sizeof(*cfg)); put(&n_steps, sizeof(n_steps)); put(tally, sizeof(*tally)); put(&ws, sizeof(ws));
    put(&ws_bytes, sizeof(ws_bytes)); put(&s, sizeof(s));
    return key;
}

}  // namespace pdq

using namespace pdq;

static int seed_impl(const pdq_field* field, const pdq_phys* phys, double charge_sigma, uint64_t seed,
                     const pdq_sample_params* params, pdq_state* st, pdq_stream_t stream, int independent) {
    if (!field || !phys || !params || !(charge_sigma >= 0)) return PDQ_ERR_INVALID_ARG;
    int rc = validate_state(st);
    if (rc) return rc;
    StepConst K;
    rc = make_step_const(field, phys, st, &K);
    if (rc) return rc;
    SeedArgs A;
    memset(&A, 0, sizeof(A));
    A.offset = st->offset; A.count = st->count; A.ctl = st->ctl; A.params = params;
    A.pos = st->pos[0]; A.vel = st->vel[0]; A.xy = (double2*)st->xy[0]; A.tag = (int2*)st->tag;
    A.capacity = st->capacity; A.S = st->n_samples; A.C = st->n_classes; A.sigma = charge_sigma;
    A.neg_frac = phys->neg_charge_frac;
    A.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    A.independent = independent;
    A.R = K.R; A.L = K.L;
    for (int c = 0; c < st->n_classes; ++c) { A.half_d[c] = K.cls[c].half_d; A.qfac[c] = K.cls[c].qfac; }
    const int64_t n = st->capacity > st->n_samples ? st->capacity : st->n_samples;
    const unsigned blocks = (unsigned)((n + 255) / 256) + 1;
    cudaStream_t s = (cudaStream_t)stream;
    if (st->precision == PDQ_FP64) k_seed<PDQ_FP64><<<blocks, 256, 0, s>>>(A);
    else k_seed<PDQ_MIXED><<<blocks, 256, 0, s>>>(A);
    PDQ_CUDA(cudaGetLastError());
    st->cur = 0;
    st->step = 0;
    return PDQ_OK;
}

extern "C" int pdq_seed_particles(const pdq_field* field, const pdq_phys* phys, double charge_sigma, uint64_t seed,
                                  const pdq_sample_params* params, pdq_state* st, pdq_stream_t stream) {
    return seed_impl(field, phys, charge_sigma, seed, params, st, stream, 0);
}

extern "C" int pdq_seed_particles_independent(const pdq_field* field, const pdq_phys* phys, double charge_sigma,
                                              uint64_t seed, const pdq_sample_params* params, pdq_state* st,
                                              pdq_stream_t stream) {
    if (st && st->n_samples > 0x7ffffffe) return PDQ_ERR_INVALID_ARG;
    return seed_impl(field, phys, charge_sigma, seed, params, st, stream, 1);
}

extern "C" int pdq_step_workspace_size(const pdq_state* st, const pdq_step_cfg* cfg, size_t* bytes) {
    if (!bytes) return PDQ_ERR_INVALID_ARG;
    int rc = validate_state(st);
    if (rc) return rc;
    size_t ib, tot;
    // sized for the narrower of the configured tile and 4 particles per thread (the given-sums
    // step of the P3M driver uses 4), so one workspace serves both step entry points
    workspace_layout(st, tile_threads(st, cfg) * std::min(tile_ilp(st, cfg), 4), &ib, &tot, nullptr, nullptr,
                     cfg && (cfg->forces & PDQ_F_CONTACT), nullptr, newton_pairs(st, cfg));
    *bytes = tot;
    return PDQ_OK;
}

extern "C" int pdq_compact(pdq_state* st, pdq_stream_t stream) {
    int rc = validate_state(st);
    if (rc) return rc;
    enqueue_compact(st, (cudaStream_t)stream);
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

namespace pdq {
// The step; ext (optional, device [capacity][3]) replaces the all-pairs Coulomb sums.
int step_impl(const pdq_field* field, const pdq_phys* phys, pdq_state* st, const pdq_sample_params* params,
              const pdq_step_cfg* cfg, int64_t n_steps, pdq_tally* tally, void* workspace, size_t workspace_bytes,
              pdq_stream_t stream, const double* ext, bool bin) {
    if (!field || !phys || !params || !cfg || !tally || !tally->n_dep || !tally->n_alive || n_steps < 0)
        return PDQ_ERR_INVALID_ARG;
    int rc = validate_state(st);
    if (rc) return rc;
    if (!(cfg->dt > 0) || (cfg->mode != PDQ_STICK && cfg->mode != PDQ_REBOUND) ||
        (cfg->forces & ~(PDQ_F_ALL | PDQ_F_CONTACT)) || cfg->compact_every < 0 || cfg->variant < 0 || cfg->variant > 3 ||
        cfg->use_graph < 0 || cfg->use_graph > 2)
        return PDQ_ERR_INVALID_ARG;
    const bool contact = (cfg->forces & PDQ_F_CONTACT) != 0;
    if (contact && (!(phys->restitution > 0.0 && phys->restitution <= 1.0) || !(phys->tau_col_steps > 0.0)))
        return PDQ_ERR_INVALID_ARG;
    if (ext && (contact || cfg->use_graph)) return PDQ_ERR_INVALID_ARG;
    const int NT = tile_threads(st, cfg);
    const int U = ext ? (st->precision == PDQ_FP64 ? 1 : 4) : tile_ilp(st, cfg);   // given sums: 4 per thread
    if (NT != 64 && NT != 128 && NT != 256 && !(NT == 32 && st->precision == PDQ_FP64)) return PDQ_ERR_INVALID_ARG;
    const bool newton = !ext && newton_pairs(st, cfg);
    if (newton && NT != 64 && NT != 128) return PDQ_ERR_INVALID_ARG;   // its update step runs 2 NT threads
    size_t items_bytes, need, cnt_off = 0, part_off = 0, acc_off = 0;
    workspace_layout(st, NT * U, &items_bytes, &need, &cnt_off, &part_off, contact, &acc_off, newton);
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return PDQ_ERR_WORKSPACE;
    const int JS = newton ? newton_chunks(st, NT * U) : j_split(st, NT * U, contact || ext);
    if (n_steps == 0) return PDQ_OK;
    StepArgs A;
    memset(&A, 0, sizeof(A));
    rc = make_step_const(field, phys, st, &A.K);
    if (rc) return rc;
    A.K.dt = cfg->dt;
    A.K.forces = cfg->forces;
    A.K.mode = cfg->mode;
    A.K.window_start = cfg->window_start;
    const double gplus = phys->g * phys->nu / pow(phys->re_tau * phys->nu / phys->radius, 3);
    for (int k = 0; k < 3; ++k) { A.K.grav[k] = gplus * cfg->gravity[k]; A.K.gravf[k] = (float)A.K.grav[k]; }
    A.K.dtf = (float)cfg->dt;
    if (contact) {   // K = (pi^2 + ln^2 e)/tau_col^2, H = -2 ln e/tau_col (damped oscillator, App. A.2)
        const double tc = phys->tau_col_steps * cfg->dt, le = log(phys->restitution);
        A.K.col_k = (kPi * kPi + le * le) / (tc * tc);
        A.K.col_h = -2.0 * le / tc;
    }
    A.tag = (const int2*)st->tag; A.offset = st->offset; A.count = st->count; A.params = params;
    A.items = (const int2*)workspace; A.ctl = st->ctl;
    A.n_dep = (unsigned long long*)tally->n_dep; A.n_alive = (unsigned long long*)tally->n_alive;
    A.jsplit = JS;
    A.cap = st->capacity;
    A.ext = ext;
    if (newton && st->precision == PDQ_MIXED) A.acc4 = (float4*)((char*)workspace + acc_off);
    if (newton && st->precision == PDQ_FP64) A.acc64 = (double*)((char*)workspace + acc_off);
    A.max_items = (st->capacity / (NT * U) + st->n_samples + 1) * JS;
    if (JS > 1 && !newton) {
        A.tile_cnt = (int*)((char*)workspace + cnt_off);
        A.part = (double*)((char*)workspace + part_off);
    }
    int2* items = (int2*)workspace;
    int32_t* order = (int32_t*)((char*)workspace + items_bytes);
    cudaStream_t s = (cudaStream_t)stream;

    // Particles are z-binned at the start of the call and every rebin_interval steps (compacted
    // at the same time when compaction is on) so that most tile pairs skip the per-pair minimum
    // image.  Not with given Coulomb sums: the P3M driver has its own cell list.
    const bool binned = bin && !ext;
    const bool compact = cfg->compact_every > 0;
    const int64_t rebin = binned ? rebin_interval(cfg) : cfg->compact_every;
    int2* tag_scratch = (int2*)((char*)workspace + items_bytes + align256(sizeof(int32_t) * (size_t)st->n_samples));
    const float bins_per_length = (float)(kZBins / A.K.L);
    auto enqueue = [&]() -> int {
        if (binned) {
            const int r = enqueue_sort_compact(st, tag_scratch, bins_per_length, compact, s);
            if (r) return r;
        }
        int cur = st->cur;
        int64_t stepi = st->step;
        if (JS > 1 && !newton) {   // each tile's last chunk resets its counter, so zeroing once per call suffices
            const cudaError_t e = cudaMemsetAsync(A.tile_cnt, 0, sizeof(int) * (size_t)(st->capacity / (NT * U) +
                                                                                          st->n_samples + 1), s);
            if (e != cudaSuccess) return cuda_status(e);
        }
        k_build_items<<<1, 1024, 0, s>>>(st->count, st->n_samples, NT * U, JS, order, items, st->ctl);
        for (int64_t k = 0; k < n_steps; ++k) {
            A.pos_in = st->pos[cur]; A.vel_in = st->vel[cur]; A.xy_in = (const double2*)st->xy[cur];
            A.pos_out = st->pos[cur ^ 1]; A.vel_out = st->vel[cur ^ 1]; A.xy_out = (double2*)st->xy[cur ^ 1];
            const int r = dispatch_step(st->precision, NT, cfg->variant, contact, A, s);
            if (r) return r;
            cur ^= 1;
            ++stepi;
            if (rebin > 0 && stepi % rebin == 0 && k + 1 < n_steps) {
                st->cur = cur;
                if (binned) {
                    const int r = enqueue_sort_compact(st, tag_scratch, bins_per_length, compact, s);
                    if (r) return r;
                    cur = st->cur;
                } else {
                    enqueue_compact(st, s);
                }
                k_build_items<<<1, 1024, 0, s>>>(st->count, st->n_samples, NT * U, JS, order, items, st->ctl);
            }
        }
        st->cur = cur;
        st->step = stepi;
        return PDQ_OK;
    };
    if (!cfg->use_graph) {
        rc = enqueue();
        if (rc) return rc;
        PDQ_CUDA(cudaGetLastError());
        return PDQ_OK;
    }
    // Graph mode: the whole call (binning, work lists, n_steps step launches, compactions) is
    // captured once per distinct argument set and replayed afterwards.  use_graph = 2 only
    // prepares: it captures and instantiates the graph (if not cached) and leaves the state as
    // it was, so that a later use_graph = 1 call with the same arguments is a replay.
    const bool prepare_only = cfg->use_graph == 2;
    pdq_step_cfg kcfg = *cfg;
    kcfg.use_graph = 1;                     // both modes share one cache entry
    const std::string key = graph_key(field, phys, st, params, &kcfg, n_steps, tally, workspace, workspace_bytes, s);
    {
        std::lock_guard<std::mutex> lock(g_graph_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) {
            if (prepare_only) return PDQ_OK;
            PDQ_CUDA(cudaGraphLaunch(it->second.exec, s));
            st->cur = it->second.cur_after;
            st->step += n_steps;
            return PDQ_OK;
        }
    }
    const int cur0 = st->cur;
    const int64_t step0 = st->step;
    PDQ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    rc = enqueue();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        st->cur = cur0;
        st->step = step0;
        return rc ? rc : cuda_status(e);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        st->cur = cur0;
        st->step = step0;
        return cuda_status(e);
    }
    if (prepare_only) {
        const int cur_after = st->cur;
        st->cur = cur0;
        st->step = step0;
        std::lock_guard<std::mutex> lock(g_graph_mu);
        g_graphs[key] = GraphEntry{exec, cur_after};
        return PDQ_OK;
    }
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        st->cur = cur0;
        st->step = step0;
        return cuda_status(e);
    }
    std::lock_guard<std::mutex> lock(g_graph_mu);
    g_graphs[key] = GraphEntry{exec, st->cur};
    return PDQ_OK;
}

// Compaction entry for the P3M driver (unsorted, stream-ordered).
int compact_state(pdq_state* st, cudaStream_t s) { return enqueue_compact(st, s); }
}  // namespace pdq

extern "C" int pdq_step_particles(const pdq_field* field, const pdq_phys* phys, pdq_state* st,
                                  const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                                  pdq_tally* tally, void* workspace, size_t workspace_bytes, pdq_stream_t stream) {
    return pdq::step_impl(field, phys, st, params, cfg, n_steps, tally, workspace, workspace_bytes, stream, nullptr,
                          true);
}

extern "C" int pdq_release_graphs(void) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second.exec);
    g_graphs.clear();
    return PDQ_OK;
}

extern "C" int pdq_check_state(pdq_state* st, pdq_stream_t stream) {
    if (!st || !st->ctl) return PDQ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t word = 0;
    PDQ_CUDA(cudaMemcpyAsync(&word, st->ctl + CTL_ERROR, sizeof(word), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    if (word) {
        const int64_t zero = 0;
        PDQ_CUDA(cudaMemcpy(st->ctl + CTL_ERROR, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    }
    if (word & ERR_NONFINITE) return PDQ_ERR_NAN;
    return word ? PDQ_ERR_TIMEOUT : PDQ_OK;
}

extern "C" int pdq_deposition_tally(const pdq_tally* t, int32_t S, int32_t C, double dt, double r_plus, double* vdep,
                                    double* mean, double* se, pdq_stream_t stream) {
    if (!t || !t->n_dep || !t->n_alive || S < 1 || C < 1 || !(dt > 0) || !(r_plus > 0) || !vdep)
        return PDQ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = S * C;
    k_vdep<<<(n + 255) / 256, 256, 0, s>>>(t->n_dep, t->n_alive, n, 0.5 * r_plus / dt, vdep);
    if (mean || se) k_vdep_stats<<<C, 32, 0, s>>>(vdep, S, C, mean, se);
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times one step of every (block, pair variant) candidate on the caller's
// state (best of three after a warm-up) and writes the fastest into cfg.  Each timed step writes the
// scratch half of the double buffer and a scratch tally, then the state's
// current half, step counter and control block are restored, so the state is
// unchanged apart from one z-binning (a compaction too when compaction is on),
// which only reorders live particles.  Results are cached per (precision,
// log2 capacity, log2 samples, forces) for the process lifetime.
// ---------------------------------------------------------------------------
#include <map>
#include <mutex>
#include <tuple>

namespace pdq {
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;
static int ilog2(int64_t v) { int r = 0; while (v > 1) { v >>= 1; ++r; } return r; }
static int min_tile(const pdq_state* st) { return st->precision == PDQ_FP64 ? 32 : 64 * tile_ilp(st); }
// largest step workspace over the candidate tiles (the FP64 j-split makes it grow with the tile)
static size_t autotune_scratch_offset(const pdq_state* st) {
    const bool f64 = st->precision == PDQ_FP64;
    const int tiles_f64[4] = {32, 64, 128, 256};
    const int tiles_mixed[6] = {64 * 4, 128 * 4, 256 * 4, 64 * 8, 128 * 8, 256 * 8};
    size_t best = 0;
    for (int k = 0; k < (f64 ? 4 : 6); ++k) {
        for (int nw = 0; nw < 2; ++nw) {      // one-sided and Newton-pair layouts
            size_t ib, tot;
            const int TI = f64 ? tiles_f64[k] * (nw ? 2 : 1) : tiles_mixed[k];
            workspace_layout(st, TI, &ib, &tot, nullptr, nullptr, false, nullptr, nw == 1);
            if (tot > best) best = tot;
        }
    }
    return best;
}
}  // namespace pdq

extern "C" int pdq_autotune_workspace_size(const pdq_state* st, size_t* bytes) {
    if (!bytes) return PDQ_ERR_INVALID_ARG;
    int rc = validate_state(st);
    if (rc) return rc;
    *bytes = autotune_scratch_offset(st) + 2 * align256(sizeof(int64_t) * (size_t)st->n_samples * st->n_classes);
    return PDQ_OK;
}

extern "C" int pdq_autotune(const pdq_field* field, const pdq_phys* phys, pdq_state* st,
                            const pdq_sample_params* params, pdq_step_cfg* cfg, void* workspace,
                            size_t workspace_bytes, pdq_stream_t stream) {
    if (!field || !phys || !params || !cfg) return PDQ_ERR_INVALID_ARG;
    size_t need = 0;
    int rc = pdq_autotune_workspace_size(st, &need);
    if (rc) return rc;
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return PDQ_ERR_WORKSPACE;
    const auto key = std::make_tuple(st->precision, ilog2(st->capacity), ilog2(st->n_samples), cfg->forces);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            cfg->block = it->second.first;
            cfg->variant = it->second.second;
            return PDQ_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t step_ws = autotune_scratch_offset(st);
    const size_t tb = align256(sizeof(int64_t) * (size_t)st->n_samples * st->n_classes);
    pdq_tally scratch;
    scratch.n_dep = (int64_t*)((char*)workspace + step_ws);
    scratch.n_alive = (int64_t*)((char*)workspace + step_ws + tb);
    {   // bin the state once (as a step call would), then time unbinned single steps on it
        StepConst K;
        rc = make_step_const(field, phys, st, &K);
        if (rc) return rc;
        size_t ib, tot;
        workspace_layout(st, min_tile(st), &ib, &tot);
        int2* tag_scratch = (int2*)((char*)workspace + ib + align256(sizeof(int32_t) * (size_t)st->n_samples));
        rc = enqueue_sort_compact(st, tag_scratch, (float)(kZBins / K.L), cfg->compact_every > 0, s);
        if (rc) return rc;
    }
    const int blocks[4] = {64, 128, 256, 32};
    const int n_blk = st->precision == PDQ_FP64 ? 4 : 3;    // 32-thread tiles: FP64 only
    // candidate pair variants: MIXED 0-3, FP64 0 and 3 (Newton pairs); contact runs: MIXED 0 and 3,
    // FP64 0
    const bool contact_run = (cfg->forces & PDQ_F_CONTACT) != 0;
    const int vars_mixed[4] = {0, 1, 2, 3}, vars_03[2] = {0, 3};
    const int* vars = st->precision == PDQ_MIXED && !contact_run ? vars_mixed : vars_03;
    const int n_var = contact_run ? (st->precision == PDQ_MIXED ? 2 : 1) : (st->precision == PDQ_MIXED ? 4 : 2);
    cudaEvent_t e0, e1;
    PDQ_CUDA(cudaEventCreate(&e0));
    PDQ_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_b = tile_threads(st, nullptr), best_v = 0;
    const int cur0 = st->cur;
    const int64_t step0 = st->step;
    for (int bi = 0; bi < n_blk && rc == PDQ_OK; ++bi) {
        for (int vi = 0; vi < n_var && rc == PDQ_OK; ++vi) {
            const int v = vars[vi];
            if (v == 3 && blocks[bi] != 64 && blocks[bi] != 128) continue;       // Newton pairs: 64 or 128 threads
            pdq_step_cfg c = *cfg;
            c.block = blocks[bi];
            c.variant = v;
            c.compact_every = 0;
            c.use_graph = 0;
            float ms = 1e30f;
            for (int rep = 0; rep < 4 && rc == PDQ_OK; ++rep) {      // rep 0 warms up; best of the other 3
                cudaEventRecord(e0, s);
                rc = step_impl(field, phys, st, params, &c, 1, &scratch, workspace, step_ws, stream, nullptr, false);
                cudaEventRecord(e1, s);
                st->cur = cur0;
                st->step = step0;
                cudaMemcpyAsync(st->ctl, &step0, sizeof(int64_t), cudaMemcpyHostToDevice, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = PDQ_ERR_CUDA;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            if (rc == PDQ_OK && ms < best) { best = ms; best_b = blocks[bi]; best_v = v; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    cfg->block = best_b;
    cfg->variant = best_v;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = std::make_pair(best_b, best_v);
    return PDQ_OK;
}

// ---------------------------------------------------------------------------
// Capture efficiency (Sec. 4.3): CE = (4 L / D) (u* / U_b) V_dep+|stick, where the
// tallies of a rebound-mode run count only the particles that stick.
// ---------------------------------------------------------------------------
namespace pdq {
__global__ void k_scale(const double* __restrict__ in, int64_t n, double f, double* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = f * in[k];
}
}  // namespace pdq

extern "C" int pdq_capture_efficiency(const pdq_field* field, const pdq_phys* phys, const double* vdep, int64_t n,
                                      double* ce, pdq_stream_t stream) {
    if (!field || !phys || !vdep || !ce || n < 0 || !(phys->u_bulk > 0)) return PDQ_ERR_INVALID_ARG;
    const double ustar = phys->re_tau * phys->nu / phys->radius;
    const double f = 4.0 * (field->desc.l_plus / (2.0 * field->desc.r_plus)) * (ustar / phys->u_bulk);
    if (n == 0) return PDQ_OK;
    k_scale<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(vdep, n, f, ce);
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}
