// pdq_device.cuh -- device-side physics shared by the forward step and the
// adjoint kernels: time-integration weights, field interpolation and the
// scalar Coulomb pair.
#pragma once

#include <type_traits>

#include "pdq_common.cuh"

namespace pdq {

template <int P> struct Real;
template <> struct Real<PDQ_FP64> { typedef double T; typedef double4_32a T4; };
template <> struct Real<PDQ_MIXED> { typedef float T; typedef float4 T4; };

// ---------------------------------------------------------------------------
// Device physics helpers.
// ---------------------------------------------------------------------------
// phi1(z) = (e^z - 1)/z and phi2(z) = (e^z - 1 - z)/z^2: Taylor series near 0
// (where the closed forms cancel), expm1 elsewhere.
__device__ __forceinline__ void phi12(double z, double& p1, double& p2) {
    if (fabs(z) < 0.05) {
        // Horner with explicit coefficients (1/(k+1)! and 1/(k+2)!).
        const double c1[11] = {1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
                               1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800};
        p1 = c1[10];
        p2 = 1.0 / 479001600;
        for (int k = 9; k >= 0; --k) p1 = p1 * z + c1[k];
        for (int k = 9; k >= 0; --k) p2 = p2 * z + c1[k + 1];
        return;
    }
    const double em = expm1(z);
    p1 = em / z;
    p2 = (em - z) / (z * z);
}
__device__ __forceinline__ void phi12(float z, float& p1, float& p2) {
    if (fabsf(z) < 0.1f) {
        const float c[10] = {1.f, 1.f / 2, 1.f / 6, 1.f / 24, 1.f / 120, 1.f / 720, 1.f / 5040, 1.f / 40320,
                             1.f / 362880, 1.f / 3628800};
        p1 = c[8];
        p2 = c[9];
        for (int k = 7; k >= 0; --k) p1 = fmaf(p1, z, c[k]);
        for (int k = 8; k >= 1; --k) p2 = fmaf(p2, z, c[k]);
        return;
    }
    const float em = expm1f(z);
    p1 = em / z;
    p2 = (em - z) / (z * z);
}

__device__ __forceinline__ double atanh_(double x) { return atanh(x); }
__device__ __forceinline__ float atanh_(float x) { return atanhf(x); }
__device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double floor_(double x) { return floor(x); }
__device__ __forceinline__ float floor_(float x) { return floorf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }

__device__ __forceinline__ double4_32a grid_at(const StepConst& K, const double4_32a*, int64_t i) { return K.grid64[i]; }
__device__ __forceinline__ float4 grid_at(const StepConst& K, const float4*, int64_t i) { return __ldg(K.grid32 + i); }

// Trilinear interpolation in (s(r), theta, z) index space: s = atanh(r tanh(beta)/R)/beta
// inverts the node stretching; theta and z are periodic; s is clamped to [0, 1].
// The field-geometry constants in T: for float the FP32 copies rounded once on the host (the
// same values as converting the doubles here, without the per-particle conversions and the FP64
// division n_th / 2 pi); for double the doubles.
template <class T>
struct GridT {
    T R, tanh_b, inv_b, th_scale, z_scale;
    __device__ __forceinline__ explicit GridT(const StepConst& K) {
        if constexpr (std::is_same<T, float>::value) {
            R = K.Rf; tanh_b = K.tanh_beta_f; inv_b = K.inv_beta_f; th_scale = K.th_scale_f; z_scale = K.z_scale_f;
        } else {
            R = K.R; tanh_b = K.tanh_beta; inv_b = K.inv_beta; th_scale = K.n_th / (2.0 * kPi);
            z_scale = K.n_z * K.invL;
        }
    }
};

template <class T, class T4>
__device__ __forceinline__ void interp(const StepConst& K, T r, T x, T y, T z, T u[3]) {
    if (!(isfinite(r) && isfinite(x) && isfinite(y) && isfinite(z))) {
        // a non-finite position (reported through the error word) never forms a cell index
        u[0] = u[1] = u[2] = (T)NAN;
        return;
    }
    const GridT<T> G(K);
    const T R = G.R, tanh_b = G.tanh_b, inv_b = G.inv_b, th_scale = G.th_scale, z_scale = G.z_scale;
    const T rho = fmin(r / R, (T)1);
    const T s = atanh_(rho * tanh_b) * inv_b;
    const T fi = s * (T)(K.n_r - 1);
    int i0 = (int)floor_(fi);
    i0 = i0 < 0 ? 0 : (i0 > K.n_r - 2 ? K.n_r - 2 : i0);
    const T tr = fi - (T)i0;
    T fj = atan2_(y, x) * th_scale;
    if (fj < (T)0) fj += (T)K.n_th;
    int j0 = (int)floor_(fj);
    const T tt = fj - (T)j0;
    j0 %= K.n_th;                    // any int (also a non-finite input's) maps into [0, n_th)
    if (j0 < 0) j0 += K.n_th;
    const int j1 = (j0 + 1 == K.n_th) ? 0 : j0 + 1;
    const T fk = z * z_scale;
    int k0 = (int)floor_(fk);
    const T tz = fk - (T)k0;
    k0 %= K.n_z;
    if (k0 < 0) k0 += K.n_z;
    const int k1 = (k0 + 1 == K.n_z) ? 0 : k0 + 1;
    const int64_t nr = K.n_r, plane = (int64_t)K.n_r * K.n_th;
    const int64_t b00 = k0 * plane + j0 * nr + i0, b01 = k0 * plane + j1 * nr + i0;
    const int64_t b10 = k1 * plane + j0 * nr + i0, b11 = k1 * plane + j1 * nr + i0;
    const T4* tag = nullptr;
    const T4 g000 = grid_at(K, tag, b00), g001 = grid_at(K, tag, b00 + 1);
    const T4 g010 = grid_at(K, tag, b01), g011 = grid_at(K, tag, b01 + 1);
    const T4 g100 = grid_at(K, tag, b10), g101 = grid_at(K, tag, b10 + 1);
    const T4 g110 = grid_at(K, tag, b11), g111 = grid_at(K, tag, b11 + 1);
    const T wr0 = (T)1 - tr, wt0 = (T)1 - tt, wz0 = (T)1 - tz;
    const T w000 = wr0 * wt0 * wz0, w001 = tr * wt0 * wz0, w010 = wr0 * tt * wz0, w011 = tr * tt * wz0;
    const T w100 = wr0 * wt0 * tz, w101 = tr * wt0 * tz, w110 = wr0 * tt * tz, w111 = tr * tt * tz;
    u[0] = w000 * g000.x + w001 * g001.x + w010 * g010.x + w011 * g011.x + w100 * g100.x + w101 * g101.x +
           w110 * g110.x + w111 * g111.x;
    u[1] = w000 * g000.y + w001 * g001.y + w010 * g010.y + w011 * g011.y + w100 * g100.y + w101 * g101.y +
           w110 * g110.y + w111 * g111.y;
    u[2] = w000 * g000.z + w001 * g001.z + w010 * g010.z + w011 * g011.z + w100 * g100.z + w101 * g101.z +
           w110 * g110.z + w111 * g111.z;
}

// One ordered pair of the Coulomb sum: acc += q_j (x_i - x_j) / max(|x_i - x_j|, d_c)^3,
// minimum image in z by the round-to-nearest trick (t + M) - M.
// Hardware reciprocal square root without the denormal fix-up path (arguments
// here are clamped away from zero by the contact distance).
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rsqrt_ftz(double x) { return rsqrt(x); }

__device__ __forceinline__ void coulomb_pair(float xi, float yi, float zi, const float4 pj, float L, float invL,
                                             float c2, float& ax, float& ay, float& az) {
    const float dx = xi - pj.x, dy = yi - pj.y;
    float dz = zi - pj.z;
    const float t = __fadd_rn(__fmaf_rn(dz, invL, 12582912.0f), -12582912.0f);
    dz = __fmaf_rn(-L, t, dz);
    const float r2 = fmaxf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))), c2);
    const float ri = rsqrt_ftz(r2);
    const float s = __fmul_rn(__fmul_rn(pj.w, ri), __fmul_rn(ri, ri));
    ax = __fmaf_rn(s, dx, ax);
    ay = __fmaf_rn(s, dy, ay);
    az = __fmaf_rn(s, dz, az);
}
__device__ __forceinline__ void coulomb_pair(double xi, double yi, double zi, const double4_32a pj, double L, double invL,
                                             double c2, double& ax, double& ay, double& az) {
    const double dx = xi - pj.x, dy = yi - pj.y;
    double dz = zi - pj.z;
    const double t = __dadd_rn(__fma_rn(dz, invL, 6755399441055744.0), -6755399441055744.0);
    dz = __fma_rn(-L, t, dz);
    const double r2 = fmax(__fma_rn(dx, dx, __fma_rn(dy, dy, dz * dz)), c2);
    const double ri = rsqrt(r2);
    const double s = pj.w * ri * (ri * ri);
    ax = __fma_rn(s, dx, ax);
    ay = __fma_rn(s, dy, ay);
    az = __fma_rn(s, dz, az);
}


// Initial state of local particle j (Sec. 2.1: uniform in the pipe, at rest):
// Philox4x32-10 counter (j, 0, 0, w3) gives (r, theta, z) = ((R - d/2) sqrt(u0),
// 2 pi u1, L u2); counter (j, 1, 0, w3) the lognormal charge factor
// exp(sigma sqrt(-2 ln u0) cos(2 pi u1)); counter (j, 2, 0, w3) the sign when neg_frac > 0.
// w3 = 0: every sample draws the same particles (common random numbers); w3 = s + 1 gives
// sample s a stream of its own.  qhat = charge per unit xi (units of q_unit).
__device__ __forceinline__ void seed_particle(uint2 key, uint32_t j, double sigma, double neg_frac, double R, double L,
                                              double half_d, double qfac, double& x, double& y, double& z,
                                              double& qhat, uint32_t w3 = 0u) {
    const uint4 a = philox4x32_10(make_uint4(j, 0u, 0u, w3), key);
    double lam = 1.0;
    if (neg_frac > 0.0) {      // negative charge with probability neg_frac (counter word 2)
        const uint4 b = philox4x32_10(make_uint4(j, 2u, 0u, w3), key);
        if (unit_open(b.x) < neg_frac) lam = -1.0;
    }
    if (sigma > 0.0) {
        const uint4 b = philox4x32_10(make_uint4(j, 1u, 0u, w3), key);
        lam *= exp(sigma * sqrt(-2.0 * log(unit_open(b.x))) * cos(2.0 * kPi * unit_open(b.y)));
    }
    const double rr = (R - half_d) * sqrt(unit_open(a.x));
    double sth, cth;
    sincos(2.0 * kPi * unit_open(a.y), &sth, &cth);
    x = rr * cth;
    y = rr * sth;
    z = L * unit_open(a.z);
    qhat = qfac * lam;
}

// Packed FP32 pairs (sm_100+ f32x2 instructions): one 64-bit register holds the
// same quantity for two particles, so each FMA-pipe instruction does two lanes' work.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { f2 d; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) { f2 d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) { f2 d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}


// Two ordered pairs (i_a, j), (i_b, j) of the Coulomb sum in packed form.
// j = (xj, xj), (yj, yj), (zj, zj), (qj, qj); the minimum image in z uses
// (dz/L + M) - M = rint(dz/L) with M = 1.5 * 2^23.
// TRACK: also keep the smallest nonzero r^2 seen (contact-force runs look for near pairs; the
// self pair, r = 0, is left out).
template <bool TRACK = false>
__device__ __forceinline__ void coulomb_pair_x2(f2 xi, f2 yi, f2 zi, f2 xj, f2 yj, f2 zj, f2 qj, f2 invL2, f2 M2,
                                                f2 nM2, f2 nL2, float c2, f2& ax, f2& ay, f2& az, float& mn) {
    const f2 dx = f2_sub(xi, xj), dy = f2_sub(yi, yj);
    f2 dz = f2_sub(zi, zj);
    const f2 t = f2_add(f2_fma(dz, invL2, M2), nM2);
    dz = f2_fma(nL2, t, dz);
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    if constexpr (TRACK) mn = fminf(mn, fminf(ra > 0.f ? ra : INFINITY, rb > 0.f ? rb : INFINITY));   // not self
    const f2 ri = f2_pack(rsqrt_ftz(fmaxf(ra, c2)), rsqrt_ftz(fmaxf(rb, c2)));
    const f2 s = f2_mul(f2_mul(ri, qj), f2_mul(ri, ri));
    ax = f2_fma(s, dx, ax);
    ay = f2_fma(s, dy, ay);
    az = f2_fma(s, dz, az);
}

// Same pairs when no pair of the (i-tile, j-tile) combination needs the
// periodic image: dz = (z_i - shift) - z_j directly (the shift is folded into zi).
// CLAMP = false when every |dz| of the tile pair exceeds the contact distance, so
// r^2 > c2 and the clamp could not change a result.
template <bool CLAMP, bool TRACK = false>
__device__ __forceinline__ void coulomb_pair_x2_direct(f2 xi, f2 yi, f2 zi, f2 xj, f2 yj, f2 zj, f2 qj, float c2,
                                                       f2& ax, f2& ay, f2& az, float& mn) {
    const f2 dx = f2_sub(xi, xj), dy = f2_sub(yi, yj), dz = f2_sub(zi, zj);
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    if constexpr (TRACK) mn = fminf(mn, fminf(ra > 0.f ? ra : INFINITY, rb > 0.f ? rb : INFINITY));   // not self
    if constexpr (CLAMP) { ra = fmaxf(ra, c2); rb = fmaxf(rb, c2); }
    const f2 ri = f2_pack(rsqrt_ftz(ra), rsqrt_ftz(rb));
    const f2 s = f2_mul(f2_mul(ri, qj), f2_mul(ri, ri));
    ax = f2_fma(s, dx, ax);
    ay = f2_fma(s, dy, ay);
    az = f2_fma(s, dz, az);
}

}  // namespace pdq
