// pdq_p3m.cu -- P3M electrostatics for the periodic pipe (App. A.2: the
// particle-particle particle-mesh method the paper uses for large samples).
//
// The pipe is periodic along z (period L) and isolated across.  The Coulomb
// kernel d/r^3 is split with a Gaussian screening of width 1/alpha,
//   K_L(d) = d [erf(alpha r)/r^3 - 2 alpha/sqrt(pi) exp(-alpha^2 r^2)/r^2],
//   K_S(d) = d/max(r, d_c)^3 - K_L(d)  (negligible beyond r_cut),
// K_L handled on a mesh, K_S pair by pair:
//   plan:  K_L summed over the z images at every node offset of a mesh that is
//          periodic in z and twice the charge region across (so the FFT's
//          circular convolution is the open one), transformed, divided by the
//          squared TSC window (sinc^3 per axis) and by the transform size;
//   solve: TSC charge assignment (atomics) -> FFT -> product with each kernel
//          component -> inverse FFT -> TSC interpolation; then a cell list
//          (cells >= r_cut, stable per-cell order, particles copied in cell
//          order) and the direct short-range sum with the minimum image along z.
// FP64 throughout; cuFFT does the transforms.  One sample at a time.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "pdq_common.cuh"
#include "pdq_device.cuh"

struct pdq_p3m {
    int device;
    double R, L, h, hz, x0, alpha, rc;
    int M, Mx, Nx, Nz, n_img;
    int64_t max_n;
    size_t nreal, ncplx;
    cufftHandle fwd, inv;
    bool have_fwd, have_inv;
    cufftDoubleComplex* Gh;     // [3][ncplx] influence function
    double* Q;                  // [nreal] charges
    cufftDoubleComplex* Qh;     // [ncplx]
    cufftDoubleComplex* Ah;     // [ncplx]
    double* A;                  // [nreal]
    int ncx, ncz;
    int64_t ncells;
    int* cell_count;            // [ncells]
    int* cell_start;            // [ncells + 1]
    int* cell_fill;             // [ncells]
    int* cell_list;             // [max_n]
    double4_32a* sorted64;          // [max_n] live particles in cell order: x, y, z, q
    double2* lf_tab;                // [kTab + 1] K_L factor and its u-derivative at u = k (alpha r_cut)^2 / kTab
    float4* sorted32;           // [max_n] the same positions in FP32 (distance pre-filter)
    double* sums;               // [sums_cap][3], for the step driver
    int64_t sums_cap;
};

namespace pdq {
namespace {

struct P3MGeom {
    double R, L, h, hz, x0, alpha, rc, contact;
    int Mx, Nx, Nz, n_img, ncx, ncz;
    const double2* lf_tab;
};

// The short-range pairs read the long-range factor from a cubic Hermite table in
// u = (alpha r)^2 (relative interpolation error ~1e-13) instead of FP64 erf and exp.
constexpr int kTab = 4096;

struct P3MPart {                // the particles of one sample, current half of the state
    const void* pos;
    const void* vel;
    const double2* xy;
    int64_t o, n;
    int precision;
};

__device__ __forceinline__ bool load_particle(const P3MPart& S, int64_t g, double& x, double& y, double& z,
                                              double& q) {
    if (S.precision == PDQ_FP64) {
        const double4_32a p = ((const double4_32a*)S.pos)[g];
        const double4_32a v = ((const double4_32a*)S.vel)[g];
        x = p.x; y = p.y; z = p.z; q = p.w;
        return v.w > 0.5;
    }
    const float4 p = ((const float4*)S.pos)[g];
    const float4 v = ((const float4*)S.vel)[g];
    const double2 xy = S.xy[g];
    x = xy.x; y = xy.y; z = (double)p.z; q = (double)p.w;
    return v.w > 0.5f;
}

// K_L(d) / |d| factor: erf(ar)/r^3 - 2a/sqrt(pi) e^{-a^2 r^2}/r^2; Taylor series near 0, 1/r^3 far out.
__device__ __forceinline__ double long_factor(double r2, double alpha) {
    const double r = sqrt(r2), ar = alpha * r;
    const double c = 1.1283791670955126;      // 2 / sqrt(pi)
    if (ar < 0.05) {                          // Taylor series where the closed form cancels
        const double u = ar * ar;
        return c * alpha * alpha * alpha * (2.0 / 3.0) * (1.0 - 0.6 * u + (3.0 / 14.0) * u * u);
    }
    const double ir2 = 1.0 / r2, ir3 = ir2 / r;
    if (ar > 6.5) return ir3;                 // erf = 1, the Gaussian below 1e-18
    return erf(ar) * ir3 - c * alpha * exp(-ar * ar) * ir2;
}

__global__ void k_p3m_kernel(const P3MGeom G, double* gx, double* gy, double* gz) {
    const int64_t nreal = (int64_t)G.Nx * G.Nx * G.Nz;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nreal) return;
    const int iz = (int)(idx % G.Nz);
    const int iy = (int)((idx / G.Nz) % G.Nx);
    const int ix = (int)(idx / ((int64_t)G.Nz * G.Nx));
    if (2 * ix == G.Nx || 2 * iy == G.Nx) { gx[idx] = 0.0; gy[idx] = 0.0; gz[idx] = 0.0; return; }
    const double dx = (ix > G.Nx / 2 ? ix - G.Nx : ix) * G.h;
    const double dy = (iy > G.Nx / 2 ? iy - G.Nx : iy) * G.h;
    const double dz0 = (iz > G.Nz / 2 ? iz - G.Nz : iz) * G.hz;
    const double rho2 = dx * dx + dy * dy;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int k = -G.n_img; k <= G.n_img; ++k) {
        const double dz = dz0 - k * G.L;
        const double r2 = rho2 + dz * dz;
        const double f = long_factor(r2, G.alpha);
        sx += f * dx; sy += f * dy; sz += f * dz;
    }
    const double tail = 1.0 / (2.0 * (G.n_img + 0.5) * (G.n_img + 0.5)) / (G.L * G.L * G.L);
    sx += 2.0 * dx * tail;
    sy += 2.0 * dy * tail;
    sz += -4.0 * dz0 * tail;
    if (2 * iz == G.Nz) sz = 0.0;              // half a period: the odd z-component vanishes
    gx[idx] = sx; gy[idx] = sy; gz[idx] = sz;
}

__device__ __forceinline__ double sinc6(double m) {
    if (m == 0.0) return 1.0;
    const double a = kPi * m, s = sin(a) / a;
    const double s3 = s * s * s;
    return s3 * s3;
}

// Divide the kernel transforms by the squared TSC window and the transform size.
__global__ void k_p3m_deconv(const P3MGeom G, cufftDoubleComplex* gh, int64_t ncplx) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncplx) return;
    const int nzh = G.Nz / 2 + 1;
    const int iz = (int)(idx % nzh);
    const int iy = (int)((idx / nzh) % G.Nx);
    const int ix = (int)(idx / ((int64_t)nzh * G.Nx));
    const double mx = (double)min(ix, G.Nx - ix) / G.Nx, my = (double)min(iy, G.Nx - iy) / G.Nx;
    const double mz = (double)iz / G.Nz;
    const double w = sinc6(mx) * sinc6(my) * sinc6(mz) * ((double)G.Nx * G.Nx * G.Nz);
    for (int c = 0; c < 3; ++c) {
        cufftDoubleComplex& v = gh[c * ncplx + idx];
        v.x /= w;
        v.y /= w;
    }
}

// TSC: nearest node and weights of a coordinate in node units.
__device__ __forceinline__ int tsc(double t, int lo, int hi, double w[3]) {
    int i0 = (int)rint(t);
    const double d = t - i0;
    w[0] = 0.5 * (0.5 - d) * (0.5 - d);
    w[1] = 0.75 - d * d;
    w[2] = 0.5 * (0.5 + d) * (0.5 + d);
    return i0 < lo ? lo : (i0 > hi ? hi : i0);   // particles are inside the pipe; the clamp is a guard
}

__global__ void k_p3m_assign(const P3MGeom G, const P3MPart S, double* Q) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.n) return;
    double x, y, z, q;
    if (!load_particle(S, S.o + k, x, y, z, q) || q == 0.0) return;
    double wx[3], wy[3], wz[3];
    const int ix = tsc((x - G.x0) / G.h, 1, G.Mx - 2, wx);
    const int iy = tsc((y - G.x0) / G.h, 1, G.Mx - 2, wy);
    const int iz = tsc(z / G.hz, -1 << 30, 1 << 30, wz);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int64_t rowb = ((int64_t)(ix + a - 1) * G.Nx + (iy + b - 1)) * G.Nz;
            for (int c = 0; c < 3; ++c) {
                int zz = (iz + c - 1) % G.Nz;
                if (zz < 0) zz += G.Nz;
                atomicAdd(&Q[rowb + zz], q * wx[a] * wy[b] * wz[c]);
            }
        }
}

__global__ void k_p3m_mul(const cufftDoubleComplex* __restrict__ Qh, const cufftDoubleComplex* __restrict__ gh,
                          cufftDoubleComplex* __restrict__ Ah, int64_t ncplx) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncplx) return;
    const cufftDoubleComplex a = Qh[idx], b = gh[idx];
    Ah[idx] = make_cuDoubleComplex(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Long-range sum, component c, interpolated with the assignment weights (written, not added).
__global__ void k_p3m_interp(const P3MGeom G, const P3MPart S, const double* __restrict__ A, int c, double* sums) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.n) return;
    const int64_t g = S.o + k;
    double x, y, z, q;
    if (!load_particle(S, g, x, y, z, q)) return;
    double wx[3], wy[3], wz[3];
    const int ix = tsc((x - G.x0) / G.h, 1, G.Mx - 2, wx);
    const int iy = tsc((y - G.x0) / G.h, 1, G.Mx - 2, wy);
    const int iz = tsc(z / G.hz, -1 << 30, 1 << 30, wz);
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int64_t rowb = ((int64_t)(ix + a - 1) * G.Nx + (iy + b - 1)) * G.Nz;
            for (int cc = 0; cc < 3; ++cc) {
                int zz = (iz + cc - 1) % G.Nz;
                if (zz < 0) zz += G.Nz;
                s += A[rowb + zz] * wx[a] * wy[b] * wz[cc];
            }
        }
    sums[3 * g + c] = s;
}

__device__ __forceinline__ int cell_of(const P3MGeom& G, double x, double y, double z) {
    const double wxy = 2.0 * G.R / G.ncx, wz = G.L / G.ncz;
    int cx = (int)floor((x + G.R) / wxy), cy = (int)floor((y + G.R) / wxy), cz = (int)floor(z / wz);
    cx = cx < 0 ? 0 : (cx >= G.ncx ? G.ncx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= G.ncx ? G.ncx - 1 : cy);
    cz = cz < 0 ? 0 : (cz >= G.ncz ? G.ncz - 1 : cz);
    return (cx * G.ncx + cy) * G.ncz + cz;
}

__global__ void k_cell_count(const P3MGeom G, const P3MPart S, int* count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.n) return;
    double x, y, z, q;
    if (!load_particle(S, S.o + k, x, y, z, q)) return;
    atomicAdd(&count[cell_of(G, x, y, z)], 1);
}

// Exclusive scan of the cell counts (one CTA of 1024 threads, chunks in order).
__global__ void __launch_bounds__(1024) k_cell_scan(const int* count, int64_t ncells, int* start) {
    __shared__ int warp_sum[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < ncells; c0 += 1024) {
        const int64_t c = c0 + tid;
        const int v = c < ncells ? count[c] : 0;
        int incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = warp_sum[lane], wi = w;
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= d) wi += t;
            }
            warp_sum[lane] = wi - w;
        }
        __syncthreads();
        if (c < ncells) start[c] = carry + warp_sum[warp] + incl - v;
        __syncthreads();
        if (tid == 1023) carry += warp_sum[31] + incl;
        __syncthreads();
    }
    if (tid == 0) start[ncells] = carry;
}

__global__ void k_cell_fill(const P3MGeom G, const P3MPart S, const int* start, int* fill, int* list) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.n) return;
    double x, y, z, q;
    if (!load_particle(S, S.o + k, x, y, z, q)) return;
    const int c = cell_of(G, x, y, z);
    list[start[c] + atomicAdd(&fill[c], 1)] = (int)k;
}

// Each cell's particles in increasing index (the fill order above is not deterministic).
__global__ void k_cell_sort(const int* start, int64_t ncells, int* list) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int b = start[c], e = start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        const int v = list[i];
        int j = i - 1;
        while (j >= b && list[j] > v) { list[j + 1] = list[j]; --j; }
        list[j + 1] = v;
    }
}

// Live particles copied in cell order (FP64 and an FP32 copy of the positions).
__global__ void k_cell_gather(const P3MPart S, const int* start, int64_t ncells, const int* list, double4_32a* s64,
                              float4* s32) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= start[ncells]) return;
    double x, y, z, q;
    load_particle(S, S.o + list[t], x, y, z, q);
    s64[t] = make_double4_32a(x, y, z, q);
    s32[t] = make_float4((float)x, (float)y, (float)z, 0.f);
}

// K_L factor and d/du at u = (alpha r)^2, for the table: the series (2 alpha^3 c / 3)
// (1 - 3u/5 + 3u^2/14) below u = 2.5e-3, the closed form above.
__device__ __forceinline__ double2 long_factor_u(double u, double alpha) {
    const double c = 1.1283791670955126, a3 = alpha * alpha * alpha;
    if (u < 2.5e-3) return make_double2((2.0 / 3.0) * c * a3 * (1.0 - 0.6 * u + (3.0 / 14.0) * u * u),
                                        (2.0 / 3.0) * c * a3 * (-0.6 + (3.0 / 7.0) * u));
    const double r = sqrt(u) / alpha, e = exp(-u), er = erf(sqrt(u));
    const double f = er / (r * r * r) - c * alpha * e / (r * r);
    const double dfdr = -3.0 * er / (r * r * r * r) + 3.0 * c * alpha * e / (r * r * r) + 2.0 * c * a3 * e / r;
    return make_double2(f, dfdr / (2.0 * r * alpha * alpha));   // d/du = (d/dr) / (2 r alpha^2)
}

__global__ void k_lf_table(double alpha, double umax, double2* tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kTab) return;
    tab[k] = long_factor_u(umax * k / kTab, alpha);
}

__device__ __forceinline__ double long_factor_tab(const P3MGeom& G, double r2) {
    const double umax = G.alpha * G.alpha * G.rc * G.rc, hu = umax / kTab;
    const double x = G.alpha * G.alpha * r2 / hu;
    int k = (int)x;
    k = k < 0 ? 0 : (k >= kTab ? kTab - 1 : k);
    const double t = x - k, t2 = t * t, t3 = t2 * t;
    const double2 a = G.lf_tab[k], b = G.lf_tab[k + 1];
    return (2.0 * t3 - 3.0 * t2 + 1.0) * a.x + (t3 - 2.0 * t2 + t) * hu * a.y + (-2.0 * t3 + 3.0 * t2) * b.x +
           (t3 - t2) * hu * b.y;
}

// One short-range pair: q_j (d / max(r, d_c)^3 - K_L(d)) when r < r_cut (FP64).
__device__ __forceinline__ void pp_pair(const P3MGeom& G, const double4_32a& pi, const double4_32a& pj, double invL,
                                        double rc2, double dc2, double& sx, double& sy, double& sz) {
    const double dx = pi.x - pj.x, dy = pi.y - pj.y;
    double dz = pi.z - pj.z;
    dz -= G.L * rint(dz * invL);
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < rc2)) return;
    const double ic = rsqrt(fmax(r2, dc2));             // 1 / max(r, d_c)
    const double f = pj.w * (ic * ic * ic - long_factor_tab(G, r2));
    sx += f * dx; sy += f * dy; sz += f * dz;
}

// Short-range part: q_j (d / max(r, d_c)^3 - K_L(d)) over j != i closer than r_cut, added to sums.
// One warp per particle i (cell order): the lanes screen 32 candidates of the 27 neighbour cells
// at a time in FP32 (r^2 < (r_cut + 1e-3)^2 + 1e-3), the survivors go to a per-warp queue in
// shared memory, and every 32 queued pairs are evaluated in FP64 with all lanes busy; the lanes'
// partial sums are reduced in a fixed order.
constexpr int kPPWarps = 8;
__global__ void __launch_bounds__(32 * kPPWarps) k_p3m_pp(const P3MGeom G, const P3MPart S, const int* start,
                                                          int64_t ncells, const int* list,
                                                          const double4_32a* __restrict__ s64,
                                                          const float4* __restrict__ s32, double* sums) {
    __shared__ int queue[kPPWarps][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* qw = queue[w];
    const int n_live = start[ncells];
    const double rc2 = G.rc * G.rc, dc2 = G.contact * G.contact, invL = 1.0 / G.L;
    const float rcf = (float)G.rc + 1e-3f, rc2f = rcf * rcf + 1e-3f, Lf = (float)G.L, invLf = 1.0f / Lf;
    const unsigned lt = (1u << lane) - 1u;
    for (int t = blockIdx.x * kPPWarps + w; t < n_live; t += gridDim.x * kPPWarps) {
        const double4_32a pi = s64[t];
        const float4 fi = s32[t];
        const int ci = cell_of(G, pi.x, pi.y, pi.z);
        const int cz = ci % G.ncz, cy = (ci / G.ncz) % G.ncx, cx = ci / (G.ncz * G.ncx);
        double sx = 0.0, sy = 0.0, sz = 0.0;
        int qn = 0;
        const int nz = G.ncz >= 3 ? 3 : G.ncz;
        for (int a = cx - 1; a <= cx + 1; ++a) {
            if (a < 0 || a >= G.ncx) continue;
            for (int b = cy - 1; b <= cy + 1; ++b) {
                if (b < 0 || b >= G.ncx) continue;
                for (int u = 0; u < nz; ++u) {
                    int cc = G.ncz >= 3 ? cz - 1 + u : u;
                    if (cc < 0) cc += G.ncz;
                    if (cc >= G.ncz) cc -= G.ncz;
                    const int cell = (a * G.ncx + b) * G.ncz + cc;
                    const int pe = start[cell + 1];
                    for (int p0 = start[cell]; p0 < pe; p0 += 32) {
                        const int p = p0 + lane;
                        bool pass = false;
                        if (p < pe && p != t) {
                            const float4 fj = s32[p];
                            const float ex = fi.x - fj.x, ey = fi.y - fj.y;
                            float ez = fi.z - fj.z;
                            ez -= Lf * rintf(ez * invLf);
                            pass = ex * ex + ey * ey + ez * ez < rc2f;
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, pass);
                        if (pass) qw[qn + __popc(m & lt)] = p;
                        qn += __popc(m);
                        __syncwarp();
                        if (qn >= 32) {
                            pp_pair(G, pi, s64[qw[lane]], invL, rc2, dc2, sx, sy, sz);
                            __syncwarp();
                            if (lane < qn - 32) qw[lane] = qw[32 + lane];
                            qn -= 32;
                            __syncwarp();
                        }
                    }
                }
            }
        }
        if (lane < qn) pp_pair(G, pi, s64[qw[lane]], invL, rc2, dc2, sx, sy, sz);
        __syncwarp();
        for (int d = 16; d > 0; d >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, d);
            sy += __shfl_xor_sync(0xffffffffu, sy, d);
            sz += __shfl_xor_sync(0xffffffffu, sz, d);
        }
        if (lane == 0) {
            const int64_t gi = S.o + list[t];
            sums[3 * gi] += sx;
            sums[3 * gi + 1] += sy;
            sums[3 * gi + 2] += sz;
        }
    }
}

unsigned grid_of(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

int cufft_status(cufftResult r) { return r == CUFFT_SUCCESS ? PDQ_OK : (r == CUFFT_ALLOC_FAILED ? PDQ_ERR_OOM : PDQ_ERR_CUDA); }

P3MGeom geom_of(const pdq_p3m* P, double contact) {
    P3MGeom G;
    G.R = P->R; G.L = P->L; G.h = P->h; G.hz = P->hz; G.x0 = P->x0; G.alpha = P->alpha; G.rc = P->rc;
    G.contact = contact; G.Mx = P->Mx; G.Nx = P->Nx; G.Nz = P->Nz; G.n_img = P->n_img;
    G.ncx = P->ncx; G.ncz = P->ncz;
    G.lf_tab = P->lf_tab;
    return G;
}

void free_plan(pdq_p3m* P) {
    if (!P) return;
    if (P->have_fwd) cufftDestroy(P->fwd);
    if (P->have_inv) cufftDestroy(P->inv);
    cudaFree(P->Gh); cudaFree(P->Q); cudaFree(P->Qh); cudaFree(P->Ah); cudaFree(P->A);
    cudaFree(P->cell_count); cudaFree(P->cell_start); cudaFree(P->cell_fill); cudaFree(P->cell_list);
    cudaFree(P->sorted64); cudaFree(P->sorted32); cudaFree(P->lf_tab);
    cudaFree(P->sums);
    delete P;
}

}  // namespace
}  // namespace pdq

using namespace pdq;

extern "C" int pdq_p3m_create(const pdq_field* field, const pdq_p3m_desc* d, int64_t max_particles,
                              pdq_stream_t stream, pdq_p3m** out) {
    if (!field || !d || !out || max_particles < 1 || max_particles > ((int64_t)1 << 31) - 1 || d->M < 4 ||
        d->Nz < 4 || d->alpha < 0 || d->r_cut < 0 || d->n_img < 0)
        return PDQ_ERR_INVALID_ARG;
    *out = nullptr;
    pdq_p3m* P = new pdq_p3m();
    memset(P, 0, sizeof(*P));
    cudaGetDevice(&P->device);
    P->R = field->desc.r_plus;
    P->L = field->desc.l_plus;
    P->M = d->M;
    P->Nz = d->Nz;
    P->h = 2.0 * P->R / P->M;
    P->hz = P->L / P->Nz;
    P->Mx = P->M + 5;
    P->x0 = -P->R - 2.0 * P->h;
    P->Nx = 2 * P->Mx;
    P->alpha = d->alpha > 0 ? d->alpha : 0.5 / P->h;
    P->rc = d->r_cut > 0 ? d->r_cut : 3.3 / P->alpha;
    P->n_img = d->n_img > 0 ? d->n_img : 200;
    P->max_n = max_particles;
    if (!(P->rc < 0.5 * P->L)) { delete P; return PDQ_ERR_INVALID_ARG; }
    P->nreal = (size_t)P->Nx * P->Nx * P->Nz;
    P->ncplx = (size_t)P->Nx * P->Nx * (P->Nz / 2 + 1);
    P->ncx = std::max(1, (int)floor(2.0 * P->R / P->rc));
    P->ncz = std::max(1, (int)floor(P->L / P->rc));
    P->ncells = (int64_t)P->ncx * P->ncx * P->ncz;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = PDQ_OK;
    double* Gr = nullptr;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc == PDQ_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = PDQ_ERR_OOM;
    };
    alloc((void**)&P->Gh, 3 * P->ncplx * sizeof(cufftDoubleComplex));
    alloc((void**)&P->Q, P->nreal * sizeof(double));
    alloc((void**)&P->Qh, P->ncplx * sizeof(cufftDoubleComplex));
    alloc((void**)&P->Ah, P->ncplx * sizeof(cufftDoubleComplex));
    alloc((void**)&P->A, P->nreal * sizeof(double));
    alloc((void**)&P->cell_count, P->ncells * sizeof(int));
    alloc((void**)&P->cell_start, (P->ncells + 1) * sizeof(int));
    alloc((void**)&P->cell_fill, P->ncells * sizeof(int));
    alloc((void**)&P->cell_list, P->max_n * sizeof(int));
    alloc((void**)&P->sorted64, P->max_n * sizeof(double4_32a));
    alloc((void**)&P->sorted32, P->max_n * sizeof(float4));
    alloc((void**)&P->lf_tab, (kTab + 1) * sizeof(double2));
    alloc((void**)&Gr, 3 * P->nreal * sizeof(double));
    if (rc == PDQ_OK) rc = cufft_status(cufftPlan3d(&P->fwd, P->Nx, P->Nx, P->Nz, CUFFT_D2Z));
    if (rc == PDQ_OK) P->have_fwd = true;
    if (rc == PDQ_OK) rc = cufft_status(cufftPlan3d(&P->inv, P->Nx, P->Nx, P->Nz, CUFFT_Z2D));
    if (rc == PDQ_OK) P->have_inv = true;
    if (rc == PDQ_OK) rc = cufft_status(cufftSetStream(P->fwd, s));
    if (rc == PDQ_OK) {
        const P3MGeom G = geom_of(P, 0.0);
        k_p3m_kernel<<<grid_of(P->nreal, 256), 256, 0, s>>>(G, Gr, Gr + P->nreal, Gr + 2 * P->nreal);
        k_lf_table<<<grid_of(kTab + 1, 256), 256, 0, s>>>(P->alpha, P->alpha * P->alpha * P->rc * P->rc, P->lf_tab);
        for (int c = 0; c < 3 && rc == PDQ_OK; ++c)
            rc = cufft_status(cufftExecD2Z(P->fwd, Gr + c * P->nreal, P->Gh + c * P->ncplx));
        if (rc == PDQ_OK) k_p3m_deconv<<<grid_of(P->ncplx, 256), 256, 0, s>>>(G, P->Gh, (int64_t)P->ncplx);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = PDQ_ERR_CUDA;
    }
    cudaFree(Gr);
    if (rc != PDQ_OK) { free_plan(P); return rc; }
    *out = P;
    return PDQ_OK;
}

extern "C" int pdq_p3m_destroy(pdq_p3m* plan) {
    free_plan(plan);
    return PDQ_OK;
}

extern "C" int pdq_p3m_params(const pdq_p3m* P, double* alpha, double* r_cut, int32_t* n_img, int32_t* nx) {
    if (!P) return PDQ_ERR_INVALID_ARG;
    if (alpha) *alpha = P->alpha;
    if (r_cut) *r_cut = P->rc;
    if (n_img) *n_img = P->n_img;
    if (nx) *nx = P->Nx;
    return PDQ_OK;
}

extern "C" int pdq_p3m_coulomb(pdq_p3m* P, const pdq_phys* phys, const pdq_state* st, double* sums,
                               pdq_stream_t stream) {
    if (!P || !phys || !st || !sums || !st->count || !st->offset || st->n_samples < 1 ||
        (st->cur != 0 && st->cur != 1) || !st->pos[st->cur] || !st->vel[st->cur] ||
        (st->precision != PDQ_FP64 && st->precision != PDQ_MIXED) ||
        (st->precision == PDQ_MIXED && !st->xy[st->cur]))
        return PDQ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (st->n_classes < 1 || st->n_classes > PDQ_MAX_CLASSES) return PDQ_ERR_INVALID_ARG;
    int rc = PDQ_OK;
    const P3MGeom G = geom_of(P, contact_distance(phys, st));
    std::vector<int64_t> off(st->n_samples + 1);
    std::vector<int32_t> cnt(st->n_samples);
    PDQ_CUDA(cudaMemcpyAsync(off.data(), st->offset, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaMemcpyAsync(cnt.data(), st->count, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < st->n_samples; ++k)
        if (cnt[k] < 0 || cnt[k] > P->max_n) return PDQ_ERR_INVALID_ARG;
    PDQ_CUDA(cudaMemsetAsync(sums, 0, (size_t)st->capacity * 3 * sizeof(double), s));
    PDQ_CUDA(cufftSetStream(P->fwd, s) == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown);
    PDQ_CUDA(cufftSetStream(P->inv, s) == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown);
    const int h = st->cur;
    for (int k = 0; k < st->n_samples; ++k) {
        if (cnt[k] == 0) continue;
        P3MPart S;
        S.pos = st->pos[h]; S.vel = st->vel[h]; S.xy = (const double2*)st->xy[h];
        S.o = off[k]; S.n = cnt[k]; S.precision = st->precision;
        const unsigned gp = grid_of(S.n, 256);
        // long range: assign, transform, multiply, transform back, interpolate
        PDQ_CUDA(cudaMemsetAsync(P->Q, 0, P->nreal * sizeof(double), s));
        k_p3m_assign<<<gp, 256, 0, s>>>(G, S, P->Q);
        rc = cufft_status(cufftExecD2Z(P->fwd, P->Q, P->Qh));
        if (rc) return rc;
        for (int c = 0; c < 3; ++c) {
            k_p3m_mul<<<grid_of(P->ncplx, 256), 256, 0, s>>>(P->Qh, P->Gh + c * P->ncplx, P->Ah, (int64_t)P->ncplx);
            rc = cufft_status(cufftExecZ2D(P->inv, P->Ah, P->A));
            if (rc) return rc;
            k_p3m_interp<<<gp, 256, 0, s>>>(G, S, P->A, c, sums);
        }
        // short range: cell list, then the direct sum
        PDQ_CUDA(cudaMemsetAsync(P->cell_count, 0, P->ncells * sizeof(int), s));
        PDQ_CUDA(cudaMemsetAsync(P->cell_fill, 0, P->ncells * sizeof(int), s));
        k_cell_count<<<gp, 256, 0, s>>>(G, S, P->cell_count);
        k_cell_scan<<<1, 1024, 0, s>>>(P->cell_count, P->ncells, P->cell_start);
        k_cell_fill<<<gp, 256, 0, s>>>(G, S, P->cell_start, P->cell_fill, P->cell_list);
        k_cell_sort<<<grid_of(P->ncells, 128), 128, 0, s>>>(P->cell_start, P->ncells, P->cell_list);
        k_cell_gather<<<gp, 256, 0, s>>>(S, P->cell_start, P->ncells, P->cell_list, P->sorted64, P->sorted32);
        k_p3m_pp<<<(unsigned)std::min<int64_t>(grid_of(S.n, kPPWarps), 16 * 152), 32 * kPPWarps, 0, s>>>(
            G, S, P->cell_start, P->ncells, P->cell_list, P->sorted64, P->sorted32, sums);
    }
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

extern "C" int pdq_step_particles_p3m(const pdq_field* field, const pdq_phys* phys, pdq_state* st,
                                      const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                                      pdq_tally* tally, pdq_p3m* P, void* workspace, size_t workspace_bytes,
                                      pdq_stream_t stream) {
    if (!P || !cfg || !st || n_steps < 0 || cfg->use_graph || (cfg->forces & PDQ_F_CONTACT))
        return PDQ_ERR_INVALID_ARG;
    if (st->capacity > P->sums_cap) {
        cudaFree(P->sums);
        P->sums = nullptr;
        P->sums_cap = 0;
        if (cudaMalloc(&P->sums, (size_t)std::max<int64_t>(st->capacity, 1) * 3 * sizeof(double)) != cudaSuccess)
            return PDQ_ERR_OOM;
        P->sums_cap = st->capacity;
    }
    pdq_step_cfg c1 = *cfg;
    c1.compact_every = 0;
    c1.variant = 0;
    for (int64_t k = 0; k < n_steps; ++k) {
        int rc = PDQ_OK;
        if (cfg->forces & PDQ_F_COULOMB) {
            rc = pdq_p3m_coulomb(P, phys, st, P->sums, stream);
            if (rc) return rc;
        }
        rc = step_impl(field, phys, st, params, &c1, 1, tally, workspace, workspace_bytes, stream,
                       (cfg->forces & PDQ_F_COULOMB) ? P->sums : nullptr, false);
        if (rc) return rc;
        if (cfg->compact_every > 0 && st->step % cfg->compact_every == 0 && k + 1 < n_steps) {
            rc = compact_state(st, (cudaStream_t)stream);
            if (rc) return rc;
        }
    }
    return PDQ_OK;
}
