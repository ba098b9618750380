// pdq_lf.cu -- the 1-D Eulerian low-fidelity deposition model of App. B,
// batched over (sample, size class) items.
//
// Per item the model is two ODEs in the wall distance y of the particle
// centre (wall units; V = mean wall-normal particle velocity, < 0 toward the
// wall; rho = particle density over its value on the axis):
//   momentum   d/dy(V^2/2 + R v_f'^2 + Phi) = -V/tau_1     (Eq. mom_modified,
//              Phi the potentials of F_elec and F_vdw, R v_f'^2 the
//              turbophoretic term),
//   continuity J = -(D_B + eps) rho' + rho V = const, V_dep+ = -J, with the
//              kinetic wall condition J = rho_w K(V_w) at contact y = d/2.
// The closures App. B cites but does not print: v_f'^2 = (theta, z) variance
// of the synthetic field's radial velocity, R = T_L/(T_L + tau_p),
// eps = v_f'^2 T_L, tau_1 = tau_p, D_B = k_B T tau_p/m_p, isothermal gas,
// M_r = -V_w/(sqrt(2) sigma) with sigma^2 = R v_f'^2 + k_B T/m_p at contact.
//
// Layout: CTAs per class in one wave, each walking blocks of 256 samples.  A
// CTA first writes the class's per-cell table into shared memory (differences
// of the turbophoretic term and of the two potential shapes, dy/tau and dy/D
// across each cell: 40 B per cell in FP64, 20 B in FP32); then each thread
// marches one sample from the axis (V = 0) to the wall.  At every cell it solves the implicit momentum step
//   V_k^2/2 - a V_k = c,  a = dy/tau,  c = V_{k+1}^2/2 + dw + dPhi,
// taking the root V_k <= 0 in the cancellation-free form -2c/(a + sqrt(a^2+2c))
// (V_k = 0 where c < 0), and composes the exact cell solution of the flux
// equation with V and D at their cell means (exponential fitting):
//   rho_{k+1} = E_k rho_k - J G_k,  E_k = e^{a'}, G_k = (e^{a'} - 1)/V_m,
//   a' = V_m dy/D_m,
// inward as rho_axis = P rho_k - J Q (P <- P E_k, Q <- Q + P G_k), so nothing
// per node is stored.  At the wall J = rho_w K and rho_axis = 1 give
// V_dep+ = -K/(P - K Q).  PDQ_FP64 marches in FP64 (bound by the FP64 pipe);
// PDQ_MIXED marches in FP32 with the wall condition and the final ratio in
// FP64.  Either way the ~2,000 cells per item are tiny next to one
// high-fidelity sample.
#include <math.h>
#include <string.h>

#include "pdq_common.cuh"

namespace pdq {

constexpr double kBoltzmann = 1.380649e-23;   // J/K
constexpr int kLfThreads = 256;

struct LfClass {
    double tau;       // tau_p+ = tau_1+
    double y_w;       // contact distance d+/2
    double resp;      // R = T_L/(T_L + tau_p)
    double d_b;       // D_B / nu
    double thermal;   // k_B T / (m u*^2)
    double ce;        // Phi_elec+ = -ce xi^2 / y+
    double cv;        // Phi_vdw+ = -cv zeta psi(gap+)
};

struct LfArgs {
    LfClass cls[PDQ_MAX_CLASSES];
    int32_t C, n_y, n_r;
    int64_t S;
    double R, beta, tanh_beta, stretch, em1_stretch, t_lagr, cut;
    const double* var;                    // [n_r], at the field's radial nodes
    const pdq_sample_params* params;      // [S]
    double* vdep;                         // [S][C]
};

// Fluid variance at wall distance y: linear in the stretched radial coordinate
// s = atanh(r tanh(beta)/R)/beta between the field's nodes s_i = i/(n_r - 1).
__device__ __forceinline__ double lf_var_at(const LfArgs& A, double y) {
    const double r = A.R - y;
    const double s = atanh(r * A.tanh_beta / A.R) / A.beta;
    const double t = s * (double)(A.n_r - 1);
    int i = (int)floor(t);
    i = i > A.n_r - 2 ? A.n_r - 2 : i;
    i = i < 0 ? 0 : i;
    const double f = t - (double)i;
    return (1.0 - f) * A.var[i] + f * A.var[i + 1];
}

// vdW potential shape: psi = 1/gap beyond the cutoff, linear inside it (force held constant).
__device__ __forceinline__ double lf_psi(double gap, double cut) {
    return gap >= cut ? 1.0 / gap : 2.0 / cut - gap / (cut * cut);
}

struct LfNode {
    double y, w, D, inv_y, psi;
};

__device__ __forceinline__ LfNode lf_node(const LfArgs& A, const LfClass& K, int k) {
    LfNode n;
    const double s = (double)k / (double)(A.n_y - 1);
    n.y = K.y_w + (A.R - K.y_w) * expm1(A.stretch * s) / A.em1_stretch;
    const double v = lf_var_at(A, n.y);
    n.w = K.resp * v;
    n.D = K.d_b + v * A.t_lagr;
    n.inv_y = 1.0 / n.y;
    n.psi = lf_psi(n.y - K.y_w, A.cut);
    return n;
}

// One cell of the class table: differences of R v_f'^2 and of the two potential
// shapes across the cell and dy/tau (16 B in FP32, one shared-memory load; the
// cell's dy/D_m sits in a second array).
template <typename T>
struct __align__(16) LfCell {
    T dw, de, dv, a;
};

// exp(x) - 1 over x, for the FP32 march (x <= 0): Taylor polynomial below
// |x| = 0.5 (terms to x^8/9!, truncation < 1e-9 relative), the approximate
// exponential beyond (E - 1 then stays below -0.39, so its relative rounding
// does not grow).  Returns phi and E = 1 + x phi.
__device__ __forceinline__ float lf_phi(float x, float* E) {
    if (x > -0.5f) {
        float p = 2.7557319e-6f;                  // 1/9!
        p = fmaf(p, x, 2.4801587e-5f);            // 1/8!
        p = fmaf(p, x, 1.9841270e-4f);            // 1/7!
        p = fmaf(p, x, 1.3888889e-3f);            // 1/6!
        p = fmaf(p, x, 8.3333333e-3f);            // 1/5!
        p = fmaf(p, x, 4.1666667e-2f);            // 1/4!
        p = fmaf(p, x, 1.6666667e-1f);            // 1/3!
        p = fmaf(p, x, 0.5f);                     // 1/2!
        p = fmaf(p, x, 1.0f);
        *E = fmaf(x, p, 1.0f);
        return p;
    }
    const float e = __expf(x);
    *E = e;
    return __fdividef(e - 1.0f, x);
}

// T = double: the march in FP64.  T = float (PDQ_MIXED): the cell table and the
// march in FP32 (root by x rsqrt(x) and an approximate division, the cell's
// exponential by lf_phi; Q summed with Kahan compensation), the wall
// condition and the final ratio in FP64.  Each CTA builds its class's table
// once and walks blocks of 256 samples blockIdx.x, blockIdx.x + gridDim.x, ...
template <typename T>
__global__ void __launch_bounds__(kLfThreads) k_lf_vdep(const LfArgs A) {
    extern __shared__ __align__(16) unsigned char lf_smem[];
    const int c = blockIdx.y;
    const LfClass K = A.cls[c];
    const int ncell = A.n_y - 1;
    LfCell<T>* cell = reinterpret_cast<LfCell<T>*>(lf_smem);
    T* t_h = reinterpret_cast<T*>(cell + ncell);
    __shared__ double s_sigma;
    for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
        const LfNode lo = lf_node(A, K, k), hi = lf_node(A, K, k + 1);
        const double dy = hi.y - lo.y;
        LfCell<T> e;
        e.dw = (T)(hi.w - lo.w);
        e.de = (T)(hi.inv_y - lo.inv_y);
        e.dv = (T)(hi.psi - lo.psi);
        e.a = (T)(dy / K.tau);
        cell[k] = e;
        t_h[k] = (T)(dy / (0.5 * (lo.D + hi.D)));
        if (k == 0) s_sigma = sqrt(K.resp * lf_var_at(A, lo.y) + K.thermal);
    }
    __syncthreads();
    const double sg = s_sigma;
    const int64_t nblk = (A.S + kLfThreads - 1) / kLfThreads;
    for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int64_t s = b * kLfThreads + threadIdx.x;
        if (s >= A.S) continue;
        const double xi = A.params[s].xi, zeta = A.params[s].zeta;
        const T ae = (T)(-K.ce * xi * xi), av = (T)(-K.cv * zeta);
        const T half = (T)0.5, two = (T)2, zero = (T)0, one = (T)1;
        T v_out = zero;   // V at node k + 1 (the axis: 0)
        T P = one, Q = zero, Qc = zero;
        for (int k = ncell - 1; k >= 0; --k) {
            const LfCell<T> e = cell[k];
            const T h = t_h[k];
            // momentum: implicit drag, root <= 0 of V^2/2 - a V = c
            const T c2 = half * v_out * v_out + e.dw + (ae * e.de + av * e.dv);
            T v_in = zero;
            T G, E;
            if constexpr (sizeof(T) == sizeof(double)) {
                if (c2 > zero) v_in = -two * c2 / (e.a + sqrt(fma(e.a, e.a, two * c2)));
                // continuity: exact cell solution with the cell-mean V and D
                const T vm = half * (v_in + v_out);
                const T am = vm * h;
                G = h;
                E = one;
                if (am != zero) {
                    const T em = expm1(am);
                    G = em / vm;
                    E = one + em;
                }
                Q = fma(P, G, Q);
            } else {
                if (c2 > zero) {
                    const float x = fmaf(e.a, e.a, two * c2);
                    v_in = __fdividef(-two * c2, e.a + x * rsqrtf(x));
                }
                const float am = half * (v_in + v_out) * h;   // <= 0
                G = h * lf_phi(am, &E);
                const T yq = fma(P, G, -Qc);
                const T tq = Q + yq;
                Qc = (tq - Q) - yq;
                Q = tq;
            }
            P *= E;
            v_out = v_in;
        }
        // kinetic wall condition: one-way flux of a Gaussian velocity (mean V_w, sd sigma), FP64
        const double u = -(double)v_out;
        const double M = u / (1.4142135623730951 * sg);
        const double Kw = -(0.5 * u * (1.0 + erf(M)) + sg * exp(-M * M) * 0.3989422804014327);
        const double Qd = (double)Q - (double)Qc;
        A.vdep[s * A.C + c] = -Kw / ((double)P - Kw * Qd);
    }
}

// Population variance over (theta, z) of u_r = cos(theta) u_x + sin(theta) u_y
// at radial node blockIdx.x, two passes (mean, then centred squares), fixed
// reduction order.
__global__ void __launch_bounds__(256) k_lf_variance(const double4_32a* __restrict__ g, int n_r, int n_th, int n_z,
                                                     double* __restrict__ var) {
    const int i = blockIdx.x;
    const int64_t n = (int64_t)n_th * n_z;
    __shared__ double red[256];
    double mean = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        double acc = 0.0;
        for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
            const int j = (int)(t % n_th);
            const double4_32a u = g[t * n_r + i];
            double sn, cs;
            sincos(2.0 * kPi * j / n_th, &sn, &cs);
            const double ur = cs * u.x + sn * u.y;
            const double e = pass == 0 ? ur : ur - mean;
            acc += pass == 0 ? e : e * e;
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        const double tot = red[0] / (double)n;
        __syncthreads();
        if (pass == 0) mean = tot;
        else if (threadIdx.x == 0) var[i] = tot;
    }
}

}  // namespace pdq

using namespace pdq;

extern "C" void pdq_lf_desc_default(pdq_lf_desc* out) {
    if (!out) return;
    memset(out, 0, sizeof(*out));
    out->n_y = 2048;
    out->precision = PDQ_FP64;
    out->stretch = 8.0;
    out->t_lagr = 10.0;
    out->temperature = 293.15;
    out->vdw_cutoff = 1e-12;
}

extern "C" int pdq_lf_fluid_variance(const pdq_field* field, double* var, pdq_stream_t stream) {
    if (!field || !var) return PDQ_ERR_INVALID_ARG;
    const pdq_field_desc& d = field->desc;
    k_lf_variance<<<d.n_r, 256, 0, (cudaStream_t)stream>>>(field->grid64, d.n_r, d.n_th, d.n_z, var);
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

static size_t lf_shared_bytes(int32_t n_y, size_t elem) { return (size_t)5 * (size_t)(n_y - 1) * elem; }

// One wave: as many CTAs per class as fit on the GPU at once (its SMs times the
// resident CTAs per SM, divided among the classes), each building its class's
// table once and walking ceil(blocks / CTAs) sample blocks.
template <typename T>
static int launch_lf(const LfArgs& A, pdq_stream_t stream) {
    const size_t smem = lf_shared_bytes(A.n_y, sizeof(T));
    PDQ_CUDA(cudaFuncSetAttribute(k_lf_vdep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    PDQ_CUDA(cudaGetDevice(&dev));
    PDQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PDQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lf_vdep<T>, kLfThreads, smem));
    const int64_t nblk = (A.S + kLfThreads - 1) / kLfThreads;
    int64_t gx = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) / A.C;
    if (gx < 1) gx = 1;
    if (gx > nblk) gx = nblk;
    const dim3 grid((unsigned)gx, (unsigned)A.C);
    k_lf_vdep<T><<<grid, kLfThreads, smem, (cudaStream_t)stream>>>(A);
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}

extern "C" int pdq_lf_vdep(const pdq_field* field, const pdq_phys* phys, const pdq_lf_desc* lf, const double* var,
                           int32_t n_classes, const double* st_plus, int64_t n_samples,
                           const pdq_sample_params* params, double* vdep, pdq_stream_t stream) {
    if (!field || !phys || !lf || !var || !st_plus || n_samples < 0) return PDQ_ERR_INVALID_ARG;
    if (n_classes < 1 || n_classes > PDQ_MAX_CLASSES) return PDQ_ERR_INVALID_ARG;
    if (lf->n_y < 3 || lf->n_y > PDQ_LF_MAX_NODES) return PDQ_ERR_INVALID_ARG;
    if (lf->precision != PDQ_FP64 && lf->precision != PDQ_MIXED) return PDQ_ERR_INVALID_ARG;
    if (!(lf->stretch > 0.0) || !(lf->stretch <= 700.0) || !(lf->t_lagr > 0.0) || !(lf->temperature > 0.0) ||
        !(lf->vdw_cutoff > 0.0))
        return PDQ_ERR_INVALID_ARG;
    if (field->desc.n_r < 2) return PDQ_ERR_INVALID_ARG;
    if (fabs(field->desc.r_plus - phys->re_tau) > 1e-9 * phys->re_tau) return PDQ_ERR_INVALID_ARG;
    if (n_samples == 0) return PDQ_OK;
    if (!params || !vdep) return PDQ_ERR_INVALID_ARG;
    const double ustar = phys->re_tau * phys->nu / phys->radius;
    const double ell = phys->nu / ustar;
    const double tauf = phys->nu / (ustar * ustar);
    const double acc = phys->nu / (ustar * ustar * ustar);
    LfArgs A;
    memset(&A, 0, sizeof(A));
    for (int c = 0; c < n_classes; ++c) {
        const double tau = st_plus[c];
        if (!(tau > 0.0)) return PDQ_ERR_INVALID_ARG;
        // tau_p = rho_p d^2/(18 rho_f nu), tau_p+ = tau_p/tau_f (Sec. 2.1)
        const double d = sqrt(18.0 * phys->rho_f * phys->nu * tau * tauf / phys->rho_p);
        const double m = phys->rho_p * kPi * d * d * d / 6.0;
        const double q1 = phys->q_unit * (d * 1e6) * (d * 1e6);     // q_max of the class
        LfClass& K = A.cls[c];
        K.tau = tau;
        K.y_w = 0.5 * d / ell;
        if (!(K.y_w < field->desc.r_plus)) return PDQ_ERR_INVALID_ARG;
        K.resp = lf->t_lagr / (lf->t_lagr + tau);
        K.d_b = kBoltzmann * lf->temperature * (tau * tauf) / m / phys->nu;
        K.thermal = kBoltzmann * lf->temperature / m / (ustar * ustar);
        // F_elec = -3 q^2/(8 pi^2 eps0 rho_p d^3 y^2), F_vdw = -A d/(12 m gap^2) per unit mass (App. B)
        K.ce = 3.0 * q1 * q1 / (8.0 * kPi * kPi * phys->eps0 * phys->rho_p * d * d * d) * acc / (ell * ell);
        K.cv = phys->hamaker0 * d / (12.0 * m) * acc / (ell * ell);
    }
    A.C = n_classes;
    A.n_y = lf->n_y;
    A.n_r = field->desc.n_r;
    A.S = n_samples;
    A.R = field->desc.r_plus;
    A.beta = field->desc.beta;
    A.tanh_beta = tanh(field->desc.beta);
    A.stretch = lf->stretch;
    A.em1_stretch = expm1(lf->stretch);
    A.t_lagr = lf->t_lagr;
    A.cut = lf->vdw_cutoff / ell;
    A.var = var;
    A.params = params;
    A.vdep = vdep;
    if (lf->precision == PDQ_FP64) return launch_lf<double>(A, stream);
    return launch_lf<float>(A, stream);
}
