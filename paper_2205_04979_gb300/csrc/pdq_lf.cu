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
// Layout: one CTA per (class, block of 256 samples).  The CTA first writes the
// class's per-cell table into shared memory (differences of the turbophoretic
// term and of the two potential shapes, dy/tau and dy/D across each cell: 40 B
// per cell); then each thread marches one sample from the axis (V = 0) to the
// wall.  At every cell it solves the implicit momentum step
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

// T = double: the march in FP64.  T = float (PDQ_MIXED): the cell table and the
// march in FP32 (IEEE square root, division and expm1f; Q summed with Kahan
// compensation), the wall condition and the final ratio in FP64.
template <typename T>
__global__ void __launch_bounds__(kLfThreads) k_lf_vdep(const LfArgs A) {
    extern __shared__ __align__(16) unsigned char lf_smem[];
    T* tab = reinterpret_cast<T*>(lf_smem);   // 5 arrays of n_y - 1 cells: dw, dinv_y, dpsi, dy/tau, dy/D_m
    const int c = blockIdx.y;
    const LfClass K = A.cls[c];
    const int ncell = A.n_y - 1;
    T* t_dw = tab;
    T* t_de = tab + ncell;
    T* t_dv = tab + 2 * ncell;
    T* t_a = tab + 3 * ncell;
    T* t_h = tab + 4 * ncell;
    __shared__ double s_sigma;
    for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
        const LfNode lo = lf_node(A, K, k), hi = lf_node(A, K, k + 1);
        const double dy = hi.y - lo.y;
        t_dw[k] = (T)(hi.w - lo.w);
        t_de[k] = (T)(hi.inv_y - lo.inv_y);
        t_dv[k] = (T)(hi.psi - lo.psi);
        t_a[k] = (T)(dy / K.tau);
        t_h[k] = (T)(dy / (0.5 * (lo.D + hi.D)));
        if (k == 0) s_sigma = sqrt(K.resp * lf_var_at(A, lo.y) + K.thermal);
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    const double xi = A.params[s].xi, zeta = A.params[s].zeta;
    const T ae = (T)(-K.ce * xi * xi), av = (T)(-K.cv * zeta);
    const T half = (T)0.5, two = (T)2, zero = (T)0, one = (T)1;
    T v_out = zero;   // V at node k + 1 (the axis: 0)
    T P = one, Q = zero, Qc = zero;
    for (int k = ncell - 1; k >= 0; --k) {
        // momentum: implicit drag, root <= 0 of V^2/2 - a V = c
        const T a = t_a[k];
        const T c2 = half * v_out * v_out + t_dw[k] + (ae * t_de[k] + av * t_dv[k]);
        T v_in = zero;
        if (c2 > zero) v_in = -two * c2 / (a + sqrt(fma(a, a, two * c2)));
        // continuity: exact cell solution with the cell-mean V and D
        const T vm = half * (v_in + v_out);
        const T am = vm * t_h[k];
        T G = t_h[k], E = one;
        if (am != zero) {
            const T em = expm1(am);
            G = em / vm;
            E = one + em;
        }
        if constexpr (sizeof(T) == sizeof(double)) {
            Q = fma(P, G, Q);
        } else {
            const T yq = fma(P, G, -Qc);
            const T tq = Q + yq;
            Qc = (tq - Q) - yq;
            Q = tq;
        }
        P *= E;
        v_out = v_in;
    }
    // kinetic wall condition: one-way flux of a Gaussian velocity (mean V_w, sd sigma), FP64
    const double u = -(double)v_out, sg = s_sigma;
    const double M = u / (1.4142135623730951 * sg);
    const double Kw = -(0.5 * u * (1.0 + erf(M)) + sg * exp(-M * M) * 0.3989422804014327);
    const double Qd = (double)Q - (double)Qc;
    A.vdep[s * A.C + c] = -Kw / ((double)P - Kw * Qd);
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
    if ((n_samples + kLfThreads - 1) / kLfThreads > 0x7fffffff) return PDQ_ERR_INVALID_ARG;
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
    const dim3 grid((unsigned)((n_samples + kLfThreads - 1) / kLfThreads), (unsigned)n_classes);
    if (lf->precision == PDQ_FP64) {
        const size_t smem = lf_shared_bytes(lf->n_y, sizeof(double));
        PDQ_CUDA(cudaFuncSetAttribute(k_lf_vdep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lf_vdep<double><<<grid, kLfThreads, smem, (cudaStream_t)stream>>>(A);
    } else {
        const size_t smem = lf_shared_bytes(lf->n_y, sizeof(float));
        PDQ_CUDA(cudaFuncSetAttribute(k_lf_vdep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lf_vdep<float><<<grid, kLfThreads, smem, (cudaStream_t)stream>>>(A);
    }
    PDQ_CUDA(cudaGetLastError());
    return PDQ_OK;
}
