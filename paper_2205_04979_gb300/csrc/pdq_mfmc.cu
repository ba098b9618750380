// pdq_mfmc.cu -- multi-fidelity Monte Carlo allocation and Sobol' estimators
// (Sec. 3 of the paper): FP64 pick-freeze sums on the device, estimator
// assembly on the host.
//
// Model i's evaluations are laid out as y_i[g][col][c]: group g (a shared
// sample sequence, nested across models), column 0 = f(x), 1 = f(x'),
// 2 + j = f(z^(j)) with z^(j) = x' except input j from x, class/output c.
// For every model i and both prefix lengths m_{i-1} and m_i, one CTA reduces,
// per output c, the sums
//   S1 = sum f(x), S2 = sum f(x)^2, R1 = sum f(x'), R2 = sum f(x')^2,
//   P_j = sum f(x) f(z^(j)), Q_j = sum (f(x') - f(z^(j)))^2,
// in a fixed order (deterministic).  Bootstrap replicate b >= 1 replaces group
// position t by an index drawn from word = Philox4x32-10 counter (t, b, 0, 2),
// key = seed, resampled within its nesting block: position t in
// [m_{l-1}, m_l) maps to m_{l-1} + ((word (m_l - m_{l-1})) >> 32); model i
// reads positions t < m_i, so it only touches its own evaluations and the
// nesting of the samples is kept.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pdq_common.cuh"

namespace pdq {

constexpr int kMaxInputs = 16;

struct SumArgs {
    const double* y[8];     // per model, device [n_i][d+2][C]
    int64_t m[8];           // nested counts
    int32_t k, d, C;
    uint2 key;
    double* sums;           // [1+B][k][2][C][4+2d]
};

__global__ void __launch_bounds__(256) k_mfmc_sums(const SumArgs A) {
    const int c = blockIdx.x;
    const int ip = blockIdx.y;           // model i = ip / 2, prefix p = ip % 2
    const int b = blockIdx.z;            // 0 = the sample itself, >= 1 bootstrap
    const int i = ip >> 1, p = ip & 1;
    const int d = A.d, C = A.C, ncol = d + 2, nq = 4 + 2 * d;
    const int64_t m = p ? A.m[i] : (i > 0 ? A.m[i - 1] : A.m[0]);
    const double* __restrict__ y = A.y[i];
    double acc[4 + 2 * kMaxInputs];
    for (int q = 0; q < nq; ++q) acc[q] = 0.0;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        int64_t g = t;
        if (b > 0) {
            // block-wise resampling: position t in [m_{l-1}, m_l) draws from the same block,
            // so every index stays below m_i for the positions model i reads
            int l = 0;
            while (t >= A.m[l]) ++l;
            const int64_t lo = l > 0 ? A.m[l - 1] : 0;
            const uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)b, 0u, 2u), A.key);
            g = lo + (int64_t)(((uint64_t)w.x * (uint64_t)(A.m[l] - lo)) >> 32);
        }
        const double* row = y + g * ncol * C + c;
        const double fx = row[0], fxp = row[C];
        acc[0] += fx; acc[1] += fx * fx; acc[2] += fxp; acc[3] += fxp * fxp;
        for (int j = 0; j < d; ++j) {
            const double fz = row[(2 + j) * C];
            acc[4 + j] += fx * fz;
            const double e = fxp - fz;
            acc[4 + d + j] += e * e;
        }
    }
    __shared__ double red[256];
    double* out = A.sums + ((((int64_t)b * A.k + i) * 2 + p) * C + c) * nq;
    for (int q = 0; q < nq; ++q) {
        red[threadIdx.x] = acc[q];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = red[0];
        __syncthreads();
    }
}

// Host assembly of one replicate: mean, variance, main and total indices per output.
struct Estimates {
    std::vector<double> mean, var, smain, stot;   // [C], [C], [d][C], [d][C]
};

static void assemble(const double* sums, int k, int d, int C, const int64_t* m, const double* alpha, Estimates* e) {
    const int nq = 4 + 2 * d;
    e->mean.assign(C, 0.0); e->var.assign(C, 0.0);
    e->smain.assign((size_t)d * C, 0.0); e->stot.assign((size_t)d * C, 0.0);
    for (int c = 0; c < C; ++c) {
        std::vector<double> Vj(d, 0.0), Tj(d, 0.0);
        double mean = 0.0, var = 0.0;
        for (int i = 0; i < k; ++i) {
            for (int p = 1; p >= (i > 0 ? 0 : 1); --p) {
                const double mm = (double)(p ? m[i] : m[i - 1]);
                const double* s = sums + (((int64_t)i * 2 + p) * C + c) * nq;
                const double E = s[0] / mm, Ep = s[2] / mm;
                const double V = (s[1] - mm * E * E) / (mm - 1.0), Vp = (s[3] - mm * Ep * Ep) / (mm - 1.0);
                // term sign/weight: model 1 enters once; model i >= 2 as alpha_i (y_{m_i} - y_{m_{i-1}})
                const double wgt = i == 0 ? 1.0 : (p ? alpha[i] : -alpha[i]);
                mean += wgt * E;
                var += wgt * V;
                for (int j = 0; j < d; ++j) {
                    // Owen's main-effect estimator and Jansen's total-effect estimator (Sec. 3.3)
                    const double vj = 2.0 * mm / (2.0 * mm - 1.0) *
                                      (s[4 + j] / mm - 0.25 * (E + Ep) * (E + Ep) + (V + Vp) / (4.0 * mm));
                    const double tj = s[4 + d + j] / (2.0 * mm);
                    Vj[j] += wgt * vj;
                    Tj[j] += wgt * tj;
                }
            }
        }
        e->mean[c] = mean;
        e->var[c] = var;
        for (int j = 0; j < d; ++j) {
            e->smain[(size_t)j * C + c] = Vj[j] / var;
            e->stot[(size_t)j * C + c] = Tj[j] / var;
        }
    }
}

}  // namespace pdq

using namespace pdq;

extern "C" int pdq_mfmc_allocate(int32_t k, const double* rho, const double* sigma, const double* w, double budget,
                                 int32_t d_inputs, int64_t* m_out, double* alpha_out, double* m_real_out,
                                 double* gamma_out) {
    if (k < 1 || k > 8 || !rho || !sigma || !w || !m_out || !alpha_out || !(budget > 0) || d_inputs < 0)
        return PDQ_ERR_INVALID_ARG;
    for (int i = 0; i < k; ++i)
        if (!(sigma[i] > 0) || !(w[i] > 0) || !(fabs(rho[i]) <= 1.0)) return PDQ_ERR_INVALID_ARG;
    // rho_{1,1} = 1; rho_{1,k+1} taken as 0.
    std::vector<double> r2(k + 1, 0.0);
    for (int i = 0; i < k; ++i) r2[i] = i == 0 ? 1.0 : rho[i] * rho[i];
    for (int i = 1; i < k; ++i)
        if (!(r2[i] < r2[i - 1])) return PDQ_ERR_PRECOND;                    // models sorted by correlation
    // Eq. (mf-precond): w_{i-1}/w_i > (rho_{i-1}^2 - rho_i^2)/(rho_i^2 - rho_{i+1}^2), i = 2..k
    for (int i = 1; i < k; ++i) {
        const double lhs = w[i - 1] / w[i];
        const double rhs = (r2[i - 1] - r2[i]) / (r2[i] - r2[i + 1]);
        if (!(lhs > rhs)) return PDQ_ERR_PRECOND;
    }
    const double p = d_inputs > 0 ? budget / (d_inputs + 2) : budget;   // effective budget for Sobol' (d+2 runs)
    std::vector<double> r(k);
    double wr = 0.0;
    for (int i = 0; i < k; ++i) {
        // Eq. (opt2): r_i = sqrt(w_1 (rho_i^2 - rho_{i+1}^2) / (w_i (1 - rho_2^2)))
        r[i] = sqrt(w[0] * (r2[i] - r2[i + 1]) / (w[i] * (1.0 - r2[1])));
        wr += w[i] * r[i];
    }
    const double m1 = p / wr;                                             // m_1 = p / (w^T r)
    for (int i = 0; i < k; ++i) {
        const double mi = m1 * r[i];                                      // Eq. (opt3)
        if (m_real_out) m_real_out[i] = mi;
        m_out[i] = (int64_t)floor(mi);
        if (i > 0 && m_out[i] < m_out[i - 1]) m_out[i] = m_out[i - 1];
        alpha_out[i] = i == 0 ? 1.0 : rho[i] * sigma[0] / sigma[i];        // Eq. (opt1)
    }
    if (gamma_out) {
        // MSE of the MFMC mean with the real-valued optimum, relative to MC with the same budget:
        // MSE = sigma_1^2/m_1 + sum_i (1/m_{i-1} - 1/m_i)(alpha_i^2 sigma_i^2 - 2 alpha_i rho_i sigma_1 sigma_i)
        double mse = sigma[0] * sigma[0] / m1;
        for (int i = 1; i < k; ++i) {
            const double a = alpha_out[i];
            mse += (1.0 / (m1 * r[i - 1]) - 1.0 / (m1 * r[i])) *
                   (a * a * sigma[i] * sigma[i] - 2.0 * a * rho[i] * sigma[0] * sigma[i]);
        }
        *gamma_out = mse / (sigma[0] * sigma[0] * w[0] / p);
    }
    return PDQ_OK;
}

extern "C" int pdq_mfmc_workspace_size(int32_t k, int32_t d, int32_t C, int32_t n_boot, size_t* bytes) {
    if (!bytes || k < 1 || k > 8 || d < 1 || d > kMaxInputs || C < 1 || n_boot < 0) return PDQ_ERR_INVALID_ARG;
    *bytes = sizeof(double) * (size_t)(1 + n_boot) * k * 2 * C * (4 + 2 * d);
    return PDQ_OK;
}

extern "C" int pdq_mfmc_sobol(int32_t k, const double* const* y, const int64_t* m, const double* alpha, int32_t d,
                              int32_t C, int32_t n_boot, uint64_t seed, double* mean, double* var, double* s_main,
                              double* s_total, double* s_main_ci, double* s_total_ci, void* workspace,
                              size_t workspace_bytes, pdq_stream_t stream) {
    size_t need = 0;
    int rc = pdq_mfmc_workspace_size(k, d, C, n_boot, &need);
    if (rc) return rc;
    if (!y || !m || !alpha || !mean || !var || !s_main || !s_total) return PDQ_ERR_INVALID_ARG;
    if (n_boot > 0 && (!s_main_ci || !s_total_ci)) return PDQ_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return PDQ_ERR_WORKSPACE;
    for (int i = 0; i < k; ++i) {
        if (!y[i] || m[i] < 2 || (i > 0 && m[i] < m[i - 1])) return PDQ_ERR_INVALID_ARG;
    }
    if ((uint64_t)m[k - 1] > 0xffffffffull) return PDQ_ERR_INVALID_ARG;
    SumArgs A;
    memset(&A, 0, sizeof(A));
    for (int i = 0; i < k; ++i) { A.y[i] = y[i]; A.m[i] = m[i]; }
    A.k = k; A.d = d; A.C = C;
    A.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    A.sums = (double*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    k_mfmc_sums<<<dim3(C, 2 * k, 1 + n_boot), 256, 0, s>>>(A);
    PDQ_CUDA(cudaGetLastError());
    std::vector<double> h(need / sizeof(double));
    PDQ_CUDA(cudaMemcpyAsync(h.data(), workspace, need, cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    const size_t per_rep = (size_t)k * 2 * C * (4 + 2 * d);
    Estimates e;
    assemble(h.data(), k, d, C, m, alpha, &e);
    for (int c = 0; c < C; ++c) { mean[c] = e.mean[c]; var[c] = e.var[c]; }
    for (size_t q = 0; q < (size_t)d * C; ++q) { s_main[q] = e.smain[q]; s_total[q] = e.stot[q]; }
    if (n_boot > 0) {
        // percentile interval: sorted replicate values at ranks round(0.025 (B-1)) and round(0.975 (B-1))
        std::vector<std::vector<double>> bm((size_t)d * C), bt((size_t)d * C);
        for (int b = 1; b <= n_boot; ++b) {
            Estimates eb;
            assemble(h.data() + per_rep * b, k, d, C, m, alpha, &eb);
            for (size_t q = 0; q < (size_t)d * C; ++q) { bm[q].push_back(eb.smain[q]); bt[q].push_back(eb.stot[q]); }
        }
        const int lo = (int)lround(0.025 * (n_boot - 1)), hi = (int)lround(0.975 * (n_boot - 1));
        for (size_t q = 0; q < (size_t)d * C; ++q) {
            std::sort(bm[q].begin(), bm[q].end());
            std::sort(bt[q].begin(), bt[q].end());
            s_main_ci[2 * q] = bm[q][lo]; s_main_ci[2 * q + 1] = bm[q][hi];
            s_total_ci[2 * q] = bt[q][lo]; s_total_ci[2 * q + 1] = bt[q][hi];
        }
    }
    return PDQ_OK;
}

// ---------------------------------------------------------------------------
// Derivative-based global sensitivity (DGSM) bounds on the total Sobol'
// indices (Sobol' & Kucherenko): for inputs uniform on [a_j, b_j],
//   s_j^t <= (b_j - a_j)^2 nu_j / (pi^2 Var f),  nu_j = E[(df/dx_j)^2],
// from S samples of the gradient.  One CTA per (output c, input j) reduces
// sum (df/dx_j)^2; one CTA per output computes the sample variance (two
// passes, divisor S - 1); fixed-order reductions.
// ---------------------------------------------------------------------------
namespace pdq {
__device__ __forceinline__ double block_sum_256(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_dgsm(const double* __restrict__ grad, const double* __restrict__ y, int S,
                                              int C, int d, double* __restrict__ out /*[d+1][C]*/) {
    __shared__ double red[256];
    const int c = blockIdx.x, j = blockIdx.y;   // j == d: variance of y
    if (j < d) {
        double acc = 0.0;
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const double gv = grad[((int64_t)s * C + c) * d + j];
            acc += gv * gv;
        }
        const double tot = block_sum_256(acc, red);
        if (threadIdx.x == 0) out[(int64_t)j * C + c] = tot / S;
    } else {
        double acc = 0.0;
        for (int s = threadIdx.x; s < S; s += blockDim.x) acc += y[(int64_t)s * C + c];
        const double mu = block_sum_256(acc, red) / S;
        double acc2 = 0.0;
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const double e = y[(int64_t)s * C + c] - mu;
            acc2 += e * e;
        }
        const double tot = block_sum_256(acc2, red);
        if (threadIdx.x == 0) out[(int64_t)d * C + c] = tot / (S - 1);
    }
}
}  // namespace pdq

extern "C" int pdq_dgsm_workspace_size(int32_t C, int32_t d, size_t* bytes) {
    if (C < 1 || d < 1 || d > 64 || !bytes) return PDQ_ERR_INVALID_ARG;
    *bytes = sizeof(double) * (size_t)(d + 1) * (size_t)C;
    return PDQ_OK;
}

extern "C" int pdq_dgsm_bounds(int32_t S, int32_t C, int32_t d, const double* grad, const double* y,
                               const double* width, double* nu, double* bound, void* workspace,
                               size_t workspace_bytes, pdq_stream_t stream) {
    if (S < 2 || C < 1 || d < 1 || d > 64 || !grad || !y || !width || !nu || !bound) return PDQ_ERR_INVALID_ARG;
    size_t need = 0;
    pdq_dgsm_workspace_size(C, d, &need);
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 7)) return PDQ_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double* dev = (double*)workspace;   // (d+1) x C results: nu per input, then Var f
    k_dgsm<<<dim3(C, d + 1), 256, 0, s>>>(grad, y, S, C, d, dev);
    std::vector<double> h((size_t)(d + 1) * C);
    PDQ_CUDA(cudaGetLastError());
    PDQ_CUDA(cudaMemcpyAsync(h.data(), dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    PDQ_CUDA(cudaStreamSynchronize(s));
    const double pi2 = kPi * kPi;
    for (int j = 0; j < d; ++j)
        for (int c = 0; c < C; ++c) {
            const double n = h[(size_t)j * C + c], var = h[(size_t)d * C + c];
            nu[(size_t)j * C + c] = n;
            bound[(size_t)j * C + c] = var > 0 ? width[j] * width[j] * n / (pi2 * var) : NAN;
        }
    return PDQ_OK;
}
