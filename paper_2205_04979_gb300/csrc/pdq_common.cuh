// pdq_common.cuh -- internal definitions shared by the libpdq translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pdq.h"

namespace pdq {

constexpr double kPi = 3.14159265358979323846;

// cudaError_t -> status, remembering the last CUDA error text for pdq_strerror.
int cuda_status(cudaError_t e);
#define PDQ_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::pdq::cuda_status(e_); \
    } while (0)

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
// 32-bit word to a double in (0, 1): (w + 1/2) * 2^-32, exact.
__device__ __forceinline__ double unit_open(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

// ---------------------------------------------------------------------------
// Field handle.
// ---------------------------------------------------------------------------
}  // namespace pdq

struct pdq_field {
    pdq_field_desc desc;
    int device;
    double* modes;     // [n_modes][7]
    double4_32a* grid64;   // [n_z][n_th][n_r]
    float4* grid32;
    double y_cross;    // sublayer / log-law crossing
};

namespace pdq {

// ---------------------------------------------------------------------------
// Per-class constants, built on the host from pdq_phys and the class St+.
// ---------------------------------------------------------------------------
struct ClassK {
    double tau;       // tau_p+
    double d_plus;    // diameter, wall units
    double half_d;    // d+/2
    double d_m;       // diameter, m
    double mass;      // kg
    double qfac;      // (d/1um)^2: q_max / q_unit
    double coul;      // Coulomb: a+ = coul * q_i * sum_j q_j r_ij / |r_ij|^3 (q in q_unit, r in wall units)
    double vdw;       // vdW: a+ = zeta * vdw * d^6 / (delta^2 (2d+delta)^2 (d+delta)^3)  (SI lengths)
    double stick;     // 2 A_cont gamma_c / (m zeta) = pi d^2 A0 / (24 pi delta_c^2 m) * ... (m^2/s^2 per unit zeta)
    double d3;        // d+^3 (mass ratios of the contact forces)
    double vdw_pp;    // particle-particle vdW: a+ = zeta * vdw_pp * d^6 / (delta^2 (2d+delta)^2 (d+delta)^3), SI lengths
    double wall2;     // (R+ - d+/2)^2: contact when x^2 + y^2 reaches it (MIXED)
    float tau_f, inv_tau_f, d_plus_f, half_d_f, coul_f, img_f;
    float vdw_reach_f;  // R+ - r below which the wall vdW term may act (3/4 d+, with a margin; MIXED screen)
};

struct StepConst {
    ClassK cls[PDQ_MAX_CLASSES];
    int32_t n_classes;
    int32_t forces;
    int32_t mode;
    int32_t n_r, n_th, n_z;
    int64_t window_start;
    double dt;
    double R, L, invL;       // pipe radius, length (wall units)
    double ell;              // metres per wall unit
    double delta_min;        // m
    double ustar;            // m/s
    double elastic0;         // sigma_y0^2 / (rho_p E), m^2/s^2
    double grav[3];          // gravity acceleration vector, wall units
    double contact2;         // (largest class diameter)^2, wall units
    double near;             // range of the contact forces: 1.25 x largest diameter, wall units
    double col_k, col_h;     // collision spring and damping rates per unit effective mass (wall units)
    double inv_beta, tanh_beta;
    double R2;               // R^2
    float Rf, Lf, invLf, contact2f, dtf, inv_beta_f, tanh_beta_f, gravf[3];
    float th_scale_f, z_scale_f;   // n_th / (2 pi) and n_z / L: cell index per radian and per unit z
    const double4_32a* grid64;
    const float4* grid32;
};

// Fill a StepConst (everything but dt/forces/mode/window and the grids).
int make_step_const(const pdq_field* f, const pdq_phys* p, const pdq_state* st, StepConst* K);

// The particle step with optional given Coulomb sums ext (device [capacity][3]) in place of
// the all-pairs loop (bin = false: no z-binning), and an unsorted compaction (pdq_particles.cu).
int step_impl(const pdq_field* field, const pdq_phys* phys, pdq_state* st, const pdq_sample_params* params,
              const pdq_step_cfg* cfg, int64_t n_steps, pdq_tally* tally, void* workspace, size_t workspace_bytes,
              pdq_stream_t stream, const double* ext, bool bin);
int compact_state(pdq_state* st, cudaStream_t s);
// Largest class diameter of a state in wall units (pdq_particles.cu).
double contact_distance(const pdq_phys* p, const pdq_state* st);

}  // namespace pdq
