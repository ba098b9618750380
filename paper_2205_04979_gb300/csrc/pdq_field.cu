// pdq_field.cu -- synthetic carrier field: random Fourier modes and the gridded
// velocity (the stand-in for the paper's DNS field, App. A.1).
//
// u = U+(R - r) e_z + curl( (1 - r^2/R^2)^2 sum_n b_n cos(k_n . x + phi_n) ).
// The curl of one mode expands to cos(.) (grad f x b) - f sin(.) (k x b); both
// f and grad f vanish at r = R, so the fluctuation obeys no-slip, and the curl
// makes it divergence-free.
#include <math.h>
#include <stdlib.h>

#include "pdq_common.cuh"

namespace pdq {

// One thread per mode: draw (k, b, phi) from Philox counters (n, 0, 0, 1) and (n, 1, 0, 1).
__global__ void k_field_modes(pdq_field_desc d, uint2 key, double* __restrict__ modes) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.n_modes) return;
    const uint4 a = philox4x32_10(make_uint4((uint32_t)n, 0u, 0u, 1u), key);
    const uint4 b = philox4x32_10(make_uint4((uint32_t)n, 1u, 0u, 1u), key);
    const double twopi = 2.0 * kPi;
    const double kmag = d.k_min * pow(d.k_max / d.k_min, unit_open(a.x));
    const double ct = 2.0 * unit_open(a.y) - 1.0;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sph, cph;
    sincos(twopi * unit_open(a.z), &sph, &cph);
    double k[3] = {kmag * st * cph, kmag * st * sph, kmag * ct};
    const double dkz = twopi / d.l_plus;
    k[2] = dkz * rint(k[2] / dkz);                 // lattice of the periodic length
    const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    const double kp = sqrt(k[0] * k[0] + k[1] * k[1]);
    double e1[3];
    if (kp > 0.0) { e1[0] = k[1] / kp; e1[1] = -k[0] / kp; e1[2] = 0.0; }
    else { e1[0] = 1.0; e1[1] = 0.0; e1[2] = 0.0; }
    const double h[3] = {k[0] / kn, k[1] / kn, k[2] / kn};
    const double e2[3] = {h[1] * e1[2] - h[2] * e1[1], h[2] * e1[0] - h[0] * e1[2], h[0] * e1[1] - h[1] * e1[0]};
    double sps, cps;
    sincos(twopi * unit_open(a.w), &sps, &cps);
    const double bm = d.u_rms * sqrt(6.0 / d.n_modes) / kn;
    double* m = modes + 7 * n;
    m[0] = k[0]; m[1] = k[1]; m[2] = k[2];
    for (int c = 0; c < 3; ++c) m[3 + c] = bm * (cps * e1[c] + sps * e2[c]);
    m[6] = twopi * unit_open(b.x);
}

// One thread per node; the mode table is staged in shared memory with k x b.
__global__ void k_field_grid(pdq_field_desc d, double y_cross, const double* __restrict__ modes,
                             double4_32a* __restrict__ g64, float4* __restrict__ g32) {
    extern __shared__ double sm[];   // [n_modes][10]: k, b, phi, k x b
    for (int t = threadIdx.x; t < d.n_modes; t += blockDim.x) {
        const double* m = modes + 7 * t;
        double* s = sm + 10 * t;
        for (int c = 0; c < 7; ++c) s[c] = m[c];
        s[7] = m[1] * m[5] - m[2] * m[4];
        s[8] = m[2] * m[3] - m[0] * m[5];
        s[9] = m[0] * m[4] - m[1] * m[3];
    }
    __syncthreads();
    const int64_t nodes = (int64_t)d.n_r * d.n_th * d.n_z;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nodes) return;
    const int i = (int)(id % d.n_r);
    const int j = (int)((id / d.n_r) % d.n_th);
    const int kz = (int)(id / ((int64_t)d.n_r * d.n_th));
    const double R = d.r_plus;
    const double r = R * tanh(d.beta * ((double)i / (d.n_r - 1))) / tanh(d.beta);
    double sth, cth;
    sincos(2.0 * kPi * j / d.n_th, &sth, &cth);
    const double x = r * cth, y = r * sth, z = d.l_plus * kz / d.n_z;
    const double one_m = 1.0 - (x * x + y * y) / (R * R);
    double f = 0.0, gx = 0.0, gy = 0.0;
    if (r < R) { f = one_m * one_m; gx = -4.0 * one_m * x / (R * R); gy = -4.0 * one_m * y / (R * R); }
    double S0 = 0, S1 = 0, S2 = 0, T0 = 0, T1 = 0, T2 = 0;
    for (int n = 0; n < d.n_modes; ++n) {
        const double* s = sm + 10 * n;
        double sa, ca;
        sincos(s[0] * x + s[1] * y + s[2] * z + s[6], &sa, &ca);
        S0 += ca * s[3]; S1 += ca * s[4]; S2 += ca * s[5];
        T0 += sa * s[7]; T1 += sa * s[8]; T2 += sa * s[9];
    }
    // grad f = (gx, gy, 0)
    double ux = gy * S2 - f * T0;
    double uy = -gx * S2 - f * T1;
    double uz = gx * S1 - gy * S0 - f * T2;
    const double yp = fmax(R - r, 0.0);
    uz += (yp <= y_cross) ? yp : log(yp) / d.kappa + d.b_log;
    g64[id] = make_double4_32a(ux, uy, uz, 0.0);
    g32[id] = make_float4((float)ux, (float)uy, (float)uz, 0.0f);
}

// Crossing of U+ = y+ and U+ = ln(y+)/kappa + B (the larger root), by Newton from y = 30.
static double law_of_wall_crossing(double kappa, double B) {
    double y = 30.0;
    for (int it = 0; it < 100; ++it) {
        const double g = y - log(y) / kappa - B;
        const double dg = 1.0 - 1.0 / (kappa * y);
        const double yn = y - g / dg;
        if (fabs(yn - y) <= 1e-15 * y) { y = yn; break; }
        y = yn;
    }
    return y;
}

}  // namespace pdq

using namespace pdq;

extern "C" int pdq_create_pipe_field(const pdq_field_desc* desc, uint64_t seed, pdq_stream_t stream, pdq_field** out) {
    if (!desc || !out) return PDQ_ERR_INVALID_ARG;
    const pdq_field_desc d = *desc;
    if (d.n_r < 2 || d.n_th < 1 || d.n_z < 1 || d.n_modes < 0 || d.n_modes > 4096 || !(d.r_plus > 0) ||
        !(d.l_plus > 0) || !(d.beta > 0) || !(d.kappa > 0) || !(d.k_min > 0) || !(d.k_max >= d.k_min) ||
        !(d.u_rms >= 0))
        return PDQ_ERR_INVALID_ARG;
    const int64_t nodes = (int64_t)d.n_r * d.n_th * d.n_z;
    if (nodes > (int64_t)1 << 31) return PDQ_ERR_INVALID_ARG;
    pdq_field* f = (pdq_field*)calloc(1, sizeof(pdq_field));
    if (!f) return PDQ_ERR_OOM;
    f->desc = d;
    f->y_cross = law_of_wall_crossing(d.kappa, d.b_log);
    cudaGetDevice(&f->device);
    cudaStream_t s = (cudaStream_t)stream;
    int st = PDQ_OK;
    if (cudaMalloc(&f->modes, sizeof(double) * 7 * (d.n_modes > 0 ? d.n_modes : 1)) != cudaSuccess ||
        cudaMalloc(&f->grid64, sizeof(double4_32a) * nodes) != cudaSuccess ||
        cudaMalloc(&f->grid32, sizeof(float4) * nodes) != cudaSuccess) {
        cudaGetLastError();
        st = PDQ_ERR_OOM;
    }
    if (st == PDQ_OK) {
        const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        if (d.n_modes > 0) k_field_modes<<<(d.n_modes + 63) / 64, 64, 0, s>>>(d, key, f->modes);
        const size_t smem = sizeof(double) * 10 * (d.n_modes > 0 ? d.n_modes : 1);
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_field_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_field_grid<<<(unsigned)((nodes + 255) / 256), 256, smem, s>>>(d, f->y_cross, f->modes, f->grid64, f->grid32);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    if (st != PDQ_OK) {
        pdq_destroy_pipe_field(f);
        return st;
    }
    *out = f;
    return PDQ_OK;
}

extern "C" int pdq_destroy_pipe_field(pdq_field* f) {
    if (!f) return PDQ_ERR_INVALID_ARG;
    if (f->modes) cudaFree(f->modes);
    if (f->grid64) cudaFree(f->grid64);
    if (f->grid32) cudaFree(f->grid32);
    free(f);
    return PDQ_OK;
}

extern "C" int pdq_field_views(const pdq_field* f, pdq_field_desc* desc, const void** grid64, const void** grid32,
                               const double** modes) {
    if (!f) return PDQ_ERR_INVALID_ARG;
    if (desc) *desc = f->desc;
    if (grid64) *grid64 = f->grid64;
    if (grid32) *grid32 = f->grid32;
    if (modes) *modes = f->modes;
    return PDQ_OK;
}

extern "C" int pdq_field_copy(const pdq_field* f, void* grid64, void* grid32, void* modes, pdq_stream_t stream) {
    if (!f) return PDQ_ERR_INVALID_ARG;
    const size_t nodes = (size_t)f->desc.n_r * f->desc.n_th * f->desc.n_z;
    cudaStream_t s = (cudaStream_t)stream;
    if (grid64) PDQ_CUDA(cudaMemcpyAsync(grid64, f->grid64, nodes * sizeof(double4_32a), cudaMemcpyDefault, s));
    if (grid32) PDQ_CUDA(cudaMemcpyAsync(grid32, f->grid32, nodes * sizeof(float4), cudaMemcpyDefault, s));
    if (modes && f->desc.n_modes > 0)
        PDQ_CUDA(cudaMemcpyAsync(modes, f->modes, sizeof(double) * 7 * f->desc.n_modes, cudaMemcpyDefault, s));
    return PDQ_OK;
}
