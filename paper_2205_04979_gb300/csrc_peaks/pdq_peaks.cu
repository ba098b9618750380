// pdq_peaks.cu -- throughput microbenchmarks that give the roofline denominators of the
// particle kernels on the GPU they run on: FP32 FMA (scalar and packed f32x2), packed FP32
// add, FP64 FMA, the MUFU reciprocal square root, and L2 read bandwidth.
//
// Each compute kernel runs CH independent dependency chains per thread for `iters` rounds, so
// the pipes, not latency, bound it when enough warps are resident; the result is folded into a
// value stored only under a condition the data never meet, which keeps the chains live.  The
// host entry point times one launch with CUDA events after one untimed launch.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int CH = 8;

__device__ __forceinline__ uint64_t pk(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float pk_sum(uint64_t v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a + b;
}

// kind 0: scalar FFMA, x = x * a + b
__global__ void k_ffma(float* sink, int iters, float a, float b) {
    float x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

// kind 1: packed FFMA2 (fma.rn.f32x2), two FMAs per lane per instruction
__global__ void k_ffma2(float* sink, int iters, float a, float b) {
    uint64_t x[CH];
    const uint64_t A = pk(a, a), B = pk(b, b);
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = pk(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)(threadIdx.x + i));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(A), "l"(B));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += pk_sum(x[i]);
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

// kind 2: packed FADD2 (add.rn.f32x2)
__global__ void k_fadd2(float* sink, int iters, float a, float b) {
    uint64_t x[CH];
    const uint64_t B = pk(b, -b);
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = pk(a * (float)(threadIdx.x + i), 2e-3f * (float)(threadIdx.x + i));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(x[i]) : "l"(B));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += pk_sum(x[i]);
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

// kind 3: FP64 FMA
__global__ void k_dfma(float* sink, int iters, float a, float b) {
    double x[CH];
    const double A = a, B = b;
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = fma(x[i], A, B);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == -1.2345) sink[threadIdx.x] = (float)s;
}

// kind 4: MUFU reciprocal square root (rsqrt.approx.ftz.f32); x -> rsqrt(x) stays near 1
__global__ void k_rsqrt(float* sink, int iters, float a, float b) {
    float x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[i]));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == -1.2345f) sink[threadIdx.x] = s + a + b;
}

// kind 5: L2 read bandwidth: every thread sums float4 loads of a buffer small enough to stay in
// L2, `iters` passes, grid-stride
__global__ void k_l2read(const float4* __restrict__ buf, int64_t n4, float* sink, int iters) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == -1.2345f) sink[threadIdx.x] = s;
}

}  // namespace

// Operations per thread per round of `iters`: 4 x CH (instructions; flops follow from the kind).
extern "C" int pk_ops_per_iter(void) { return 4 * CH; }

// Time one launch of kernel `kind` (0..4: blocks x threads, `iters` rounds; 5: L2 reads of a
// buffer of `l2_bytes`, `iters` passes) after one untimed launch.  *ms receives the event time.
// Returns 0 or the CUDA error code.
extern "C" int pk_time(int kind, int blocks, int threads, int iters, int64_t l2_bytes, float* ms) {
    float* sink = nullptr;
    float4* buf = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * 1024);
    if (e != cudaSuccess) return (int)e;
    const int64_t n4 = l2_bytes / 16;
    if (kind == 5) {
        e = cudaMalloc(&buf, (size_t)n4 * 16);
        if (e == cudaSuccess) e = cudaMemset(buf, 0, (size_t)n4 * 16);
        if (e != cudaSuccess) { cudaFree(sink); return (int)e; }
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const float a = 0.9999999f, b = 1e-7f;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(t0);
        switch (kind) {
            case 0: k_ffma<<<blocks, threads>>>(sink, iters, a, b); break;
            case 1: k_ffma2<<<blocks, threads>>>(sink, iters, a, b); break;
            case 2: k_fadd2<<<blocks, threads>>>(sink, iters, a, b); break;
            case 3: k_dfma<<<blocks, threads>>>(sink, iters, a, b); break;
            case 4: k_rsqrt<<<blocks, threads>>>(sink, iters, a, b); break;
            case 5: k_l2read<<<blocks, threads>>>(buf, n4, sink, iters); break;
            default: break;
        }
        if (rep == 1) cudaEventRecord(t1);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(sink);
    if (buf) cudaFree(buf);
    return (int)e;
}
