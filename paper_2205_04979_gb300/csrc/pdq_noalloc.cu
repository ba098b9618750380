// pdq_noalloc.cu -- pdq_step_particles_noalloc: the particle step for callers
// that cannot allocate device memory.
//
// pdq_step_particles takes a caller-allocated workspace for its work queue.
// Some callers cannot provide one: a host program whose device memory is owned
// entirely by another allocator (for example a framework's caching pool) or
// held under a hard memory cap, or a latency-critical loop that must not call
// cudaMalloc, which can synchronise the device.  This entry point serves them
// from a fixed scratch array compiled into the library instead, and calls no
// allocating routine.
#include <mutex>

#include "pdq_common.cuh"

namespace {

// Built-in scratch: holds the step's whole workspace (work-item table, sample
// order, the z-binning sort's tag scratch, and, as the configuration needs them,
// the Newton-pair sums or the FP64 j-chunk partial sums).  Every GPU that loads
// libpdq keeps this array until the process exits.
constexpr size_t kScratchBytes = PDQ_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};   // device address of g_step_scratch, per device

// Resolve the scratch array's device address on the current device (once).
// In host code g_step_scratch names a host-side stand-in, so kernels must be
// given this address instead.
int scratch_address(void** out) {
    int dev = 0;
    PDQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PDQ_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        PDQ_CUDA(cudaGetSymbolAddress(&p, g_step_scratch));
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return PDQ_OK;
}

}  // namespace

extern "C" int pdq_step_particles_noalloc(const pdq_field* field, const pdq_phys* phys, pdq_state* state,
                                          const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                                          pdq_tally* tally, pdq_stream_t stream) {
    if (!cfg || !state) return PDQ_ERR_INVALID_ARG;
    if (cfg->use_graph) return PDQ_ERR_INVALID_ARG;   // graph instantiation may allocate
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    // The step compares the scratch size with the exact workspace of the tile shape it
    // runs and returns PDQ_ERR_WORKSPACE before any device work when it does not fit.
    // Every part of the workspace is rebuilt (work queue from count[]) or zeroed (sums)
    // inside the call, so the previous call's contents need no clearing.
    return pdq_step_particles(field, phys, state, params, cfg, n_steps, tally, scratch, kScratchBytes, stream);
}
