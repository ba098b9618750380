// pdq_capi.cu -- status codes, version and default physical constants of libpdq.
#include <stdio.h>

#include "pdq_common.cuh"

namespace pdq {
static thread_local char g_cuda_msg[256];
static thread_local int g_have_msg = 0;

int cuda_status(cudaError_t e) {
    snprintf(g_cuda_msg, sizeof(g_cuda_msg), "CUDA error %d: %s", (int)e, cudaGetErrorString(e));
    g_have_msg = 1;
    if (e == cudaErrorMemoryAllocation) return PDQ_ERR_OOM;
    return PDQ_ERR_CUDA;
}
}  // namespace pdq

extern "C" const char* pdq_strerror(int status) {
    switch (status) {
        case PDQ_OK: return "ok";
        case PDQ_ERR_INVALID_ARG: return "invalid argument";
        case PDQ_ERR_CUDA: return pdq::g_have_msg ? pdq::g_cuda_msg : "CUDA error";
        case PDQ_ERR_OOM: return "out of device memory";
        case PDQ_ERR_NAN: return "non-finite particle state";
        case PDQ_ERR_TIMEOUT: return "bounded device wait gave up";
        case PDQ_ERR_PRECOND: return "MFMC precondition violated";
        case PDQ_ERR_UNSUPPORTED: return "unsupported request";
        case PDQ_ERR_WORKSPACE: return "workspace too small or misaligned";
        default: return "unknown status";
    }
}

extern "C" int pdq_version(void) { return 100; }

// Constants of Sec. 2.1, 2.2 and 4.3; rho_f = 1.2 kg/m^3 is the reading that
// reproduces the printed tau_p+ (the paper does not print it).
extern "C" void pdq_phys_default(pdq_phys* p) {
    if (!p) return;
    p->nu = 1.5e-5;
    p->radius = 0.01;
    p->re_tau = 180.0;
    p->u_bulk = 4.0;
    p->rho_p = 2650.0;
    p->rho_f = 1.2;
    p->eps0 = 8.854e-12;
    p->q_unit = 500.0 * 1.6e-19;
    p->hamaker0 = 1e-18;
    p->delta_min = 1e-9;
    p->young = 70e9;
    p->delta_c = 0.165e-9;
    p->sigma_y0 = 200e6;
    p->g = 9.81;
    p->restitution = 0.9;
    p->tau_col_steps = 15.0;
    p->neg_charge_frac = 0.0;
    p->contact_scale = 1.0;
}
