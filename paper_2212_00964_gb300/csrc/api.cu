// api.cu -- error reporting, status strings, option defaults, launch counter.
#include <cstdio>
#include <string>

#include "fem_internal.cuh"

namespace femgb {

std::atomic<int64_t> g_launches{0};
thread_local bool t_capturing = false;
static thread_local std::string t_last_error;

void set_error(const std::string &msg) { t_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    t_last_error = buf;
    if (e == cudaErrorMemoryAllocation) return FEM_ERR_NOMEM;
    return FEM_ERR_CUDA;
}

}  // namespace femgb

extern "C" const char *fem_status_string(int status)
{
    switch (status) {
    case FEM_OK: return "ok";
    case FEM_ERR_ARG: return "invalid argument";
    case FEM_ERR_CUDA: return "CUDA error";
    case FEM_ERR_NOT_CONVERGED: return "not converged";
    case FEM_ERR_INVERTED: return "inverted element (det F <= 0)";
    case FEM_ERR_BREAKDOWN: return "CG breakdown (p^T K p <= 0)";
    case FEM_ERR_NONFINITE: return "non-finite residual";
    case FEM_ERR_TIMEOUT: return "timeout";
    case FEM_ERR_NOMEM: return "out of device memory";
    }
    return "unknown status";
}

extern "C" const char *fem_last_error(void) { return femgb::t_last_error.c_str(); }

extern "C" int64_t fem_kernel_launches(void) { return femgb::g_launches.load(); }

extern "C" void fem_default_options(fem_options *o)
{
    if (!o) return;
    o->precision = FEM_MIXED;
    o->newton_rtol = 1e-10;
    o->newton_atol = 0.0;
    o->newton_maxit = 30;
    o->pcg_rtol = 3e-4;
    o->pcg_maxit = 5000;
    o->pcg_chunk = 16;
    o->step_begin = 1;
    o->apply_kernel = 0;
    o->cg_fused = 0;
    o->timeout_s = 0.0;
    o->newton_res32 = 1;
    o->graph_loop = 1;
    o->pcg_rtol_max = 0.1;
    o->cta_cells = 0;
}
