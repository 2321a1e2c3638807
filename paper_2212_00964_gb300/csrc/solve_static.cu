// solve_static.cu -- fem_solve_static: the load-stepped Newton solve of
// fem_solve for one box mesh, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc when they solve.  Examples:
//  - a process whose device memory is owned by another framework's caching
//    allocator;
//  - a real-time loop that forbids allocation after start-up;
//  - code that runs while a stream capture in global mode makes allocation
//    illegal.
// This entry point needs neither a mesh handle nor a workspace.  Its scratch
// (CG vectors, the FP64 residual, the control block) lives in one file-scope
// device array of FEM_STATIC_SCRATCH_BYTES.  Every GPU that loads the library
// holds that array until the process exits.
//
// It also makes no synchronisation call: each of its host round trips is a
// device-to-host copy into pageable host memory, which the CUDA runtime
// returns from only once the copy is complete.  While another thread holds
// a global-mode stream capture open, cudaMalloc, cudaStreamSynchronize,
// cudaStreamQuery and cudaEventSynchronize are refused (and invalidate that
// capture); kernel launches, memsets and pageable copies on another stream
// are not.
#include <cstdio>
#include <mutex>

#include "cell_ops.cuh"
#include "fem_internal.cuh"

namespace femgb {
size_t region_bytes(const InstDesc &d, int precision, bool has_cp);
int solve_in_region(const InstDesc &d, int n_steps, const fem_bc &bc, const double *cp64,
                    const fem_options &o, double *u64, void *region, fem_stats *stats, cudaStream_t s);
int check_solver_options(const fem_options &o);
}  // namespace femgb

using namespace femgb;

// The shared scratch of every fem_solve_static call on a device.
static __device__ __align__(256) unsigned char g_static_scratch[FEM_STATIC_SCRATCH_BYTES];

// In host code g_static_scratch names a host-side stand-in, not device
// memory.  So the device address is looked up once per device, with that
// device current, and kept here.
static std::mutex g_static_mu;
static void *g_static_ptr[64] = {};

static int static_scratch(void **out)
{
    int dev = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return (set_error("fem_solve_static: device ordinal out of range"), FEM_ERR_ARG);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
        if (!p) return (set_error("fem_solve_static: null scratch address"), FEM_ERR_CUDA);
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return FEM_OK;
}

extern "C" int fem_solve_static(int nx, int ny, int nz, double lx, double ly, double lz, const fem_material *mat,
                                const fem_bc *bc, const double *cell_param, int n_steps, const fem_options *opt,
                                double *u_inout, fem_stats *stats, void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0) || !(ly > 0) || !(lz > 0))
        return (set_error("fem_solve_static: sizes must be >= 1 and lengths > 0"), FEM_ERR_ARG);
    if (!bc || !bc->mask || !bc->u_bar || !u_inout || n_steps < 1)
        return (set_error("fem_solve_static: mask, u_bar, u_inout required and n_steps >= 1"), FEM_ERR_ARG);
    if (int rc = check_material(mat)) return rc;
    fem_options o;
    fem_default_options(&o);
    if (opt) o = *opt;
    if (int rc = check_solver_options(o)) return rc;
    InstDesc d{};
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.kind = mat->kind;
    d.E = mat->E; d.nu = mat->nu; d.p = mat->simp_p; d.emin = mat->simp_emin;
    d.hx = lx / nx; d.hy = ly / ny; d.hz = lz / nz;
    d.derive();
    if (d.n_dofs() >= (int64_t)INT32_MAX)
        return (set_error("fem_solve_static: mesh too large"), FEM_ERR_ARG);
    const size_t need = region_bytes(d, o.precision, cell_param != nullptr);
    if (need > (size_t)FEM_STATIC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "fem_solve_static: %dx%dx%d needs %zu bytes of scratch, more than the %zu-byte static array; "
                 "use fem_solve",
                 nx, ny, nz, need, (size_t)FEM_STATIC_SCRATCH_BYTES);
        set_error(buf);
        return FEM_ERR_ARG;
    }
    void *scratch = nullptr;
    if (int rc = static_scratch(&scratch)) return rc;
    return solve_in_region(d, n_steps, *bc, cell_param, o, u_inout, scratch, stats, (cudaStream_t)stream);
}
