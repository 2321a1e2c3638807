// cell_ops.cuh -- launcher interface shared by the cell operators and the solvers.
#pragma once

#include <utility>

#include "cell_kernels.cuh"

struct fem_mesh_s;

namespace femgb {

template <typename T>
cudaError_t launch_cell(int mode, bool nh, const CellArgs<T> &a, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_brick(bool nh, const CellArgs<T> &a, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_cell4(bool nh, const CellArgs<T> &a, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_kin(bool nh, const CellArgs<T> &a, cudaStream_t s, bool four_ctas = false);

cudaError_t launch_apply_x2(bool nh, int kin, const CellArgs<float> &a, cudaStream_t s, bool stage = false,
                            int nt = CELL_BLOCK);
cudaError_t launch_apply_x2h(const CellArgs<float> &a, cudaStream_t s);
cudaError_t launch_le_k0(const InstDesc &d, float *k0, cudaStream_t s);
cudaError_t launch_apply_le_tc(const CellArgs<float> &a, const float *k0, cudaStream_t s, bool pcg = true);

// What the diagonal kernel stores for CG apply kernel `variant` (CellArgs::kin_mode):
// 0 nothing, 1 cof(F) + scalars, 2 scalars, 3 scalars + displacement gradient.
inline int kin_mode_of(int variant)
{
    switch (variant) {
    case 4: return 1;
    case 5: return 2;
    case 6: case 7: case 9: case 10: case 12: return 3;
    }
    return 0;
}

// Launch with programmatic stream serialisation (the kernel must begin with
// pdl_wait() before it reads anything its predecessor wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int device_sms();
void warm_occupancy(bool nh);
int resident_grid(const void *func, int block, size_t smem);
int check_material(const fem_material *mat);
InstDesc make_desc(const fem_mesh_s *m, const fem_material *mat);

}  // namespace femgb
