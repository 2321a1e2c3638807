// cell_ops.cuh -- launcher interface shared by the cell operators and the solvers.
#pragma once

#include "cell_kernels.cuh"

struct fem_mesh_s;

namespace femgb {

template <typename T>
cudaError_t launch_cell(int mode, bool nh, const CellArgs<T> &a, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_brick(bool nh, const CellArgs<T> &a, cudaStream_t s);

template <typename T>
cudaError_t launch_apply_cell4(bool nh, const CellArgs<T> &a, cudaStream_t s);

int device_sms();
void warm_occupancy(bool nh);
int resident_grid(const void *func, int block, size_t smem);
int check_material(const fem_material *mat);
InstDesc make_desc(const fem_mesh_s *m, const fem_material *mat);

}  // namespace femgb
