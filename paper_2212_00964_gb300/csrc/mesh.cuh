// mesh.cuh -- the mesh handle and the per-handle scratch workspace.
#pragma once

#include <mutex>

#include "fem_internal.cuh"

namespace femgb {

// Named device buffers that grow on demand and are never shrunk.
// Slots 0..31 belong to the solvers, WS_BICG0.. to the assembled-matrix
// solver, 48..63 to the scalar Poisson path, 64..79 and 88..97 to J2
// plasticity, 80..87 to the topology-optimisation step, WS_APPLY_K0 to the
// standalone tensor-core tangent apply.
enum { WS_BICG0 = 32, WS_APPLY_K0 = 100 };

struct Workspace {
    enum { N_SLOTS = 128 };
    void *ptr[N_SLOTS] = {};
    size_t cap[N_SLOTS] = {};

    // Returns nullptr (with the error text set) when cudaMalloc fails or the
    // slot does not exist.
    void *get(int slot, size_t bytes)
    {
        if (slot < 0 || slot >= N_SLOTS) {
            set_error("workspace: slot out of range");
            return nullptr;
        }
        if (bytes == 0) bytes = 16;
        if (cap[slot] >= bytes) return ptr[slot];
        if (ptr[slot]) cudaFree(ptr[slot]);
        ptr[slot] = nullptr;
        cap[slot] = 0;
        size_t b = (bytes + 255) & ~(size_t)255;
        if (cudaMalloc(&ptr[slot], b) != cudaSuccess) {
            cudaGetLastError();
            set_error("workspace: cudaMalloc failed");
            return nullptr;
        }
        cap[slot] = b;
        return ptr[slot];
    }
    void release()
    {
        for (int i = 0; i < N_SLOTS; ++i) {
            if (ptr[i]) cudaFree(ptr[i]);
            ptr[i] = nullptr;
            cap[i] = 0;
        }
    }
};

}  // namespace femgb

struct fem_mesh_s {
    int nx = 0, ny = 0, nz = 0;
    double lx = 0, ly = 0, lz = 0;
    int64_t n_nodes = 0, n_cells = 0, nnz = 0;
    int32_t *conn = nullptr;
    double *X = nullptr;
    int32_t *colour_ptr = nullptr;
    int32_t colour_ptr_h[9] = {};
    int32_t *cell_perm = nullptr;
    int32_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    bool det = false;  // FEM_MESH_DETERMINISTIC: colour-ordered cell operators
    bool tc = false;   // FEM_MESH_TENSOR_CORES: FP32 LE/SIMP applies on the tensor cores
    femgb::Workspace ws;
    std::mutex mu;  // one solve per handle at a time

    int64_t n_dofs() const { return 3 * n_nodes; }
    void release()
    {
        if (conn) cudaFree(conn);
        if (X) cudaFree(X);
        if (colour_ptr) cudaFree(colour_ptr);
        if (cell_perm) cudaFree(cell_perm);
        if (row_ptr) cudaFree(row_ptr);
        if (col) cudaFree(col);
        conn = nullptr; X = nullptr; colour_ptr = nullptr; cell_perm = nullptr; row_ptr = nullptr; col = nullptr;
        ws.release();
    }
};
