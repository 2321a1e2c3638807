// mesh.cu -- structured HEX8 box mesh on the device: connectivity, coordinates,
// cell colouring, CSR pattern and scatter map of the global tangent
// (Algorithm 1's sparse K), external loads of the weak form (Eq. (2)).
//
// The box's numbering makes every integer output a closed form of the node
// or cell coordinates, so each kernel is one thread per output row/cell with
// no search, sort or scan.
#include <algorithm>
#include <cstring>

#include "mesh.cuh"

namespace femgb {

// VTK hexahedron local order -> (p, q, r) offsets
__constant__ int c_vtk_off[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                    {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

__global__ void k_mesh_nodes(int nx, int ny, int nz, double lx, double ly, double lz, double *X)
{
    const int64_t n_nodes = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(n % (nx + 1));
        int j = (int)((n / (nx + 1)) % (ny + 1));
        int k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
        X[3 * n + 0] = __ddiv_rn(__dmul_rn(lx, (double)i), (double)nx);
        X[3 * n + 1] = __ddiv_rn(__dmul_rn(ly, (double)j), (double)ny);
        X[3 * n + 2] = __ddiv_rn(__dmul_rn(lz, (double)k), (double)nz);
    }
}

__global__ void k_mesh_conn(int nx, int ny, int nz, int32_t *conn)
{
    const int64_t ne = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
        for (int a = 0; a < 8; ++a) {
            int64_t n = (i + c_vtk_off[a][0]) +
                        (int64_t)(nx + 1) * ((j + c_vtk_off[a][1]) + (int64_t)(ny + 1) * (k + c_vtk_off[a][2]));
            conn[8 * e + a] = (int32_t)n;
        }
    }
}

// number of indices t in [0, n) with t % 2 == par
__host__ __device__ inline int64_t par_count(int n, int par) { return (n - par + 1) / 2; }

__global__ void k_colour_perm(int nx, int ny, int nz, const int32_t *colour_ptr, int32_t *perm)
{
    const int64_t ne = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
        int a = i & 1, b = j & 1, c = k & 1;
        int col = a + 2 * b + 4 * c;
        int64_t ni = par_count(nx, a), nj = par_count(ny, b);
        int64_t pos = (i >> 1) + ni * ((j >> 1) + nj * (int64_t)(k >> 1));
        perm[colour_ptr[col] + pos] = (int32_t)e;
    }
}

__host__ __device__ inline int64_t win_len_h(int a, int n) { return 1 + (a > 0) + (a < n); }
// sum of window lengths of node coordinates 0..a-1 (a <= n)
__host__ __device__ inline int64_t win_prefix(int a, int n) { return a == 0 ? 0 : 3LL * a - 1; }

__device__ inline int64_t csr_node_start(int nx, int ny, int nz, int I, int J, int K)
{
    const int64_t SX = 3LL * nx + 1, SY = 3LL * ny + 1;
    return 9 * (SX * SY * win_prefix(K, nz) +
                win_len_h(K, nz) * (SX * win_prefix(J, ny) + win_len_h(J, ny) * win_prefix(I, nx)));
}

__global__ void k_csr_rows(int nx, int ny, int nz, int32_t *row_ptr, int32_t *col)
{
    const int64_t n_nodes = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_nodes;
         n += (int64_t)gridDim.x * blockDim.x) {
        int I = (int)(n % (nx + 1)), J = (int)((n / (nx + 1)) % (ny + 1)),
            K = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
        int64_t start = csr_node_start(nx, ny, nz, I, J, K);
        int64_t len = 3 * win_len_h(I, nx) * win_len_h(J, ny) * win_len_h(K, nz);
        for (int c = 0; c < 3; ++c) row_ptr[3 * n + c] = (int32_t)(start + c * len);
        if (n == n_nodes - 1) row_ptr[3 * n_nodes] = (int32_t)(start + 3 * len);
        if (col) {
            for (int c = 0; c < 3; ++c) {
                int64_t o = start + c * len;
                for (int K2 = max(K - 1, 0); K2 <= min(K + 1, nz); ++K2)
                    for (int J2 = max(J - 1, 0); J2 <= min(J + 1, ny); ++J2)
                        for (int I2 = max(I - 1, 0); I2 <= min(I + 1, nx); ++I2) {
                            int64_t m = I2 + (int64_t)(nx + 1) * (J2 + (int64_t)(ny + 1) * K2);
                            for (int j = 0; j < 3; ++j) col[o++] = (int32_t)(3 * m + j);
                        }
            }
        }
    }
}

__global__ void k_csr_map(int nx, int ny, int nz, const int32_t *row_ptr, int32_t *map)
{
    const int64_t ne = (int64_t)nx * ny * nz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ne * 64;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = t / 64;
        int a = (int)((t / 8) % 8), b = (int)(t % 8);
        int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
        int aI = i + c_vtk_off[a][0], aJ = j + c_vtk_off[a][1], aK = k + c_vtk_off[a][2];
        int bI = i + c_vtk_off[b][0], bJ = j + c_vtk_off[b][1], bK = k + c_vtk_off[b][2];
        int64_t na = aI + (int64_t)(nx + 1) * (aJ + (int64_t)(ny + 1) * aK);
        int64_t wx = win_len_h(aI, nx), wy = win_len_h(aJ, ny);
        int64_t pos = ((bK - (aK > 0 ? aK - 1 : 0)) * wy + (bJ - (aJ > 0 ? aJ - 1 : 0))) * wx +
                      (bI - (aI > 0 ? aI - 1 : 0));
        for (int ci = 0; ci < 3; ++ci)
            for (int cj = 0; cj < 3; ++cj)
                map[576 * e + 24 * (3 * a + ci) + 3 * b + cj] = row_ptr[3 * na + ci] + (int32_t)(3 * pos + cj);
    }
}

// Uniform traction on one face: every face cell adds t * area / 4 to each of
// its 4 face nodes (exact integral of the bilinear face shape functions).
__global__ void k_traction(int nx, int ny, int nz, int face, double tx, double ty, double tz, double area,
                           double *f)
{
    const int d = face / 2, side = face % 2;
    const int n[3] = {nx, ny, nz};
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const int64_t nf = (int64_t)n[d1] * n[d2];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        int a = (int)(t % n[d1]), b = (int)(t / n[d1]);
        for (int da = 0; da < 2; ++da)
            for (int db = 0; db < 2; ++db) {
                int idx[3];
                idx[d] = side ? n[d] : 0;
                idx[d1] = a + da;
                idx[d2] = b + db;
                int64_t node = idx[0] + (int64_t)(nx + 1) * (idx[1] + (int64_t)(ny + 1) * idx[2]);
                red_add(&f[3 * node + 0], tx * area * 0.25);
                red_add(&f[3 * node + 1], ty * area * 0.25);
                red_add(&f[3 * node + 2], tz * area * 0.25);
            }
    }
}

// Uniform body force: every cell adds b * volume / 8 to each of its nodes.
__global__ void k_body(int nx, int ny, int nz, double bx, double by, double bz, double vol, double *f)
{
    const int64_t ne = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
        for (int a = 0; a < 8; ++a) {
            int64_t node = (i + c_vtk_off[a][0]) +
                           (int64_t)(nx + 1) * ((j + c_vtk_off[a][1]) + (int64_t)(ny + 1) * (k + c_vtk_off[a][2]));
            red_add(&f[3 * node + 0], bx * vol * 0.125);
            red_add(&f[3 * node + 1], by * vol * 0.125);
            red_add(&f[3 * node + 2], bz * vol * 0.125);
        }
    }
}

static int grid_for(int64_t n, int bs)
{
    int64_t g = (n + bs - 1) / bs;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 64));
}

}  // namespace femgb

using namespace femgb;

extern "C" int fem_mesh(int nx, int ny, int nz, double lx, double ly, double lz, int flags, void *stream,
                        fem_mesh_t *out)
{
    if (!out) return (set_error("fem_mesh: out is NULL"), FEM_ERR_ARG);
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0) || !(ly > 0) || !(lz > 0))
        return (set_error("fem_mesh: sizes must be >= 1 and lengths > 0"), FEM_ERR_ARG);
    const int64_t n_nodes = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    const int64_t n_cells = (int64_t)nx * ny * nz;
    if (3 * n_nodes >= (int64_t)INT32_MAX || n_cells * 8 >= (int64_t)INT32_MAX)
        return (set_error("fem_mesh: mesh too large for int32 indexing"), FEM_ERR_ARG);
    const int64_t nnz = 9LL * (3LL * nx + 1) * (3LL * ny + 1) * (3LL * nz + 1);
    const bool csr = (flags & FEM_MESH_CSR) != 0;
    if (csr && (nnz >= (int64_t)INT32_MAX || n_cells * 576 >= (int64_t)INT64_MAX / 4))
        return (set_error("fem_mesh: CSR pattern exceeds int32 range"), FEM_ERR_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    fem_mesh_s *m = new fem_mesh_s();
    m->nx = nx; m->ny = ny; m->nz = nz;
    m->lx = lx; m->ly = ly; m->lz = lz;
    m->n_nodes = n_nodes; m->n_cells = n_cells; m->nnz = csr ? nnz : 0;
    m->det = (flags & FEM_MESH_DETERMINISTIC) != 0;
    m->tc = (flags & FEM_MESH_TENSOR_CORES) != 0;
    auto fail = [&](cudaError_t e, const char *what) {
        int rc = cuda_fail(e, what, __FILE__, __LINE__);
        fem_mesh_destroy(m);
        return rc;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&m->conn, sizeof(int32_t) * 8 * n_cells)) != cudaSuccess) return fail(e, "malloc conn");
    if ((e = cudaMalloc(&m->X, sizeof(double) * 3 * n_nodes)) != cudaSuccess) return fail(e, "malloc X");
    if ((e = cudaMalloc(&m->colour_ptr, sizeof(int32_t) * 9)) != cudaSuccess) return fail(e, "malloc colour");
    if ((e = cudaMalloc(&m->cell_perm, sizeof(int32_t) * n_cells)) != cudaSuccess) return fail(e, "malloc perm");
    int64_t off = 0;
    for (int c = 0; c < 8; ++c) {
        m->colour_ptr_h[c] = (int32_t)off;
        off += par_count(nx, c & 1) * par_count(ny, (c >> 1) & 1) * par_count(nz, c >> 2);
    }
    m->colour_ptr_h[8] = (int32_t)off;
    if ((e = cudaMemcpyAsync(m->colour_ptr, m->colour_ptr_h, sizeof(int32_t) * 9, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return fail(e, "copy colour_ptr");
    k_mesh_nodes<<<grid_for(n_nodes, 256), 256, 0, s>>>(nx, ny, nz, lx, ly, lz, m->X);
    k_mesh_conn<<<grid_for(n_cells, 256), 256, 0, s>>>(nx, ny, nz, m->conn);
    k_colour_perm<<<grid_for(n_cells, 256), 256, 0, s>>>(nx, ny, nz, m->colour_ptr, m->cell_perm);
    count_launch(3);
    if (csr) {
        if ((e = cudaMalloc(&m->row_ptr, sizeof(int32_t) * (3 * n_nodes + 1))) != cudaSuccess) return fail(e, "malloc row_ptr");
        if ((e = cudaMalloc(&m->col, sizeof(int32_t) * nnz)) != cudaSuccess) return fail(e, "malloc col");
        k_csr_rows<<<grid_for(n_nodes, 128), 128, 0, s>>>(nx, ny, nz, m->row_ptr, m->col);
        count_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "mesh kernels");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "mesh sync");
    *out = m;
    return FEM_OK;
}

extern "C" int fem_mesh_info(fem_mesh_t m, int64_t *n_nodes, int64_t *n_cells, int64_t *nnz)
{
    if (!m) return (set_error("fem_mesh_info: NULL mesh"), FEM_ERR_ARG);
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_cells) *n_cells = m->n_cells;
    if (nnz) *nnz = m->nnz;
    return FEM_OK;
}

extern "C" int fem_mesh_export(fem_mesh_t m, int32_t *conn, double *X, int32_t *colour_ptr, int32_t *cell_perm,
                               int32_t *row_ptr, int32_t *col, int32_t *map, void *stream)
{
    if (!m) return (set_error("fem_mesh_export: NULL mesh"), FEM_ERR_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    if ((row_ptr || col || map) && !m->row_ptr)
        return (set_error("fem_mesh_export: mesh built without FEM_MESH_CSR"), FEM_ERR_ARG);
    if (conn) FEM_CUDA(cudaMemcpyAsync(conn, m->conn, sizeof(int32_t) * 8 * m->n_cells, cudaMemcpyDeviceToDevice, s));
    if (X) FEM_CUDA(cudaMemcpyAsync(X, m->X, sizeof(double) * 3 * m->n_nodes, cudaMemcpyDeviceToDevice, s));
    if (colour_ptr) FEM_CUDA(cudaMemcpyAsync(colour_ptr, m->colour_ptr, sizeof(int32_t) * 9, cudaMemcpyDeviceToDevice, s));
    if (cell_perm) FEM_CUDA(cudaMemcpyAsync(cell_perm, m->cell_perm, sizeof(int32_t) * m->n_cells, cudaMemcpyDeviceToDevice, s));
    if (row_ptr) FEM_CUDA(cudaMemcpyAsync(row_ptr, m->row_ptr, sizeof(int32_t) * (3 * m->n_nodes + 1), cudaMemcpyDeviceToDevice, s));
    if (col) FEM_CUDA(cudaMemcpyAsync(col, m->col, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToDevice, s));
    if (map) {
        k_csr_map<<<grid_for(m->n_cells * 64, 256), 256, 0, s>>>(m->nx, m->ny, m->nz, m->row_ptr, map);
        count_launch();
        FEM_CUDA(cudaGetLastError());
    }
    return FEM_OK;
}

extern "C" int fem_mesh_destroy(fem_mesh_t m)
{
    if (!m) return FEM_OK;
    m->release();
    delete m;
    return FEM_OK;
}

extern "C" int fem_load_traction(fem_mesh_t m, int face, const double *t, double *f_ext, void *stream)
{
    if (!m || !t || !f_ext || face < 0 || face > 5) return (set_error("fem_load_traction: bad argument"), FEM_ERR_ARG);
    const double h[3] = {m->lx / m->nx, m->ly / m->ny, m->lz / m->nz};
    const int d = face / 2, d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const int n[3] = {m->nx, m->ny, m->nz};
    const int64_t nf = (int64_t)n[d1] * n[d2];
    k_traction<<<grid_for(nf, 256), 256, 0, (cudaStream_t)stream>>>(m->nx, m->ny, m->nz, face, t[0], t[1], t[2],
                                                                    h[d1] * h[d2], f_ext);
    count_launch();
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}

extern "C" int fem_load_body(fem_mesh_t m, const double *b, double *f_ext, void *stream)
{
    if (!m || !b || !f_ext) return (set_error("fem_load_body: bad argument"), FEM_ERR_ARG);
    const double vol = (m->lx / m->nx) * (m->ly / m->ny) * (m->lz / m->nz);
    k_body<<<grid_for(m->n_cells, 256), 256, 0, (cudaStream_t)stream>>>(m->nx, m->ny, m->nz, b[0], b[1], b[2], vol, f_ext);
    count_launch();
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
}
