// fmm_forces_noalloc: the leaf-force pass (potential, field and the FP64
// conservation sums) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// available -- a host framework that owns all device memory through its own
// pool and forbids side allocations, a foreign-language caller (Fortran, a
// plugin ABI) that can pass pointers but not manage CUDA allocations, or
// work enqueued where an allocation would block or fail.  Such a caller
// still hands in every input and output buffer; the only other memory this
// pass needs, the per-leaf-node partial sums, lives in a fixed array below.
//
// The scratch array is a file-scope __device__ array of kMaxLeafNodes x 8
// doubles (4 MiB).  Every GPU that loads the library holds it until the
// process exits, and every call shares it: each call overwrites the rows it
// uses before reading them (nothing has to start at zero), and two calls
// whose work overlaps on the GPU -- on different streams, or from different
// threads -- race on it.  Serialise the calls.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device asks the runtime for the address (cudaGetSymbolAddress,
// with that device current) and keeps it; make that first call before any
// stream capture.  The arithmetic per cell and per sum matches fmm_forces.
#include <mutex>
#include <string>

#include "fmm_internal.h"

namespace {

constexpr int64_t kMaxLeafNodes = 65536;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 128;          // 4 cells per thread, as fmm_forces

static __device__ __align__(256) double g_noalloc_partials[kMaxLeafNodes * 8];

std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};

int noalloc_fail(int code, const std::string &msg)
{
    fmm::record_error(msg);            // readable through fmm_last_error()
    return code;
}

__device__ __forceinline__ void block_sum8(double v[8], double (*sh)[8])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 8; ++k) {
            double s = 0.0;
            for (int w = 0; w < int(blockDim.x) / 32; ++w) s += sh[w][k];
            v[k] = s;
        }
    }
}

// a leaf-table row the pass can use: node inside the caller's node-indexed
// buffers, level 1..20, coordinates inside that level's grid, tree inside
// the totals
__device__ __forceinline__ bool row_valid(const int32_t *lt, int64_t n_nodes, int32_t n_trees)
{
    const int level = lt[1];
    if (lt[0] < 0 || int64_t(lt[0]) >= n_nodes || level < 1 || level > 20) return false;
    const int side = 1 << (level - 1);
    return lt[2] >= 0 && lt[2] < side && lt[3] >= 0 && lt[3] < side && lt[4] >= 0 &&
           lt[4] < side && lt[5] >= 0 && lt[5] < n_trees;
}

// One CTA per leaf node (leaf table row r = leaf row r): phi, g and the
// node's 8 partial sums into the static scratch rows.  A row that fails
// row_valid reads nothing through its node index: its phi and g rows and its
// partial sums are NaN.
__global__ void __launch_bounds__(kThreads) noalloc_leaf_kernel(
    const int32_t *__restrict__ leaf_table, int64_t n_nodes, int32_t n_trees,
    const double *__restrict__ L64, const double *__restrict__ dacc,
    const double *__restrict__ rho, double *__restrict__ phi, double *__restrict__ g,
    double *__restrict__ partials, double box_size)
{
    __shared__ double sh[kThreads / 32][8];
    const int row = blockIdx.x;
    const int32_t *lt = leaf_table + size_t(row) * 6;
    if (!row_valid(lt, n_nodes, n_trees)) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (int c = threadIdx.x; c < fmm::NCELL; c += kThreads) {
            phi[size_t(row) * fmm::NCELL + c] = nan;
#pragma unroll
            for (int a = 0; a < 3; ++a) g[(size_t(row) * 3 + a) * fmm::NCELL + c] = nan;
        }
        if (threadIdx.x < 8) partials[size_t(row) * 8 + threadIdx.x] = nan;
        return;
    }
    const int node = lt[0], level = lt[1], ix = lt[2], iy = lt[3], iz = lt[4];
    const double h = box_size / (8.0 * double(1u << (level - 1)));
    const double h3 = h * h * h;
    const double half = 0.5 * box_size;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float nf = 0.f, nt = 0.f;
#pragma unroll
    for (int r = 0; r < fmm::NCELL / kThreads; ++r) {
        const int c = threadIdx.x + r * kThreads;
        const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
        const double m = rho[size_t(row) * fmm::NCELL + c] * h3;
        phi[size_t(row) * fmm::NCELL + c] = L64[(size_t(node) * fmm::NCOMP) * fmm::NCELL + c];
        double gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gv[a] = -(L64[(size_t(node) * fmm::NCOMP + 1 + a) * fmm::NCELL + c] +
                      dacc[(size_t(node) * 3 + a) * fmm::NCELL + c]);
            g[(size_t(row) * 3 + a) * fmm::NCELL + c] = gv[a];
        }
        const double X[3] = {(8.0 * ix + x + 0.5) * h - half, (8.0 * iy + y + 0.5) * h - half,
                             (8.0 * iz + z + 0.5) * h - half};
        const double u[3] = {X[1] * gv[2] - X[2] * gv[1], X[2] * gv[0] - X[0] * gv[2],
                             X[0] * gv[1] - X[1] * gv[0]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] += m * gv[a];
            v[3 + a] += m * u[a];
        }
        const float mf = float(m);
        const float gf[3] = {float(gv[0]), float(gv[1]), float(gv[2])};
        const float uf[3] = {float(u[0]), float(u[1]), float(u[2])};
        nf += mf * sqrtf(gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2]);
        nt += mf * sqrtf(uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
    }
    v[6] = double(nf);
    v[7] = double(nt);
    block_sum8(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) partials[size_t(row) * 8 + k] = v[k];
}

// One CTA per tree: the tree's rows of the scratch array in ascending row
// order (fixed order, deterministic).  If any row of the table is invalid,
// every tree's totals are NaN (a row with a bad tree id belongs to no tree,
// so no single tree could carry the error).
__global__ void __launch_bounds__(512) noalloc_reduce_kernel(const int32_t *__restrict__ leaf_table,
                                                             int64_t n_leaf, int64_t n_nodes,
                                                             int32_t n_trees,
                                                             const double *__restrict__ partials,
                                                             double *__restrict__ totals)
{
    __shared__ double sh[16][8];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const int tree = blockIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int bad = 0;
    for (int64_t i = threadIdx.x; i < n_leaf; i += blockDim.x) {
        if (!row_valid(leaf_table + i * 6, n_nodes, n_trees)) {
            bad = 1;
            continue;
        }
        if (leaf_table[i * 6 + 5] == tree)
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] += partials[size_t(i) * 8 + k];
    }
    if (bad) atomicOr(&s_bad, 1);
    block_sum8(v, sh);          // its barrier publishes s_bad
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (int k = 0; k < 8; ++k) totals[size_t(tree) * 8 + k] = s_bad ? nan : v[k];
    }
}

// device address of the scratch array for the current device (set-up on
// first use per device)
int scratch_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FMM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FMM_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return noalloc_fail(FMM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = static_cast<double *>(p);
    }
    *out = g_scratch[dev];
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_forces_noalloc(const int32_t *leaf_table, int64_t n_leaf, int64_t n_nodes,
                       int32_t n_trees, double box_size, const double *L64,
                       const double *dL1_acc, const double *rho, double *phi, double *g,
                       double *totals, fmm_stream_t stream)
{
    if (!leaf_table || !L64 || !dL1_acc || !rho || !phi || !g || !totals)
        return noalloc_fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    if (n_leaf < 1 || n_leaf > kMaxLeafNodes)
        return noalloc_fail(FMM_ERR_INVALID_ARG,
                            "n_leaf must lie in 1.." + std::to_string(kMaxLeafNodes) +
                                " (the size of the fixed scratch array)");
    if (n_nodes < n_leaf) return noalloc_fail(FMM_ERR_INVALID_ARG, "n_nodes must be >= n_leaf");
    if (n_trees < 1 || n_trees > 65535)
        return noalloc_fail(FMM_ERR_INVALID_ARG, "n_trees must lie in 1..65535");
    if (!(box_size > 0.0)) return noalloc_fail(FMM_ERR_INVALID_ARG, "box_size must be positive");
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_leaf_kernel<<<unsigned(n_leaf), kThreads, 0, s>>>(leaf_table, n_nodes, n_trees, L64,
                                                              dL1_acc, rho, phi, g, scratch,
                                                              box_size);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(FMM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    noalloc_reduce_kernel<<<unsigned(n_trees), 512, 0, s>>>(leaf_table, n_leaf, n_nodes, n_trees,
                                                            scratch, totals);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(FMM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return FMM_OK;
}

}  // extern "C"
