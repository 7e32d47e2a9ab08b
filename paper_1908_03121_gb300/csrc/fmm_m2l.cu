// Same-level pass (Sec. 4.3, second step; Sec. 5.1 moves it to the GPU).
//
// Every cell A gathers, from each same-level source B that the opening rule
// selects, the order-3 Taylor coefficients of B's potential at A's centre of
// mass, in level units (lengths in cell widths, G factored out):
//   L^(n)_A -= sum_{m: n+m<=3} ((-1)^m / m!) M_B^(m) . D^(n+m)(R),
//   R = X_A - X_B,
// and the angular-momentum correction
//   dL1_A,i += (1/6) sum_jkl D4_ijkl(R) [M3_B - (M0_B / M0_A) M3_A]_jkl.
// Sec. 4.3 lists four kinds by node refinement; this file has one kernel per
// kind of target, as the paper's GPU port fuses multipole<-multipole with
// multipole<-monopole:
//   mp_kernel    refined targets: multipole<-multipole (well-separated
//                sources) and multipole<-monopole (all candidate leaf
//                sources) -- the "455 flop" kernel of Sec. 4.3;
//   mono_kernel  leaf targets, leaf sources: monopole<-monopole, a 1-in,
//                4-out convolution whose per-offset weights are tabulated;
//   mx_kernel    leaf targets next to refined nodes: monopole<-multipole;
//   root_kernel  the single node of level 1 of each tree (all pairs are
//                candidates there).
// Design (GB300-first, unlike the paper's 8x64-thread launches per node fed
// from 128 streams): persistent CTAs pull whole sub-grids from cost-sorted
// work queues; a warp holds 32 targets of one child parity so the stencil
// loop is warp-uniform; leaf-source masses of the 26-neighbour halo are staged
// once per sub-grid into a parity-split, bank-padded shared-memory window;
// refined-source moments stream through L1 as four vector loads from a
// parity-split packed layout, so a warp's loads are contiguous.  Orders 2-4
// of the derivative tensors are traceless, so the contraction works in
// traceless bases (fmm_tensor.cuh): 16 accumulated components instead of 20,
// 16 packed source values instead of 20, and about a quarter fewer products.
// Mixed precision: offsets are formed from double-precision centres of mass
// (packed as offsets from the cell centre, in cell widths), the contraction
// runs in float with per-chunk sums folded into (hi, lo) pairs by TwoSum, and
// the correction's compensated sum is stored and carried down in double.
// Conserving precision: the same kernels instantiated on dfloat (pairs of
// floats, fmm_dfloat.cuh) evaluate offsets, derivative tensors, contraction
// and sums in double-float, so each pair's contributions to A and to B cancel
// in momentum and angular momentum to about 1e-13, as in FP64.
#include <cstdio>
#include <type_traits>

#include "fmm_convert.cuh"
#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

// element types of the three precisions: float (mixed), dfloat (conserving),
// double (FP64)
template <typename T> constexpr bool kF32 = std::is_same<T, float>::value;
template <typename T> constexpr bool kDF = std::is_same<T, dfloat>::value;

template <typename T>
__device__ __forceinline__ T ldg_t(const T *p)
{
    if constexpr (kDF<T>) {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(p));
        return dfloat(f.x, f.y);
    } else {
        return __ldg(p);
    }
}

constexpr int kThreads = 256;   // 8 warps = the 8 child parities
constexpr int kChunk = 16;      // stencil entries per compensated chunk
constexpr int Q_MP = 0, Q_MONO = 1, Q_MX = 2;   // work-queue heads (Q_MX: the fused launch)

struct KParams {
    const NodeInfo *info;
    const int32_t *nbr;
    const int32_t *list;
    int32_t n_items;
    int32_t *counter;
    const StencilEntry *stencil;
    const float4 *stencil_f;  // the same, offsets as floats, window offset's bits in w
    const void *coef;        // monopole weights of parity 0
    const int32_t *mono_woff;  // [8][ent_stride] window offsets in parity 0's order, reflected
    int n_far, n_near;       // identical for every parity
    int ent_stride;          // entries reserved per parity
    const int4 *mx_targets;  // monopole<-multipole targets (node, cell, warp's pair base, count)
    int32_t n_mx;            // monopole<-multipole targets the multipole launch takes (0: none)
    int32_t *mx_counter;     // their queue head
    const int2 *mx_pairs;    // (packed-moment offset, stencil entry); pair k of target
                             // 32 w + j at its warp's base + 32 k + j
    int reach, py, pz, sub_stride;
    const void *mass;
    const void *mp;
    int mp_limit;            // elements of mp: decoded window offsets below it only; the
                             // row starting there holds zeros
    void *L;
    float *Lc;
    double *dL1;
    int far_o2;              // cells at squared offset >= far_o2 are well separated
};

// ------------------------------------------------------------------ pack
// a double as the element type (double-float: split with the conversions on
// the integer pipe)
template <typename T>
__device__ __forceinline__ T elem_from_double(double v)
{
    if constexpr (kDF<T>) return df_from_double(v);
    else return T(v);
}

// Mixed precision: everything but the centre-of-mass offset in float, with
// the double -> float conversions on the integer pipe (GB300's FP64 unit,
// which also runs conversions, would otherwise bound this pass); the
// moments' float rounding is the contraction's own precision.
// (the FP64 moments are read once, with the evict-first hint, so that they
// do not push the packed values just written out of L2, where the
// multipole kernel reads them next)
__device__ __forceinline__ void pack_float(const NodeInfo &ni, const double *__restrict__ levels,
                                           const double *__restrict__ Mn,
                                           const double *__restrict__ comc, int x, int y, int z,
                                           int pi, float *__restrict__ mass_node,
                                           float *__restrict__ mp, double lo_x, double lo_y,
                                           double lo_z)
{
    mass_node[pi] = d2f_rn(__ldcs(Mn));
    if (ni.mp_row < 0) return;
    const double h = levels[ni.level * LEVEL_FIELDS + LV_H];
    const float ih = d2f_rn(levels[ni.level * LEVEL_FIELDS + LV_IH]);
    const double ctr[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * h, lo_y + (8.0 * ni.iy + y + 0.5) * h,
                           lo_z + (8.0 * ni.iz + z + 0.5) * h};
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = d2f_rn(__ldcs(comc + a * NCELL) - ctr[a]) * ih;
    const float w2 = 0.5f * ih * ih, w3 = (1.0f / 6.0f) * ih * ih * ih;
    float A2[6], A3[10];
#pragma unroll
    for (int q = 0; q < 6; ++q) A2[q] = d2f_rn(__ldcs(Mn + (4 + q) * NCELL)) * (float(mult2(q)) * w2);
#pragma unroll
    for (int q = 0; q < 10; ++q) A3[q] = d2f_rn(__ldcs(Mn + (10 + q) * NCELL)) * (float(mult3(q)) * w3);
    const float v[16] = {d[0],          d[1],          d[2],          mass_node[pi],
                         A2[0] - A2[5], A2[3] - A2[5], A2[1],         A2[2],
                         A2[4],         A3[0] - A3[5], A3[1] - A3[8], A3[2] - A3[9],
                         A3[3] - A3[5], A3[4],         A3[6] - A3[8], A3[7] - A3[9]};
    float4 *out = reinterpret_cast<float4 *>(mp + (size_t(ni.mp_row) * 4 * NCELL + pi) * 4);
#pragma unroll
    for (int g = 0; g < 4; ++g)
        out[size_t(g) * NCELL] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
}

// mass[node][pi] = M0 for every node.  Refined nodes also get, in level
// units, four groups of four values at mp[row][g][pi][0..3]:
//   g0 = (delta, M0), delta = (X - centre) / h (first, so that its x and y
//        land in an aligned register pair for the paired FP32 subtraction),
//   g1 = B2[0..3], g2 = (B2[4], B3[0..2]), g3 = B3[3..6],
// the traceless projections of A2 = mult M2 / (2 h^2), A3 = mult M3 / (6 h^3).
template <typename T>
__global__ void __launch_bounds__(512) pack_kernel(const NodeInfo *__restrict__ info,
                                                   const int32_t *__restrict__ nodes,
                                                   const double *__restrict__ levels,
                                                   const double *__restrict__ M,
                                                   const double *__restrict__ com,
                                                   T *__restrict__ mass, T *__restrict__ mp,
                                                   double lo_x, double lo_y, double lo_z)
{
    const int node = nodes ? nodes[blockIdx.x] : int(blockIdx.x);   // a list, or every node
    const NodeInfo ni = info[node];
    const int c = threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int pi = parity_index(x, y, z);
    const double *Mn = M + size_t(node) * NCOMP * NCELL + c;
    if constexpr (kF32<T>) {
        pack_float(ni, levels, Mn, com + size_t(node) * 3 * NCELL + c, x, y, z, pi, mass + size_t(node) * NCELL,
                   mp, lo_x, lo_y, lo_z);
        return;
    }
    mass[size_t(node) * NCELL + pi] = elem_from_double<T>(Mn[0]);
    if (ni.mp_row < 0) return;
    const double h = levels[ni.level * LEVEL_FIELDS + LV_H];
    const double ih = levels[ni.level * LEVEL_FIELDS + LV_IH];
    const double ctr[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * h, lo_y + (8.0 * ni.iy + y + 0.5) * h,
                           lo_z + (8.0 * ni.iz + z + 0.5) * h};
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = (com[(size_t(node) * 3 + a) * NCELL + c] - ctr[a]) * ih;
    const double w2 = 0.5 * ih * ih, w3 = (1.0 / 6.0) * ih * ih * ih;
    double A2[6], A3[10];
#pragma unroll
    for (int q = 0; q < 6; ++q) A2[q] = mult2(q) * w2 * Mn[(4 + q) * NCELL];
#pragma unroll
    for (int q = 0; q < 10; ++q) A3[q] = mult3(q) * w3 * Mn[(10 + q) * NCELL];
    // symmetric order: A2 xx xy xz yy yz zz; A3 xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    const double v[16] = {d[0],          d[1],          d[2],          Mn[0],
                          A2[0] - A2[5], A2[3] - A2[5], A2[1],         A2[2],
                          A2[4],         A3[0] - A3[5], A3[1] - A3[8], A3[2] - A3[9],
                          A3[3] - A3[5], A3[4],         A3[6] - A3[8], A3[7] - A3[9]};
    T *out = mp + (size_t(ni.mp_row) * 4 * NCELL + pi) * 4;
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[size_t(g) * NCELL * 4 + j] = elem_from_double<T>(v[4 * g + j]);
}

// ------------------------------------------------------------ common bits
__device__ __forceinline__ int pull_item(int32_t *counter, int *s_item)
{
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    return *s_item;
}

// Stage the halo window of leaf-cell masses around a target node: window
// cell u in [0, 8 + 2R)^3 holds the source at node-local position u - R, or 0
// when that source is refined or absent.  Layout: parity sub-window
// q = (ux&1) + 2(uy&1) + 4(uz&1), then (ux>>1) + py (uy>>1) + pz (uz>>1).
// One (ux, uy) column per thread pass, z innermost; the parity index and the
// window address both split into an (x, y) part and a z part.  The copies go
// through cp.async (global -> shared without registers; sources that are
// refined or absent are zero-filled by a zero source size), so every load of
// the window is in flight at once.  The caller commits and waits.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element size");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src),
                 "n"(int(sizeof(T))), "r"(valid ? int(sizeof(T)) : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// With s_row given (the multipole-target kernel), a refined source's cell
// holds instead the offset of its packed moments (row and parity index),
// encoded by window_index as a value with the sign bit set (masses are not
// negative); without, it holds 0.  The kernels use a decoded offset only
// below mp_limit, so an invalid negative density can give wrong results but
// no access outside the packed moments.
template <typename T>
__device__ __forceinline__ T window_index(int idx)
{
    if constexpr (kF32<T>) {
        return __int_as_float(-1 - idx);
    } else if constexpr (kDF<T>) {
        return dfloat(__int_as_float(-1 - idx), 0.f);
    } else {
        return __longlong_as_double(-1ll - idx);
    }
}

// the moment offset encoded in a window cell, or -1 for a mass
template <typename T>
__device__ __forceinline__ int window_decode(T v)
{
    if constexpr (kF32<T>) {
        const int b = __float_as_int(v);
        return b < 0 ? -1 - b : -1;
    } else if constexpr (kDF<T>) {
        const int b = __float_as_int(v.hi);
        return b < 0 ? -1 - b : -1;
    } else {
        const long long b = __double_as_longlong(v);
        return b < 0 ? int(-1ll - b) : -1;
    }
}

// whether a window value is a refined source's moment offset below limit,
// and that offset: -1 - bits is the offset for a refined source and
// negative (a large unsigned value) for a mass, whose bits are not
// negative, so one unsigned comparison tells both apart and bounds the
// offset
template <typename T>
__device__ __forceinline__ bool window_moments(T v, int limit, int &idx)
{
    if constexpr (kF32<T>) {
        const unsigned u = unsigned(-1 - __float_as_int(v));
        idx = int(u);
        return u < unsigned(limit);
    } else if constexpr (kDF<T>) {
        const unsigned u = unsigned(-1 - __float_as_int(v.hi));
        idx = int(u);
        return u < unsigned(limit);
    } else {
        const unsigned long long u = static_cast<unsigned long long>(-1ll - __double_as_longlong(v));
        idx = int(u);
        return u < static_cast<unsigned long long>(limit);
    }
}

// whether a window value encodes a refined source (sign bit set)
template <typename T>
__device__ __forceinline__ bool window_refined(T v)
{
    if constexpr (kF32<T>) {
        return __float_as_int(v) < 0;
    } else if constexpr (kDF<T>) {
        return __float_as_int(v.hi) < 0;
    } else {
        return __double_as_longlong(v) < 0;
    }
}

// Window geometry of reach R: the host's pitches (same pad_to), as
// compile-time constants; RR = 0 takes them from the kernel parameters.
template <int RR>
struct WinGeo {
    static constexpr int R = RR, SUB = 4 + RR, E = 8 + 2 * RR;
    static constexpr int PY = pad_to(SUB, 12), PZ = pad_to(SUB * PY, 16), SUB_STRIDE = SUB * PZ;
};

template <typename T, int RR = 0>
__device__ __forceinline__ void stage_window_async(T *W, const int *s_nbr, const int *s_leaf,
                                                   const T *__restrict__ mass, const KParams &P,
                                                   const int *s_row = nullptr)
{
    using G = WinGeo<RR>;
    const int R = RR ? G::R : P.reach;
    const int E = RR ? G::E : 8 + 2 * R;
    const int py = RR ? G::PY : P.py, pz = RR ? G::PZ : P.pz;
    const int sub_stride = RR ? G::SUB_STRIDE : P.sub_stride;
    for (int t = threadIdx.x; t < E * E; t += blockDim.x) {
        const int ux = t % E, uy = t / E;
        const int bx = ux - R + 8, by = uy - R + 8;           // >= 1
        const int sxy = (bx >> 3) + 3 * (by >> 3);
        const int lx = bx & 7, ly = by & 7;
        const int pxy = ((lx & 1) + 2 * (ly & 1)) * 64 + (lx >> 1) + 4 * (ly >> 1);
        const int wxy = ((ux & 1) + 2 * (uy & 1)) * sub_stride + (ux >> 1) + py * (uy >> 1);
#pragma unroll 4
        for (int uz = 0; uz < E; ++uz) {
            const int bz = uz - R + 8;
            const int slot = sxy + 9 * (bz >> 3);
            const int lz = bz & 7;
            const bool ok = s_leaf[slot] != 0;
            const int pi = pxy + 256 * (lz & 1) + 16 * (lz >> 1);
            const T *src = ok ? mass + size_t(s_nbr[slot]) * NCELL + pi : mass;
            const int wi = wxy + 4 * (uz & 1) * sub_stride + pz * (uz >> 1);
            const int row = s_row ? s_row[slot] : -1;
            if (row >= 0)
                W[wi] = window_index<T>((row * 4 * NCELL + pi) * 4);
            else
                cp_async_elem<T>(W + wi, src, ok);
        }
    }
}

// neighbour tables of the current target node into shared memory; returns,
// in threads 0-26, whether that thread's neighbour is a leaf (0 elsewhere)
__device__ __forceinline__ int load_slots(int node, const KParams &P, int *s_nbr, int *s_leaf,
                                          int *s_row)
{
    int is_leaf = 0;
    if (threadIdx.x < 27) {
        const int nb = P.nbr[node * 27 + threadIdx.x];
        s_nbr[threadIdx.x] = nb;
        int leaf = 0, row = -1;
        if (nb >= 0) {
            const NodeInfo ni = P.info[nb];
            leaf = ni.leaf_row >= 0;
            row = ni.mp_row;
        }
        s_leaf[threadIdx.x] = leaf;
        s_row[threadIdx.x] = row;
        is_leaf = leaf;
    }
    return is_leaf;
}

// a window value that is a nonzero mass or a moment offset (an absent
// source's cell holds 0 and contributes nothing)
template <typename T>
__device__ __forceinline__ bool window_nonzero(T v)
{
    if constexpr (kDF<T>) {
        return v.hi != 0.f;
    } else {
        return v != T(0);
    }
}

// Compensated accumulator: float partial sums per chunk, folded into a
// (hi, lo) pair by TwoSum; in double precision a plain sum.
template <typename T, int N>
struct Acc {
    T part[N];
    T hi[N];
    T lo[N];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) part[k] = hi[k] = lo[k] = T(0);
    }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if constexpr (kF32<T>) {
                float s, e;
                two_sum(hi[k], part[k], s, e);
                hi[k] = s;
                lo[k] += e;
            } else {
                hi[k] += part[k];
            }
            part[k] = T(0);
        }
    }
};

// double-float: every term already lands in a double-float running sum,
// so there is nothing to fold
template <int N>
struct Acc<dfloat, N> {
    dfloat part[N];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) part[k] = dfloat(0.f);
    }
    // the running sums take unnormalised terms (fmadd_u, add_u): restore
    // the canonical (hi, lo) form every chunk
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) part[k] = renorm(part[k]);
    }
};

// the (hi, lo) value of accumulator k
template <typename T, int N>
__device__ __forceinline__ T acc_hi(const Acc<T, N> &a, int k) { return a.hi[k]; }
template <int N>
__device__ __forceinline__ dfloat acc_hi(const Acc<dfloat, N> &a, int k) { return a.part[k]; }
template <typename T, int N>
__device__ __forceinline__ T acc_lo(const Acc<T, N> &a, int k) { return a.lo[k]; }
template <int N>
__device__ __forceinline__ dfloat acc_lo(const Acc<dfloat, N> &, int) { return dfloat(0.f); }

// Float accumulator whose (hi, lo) pairs live in shared memory, in this
// thread's column of a [components][2][threads] array: only the chunk sums
// take registers.  The first NC components are compensated; the others
// (the multipole target's orders 2-3, which reach the forces only through
// the downward shifts, scaled by the small child offsets) are plain float
// sums in registers.  Fewer pairs leave more of the SM's shared memory to
// L1, where the multipole kernel rereads the sources' packed moments.
template <int N, int NC = N>
struct SmemAcc {
    float part[N];
    float *col;                       // the (hi, lo) pairs of component k < NC at col[k * 2 * kThreads]
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) part[k] = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            col[k * 2 * kThreads] = 0.f;
            col[(k * 2 + 1) * kThreads] = 0.f;
        }
    }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            float s, e;
            two_sum(col[k * 2 * kThreads], part[k], s, e);
            col[k * 2 * kThreads] = s;
            col[(k * 2 + 1) * kThreads] += e;
            part[k] = 0.f;
        }
    }
};
template <int N, int NC>
__device__ __forceinline__ float acc_hi(const SmemAcc<N, NC> &a, int k)
{
    return k < NC ? a.col[k * 2 * kThreads] : a.part[k];
}
template <int N, int NC>
__device__ __forceinline__ float acc_lo(const SmemAcc<N, NC> &a, int k)
{
    return k < NC ? a.col[(k * 2 + 1) * kThreads] : 0.f;
}

// the multipole kernel's accumulators: for float, shared-memory pairs for
// orders 0-1 and the correction
template <typename T, int N>
struct MpAcc {
    using type = Acc<T, N>;
};
template <int N>
struct MpAcc<float, N> {
    using type = SmemAcc<N, N == 16 ? 4 : N>;
};
constexpr int kMpPairs = 4 + 3;      // compensated float components of mp_kernel

// store component k of a target cell: level units; (hi, lo) float pairs for
// float (renormalised) and double-float (lo is zero there), else double
// Same-level results are stored with the evict-first (streaming) hint: they
// are read once, much later, by the downward pass, and left in L2 they would
// push out the packed source moments that the multipole kernel rereads.
template <typename T>
__device__ __forceinline__ void store_L(const KParams &P, int node, int k, int cell, T hi, T lo)
{
    const size_t idx = (size_t(node) * NCOMP + k) * NCELL + cell;
    if constexpr (kF32<T>) {
        // renormalise so that |lo| <= ulp(hi)/2
        float s = hi + lo;
        float e = lo - (s - hi);
        __stcs(static_cast<float *>(P.L) + idx, s);
        __stcs(P.Lc + idx, e);
    } else if constexpr (kDF<T>) {
        __stcs(static_cast<float *>(P.L) + idx, hi.hi);
        __stcs(P.Lc + idx, hi.lo);
    } else {
        __stcs(static_cast<double *>(P.L) + idx, hi);
    }
}

// store -(a + b) for a traceless-dependent component
template <typename T>
__device__ __forceinline__ void store_neg_sum(const KParams &P, int node, int k, int cell,
                                              const T hi[16], const T lo[16], int a, int b)
{
    if constexpr (kF32<T>) {
        float s, e;
        two_sum(hi[a], hi[b], s, e);
        store_L<T>(P, node, k, cell, -s, -(lo[a] + lo[b] + e));
    } else {
        store_L<T>(P, node, k, cell, -(hi[a] + hi[b]), T(0));
    }
}

// the 16 traceless values of a multipole target -> 20 stored components
// values: 0 L0 | 1-3 L1 | 4-8 L2 (xx yy xy xz yz) | 9-15 L3 (xxx xxy
// xxz xyy xyz yyy yyz)
template <typename T>
__device__ __forceinline__ void store_target_values(const KParams &P, int node, int cell,
                                                    const T hi[16], const T lo[16])
{
    constexpr int direct[16] = {0, 1, 2, 3, 4, 7, 5, 6, 8, 10, 11, 12, 13, 14, 16, 17};
#pragma unroll
    for (int k = 0; k < 16; ++k) store_L<T>(P, node, direct[k], cell, hi[k], lo[k]);
    store_neg_sum<T>(P, node, 9, cell, hi, lo, 4, 5);      // zz  = -(xx + yy)
    store_neg_sum<T>(P, node, 15, cell, hi, lo, 9, 12);    // xzz = -(xxx + xyy)
    store_neg_sum<T>(P, node, 18, cell, hi, lo, 10, 14);   // yzz = -(xxy + yyy)
    store_neg_sum<T>(P, node, 19, cell, hi, lo, 11, 15);   // zzz = -(xxz + yyz)
}

template <typename T, class LA>
__device__ __forceinline__ void store_target(const KParams &P, int node, int cell, const LA &L)
{
    T hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        hi[k] = acc_hi(L, k);
        lo[k] = acc_lo(L, k);
    }
    store_target_values<T>(P, node, cell, hi, lo);
}

// packed data of one source cell (level units)
template <typename T>
struct Src {
    T m0, d[3], B2[5], B3[7];
};

template <typename T>
__device__ __forceinline__ void load4(const T *p, T v[4])
{
    if constexpr (kF32<T>) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else if constexpr (kDF<T>) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w);
        v[2] = dfloat(b.x, b.y); v[3] = dfloat(b.z, b.w);
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void load_source_at(const T *base, Src<T> &s)
{
    T v[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) load4<T>(base + size_t(g) * NCELL * 4, v + 4 * g);
    s.d[0] = v[0]; s.d[1] = v[1]; s.d[2] = v[2];
    s.m0 = v[3];
#pragma unroll
    for (int k = 0; k < 5; ++k) s.B2[k] = v[4 + k];
#pragma unroll
    for (int q = 0; q < 7; ++q) s.B3[q] = v[9 + q];
}

template <typename T>
__device__ __forceinline__ void load_source(const KParams &P, int row, int pi, Src<T> &s)
{
    load_source_at<T>(static_cast<const T *>(P.mp) + (size_t(row) * 4 * NCELL + pi) * 4, s);
}

template <typename T>
__device__ __forceinline__ void zero_moments(Src<T> &s)
{
    s.d[0] = s.d[1] = s.d[2] = T(0);
#pragma unroll
    for (int k = 0; k < 5; ++k) s.B2[k] = T(0);
#pragma unroll
    for (int q = 0; q < 7; ++q) s.B3[q] = T(0);
}

// One source (multipole if SRC_MP, else a point mass m0 = s.m0) into a
// multipole target's 16 traceless accumulators and the correction sum
//   S_i += sum_q (B3_B - M0_B a3_A)_q D4[i, q],  a3_A = B3_A / M0_A,
// with the sign of L folded in:
//   L0 -= M0 D0 + B2.D2 - B3.D3,  L1_i -= M0 D1_i + B2.D3[i,.],
//   L2 -= M0 D2,  L3 -= M0 D3.
// Orders 0 and 1 (potential and field) sum each source's terms first and
// add that sum to the chunk sum once, so every source costs one rounding at
// the chunk sum's magnitude; orders 2-3 and the correction take each product
// straight into their sums as one fused multiply-add.
//
// Expansion order 2 (ORDER = 2; truncation n + m <= 2): L0 -= M0 D0 + B2.D2,
// L1 -= M0 D1, L2 -= M0 D2, no L3, and the correction is the dropped
// n = 1, m = 2 term with the target's share added (D3 is odd):
//   S_i -= sum_k (B2_B + M0_B a2_A)_k D3[i, k],  a2_A = B2_A / M0_A
// (aA holds a2_A in its first five entries then).
template <typename T, bool SRC_MP, int ORDER = 3, class LA, class SA>
__device__ __forceinline__ void acc_mp(T Rx, T Ry, T Rz, const Src<T> &s, const T aA[7], LA &L,
                                       SA &S)
{
    DTraceless<T> D;
    D.template eval<ORDER == 3>(Rx, Ry, Rz);
    const T nm0 = -s.m0;
    // float: each term straight into the chunk sum (one fused multiply-add
    // per term); double-float and double: each source's terms summed first
    T a = kF32<T> ? fmadd(nm0, D.D0, L.part[0]) : nm0 * D.D0;
    if (SRC_MP) {
#pragma unroll
        for (int k = 0; k < 5; ++k) a = fmadd_u(-s.B2[k], D.D2[k], a);
        if (ORDER == 3) {
#pragma unroll
            for (int q = 0; q < 7; ++q) a = fmadd_u(s.B3[q], D.D3[q], a);
        }
    }
    L.part[0] = kF32<T> ? a : add_u(L.part[0], renorm(a));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T b = kF32<T> ? fmadd(nm0, D.D1[i], L.part[1 + i]) : nm0 * D.D1[i];
        if (SRC_MP && ORDER == 3) {
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmadd_u(-s.B2[k], D.d3slice(i, k), b);
        }
        L.part[1 + i] = kF32<T> ? b : add_u(L.part[1 + i], renorm(b));
    }
    if constexpr (ORDER == 2) {
#pragma unroll
        for (int k = 0; k < 5; ++k) L.part[4 + k] = fmadd_u(nm0, D.D2[k], L.part[4 + k]);
        T wn[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) wn[k] = SRC_MP ? fmadd(nm0, aA[k], -s.B2[k]) : nm0 * aA[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T c = S.part[i];
#pragma unroll
            for (int k = 0; k < 5; ++k) c = fmadd_u(wn[k], D.d3slice(i, k), c);
            S.part[i] = renorm(c);
        }
        return;
    }
    const T *a3A = aA;
    if constexpr (kF32<T>) {
        // orders 2-3 (12 components): the pairs in which the derivative
        // tensors come out of DTraceless<float> (xx yy | xz yz of D2, xxx yyy
        // | xxz yyz of D3) on the paired FP32 pipe (fma.rn.f32x2: each half
        // rounds as fmaf does), the other four scalar
        constexpr int pair_a[4] = {4, 7, 9, 11}, pair_b[4] = {5, 8, 14, 15};
        const float dv[16] = {0.f, 0.f, 0.f, 0.f, D.D2[0], D.D2[1], D.D2[2], D.D2[3],
                              D.D2[4], D.D3[0], D.D3[1], D.D3[2], D.D3[3], D.D3[4],
                              D.D3[5], D.D3[6]};
        const float2 nm2 = make_float2(nm0, nm0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = pair_a[j], b = pair_b[j];
            const float2 r = __ffma2_rn(nm2, make_float2(dv[a], dv[b]),
                                        make_float2(L.part[a], L.part[b]));
            L.part[a] = r.x;
            L.part[b] = r.y;
        }
        L.part[6] = fmaf(nm0, dv[6], L.part[6]);
        L.part[10] = fmaf(nm0, dv[10], L.part[10]);
        L.part[12] = fmaf(nm0, dv[12], L.part[12]);
        L.part[13] = fmaf(nm0, dv[13], L.part[13]);
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) L.part[4 + k] = fmadd_u(nm0, D.D2[k], L.part[4 + k]);
#pragma unroll
        for (int q = 0; q < 7; ++q) L.part[9 + q] = fmadd_u(nm0, D.D3[q], L.part[9 + q]);
    }
    T w[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) w[q] = SRC_MP ? fmadd(nm0, a3A[q], s.B3[q]) : nm0 * a3A[q];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T c = S.part[i];
#pragma unroll
        for (int q = 0; q < 7; ++q) c = fmadd_u(w[q], D.U[i][q], c);
        S.part[i] = renorm(c);
    }
}

// One multipole source into a leaf target (orders 0-1 and the correction;
// the target has no third moment)
// (ORDER = 2: L0 -= M0 D0 + B2.D2, L1 -= M0 D1, S_i -= B2 . D3[i, .])
template <typename T, int ORDER = 3>
__device__ __forceinline__ void acc_mx(T Rx, T Ry, T Rz, const Src<T> &s, Acc<T, 4> &L,
                                       Acc<T, 3> &S)
{
    DTraceless<T> D;
    D.template eval<ORDER == 3>(Rx, Ry, Rz);
    T a = -s.m0 * D.D0;
#pragma unroll
    for (int k = 0; k < 5; ++k) a = fmadd_u(-s.B2[k], D.D2[k], a);
    if (ORDER == 3) {
#pragma unroll
        for (int q = 0; q < 7; ++q) a = fmadd_u(s.B3[q], D.D3[q], a);
    }
    L.part[0] = add_u(L.part[0], renorm(a));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T b = -s.m0 * D.D1[i];
        T c = S.part[i];
        if (ORDER == 3) {
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmadd_u(-s.B2[k], D.d3slice(i, k), b);
#pragma unroll
            for (int q = 0; q < 7; ++q) c = fmadd_u(s.B3[q], D.U[i][q], c);
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) c = fmadd_u(-s.B2[k], D.d3slice(i, k), c);
        }
        L.part[1 + i] = add_u(L.part[1 + i], renorm(b));
        S.part[i] = renorm(c);
    }
}

// target-to-source separation in cell widths, R = (dA - d) - E, in that
// order; float takes x and y as one pair (the offsets' x and y sit in
// aligned register pairs: first in their 16-byte groups)
template <typename T>
__device__ __forceinline__ void separation(const T dA[3], const T d[3], const float4 &E, T R[3])
{
    if constexpr (kF32<T>) {
        const float2 u = fsub2_rn(make_float2(dA[0], dA[1]), make_float2(d[0], d[1]));
        const float2 r = fsub2_rn(u, make_float2(E.x, E.y));
        R[0] = r.x;
        R[1] = r.y;
        R[2] = dA[2] - d[2] - E.z;
    } else {
        R[0] = dA[0] - d[0] - T(E.x);
        R[1] = dA[1] - d[1] - T(E.y);
        R[2] = dA[2] - d[2] - T(E.z);
    }
}

// own packed data of a multipole target: centre-of-mass offset and
// a3 = B3/M0 (order 3) or a2 = B2/M0 in the first five entries (order 2)
template <typename T, int ORDER = 3>
__device__ __forceinline__ void load_target(const KParams &P, int row, int pi, T dA[3], T aA[7])
{
    Src<T> own;
    load_source<T>(P, row, pi, own);
    const T im0 = T(1) / own.m0;
#pragma unroll
    for (int a = 0; a < 3; ++a) dA[a] = own.d[a];
    if (ORDER == 3) {
#pragma unroll
        for (int q = 0; q < 7; ++q) aA[q] = own.B3[q] * im0;
    } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) aA[q] = own.B2[q] * im0;
        aA[5] = aA[6] = T(0);
    }
}

__device__ __forceinline__ double to_double(float v) { return double(v); }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(dfloat v) { return v.to_double(); }

template <typename T, class SA>
__device__ __forceinline__ double acc_value(const SA &S, int i)
{
    return to_double(acc_hi(S, i)) + to_double(acc_lo(S, i));
}

// ------------------------------------------------- monopole<-multipole
// One leaf target cell with refined sources (one lane): its own list of
// (packed-moment offset, stencil entry) pairs, orders 0-1 and the correction
// added to what the monopole kernel stored for the cell.
template <typename T, int ORDER = 3>
__device__ __forceinline__ void mx_target(const KParams &P, int t)
{
    const T *mp = static_cast<const T *>(P.mp);
    const int4 tg = __ldg(P.mx_targets + t);       // node, cell, pair offset, count
    const int x = tg.y & 7, y = (tg.y >> 3) & 7, z = tg.y >> 6;
    const int p = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
    const float4 *ent = P.stencil_f + p * P.ent_stride;   // float offsets: no conversions
    Acc<T, 4> L;
    Acc<T, 3> S;
    L.zero();
    S.zero();
    int done = 0;
    // this lane's pairs, interleaved with its warp's: pair k at base + 32 k + lane;
    // the next pair is fetched while the current one is evaluated
    const int2 *pairs = P.mx_pairs + size_t(tg.z) + (t & 31);
    int2 next = tg.w > 0 ? __ldg(pairs) : make_int2(0, 0);
    for (int k = 0; k < tg.w; ++k) {
        const int2 pr = next;
        if (k + 1 < tg.w) next = __ldg(pairs + size_t(k + 1) * 32);
        const float4 E = __ldg(ent + pr.y);
        Src<T> src;
        load_source_at<T>(mp + pr.x, src);
        acc_mx<T, ORDER>(-T(E.x) - src.d[0], -T(E.y) - src.d[1], -T(E.z) - src.d[2], src, L, S);
        if (++done == kChunk) {
            L.flush();
            S.flush();
            done = 0;
        }
    }
    L.flush();
    S.flush();
    const int node = tg.x, cell = tg.y;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t idx = (size_t(node) * NCOMP + k) * NCELL + cell;
        if constexpr (kF32<T>) {
            float *Lh = static_cast<float *>(P.L);
            float s, e;
            two_sum(Lh[idx], L.hi[k], s, e);
            const float lo = P.Lc[idx] + L.lo[k] + e;
            const float s2 = s + lo;
            Lh[idx] = s2;
            P.Lc[idx] = lo - (s2 - s);
        } else if constexpr (kDF<T>) {
            float *Lh = static_cast<float *>(P.L);
            const dfloat v = dfloat(Lh[idx], P.Lc[idx]) + L.part[k];
            Lh[idx] = v.hi;
            P.Lc[idx] = v.lo;
        } else {
            static_cast<double *>(P.L)[idx] += L.hi[k];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) P.dL1[(size_t(node) * 3 + i) * NCELL + cell] = acc_value<T>(S, i);
}

// ------------------------------------------------------------ mp_kernel
// HALVES: item k is half k & 1 (cells of z < 4 or z >= 4) of node list[k >> 1],
// else item k is all of node list[k]
template <typename T, int ORDER, bool HALVES>
// float: three CTAs per SM (at most 85 registers): the compensation pairs,
// touched once per chunk, live in shared memory after the window
__global__ void __launch_bounds__(kThreads, kF32<T> ? 3 : 1) mp_kernel(KParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *W = reinterpret_cast<T *>(smem_raw);
    float *Cs = reinterpret_cast<float *>(W + 8 * P.sub_stride) + threadIdx.x;   // float only
    __shared__ int s_nbr[27], s_leaf[27], s_row[27], s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz0 = lane >> 4;
    const float4 *ent = P.stencil_f + p * P.ent_stride;   // float offsets: no conversions
    const T *mass = static_cast<const T *>(P.mass);
    const T *mp = static_cast<const T *>(P.mp);
    for (;;) {
        const int item = pull_item(P.counter, &s_item);
        if (item >= P.n_items) break;
        const int node = P.list[HALVES ? item >> 1 : item];
        const NodeInfo ti = P.info[node];
        // near sources contribute only if some neighbour is a leaf
        const int any_leaf = __syncthreads_or(load_slots(node, P, s_nbr, s_leaf, s_row));
        stage_window_async<T>(W, s_nbr, s_leaf, mass, P, s_row);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int half0 = HALVES ? item & 1 : 0;
        const int half1 = HALVES ? half0 + 1 : 2;
        for (int half = half0; half < half1; ++half) {
            const int cz = cz0 + 2 * half;
            const int ax = 2 * cx + px, ay = 2 * cy + py, az = 2 * cz + pz;
            const int base = cx + P.py * cy + P.pz * cz;
            T dA[3], a3A[7];
            load_target<T, ORDER>(P, ti.mp_row, parity_index(ax, ay, az), dA, a3A);
            typename MpAcc<T, 16>::type L;
            typename MpAcc<T, 3>::type S;
            if constexpr (kF32<T>) {
                L.col = Cs;
                S.col = Cs + 4 * 2 * kThreads;
            }
            L.zero();
            S.zero();
            // well-separated sources: refined (full moments) or leaf (mass).
            // In float, a vote classifies the warp's 32 sources of one
            // entry: all refined take the moments without a branch, all
            // leaves the mass-only form (the same operations less the zero
            // moments' terms, so the same values), a mix the general form
            // with zero moments for the leaves, and an entry with only
            // absent sources (mass 0) is skipped.
            for (int e0 = 0; e0 < P.n_far; e0 += kChunk) {
                const int e1 = min(e0 + kChunk, P.n_far);
                for (int e = e0; e < e1; ++e) {
                    const float4 E = __ldg(ent + e);
                    const T wv = W[base + __float_as_int(E.w)];
                    int idx;
                    const bool is_mp = window_moments<T>(wv, P.mp_limit, idx);
                    // (the double-float and double bodies are several times
                    // larger, and extra copies of them cost more in
                    // instruction fetch than they save: general form only)
                    const bool all_mp = kF32<T> && __all_sync(0xffffffffu, is_mp);
                    Src<T> src;
                    T R[3];
                    if (all_mp) {
                        load_source_at<T>(mp + idx, src);
                        separation<T>(dA, src.d, E, R);
                        acc_mp<T, true, ORDER>(R[0], R[1], R[2], src, a3A, L, S);
                    } else if (kF32<T> && !__any_sync(0xffffffffu, is_mp)) {
                        if (__any_sync(0xffffffffu, window_nonzero<T>(wv))) {
                            src.m0 = wv;
                            acc_mp<T, false, ORDER>(dA[0] - T(E.x), dA[1] - T(E.y),
                                                    dA[2] - T(E.z), src, a3A, L, S);
                        }
                    } else {
                        if constexpr (kF32<T>) {
                            if (is_mp) {
                                load_source_at<T>(mp + idx, src);
                            } else {
                                src.m0 = wv;
                                zero_moments<T>(src);
                            }
                        } else {
                            // leaf lanes read zero moments from the zero row
                            // (no branch; the warp issues the loads anyway):
                            // faster for the wider types, slower for float
                            load_source_at<T>(mp + (is_mp ? idx : P.mp_limit), src);
                            if (!is_mp) src.m0 = wv;
                        }
                        separation<T>(dA, src.d, E, R);
                        acc_mp<T, true, ORDER>(R[0], R[1], R[2], src, a3A, L, S);
                    }
                }
                L.flush();
                S.flush();
            }
            // near sources: leaf cells only (refined ones contribute nothing
            // here: their children interact one level down); skipped when no
            // neighbour is a leaf, and entry by entry when none of the
            // warp's 32 sources is a leaf with mass (skipping exact zeros
            // changes no sum)
            for (int e0 = P.n_far; any_leaf && e0 < P.n_far + P.n_near; e0 += kChunk) {
                const int e1 = min(e0 + kChunk, P.n_far + P.n_near);
                for (int e = e0; e < e1; ++e) {
                    const float4 E = __ldg(ent + e);
                    const T wv = W[base + __float_as_int(E.w)];
                    Src<T> src;
                    src.m0 = window_refined<T>(wv) ? T(0) : wv;
                    if (!__any_sync(0xffffffffu, window_nonzero<T>(src.m0))) continue;
                    acc_mp<T, false, ORDER>(dA[0] - T(E.x), dA[1] - T(E.y), dA[2] - T(E.z), src, a3A,
                                     L, S);
                }
                L.flush();
                S.flush();
            }
            const int cell = ax + 8 * ay + 64 * az;
            store_target<T>(P, node, cell, L);
#pragma unroll
            for (int i = 0; i < 3; ++i)
                __stcs(P.dL1 + (size_t(node) * 3 + i) * NCELL + cell, acc_value<T>(S, i));
        }
        __syncthreads();
    }
    // fmm_step also hands this launch the monopole<-multipole targets: once
    // the multipole queue is empty, each warp pulls 32 of them at a time
    // from their own queue, which fills the tail that the coarse multipole
    // items leave (the monopole kernel, whose results they add to, has
    // finished before this launch)
    if (P.n_mx > 0) {
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(P.mx_counter, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w * 32 >= P.n_mx) break;
            if (w * 32 + lane < P.n_mx) mx_target<T, ORDER>(P, w * 32 + lane);
        }
    }
}

// ----------------------------------------------------------- mp2_kernel
// The multipole kernel (float) with each thread's two target cells (z and
// z + 4 of one parity) walked through the stencil together instead of one
// after the other: one stencil-entry load serves both, and the two cells'
// independent loads and arithmetic interleave, so each warp has twice the
// work in flight between its dependent steps.  Two CTAs per SM (at most 128
// registers) and both cells' compensation pairs in shared memory.  Every
// cell's operations and their order are those of mp_kernel, so the results
// are the same bits.
constexpr int kMp2Pairs = 2 * kMpPairs;

__device__ __forceinline__ void mp2_source(const KParams &P, const float *mp, float wv, Src<float> &src)
{
    // masses are not negative, so a mass's decoded offset is out of range
    const unsigned idx = unsigned(-1 - __float_as_int(wv));
    if (idx < unsigned(P.mp_limit)) {
        load_source_at<float>(mp + idx, src);
    } else {
        src.m0 = wv;
        zero_moments<float>(src);
    }
}

__global__ void __launch_bounds__(kThreads, 2) mp2_kernel(KParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *W = reinterpret_cast<float *>(smem_raw);
    float *Cs = W + 8 * P.sub_stride + threadIdx.x;
    __shared__ int s_nbr[27], s_leaf[27], s_row[27], s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz0 = lane >> 4;
    const float4 *ent = P.stencil_f + p * P.ent_stride;
    const float *mass = static_cast<const float *>(P.mass);
    const float *mp = static_cast<const float *>(P.mp);
    for (;;) {
        const int item = pull_item(P.counter, &s_item);
        if (item >= P.n_items) break;
        const int node = P.list[item];
        const NodeInfo ti = P.info[node];
        const int any_leaf = __syncthreads_or(load_slots(node, P, s_nbr, s_leaf, s_row));
        stage_window_async<float>(W, s_nbr, s_leaf, mass, P, s_row);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int ax = 2 * cx + px, ay = 2 * cy + py;
        const int az0 = 2 * cz0 + pz, az1 = az0 + 4;
        const int base0 = cx + P.py * cy + P.pz * cz0, base1 = base0 + 2 * P.pz;
        float dA0[3], a3A0[7], dA1[3], a3A1[7];
        load_target<float>(P, ti.mp_row, parity_index(ax, ay, az0), dA0, a3A0);
        load_target<float>(P, ti.mp_row, parity_index(ax, ay, az1), dA1, a3A1);
        MpAcc<float, 16>::type L0, L1;
        MpAcc<float, 3>::type S0, S1;
        L0.col = Cs;
        S0.col = Cs + 4 * 2 * kThreads;
        L1.col = Cs + kMpPairs * 2 * kThreads;
        S1.col = Cs + (kMpPairs + 4) * 2 * kThreads;
        L0.zero();
        S0.zero();
        L1.zero();
        S1.zero();
        for (int e0 = 0; e0 < P.n_far; e0 += kChunk) {
            const int e1 = min(e0 + kChunk, P.n_far);
            for (int e = e0; e < e1; ++e) {
                const float4 E = __ldg(ent + e);
                const int woff = __float_as_int(E.w);
                const float w0 = W[base0 + woff], w1 = W[base1 + woff];
                const unsigned i0 = unsigned(-1 - __float_as_int(w0));
                const unsigned i1 = unsigned(-1 - __float_as_int(w1));
                Src<float> s0, s1;
                // the warp's 64 sources all refined: the moments without a
                // branch (the same values as the general form)
                if (__all_sync(0xffffffffu, i0 < unsigned(P.mp_limit) && i1 < unsigned(P.mp_limit))) {
                    load_source_at<float>(mp + i0, s0);
                    load_source_at<float>(mp + i1, s1);
                } else {
                    mp2_source(P, mp, w0, s0);
                    mp2_source(P, mp, w1, s1);
                }
                float R0[3], R1[3];
                separation<float>(dA0, s0.d, E, R0);
                separation<float>(dA1, s1.d, E, R1);
                acc_mp<float, true>(R0[0], R0[1], R0[2], s0, a3A0, L0, S0);
                acc_mp<float, true>(R1[0], R1[1], R1[2], s1, a3A1, L1, S1);
            }
            L0.flush();
            S0.flush();
            L1.flush();
            S1.flush();
        }
        for (int e0 = P.n_far; any_leaf && e0 < P.n_far + P.n_near; e0 += kChunk) {
            const int e1 = min(e0 + kChunk, P.n_far + P.n_near);
            for (int e = e0; e < e1; ++e) {
                const float4 E = __ldg(ent + e);
                const int woff = __float_as_int(E.w);
                const float w0 = W[base0 + woff], w1 = W[base1 + woff];
                Src<float> s0, s1;
                s0.m0 = unsigned(-1 - __float_as_int(w0)) < unsigned(P.mp_limit) ? 0.f : w0;
                s1.m0 = unsigned(-1 - __float_as_int(w1)) < unsigned(P.mp_limit) ? 0.f : w1;
                if (!__any_sync(0xffffffffu, s0.m0 != 0.f || s1.m0 != 0.f)) continue;
                acc_mp<float, false>(dA0[0] - E.x, dA0[1] - E.y, dA0[2] - E.z, s0, a3A0, L0, S0);
                acc_mp<float, false>(dA1[0] - E.x, dA1[1] - E.y, dA1[2] - E.z, s1, a3A1, L1, S1);
            }
            L0.flush();
            S0.flush();
            L1.flush();
            S1.flush();
        }
        const int cell0 = ax + 8 * ay + 64 * az0, cell1 = ax + 8 * ay + 64 * az1;
        store_target<float>(P, node, cell0, L0);
        store_target<float>(P, node, cell1, L1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            P.dL1[(size_t(node) * 3 + i) * NCELL + cell0] = acc_value<float>(S0, i);
            P.dL1[(size_t(node) * 3 + i) * NCELL + cell1] = acc_value<float>(S1, i);
        }
        __syncthreads();
    }
    if (P.n_mx > 0) {
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(P.mx_counter, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w * 32 >= P.n_mx) break;
            if (w * 32 + lane < P.n_mx) mx_target<float>(P, w * 32 + lane);
        }
    }
}

// ---------------------------------------------------------- mono_kernel
// Leaf target, leaf sources: R = -o exactly, so L0 += c0(o) m and
// L1 += c1(o) m with per-offset weights c0 = -1/|o|, c1 = -o/|o|^3.
// Every parity's stencil is parity 0's reflected along its odd axes, so a
// warp of parity p walks parity 0's entries, reflected (mono_woff holds
// their window offsets), and one weight table (parity 0's) serves all eight
// warps: the warp accumulates with parity 0's first-order weights and flips
// the signs of its L1 components along p's odd axes at the end (exact).  The
// table and the window offsets sit in shared memory, loaded once per CTA;
// every access to them is a warp-uniform broadcast.
// Each pass takes NB sub-grids (consecutive in the cost-sorted queue), each
// with its own halo window, staged by cp.async so that every load of the
// window is in flight at once; every thread holds two target cells (z and
// z+4 of one parity) per sub-grid, so each weight feeds 2 NB cells.
template <typename T>
__device__ __forceinline__ void load4_shared(const T *p, T v[4])
{
    if constexpr (kF32<T>) {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else if constexpr (kDF<T>) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w);
        v[2] = dfloat(b.x, b.y); v[3] = dfloat(b.z, b.w);
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

// Wb = the window at this thread's first target cell; the NB windows are
// WSTRIDE apart and the second target cell DZ1 further on (compile-time
// offsets, folded into the shared-memory loads)
template <typename T, int NB, int WSTRIDE, int DZ1>
__device__ __forceinline__ void mono_entry(const T *Wb, const int *woff, const T *coef, int e,
                                           Acc<T, 4> (&A)[NB], Acc<T, 4> (&B)[NB])
{
    const T *src = Wb + woff[e];
    T c[4];
    load4_shared<T>(coef + 4 * e, c);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const T m0 = src[b * WSTRIDE];
        const T m1 = src[b * WSTRIDE + DZ1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            A[b].part[k] = fmadd_u(c[k], m0, A[b].part[k]);
            B[b].part[k] = fmadd_u(c[k], m1, B[b].part[k]);
        }
    }
}

// dynamic shared memory of mono_kernel<T, NB, R>: NB windows, the weight table
// of parity 0 and the window offsets of all parities
template <typename T>
size_t mono_smem_bytes(int nb, size_t window_bytes, int ent_stride)
{
    return nb * window_bytes + size_t(ent_stride) * 4 * sizeof(T) + size_t(8) * ent_stride * sizeof(int);
}

template <typename T, int NB, int RR>
__global__ void __launch_bounds__(kThreads) mono_kernel(KParams P)
{
    using G = WinGeo<RR>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int wstride = 8 * G::SUB_STRIDE;
    T *W = reinterpret_cast<T *>(smem_raw);
    T *s_coef = W + NB * wstride;
    int *s_woff = reinterpret_cast<int *>(s_coef + 4 * P.ent_stride);
    __shared__ int s_nbr[NB][27], s_leaf[NB][27], s_row[NB][27], s_item;
    const int n_ent = P.n_far + P.n_near;
    {
        const T *gcoef = static_cast<const T *>(P.coef);          // parity 0 first
        for (int i = threadIdx.x; i < 4 * n_ent; i += blockDim.x) s_coef[i] = ldg_t(gcoef + i);
        for (int i = threadIdx.x; i < 8 * P.ent_stride; i += blockDim.x)
            s_woff[i] = __ldg(P.mono_woff + i);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz = lane >> 4;
    const int *woff = s_woff + p * P.ent_stride;
    const T *mass = static_cast<const T *>(P.mass);
    const int base0 = cx + G::PY * cy + G::PZ * cz;
    constexpr int dz1 = 2 * G::PZ;              // the second target cell, z + 4
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.counter, NB);
        __syncthreads();
        const int item0 = s_item;
        if (item0 >= P.n_items) break;
        int nodes[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) nodes[b] = item0 + b < P.n_items ? P.list[item0 + b] : -1;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (nodes[b] >= 0) load_slots(nodes[b], P, s_nbr[b], s_leaf[b], s_row[b]);
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (nodes[b] >= 0) stage_window_async<T, RR>(W + b * wstride, s_nbr[b], s_leaf[b], mass, P);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        Acc<T, 4> A[NB], B[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            A[b].zero();
            B[b].zero();
        }
        // float: 32 entries per compensated chunk (the TwoSum folds are a
        // fifth of this kernel's instructions at 16); double-float keeps 16
        constexpr int chunk = kF32<T> ? 2 * kChunk : kChunk;
        int e = 0;
        for (; e + chunk <= n_ent; e += chunk) {
#pragma unroll
            for (int j = 0; j < chunk; ++j)
                mono_entry<T, NB, wstride, dz1>(W + base0, woff, s_coef, e + j, A, B);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                A[b].flush();
                B[b].flush();
            }
        }
        for (; e < n_ent; ++e) mono_entry<T, NB, wstride, dz1>(W + base0, woff, s_coef, e, A, B);
        const int ax = 2 * cx + px, ay = 2 * cy + py;
        const int cell0 = ax + 8 * ay + 64 * (2 * cz + pz);
        const int cell1 = cell0 + 64 * 4;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (nodes[b] < 0) continue;
            A[b].flush();
            B[b].flush();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // first-order weights were parity 0's: undo the reflection
                const bool flip = k > 0 && ((p >> (k - 1)) & 1);
                const T ah = acc_hi(A[b], k), al = acc_lo(A[b], k);
                const T bh = acc_hi(B[b], k), bl = acc_lo(B[b], k);
                store_L<T>(P, nodes[b], k, cell0, flip ? -ah : ah, flip ? -al : al);
                store_L<T>(P, nodes[b], k, cell1, flip ? -bh : bh, flip ? -bl : bl);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                __stcs(P.dL1 + (size_t(nodes[b]) * 3 + i) * NCELL + cell0, 0.0);
                __stcs(P.dL1 + (size_t(nodes[b]) * 3 + i) * NCELL + cell1, 0.0);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ mx_kernel
// Leaf targets, refined sources (monopole<-multipole): orders 0-1 and the
// correction (the target has no third moment).  Adds to what mono_kernel
// stored for the same cells, so it runs after it on the same stream.  Few
// targets of a node see refined sources, and those see few (16 on average
// on the workloads), so instead of walking every stencil entry with most
// lanes masked off, each lane takes one target cell and walks that cell's
// own list of (packed-moment offset, stencil entry) pairs, built on the
// host; targets are sorted by list length, so a warp's lanes finish together,
// and a warp's lists are interleaved, so each step of the walk reads the
// warp's 32 pairs as one contiguous block.
template <typename T, int ORDER>
__global__ void __launch_bounds__(kThreads) mx_kernel(KParams P)
{
    const int lane = threadIdx.x & 31;
    const int warps = int(gridDim.x) * (kThreads / 32);
    for (int w = int(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); w * 32 < P.n_items;
         w += warps) {
        const int t = w * 32 + lane;
        if (t < P.n_items) mx_target<T, ORDER>(P, t);
    }
}

// ---------------------------------------------------------- root_kernel
// Level 1 holds one node per tree and every pair is a candidate: a refined
// root evaluates its well-separated pairs, a leaf root all pairs.  The
// 512 x 511 pairs of one root are spread over 16 CTAs of 32 targets, each
// target's 512 sources over 8 warps; the 8 partial sums are folded in a
// fixed order (deterministic).
constexpr int kRootSlices = 8;
constexpr int kRootThreads = 32 * kRootSlices;
constexpr int kRootGroups = NCELL / 32;

template <typename T, int ORDER>
__global__ void __launch_bounds__(kRootThreads) root_kernel(KParams P)
{
    constexpr int NV = 16 + 3;                      // L (traceless), S
    __shared__ T sh_hi[kRootSlices][NV][32];
    __shared__ T sh_lo[kRootSlices][kF32<T> ? NV : 1][32];   // float only
    const int node = P.list[blockIdx.x];
    const NodeInfo ti = P.info[node];
    const bool leaf = ti.leaf_row >= 0;
    const T *mass = static_cast<const T *>(P.mass);
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int cell = blockIdx.y * 32 + lane;
    const int ax = cell & 7, ay = (cell >> 3) & 7, az = cell >> 6;
    T dA[3] = {T(0), T(0), T(0)}, a3A[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    if (!leaf) load_target<T, ORDER>(P, ti.mp_row, parity_index(ax, ay, az), dA, a3A);
    Acc<T, 16> L;
    Acc<T, 3> S;
    L.zero();
    S.zero();
    int done = 0;
    const int b0 = slice * (NCELL / kRootSlices);
    for (int b = b0; b < b0 + NCELL / kRootSlices; ++b) {
        const int ox = (b & 7) - ax, oy = ((b >> 3) & 7) - ay, oz = (b >> 6) - az;
        const bool far = ox * ox + oy * oy + oz * oz >= P.far_o2;
        if (b == cell || !(far || leaf)) continue;
        const int pi = parity_index(b & 7, (b >> 3) & 7, b >> 6);
        Src<T> src;
        if (!leaf) {
            load_source<T>(P, ti.mp_row, pi, src);
        } else {
            src.m0 = mass[size_t(node) * NCELL + pi];
            zero_moments<T>(src);
        }
        acc_mp<T, true, ORDER>(dA[0] - src.d[0] - T(ox), dA[1] - src.d[1] - T(oy),
                        dA[2] - src.d[2] - T(oz), src, a3A, L, S);
        if (++done == kChunk) {
            L.flush();
            S.flush();
            done = 0;
        }
    }
    L.flush();
    S.flush();
    for (int k = 0; k < 16; ++k) {
        sh_hi[slice][k][lane] = acc_hi(L, k);
        if constexpr (kF32<T>) sh_lo[slice][k][lane] = acc_lo(L, k);
    }
    for (int i = 0; i < 3; ++i) {
        sh_hi[slice][16 + i][lane] = acc_hi(S, i);
        if constexpr (kF32<T>) sh_lo[slice][16 + i][lane] = acc_lo(S, i);
    }
    __syncthreads();
    if (slice != 0) return;
    T Fh[NV], Fl[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T hi = T(0), lo = T(0);
        for (int sl = 0; sl < kRootSlices; ++sl) {
            if constexpr (kF32<T>) {
                float sum, err;
                two_sum(hi, sh_hi[sl][k][lane], sum, err);
                hi = sum;
                lo += err + sh_lo[sl][k][lane];
            } else {
                hi += sh_hi[sl][k][lane];
            }
        }
        Fh[k] = hi;
        Fl[k] = lo;
    }
    if (leaf) {
        for (int k = 0; k < 4; ++k) store_L<T>(P, node, k, cell, Fh[k], Fl[k]);
    } else {
        store_target_values<T>(P, node, cell, Fh, Fl);
    }
    for (int i = 0; i < 3; ++i)
        P.dL1[(size_t(node) * 3 + i) * NCELL + cell] = to_double(Fh[16 + i]) + to_double(Fl[16 + i]);
}

// ---------------------------------------------------------- launching
// opt-in dynamic shared memory of a kernel, raised once to the largest size
// asked for so far
template <typename Kern>
cudaError_t allow_smem(Kern k, size_t bytes, size_t &done)
{
    if (bytes <= done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) done = bytes;
    return e;
}

template <typename T>
struct Kernels {
    template <int ORDER, bool HALVES>
    static cudaError_t mp(size_t bytes)
    {
        static size_t done = 0;
        return allow_smem(mp_kernel<T, ORDER, HALVES>, bytes, done);
    }
    static cudaError_t mp2(size_t bytes)
    {
        static size_t done = 0;
        return allow_smem(mp2_kernel, bytes, done);
    }
    template <int NB, int RR>
    static cudaError_t mono(size_t bytes)
    {
        static size_t done = 0;
        return allow_smem(mono_kernel<T, NB, RR>, bytes, done);
    }
};

// persistent grid: SMs x resident CTAs (optionally capped by the tuning)
template <typename Kern>
int persistent_grid(Kern k, size_t smem, int64_t items, int sms, int cap_per_sm)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (cap_per_sm > 0 && cap_per_sm < per_sm) per_sm = cap_per_sm;
    int64_t g = int64_t(per_sm) * sms;
    return int(items < g ? items : g);
}

template <typename T, int NB, int RR>
cudaError_t launch_mono_r(const KParams &K, size_t wbytes, int sms, int cap, cudaStream_t s)
{
    // the compile-time window geometry must be the host's
    using G = WinGeo<RR>;
    if (K.reach != G::R || K.py != G::PY || K.pz != G::PZ || K.sub_stride != G::SUB_STRIDE)
        return cudaErrorInvalidValue;
    const size_t bytes = mono_smem_bytes<T>(NB, wbytes, K.ent_stride);
    cudaError_t e = Kernels<T>::template mono<NB, RR>(bytes);
    if (e != cudaSuccess) return e;
    const int64_t passes = (K.n_items + NB - 1) / NB;
    const int g = persistent_grid(mono_kernel<T, NB, RR>, bytes, passes, sms, cap);
    mono_kernel<T, NB, RR><<<g, kThreads, bytes, s>>>(K);
    return cudaGetLastError();
}

// theta in (0.25, 1/sqrt(3)] gives reach 2 floor(1/theta) + 1 = 3, 5 or 7
template <typename T, int NB>
cudaError_t launch_mono(const KParams &K, size_t wbytes, int sms, int cap, cudaStream_t s)
{
    switch (K.reach) {
    case 3: return launch_mono_r<T, NB, 3>(K, wbytes, sms, cap, s);
    case 5: return launch_mono_r<T, NB, 5>(K, wbytes, sms, cap, s);
    case 7: return launch_mono_r<T, NB, 7>(K, wbytes, sms, cap, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int ORDER>
cudaError_t launch_all(const fmm_tree_s *t, void *L, float *Lc, double *dL1, cudaStream_t s,
                       int *n_launches, int parts)
{
    const Plan &Pl = t->plan;
    const DeviceTables &d = t->dev;
    KParams P{};
    P.info = d.info;
    P.nbr = d.nbr;
    P.stencil = d.stencil;
    P.stencil_f = reinterpret_cast<const float4 *>(d.stencil_f);
    P.coef = kF32<T> ? static_cast<const void *>(d.coef32)
             : kDF<T> ? static_cast<const void *>(d.coefdf)
                      : static_cast<const void *>(d.coef64);
    P.n_far = Pl.n_far[0];
    P.n_near = Pl.n_near[0];
    P.ent_stride = Pl.ent_stride;
    P.reach = Pl.reach;
    P.py = Pl.py;
    P.pz = Pl.pz;
    P.sub_stride = Pl.sub_stride;
    P.mass = d.mass;
    P.mp = d.mp;
    P.mp_limit = int(t->n_refined * 4 * NCELL * 4);
    P.L = L;
    P.Lc = Lc;
    P.dL1 = dL1;
    P.far_o2 = t->plan.far_o2;
    P.mx_targets = d.mx_targets;
    P.mx_pairs = d.mx_pairs;
    P.mono_woff = d.mono_woff;
    const int cap = t->tuning.ctas_per_sm;
    const size_t wbytes = size_t(8) * Pl.sub_stride * sizeof(T);
    // mp_kernel: one window (masses of leaf sources, moment offsets of
    // refined ones); float adds its compensation pairs, [7][2][threads]
    const size_t mp_bytes = wbytes + (kF32<T> ? size_t(kMpPairs) * 2 * kThreads * sizeof(float) : 0);
    cudaError_t e = Kernels<T>::template mp<ORDER, false>(mp_bytes);
    if (e == cudaSuccess) e = Kernels<T>::template mp<ORDER, true>(mp_bytes);
    if (e != cudaSuccess) return e;
    if (parts & M2L_RESET) {
        e = cudaMemsetAsync(d.counters, 0, 4 * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    const int sms = sm_count_of_current_device();
    int nl = 0;
    // M2L_MPX: the monopole<-multipole targets ride in the multipole launch
    // when there is one, else they get their own
    const bool mx_in_mp = (parts & M2L_MPX) && (parts & M2L_MP) && Pl.work_mp.count > 0;
    if ((parts & M2L_ROOT) && Pl.roots.count) {
        KParams R = P;
        R.list = d.lists + Pl.roots.off;
        R.n_items = int32_t(Pl.roots.count);
        timing_begin(t, FMM_K_ROOT, s);
        root_kernel<T, ORDER><<<dim3(unsigned(Pl.roots.count), kRootGroups), kRootThreads, 0, s>>>(R);
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((parts & M2L_MP) && Pl.work_mp.count) {
        KParams K = P;
        K.list = d.lists + Pl.work_mp.off;
        K.n_items = int32_t(Pl.work_mp.count);
        K.counter = d.counters + Q_MP;
        if (mx_in_mp) {
            K.n_mx = int32_t(Pl.n_mx_targets);
            K.mx_counter = d.counters + Q_MX;
        }
        timing_begin(t, FMM_K_MULTIPOLE, s);
        if (kF32<T> && ORDER == 3 && t->tuning.mp_pair_targets) {
            // both target cells of a thread together (float only)
            const size_t b2 = wbytes + size_t(kMp2Pairs) * 2 * kThreads * sizeof(float);
            if ((e = Kernels<T>::mp2(b2)) != cudaSuccess) return e;
            int g = persistent_grid(mp2_kernel, b2, Pl.work_mp.count, sms, cap);
            mp2_kernel<<<g, kThreads, b2, s>>>(K);
        } else {
            // half sub-grids per item where whole ones would leave CTA slots
            // idle or unbalanced (fewer nodes than twice the slots)
            const int64_t slots =
                persistent_grid(mp_kernel<T, ORDER, false>, mp_bytes, INT32_MAX, sms, cap);
            const int mode = t->tuning.mp_items;
            if (mode == 2 || (mode == 0 && Pl.work_mp.count < 2 * slots)) {
                K.n_items = int32_t(2 * Pl.work_mp.count);
                int g = persistent_grid(mp_kernel<T, ORDER, true>, mp_bytes, K.n_items, sms, cap);
                mp_kernel<T, ORDER, true><<<g, kThreads, mp_bytes, s>>>(K);
            } else {
                int g = persistent_grid(mp_kernel<T, ORDER, false>, mp_bytes, K.n_items, sms, cap);
                mp_kernel<T, ORDER, false><<<g, kThreads, mp_bytes, s>>>(K);
            }
        }
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((parts & M2L_MONO) && Pl.work_mono.count) {
        KParams K = P;
        K.list = d.lists + Pl.work_mono.off;
        K.n_items = int32_t(Pl.work_mono.count);
        K.counter = d.counters + Q_MONO;
        int nb = t->tuning.mono_subgrids;
        if (nb != 1 && nb != 2 && nb != 4) nb = kF32<T> ? 2 : 1;
        if (!kF32<T> && nb == 4) nb = 2;
        // fewer sub-grids per pass where their windows do not fit
        const size_t smem_max = max_smem_optin_of_current_device();
        while (nb > 1 && mono_smem_bytes<T>(nb, wbytes, Pl.ent_stride) > smem_max) nb /= 2;
        timing_begin(t, FMM_K_MONOPOLE, s);
        e = nb == 1 ? launch_mono<T, 1>(K, wbytes, sms, cap, s)
            : nb == 2 ? launch_mono<T, 2>(K, wbytes, sms, cap, s)
                      : launch_mono<T, kF32<T> ? 4 : 2>(K, wbytes, sms, cap, s);
        timing_end(t, s);
        ++nl;
        if (e != cudaSuccess) return e;
    }
    if ((parts & (M2L_MX | M2L_MPX)) && !mx_in_mp && Pl.n_mx_targets) {
        KParams K = P;
        K.n_items = int32_t(Pl.n_mx_targets);
        const int64_t warps = (K.n_items + 31) / 32;
        int g = persistent_grid(mx_kernel<T, ORDER>, 0, (warps + kThreads / 32 - 1) / (kThreads / 32), sms,
                                cap);
        timing_begin(t, FMM_K_MONO_MULTI, s);
        mx_kernel<T, ORDER><<<g, kThreads, 0, s>>>(K);
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_launches) *n_launches = nl;
    return cudaSuccess;
}

template <typename T>
void launch_pack_t(const fmm_tree_s *t, const double *M, const double *com, cudaStream_t s,
                   const int32_t *nodes, int64_t count)
{
    const auto &c = t->cfg;
    pack_kernel<T><<<unsigned(count), 512, 0, s>>>(t->dev.info, nodes, t->dev.levels, M, com,
                                                   static_cast<T *>(t->dev.mass),
                                                   static_cast<T *>(t->dev.mp), c.box_lo[0],
                                                   c.box_lo[1], c.box_lo[2]);
}

}  // namespace

cudaError_t launch_pack(const fmm_tree_s *t, const double *M, const double *com, cudaStream_t s,
                        int which)
{
    const int32_t *nodes = nullptr;
    int64_t count = t->n;
    if (which == PACK_LEAVES) {
        nodes = t->dev.lists + t->plan.leaves.off;
        count = t->plan.leaves.count;
    } else if (which == PACK_REFINED) {
        nodes = t->dev.lists + t->plan.refined.off;
        count = t->plan.refined.count;
    }
    if (count == 0) return cudaSuccess;
    switch (t->cfg.precision) {
    case FMM_MIXED: launch_pack_t<float>(t, M, com, s, nodes, count); break;
    case FMM_DFLOAT: launch_pack_t<dfloat>(t, M, com, s, nodes, count); break;
    default: launch_pack_t<double>(t, M, com, s, nodes, count); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_m2l(const fmm_tree_s *t, void *L, float *Lc, double *dL1, cudaStream_t s,
                       int *n_launches, int parts)
{
    const bool o2 = t->cfg.order == 2;
    switch (t->cfg.precision) {
    case FMM_MIXED:
        return o2 ? launch_all<float, 2>(t, L, Lc, dL1, s, n_launches, parts)
                  : launch_all<float, 3>(t, L, Lc, dL1, s, n_launches, parts);
    case FMM_DFLOAT:
        return o2 ? launch_all<dfloat, 2>(t, L, Lc, dL1, s, n_launches, parts)
                  : launch_all<dfloat, 3>(t, L, Lc, dL1, s, n_launches, parts);
    default:
        return o2 ? launch_all<double, 2>(t, L, Lc, dL1, s, n_launches, parts)
                  : launch_all<double, 3>(t, L, Lc, dL1, s, n_launches, parts);
    }
}

}  // namespace fmm
