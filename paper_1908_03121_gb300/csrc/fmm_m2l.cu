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
// refined-source moments stream through L1 from a parity-split packed
// layout, so a warp's 32 loads of one field are contiguous.
// Mixed precision: offsets are formed from double-precision centres of mass
// (packed as offsets from the cell centre, in cell widths), the contraction
// runs in float with per-chunk sums folded into (hi, lo) pairs by TwoSum, and
// the correction is finished in double.
#include <cstdio>

#include "fmm_internal.h"
#include "fmm_tensor.cuh"

namespace fmm {

namespace {

constexpr int kThreads = 256;   // 8 warps = the 8 child parities
constexpr int kChunk = 16;      // stencil entries per compensated chunk
constexpr int Q_MP = 0, Q_MONO = 1, Q_MX = 2;   // work-queue heads

struct KParams {
    const NodeInfo *info;
    const int32_t *nbr;
    const int32_t *list;
    int32_t n_items;
    int32_t *counter;
    const StencilEntry *stencil;
    const void *coef;
    int n_far, n_near;       // identical for every parity
    int ent_stride;          // entries reserved per parity
    const int32_t *slot_mask;  // [8][2][ent_stride] neighbour slots an entry can reach
    int reach, py, pz, sub_stride;
    const void *mass;
    const void *mp;
    void *L;
    float *Lc;
    double *dL1;
    double theta2;
};

// ------------------------------------------------------------------ pack
// mass[node][pi] = M0; refined nodes also get delta = (X - centre)/h,
// A2 = mult M2 / (2 h^2), A3 = mult M3 / (6 h^3) at mp[row][field][pi].
template <typename T>
__global__ void __launch_bounds__(512) pack_kernel(const NodeInfo *__restrict__ info,
                                                   const double *__restrict__ levels,
                                                   const double *__restrict__ M,
                                                   const double *__restrict__ com,
                                                   T *__restrict__ mass, T *__restrict__ mp,
                                                   double lo_x, double lo_y, double lo_z)
{
    const int node = blockIdx.x;
    const NodeInfo ni = info[node];
    const int c = threadIdx.x;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int pi = parity_index(x, y, z);
    const double *Mn = M + size_t(node) * NCOMP * NCELL + c;
    mass[size_t(node) * NCELL + pi] = T(Mn[0]);
    if (ni.mp_row < 0) return;
    const double h = levels[ni.level * LEVEL_FIELDS + LV_H];
    const double ih = levels[ni.level * LEVEL_FIELDS + LV_IH];
    T *out = mp + size_t(ni.mp_row) * NMP * NCELL + pi;
    const double ctr[3] = {lo_x + (8.0 * ni.ix + x + 0.5) * h, lo_y + (8.0 * ni.iy + y + 0.5) * h,
                           lo_z + (8.0 * ni.iz + z + 0.5) * h};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        out[a * NCELL] = T((com[(size_t(node) * 3 + a) * NCELL + c] - ctr[a]) * ih);
    const double w2 = 0.5 * ih * ih, w3 = (1.0 / 6.0) * ih * ih * ih;
#pragma unroll
    for (int q = 0; q < 6; ++q) out[(3 + q) * NCELL] = T(mult2(q) * w2 * Mn[(4 + q) * NCELL]);
#pragma unroll
    for (int q = 0; q < 10; ++q) out[(9 + q) * NCELL] = T(mult3(q) * w3 * Mn[(10 + q) * NCELL]);
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
template <typename T>
__device__ __forceinline__ void stage_window(T *W, const int *s_nbr, const int *s_leaf,
                                             const T *__restrict__ mass, const KParams &P)
{
    const int R = P.reach;
    const int E = 8 + 2 * R;
    // one (ux, uy) column per thread pass, z innermost; the parity index and
    // the window address both split into an (x, y) part and a z part
    for (int t = threadIdx.x; t < E * E; t += blockDim.x) {
        const int ux = t % E, uy = t / E;
        const int bx = ux - R + 8, by = uy - R + 8;           // >= 1
        const int sxy = (bx >> 3) + 3 * (by >> 3);
        const int lx = bx & 7, ly = by & 7;
        const int pxy = ((lx & 1) + 2 * (ly & 1)) * 64 + (lx >> 1) + 4 * (ly >> 1);
        const int wxy = ((ux & 1) + 2 * (uy & 1)) * P.sub_stride + (ux >> 1) + P.py * (uy >> 1);
        for (int uz = 0; uz < E; ++uz) {
            const int bz = uz - R + 8;
            const int slot = sxy + 9 * (bz >> 3);
            const int lz = bz & 7;
            T v = T(0);
            if (s_leaf[slot])
                v = __ldg(mass + size_t(s_nbr[slot]) * NCELL + pxy + 256 * (lz & 1) + 16 * (lz >> 1));
            W[wxy + 4 * (uz & 1) * P.sub_stride + P.pz * (uz >> 1)] = v;
        }
    }
}

// neighbour tables of the current target node into shared memory
__device__ __forceinline__ void load_slots(int node, const KParams &P, int *s_nbr, int *s_leaf,
                                           int *s_row)
{
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
            if constexpr (sizeof(T) == 4) {
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

// store component k of a target cell: level units, (hi, lo) for float
template <typename T>
__device__ __forceinline__ void store_L(const KParams &P, int node, int k, int cell, T hi, T lo)
{
    const size_t idx = (size_t(node) * NCOMP + k) * NCELL + cell;
    if constexpr (sizeof(T) == 4) {
        // renormalise so that |lo| <= ulp(hi)/2
        float s = hi + lo;
        float e = lo - (s - hi);
        static_cast<float *>(P.L)[idx] = s;
        P.Lc[idx] = e;
    } else {
        static_cast<double *>(P.L)[idx] = hi;
    }
}

// One multipole or monopole source, accumulated into the full order-3
// expansion plus the two correction sums S1 (sum D4 : A3_B) and
// S2 (sum M0_B D4), all with the sign of L folded in.
template <typename T, bool SRC_MP>
__device__ __forceinline__ void accumulate_mp(T Rx, T Ry, T Rz, T m0, const T *A2, const T *A3,
                                              Acc<T, 20> &L, T *S1, T *S2)
{
    DTensors<T, true> D;
    D.eval(Rx, Ry, Rz);
    // L0 = -(M0 D0 + A2.D2 - A3.D3)
    T l0 = m0 * D.D0;
    if (SRC_MP) {
#pragma unroll
        for (int q = 0; q < 6; ++q) l0 += A2[q] * D.D2[q];
#pragma unroll
        for (int q = 0; q < 10; ++q) l0 -= A3[q] * D.D3[q];
    }
    L.part[0] -= l0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T l1 = m0 * D.D1[i];
        if (SRC_MP) {
#pragma unroll
            for (int q = 0; q < 6; ++q) l1 += A2[q] * D.D3[r3_of(i, q)];
        }
        L.part[1 + i] -= l1;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) L.part[4 + q] -= m0 * D.D2[q];
#pragma unroll
    for (int q = 0; q < 10; ++q) L.part[10 + q] -= m0 * D.D3[q];
    if (SRC_MP) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T s = T(0);
#pragma unroll
            for (int q = 0; q < 10; ++q) s += A3[q] * D.D4[r4_of(i, q)];
            S1[i] += s;
        }
    }
#pragma unroll
    for (int q = 0; q < 15; ++q) S2[q] += m0 * D.D4[q];
}

// load the packed data of one refined source cell
template <typename T>
__device__ __forceinline__ void load_source(const KParams &P, int node, int row, int pi, T &m0,
                                            T *dB, T *A2, T *A3)
{
    const T *mass = static_cast<const T *>(P.mass);
    const T *mp = static_cast<const T *>(P.mp) + size_t(row) * NMP * NCELL + pi;
    m0 = __ldg(mass + size_t(node) * NCELL + pi);
#pragma unroll
    for (int a = 0; a < 3; ++a) dB[a] = __ldg(mp + a * NCELL);
#pragma unroll
    for (int q = 0; q < 6; ++q) A2[q] = __ldg(mp + (3 + q) * NCELL);
#pragma unroll
    for (int q = 0; q < 10; ++q) A3[q] = __ldg(mp + (9 + q) * NCELL);
}

// per-lane source position: slot of the neighbour node and parity index
__device__ __forceinline__ void source_cell(int ax, int ay, int az, int ox, int oy, int oz,
                                            int &slot, int &pi)
{
    const int bx = ax + ox + 8, by = ay + oy + 8, bz = az + oz + 8;   // >= 1
    slot = (bx >> 3) + 3 * (by >> 3) + 9 * (bz >> 3);
    pi = parity_index(bx & 7, by & 7, bz & 7);
}

// ------------------------------------------------------------ mp_kernel
template <typename T>
// float: two CTAs per SM (128 registers; the (hi, lo) pairs, touched once per
// chunk, are what the register budget squeezes)
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) mp_kernel(KParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *W = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_nbr[27], s_leaf[27], s_row[27], s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz0 = lane >> 4;
    const StencilEntry *ent = P.stencil + p * P.ent_stride;
    const T *mass = static_cast<const T *>(P.mass);
    const T *mpd = static_cast<const T *>(P.mp);
    for (;;) {
        const int item = pull_item(P.counter, &s_item);
        if (item >= P.n_items) break;
        const int node = P.list[item];
        const NodeInfo ti = P.info[node];
        load_slots(node, P, s_nbr, s_leaf, s_row);
        __syncthreads();
        stage_window<T>(W, s_nbr, s_leaf, mass, P);
        __syncthreads();
        for (int half = 0; half < 2; ++half) {
            const int cz = cz0 + 2 * half;
            const int ax = 2 * cx + px, ay = 2 * cy + py, az = 2 * cz + pz;
            const int base = cx + P.py * cy + P.pz * cz;
            const int tpi = parity_index(ax, ay, az);
            const T *own = mpd + size_t(ti.mp_row) * NMP * NCELL + tpi;
            const T dAx = own[0], dAy = own[NCELL], dAz = own[2 * NCELL];
            Acc<T, 20> L;
            L.zero();
            T S1[3] = {T(0), T(0), T(0)};
            T S2[15];
#pragma unroll
            for (int q = 0; q < 15; ++q) S2[q] = T(0);
            // well-separated sources: refined (full moments) or leaf (mass)
            for (int e0 = 0; e0 < P.n_far; e0 += kChunk) {
                const int e1 = min(e0 + kChunk, P.n_far);
                for (int e = e0; e < e1; ++e) {
                    const int4 E = __ldg(reinterpret_cast<const int4 *>(ent + e));
                    int slot, pi;
                    source_cell(ax, ay, az, E.x, E.y, E.z, slot, pi);
                    const int row = s_row[slot];
                    T m0, dB[3] = {T(0), T(0), T(0)}, A2[6], A3[10];
                    if (row >= 0) {
                        load_source<T>(P, s_nbr[slot], row, pi, m0, dB, A2, A3);
                    } else {
                        m0 = W[base + E.w];
#pragma unroll
                        for (int q = 0; q < 6; ++q) A2[q] = T(0);
#pragma unroll
                        for (int q = 0; q < 10; ++q) A3[q] = T(0);
                    }
                    accumulate_mp<T, true>(dAx - dB[0] - T(E.x), dAy - dB[1] - T(E.y),
                                           dAz - dB[2] - T(E.z), m0, A2, A3, L, S1, S2);
                }
                L.flush();
            }
            // near sources: leaf cells only (the window holds 0 elsewhere)
            for (int e0 = P.n_far; e0 < P.n_far + P.n_near; e0 += kChunk) {
                const int e1 = min(e0 + kChunk, P.n_far + P.n_near);
                for (int e = e0; e < e1; ++e) {
                    const int4 E = __ldg(reinterpret_cast<const int4 *>(ent + e));
                    const T m0 = W[base + E.w];
                    accumulate_mp<T, false>(dAx - T(E.x), dAy - T(E.y), dAz - T(E.z), m0, nullptr,
                                            nullptr, L, S1, S2);
                }
                L.flush();
            }
            const int cell = ax + 8 * ay + 64 * az;
#pragma unroll
            for (int k = 0; k < 20; ++k) store_L<T>(P, node, k, cell, L.hi[k], L.lo[k]);
            // correction, finished in double:
            //   dL1_i = S1_i - (1/M0_A) sum_q A3_A,q S2_(i,q)
            const double m0A = double(mass[size_t(node) * NCELL + tpi]);
            double A3A[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) A3A[q] = double(own[(9 + q) * NCELL]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < 10; ++q) s += A3A[q] * double(S2[r4_of(i, q)]);
                P.dL1[(size_t(node) * 3 + i) * NCELL + cell] = double(S1[i]) - s / m0A;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- mono_kernel
// Leaf target, leaf sources: R = -o exactly, so L0 += c0(o) m and
// L1 += c1(o) m with per-offset weights c0 = -1/|o|, c1 = -o/|o|^3.
// Each pass takes NB sub-grids (consecutive in the cost-sorted queue), each
// with its own staged window; every thread holds two target cells (z and
// z+4 of one parity) per sub-grid, so each loaded weight feeds 2 NB cells.
template <typename T, int NB>
__device__ __forceinline__ void mono_entry(const T *W, int wstride, int base0, int base1,
                                           const StencilEntry *ent, const T *coef, int e,
                                           Acc<T, 4> (&A)[NB], Acc<T, 4> (&B)[NB])
{
    const int w = __ldg(&ent[e].woff);
    T c[4];
    if constexpr (sizeof(T) == 4) {
        const float4 cc = __ldg(reinterpret_cast<const float4 *>(coef) + e);
        c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
    } else {
        const double2 c01 = __ldg(reinterpret_cast<const double2 *>(coef) + 2 * e);
        const double2 c23 = __ldg(reinterpret_cast<const double2 *>(coef) + 2 * e + 1);
        c[0] = c01.x; c[1] = c01.y; c[2] = c23.x; c[3] = c23.y;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const T m0 = W[b * wstride + base0 + w];
        const T m1 = W[b * wstride + base1 + w];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            A[b].part[k] += c[k] * m0;
            B[b].part[k] += c[k] * m1;
        }
    }
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) mono_kernel(KParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *W = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_nbr[NB][27], s_leaf[NB][27], s_row[NB][27], s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz = lane >> 4;
    const StencilEntry *ent = P.stencil + p * P.ent_stride;
    const T *coef = static_cast<const T *>(P.coef) + size_t(p) * P.ent_stride * 4;
    const T *mass = static_cast<const T *>(P.mass);
    const int n_ent = P.n_far + P.n_near;
    const int wstride = 8 * P.sub_stride;
    const int base0 = cx + P.py * cy + P.pz * cz;
    const int base1 = base0 + 2 * P.pz;
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
            if (nodes[b] >= 0) stage_window<T>(W + b * wstride, s_nbr[b], s_leaf[b], mass, P);
        __syncthreads();
        Acc<T, 4> A[NB], B[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            A[b].zero();
            B[b].zero();
        }
        int e = 0;
        for (; e + kChunk <= n_ent; e += kChunk) {
#pragma unroll
            for (int j = 0; j < kChunk; ++j)
                mono_entry<T, NB>(W, wstride, base0, base1, ent, coef, e + j, A, B);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                A[b].flush();
                B[b].flush();
            }
        }
        for (; e < n_ent; ++e) mono_entry<T, NB>(W, wstride, base0, base1, ent, coef, e, A, B);
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
                store_L<T>(P, nodes[b], k, cell0, A[b].hi[k], A[b].lo[k]);
                store_L<T>(P, nodes[b], k, cell1, B[b].hi[k], B[b].lo[k]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                P.dL1[(size_t(nodes[b]) * 3 + i) * NCELL + cell0] = 0.0;
                P.dL1[(size_t(nodes[b]) * 3 + i) * NCELL + cell1] = 0.0;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ mx_kernel
// Leaf target, refined sources (monopole<-multipole): orders 0-1 and the
// correction S1 (the target has no third moment).  Adds to what mono_kernel
// stored for the same node, so it runs after it on the same stream.  Work
// items are node halves (z < 4, z >= 4); a host table gives, per parity,
// half and stencil entry, the neighbour slots its sources can fall in, so a
// warp skips (uniformly) every entry that cannot reach a refined neighbour.
template <typename T>
__global__ void __launch_bounds__(kThreads) mx_kernel(KParams P)
{
    __shared__ int s_nbr[27], s_leaf[27], s_row[27], s_item, s_mask;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = warp;
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    const int cx = lane & 3, cy = (lane >> 2) & 3, cz0 = lane >> 4;
    const StencilEntry *ent = P.stencil + p * P.ent_stride;
    const int n_ent = P.n_far + P.n_near;
    for (;;) {
        const int item = pull_item(P.counter, &s_item);
        if (item >= P.n_items) break;
        const int node = P.list[item >> 1];
        const int half = item & 1;
        load_slots(node, P, s_nbr, s_leaf, s_row);
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned bits = __ballot_sync(0xffffffffu, threadIdx.x < 27 && s_row[threadIdx.x] >= 0);
            if (threadIdx.x == 0) s_mask = int(bits);
        }
        __syncthreads();
        const int rmask = s_mask;
        const int32_t *smask = P.slot_mask + (size_t(p) * 2 + half) * P.ent_stride;
        const int cz = cz0 + 2 * half;
        const int ax = 2 * cx + px, ay = 2 * cy + py, az = 2 * cz + pz;
        Acc<T, 4> L;
        L.zero();
        T S1[3] = {T(0), T(0), T(0)};
        int done = 0;
        for (int e = 0; e < n_ent; ++e) {
            if (!(__ldg(&smask[e]) & rmask)) continue;
            const int4 E = __ldg(reinterpret_cast<const int4 *>(ent + e));
            int slot, pi;
            source_cell(ax, ay, az, E.x, E.y, E.z, slot, pi);
            const int row = s_row[slot];
            T m0 = T(0), dB[3] = {T(0), T(0), T(0)}, A2[6], A3[10];
#pragma unroll
            for (int q = 0; q < 6; ++q) A2[q] = T(0);
#pragma unroll
            for (int q = 0; q < 10; ++q) A3[q] = T(0);
            if (row >= 0) load_source<T>(P, s_nbr[slot], row, pi, m0, dB, A2, A3);
            DTensors<T, true> D;
            D.eval(-T(E.x) - dB[0], -T(E.y) - dB[1], -T(E.z) - dB[2]);
            T l0 = m0 * D.D0;
#pragma unroll
            for (int q = 0; q < 6; ++q) l0 += A2[q] * D.D2[q];
#pragma unroll
            for (int q = 0; q < 10; ++q) l0 -= A3[q] * D.D3[q];
            L.part[0] -= l0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T l1 = m0 * D.D1[i];
#pragma unroll
                for (int q = 0; q < 6; ++q) l1 += A2[q] * D.D3[r3_of(i, q)];
                L.part[1 + i] -= l1;
                T sacc = T(0);
#pragma unroll
                for (int q = 0; q < 10; ++q) sacc += A3[q] * D.D4[r4_of(i, q)];
                S1[i] += sacc;
            }
            if (++done == kChunk) {
                L.flush();
                done = 0;
            }
        }
        L.flush();
        const int cell = ax + 8 * ay + 64 * az;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const size_t idx = (size_t(node) * NCOMP + k) * NCELL + cell;
            if constexpr (sizeof(T) == 4) {
                float *Lh = static_cast<float *>(P.L);
                float s, e;
                two_sum(Lh[idx], L.hi[k], s, e);
                const float lo = P.Lc[idx] + L.lo[k] + e;
                const float s2 = s + lo;
                Lh[idx] = s2;
                P.Lc[idx] = lo - (s2 - s);
            } else {
                static_cast<double *>(P.L)[idx] += L.hi[k];
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) P.dL1[(size_t(node) * 3 + i) * NCELL + cell] = double(S1[i]);
        __syncthreads();
    }
}

// ---------------------------------------------------------- root_kernel
// Level 1 holds one node per tree and every pair is a candidate: a refined
// root evaluates its well-separated pairs, a leaf root all pairs.  The
// 512 x 511 pairs of one root are spread over 16 CTAs of 32 targets, each
// target's 512 sources over 4 warps; the 4 partial sums are folded in a
// fixed order (deterministic).
constexpr int kRootSlices = 4;
constexpr int kRootThreads = 32 * kRootSlices;
constexpr int kRootGroups = NCELL / 32;

template <typename T>
__global__ void __launch_bounds__(kRootThreads) root_kernel(KParams P)
{
    constexpr int NV = 20 + 3 + 15;                 // L, S1, S2
    __shared__ T sh_hi[kRootSlices][NV][32];
    __shared__ T sh_lo[kRootSlices][sizeof(T) == 4 ? 20 : 1][32];   // float only
    const int node = P.list[blockIdx.x];
    const NodeInfo ti = P.info[node];
    const bool leaf = ti.leaf_row >= 0;
    const T *mass = static_cast<const T *>(P.mass);
    const T *mpd = static_cast<const T *>(P.mp);
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int cell = blockIdx.y * 32 + lane;
    const int ax = cell & 7, ay = (cell >> 3) & 7, az = cell >> 6;
    const int tpi = parity_index(ax, ay, az);
    T dA[3] = {T(0), T(0), T(0)};
    if (!leaf)
        for (int a = 0; a < 3; ++a) dA[a] = mpd[(size_t(ti.mp_row) * NMP + a) * NCELL + tpi];
    Acc<T, 20> L;
    L.zero();
    T S1[3] = {T(0), T(0), T(0)}, S2[15];
    for (int q = 0; q < 15; ++q) S2[q] = T(0);
    int done = 0;
    const int b0 = slice * (NCELL / kRootSlices);
    for (int b = b0; b < b0 + NCELL / kRootSlices; ++b) {
        const int ox = (b & 7) - ax, oy = ((b >> 3) & 7) - ay, oz = (b >> 6) - az;
        const double o2 = double(ox * ox + oy * oy + oz * oz);
        const bool far = P.theta2 * o2 > 1.0;
        if (b == cell || !(far || leaf)) continue;
        const int pi = parity_index(b & 7, (b >> 3) & 7, b >> 6);
        T m0, dB[3] = {T(0), T(0), T(0)}, A2[6], A3[10];
        for (int q = 0; q < 6; ++q) A2[q] = T(0);
        for (int q = 0; q < 10; ++q) A3[q] = T(0);
        if (!leaf) load_source<T>(P, node, ti.mp_row, pi, m0, dB, A2, A3);
        else m0 = mass[size_t(node) * NCELL + pi];
        accumulate_mp<T, true>(dA[0] - dB[0] - T(ox), dA[1] - dB[1] - T(oy), dA[2] - dB[2] - T(oz),
                               m0, A2, A3, L, S1, S2);
        if (++done == kChunk) {
            L.flush();
            done = 0;
        }
    }
    L.flush();
    for (int k = 0; k < 20; ++k) {
        sh_hi[slice][k][lane] = L.hi[k];
        if constexpr (sizeof(T) == 4) sh_lo[slice][k][lane] = L.lo[k];
    }
    for (int i = 0; i < 3; ++i) sh_hi[slice][20 + i][lane] = S1[i];
    for (int q = 0; q < 15; ++q) sh_hi[slice][23 + q][lane] = S2[q];
    __syncthreads();
    if (slice != 0) return;
    const int nk = leaf ? 4 : 20;
    for (int k = 0; k < nk; ++k) {
        T hi = T(0), lo = T(0);
        for (int sl = 0; sl < kRootSlices; ++sl) {
            if constexpr (sizeof(T) == 4) {
                float sum, err;
                two_sum(hi, sh_hi[sl][k][lane], sum, err);
                hi = sum;
                lo += err + sh_lo[sl][k][lane];
            } else {
                hi += sh_hi[sl][k][lane];
            }
        }
        store_L<T>(P, node, k, cell, hi, lo);
    }
    double s1[3] = {0.0, 0.0, 0.0}, s2[15];
    for (int q = 0; q < 15; ++q) s2[q] = 0.0;
    for (int sl = 0; sl < kRootSlices; ++sl) {
        for (int i = 0; i < 3; ++i) s1[i] += double(sh_hi[sl][20 + i][lane]);
        for (int q = 0; q < 15; ++q) s2[q] += double(sh_hi[sl][23 + q][lane]);
    }
    double corr[3] = {s1[0], s1[1], s1[2]};
    if (!leaf) {
        const double m0A = double(mass[size_t(node) * NCELL + tpi]);
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int q = 0; q < 10; ++q)
                acc += double(mpd[(size_t(ti.mp_row) * NMP + 9 + q) * NCELL + tpi]) * s2[r4_of(i, q)];
            corr[i] -= acc / m0A;
        }
    }
    for (int i = 0; i < 3; ++i) P.dL1[(size_t(node) * 3 + i) * NCELL + cell] = corr[i];
}

// ---------------------------------------------------------- launching
template <typename T>
struct Kernels {
    static cudaError_t configure(size_t window_bytes)
    {
        static size_t done_bytes = 0;
        if (done_bytes >= window_bytes) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(mp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(window_bytes))) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(mono_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(window_bytes))) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(mono_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(2 * window_bytes))) != cudaSuccess)
            return e;
        if (sizeof(T) == 4 &&
            (e = cudaFuncSetAttribute(mono_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(4 * window_bytes))) != cudaSuccess)
            return e;
        done_bytes = window_bytes;
        return cudaSuccess;
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

template <typename T, int NB>
cudaError_t launch_mono(const KParams &K, size_t wbytes, int sms, int cap, cudaStream_t s)
{
    const int64_t passes = (K.n_items + NB - 1) / NB;
    const int g = persistent_grid(mono_kernel<T, NB>, NB * wbytes, passes, sms, cap);
    mono_kernel<T, NB><<<g, kThreads, NB * wbytes, s>>>(K);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_all(const fmm_tree_s *t, void *L, float *Lc, double *dL1, cudaStream_t s,
                       int *n_launches)
{
    const Plan &Pl = t->plan;
    const DeviceTables &d = t->dev;
    KParams P{};
    P.info = d.info;
    P.nbr = d.nbr;
    P.stencil = d.stencil;
    P.coef = sizeof(T) == 4 ? static_cast<const void *>(d.coef32) : static_cast<const void *>(d.coef64);
    P.n_far = Pl.n_far[0];
    P.n_near = Pl.n_near[0];
    P.ent_stride = Pl.ent_stride;
    P.reach = Pl.reach;
    P.py = Pl.py;
    P.pz = Pl.pz;
    P.sub_stride = Pl.sub_stride;
    P.mass = d.mass;
    P.mp = d.mp;
    P.L = L;
    P.Lc = Lc;
    P.dL1 = dL1;
    P.theta2 = t->cfg.theta * t->cfg.theta;
    P.slot_mask = d.slot_mask;
    const int cap = t->tuning.ctas_per_sm;
    const size_t wbytes = size_t(8) * Pl.sub_stride * sizeof(T);
    cudaError_t e = Kernels<T>::configure(wbytes);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d.counters, 0, 4 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int sms = sm_count_of_current_device();
    int nl = 0;
    if (Pl.roots.count) {
        KParams R = P;
        R.list = d.lists + Pl.roots.off;
        R.n_items = int32_t(Pl.roots.count);
        timing_begin(t, FMM_K_ROOT, s);
        root_kernel<T><<<dim3(unsigned(Pl.roots.count), kRootGroups), kRootThreads, 0, s>>>(R);
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (Pl.work_mp.count) {
        KParams K = P;
        K.list = d.lists + Pl.work_mp.off;
        K.n_items = int32_t(Pl.work_mp.count);
        K.counter = d.counters + Q_MP;
        int g = persistent_grid(mp_kernel<T>, wbytes, Pl.work_mp.count, sms, cap);
        timing_begin(t, FMM_K_MULTIPOLE, s);
        mp_kernel<T><<<g, kThreads, wbytes, s>>>(K);
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (Pl.work_mono.count) {
        KParams K = P;
        K.list = d.lists + Pl.work_mono.off;
        K.n_items = int32_t(Pl.work_mono.count);
        K.counter = d.counters + Q_MONO;
        int nb = t->tuning.mono_subgrids;
        if (nb != 1 && nb != 2 && nb != 4) nb = sizeof(T) == 4 ? 2 : 1;
        if (sizeof(T) != 4 && nb == 4) nb = 2;
        timing_begin(t, FMM_K_MONOPOLE, s);
        e = nb == 1 ? launch_mono<T, 1>(K, wbytes, sms, cap, s)
            : nb == 2 ? launch_mono<T, 2>(K, wbytes, sms, cap, s)
                      : launch_mono<T, sizeof(T) == 4 ? 4 : 2>(K, wbytes, sms, cap, s);
        timing_end(t, s);
        ++nl;
        if (e != cudaSuccess) return e;
    }
    if (Pl.work_mx.count) {
        KParams K = P;
        K.list = d.lists + Pl.work_mx.off;
        K.n_items = int32_t(2 * Pl.work_mx.count);       // node halves
        K.counter = d.counters + Q_MX;
        int g = persistent_grid(mx_kernel<T>, 0, K.n_items, sms, cap);
        timing_begin(t, FMM_K_MONO_MULTI, s);
        mx_kernel<T><<<g, kThreads, 0, s>>>(K);
        timing_end(t, s);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_launches) *n_launches = nl;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_pack(const fmm_tree_s *t, const double *M, const double *com, cudaStream_t s)
{
    const auto &c = t->cfg;
    if (c.precision == FMM_MIXED)
        pack_kernel<float><<<unsigned(t->n), 512, 0, s>>>(
            t->dev.info, t->dev.levels, M, com, static_cast<float *>(t->dev.mass),
            static_cast<float *>(t->dev.mp), c.box_lo[0], c.box_lo[1], c.box_lo[2]);
    else
        pack_kernel<double><<<unsigned(t->n), 512, 0, s>>>(
            t->dev.info, t->dev.levels, M, com, static_cast<double *>(t->dev.mass),
            static_cast<double *>(t->dev.mp), c.box_lo[0], c.box_lo[1], c.box_lo[2]);
    return cudaGetLastError();
}

cudaError_t launch_m2l(const fmm_tree_s *t, void *L, float *Lc, double *dL1, cudaStream_t s,
                       int *n_launches)
{
    if (t->cfg.precision == FMM_MIXED) return launch_all<float>(t, L, Lc, dL1, s, n_launches);
    return launch_all<double>(t, L, Lc, dL1, s, n_launches);
}

}  // namespace fmm
