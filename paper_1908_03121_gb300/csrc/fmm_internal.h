// Internal declarations of the GB300 FMM library (not part of the C ABI).
//
// Layouts used inside the library, beyond the caller-visible ones described
// in include/fmm_gb300.h:
//   - "parity-split" cell order inside a node: cell (x,y,z) sits at
//       ((x&1) + 2(y&1) + 4(z&1)) * 64 + (x>>1) + 4(y>>1) + 16(z>>1),
//     so the 64 cells of one parity class (which share one stencil) are
//     contiguous;
//   - packed same-level source data (workspace), in level units:
//       mass[node][512]            cell mass (all nodes)
//       mp[mp_row][4][512][4]      refined nodes only, four groups of four:
//                                  (centre-of-mass offset from the cell
//                                  centre in cell widths, M0), then the traceless
//                                  projections B2 (5) and B3 (7) of
//                                  A2 = mult * M2 / (2 h^2), A3 = mult * M3 / (6 h^3)
//     where mult is the number of index permutations of a symmetric
//     component (so full-tensor contractions become plain dot products).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fmm_gb300.h"

namespace fmm {

constexpr int NSIDE = 8;
constexpr int NCELL = 512;
constexpr int NCOMP = 20;
constexpr int NMP = 16;          // packed same-level values per refined cell
constexpr int kReduceRows = 1024;   // leaf rows per CTA of the first force-sum stage

// pad a pitch up to the next value congruent to want (mod 32): the halo
// window's row and plane pitches, chosen so that the 32 lanes of a warp hit
// distinct shared-memory banks
__host__ __device__ constexpr int pad_to(int min_value, int want)
{
    int v = min_value;
    while (((v % 32) + 32) % 32 != want) ++v;
    return v;
}

// per-level geometry table (device, [level][LEVEL_FIELDS] doubles), filled on
// the host so that no kernel divides: h, 1/h, h^3, the level-unit ->
// physical scales G h^-(n+1) of orders n = 0..3 and their inverses
constexpr int LEVEL_FIELDS = 12;
enum { LV_H = 0, LV_IH, LV_H3, LV_S0, LV_S1, LV_S2, LV_S3, LV_R0, LV_R1, LV_R2, LV_R3 };
// the same h, inverse scales R0..R3 and scales S0..S3 as double-float
// (hi, lo) pairs, [level][LEVEL_DF_FIELDS][2] floats
constexpr int LEVEL_DF_FIELDS = 9;

// per-node table row (device and host)
struct NodeInfo {
    int32_t level, ix, iy, iz;
    int32_t parent;
    int32_t leaf_row;    // density / potential row, -1 for refined nodes
    int32_t mp_row;      // row in the packed multipole workspace, -1 for leaves
    int32_t tree;
};

// stencil entry of one parity class; far entries come first
struct StencilEntry {
    int32_t ox, oy, oz;  // source offset in cell widths
    int32_t woff;        // offset inside the parity-split halo window
};

struct DeviceTables {
    NodeInfo *info = nullptr;        // [n]
    int32_t *children = nullptr;     // [n][8]
    int32_t *nbr = nullptr;          // [n][27], slot (dx+1)+3(dy+1)+9(dz+1)
    int32_t *lists = nullptr;        // all node-index lists, see Plan offsets
    StencilEntry *stencil = nullptr; // [8][ent_stride]
    float *stencil_f = nullptr;      // [8][ent_stride][4] the same entries with the offset
                                     // as floats (window offset's int bits in the fourth)
    float *coef32 = nullptr;         // [ent_stride][4] monopole weights of parity 0
    double *coef64 = nullptr;        // [ent_stride][4]
    float *coefdf = nullptr;         // [ent_stride][4][hi, lo]
    int32_t *mono_woff = nullptr;    // [8][ent_stride] window offsets, parity 0's order reflected
    int32_t *tree_leaf_off = nullptr;   // [n_trees + 1]
    int32_t *tree_leaf_rows = nullptr;  // [n_leaf]
    double *levels = nullptr;        // [max_level + 1][LEVEL_FIELDS]
    float *levels_df = nullptr;      // [max_level + 1][LEVEL_DF_FIELDS][2]
    int4 *mx_targets = nullptr;      // monopole<-multipole targets (node, cell, warp base, count)
    int2 *mx_pairs = nullptr;        // their pairs (packed-moment offset, stencil entry),
                                     // interleaved by warp (fmm_tree_s::mx_pairs)
    // workspace
    void *mass = nullptr;            // [n][512] float or double
    void *mp = nullptr;              // [n_refined][4][512][4] packed sources: float,
                                     // double-float pairs or double
    int32_t *counters = nullptr;     // work-queue heads; [kStatusSlot]: FMM_STATUS_* bits
    double *partials = nullptr;      // [n_leaf][8]
    double *chunk_sums = nullptr;    // [n_trees][reduce_chunks][8]
    float *up = nullptr;             // mixed, dfloat: [n_refined][20][512] double-float
                                     // (hi, lo) results of the upward pass per refined cell
    int32_t *dflow_items = nullptr;  // dataflow downward queue: refined (node, slice) items
                                     // node * 8 + slice, root level first, then leaf nodes
                                     // by level
    int32_t *dflow_ready = nullptr;  // [n]: slices of the node's shift completed this step
    float *down = nullptr;           // mixed and double-float: [n_refined][23][512]
                                     // (hi, lo) pairs of each refined cell's final
                                     // expansion (20) and centre-of-mass offset from
                                     // its centre (3)
    size_t workspace_bytes = 0;
};

// offsets of the node lists inside DeviceTables::lists
// the slot of DeviceTables::counters that holds the status word (the work
// queues use slots 0-3, which every step resets)
constexpr int kStatusSlot = 8;
// the dataflow downward pass's queue head and abort flag (reset every step)
constexpr int kDflowHeadSlot = 16;
constexpr int kDflowAbortSlot = 17;
// default budget of one device-side wait of the dataflow pass
constexpr long long kDefaultWaitBudgetNs = 1000000000ll;

struct ListRange {
    int64_t off = 0, count = 0;
};

struct Plan {
    // window geometry
    int reach = 5;                   // largest per-axis offset
    int far_o2 = 5;                  // smallest well-separated squared offset
    int reduce_chunks = 1;           // leaf-row chunks per tree of the force sums
    int sub = 9;                     // parity sub-window edge = 4 + reach
    int py = 12, pz = 112;           // padded pitches of a sub-window
    int sub_stride = 1008;           // elements per sub-window
    int n_far[8] = {0}, n_near[8] = {0};
    int ent_stride = 0;              // entries reserved per parity
    int64_t stencil_union = 0;
    // node lists
    ListRange leaves;                // all leaf nodes (P2M, forces)
    std::vector<ListRange> refined_at;   // [level] refined nodes (M2M)
    std::vector<ListRange> leafkids_at;  // [level] refined nodes whose 8 children are leaves
    std::vector<ListRange> mixedkids_at; // [level] the other refined nodes
    std::vector<ListRange> nodes_at;     // [level] all nodes (L2L)
    ListRange work_mp, work_mono, work_mx, roots;
    ListRange refined;                    // every refined node (roots included)
    int64_t n_mx_targets = 0;             // leaf cells with refined sources
    int64_t dflow_refined_items = 0;      // refined (node, slice) items of the dataflow queue
    int64_t dflow_items = 0;              // all its items (the leaf nodes after them)
    int64_t interactions[4] = {0, 0, 0, 0};
    int64_t kernel_interactions[4] = {0, 0, 0, 0};  // multipole, monopole, mono<-multi, root
};

}  // namespace fmm

namespace fmm {
// event pairs around timed launches (FMM_FLAG_TIMING)
struct TimerState {
    std::vector<cudaEvent_t> ev;     // 2 per record
    std::vector<int> slot;           // kernel slot per record
    int used = 0;
    int open_slot = -1;
    double ms[16] = {0};
    int64_t launches[16] = {0};
};
}  // namespace fmm

struct fmm_tree_s {
    fmm_config cfg;
    int64_t n = 0, n_leaf = 0, n_refined = 0;
    int32_t n_trees = 0, max_level = 0;
    std::vector<fmm::NodeInfo> info;
    std::vector<int32_t> children, nbr, lists;
    std::vector<fmm::StencilEntry> stencil;
    std::vector<float> stencil_f;
    std::vector<float> coef32;
    std::vector<double> coef64;
    std::vector<float> coefdf;
    std::vector<int32_t> mono_woff;
    std::vector<int32_t> tree_leaf_off, tree_leaf_rows;
    std::vector<double> levels;
    std::vector<float> levels_df;
    std::vector<int32_t> mx_targets;     // [n_mx_targets][4]: node, cell, the warp's pair base, count
    std::vector<int32_t> mx_pairs;       // [slots][2]: packed-moment offset, stencil entry; pair k
                                         // of target 32 w + j at base_w + 32 k + j
    std::vector<int32_t> dflow_items;    // the dataflow downward queue (DeviceTables)
    fmm::Plan plan;
    fmm_tuning tuning{};
    bool host_only = false;
    int device = -1;
    fmm::DeviceTables dev;
    mutable fmm::TimerState timer;
    // fmm_step's second stream and its fork/join events (device trees only)
    cudaStream_t aux = nullptr;
    cudaEvent_t step_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace fmm {

// kernels (each returns a cudaError_t from the launch)
// pack_leaves: also store the leaf masses in the same-level pass's packed
// form (what launch_pack does for the leaves)
cudaError_t launch_p2m(const fmm_tree_s *t, const double *rho, double *M, cudaStream_t s,
                       bool pack_leaves = false);
cudaError_t launch_m2m_level(const fmm_tree_s *t, int level, double *M, double *com,
                             cudaStream_t s);
// which nodes a pack launch covers
enum { PACK_ALL = 0, PACK_LEAVES = 1, PACK_REFINED = 2 };
cudaError_t launch_pack(const fmm_tree_s *t, const double *M, const double *com,
                        cudaStream_t s, int which = PACK_ALL);
// parts of the same-level pass (bits; M2L_ALL = all, counters reset first)
// M2L_MPX: the multipole launch also takes the monopole<-multipole targets
// (after its own queue; the monopole kernel must have finished)
enum { M2L_RESET = 1, M2L_ROOT = 2, M2L_MP = 4, M2L_MONO = 8, M2L_MX = 16, M2L_ALL = 31,
       M2L_MPX = 32 };
cudaError_t launch_m2l(const fmm_tree_s *t, void *L, float *Lc, double *dL1,
                       cudaStream_t s, int *n_launches, int parts = M2L_ALL);
cudaError_t launch_l2l_level(const fmm_tree_s *t, int level, const void *L,
                             const float *Lc, const double *dL1, const double *com,
                             double *L64, double *dacc, cudaStream_t s);
cudaError_t launch_l2l_nodes(const fmm_tree_s *t, const ListRange &r, const void *L,
                             const float *Lc, const double *dL1, const double *com,
                             double *L64, double *dacc, cudaStream_t s);
cudaError_t launch_leaf_finish(const fmm_tree_s *t, const void *L, const float *Lc,
                               const double *dL1, const double *com, double *L64, double *dacc,
                               const double *M, double *phi, double *g, cudaStream_t s);
cudaError_t launch_force_sums(const fmm_tree_s *t, double *totals, cudaStream_t s);
// the refined levels' shifts and every leaf's shift and forces in one
// persistent launch ordered by per-node readiness counters
cudaError_t launch_downward_dataflow(const fmm_tree_s *t, const void *L, const float *Lc,
                                     const double *dL1, const double *com, double *L64,
                                     double *dacc, const double *M, double *phi, double *g,
                                     cudaStream_t s);
cudaError_t launch_forces(const fmm_tree_s *t, const double *L64, const double *dacc,
                          const double *rho, double *phi, double *g, double *totals,
                          cudaStream_t s);

int sm_count_of_current_device();
size_t max_smem_optin_of_current_device();

// set the calling thread's fmm_last_error() message
void record_error(const std::string &msg);

// FMM_FLAG_TIMING hooks around one kernel launch (no-ops otherwise)
void timing_begin(const fmm_tree_s *t, int slot, cudaStream_t s);
void timing_end(const fmm_tree_s *t, cudaStream_t s);

}  // namespace fmm
