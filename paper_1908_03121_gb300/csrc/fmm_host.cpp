// Host side of the C ABI: descriptor validation, planning (neighbour tables,
// per-parity stencils of the opening rule, level schedules, cost-sorted work
// lists, exact interaction counts), device upload and launch sequencing.
//
// Method: Octo-Tiger's cell-based FMM (arXiv 1908.03121, Sec. 4.3).  The
// opening rule gives every cell of a level the same set of same-level
// partners ("constant on each level", Sec. 4.3), which is why it can be
// tabulated once per child parity and applied as a stencil.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <unordered_map>

#include "fmm_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(FMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline int64_t floordiv2(int64_t v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

// node key inside one tree
inline uint64_t node_key(int level, int64_t ix, int64_t iy, int64_t iz)
{
    return (uint64_t(level) << 60) | (uint64_t(ix) << 40) | (uint64_t(iy) << 20) | uint64_t(iz);
}

bool well_separated(double theta, int64_t ox, int64_t oy, int64_t oz)
{
    double o2 = double(ox * ox + oy * oy + oz * oz);
    return theta * theta * o2 > 1.0;
}

// pad a pitch up to the next value congruent to want (mod 32)

// Monopole-monopole coefficients of one offset o (target minus source
// position is -o cell widths): L0 += c0 m, L1 += c1 m in level units.
void mono_coef(int ox, int oy, int oz, double c[4])
{
    double r2 = double(ox * ox + oy * oy + oz * oz);
    double r = std::sqrt(r2);
    double ir3 = 1.0 / (r2 * r);
    c[0] = -1.0 / r;
    c[1] = -ox * ir3;
    c[2] = -oy * ir3;
    c[3] = -oz * ir3;
}

}  // namespace

namespace fmm {

void record_error(const std::string &msg) { g_last_error = msg; }

int sm_count_of_current_device()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

size_t max_smem_optin_of_current_device()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 48 * 1024;
    return size_t(n);
}

static void timing_fold(const fmm_tree_s *t)
{
    TimerState &T = t->timer;
    if (T.used == 0) return;
    cudaEventSynchronize(T.ev[size_t(2 * T.used - 1)]);
    for (int i = 0; i < T.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, T.ev[size_t(2 * i)], T.ev[size_t(2 * i + 1)]) == cudaSuccess) {
            T.ms[T.slot[size_t(i)]] += ms;
            T.launches[T.slot[size_t(i)]]++;
        }
    }
    T.used = 0;
}

void timing_begin(const fmm_tree_s *t, int slot, cudaStream_t s)
{
    if (!(t->cfg.flags & FMM_FLAG_TIMING)) return;
    TimerState &T = t->timer;
    if (2 * T.used + 2 > int(T.ev.size())) timing_fold(t);
    cudaEventRecord(T.ev[size_t(2 * T.used)], s);
    T.slot[size_t(T.used)] = slot;
    T.open_slot = slot;
}

void timing_end(const fmm_tree_s *t, cudaStream_t s)
{
    if (!(t->cfg.flags & FMM_FLAG_TIMING)) return;
    TimerState &T = t->timer;
    if (T.open_slot < 0) return;
    cudaEventRecord(T.ev[size_t(2 * T.used + 1)], s);
    T.used++;
    T.open_slot = -1;
}

}  // namespace fmm

using namespace fmm;

static int validate_config(const fmm_config *cfg)
{
    if (!(cfg->theta > 0.25 && cfg->theta <= 1.0 / std::sqrt(3.0) + 1e-12))
        return fail(FMM_ERR_INVALID_ARG,
                    "theta must lie in (0.25, 1/sqrt(3)]: sources within the 26 neighbour "
                    "nodes and each leaf pair evaluated once");
    if (!(cfg->box_size > 0.0) || !std::isfinite(cfg->box_size))
        return fail(FMM_ERR_INVALID_ARG, "box_size must be positive and finite");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(cfg->box_lo[a])) return fail(FMM_ERR_INVALID_ARG, "box_lo not finite");
    if (!std::isfinite(cfg->G)) return fail(FMM_ERR_INVALID_ARG, "G not finite");
    if (cfg->precision != FMM_FP64 && cfg->precision != FMM_MIXED && cfg->precision != FMM_DFLOAT)
        return fail(FMM_ERR_INVALID_ARG, "precision must be FMM_FP64, FMM_MIXED or FMM_DFLOAT");
    if (cfg->max_level < 1 || cfg->max_level > 20)
        return fail(FMM_ERR_INVALID_ARG, "max_level must lie in 1..20");
    if (cfg->order != 0 && cfg->order != 2 && cfg->order != 3)
        return fail(FMM_ERR_INVALID_ARG, "order must be 2 or 3 (0 selects 3)");
    return FMM_OK;
}

// ------------------------------------------------------------ validation
static int validate_nodes(const fmm_node_desc *d, int64_t n, const fmm_config *cfg,
                          fmm_tree_s *t, std::vector<std::unordered_map<uint64_t, int32_t>> &maps)
{
    int32_t max_tree = -1;
    for (int64_t i = 0; i < n; ++i) {
        const fmm_node_desc &x = d[i];
        if (x.level < 1 || x.level > cfg->max_level)
            return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": level outside 1..max_level");
        int64_t side = int64_t(1) << (x.level - 1);
        if (x.ix < 0 || x.iy < 0 || x.iz < 0 || x.ix >= side || x.iy >= side || x.iz >= side)
            return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": coordinates outside its level");
        if (x.tree_id < 0 || x.tree_id >= n)
            return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": tree_id out of range");
        max_tree = std::max(max_tree, x.tree_id);
    }
    t->n_trees = max_tree + 1;
    maps.assign(size_t(t->n_trees), {});
    std::vector<int> roots(size_t(t->n_trees), 0);
    for (int64_t i = 0; i < n; ++i) {
        const fmm_node_desc &x = d[i];
        auto &m = maps[size_t(x.tree_id)];
        auto ins = m.emplace(node_key(x.level, x.ix, x.iy, x.iz), int32_t(i));
        if (!ins.second)
            return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": duplicate of node " +
                                          std::to_string(ins.first->second));
        if (x.level == 1) {
            if (x.parent != -1) return fail(FMM_ERR_TREE, "root node with a parent");
            roots[size_t(x.tree_id)]++;
        } else {
            if (x.parent < 0 || x.parent >= n)
                return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": parent out of range");
            const fmm_node_desc &p = d[x.parent];
            if (p.level != x.level - 1 || p.tree_id != x.tree_id)
                return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": parent level/tree mismatch");
            if (p.ix != x.ix / 2 || p.iy != x.iy / 2 || p.iz != x.iz / 2)
                return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": not inside its parent");
            int k = (x.ix & 1) + 2 * (x.iy & 1) + 4 * (x.iz & 1);
            if (p.child[k] != i)
                return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": parent does not list it");
        }
        int nchild = 0;
        for (int k = 0; k < 8; ++k) nchild += x.child[k] >= 0;
        if (nchild != 0 && nchild != 8)
            return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": partially refined");
        for (int k = 0; k < 8 && nchild; ++k) {
            int32_t c = x.child[k];
            if (c >= n) return fail(FMM_ERR_TREE, "child index out of range");
            const fmm_node_desc &ch = d[c];
            if (ch.parent != i || ch.level != x.level + 1 || ch.ix != 2 * x.ix + (k & 1) ||
                ch.iy != 2 * x.iy + ((k >> 1) & 1) || ch.iz != 2 * x.iz + ((k >> 2) & 1))
                return fail(FMM_ERR_TREE, "node " + std::to_string(i) + ": inconsistent child " +
                                              std::to_string(k));
        }
    }
    for (int32_t tr = 0; tr < t->n_trees; ++tr)
        if (roots[size_t(tr)] != 1)
            return fail(FMM_ERR_TREE, "tree " + std::to_string(tr) + " does not have exactly one root");
    return FMM_OK;
}

// ------------------------------------------------------------- stencils
// Per child parity p: all offsets o whose parent offset floor((p+o)/2) is
// not well separated, split into well-separated (far) and near offsets, each
// in lexicographic order (neighbouring warps then walk the halo in the same
// spatial order, which keeps the multipole kernel's source reads in L1).
// Reflecting o along the axes where p is odd maps parity 0's stencil onto
// parity p's (floor((1+o)/2) = -floor(-o/2), and both tests depend on |.|
// only); the monopole kernel walks every parity in parity 0's order,
// reflected, so that one weight table (parity 0's) serves all parities, and
// gets its own table of window offsets in that order.
static void build_stencils(fmm_tree_s *t)
{
    Plan &P = t->plan;
    double theta = t->cfg.theta;
    int R = 2 * int(std::floor(1.0 / theta)) + 1;
    P.reach = R;
    P.sub = 4 + R;
    P.py = pad_to(P.sub, 12);
    P.pz = pad_to(P.sub * P.py, 16);
    P.sub_stride = P.sub * P.pz;
    auto in_stencil = [&](const int pp[3], const int o[3]) {
        int64_t po[3];
        for (int a = 0; a < 3; ++a) po[a] = floordiv2(pp[a] + o[a]);
        return !well_separated(theta, po[0], po[1], po[2]);
    };
    // window offset of the source relative to the lane base
    auto entry = [&](const int pp[3], int ox, int oy, int oz) {
        const int o[3] = {ox, oy, oz};
        int u[3], q = 0;
        for (int a = 0; a < 3; ++a) {
            u[a] = pp[a] + o[a] + R;       // >= 0
            q |= (u[a] & 1) << a;
        }
        const int woff = q * P.sub_stride + (u[0] >> 1) + P.py * (u[1] >> 1) + P.pz * (u[2] >> 1);
        return StencilEntry{ox, oy, oz, woff};
    };
    std::vector<char> in_union(size_t(2 * R + 1) * (2 * R + 1) * (2 * R + 1), 0);
    std::vector<StencilEntry> lists[8];
    for (int p = 0; p < 8; ++p) {
        const int pp[3] = {p & 1, (p >> 1) & 1, (p >> 2) & 1};
        std::vector<StencilEntry> far, nearv;
        for (int oz = -R; oz <= R; ++oz)
            for (int oy = -R; oy <= R; ++oy)
                for (int ox = -R; ox <= R; ++ox) {
                    if (!ox && !oy && !oz) continue;
                    const int o[3] = {ox, oy, oz};
                    if (!in_stencil(pp, o)) continue;
                    (well_separated(theta, ox, oy, oz) ? far : nearv).push_back(entry(pp, ox, oy, oz));
                    in_union[size_t((oz + R) * (2 * R + 1) + (oy + R)) * (2 * R + 1) + (ox + R)] = 1;
                }
        P.n_far[p] = int(far.size());
        P.n_near[p] = int(nearv.size());
        lists[p] = far;
        lists[p].insert(lists[p].end(), nearv.begin(), nearv.end());
    }
    // the kernels rely on every parity having the same far/near counts
    // (the reflection above maps one parity's stencil onto another's)
    for (int p = 1; p < 8; ++p)
        if (P.n_far[p] != P.n_far[0] || P.n_near[p] != P.n_near[0]) std::abort();
    int stride = 0;
    for (int p = 0; p < 8; ++p) stride = std::max(stride, int(lists[p].size()));
    P.ent_stride = (stride + 3) & ~3;
    t->stencil.assign(size_t(8) * P.ent_stride, StencilEntry{0, 0, 0, 0});
    for (int p = 0; p < 8; ++p)
        for (size_t k = 0; k < lists[p].size(); ++k) t->stencil[size_t(p) * P.ent_stride + k] = lists[p][k];
    t->stencil_f.assign(t->stencil.size() * 4, 0.f);
    for (size_t i = 0; i < t->stencil.size(); ++i) {
        const StencilEntry &e = t->stencil[i];
        t->stencil_f[4 * i] = float(e.ox);
        t->stencil_f[4 * i + 1] = float(e.oy);
        t->stencil_f[4 * i + 2] = float(e.oz);
        std::memcpy(&t->stencil_f[4 * i + 3], &e.woff, sizeof(float));
    }
    // monopole kernel: parity 0's weights, every parity in parity 0's order
    t->coef32.assign(size_t(P.ent_stride) * 4, 0.f);
    t->coef64.assign(size_t(P.ent_stride) * 4, 0.0);
    t->coefdf.assign(size_t(P.ent_stride) * 8, 0.f);
    t->mono_woff.assign(size_t(8) * P.ent_stride, 0);
    for (size_t k = 0; k < lists[0].size(); ++k) {
        const StencilEntry &e = lists[0][k];
        double c[4];
        mono_coef(e.ox, e.oy, e.oz, c);
        for (int j = 0; j < 4; ++j) {
            t->coef64[k * 4 + j] = c[j];
            t->coef32[k * 4 + j] = float(c[j]);
            // double-float (hi, lo) pairs
            t->coefdf[k * 8 + 2 * j] = float(c[j]);
            t->coefdf[k * 8 + 2 * j + 1] = float(c[j] - double(float(c[j])));
        }
        for (int p = 0; p < 8; ++p) {
            const int pp[3] = {p & 1, (p >> 1) & 1, (p >> 2) & 1};
            const int o[3] = {pp[0] ? -e.ox : e.ox, pp[1] ? -e.oy : e.oy, pp[2] ? -e.oz : e.oz};
            // the reflected entry is in parity p's stencil, on the same side
            // of the far/near split
            if (!in_stencil(pp, o) ||
                well_separated(theta, o[0], o[1], o[2]) != (int(k) < P.n_far[0]))
                std::abort();
            t->mono_woff[size_t(p) * P.ent_stride + k] = entry(pp, o[0], o[1], o[2]).woff;
        }
    }
    P.stencil_union = 0;
    for (char c : in_union) P.stencil_union += c;
    // the opening test on an integer squared offset n, as a threshold: the
    // smallest n that is well separated (kernels compare integers only)
    // (the same expression as well_separated on o2 = far_o2)
    P.far_o2 = 1;
    while (!(theta * theta * double(P.far_o2) > 1.0)) ++P.far_o2;
}

// --------------------------------------------------- interaction counting
// For every parity, far/near list and neighbour slot, the number of
// (target cell, entry) pairs whose source falls into that slot.
static void slot_tables(const fmm_tree_s *t, std::vector<int64_t> &tab)
{
    const Plan &P = t->plan;
    tab.assign(size_t(8) * 2 * 27, 0);
    for (int p = 0; p < 8; ++p) {
        int pp[3] = {p & 1, (p >> 1) & 1, (p >> 2) & 1};
        for (int e = 0; e < P.n_far[p] + P.n_near[p]; ++e) {
            const StencilEntry &s = t->stencil[size_t(p) * P.ent_stride + e];
            int o[3] = {s.ox, s.oy, s.oz};
            int64_t cnt[3][3] = {{0}};
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 4; ++c) {
                    int b = 2 * c + pp[a] + o[a];
                    int slot = (b + 8) / 8;   // b in [-7, 14]
                    cnt[a][slot]++;
                }
            int fn = e < P.n_far[p] ? 0 : 1;
            for (int sz = 0; sz < 3; ++sz)
                for (int sy = 0; sy < 3; ++sy)
                    for (int sx = 0; sx < 3; ++sx)
                        tab[(size_t(p) * 2 + fn) * 27 + sx + 3 * sy + 9 * sz] +=
                            cnt[0][sx] * cnt[1][sy] * cnt[2][sz];
        }
    }
}

// Flop model: operations of one interaction of each kind as the kernels
// evaluate it, counted from their source (fused multiply-add = 2, the
// reciprocal square root = 1), compensation excluded.  The contraction works
// in traceless bases (D2 5, D3 7 + 2 dependent, 12 slice values of D4):
//   derivative tensors from R: 92; offset R: 3 (leaf source) or 6;
//   multipole<-multipole: orders 0-3 (86) + correction weights and sum (56) -> 240
//   multipole<-monopole:  M0 D^(n) (32) + weights (7) and sum (42)         -> 176
//   monopole<-monopole:   tabulated weights, 4 FMAs                        ->   8
//   monopole<-multipole:  orders 0-1 (62) + correction sum (42)            -> 199
// (Sec. 4.3 quotes 455 and 12 for the paper's own kernels.)
// Order 2 (no D4, no third orders): derivative tensors 51; multipole<-
// multipole 6 + 51 + orders 0-2 (28) + correction weights and sum (40) -> 125;
// multipole<-monopole 3 + 51 + 18 + 35 -> 107; monopole<-multipole
// 3 + 51 + 18 + 30 -> 102.
static const double kFlops[4] = {240.0, 176.0, 8.0, 199.0};
static const double kFlops2[4] = {125.0, 107.0, 8.0, 102.0};

// Monopole<-multipole work as pair lists: for every cell of a leaf node next
// to a refined node, the stencil entries whose source cell is refined, each
// with the source's packed-moment offset.  Targets are sorted by pair count
// (longest first) so that the 32 targets of a warp have nearly equal counts.
static void build_mx_pairs(fmm_tree_s *t, const std::vector<int32_t> &mx_nodes)
{
    const Plan &P = t->plan;
    struct Target { int32_t node, cell, off, count; };
    std::vector<Target> targets;
    std::vector<int32_t> pairs;              // (source offset, entry) interleaved
    for (int32_t node : mx_nodes) {
        const int32_t *nb = &t->nbr[size_t(node) * 27];
        for (int cell = 0; cell < NCELL; ++cell) {
            const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
            const int p = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
            const int n_ent = P.n_far[p] + P.n_near[p];
            const int32_t off = int32_t(pairs.size() / 2);
            for (int k = 0; k < n_ent; ++k) {
                const StencilEntry &e = t->stencil[size_t(p) * P.ent_stride + k];
                const int bx = x + e.ox + 8, by = y + e.oy + 8, bz = z + e.oz + 8;
                const int slot = (bx >> 3) + 3 * (by >> 3) + 9 * (bz >> 3);
                const int32_t src = nb[slot];
                if (src < 0 || t->info[size_t(src)].leaf_row >= 0) continue;
                // the kernels' parity-split cell order (parity_index)
                const int lx = bx & 7, ly = by & 7, lz = bz & 7;
                const int pi = ((lx & 1) + 2 * (ly & 1) + 4 * (lz & 1)) * 64 + (lx >> 1) +
                               4 * (ly >> 1) + 16 * (lz >> 1);
                pairs.push_back((t->info[size_t(src)].mp_row * 4 * NCELL + pi) * 4);
                pairs.push_back(k);
            }
            const int32_t count = int32_t(pairs.size() / 2) - off;
            if (count) targets.push_back(Target{node, cell, off, count});
        }
    }
    std::stable_sort(targets.begin(), targets.end(),
                     [](const Target &a, const Target &b) { return a.count > b.count; });
    // the same count as the planner's slot tables (two independent walks)
    if (int64_t(pairs.size() / 2) != P.kernel_interactions[2]) std::abort();
    // Interleave each warp's lists: the 32 consecutive targets of warp w
    // keep pair k of lane j at base_w + 32 k + j, so a warp's k-th loads are
    // one contiguous 256-byte read.  Lists are sorted by length, so the
    // padding (slots past a lane's own count, never read) is small.
    std::vector<int32_t> inter;
    t->mx_targets.resize(targets.size() * 4);
    for (size_t w0 = 0; w0 < targets.size(); w0 += 32) {
        const size_t w1 = std::min(targets.size(), w0 + 32);
        const int32_t kmax = targets[w0].count;
        const int64_t base = int64_t(inter.size() / 2);
        inter.resize(inter.size() + size_t(kmax) * 32 * 2, -1);
        for (size_t i = w0; i < w1; ++i) {
            const int32_t lane = int32_t(i - w0);
            for (int32_t k = 0; k < targets[i].count; ++k) {
                const size_t slot = size_t(base + int64_t(k) * 32 + lane);
                inter[2 * slot] = pairs[2 * size_t(targets[i].off + k)];
                inter[2 * slot + 1] = pairs[2 * size_t(targets[i].off + k) + 1];
            }
            t->mx_targets[4 * i + 0] = targets[i].node;
            t->mx_targets[4 * i + 1] = targets[i].cell;
            t->mx_targets[4 * i + 2] = int32_t(base);
            t->mx_targets[4 * i + 3] = targets[i].count;
        }
    }
    if (inter.size() / 2 > size_t(INT32_MAX)) std::abort();
    t->mx_pairs = std::move(inter);
    t->plan.n_mx_targets = int64_t(targets.size());
}

// The dataflow downward queue: every refined node's eight slices, levels
// from the root down, then every leaf node, coarse levels first, so that each
// item's parent comes earlier in the queue.
static void plan_dataflow(fmm_tree_s *t)
{
    std::vector<int32_t> &q = t->dflow_items;
    q.clear();
    for (int lev = 1; lev <= t->max_level; ++lev)
        for (int64_t i = 0; i < t->n; ++i) {
            const NodeInfo &x = t->info[size_t(i)];
            if (x.level == lev && x.leaf_row < 0)
                for (int sl = 0; sl < 8; ++sl) q.push_back(int32_t(i * 8 + sl));
        }
    t->plan.dflow_refined_items = int64_t(q.size());
    for (int lev = 1; lev <= t->max_level; ++lev)
        for (int64_t i = 0; i < t->n; ++i) {
            const NodeInfo &x = t->info[size_t(i)];
            if (x.level == lev && x.leaf_row >= 0) q.push_back(int32_t(i));
        }
    t->plan.dflow_items = int64_t(q.size());
}

static void plan_work(fmm_tree_s *t)
{
    Plan &P = t->plan;
    std::vector<int64_t> tab;
    slot_tables(t, tab);
    const int64_t n = t->n;
    std::vector<int64_t> cost(size_t(n), 0);
    std::vector<char> has_refined_nbr(size_t(n), 0);
    for (int k = 0; k < 4; ++k) P.interactions[k] = P.kernel_interactions[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const NodeInfo &x = t->info[size_t(i)];
        bool leaf = x.leaf_row >= 0;
        if (x.level == 1) {
            // root level: every pair of the one node is a candidate
            int64_t far = 0, nearc = 0;
            for (int a = 0; a < NCELL; ++a)
                for (int b = 0; b < NCELL; ++b) {
                    if (a == b) continue;
                    int ox = (b & 7) - (a & 7), oy = ((b >> 3) & 7) - ((a >> 3) & 7),
                        oz = (b >> 6) - (a >> 6);
                    (well_separated(t->cfg.theta, ox, oy, oz) ? far : nearc)++;
                }
            if (leaf) P.interactions[2] += far + nearc;
            else P.interactions[0] += far;
            P.kernel_interactions[3] += leaf ? far + nearc : far;
            cost[size_t(i)] = leaf ? (far + nearc) : far * 40;
            continue;
        }
        const int32_t *nb = &t->nbr[size_t(i) * 27];
        int64_t c[4] = {0, 0, 0, 0};
        for (int s = 0; s < 27; ++s) {
            if (nb[s] < 0) continue;
            bool src_leaf = t->info[size_t(nb[s])].leaf_row >= 0;
            if (!src_leaf && s != 13) has_refined_nbr[size_t(i)] = 1;
            for (int p = 0; p < 8; ++p) {
                int64_t fa = tab[(size_t(p) * 2 + 0) * 27 + s];
                int64_t ne = tab[(size_t(p) * 2 + 1) * 27 + s];
                if (!leaf) {
                    if (src_leaf) c[1] += fa + ne;
                    else c[0] += fa;
                } else {
                    if (src_leaf) c[2] += fa + ne;
                    else c[3] += fa + ne;
                }
            }
        }
        for (int k = 0; k < 4; ++k) P.interactions[k] += c[k];
        if (!leaf) P.kernel_interactions[0] += c[0] + c[1];
        else {
            P.kernel_interactions[1] += c[2];
            P.kernel_interactions[2] += c[3];
        }
        cost[size_t(i)] = leaf ? c[2] + 30 * c[3] : 45 * (c[0] + c[1]);
    }
    // node lists
    std::vector<int32_t> &L = t->lists;
    L.clear();
    auto push_range = [&](const std::vector<int32_t> &v) {
        ListRange r;
        r.off = int64_t(L.size());
        r.count = int64_t(v.size());
        L.insert(L.end(), v.begin(), v.end());
        return r;
    };
    auto by_cost = [&](std::vector<int32_t> &v) {
        std::stable_sort(v.begin(), v.end(),
                         [&](int32_t a, int32_t b) { return cost[size_t(a)] > cost[size_t(b)]; });
    };
    std::vector<int32_t> leaves, mp, mono, mx, roots, refined;
    for (int64_t i = 0; i < n; ++i) {
        const NodeInfo &x = t->info[size_t(i)];
        bool leaf = x.leaf_row >= 0;
        if (leaf) leaves.push_back(int32_t(i));
        else refined.push_back(int32_t(i));
        if (x.level == 1) { roots.push_back(int32_t(i)); continue; }
        if (!leaf) mp.push_back(int32_t(i));
        else {
            mono.push_back(int32_t(i));
            if (has_refined_nbr[size_t(i)]) mx.push_back(int32_t(i));
        }
    }
    by_cost(mp);
    by_cost(mono);
    by_cost(mx);
    P.leaves = push_range(leaves);
    P.work_mp = push_range(mp);
    P.work_mono = push_range(mono);
    P.work_mx = push_range(mx);
    P.roots = push_range(roots);
    build_mx_pairs(t, mx);
    P.refined = push_range(refined);
    P.refined_at.assign(size_t(t->max_level) + 2, {});
    P.leafkids_at.assign(size_t(t->max_level) + 2, {});
    P.mixedkids_at.assign(size_t(t->max_level) + 2, {});
    P.nodes_at.assign(size_t(t->max_level) + 2, {});
    for (int lev = 1; lev <= t->max_level; ++lev) {
        std::vector<int32_t> ref, all, leafkids, mixedkids;
        for (int64_t i = 0; i < n; ++i) {
            const NodeInfo &x = t->info[size_t(i)];
            if (x.level != lev) continue;
            all.push_back(int32_t(i));
            if (x.leaf_row >= 0) continue;
            ref.push_back(int32_t(i));
            bool kids_leaves = true;
            for (int k = 0; k < 8; ++k)
                kids_leaves = kids_leaves &&
                              t->info[size_t(t->children[size_t(i) * 8 + k])].leaf_row >= 0;
            (kids_leaves ? leafkids : mixedkids).push_back(int32_t(i));
        }
        P.refined_at[size_t(lev)] = push_range(ref);
        P.leafkids_at[size_t(lev)] = push_range(leafkids);
        P.mixedkids_at[size_t(lev)] = push_range(mixedkids);
        P.nodes_at[size_t(lev)] = push_range(all);
    }
}

// ------------------------------------------------------------- upload
template <typename T>
static int upload(T **dst, const std::vector<T> &src)
{
    if (src.empty()) { *dst = nullptr; return FMM_OK; }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), src.size() * sizeof(T));
    if (e != cudaSuccess) return fail(FMM_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return FMM_OK;
}

static void free_device(fmm_tree_s *t)
{
    for (cudaEvent_t e : t->timer.ev) cudaEventDestroy(e);
    t->timer.ev.clear();
    for (cudaEvent_t &e : t->step_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (t->aux) {
        cudaStreamDestroy(t->aux);
        t->aux = nullptr;
    }
    DeviceTables &d = t->dev;
    void *ptrs[] = {d.info, d.children, d.nbr, d.lists, d.stencil, d.stencil_f, d.coef32, d.coef64, d.coefdf, d.mono_woff,
                    d.tree_leaf_off, d.tree_leaf_rows, d.levels, d.levels_df, d.mass, d.mp, d.counters,
                    d.partials, d.chunk_sums, d.up, d.down, d.mx_targets, d.mx_pairs,
                    d.dflow_items, d.dflow_ready};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    d = DeviceTables{};
}

static int upload_tree(fmm_tree_s *t)
{
    DeviceTables &d = t->dev;
    int rc;
    if ((rc = upload(&d.info, t->info)) || (rc = upload(&d.children, t->children)) ||
        (rc = upload(&d.nbr, t->nbr)) || (rc = upload(&d.lists, t->lists)) ||
        (rc = upload(&d.stencil, t->stencil)) || (rc = upload(&d.stencil_f, t->stencil_f)) ||
        (rc = upload(&d.coef32, t->coef32)) ||
        (rc = upload(&d.coef64, t->coef64)) || (rc = upload(&d.coefdf, t->coefdf)) ||
        (rc = upload(&d.mono_woff, t->mono_woff)) ||
        (rc = upload(&d.tree_leaf_off, t->tree_leaf_off)) ||
        (rc = upload(&d.tree_leaf_rows, t->tree_leaf_rows)) || (rc = upload(&d.levels, t->levels)) ||
        (rc = upload(&d.levels_df, t->levels_df)) ||
        (rc = upload(reinterpret_cast<int32_t **>(&d.mx_targets), t->mx_targets)) ||
        (rc = upload(reinterpret_cast<int32_t **>(&d.mx_pairs), t->mx_pairs)) ||
        (rc = upload(&d.dflow_items, t->dflow_items)))
        return rc;
    // packed masses and moments: float (mixed), (hi, lo) float pairs (dfloat), double
    size_t es = t->cfg.precision == FMM_MIXED ? sizeof(float) : 2 * sizeof(float);
    static_assert(2 * sizeof(float) == sizeof(double), "packed element sizes");
    size_t mass_b = size_t(t->n) * NCELL * es;
    // one row past the refined nodes' rows stays zero: the multipole
    // kernel reads a leaf source's (absent) moments there
    const size_t mp_row_b = size_t(NMP) * NCELL * es;
    size_t mp_b = size_t(t->n_refined + 1) * mp_row_b;
    size_t part_b = size_t(std::max<int64_t>(t->n_leaf, 1)) * 8 * sizeof(double);
    size_t chunk_b = size_t(t->n_trees) * t->plan.reduce_chunks * 8 * sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&d.mass, mass_b)) != cudaSuccess ||
        (e = cudaMalloc(&d.mp, mp_b)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d.counters), 64 * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d.partials), part_b)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d.chunk_sums), chunk_b)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d.dflow_ready), size_t(t->n) * sizeof(int32_t))) !=
            cudaSuccess)
        return fail(FMM_ERR_NOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
    d.workspace_bytes = mass_b + mp_b + part_b + chunk_b + 64 * sizeof(int32_t) +
                        size_t(t->n) * sizeof(int32_t);
    // work queues and the status word start at zero
    if ((e = cudaMemset(d.counters, 0, 64 * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(static_cast<char *>(d.mp) + size_t(t->n_refined) * mp_row_b, 0, mp_row_b)) !=
            cudaSuccess)
        return cuda_fail(e, "cudaMemset");
    if (t->cfg.precision != FMM_FP64) {
        size_t up_b = size_t(std::max<int64_t>(t->n_refined, 1)) * 20 * NCELL * 2 * sizeof(float);
        if ((e = cudaMalloc(reinterpret_cast<void **>(&d.up), up_b)) != cudaSuccess)
            return fail(FMM_ERR_NOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
        d.workspace_bytes += up_b;
    }
    if (t->cfg.precision != FMM_FP64) {
        // (hi, lo) float pairs
        size_t down_b = size_t(std::max<int64_t>(t->n_refined, 1)) * 23 * NCELL * 2 * sizeof(float);
        if ((e = cudaMalloc(reinterpret_cast<void **>(&d.down), down_b)) != cudaSuccess)
            return fail(FMM_ERR_NOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
        d.workspace_bytes += down_b;
    }
    // fmm_step's second stream and events (no timing: they only order work)
    if ((e = cudaStreamCreateWithFlags(&t->aux, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    for (cudaEvent_t &ev : t->step_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
    if (t->cfg.flags & FMM_FLAG_TIMING) {
        const int records = 256;
        t->timer.ev.resize(size_t(2 * records));
        t->timer.slot.assign(size_t(records), 0);
        for (auto &ev : t->timer.ev)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    return FMM_OK;
}

// ================================================================ C ABI
extern "C" {

int fmm_build_tree(const fmm_node_desc *nodes, int64_t n_nodes, const fmm_config *cfg,
                   fmm_tree_t *out)
{
    if (!out) return fail(FMM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !cfg) return fail(FMM_ERR_INVALID_ARG, "nodes or cfg is NULL");
    if (n_nodes < 1 || n_nodes > (int64_t(1) << 30))
        return fail(FMM_ERR_INVALID_ARG, "n_nodes must lie in 1..2^30");
    int rc = validate_config(cfg);
    if (rc) return rc;
    fmm_tree_s *t = new (std::nothrow) fmm_tree_s();
    if (!t) return fail(FMM_ERR_NOMEM, "host allocation failed");
    t->cfg = *cfg;
    if (t->cfg.order == 0) t->cfg.order = 3;
    t->n = n_nodes;
    t->host_only = (cfg->flags & FMM_FLAG_HOST_ONLY) != 0;
    std::vector<std::unordered_map<uint64_t, int32_t>> maps;
    rc = validate_nodes(nodes, n_nodes, cfg, t, maps);
    if (rc) { delete t; return rc; }
    // node table
    t->info.resize(size_t(n_nodes));
    t->children.assign(size_t(n_nodes) * 8, -1);
    int64_t leaf_rows = 0, mp_rows = 0;
    for (int64_t i = 0; i < n_nodes; ++i) {
        const fmm_node_desc &x = nodes[i];
        bool leaf = x.child[0] < 0;
        t->info[size_t(i)] = NodeInfo{x.level, x.ix, x.iy, x.iz, x.parent,
                                      leaf ? int32_t(leaf_rows++) : -1,
                                      leaf ? -1 : int32_t(mp_rows++), x.tree_id};
        for (int k = 0; k < 8; ++k) t->children[size_t(i) * 8 + k] = x.child[k];
        t->max_level = std::max(t->max_level, x.level);
    }
    t->n_leaf = leaf_rows;
    t->n_refined = mp_rows;
    // the same-level kernels address packed moments with 32-bit offsets
    // (row * 8192 elements)
    if (mp_rows > (int64_t(1) << 31) / (4 * NCELL * 4) - 1) {
        delete t;
        return fail(FMM_ERR_INVALID_ARG, "more than 262143 refined nodes in one tree handle");
    }
    // neighbours, and the nesting rule for refined nodes
    t->nbr.assign(size_t(n_nodes) * 27, -1);
    for (int64_t i = 0; i < n_nodes; ++i) {
        const fmm_node_desc &x = nodes[i];
        int64_t side = int64_t(1) << (x.level - 1);
        auto &m = maps[size_t(x.tree_id)];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t jx = x.ix + dx, jy = x.iy + dy, jz = x.iz + dz;
                    if (jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;
                    auto it = m.find(node_key(x.level, jx, jy, jz));
                    int s = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                    if (it != m.end()) t->nbr[size_t(i) * 27 + s] = it->second;
                    else if (x.child[0] >= 0) {
                        delete t;
                        return fail(FMM_ERR_TREE, "node " + std::to_string(i) +
                                                      " is refined but an in-domain neighbour is missing");
                    }
                }
    }
    // leaf rows grouped per tree (fixed-order reductions)
    t->tree_leaf_off.assign(size_t(t->n_trees) + 1, 0);
    for (int64_t i = 0; i < n_nodes; ++i)
        if (t->info[size_t(i)].leaf_row >= 0) t->tree_leaf_off[size_t(t->info[size_t(i)].tree) + 1]++;
    for (int32_t k = 0; k < t->n_trees; ++k) t->tree_leaf_off[size_t(k) + 1] += t->tree_leaf_off[size_t(k)];
    int64_t most = 1;
    for (int32_t k = 0; k < t->n_trees; ++k)
        most = std::max<int64_t>(most, t->tree_leaf_off[size_t(k) + 1] - t->tree_leaf_off[size_t(k)]);
    t->plan.reduce_chunks = int((most + kReduceRows - 1) / kReduceRows);
    t->tree_leaf_rows.assign(size_t(t->n_leaf), 0);
    {
        std::vector<int32_t> fill(t->tree_leaf_off.begin(), t->tree_leaf_off.end() - 1);
        for (int64_t i = 0; i < n_nodes; ++i) {
            const NodeInfo &x = t->info[size_t(i)];
            if (x.leaf_row >= 0) t->tree_leaf_rows[size_t(fill[size_t(x.tree)]++)] = x.leaf_row;
        }
    }
    build_stencils(t);
    plan_work(t);
    plan_dataflow(t);
    // per-level geometry: h = box / (8 * 2^(l-1)) is exact up to the box edge
    t->levels.assign(size_t(t->max_level + 1) * LEVEL_FIELDS, 0.0);
    for (int lev = 1; lev <= t->max_level; ++lev) {
        double *L = &t->levels[size_t(lev) * LEVEL_FIELDS];
        const double h = cfg->box_size / (8.0 * std::ldexp(1.0, lev - 1));
        L[LV_H] = h;
        L[LV_IH] = 1.0 / h;
        L[LV_H3] = h * h * h;
        L[LV_S0] = cfg->G / h;
        L[LV_S1] = L[LV_S0] / h;
        L[LV_S2] = L[LV_S1] / h;
        L[LV_S3] = L[LV_S2] / h;
        for (int k = 0; k < 4; ++k) L[LV_R0 + k] = 1.0 / L[LV_S0 + k];
    }
    // the same h, inverse scales and scales as (hi, lo) float pairs
    t->levels_df.assign(size_t(t->max_level + 1) * LEVEL_DF_FIELDS * 2, 0.f);
    for (int lev = 1; lev <= t->max_level; ++lev) {
        const double *L = &t->levels[size_t(lev) * LEVEL_FIELDS];
        const double v[LEVEL_DF_FIELDS] = {L[LV_H],  L[LV_R0], L[LV_R1], L[LV_R2], L[LV_R3],
                                           L[LV_S0], L[LV_S1], L[LV_S2], L[LV_S3]};
        for (int k = 0; k < LEVEL_DF_FIELDS; ++k) {
            float *o = &t->levels_df[(size_t(lev) * LEVEL_DF_FIELDS + k) * 2];
            o[0] = float(v[k]);
            o[1] = float(v[k] - double(o[0]));
        }
    }
    if (!t->host_only) {
        if (cudaGetDevice(&t->device) != cudaSuccess) {
            delete t;
            return fail(FMM_ERR_CUDA, "no CUDA device available (use FMM_FLAG_HOST_ONLY to plan only)");
        }
        rc = upload_tree(t);
        if (rc) { free_device(t); delete t; return rc; }
    }
    *out = t;
    return FMM_OK;
}

int fmm_get_sizes(fmm_tree_t t, fmm_sizes *o)
{
    if (!t || !o) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof *o);
    o->n_nodes = t->n;
    o->n_leaf = t->n_leaf;
    o->n_refined = t->n_refined;
    o->n_trees = t->n_trees;
    o->max_level = t->max_level;
    o->precision = t->cfg.precision;
    int64_t per = int64_t(NCELL) * 8;
    bool mixed = t->cfg.precision != FMM_FP64;     // float (hi, lo) Taylor coefficients
    o->rho_bytes = t->n_leaf * per;
    o->M_bytes = t->n * NCOMP * per;
    o->com_bytes = t->n * 3 * per;
    o->L_bytes = t->n * NCOMP * NCELL * (mixed ? 4 : 8);
    o->Lcomp_bytes = mixed ? t->n * NCOMP * NCELL * 4 : 0;
    o->dL1_bytes = t->n * 3 * per;
    o->L64_bytes = t->n * NCOMP * per;
    o->phi_bytes = t->n_leaf * per;
    o->g_bytes = t->n_leaf * 3 * per;
    o->totals_bytes = int64_t(t->n_trees) * 8 * 8;
    o->workspace_bytes = int64_t(t->dev.workspace_bytes);
    return FMM_OK;
}

int fmm_get_stats(fmm_tree_t t, fmm_stats *o)
{
    if (!t || !o) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof *o);
    const Plan &P = t->plan;
    for (int k = 0; k < 4; ++k) {
        o->interactions[k] = P.interactions[k];
        o->flops_per_interaction[k] = t->cfg.order == 2 ? kFlops2[k] : kFlops[k];
    }
    o->stencil_far = P.n_far[0];
    o->stencil_near = P.n_near[0];
    o->stencil_union = P.stencil_union;
    o->work_items[0] = P.work_mp.count;
    o->work_items[1] = P.work_mono.count;
    o->work_items[2] = P.work_mx.count;
    o->work_items[3] = P.roots.count;
    for (int k = 0; k < 4; ++k) o->kernel_interactions[k] = P.kernel_interactions[k];
    o->reach = P.reach;
    int m2l = 1 /*pack*/ + (P.roots.count > 0) + (P.work_mp.count > 0) + (P.work_mono.count > 0) +
              (P.n_mx_targets > 0);
    int up = 1;
    for (int lev = 1; lev < t->max_level; ++lev) up += P.refined_at[size_t(lev)].count > 0;
    int down = 0;
    for (int lev = 1; lev <= t->max_level; ++lev) down += P.nodes_at[size_t(lev)].count > 0;
    o->launches_m2l = m2l;
    o->launches_step = up + m2l + down + 3;
    // fmm_step: P2M also packs the leaf masses, one pack launch for the
    // refined nodes; then either the refined levels' shifts per level and
    // every leaf's shift and forces in one launch, or (dataflow tuning) all
    // of it in one persistent launch; the two force-sum launches
    int refined_levels = 0;
    for (int lev = 1; lev <= t->max_level; ++lev) refined_levels += P.refined_at[size_t(lev)].count > 0;
    // (the monopole<-multipole targets ride in the multipole launch)
    const int mx_alone = (P.n_mx_targets > 0) && (P.work_mp.count == 0);
    const int downward = t->tuning.dataflow ? 1 : refined_levels + (P.leaves.count > 0);
    o->launches_fused = up + (m2l - 1) - (P.n_mx_targets > 0) + mx_alone + (P.refined.count > 0) +
                        downward + 2;
    if ((t->cfg.flags & FMM_FLAG_TIMING) && !t->host_only) {
        o->timing = 1;
        timing_fold(t);
        for (int k = 0; k < FMM_K_COUNT; ++k) {
            o->kernel_ms[k] = t->timer.ms[k];
            o->kernel_launches[k] = t->timer.launches[k];
            t->timer.ms[k] = 0.0;
            t->timer.launches[k] = 0;
        }
    }
    return FMM_OK;
}

static int check_device_tree(fmm_tree_t t)
{
    if (!t) return fail(FMM_ERR_INVALID_ARG, "tree is NULL");
    if (t->host_only) return fail(FMM_ERR_INVALID_ARG, "tree was planned with FMM_FLAG_HOST_ONLY");
    return FMM_OK;
}

// P2M moves the density and the leaf masses as 16-byte vectors
static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int fmm_upward(fmm_tree_t t, const double *rho, double *M, double *com, fmm_stream_t stream)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!rho || !M || !com) return fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(rho) || !aligned16(M))
        return fail(FMM_ERR_INVALID_ARG, "rho and M must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    timing_begin(t, FMM_K_P2M, s);
    cudaError_t e = launch_p2m(t, rho, M, s);
    timing_end(t, s);
    if (e != cudaSuccess) return cuda_fail(e, "p2m launch");
    for (int lev = t->max_level - 1; lev >= 1; --lev) {
        if (t->plan.refined_at[size_t(lev)].count == 0) continue;
        timing_begin(t, FMM_K_M2M, s);
        e = launch_m2m_level(t, lev, M, com, s);
        timing_end(t, s);
        if (e != cudaSuccess) return cuda_fail(e, "m2m launch");
    }
    return FMM_OK;
}

int fmm_m2l(fmm_tree_t t, const double *M, const double *com, void *L, float *L_comp,
            double *dL1, fmm_stream_t stream)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!M || !com || !L || !dL1) return fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    if (t->cfg.precision != FMM_FP64 && !L_comp)
        return fail(FMM_ERR_INVALID_ARG, "L_comp is required in FMM_MIXED and FMM_DFLOAT");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    timing_begin(t, FMM_K_PACK, s);
    cudaError_t e = launch_pack(t, M, com, s);
    timing_end(t, s);
    if (e != cudaSuccess) return cuda_fail(e, "pack launch");
    int nl = 0;
    e = launch_m2l(t, L, L_comp, dL1, s, &nl);
    if (e != cudaSuccess) return cuda_fail(e, "m2l launch");
    return FMM_OK;
}

int fmm_downward(fmm_tree_t t, const void *L, const float *L_comp, const double *dL1,
                 const double *com, double *L64, double *dL1_acc, fmm_stream_t stream)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!L || !dL1 || !com || !L64 || !dL1_acc) return fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    if (t->cfg.precision != FMM_FP64 && !L_comp)
        return fail(FMM_ERR_INVALID_ARG, "L_comp is required in FMM_MIXED and FMM_DFLOAT");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int lev = 1; lev <= t->max_level; ++lev) {
        if (t->plan.nodes_at[size_t(lev)].count == 0) continue;
        timing_begin(t, FMM_K_L2L, s);
        cudaError_t e = launch_l2l_level(t, lev, L, L_comp, dL1, com, L64, dL1_acc, s);
        timing_end(t, s);
        if (e != cudaSuccess) return cuda_fail(e, "l2l launch");
    }
    return FMM_OK;
}

int fmm_forces(fmm_tree_t t, const double *L64, const double *dL1_acc, const double *rho,
               double *phi, double *g, double *totals, fmm_stream_t stream)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!L64 || !dL1_acc || !rho || !phi || !g || !totals)
        return fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    cudaError_t e = launch_forces(t, L64, dL1_acc, rho, phi, g, totals,
                                  static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "forces launch");
    return FMM_OK;
}

// The whole step as one call, with the passes' independent work overlapped on
// two streams: the monopole<-monopole kernel needs only leaf masses, so it
// runs beside the upward pass of the refined levels; the multipole launch
// also takes the monopole<-multipole targets once its own queue is empty,
// with the roots beside it on the second stream; then the refined levels'
// shifts, and every leaf's shift and forces (all levels, one fused launch).
// The same arithmetic, hence the same results, as fmm_upward, fmm_m2l,
// fmm_downward and fmm_forces in sequence.
int fmm_step(fmm_tree_t t, const double *rho, double *M, double *com, void *L, float *L_comp,
             double *dL1, double *L64, double *dL1_acc, double *phi, double *g, double *totals,
             fmm_stream_t stream)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!rho || !M || !com || !L || !dL1 || !L64 || !dL1_acc || !phi || !g || !totals)
        return fail(FMM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(rho) || !aligned16(M))
        return fail(FMM_ERR_INVALID_ARG, "rho and M must be 16-byte aligned");
    if (t->cfg.precision != FMM_FP64 && !L_comp)
        return fail(FMM_ERR_INVALID_ARG, "L_comp is required in FMM_MIXED and FMM_DFLOAT");
    if (t->cfg.flags & FMM_FLAG_TIMING) {
        // per-kernel events on one stream: the passes in sequence
        if ((rc = fmm_upward(t, rho, M, com, stream)) || (rc = fmm_m2l(t, M, com, L, L_comp, dL1, stream)) ||
            (rc = fmm_downward(t, L, L_comp, dL1, com, L64, dL1_acc, stream)))
            return rc;
        return fmm_forces(t, L64, dL1_acc, rho, phi, g, totals, stream);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream), a = t->aux;
    cudaEvent_t *ev = t->step_ev;
    const Plan &P = t->plan;
    cudaError_t e;
    int nl = 0;
#define FMM_STEP_TRY(call, what) \
    if ((e = (call)) != cudaSuccess) return cuda_fail(e, what)
    // main: reset the work queues, P2M, fork
    FMM_STEP_TRY(launch_m2l(t, L, L_comp, dL1, s, &nl, M2L_RESET), "queue reset");
    FMM_STEP_TRY(launch_p2m(t, rho, M, s, true), "p2m launch");
    FMM_STEP_TRY(cudaEventRecord(ev[0], s), "cudaEventRecord");
    // Events: 0 P2M done, 1 refined sources packed, 2 refined shifts done,
    // 3 second stream done, 4 roots done, 5 monopole kernel done.
    // aux: leaf masses, monopole<-monopole
    // (P2M has stored the leaf masses in their packed form)
    FMM_STEP_TRY(cudaStreamWaitEvent(a, ev[0], 0), "cudaStreamWaitEvent");
    FMM_STEP_TRY(launch_m2l(t, L, L_comp, dL1, a, &nl, M2L_MONO), "m2l launch");
    FMM_STEP_TRY(cudaEventRecord(ev[5], a), "cudaEventRecord");
    // main: M2M, refined sources, multipole targets
    for (int lev = t->max_level - 1; lev >= 1; --lev)
        if (P.refined_at[size_t(lev)].count)
            FMM_STEP_TRY(launch_m2m_level(t, lev, M, com, s), "m2m launch");
    FMM_STEP_TRY(launch_pack(t, M, com, s, PACK_REFINED), "pack launch");
    FMM_STEP_TRY(cudaEventRecord(ev[1], s), "cudaEventRecord");
    // the multipole targets' leaf sources read the leaf masses packed on aux;
    // the same launch then takes the monopole<-multipole targets, which add
    // to what the monopole kernel stored, so it also waits for that kernel
    // (on cfg-size trees it has finished by then).  The monopole<-multipole
    // work fills the multipole kernel's tail, where its last coarse items
    // leave SMs idle; as a launch of its own it held its SMs for its whole
    // run and delayed whichever of the multipole kernel and the shifts
    // came second.
    FMM_STEP_TRY(cudaStreamWaitEvent(s, ev[5], 0), "cudaStreamWaitEvent");
    FMM_STEP_TRY(launch_m2l(t, L, L_comp, dL1, s, &nl, M2L_MP | M2L_MPX), "m2l launch");
    // aux: the roots (16 CTAs per root) beside the multipole launch rather
    // than before it on the main stream, where the GPU idled around them
    FMM_STEP_TRY(cudaStreamWaitEvent(a, ev[1], 0), "cudaStreamWaitEvent");
    FMM_STEP_TRY(launch_m2l(t, L, L_comp, dL1, a, &nl, M2L_ROOT), "m2l launch");
    FMM_STEP_TRY(cudaEventRecord(ev[4], a), "cudaEventRecord");
    FMM_STEP_TRY(cudaStreamWaitEvent(s, ev[4], 0), "cudaStreamWaitEvent");
    if (t->tuning.dataflow) {
        // main: the refined shifts and the leaf pass in one persistent
        // launch, each item started by its parent's readiness counter; the
        // sums
        FMM_STEP_TRY(launch_downward_dataflow(t, L, L_comp, dL1, com, L64, dL1_acc, M, phi, g, s),
                     "dataflow launch");
        FMM_STEP_TRY(launch_force_sums(t, totals, s), "reduce launch");
        return FMM_OK;
    }
    // main: shifts of the refined nodes, root level first
    for (int lev = 1; lev <= t->max_level; ++lev)
        FMM_STEP_TRY(launch_l2l_nodes(t, P.refined_at[size_t(lev)], L, L_comp, dL1, com, L64,
                                      dL1_acc, s), "l2l launch");
    FMM_STEP_TRY(cudaEventRecord(ev[2], s), "cudaEventRecord");
    // aux: every leaf's shift and forces in one pass (the shifted expansion
    // feeds the forces from registers), the sums; join
    FMM_STEP_TRY(cudaStreamWaitEvent(a, ev[2], 0), "cudaStreamWaitEvent");
    FMM_STEP_TRY(launch_leaf_finish(t, L, L_comp, dL1, com, L64, dL1_acc, M, phi, g, a),
                 "leaf launch");
    FMM_STEP_TRY(launch_force_sums(t, totals, a), "reduce launch");
    FMM_STEP_TRY(cudaEventRecord(ev[3], a), "cudaEventRecord");
    FMM_STEP_TRY(cudaStreamWaitEvent(s, ev[3], 0), "cudaStreamWaitEvent");
#undef FMM_STEP_TRY
    return FMM_OK;
}

void fmm_destroy_tree(fmm_tree_t t)
{
    if (!t) return;
    if (!t->host_only) {
        cudaDeviceSynchronize();
        free_device(t);
    }
    delete t;
}

int fmm_set_tuning(fmm_tree_t t, const fmm_tuning *tu)
{
    if (!t || !tu) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    if (tu->mono_subgrids < 0 || tu->mono_subgrids > 4 || tu->mono_subgrids == 3)
        return fail(FMM_ERR_INVALID_ARG, "mono_subgrids must be 0, 1, 2 or 4");
    if (tu->ctas_per_sm < 0 || tu->ctas_per_sm > 32)
        return fail(FMM_ERR_INVALID_ARG, "ctas_per_sm must lie in 0..32");
    if (tu->dataflow < 0 || tu->dataflow > 1 || tu->drop_first_producer < 0 ||
        tu->drop_first_producer > 1 || tu->wait_budget_us < 0 || tu->mp_pair_targets < 0 ||
        tu->mp_pair_targets > 1)
        return fail(FMM_ERR_INVALID_ARG, "dataflow, drop_first_producer and mp_pair_targets "
                                         "must be 0 or 1, wait_budget_us not negative");
    if (tu->mp_items < 0 || tu->mp_items > 2)
        return fail(FMM_ERR_INVALID_ARG, "mp_items must be 0, 1 or 2");
    t->tuning = *tu;
    return FMM_OK;
}

int fmm_get_tuning(fmm_tree_t t, fmm_tuning *tu)
{
    if (!t || !tu) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    *tu = t->tuning;
    return FMM_OK;
}

int fmm_get_status(fmm_tree_t t, int32_t *status, int clear)
{
    int rc = check_device_tree(t);
    if (rc) return rc;
    if (!status) return fail(FMM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int32_t *word = t->dev.counters + kStatusSlot;
    if ((e = cudaMemcpy(status, word, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    if (clear && (e = cudaMemset(word, 0, sizeof(int32_t))) != cudaSuccess)
        return cuda_fail(e, "cudaMemset");
    if (*status & FMM_STATUS_TIMEOUT)
        return fail(FMM_ERR_TIMEOUT, "a device-side wait of the dataflow pass ran out of budget");
    return FMM_OK;
}

const char *fmm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
