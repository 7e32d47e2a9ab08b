/*
 * fmm_gb300.h -- C ABI of the GB300 (sm_103a) cell-based FMM gravity solve.
 *
 * The method is the FMM of Octo-Tiger (arXiv 1908.03121, Sec. 4.3 "The FMM
 * hotspot"): an adaptive octree whose nodes are 8x8x8-cell sub-grids; an
 * upward pass computing each cell's multipole moments and centre of mass from
 * the leaf densities; a same-level pass in which each cell collects Taylor
 * coefficients from the cells picked by the opening criterion (four kinds of
 * interaction by node refinement, Sec. 4.3); and a downward pass that hands
 * each parent's Taylor expansion to its children and accumulates it.  The
 * gravity solver also conserves angular momentum (Sec. 2, Sec. 4.2), through a
 * correction to the force coefficient that is carried down the tree.
 *
 * Conventions shared by every call
 *   - Expansion order 3: 20 packed symmetric-tensor components per cell,
 *     ordered  0 | x y z | xx xy xz yy yz zz | xxx xxy xxz xyy xyz xzz yyy
 *     yyz yzz zzz.  Moments are central moments about the cell's centre of
 *     mass, so the three dipole slots are always zero.
 *   - Cells inside a node are numbered x + 8 y + 64 z; per-node arrays are
 *     node-major, [node][component][cell], nodes in descriptor order.
 *   - Leaf rows (density, potential, field) follow the order in which leaf
 *     nodes appear in the descriptor array.
 *   - Cell width at level l (root = 1): h_l = box_size / (8 * 2^(l-1)).
 *   - Opening rule: cells at integer offset o (in cell widths) are well
 *     separated iff theta^2 |o|^2 > 1; a same-level pair is a candidate iff
 *     its parent cells are not well separated (all pairs on the root level);
 *     a candidate is evaluated iff it is well separated or either cell is a
 *     leaf cell.  theta must lie in (0.25, 1/sqrt(3)] so that sources stay in
 *     the 26 neighbour nodes and every leaf pair is evaluated exactly once.
 *
 * Memory and streams
 *   - The caller owns every data buffer (device memory, raw pointers).  The
 *     library owns only what fmm_build_tree allocates (tree tables on the
 *     device and a fixed workspace), released by fmm_destroy_tree.
 *   - fmm_upward / fmm_m2l / fmm_downward / fmm_forces only enqueue work on
 *     the given stream (a cudaStream_t; NULL = legacy default stream).  They
 *     do not allocate, free or synchronise.  A tree's workspace is shared by
 *     its calls, so calls on one tree must not overlap in time (serialise
 *     them on one stream).
 *   - Buffer sizes in bytes are reported by fmm_get_sizes.
 *
 * Errors: every int-returning call gives 0 or a negative FMM_ERR_* code;
 * fmm_last_error() returns a message for the calling thread's last failure.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_tree_s *fmm_tree_t;
typedef void *fmm_stream_t;          /* cudaStream_t */

enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = -1,        /* null pointer, bad config, host-only tree */
    FMM_ERR_TREE = -2,               /* descriptors do not form a valid octree */
    FMM_ERR_CUDA = -3,               /* a CUDA call or launch failed */
    FMM_ERR_TIMEOUT = -4,            /* a device-side wait exceeded its budget */
    FMM_ERR_NOMEM = -5               /* device or host allocation failed */
};

/* Precision of the same-level pass (the other passes are FP64 throughout):
 *   FMM_FP64    double arithmetic;
 *   FMM_MIXED   float contraction with two-sum compensated accumulation,
 *               offsets from double centres of mass, the correction finished
 *               in double; relative force error about 1e-7, net torque about
 *               1e-9 of the total;
 *   FMM_DFLOAT  conserving: every same-level operation in double-float
 *               arithmetic (pairs of floats, about 48 bits, on the FP32
 *               pipe), so that the pairwise cancellations behind momentum and
 *               angular-momentum conservation hold to about 1e-13. */
enum { FMM_FP64 = 0, FMM_MIXED = 1, FMM_DFLOAT = 2 };

enum {
    FMM_FLAG_HOST_ONLY = 1,          /* plan on the host only; no CUDA calls */
    FMM_FLAG_TIMING = 2              /* bracket every kernel launch with CUDA
                                        events on the call's stream (eager use
                                        only: do not capture such a tree in a
                                        graph); read back by fmm_get_stats */
};

/* kernel slots of fmm_stats.kernel_ms / kernel_launches */
enum {
    FMM_K_P2M = 0, FMM_K_M2M, FMM_K_PACK, FMM_K_ROOT, FMM_K_MULTIPOLE, FMM_K_MONOPOLE,
    FMM_K_MONO_MULTI, FMM_K_L2L, FMM_K_FORCES, FMM_K_REDUCE, FMM_K_COUNT
};

typedef struct {
    double theta;                    /* opening angle, (0.25, 1/sqrt(3)] */
    double G;                        /* gravitational constant */
    double box_lo[3];                /* lower corner of every tree's domain */
    double box_size;                 /* edge of the cubic domain */
    int32_t precision;               /* FMM_FP64, FMM_MIXED or FMM_DFLOAT */
    int32_t max_level;               /* deepest level allowed (1..20) */
    int32_t flags;                   /* FMM_FLAG_* */
    int32_t order;                   /* expansion order p: 3 (0 selects it), or 2: the
                                        same-level truncation n + m <= p, Taylor
                                        coefficients up to order p (the third-order
                                        slots of L stay zero at p = 2), and the
                                        correction's dropped term n = 1, m = p with
                                        the target's share signed (-1)^p (see
                                        fmm_m2l) */
} fmm_config;

/* One octree node.  child[k] covers octant (k&1, (k>>1)&1, (k>>2)&1) of the
 * node; either all eight children are -1 (leaf) or all are valid.  The root
 * of each tree is level 1 at (0,0,0) with parent -1.  tree_id groups nodes
 * of independent trees solved together (nodes of different trees never
 * interact). */
typedef struct {
    int32_t level, ix, iy, iz;
    int32_t parent;
    int32_t child[8];
    int32_t tree_id;
} fmm_node_desc;

typedef struct {
    int64_t n_nodes, n_leaf, n_refined, n_trees;
    int32_t max_level, precision;
    /* required buffer sizes in bytes */
    int64_t rho_bytes;               /* double [n_leaf][512] */
    int64_t M_bytes;                 /* double [n_nodes][20][512] */
    int64_t com_bytes;               /* double [n_nodes][3][512] */
    int64_t L_bytes;                 /* double or float [n_nodes][20][512] */
    int64_t Lcomp_bytes;             /* float [n_nodes][20][512] (mixed, dfloat), else 0 */
    int64_t dL1_bytes;               /* double [n_nodes][3][512] */
    int64_t L64_bytes;               /* double [n_nodes][20][512] */
    int64_t phi_bytes;               /* double [n_leaf][512] */
    int64_t g_bytes;                 /* double [n_leaf][3][512] */
    int64_t totals_bytes;            /* double [n_trees][8] */
    int64_t workspace_bytes;         /* device memory the tree itself holds */
} fmm_sizes;

typedef struct {
    /* evaluated directed cell pairs of each kind, in the order
     * multipole<-multipole, multipole<-monopole, monopole<-monopole,
     * monopole<-multipole (target <- source) */
    int64_t interactions[4];
    int64_t stencil_far;             /* well-separated offsets per parity */
    int64_t stencil_near;            /* near offsets per parity */
    int64_t stencil_union;           /* distinct offsets over the 8 parities */
    double flops_per_interaction[4]; /* operation count of one interaction */
    int64_t work_items[4];           /* nodes handled by each same-level kernel:
                                        multipole, monopole, monopole<-multipole, root */
    int64_t kernel_interactions[4];  /* interactions evaluated by each of those kernels */
    int32_t reach;                   /* largest per-axis stencil offset */
    int32_t launches_m2l;            /* kernel launches per fmm_m2l call */
    int32_t launches_step;           /* kernel launches per upward+m2l+downward+forces */
    int32_t timing;                  /* 1 if the tree was built with FMM_FLAG_TIMING */
    int32_t launches_fused;          /* kernel launches per fmm_step under the tree's
                                        tuning at the time of the call */
    int32_t reserved;
    /* FMM_FLAG_TIMING only: device time (ms) and launch count per kernel slot
     * (FMM_K_*), summed over the launches since the previous fmm_get_stats
     * call, which waits for those launches and then resets the sums. */
    double kernel_ms[16];
    int64_t kernel_launches[16];
} fmm_stats;

/*
 * Validate descriptors and plan the solve (Sec. 4.2: octree of N^3 sub-grids;
 * Sec. 4.3: per-level stencil of constant size).  Host work, then one upload
 * of the tables and one workspace allocation on the current device (none with
 * FMM_FLAG_HOST_ONLY).  Synchronous.
 *   nodes: host array of n_nodes descriptors (copied; the caller keeps it).
 *   cfg:   host config (copied).
 *   out:   receives the tree handle on success, NULL on failure.
 * Errors: FMM_ERR_INVALID_ARG (null pointers, n_nodes < 1, theta or box or
 * precision out of range), FMM_ERR_TREE (broken parent/child links, bad
 * levels or coordinates, duplicates, a refined node with a missing in-domain
 * neighbour, levels above cfg->max_level), FMM_ERR_NOMEM, FMM_ERR_CUDA.
 */
int fmm_build_tree(const fmm_node_desc *nodes, int64_t n_nodes,
                   const fmm_config *cfg, fmm_tree_t *out);

/* Sizes of the buffers the caller allocates for this tree (the octree of
 * Sec. 4.2: 512 cells per sub-grid) and of the tree's own workspace; host,
 * immediate.  Errors: FMM_ERR_INVALID_ARG (NULL). */
int fmm_get_sizes(fmm_tree_t tree, fmm_sizes *out);

/* Interaction counts of the opening rule, stencil sizes, the operation-count
 * model (Sec. 4.3 quotes 455 and 12 operations for its two main kernels;
 * this library reports its own counts) and launch counts (host, immediate;
 * with FMM_FLAG_TIMING it first waits for the timed launches).
 * Errors: FMM_ERR_INVALID_ARG (NULL). */
int fmm_get_stats(fmm_tree_t tree, fmm_stats *out);

/*
 * Upward pass (Sec. 4.3, first step).  Leaf cells: mass m = rho h^3 placed at
 * the cell centre (locally homogeneous density, Sec. 3 and Sec. 4.3).
 * Refined cells: mass, centre of mass and central moments of their eight
 * child cells, combined in FP64, deepest level first.
 *   rho: double [n_leaf][512], 16-byte aligned, read once, by one kernel:
 *        device memory, or page-locked host memory mapped into the device's
 *        address space (the kernel then reads it over the host link; the
 *        caller keeps it unchanged until the pass has completed on `stream`).
 *   M:   device double [n_nodes][20][512], 16-byte aligned, written.  For leaf nodes only
 *        component 0 (the cell mass) is written; their other components are
 *        zero by definition and are not touched.
 *   com: device double [n_nodes][3][512], written for refined nodes only
 *        (a leaf cell's centre of mass is its centre by definition).
 * Kernels are enqueued on `stream`; the call neither allocates nor waits.  A
 * density that is not positive sets FMM_STATUS_BAD_DENSITY (fmm_get_status).
 * Errors: FMM_ERR_INVALID_ARG (NULL tree or buffer, a FMM_FLAG_HOST_ONLY
 * tree, rho or M not 16-byte aligned), FMM_ERR_CUDA (a launch failed).
 */
int fmm_upward(fmm_tree_t tree, const double *rho, double *M, double *com,
               fmm_stream_t stream);

/*
 * Same-level pass (Sec. 4.3, second step; Sec. 5.1 runs it on the GPU).
 * Every cell A gathers, from every source cell B the opening rule selects,
 *   L^(n)_A += -G sum_{m: n+m<=p} ((-1)^m/m!) M_B^(m) . D^(n+m)(X_A - X_B),
 * D^(k) the k-th derivative tensor of 1/|R|, p the expansion order (3 by
 * default), plus the angular-momentum correction
 *   p = 3:  dL1_A,i += (G/6) sum_jkl D^(4)_ijkl(X_A - X_B) [M_B^(3) - (M_B^(0)/M_A^(0)) M_A^(3)]_jkl,
 *   p = 2:  dL1_A,i -= (G/2) sum_jk D^(3)_ijk(X_A - X_B) [M_B^(2) + (M_B^(0)/M_A^(0)) M_A^(2)]_jk
 * (the term n = 1, m = p that the truncation drops; the target's share
 * makes each pair's forces and torques cancel, its sign following the
 * parity of D^(p+1)).
 * Leaf targets only get orders 0 and 1 (nothing below them needs more).
 *   M, com: as written by fmm_upward (read).
 *   L:      device [n_nodes][20][512], written: double (FMM_FP64) or the
 *           float high part (FMM_MIXED, FMM_DFLOAT).  Values are in level units: lengths
 *           in cell widths of the target's level and G factored out, i.e.
 *           L_physical^(n) = G h^-(n+1) L^(n).  Orders 2-3 of leaf nodes are
 *           not written.
 *   L_comp: FMM_MIXED, FMM_DFLOAT: device float [n_nodes][20][512], the
 *           compensation (low) part, L = L + L_comp; FMM_FP64: ignored, may
 *           be NULL.
 *   dL1:    device double [n_nodes][3][512], written, level units
 *           (dL1_physical = G h^-2 dL1).
 * Precision: FMM_FP64 evaluates in double; FMM_MIXED forms the offsets in
 * double, contracts in float with two-sum compensated accumulation, and
 * finishes the correction in double; FMM_DFLOAT evaluates every step (offsets,
 * derivative tensors, contraction, sums) in double-float.
 * Errors: FMM_ERR_INVALID_ARG (NULL tree or buffer, L_comp NULL in FMM_MIXED
 * or FMM_DFLOAT, a FMM_FLAG_HOST_ONLY tree), FMM_ERR_CUDA (a launch failed).
 */
int fmm_m2l(fmm_tree_t tree, const double *M, const double *com, void *L,
            float *L_comp, double *dL1, fmm_stream_t stream);

/*
 * Downward pass (Sec. 4.3, third step), root level first, in FP64:
 *   L64^(n)_child = L^(n)_child + sum_{k=0}^{3-n} (1/k!) L64^(n+k)_parent . d^k,
 *   d = X_child - X_parent,   dL1_acc_child = dL1_child + dL1_acc_parent.
 *   L, L_comp, dL1: as written by fmm_m2l (read; level units).
 *   com:     as written by fmm_upward (read).
 *   L64:     device double [n_nodes][20][512], written, physical units; for
 *            leaf nodes only components 0-3 are written.
 *   dL1_acc: device double [n_nodes][3][512], written, physical units.  It
 *            may be the same buffer as dL1.
 * FMM_MIXED forms the shift increments (the k >= 1 terms) in float from float
 * copies of the parent expansion; FMM_FP64 and FMM_DFLOAT shift in double,
 * FMM_DFLOAT reading L as the double sum L + L_comp.
 * Errors: as fmm_m2l.
 */
int fmm_downward(fmm_tree_t tree, const void *L, const float *L_comp,
                 const double *dL1, const double *com, double *L64,
                 double *dL1_acc, fmm_stream_t stream);

/*
 * Potential and field at leaf cells and the conservation sums, in FP64 (the
 * end of Sec. 4.3's third step; the sums check the momentum and
 * angular-momentum conservation of Sec. 2):
 *   phi = L64^(0), g = -(L64^(1) + dL1_acc), f = m g with m = rho h^3.
 *   phi:    device double [n_leaf][512], written.
 *   g:      device double [n_leaf][3][512], written.
 *   totals: device double [n_trees][8], written: sum f (3), sum x cross f
 *           (3), sum |f|, sum |x cross f|, x measured from the box centre.
 *           The sums are FP64 in a fixed order (deterministic); the per-cell
 *           magnitudes in the last two, which only normalise the first two,
 *           are formed in float.
 *   rho:    as for fmm_upward (read).
 * Errors: FMM_ERR_INVALID_ARG (NULL tree or buffer, a FMM_FLAG_HOST_ONLY
 * tree), FMM_ERR_CUDA (a launch failed).
 */
int fmm_forces(fmm_tree_t tree, const double *L64, const double *dL1_acc,
               const double *rho, double *phi, double *g, double *totals,
               fmm_stream_t stream);

/* Launch-shape knobs of the same-level kernels, for the autotuner
 * (paper_1908_03121_gb300/autotune.py); zeros select the defaults.  No
 * counterpart in the paper: its kernels had one fixed shape (Sec. 5.1). */
typedef struct {
    int32_t mono_subgrids;           /* sub-grids per pass of the monopole kernel:
                                        1, 2 or 4 (float) / 1, 2 (double) */
    int32_t ctas_per_sm;             /* cap on persistent CTAs per SM (0 = occupancy) */
    int32_t dataflow;                /* 1: fmm_step runs the refined levels' shifts and
                                        every leaf's shift and forces as one persistent
                                        launch, each item waiting on its parent's
                                        readiness counter (the device-side counterpart
                                        of the paper's futurization, Sec. 4.1 and
                                        Sec. 5.1) instead of one launch per level */
    int32_t wait_budget_us;          /* budget of one device-side wait, microseconds
                                        (0 = 1 s); on expiry the wait gives up and
                                        FMM_STATUS_TIMEOUT is set */
    int32_t drop_first_producer;     /* test injection, host side: the dataflow queue
                                        leaves out the first node's items, so the waits
                                        on it run out (0 in normal use) */
    int32_t mp_pair_targets;         /* FMM_MIXED: 1 walks each thread's two multipole
                                        target cells through the stencil together
                                        (same results, more work in flight) */
    int32_t mp_items;                /* work item of the multipole kernel: 1 a whole
                                        sub-grid, 2 half a sub-grid (256 cells; more
                                        items to balance a tree with few refined
                                        nodes, the halo staged twice); 0 = 2 when the
                                        tree has fewer refined nodes than twice the
                                        kernel's resident CTAs, else 1.  Same results. */
    int32_t reserved;
} fmm_tuning;

/* Set / read the tree's tuning (host, immediate; affects later launches).
 * Errors: FMM_ERR_INVALID_ARG for NULL or out-of-range values. */
int fmm_set_tuning(fmm_tree_t tree, const fmm_tuning *tuning);
int fmm_get_tuning(fmm_tree_t tree, fmm_tuning *tuning);

/*
 * Input checks that the kernels make while they run (the calls stay
 * asynchronous and capturable); each sets a bit of a status word that the
 * tree keeps on the device until fmm_get_status clears it.
 *   FMM_STATUS_BAD_DENSITY: a leaf density read by the upward pass's P2M
 *     kernel (fmm_upward, fmm_step) was zero, negative or NaN.  The method
 *     needs every cell mass positive: a refined cell's centre of mass, and
 *     the correction's M_B^(0)/M_A^(0), divide by masses (Sec. 4.3 and the
 *     angular-momentum correction).  Zero-density regions take a small
 *     floor instead (the workloads use 1e-10).  The outputs of a step that
 *     set the bit are undefined.
 *   FMM_STATUS_TIMEOUT: a device-side wait of the dataflow pass (fmm_tuning
 *     .dataflow) ran past its budget; the waits give up, the kernel returns,
 *     and the step's outputs are undefined.
 */
enum { FMM_STATUS_BAD_DENSITY = 1, FMM_STATUS_TIMEOUT = 2 };

/* Wait for all work on the device, then store the status word's bits in
 * *status and, if `clear` is nonzero, clear them.  Not for use during stream
 * capture.  Returns FMM_ERR_TIMEOUT (with the bits stored) when
 * FMM_STATUS_TIMEOUT is among them.  Errors: FMM_ERR_INVALID_ARG (NULL,
 * host-only tree), FMM_ERR_CUDA. */
int fmm_get_status(fmm_tree_t tree, int32_t *status, int clear);

/*
 * The whole step of Sec. 4.3 in one call: fmm_upward, fmm_m2l, fmm_downward and
 * fmm_forces on the arguments they take (rho as for fmm_upward and
 * fmm_forces), with the same arithmetic and results.  The passes'
 * independent work is overlapped on a second stream that the tree owns and
 * that forks from and joins back into `stream` through events, so the call
 * can be captured into a CUDA graph: the monopole<-monopole kernel (it needs
 * only leaf masses) runs beside the upward pass of the refined levels, and
 * the roots beside the multipole kernel.  The multipole launch also takes
 * the monopole<-multipole targets once its own queue is empty, and every
 * leaf's shift and forces run as one fused pass, which takes the cell masses
 * from M: the step reads rho in P2M only, so rho may be page-locked host
 * memory as for fmm_upward (the whole input transfer then happens inside
 * the P2M kernel, with no separate copy).
 * With FMM_FLAG_TIMING the four passes run in sequence on `stream` instead.
 * Errors: as the four calls.
 */
int fmm_step(fmm_tree_t tree, const double *rho, double *M, double *com, void *L,
             float *L_comp, double *dL1, double *L64, double *dL1_acc, double *phi,
             double *g, double *totals, fmm_stream_t stream);

/*
 * fmm_forces_noalloc -- the leaf-force pass for callers that cannot allocate
 * device memory.  The paper has no counterpart; it exists for callers such as
 * a framework that owns all device memory through its own pool and forbids
 * side allocations, or a foreign-language host that can pass pointers but not
 * manage CUDA allocations.  Same results as fmm_forces (potential, field and
 * the FP64 conservation sums, same per-cell arithmetic), but it needs no tree
 * handle and allocates nothing: the per-leaf-node partial sums go to a fixed
 * array of 65536 x 8 doubles (4 MiB) that the library holds on every GPU that
 * loads it, until the process exits.
 *   leaf_table: device int32 [n_leaf][6], one row per leaf node in leaf-row
 *               order: node index, level, ix, iy, iz, tree_id (the tree's
 *               descriptor values).  The kernels check every row: node in
 *               [0, n_nodes), level in 1..20, ix, iy, iz in [0, 2^(level-1)),
 *               tree_id in [0, n_trees).  A row that fails is skipped without
 *               any access through it: its phi and g rows are set to NaN, and
 *               the totals of every tree come out NaN.
 *   n_leaf:     1..65536 (FMM_ERR_INVALID_ARG beyond the array's size); rho,
 *               phi and g have n_leaf rows.
 *   n_nodes:    number of nodes of the node-indexed buffers L64 and dL1_acc
 *               (>= n_leaf).
 *   n_trees:    number of trees, 1..65535; totals gets one row per tree.
 *   box_size:   edge of the domain (box_lo does not enter the sums).
 *   L64, dL1_acc, rho, phi, g, totals: as for fmm_forces.
 * Every call shares the fixed array and overwrites the rows it uses before
 * reading them; calls whose work overlaps on the GPU race on it, so serialise
 * them.  The first call on a device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 */
int fmm_forces_noalloc(const int32_t *leaf_table, int64_t n_leaf, int64_t n_nodes,
                       int32_t n_trees, double box_size, const double *L64,
                       const double *dL1_acc, const double *rho, double *phi, double *g,
                       double *totals, fmm_stream_t stream);

/*
 * fmm_check_conversions -- diagnostic, no counterpart in the paper.  The
 * downward and force passes convert between float and double through the
 * IEEE-754 bit fields on the integer pipe (GB300's FP64 unit, which also runs
 * the conversion instructions, bounds those passes).  This checks those
 * conversions against the hardware's on caller-chosen values:
 *   values:   device double [n] (read).
 *   mismatch: device int32 [1], written asynchronously: 0 when every value
 *             converts bit for bit as the hardware does (within the
 *             helpers' domain: normal magnitudes, zeros, infinities, NaNs),
 *             else a bit mask: 1 rounding to nearest, 2 truncation, 4 the
 *             exact widening of a float.
 * Errors: FMM_ERR_INVALID_ARG (NULL buffer, n < 0), FMM_ERR_CUDA.
 */
int fmm_check_conversions(const double *values, int64_t n, int32_t *mismatch,
                          fmm_stream_t stream);

/*
 * Time derivative of the potential and field (Sec. 2: the solver also needs
 * the time derivative of the gravitational field, which couples to the
 * hydrodynamics so that total energy is conserved; the paper gives no
 * formula).  Returned: the exact time derivative of this library's solve
 * along the density's rate of change,
 *   phi_dot = d/dt phi(rho + t rho_dot) at t = 0,   g_dot likewise,
 * including the motion of every refined cell's centre of mass, formed from
 * four fmm_step solves at rho + a rho_dot, a = +-eps, +-2 eps, by the
 * fourth-order central difference
 *   f'(0) ~ [8 (f(eps) - f(-eps)) - (f(2 eps) - f(-2 eps))] / (12 eps)
 * (truncation O(eps^4), rounding about the solve's relative precision / eps:
 * use FMM_FP64 or FMM_DFLOAT; the mixed precision's 1e-7 rounding makes it
 * unsuitable).
 *   rho, rho_dot: device double [n_leaf][512] (read); rho + a rho_dot must
 *            stay positive for |a| <= 2 eps (otherwise
 *            FMM_STATUS_BAD_DENSITY is set and the result is undefined).
 *   eps:     time step of the differences, > 0, in the units of rho_dot.
 *   rho_work: device double [n_leaf][512], 16-byte aligned: scratch.
 *   M ... totals: the buffers of fmm_step, used as scratch (on return they
 *            hold the solve at rho - 2 eps rho_dot).
 *   phi_dot: device double [n_leaf][512], written.
 *   g_dot:   device double [n_leaf][3][512], written.
 * Asynchronous on `stream` (no allocation).  Errors: as fmm_step, and
 * FMM_ERR_INVALID_ARG for eps not positive and finite or a NULL buffer.
 */
int fmm_field_time_derivative(fmm_tree_t tree, const double *rho, const double *rho_dot,
                              double eps, double *rho_work, double *M, double *com, void *L,
                              float *L_comp, double *dL1, double *L64, double *dL1_acc,
                              double *phi, double *g, double *totals, double *phi_dot,
                              double *g_dot, fmm_stream_t stream);

/*
 * Self-consistent-field initial models (Sec. 3 and Sec. 4.2: the initial
 * scenario is assembled with the self-consistent field technique alongside
 * the FMM solver; the method is Hachisu's 1986 SCF).  Polytropes
 * P = K rho^(1 + 1/n) in synchronous rotation about the z axis through the
 * centre of mass: inside star i the enthalpy
 *   H = (n + 1) K_i rho^(1/n) = C_i - Phi + Omega^2 w^2 / 2
 * (w: distance from the axis) vanishes on the star's surface.
 */
typedef struct {
    double n;                        /* polytropic index, > 0 */
    double rho_max[2];               /* maximum density of star 1 (> 0) and star 2
                                        (0: a single star) */
    double point_a[3];               /* surface point of star 1 (H = 0 there) */
    double point_b[3];               /* second surface point of star 1 (rotate only) */
    double point_c[3];               /* surface point of star 2 */
    double centre[2][3];             /* star i's cells: centre within r_lim[i] of
                                        centre[i], on star i's side of x_split */
    double r_lim[2];
    double x_split;                  /* star 1: x < x_split, star 2: x >= x_split */
    double rho_floor;                /* density outside the stars, >= 0 */
    int32_t rotate;                  /* 1: Omega from H = 0 at A and B; 0: Omega = 0 */
    int32_t reserved;
} fmm_scf_params;

typedef struct {
    double omega2;                   /* Omega^2 of this iteration */
    double C[2];                     /* C_1, C_2 */
    double com[3];                   /* centre of mass of the input density */
    double H_max[2];                 /* each star's largest enthalpy (K_i = H_max,i /
                                        ((n + 1) rho_max,i^(1/n))) */
    double phi_points[3];            /* potential at the cells of A, B, C */
    double mass;                     /* total mass of the input density */
} fmm_scf_result;

/*
 * One SCF iteration after a solve of the same tree (e.g. fmm_step on rho):
 *   phi:     device double [n_leaf][512], the potential of rho (read);
 *   rho:     device double [n_leaf][512], the density that phi belongs to;
 *   rho_out: device double [n_leaf][512], receives
 *            max(rho_floor, rho_max,i (H / H_max,i)^n) where H > 0 in star i,
 *            else rho_floor (may be rho itself).
 * The centre of mass is summed per leaf node on the device and over the
 * nodes on the host in a fixed order; the surface conditions hold at the
 * centres of the leaf cells containing A, B, C (w measured there); then
 *   Omega^2 = 2 (Phi_A - Phi_B) / (w_A^2 - w_B^2)   (0 unless rotate),
 *   C_1 = Phi_A - Omega^2 w_A^2 / 2,  C_2 = Phi_C - Omega^2 w_C^2 / 2.
 * Synchronises `stream` twice (the scalars need the potential at three cells
 * and the per-node sums); the density kernel is left enqueued.  Uses the
 * tree's workspace: do not overlap it with other calls on the tree.
 * Errors: FMM_ERR_INVALID_ARG (NULL, host-only tree, a batch of several
 * trees, parameters out of range, a point outside every leaf node, no
 * positive mass, a star with no positive enthalpy), FMM_ERR_CUDA.
 */
int fmm_scf_update(fmm_tree_t tree, const fmm_scf_params *params, const double *phi,
                   const double *rho, double *rho_out, fmm_scf_result *out,
                   fmm_stream_t stream);

/*
 * fmm_peak_rate -- diagnostic, no counterpart in the paper: the denominators
 * of the roofline fractions of the FP32- and FP64-bound kernels, measured on
 * the GPU in use rather than taken from a datasheet.  Enqueues one launch of
 * blocks_per_sm x (number of SMs) CTAs of 256 threads, each thread running
 * 8 independent fused multiply-add chains for iters x 16 steps:
 *   kind 0: float fmaf;  1: the paired FP32 form (two lanes per
 *   instruction);  2: double fma.
 *   sink:  device float [1], written only on a value no chain can reach (it
 *          keeps the chains live; its content is meaningless).
 *   flops: host double, receives the launch's operation count (2 per
 *          multiply-add lane); divide by the launch's CUDA-event time.
 * Changes no GPU setting.  Errors: FMM_ERR_INVALID_ARG (kind outside 0..2,
 * iters outside 1..2^40, blocks_per_sm outside 1..32, NULL pointer),
 * FMM_ERR_CUDA.
 */
int fmm_peak_rate(int32_t kind, int64_t iters, int32_t blocks_per_sm, float *sink,
                  double *flops, fmm_stream_t stream);

/* Release the tree's host and device memory, and its streams and events
 * (synchronises the device first).  NULL is ignored; no error return. */
void fmm_destroy_tree(fmm_tree_t tree);

/* Message of the calling thread's last failed call ("" if none).  The string
 * belongs to the library and stays valid until that thread's next failing
 * call. */
const char *fmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
