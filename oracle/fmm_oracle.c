/*
 * Plain, slow FP64 CPU oracle of the cell-based FMM gravity solve
 * (Octo-Tiger, arXiv 1908.03121, Sec. 4.3 "The FMM hotspot").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or constant with the CUDA library and includes none
 * of its files.
 *
 * What it computes, step by step in the paper's order (Sec. 4.3):
 *   1. upward:   cell masses from density (leaf cells, locally homogeneous
 *                density, Sec. 3 and Sec. 4.3) and, for every refined cell, the
 *                multipole moments and centre of mass of the leaf mass below
 *                it (written straight from the definition, not by shifting);
 *   2. same level (M2L): for every cell A and every same-level cell B chosen
 *                by the opening rule, the order-3 Taylor coefficients of B's
 *                potential at A's centre of mass, plus the angular-momentum
 *                correction to A's force coefficient;
 *   3. downward: the parent's Taylor expansion re-centred at each child and
 *                accumulated (Sec. 4.3, third step), then potential and force
 *                at leaf cells and the net force / torque sums.
 *
 * Conventions (readings of the paper; the paper gives no formulas):
 *   - Moments M^(m) are central moments about the cell's centre of mass X:
 *     M^(0) = sum m, M^(1) = 0, M^(2) = sum m s s, M^(3) = sum m s s s.
 *   - phi(X_A + r) = sum_n (1/n!) L^(n) . r^n, with
 *     L^(n)_A = -G sum_B sum_{m: n+m<=3} ((-1)^m / m!) M_B^(m) . D^(n+m)(X_A - X_B)
 *     and D^(k)(R) = k-th derivative tensor of 1/|R|.
 *   - Opening rule (Sec. 4.3: a constant, per-level neighbour count): cells at
 *     integer offset o (in cell widths) are well separated iff theta^2 |o|^2 > 1.
 *     A same-level pair is a candidate iff its parent cells are not well
 *     separated (every pair on the root level is a candidate).  A candidate
 *     pair is evaluated iff it is well separated or either cell is a leaf
 *     cell (its node is not refined).  This gives the four interaction kinds
 *     of Sec. 4.3 (multipole-multipole, multipole-monopole, monopole-monopole,
 *     monopole-multipole).
 *   - Angular-momentum correction (Sec. 2 and Sec. 4.2 name it; its formula is in
 *     the cited Marcello 2017 paper, not here).  Reading: the n = 1, m = 3
 *     term that the n + m <= 3 truncation drops, in the momentum-neutral form
 *       dL1_A,i = +(G/6) sum_jkl D4_ijkl(X_A - X_B) [M3_B - (M0_B/M0_A) M3_A]_jkl,
 *     carried down the tree unchanged and added to the leaf force.
 *   - Leaf force g = -(L^(1) + dL1), potential phi = L^(0), force f = m g.
 *
 * Storage shared with callers (an interface, not code): node descriptors of
 * 14 int32 (level, ix, iy, iz, parent, child[8], tree_id), cells x + 8y + 64z,
 * 20-component packed symmetric tensors (0 | x y z | xx xy xz yy yz zz |
 * xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz), node-major [node][comp][cell].
 */
#include <math.h>
#include <stdint.h>
/* The solve's arithmetic type.  Built as double (the oracle); built with
 * ORACLE_COMPLEX_STEP as double complex, so that a density rho + i h rho_dot
 * carries the exact time derivative of every stage in the imaginary parts
 * (complex-step differentiation: every operation of the solve is analytic in
 * the density, and no difference is formed, so the derivative has no
 * cancellation error). */
#ifdef ORACLE_COMPLEX_STEP
#include <complex.h>
typedef double complex real;
#define SQRT_R csqrt
#else
typedef double real;
#define SQRT_R sqrt
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NSIDE 8
#define NCELL 512
#define DCOLS 14
#define NCOMP 20

/* ------------------------------------------------------------------ tree */

typedef struct {
    int64_t n;
    const int32_t *d;
    double theta, G, lo[3], size;
    int order;              /* expansion order p: 3, or 2 (the truncation n + m <= p) */
    int64_t *leaf_row;      /* node -> density/force row, -1 if refined */
    int max_level;
    int n_trees;
    /* nodes grouped by (tree, level): index list and offsets */
    int64_t *grp_nodes;
    int64_t *grp_off;       /* (n_trees * (max_level + 1) + 1) */
} otree;

static int o_level(const otree *t, int64_t i) { return t->d[DCOLS * i + 0]; }
static int o_coord(const otree *t, int64_t i, int a) { return t->d[DCOLS * i + 1 + a]; }
static int64_t o_parent(const otree *t, int64_t i) { return t->d[DCOLS * i + 4]; }
static int o_is_leaf(const otree *t, int64_t i) { return t->d[DCOLS * i + 5] < 0; }
static int o_tree(const otree *t, int64_t i) { return t->d[DCOLS * i + 13]; }

static double o_width(const otree *t, int level)
{
    return t->size / (NSIDE * ldexp(1.0, level - 1));
}

/* global integer cell coordinates of cell c of node i */
static void o_gcell(const otree *t, int64_t i, int c, int64_t g[3])
{
    int loc[3] = { c % NSIDE, (c / NSIDE) % NSIDE, c / (NSIDE * NSIDE) };
    for (int a = 0; a < 3; ++a) g[a] = (int64_t)NSIDE * o_coord(t, i, a) + loc[a];
}

static void o_centre(const otree *t, int64_t i, int c, real x[3])
{
    int64_t g[3];
    o_gcell(t, i, c, g);
    real h = o_width(t, o_level(t, i));
    for (int a = 0; a < 3; ++a) x[a] = t->lo[a] + ((double)g[a] + 0.5) * h;
}

/* parent cell (node, local cell) of cell c of node i (i must not be a root) */
static void o_parent_cell(const otree *t, int64_t i, int c, int64_t *pn, int *pc)
{
    int64_t p = o_parent(t, i);
    int64_t g[3];
    o_gcell(t, i, c, g);
    int loc[3];
    for (int a = 0; a < 3; ++a) loc[a] = (int)((g[a] >> 1) - (int64_t)NSIDE * o_coord(t, p, a));
    *pn = p;
    *pc = loc[0] + NSIDE * loc[1] + NSIDE * NSIDE * loc[2];
}

static int o_init(otree *t, const int32_t *desc, int64_t n, const double *cfg)
{
    memset(t, 0, sizeof *t);
    t->n = n;
    t->d = desc;
    t->theta = cfg[0];
    t->G = cfg[1];
    t->lo[0] = cfg[2]; t->lo[1] = cfg[3]; t->lo[2] = cfg[4];
    t->size = cfg[5];
    t->order = (int)cfg[6];
    t->leaf_row = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t rows = 0;
    for (int64_t i = 0; i < n; ++i) {
        t->leaf_row[i] = o_is_leaf(t, i) ? rows++ : -1;
        if (o_level(t, i) > t->max_level) t->max_level = o_level(t, i);
        if (o_tree(t, i) + 1 > t->n_trees) t->n_trees = o_tree(t, i) + 1;
    }
    int64_t ng = (int64_t)t->n_trees * (t->max_level + 1);
    t->grp_off = (int64_t *)calloc((size_t)ng + 1, sizeof(int64_t));
    t->grp_nodes = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        t->grp_off[(int64_t)o_tree(t, i) * (t->max_level + 1) + o_level(t, i) + 1]++;
    for (int64_t g = 0; g < ng; ++g) t->grp_off[g + 1] += t->grp_off[g];
    int64_t *fill = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t g = (int64_t)o_tree(t, i) * (t->max_level + 1) + o_level(t, i);
        t->grp_nodes[t->grp_off[g] + fill[g]++] = i;
    }
    free(fill);
    return 0;
}

static void o_free(otree *t)
{
    free(t->leaf_row);
    free(t->grp_off);
    free(t->grp_nodes);
}

/* ------------------------------------------------------ tensor helpers */
/* Tensors are kept as full 3^k arrays, flat index i + 3 j + 9 k + 27 l. */

static const int PK2[6][2] = { {0,0},{0,1},{0,2},{1,1},{1,2},{2,2} };
static const int PK3[10][3] = { {0,0,0},{0,0,1},{0,0,2},{0,1,1},{0,1,2},
                                {0,2,2},{1,1,1},{1,1,2},{1,2,2},{2,2,2} };

/* unpack the 20 packed components of order k into a full 3^k tensor */
static void unpack(const real *p20, int k, real *full)
{
    if (k == 0) { full[0] = p20[0]; return; }
    if (k == 1) { for (int i = 0; i < 3; ++i) full[i] = p20[1 + i]; return; }
    if (k == 2) {
        for (int q = 0; q < 6; ++q) {
            int i = PK2[q][0], j = PK2[q][1];
            full[i + 3 * j] = full[j + 3 * i] = p20[4 + q];
        }
        return;
    }
    for (int q = 0; q < 10; ++q) {
        int a = PK3[q][0], b = PK3[q][1], c = PK3[q][2];
        int perm[6][3] = { {a,b,c},{a,c,b},{b,a,c},{b,c,a},{c,a,b},{c,b,a} };
        for (int s = 0; s < 6; ++s)
            full[perm[s][0] + 3 * perm[s][1] + 9 * perm[s][2]] = p20[10 + q];
    }
}

/* pack a full symmetric tensor of order k into the 20-component layout */
static void pack(const real *full, int k, real *p20)
{
    if (k == 0) { p20[0] = full[0]; return; }
    if (k == 1) { for (int i = 0; i < 3; ++i) p20[1 + i] = full[i]; return; }
    if (k == 2) {
        for (int q = 0; q < 6; ++q) p20[4 + q] = full[PK2[q][0] + 3 * PK2[q][1]];
        return;
    }
    for (int q = 0; q < 10; ++q)
        p20[10 + q] = full[PK3[q][0] + 3 * PK3[q][1] + 9 * PK3[q][2]];
}

static int ipow3(int k) { int r = 1; while (k-- > 0) r *= 3; return r; }

/*
 * Derivative tensors of 1/|R| up to order 4 (explicit Cartesian forms):
 *   D0 = 1/r
 *   D1_i = -R_i / r^3
 *   D2_ij = 3 R_i R_j / r^5 - d_ij / r^3
 *   D3_ijk = -15 R_i R_j R_k / r^7 + 3 (R_i d_jk + R_j d_ik + R_k d_ij) / r^5
 *   D4_ijkl = 105 R_i R_j R_k R_l / r^9
 *             - 15 (R_i R_j d_kl + R_i R_k d_jl + R_i R_l d_jk
 *                   + R_j R_k d_il + R_j R_l d_ik + R_k R_l d_ij) / r^7
 *             + 3 (d_ij d_kl + d_ik d_jl + d_il d_jk) / r^5
 */
void oracle_dtensors(const real R[3], real *D0, real *D1, real *D2,
                     real *D3, real *D4)
{
    real r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    real r = SQRT_R(r2);
    real i1 = 1.0 / r;
    real i3 = i1 / r2, i5 = i3 / r2, i7 = i5 / r2, i9 = i7 / r2;
#define DL(a, b) ((a) == (b) ? 1.0 : 0.0)
    D0[0] = i1;
    for (int i = 0; i < 3; ++i) D1[i] = -R[i] * i3;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            D2[i + 3 * j] = 3.0 * R[i] * R[j] * i5 - DL(i, j) * i3;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                D3[i + 3 * j + 9 * k] = -15.0 * R[i] * R[j] * R[k] * i7
                    + 3.0 * (R[i] * DL(j, k) + R[j] * DL(i, k) + R[k] * DL(i, j)) * i5;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    D4[i + 3 * j + 9 * k + 27 * l] =
                        105.0 * R[i] * R[j] * R[k] * R[l] * i9
                        - 15.0 * (R[i] * R[j] * DL(k, l) + R[i] * R[k] * DL(j, l)
                                  + R[i] * R[l] * DL(j, k) + R[j] * R[k] * DL(i, l)
                                  + R[j] * R[l] * DL(i, k) + R[k] * R[l] * DL(i, j)) * i7
                        + 3.0 * (DL(i, j) * DL(k, l) + DL(i, k) * DL(j, l)
                                 + DL(i, l) * DL(j, k)) * i5;
#undef DL
}

static const double INV_FACT[5] = { 1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0 };

/*
 * One same-level interaction, target A <- source B, in FP64.
 * MA, MB: packed 20-component moments; XA, XB: centres of mass.
 * nmax: highest Taylor order wanted at A (1 for a leaf target, the order p
 * otherwise); order: the expansion order p (3, or 2).
 * Adds to Lfull[n] (full tensors) and dL1[3].
 * The correction is the n = 1, m = p term that the truncation drops, in the
 * form that keeps each pair's forces opposite:
 *   dL1_A = -G ((-1)^p / p!) D^(p+1) : [M_B^(p) + (-1)^p (M0_B / M0_A) M_A^(p)]
 * (D^(p+1) is odd for even p and even for odd p, hence the sign of the
 * target's share); p = 3 is the reading the paper's solver is given, p = 2
 * the same construction one order lower.
 */
static void o_interact(double G, const real *MA, const real XA[3],
                       const real *MB, const real XB[3], int nmax, int order,
                       real *Lfull[4], real dL1[3])
{
    real R[3] = { XA[0] - XB[0], XA[1] - XB[1], XA[2] - XB[2] };
    real D[5][81];
    oracle_dtensors(R, D[0], D[1], D[2], D[3], D[4]);
    real Mf[4][27];
    for (int m = 0; m < 4; ++m) unpack(MB, m, Mf[m]);
    /* L^(n)_alpha += -G ((-1)^m / m!) sum_beta M^(m)_beta D^(n+m)_{alpha beta} */
    for (int n = 0; n <= nmax; ++n) {
        int na = ipow3(n);
        for (int m = 0; n + m <= order; ++m) {
            int nb = ipow3(m);
            double sgn = (m % 2) ? -1.0 : 1.0;
            double coef = -G * sgn * INV_FACT[m];
            for (int a = 0; a < na; ++a) {
                real s = 0.0;
                for (int b = 0; b < nb; ++b) s += Mf[m][b] * D[n + m][a + na * b];
                Lfull[n][a] += coef * s;
            }
        }
    }
    /* angular-momentum correction */
    if (order == 3) {
        real M3A[27];
        unpack(MA, 3, M3A);
        real ratio = MB[0] / MA[0];
        for (int i = 0; i < 3; ++i) {
            real s = 0.0;
            for (int b = 0; b < 27; ++b)
                s += D[4][i + 3 * b] * (Mf[3][b] - ratio * M3A[b]);
            dL1[i] += G / 6.0 * s;
        }
    } else {
        /* p = 2: -(G/2) D3 : [M2_B + (M0_B / M0_A) M2_A] */
        real M2A[9];
        unpack(MA, 2, M2A);
        real ratio2 = MB[0] / MA[0];
        for (int i = 0; i < 3; ++i) {
            real s = 0.0;
            for (int b = 0; b < 9; ++b)
                s += D[3][i + 3 * b] * (Mf[2][b] + ratio2 * M2A[b]);
            dL1[i] -= G / 2.0 * s;
        }
    }
}

/* opening rule: returns 0 (not evaluated) or 1 + kind, kind in 0..3:
 * 0 multipole<-multipole, 1 multipole<-monopole, 2 monopole<-monopole,
 * 3 monopole<-multipole.  far is set to the well-separated flag. */
static int o_pair(const otree *t, int level, const int64_t gA[3], int a_leaf,
                  const int64_t gB[3], int b_leaf, int *far)
{
    int64_t o[3], po[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = gB[a] - gA[a];
        po[a] = (gB[a] >> 1) - (gA[a] >> 1);   /* coordinates are >= 0 */
    }
    if (o[0] == 0 && o[1] == 0 && o[2] == 0) return 0;
    double th2 = t->theta * t->theta;
    if (level > 1) {
        double p2 = (double)(po[0] * po[0] + po[1] * po[1] + po[2] * po[2]);
        if (th2 * p2 > 1.0) return 0;          /* parents well separated */
    }
    double o2 = (double)(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    *far = th2 * o2 > 1.0;
    if (!(*far || a_leaf || b_leaf)) return 0;
    if (!a_leaf) return 1 + (b_leaf ? 1 : 0);
    return 1 + (b_leaf ? 2 : 3);
}

/* largest per-axis cell offset a candidate pair can have */
static int64_t o_reach(const otree *t)
{
    return 2 * (int64_t)floor(1.0 / t->theta) + 1;
}

/* can any cell of node j be a candidate source for a cell of node i? */
static int o_nodes_near(const otree *t, int64_t i, int64_t j)
{
    if (o_level(t, i) == 1) return 1;
    int64_t reach = o_reach(t);
    for (int a = 0; a < 3; ++a) {
        int64_t dn = (int64_t)o_coord(t, j, a) - o_coord(t, i, a);
        if (dn < 0) dn = -dn;
        int64_t gap = dn == 0 ? 0 : NSIDE * dn - (NSIDE - 1);
        if (gap > reach) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------ upward */

/*
 * Cell masses, centres of mass and central moments of every cell.
 * Leaf cells: m = rho h^3 at the cell centre (point-mass reading of the
 * locally homogeneous density; a homogeneous cube adds only an isotropic
 * M^(2), which contracts to zero with every traceless D).  Refined cells: the
 * definition summed directly over all leaf cells below them.
 * rho: [n_leaf][512]; M: [n][20][512]; com: [n][3][512].
 */
int oracle_upward(const int32_t *desc, int64_t n, const double *cfg,
                  const real *rho, real *M, real *com)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    memset(M, 0, sizeof(real) * (size_t)n * NCOMP * NCELL);
    memset(com, 0, sizeof(real) * (size_t)n * 3 * NCELL);
    real *mx = (real *)calloc((size_t)n * 3 * NCELL, sizeof(real));
    /* pass 1: mass and first moment about the origin for every ancestor */
    for (int64_t i = 0; i < n; ++i) {
        if (!o_is_leaf(t, i)) continue;
        real h = o_width(t, o_level(t, i));
        for (int c = 0; c < NCELL; ++c) {
            real m = rho[t->leaf_row[i] * NCELL + c] * h * h * h;
            real x[3];
            o_centre(t, i, c, x);
            int64_t node = i;
            int cell = c;
            for (;;) {
                M[(node * NCOMP + 0) * NCELL + cell] += m;
                for (int a = 0; a < 3; ++a) mx[(node * 3 + a) * NCELL + cell] += m * x[a];
                if (o_parent(t, node) < 0) break;
                int64_t pn; int pc;
                o_parent_cell(t, node, cell, &pn, &pc);
                node = pn; cell = pc;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < NCELL; ++c) {
            real m0 = M[(i * NCOMP + 0) * NCELL + c];
            if (o_is_leaf(t, i)) {
                real x[3];
                o_centre(t, i, c, x);
                for (int a = 0; a < 3; ++a) com[(i * 3 + a) * NCELL + c] = x[a];
            } else {
                for (int a = 0; a < 3; ++a)
                    com[(i * 3 + a) * NCELL + c] = mx[(i * 3 + a) * NCELL + c] / m0;
            }
        }
    free(mx);
    /* pass 2: second and third central moments of every refined ancestor */
    for (int64_t i = 0; i < n; ++i) {
        if (!o_is_leaf(t, i)) continue;
        real h = o_width(t, o_level(t, i));
        for (int c = 0; c < NCELL; ++c) {
            real m = rho[t->leaf_row[i] * NCELL + c] * h * h * h;
            real x[3];
            o_centre(t, i, c, x);
            int64_t node = i;
            int cell = c;
            while (o_parent(t, node) >= 0) {
                int64_t pn; int pc;
                o_parent_cell(t, node, cell, &pn, &pc);
                node = pn; cell = pc;
                real s[3];
                for (int a = 0; a < 3; ++a) s[a] = x[a] - com[(node * 3 + a) * NCELL + cell];
                for (int q = 0; q < 6; ++q)
                    M[(node * NCOMP + 4 + q) * NCELL + cell] += m * s[PK2[q][0]] * s[PK2[q][1]];
                for (int q = 0; q < 10; ++q)
                    M[(node * NCOMP + 10 + q) * NCELL + cell] +=
                        m * s[PK3[q][0]] * s[PK3[q][1]] * s[PK3[q][2]];
            }
        }
    }
    o_free(t);
    return 0;
}

/* --------------------------------------------------------------- M2L */

/* all same-level interactions of target cell c of node i: packed L20 and
 * dL1 (orders above the target's need are zero) */
static void o_m2l_target(const otree *t, const real *M, const real *com,
                         int64_t i, int c, real L20[NCOMP], real dL13[3], int64_t cnt[4])
{
    int level = o_level(t, i);
    int a_leaf = o_is_leaf(t, i);
    int nmax = a_leaf ? 1 : t->order;
    int64_t gA[3];
    o_gcell(t, i, c, gA);
    real MA[NCOMP], XA[3];
    for (int k = 0; k < NCOMP; ++k) MA[k] = M[(i * NCOMP + k) * NCELL + c];
    for (int a = 0; a < 3; ++a) XA[a] = com[(i * 3 + a) * NCELL + c];
    real Lf[4][27];
    memset(Lf, 0, sizeof Lf);
    real *Lp[4] = { Lf[0], Lf[1], Lf[2], Lf[3] };
    real d1[3] = { 0.0, 0.0, 0.0 };
    int64_t g = (int64_t)o_tree(t, i) * (t->max_level + 1) + level;
    for (int64_t q = t->grp_off[g]; q < t->grp_off[g + 1]; ++q) {
        int64_t j = t->grp_nodes[q];
        if (!o_nodes_near(t, i, j)) continue;
        int b_leaf = o_is_leaf(t, j);
        for (int cb = 0; cb < NCELL; ++cb) {
            int64_t gB[3];
            o_gcell(t, j, cb, gB);
            int far;
            int kind = o_pair(t, level, gA, a_leaf, gB, b_leaf, &far);
            if (!kind) continue;
            real MB[NCOMP], XB[3];
            for (int k = 0; k < NCOMP; ++k) MB[k] = M[(j * NCOMP + k) * NCELL + cb];
            for (int a = 0; a < 3; ++a) XB[a] = com[(j * 3 + a) * NCELL + cb];
            o_interact(t->G, MA, XA, MB, XB, nmax, t->order, Lp, d1);
            cnt[kind - 1]++;
        }
    }
    memset(L20, 0, sizeof(real) * NCOMP);
    for (int n = 0; n <= nmax; ++n) pack(Lf[n], n, L20);
    for (int a = 0; a < 3; ++a) dL13[a] = d1[a];
}

/*
 * Same-level interactions for every cell (targets == NULL) or for the listed
 * cells (targets[k] = node * 512 + cell; the other cells are left untouched).
 * L: [n][20][512] (orders 2 and 3 are zero for leaf cells, which never need
 * them); dL1: [n][3][512]; counts[4]: evaluated pairs per kind.  With
 * compact != 0 (targets given), L is [n_targets][20] and dL1 [n_targets][3].
 */
int oracle_m2l(const int32_t *desc, int64_t n, const double *cfg,
               const real *M, const real *com, real *L, real *dL1,
               int64_t *counts, const int64_t *targets, int64_t n_targets,
               int n_threads, int compact)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    int64_t total = targets ? n_targets : n * NCELL;
    if (!targets) compact = 0;
    int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : c0, c1, c2, c3)
#endif
    for (int64_t k = 0; k < total; ++k) {
        int64_t tc = targets ? targets[k] : k;
        int64_t cnt[4] = { 0, 0, 0, 0 };
        int64_t i = tc / NCELL;
        int c = (int)(tc % NCELL);
        real L20[NCOMP], d3[3];
        o_m2l_target(t, M, com, i, c, L20, d3, cnt);
        if (compact) {
            for (int q = 0; q < NCOMP; ++q) L[k * NCOMP + q] = L20[q];
            for (int a = 0; a < 3; ++a) dL1[k * 3 + a] = d3[a];
        } else {
            for (int q = 0; q < NCOMP; ++q) L[(i * NCOMP + q) * NCELL + c] = L20[q];
            for (int a = 0; a < 3; ++a) dL1[(i * 3 + a) * NCELL + c] = d3[a];
        }
        c0 += cnt[0]; c1 += cnt[1]; c2 += cnt[2]; c3 += cnt[3];
    }
    (void)n_threads;
    if (counts) { counts[0] = c0; counts[1] = c1; counts[2] = c2; counts[3] = c3; }
    o_free(t);
    return 0;
}

/*
 * Offsets (in cell widths) of every source evaluated for one target cell,
 * with flags bit0 = well separated, bit1 = source is a leaf cell.
 * Returns the number of sources (at most max_out are written).
 */
int64_t oracle_sources(const int32_t *desc, int64_t n, const double *cfg,
                       int64_t node, int cell, int32_t *offsets, int32_t *flags,
                       int64_t max_out)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    int level = o_level(t, node);
    int a_leaf = o_is_leaf(t, node);
    int64_t gA[3];
    o_gcell(t, node, cell, gA);
    int64_t cnt = 0;
    int64_t g = (int64_t)o_tree(t, node) * (t->max_level + 1) + level;
    for (int64_t q = t->grp_off[g]; q < t->grp_off[g + 1]; ++q) {
        int64_t j = t->grp_nodes[q];
        if (!o_nodes_near(t, node, j)) continue;
        int b_leaf = o_is_leaf(t, j);
        for (int cb = 0; cb < NCELL; ++cb) {
            int64_t gB[3];
            o_gcell(t, j, cb, gB);
            int far;
            if (!o_pair(t, level, gA, a_leaf, gB, b_leaf, &far)) continue;
            if (cnt < max_out) {
                for (int a = 0; a < 3; ++a) offsets[3 * cnt + a] = (int32_t)(gB[a] - gA[a]);
                flags[cnt] = far | (b_leaf << 1);
            }
            cnt++;
        }
    }
    o_free(t);
    return cnt;
}

/*
 * Coverage check of the opening rule: for weights w on leaf cells, returns
 * per leaf cell a the sum, over every evaluated pair (A, B) with a inside A,
 * of the total weight of the leaf cells inside B.  Each other leaf cell is
 * covered exactly once iff this equals sum(w) - w_a.
 */
int oracle_coverage(const int32_t *desc, int64_t n, const double *cfg,
                    const real *w, real *out)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    real *W = (real *)calloc((size_t)n * NCELL, sizeof(real));
    real *cov = (real *)calloc((size_t)n * NCELL, sizeof(real));
    for (int64_t i = 0; i < n; ++i) {
        if (!o_is_leaf(t, i)) continue;
        for (int c = 0; c < NCELL; ++c) {
            real v = w[t->leaf_row[i] * NCELL + c];
            int64_t node = i; int cell = c;
            for (;;) {
                W[node * NCELL + cell] += v;
                if (o_parent(t, node) < 0) break;
                int64_t pn; int pc;
                o_parent_cell(t, node, cell, &pn, &pc);
                node = pn; cell = pc;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        int level = o_level(t, i);
        int a_leaf = o_is_leaf(t, i);
        int64_t g = (int64_t)o_tree(t, i) * (t->max_level + 1) + level;
        for (int c = 0; c < NCELL; ++c) {
            int64_t gA[3];
            o_gcell(t, i, c, gA);
            for (int64_t q = t->grp_off[g]; q < t->grp_off[g + 1]; ++q) {
                int64_t j = t->grp_nodes[q];
                if (!o_nodes_near(t, i, j)) continue;
                int b_leaf = o_is_leaf(t, j);
                for (int cb = 0; cb < NCELL; ++cb) {
                    int64_t gB[3];
                    o_gcell(t, j, cb, gB);
                    int far;
                    if (o_pair(t, level, gA, a_leaf, gB, b_leaf, &far))
                        cov[i * NCELL + c] += W[j * NCELL + cb];
                }
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!o_is_leaf(t, i)) continue;
        for (int c = 0; c < NCELL; ++c) {
            real s = 0.0;
            int64_t node = i; int cell = c;
            for (;;) {
                s += cov[node * NCELL + cell];
                if (o_parent(t, node) < 0) break;
                int64_t pn; int pc;
                o_parent_cell(t, node, cell, &pn, &pc);
                node = pn; cell = pc;
            }
            out[t->leaf_row[i] * NCELL + c] = s;
        }
    }
    free(W);
    free(cov);
    o_free(t);
    return 0;
}

/* ----------------------------------------------------------- downward */

/*
 * Re-centre each parent expansion at the child's centre of mass and add it
 * to the child's own same-level result, root level first:
 *   L'^(n) = L_own^(n) + sum_{k=0}^{3-n} (1/k!) L_parent^(n+k) . d^k,
 *   d = X_child - X_parent;
 * the correction is carried down unchanged: dL1acc = dL1 + dL1acc_parent.
 * Leaf cells only receive orders 0 and 1.
 */
int oracle_downward(const int32_t *desc, int64_t n, const double *cfg,
                    const real *com, const real *L, const real *dL1,
                    real *L64, real *dL1acc)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    memset(L64, 0, sizeof(real) * (size_t)n * NCOMP * NCELL);
    for (int level = 1; level <= t->max_level; ++level) {
        for (int64_t i = 0; i < n; ++i) {
            if (o_level(t, i) != level) continue;
            int nmax = o_is_leaf(t, i) ? 1 : 3;
            for (int c = 0; c < NCELL; ++c) {
                real own[NCOMP];
                for (int k = 0; k < NCOMP; ++k) own[k] = L[(i * NCOMP + k) * NCELL + c];
                real out[NCOMP];
                memset(out, 0, sizeof out);
                real corr[3];
                for (int a = 0; a < 3; ++a) corr[a] = dL1[(i * 3 + a) * NCELL + c];
                if (o_parent(t, i) < 0) {
                    for (int k = 0; k < NCOMP; ++k) out[k] = own[k];
                    if (nmax == 1) for (int k = 4; k < NCOMP; ++k) out[k] = 0.0;
                } else {
                    int64_t pn; int pc;
                    o_parent_cell(t, i, c, &pn, &pc);
                    real Pp[NCOMP];
                    for (int k = 0; k < NCOMP; ++k) Pp[k] = L64[(pn * NCOMP + k) * NCELL + pc];
                    real Pf[4][27];
                    for (int k = 0; k < 4; ++k) unpack(Pp, k, Pf[k]);
                    real d[3];
                    for (int a = 0; a < 3; ++a)
                        d[a] = com[(i * 3 + a) * NCELL + c] - com[(pn * 3 + a) * NCELL + pc];
                    /* powers d^k as full tensors */
                    real dk[4][27];
                    dk[0][0] = 1.0;
                    for (int a = 0; a < 3; ++a) dk[1][a] = d[a];
                    for (int a = 0; a < 9; ++a) dk[2][a] = d[a % 3] * d[a / 3];
                    for (int a = 0; a < 27; ++a) dk[3][a] = d[a % 3] * d[(a / 3) % 3] * d[a / 9];
                    for (int nn = 0; nn <= nmax; ++nn) {
                        int na = ipow3(nn);
                        real shifted[27];
                        for (int a = 0; a < na; ++a) {
                            real s = 0.0;
                            for (int k = 0; nn + k <= 3; ++k) {
                                int nb = ipow3(k);
                                real part = 0.0;
                                for (int b = 0; b < nb; ++b) part += Pf[nn + k][a + na * b] * dk[k][b];
                                s += INV_FACT[k] * part;
                            }
                            shifted[a] = s;
                        }
                        real p20[NCOMP];
                        pack(shifted, nn, p20);
                        int k0 = nn == 0 ? 0 : nn == 1 ? 1 : nn == 2 ? 4 : 10;
                        int k1 = nn == 0 ? 1 : nn == 1 ? 4 : nn == 2 ? 10 : 20;
                        for (int k = k0; k < k1; ++k) out[k] = own[k] + p20[k];
                    }
                    for (int a = 0; a < 3; ++a) corr[a] += dL1acc[(pn * 3 + a) * NCELL + pc];
                }
                for (int k = 0; k < NCOMP; ++k) L64[(i * NCOMP + k) * NCELL + c] = out[k];
                for (int a = 0; a < 3; ++a) dL1acc[(i * 3 + a) * NCELL + c] = corr[a];
            }
        }
    }
    o_free(t);
    return 0;
}

/* ------------------------------------------------------------- forces */

/*
 * Leaf cells: phi = L^(0), g = -(L^(1) + dL1acc), f = m g with m = rho h^3.
 * totals[tree][8] = (sum f, sum x x f, sum |f|, sum |x x f|), x measured from
 * the box centre.  phi: [n_leaf][512]; g: [n_leaf][3][512].
 */
int oracle_forces(const int32_t *desc, int64_t n, const double *cfg,
                  const real *L64, const real *dL1acc, const real *rho,
                  real *phi, real *g, real *totals)
{
    otree T, *t = &T;
    o_init(t, desc, n, cfg);
    memset(totals, 0, sizeof(real) * 8 * (size_t)t->n_trees);
    real ctr[3];
    for (int a = 0; a < 3; ++a) ctr[a] = t->lo[a] + 0.5 * t->size;
    for (int64_t i = 0; i < n; ++i) {
        if (!o_is_leaf(t, i)) continue;
        int64_t row = t->leaf_row[i];
        real h = o_width(t, o_level(t, i));
        real *tot = totals + 8 * o_tree(t, i);
        for (int c = 0; c < NCELL; ++c) {
            real m = rho[row * NCELL + c] * h * h * h;
            phi[row * NCELL + c] = L64[(i * NCOMP + 0) * NCELL + c];
            real gv[3], f[3], x[3], xf[3];
            for (int a = 0; a < 3; ++a) {
                gv[a] = -(L64[(i * NCOMP + 1 + a) * NCELL + c] + dL1acc[(i * 3 + a) * NCELL + c]);
                g[(row * 3 + a) * NCELL + c] = gv[a];
                f[a] = m * gv[a];
            }
            o_centre(t, i, c, x);
            for (int a = 0; a < 3; ++a) x[a] -= ctr[a];
            xf[0] = x[1] * f[2] - x[2] * f[1];
            xf[1] = x[2] * f[0] - x[0] * f[2];
            xf[2] = x[0] * f[1] - x[1] * f[0];
            for (int a = 0; a < 3; ++a) { tot[a] += f[a]; tot[3 + a] += xf[a]; }
            tot[6] += SQRT_R(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
            tot[7] += SQRT_R(xf[0] * xf[0] + xf[1] * xf[1] + xf[2] * xf[2]);
        }
    }
    o_free(t);
    return 0;
}

/*
 * One isolated interaction for unit tests: target A (packed moments MA,
 * centre of mass XA, leaf flag) receives from source B.  Writes the packed
 * 20-component Taylor coefficients (orders above nmax left zero) and the
 * correction dL1[3].
 */
int oracle_pair_m2l(double G, int order, const real *MA, const real *XA,
                    const real *MB, const real *XB, int a_leaf,
                    real *L20, real *dL1)
{
    int nmax = a_leaf ? 1 : order;
    real Lf[4][27];
    memset(Lf, 0, sizeof Lf);
    real *Lp[4] = { Lf[0], Lf[1], Lf[2], Lf[3] };
    real d1[3] = { 0.0, 0.0, 0.0 };
    o_interact(G, MA, XA, MB, XB, nmax, order, Lp, d1);
    memset(L20, 0, sizeof(real) * NCOMP);
    for (int n = 0; n <= nmax; ++n) pack(Lf[n], n, L20);
    for (int a = 0; a < 3; ++a) dL1[a] = d1[a];
    return 0;
}
