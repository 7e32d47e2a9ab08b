"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks the oracle against a closed form, a brute-force sum, an
invariant or a fact printed in the paper, chosen so that a plausible slip
(a dropped term, a wrong sign, factorial or index, a transposed operand)
fails at least one of them.  None of these tests needs a GPU.
"""

import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from workloads import (make_config, uniform_tree, adaptive_tree,
                       leaf_cell_centres, leaf_nodes)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# --------------------------------------------------------------- helpers
# independent numpy restatement of the 20-component packing convention
_P2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
_P3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2),
       (1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)]


def unpack20(p):
    t0 = p[0]
    t1 = np.array(p[1:4])
    t2 = np.zeros((3, 3))
    for q, (i, j) in enumerate(_P2):
        t2[i, j] = t2[j, i] = p[4 + q]
    t3 = np.zeros((3, 3, 3))
    for q, idx in enumerate(_P3):
        for perm in itertools.permutations(idx):
            t3[perm] = p[10 + q]
    return t0, t1, t2, t3


def pack20(t0, t1, t2, t3):
    p = np.zeros(20)
    p[0] = t0
    p[1:4] = t1
    for q, (i, j) in enumerate(_P2):
        p[4 + q] = t2[i, j]
    for q, idx in enumerate(_P3):
        p[10 + q] = t3[idx]
    return p


def central_moments(x, m):
    """Mass, centre of mass and central moments of a point set (definition)."""
    M0 = m.sum()
    X = (m[:, None] * x).sum(0) / M0
    s = x - X
    M2 = np.einsum("p,pi,pj->ij", m, s, s)
    M3 = np.einsum("p,pi,pj,pk->ijk", m, s, s, s)
    return M0, X, M2, M3


def taylor_phi(L, r):
    t0, t1, t2, t3 = unpack20(L)
    return (t0 + t1 @ r + 0.5 * np.einsum("ij,i,j", t2, r, r)
            + np.einsum("ijk,i,j,k", t3, r, r, r) / 6.0)


def taylor_grad(L, r):
    _, t1, t2, t3 = unpack20(L)
    return t1 + t2 @ r + 0.5 * np.einsum("ijk,j,k->i", t3, r, r)


def direct_sum(pos, m, G=1.0):
    """O(N^2) point-mass potential and field, self term excluded."""
    N = len(pos)
    phi = np.zeros(N)
    g = np.zeros((N, 3))
    for s in range(0, N, 512):
        d = pos[s:s + 512, None, :] - pos[None, :, :]
        r2 = (d * d).sum(-1)
        rows = np.arange(s, min(s + 512, N))
        r2[rows - s, rows] = np.inf
        ri = 1.0 / np.sqrt(r2)
        phi[s:s + 512] = -G * (m[None, :] * ri).sum(1)
        g[s:s + 512] = -G * ((m[None, :] * ri ** 3)[:, :, None] * d).sum(1)
    return phi, g


def leaf_masses(desc, rho, box_size=1.0):
    levels = desc[leaf_nodes(desc), 0]
    h = box_size / (8 * 2.0 ** (levels - 1))
    return rho * (h ** 3)[:, None]


def flat_g(g):
    return g.transpose(0, 2, 1).reshape(-1, 3)


# ---------------------------------------------------- derivative tensors

def test_dtensors_match_finite_differences():
    rng = np.random.default_rng(10)
    for _ in range(5):
        R = rng.normal(size=3)
        R *= rng.uniform(0.7, 2.0) / np.linalg.norm(R)
        D = O.dtensors(R)
        eps = 1e-4
        for k in range(4):
            fd = np.zeros((3,) + np.shape(D[k]))
            for a in range(3):
                e = np.zeros(3)
                e[a] = eps
                # 4th-order central difference of D^(k) along axis a
                fp1, fm1 = O.dtensors(R + e)[k], O.dtensors(R - e)[k]
                fp2, fm2 = O.dtensors(R + 2 * e)[k], O.dtensors(R - 2 * e)[k]
                fd[a] = (8 * (np.asarray(fp1) - fm1) - (np.asarray(fp2) - fm2)) / (12 * eps)
            # D^(k+1)[a, ...] is the derivative of D^(k) along a
            nxt = np.asarray(D[k + 1])
            want = np.moveaxis(fd, 0, -1) if k > 0 else fd.reshape(3)
            scale = np.abs(nxt).max()
            assert np.abs(nxt - want).max() < 1e-8 * scale
        if True:
            # harmonic: every derivative tensor of order >= 2 is traceless
            assert abs(np.trace(D[2])) < 1e-13 * np.abs(D[2]).max()
            assert np.abs(np.einsum("iij->j", D[3])).max() < 1e-13 * np.abs(D[3]).max()
            assert np.abs(np.einsum("iijk->jk", D[4])).max() < 1e-13 * np.abs(D[4]).max()


def test_dtensors_first_order_closed_form():
    R = np.array([0.3, -1.1, 0.7])
    r = np.linalg.norm(R)
    D0, D1, *_ = O.dtensors(R)
    assert D0 == pytest.approx(1.0 / r, rel=1e-15)
    np.testing.assert_allclose(D1, -R / r ** 3, rtol=1e-14)


# ---------------------------------------------------- one interaction

def _point(M0, X):
    return pack20(M0, np.zeros(3), np.zeros((3, 3)), np.zeros((3, 3, 3))), np.asarray(X, float)


def test_monopole_expansion_has_fourth_order_error():
    """A point source: the local cubic Taylor polynomial misses 1/|x| by O(r^4)."""
    G, m = 1.7, 2.3
    XB = np.array([0.1, 0.2, -0.3])
    XA = XB + np.array([1.0, -0.6, 0.8])
    MA, _ = _point(1.0, XA)
    MB, _ = _point(m, XB)
    L, _ = O.pair_m2l(MA, XA, MB, XB, a_leaf=False, G=G)
    direction = np.array([0.37, 0.51, -0.78])
    errs, gerrs = [], []
    for eps in (0.04, 0.02, 0.01):
        r = eps * direction
        exact = -G * m / np.linalg.norm(XA + r - XB)
        d = XA + r - XB
        gexact = -G * m * d / np.linalg.norm(d) ** 3      # field = -grad phi
        errs.append(abs(taylor_phi(L, r) - exact))
        gerrs.append(np.linalg.norm(-taylor_grad(L, r) - gexact))
    # halving r divides the potential error by 2^4, the field error by 2^3
    for a, b in zip(errs, errs[1:]):
        assert 13.0 < a / b < 19.0
    for a, b in zip(gerrs, gerrs[1:]):
        assert 6.5 < a / b < 9.5


def _cluster(rng, K, centre, size):
    x = centre + size * rng.uniform(-1, 1, size=(K, 3))
    m = rng.uniform(0.5, 1.5, size=K)
    return x, m


def _moments20(x, m):
    M0, X, M2, M3 = central_moments(x, m)
    return pack20(M0, np.zeros(3), M2, M3), X


def test_multipole_source_far_field_orders():
    """Cluster source seen from a point: potential error O((a/R)^4) and,
    with the correction added, field error O((a/R)^4) too; without the
    correction the field error is only O((a/R)^3)."""
    rng = np.random.default_rng(11)
    xu, m = _cluster(rng, 40, np.zeros(3), 1.0)
    XA = np.array([3.1, -2.2, 1.7])
    MA, _ = _point(1.0, XA)
    phi_err, g_err, g_err_nocorr = [], [], []
    for a in (0.2, 0.1, 0.05):
        x = a * xu
        MB, XB = _moments20(x, m)
        L, dL1 = O.pair_m2l(MA, XA, MB, XB, a_leaf=False)
        d = XA - x
        rr = np.linalg.norm(d, axis=1)
        phi_exact = -(m / rr).sum()
        g_exact = -((m / rr ** 3)[:, None] * d).sum(0)
        _, L1, _, _ = unpack20(L)
        phi_err.append(abs(L[0] - phi_exact))
        g_err.append(np.linalg.norm(-(L1 + dL1) - g_exact))
        g_err_nocorr.append(np.linalg.norm(-L1 - g_exact))
    for a, b in zip(phi_err, phi_err[1:]):
        assert 13.0 < a / b < 19.0
    for a, b in zip(g_err, g_err[1:]):
        assert 13.0 < a / b < 19.0
    for a, b in zip(g_err_nocorr, g_err_nocorr[1:]):
        assert 6.5 < a / b < 9.5


def _pair_forces(xa, ma, xb, mb, use_corr=True, corr_sign=1.0, order=3):
    MA, XA = _moments20(xa, ma)
    MB, XB = _moments20(xb, mb)
    LA, dA = O.pair_m2l(MA, XA, MB, XB, a_leaf=False, order=order)
    LB, dB = O.pair_m2l(MB, XB, MA, XA, a_leaf=False, order=order)
    f = []
    for x, m, L, dl, X in ((xa, ma, LA, dA, XA), (xb, mb, LB, dB, XB)):
        for p in range(len(x)):
            g = -(taylor_grad(L, x[p] - X) + (corr_sign * dl if use_corr else 0.0))
            f.append(m[p] * g)
    f = np.array(f)
    x = np.concatenate([xa, xb])
    tau = np.cross(x, f)
    F_rel = np.linalg.norm(f.sum(0)) / np.linalg.norm(f, axis=1).sum()
    T_rel = np.linalg.norm(tau.sum(0)) / np.linalg.norm(tau, axis=1).sum()
    return F_rel, T_rel


def test_two_cluster_momentum_and_torque():
    """Two clusters, expansions evaluated at every point: net force and net
    torque vanish to rounding with the +1/6 correction; without it, or with
    its sign flipped, the net torque is large."""
    rng = np.random.default_rng(12)
    xa, ma = _cluster(rng, 30, np.array([0.1, 0.2, 0.3]), 0.3)
    xb, mb = _cluster(rng, 25, np.array([1.4, -0.7, 0.9]), 0.35)
    F, T = _pair_forces(xa, ma, xb, mb)
    assert F < 1e-14
    assert T < 1e-14
    F0, T0 = _pair_forces(xa, ma, xb, mb, use_corr=False)
    assert F0 < 1e-14          # linear momentum does not need the correction
    assert T0 > 1e-6
    _, Tm = _pair_forces(xa, ma, xb, mb, corr_sign=-1.0)
    assert Tm > 1e-6


# ------------------------------------------------ expansion order 2

def test_order2_two_cluster_momentum_and_torque():
    """At order 2 (truncation n + m <= 2) the correction is the dropped
    n = 1, m = 2 term with the target's share added, because D3 is odd:
    net force and torque then vanish to rounding; without the correction
    the torque is large (the order-3 sign of the target's share would break
    even the net force: a planted mistake in test_oracle_mutants)."""
    rng = np.random.default_rng(12)
    xa, ma = _cluster(rng, 30, np.array([0.1, 0.2, 0.3]), 0.3)
    xb, mb = _cluster(rng, 25, np.array([1.4, -0.7, 0.9]), 0.35)
    F, T = _pair_forces(xa, ma, xb, mb, order=2)
    assert F < 1e-14 and T < 1e-14
    F0, T0 = _pair_forces(xa, ma, xb, mb, use_corr=False, order=2)
    assert F0 < 1e-14 and T0 > 1e-4


def test_order2_point_source_error_orders():
    """A point source at order 2: the local quadratic misses 1/|x| by O(r^3)
    and the field by O(r^2)."""
    G, m = 1.7, 2.3
    XB = np.array([0.1, 0.2, -0.3])
    XA = XB + np.array([1.0, -0.6, 0.8])
    MA, _ = _point(1.0, XA)
    MB, _ = _point(m, XB)
    L, _ = O.pair_m2l(MA, XA, MB, XB, a_leaf=False, G=G, order=2)
    assert np.all(L[10:20] == 0.0)                  # no third-order coefficients
    direction = np.array([0.37, 0.51, -0.78])
    errs, gerrs = [], []
    for eps in (0.04, 0.02, 0.01):
        r = eps * direction
        d = XA + r - XB
        errs.append(abs(taylor_phi(L, r) + G * m / np.linalg.norm(d)))
        gerrs.append(np.linalg.norm(-taylor_grad(L, r) + G * m * d / np.linalg.norm(d) ** 3))
    for a, b in zip(errs, errs[1:]):
        assert 6.5 < a / b < 9.5
    for a, b in zip(gerrs, gerrs[1:]):
        assert 3.2 < a / b < 4.8


def test_order2_solve_conserves_and_is_less_accurate():
    """The whole order-2 solve of cfg1: net force and torque at rounding
    level; against the direct sum its field error lies above order 3's."""
    c = make_config("cfg1")
    pos = leaf_cell_centres(c["desc"]).reshape(-1, 3)
    m = leaf_masses(c["desc"], c["rho"]).reshape(-1)
    _, g_direct = direct_sum(pos, m)
    errs = {}
    for order in (2, 3):
        t = O.Tree(c["desc"], c["theta"], order=order)
        sol = O.solve(t, c["rho"])
        tot = sol["totals"][0]
        assert np.linalg.norm(tot[0:3]) / tot[6] < 1e-13
        assert np.linalg.norm(tot[3:6]) / tot[7] < 1e-13
        errs[order] = np.abs(flat_g(sol["g"]) - g_direct).max() / np.abs(g_direct).max()
    assert errs[3] < errs[2] < 1e-1, errs


# ---------------------------------------------------------- upward

def _small_adaptive():
    def want(lo, hi):
        c = np.array([0.3, 0.6, 0.45])
        d = np.clip(c, lo, hi) - c
        return float(d @ d) < 0.12 ** 2
    return adaptive_tree(want, 4)


def test_upward_matches_definition():
    desc = _small_adaptive()
    rng = np.random.default_rng(13)
    n_leaf = len(leaf_nodes(desc))
    rho = rng.uniform(0.1, 2.0, size=(n_leaf, 512))
    tree = O.Tree(desc, 0.5)
    M, com = O.upward(tree, rho)
    pos = leaf_cell_centres(desc).reshape(-1, 3)
    m = leaf_masses(desc, rho).reshape(-1)
    # cells of every refined node: collect the leaf cells inside each cell box
    for i in range(len(desc)):
        if desc[i, 5] < 0:
            continue
        level, ix, iy, iz = desc[i, :4]
        h = 1.0 / (8 * 2 ** (level - 1))
        for c in (0, 7, 100, 511):
            cx, cy, cz = c % 8, (c // 8) % 8, c // 64
            lo = (np.array([ix, iy, iz]) * 8 + [cx, cy, cz]) * h
            inside = np.all((pos >= lo) & (pos < lo + h), axis=1)
            M0, X, M2, M3 = central_moments(pos[inside], m[inside])
            want = pack20(M0, np.zeros(3), M2, M3)
            np.testing.assert_allclose(com[i, :, c], X, rtol=1e-14, atol=1e-15)
            scale = [abs(M0)] * 4 + [np.abs(M2).max()] * 6 + [np.abs(M3).max() + 1e-300] * 10
            assert np.all(np.abs(M[i, :, c] - want) <= 1e-12 * np.asarray(scale) + 1e-300)


# ---------------------------------------------------------- downward

def test_downward_recentres_cubic_exactly():
    """Random cubic on the root cells, nothing else: after the downward pass
    every cell holds the root polynomial's Taylor coefficients at its own
    centre of mass (orders 0-1 at leaf cells), and the correction passes down
    unchanged."""
    desc = _small_adaptive()
    rng = np.random.default_rng(14)
    n_leaf = len(leaf_nodes(desc))
    tree = O.Tree(desc, 0.5)
    M, com = O.upward(tree, rng.uniform(0.1, 2.0, size=(n_leaf, 512)))
    L = np.zeros((len(desc), 20, 512))
    dL1 = np.zeros((len(desc), 3, 512))
    L[0] = rng.normal(size=(20, 512))
    dL1[0] = rng.normal(size=(3, 512))
    L64, acc = O.downward(tree, com, L, dL1)
    for i in range(1, len(desc)):
        level, ix, iy, iz = desc[i, :4]
        is_leaf = desc[i, 5] < 0
        for c in (0, 63, 300, 511):
            cx, cy, cz = c % 8, (c // 8) % 8, c // 64
            g = (np.array([ix, iy, iz]) * 8 + [cx, cy, cz]) >> (level - 1)
            rc = int(g[0] + 8 * g[1] + 64 * g[2])
            Lr = L[0][:, rc]
            r = com[i, :, c] - com[0, :, rc]
            t0, t1, t2, t3 = unpack20(Lr)
            want0 = taylor_phi(Lr, r)
            want1 = taylor_grad(Lr, r)
            want2 = t2 + t3 @ r
            assert L64[i, 0, c] == pytest.approx(want0, rel=1e-12, abs=1e-12)
            np.testing.assert_allclose(L64[i, 1:4, c], want1, rtol=1e-12, atol=1e-12)
            if not is_leaf:
                np.testing.assert_allclose(L64[i, 4:10, c],
                                           [want2[a, b] for a, b in _P2], atol=1e-12)
                np.testing.assert_allclose(L64[i, 10:20, c], Lr[10:20], atol=1e-13)
            else:
                assert np.all(L64[i, 4:20, c] == 0.0)
            np.testing.assert_allclose(acc[i, :, c], dL1[0][:, rc], rtol=0, atol=1e-15)


# ----------------------------------------------------- whole solve

def _solve_cfg(name, theta=None):
    c = make_config(name, theta=theta)
    tree = O.Tree.from_config(c)
    return c, tree, O.solve(tree, c["rho"], n_threads=0)


def test_all_near_case_equals_direct_sum():
    """theta below 1/(grid diameter): every pair is a leaf-leaf point-point
    interaction, so the solve must equal the O(N^2) sum."""
    c, tree, s = _solve_cfg("cfg1", theta=0.03)
    assert s["counts"][0] == 0 and s["counts"][2] == 4096 * 4095
    pos = leaf_cell_centres(c["desc"]).reshape(-1, 3)
    m = leaf_masses(c["desc"], c["rho"]).reshape(-1)
    phi_d, g_d = direct_sum(pos, m)
    g = flat_g(s["g"])
    assert np.abs(g - g_d).max() <= 1e-13 * np.linalg.norm(g_d, axis=1).max()
    assert np.abs(s["phi"].reshape(-1) - phi_d).max() <= 1e-13 * np.abs(phi_d).max()


def test_direct_sum_error_falls_with_theta():
    c = make_config("cfg1")
    pos = leaf_cell_centres(c["desc"]).reshape(-1, 3)
    m = leaf_masses(c["desc"], c["rho"]).reshape(-1)
    _, g_d = direct_sum(pos, m)
    gmax = np.linalg.norm(g_d, axis=1).max()
    errs = []
    for th in (0.5, 0.35, 0.3):
        _, _, s = _solve_cfg("cfg1", theta=th)
        errs.append(np.abs(flat_g(s["g"]) - g_d).max() / gmax)
    assert errs[0] < 1e-2
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_momentum_invariants(name):
    _, _, s = _solve_cfg(name)
    tot = s["totals"][0]
    assert np.linalg.norm(tot[0:3]) <= 1e-13 * tot[6]
    assert np.linalg.norm(tot[3:6]) <= 1e-13 * tot[7]


def test_mirror_symmetry():
    """Density mirror-symmetric in x: g_x antisymmetric, g_y, g_z symmetric."""
    desc = uniform_tree(2)
    pos = leaf_cell_centres(desc)
    c1 = np.array([0.35, 0.52, 0.47])
    c2 = np.array([0.65, 0.52, 0.47])
    rho = (np.exp(-np.sum((pos - c1) ** 2, -1) / 0.02)
           + np.exp(-np.sum((pos - c2) ** 2, -1) / 0.02) + 1e-10)
    tree = O.Tree(desc, 0.5)
    s = O.solve(tree, rho)
    g = flat_g(s["g"])
    p = pos.reshape(-1, 3)
    key = np.round(p * 1024).astype(np.int64)
    index = {tuple(k): n for n, k in enumerate(key)}
    mirror = np.array([index[(1024 - k[0], k[1], k[2])] for k in key])
    scale = np.linalg.norm(g, axis=1).max()
    assert np.abs(g[:, 0] + g[mirror, 0]).max() < 1e-13 * scale
    assert np.abs(g[:, 1:] - g[mirror, 1:]).max() < 1e-13 * scale


@pytest.mark.parametrize("level,tol", [(2, 1.5e-2), (3, 1.0e-2)])
def test_uniform_sphere_interior_field(level, tol):
    """Uniform sphere (R = 0.25, rho = 1, centred): inside, g = -G M r / R^3
    with M the discrete mass (R taken from it); voxelisation limits the match."""
    desc = uniform_tree(level)
    pos = leaf_cell_centres(desc)
    r = np.linalg.norm(pos - 0.5, axis=-1)
    rho = np.where(r < 0.25, 1.0, 0.0) + 1e-10
    tree = O.Tree(desc, 0.5)
    s = O.solve(tree, rho)
    h = 1.0 / (8 * 2 ** (level - 1))
    Mtot = (rho * h ** 3).sum()
    Reff = (3 * Mtot / (4 * np.pi)) ** (1.0 / 3.0)
    p = (pos - 0.5).reshape(-1, 3)
    rr = r.reshape(-1)
    g_exact = -Mtot * p / Reff ** 3
    inside = rr < 0.8 * Reff
    g = flat_g(s["g"])
    err = np.abs(g[inside] - g_exact[inside]).max() / (Mtot / Reff ** 2)
    assert err < tol
    # inside, phi = -G M (3 R^2 - r^2) / (2 R^3): fit a + b r^2 over interior
    # cells (the point-mass reading drops each cell's own, constant, self
    # potential, which only moves a) and check the curvature b = G M / (2 R^3)
    phi = s["phi"].reshape(-1)[inside]
    A = np.stack([np.ones(inside.sum()), rr[inside] ** 2], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, phi, rcond=None)
    assert b == pytest.approx(0.5 * Mtot / Reff ** 3, rel=2 * tol)
    resid = np.abs(A @ np.array([a, b]) - phi).max()
    assert resid < tol * 1.5 * Mtot / Reff


@pytest.mark.parametrize("theta", [0.5, 0.35])
def test_every_leaf_pair_covered_exactly_once(theta):
    desc = _small_adaptive()
    rng = np.random.default_rng(15)
    n_leaf = len(leaf_nodes(desc))
    w = rng.uniform(0.0, 1.0, size=(n_leaf, 512))
    tree = O.Tree(desc, theta)
    cov = O.coverage(tree, w)
    want = w.sum() - w
    assert np.abs(cov - want).max() < 1e-10 * w.sum()


def test_paper_stencil_size_at_theta_035():
    """The union over the 8 child parities of the same-level partners of an
    interior cell is the paper's 1074-point stencil at theta = 0.35."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    desc = uniform_tree(3)
    tree = O.Tree(desc, 0.35)
    node = [i for i in range(len(desc))
            if desc[i, 0] == 3 and tuple(desc[i, 1:4]) == (1, 1, 1)][0]
    union = set()
    per = []
    for px, py, pz in itertools.product((0, 1), repeat=3):
        off, _ = O.sources(tree, node, px + 8 * py + 64 * pz)
        per.append(len(off))
        union |= {tuple(o) for o in off}
    assert len(union) == facts["stencil_neighbours"]["value"]
    assert 512 * len(union) == facts["interactions_per_launch"]["value"]
    assert len(set(per)) == 1


def test_paper_stencil_theta_05_counts():
    """theta = 0.5: 231 well-separated + 32 near partners per interior cell."""
    desc = uniform_tree(3)
    tree = O.Tree(desc, 0.5)
    node = [i for i in range(len(desc))
            if desc[i, 0] == 3 and tuple(desc[i, 1:4]) == (1, 1, 1)][0]
    off, flg = O.sources(tree, node, 3 + 8 * 4 + 64 * 5)
    far = (flg & 1).astype(bool)
    assert far.sum() == 231 and (~far).sum() == 32
    # near partners are exactly the lattice points with 0 < |o|^2 <= 4
    near = {tuple(o) for o in off[~far]}
    lattice = {o for o in itertools.product(range(-2, 3), repeat=3)
               if 0 < sum(v * v for v in o) <= 4}
    assert near == lattice
