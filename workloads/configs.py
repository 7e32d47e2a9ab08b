"""The five seeded workloads (plus theta variants) used by the tests and bench.

Each workload stands in for the paper's V1309 level-14 binary (not available)
with a seeded synthetic field of the same kind -- Gaussian blobs or binaries of
n = 1.5 polytropes -- on octrees of 8^3 sub-grids:

  cfg1  root + 8 leaves (16^3 = 4096 leaf cells); two Gaussians (sigma 0.1,
        peak 1) with centres U[0.3, 0.7]^3 from seed 1; theta = 0.5.
  cfg2  uniform level-3 tree (64 leaves, 32^3 cells); polytrope binary,
        q = 0.3, separation 0.4 along x about the box centre, centres jittered
        by U(-0.01, 0.01)^3 from seed 2; theta = 0.5.
  cfg3  the cfg2 binary on an adaptive tree to level 5: a node is refined iff
        it meets either star's sphere of 1.5 R (about 1500 leaves).
  cfg4  16 independent adaptive trees, seeds 100..115, q = linspace(0.1, 1, 16),
        maximum level cycling 4, 5, 6, 7 (3 to 6 levels below the root),
        100-2000 leaves each.
  cfg5  contact binary (q = 0.3, separation R1 + R2 - 0.1 R1) on an adaptive
        tree to level 7 (about 12000 leaves, 6.1M cells).

Radii: R1 = 0.12 and R2 = R1 q^(-1/3) (equal-K n = 1.5 polytropes have
R ~ M^(-1/3)); central densities rho_c1 = 1 and rho_c2 = q^2 (rho_c ~ M^2 at
fixed K); floor 1e-10 everywhere.
"""

import numpy as np

from .trees import (uniform_tree, adaptive_tree, concat_trees, leaf_cell_centres,
                    count_leaves)
from .density import gaussian_blobs, polytrope_binary

CONFIG_NAMES = ("cfg1", "cfg2", "cfg3", "cfg4", "cfg5")

R1 = 0.12


def _sphere_hit(centre, radius):
    c = np.asarray(centre, dtype=np.float64)

    def hit(lo, hi):
        d = np.clip(c, lo, hi) - c
        return float(d @ d) <= radius * radius
    return hit


def _binary_params(q, separation, seed, jitter=0.01):
    rng = np.random.default_rng(seed)
    r2 = R1 * q ** (-1.0 / 3.0)
    c1 = np.array([0.5 - 0.5 * separation, 0.5, 0.5]) + rng.uniform(-jitter, jitter, 3)
    c2 = np.array([0.5 + 0.5 * separation, 0.5, 0.5]) + rng.uniform(-jitter, jitter, 3)
    return dict(c1=c1, c2=c2, r1=R1, r2=r2, rho_c1=1.0, rho_c2=q * q)


def _binary_tree(p, factor, max_level, tree_id=0):
    h1 = _sphere_hit(p["c1"], factor * p["r1"])
    h2 = _sphere_hit(p["c2"], factor * p["r2"])
    return adaptive_tree(lambda lo, hi: h1(lo, hi) or h2(lo, hi), max_level,
                         tree_id=tree_id)


def _binary_rho(desc, p):
    pos = leaf_cell_centres(desc)
    return polytrope_binary(pos, p["c1"], p["c2"], p["r1"], p["r2"],
                            p["rho_c1"], p["rho_c2"])


# cfg4 refinement factors, tried in order; each tree takes the first one that
# keeps it at or under 2000 leaves
_CFG4_FACTORS = (1.6, 1.4, 1.2, 1.0, 0.85, 0.7, 0.6, 0.5, 0.42, 0.35, 0.3,
                 0.25, 0.2)


def make_config(name, theta=None):
    """Return a dict with desc, rho (n_leaf x 512), theta, G, box and metadata."""
    box_lo = (0.0, 0.0, 0.0)
    box_size = 1.0
    G = 1.0
    if name == "cfg1":
        rng = np.random.default_rng(1)
        centres = rng.uniform(0.3, 0.7, size=(2, 3))
        desc = uniform_tree(2)
        rho = gaussian_blobs(leaf_cell_centres(desc), centres, 0.1, 1.0)
        th = 0.5
        info = dict(centres=centres)
    elif name == "cfg2":
        p = _binary_params(0.3, 0.4, seed=2)
        desc = uniform_tree(3)
        rho = _binary_rho(desc, p)
        th = 0.5
        info = p
    elif name == "cfg3":
        p = _binary_params(0.3, 0.4, seed=2)
        desc = _binary_tree(p, 1.5, 5)
        rho = _binary_rho(desc, p)
        th = 0.5
        info = p
    elif name == "cfg4":
        qs = np.linspace(0.1, 1.0, 16)
        trees, rhos, infos = [], [], []
        for i in range(16):
            max_level = 4 + (i % 4)
            p = _binary_params(float(qs[i]), 0.4, seed=100 + i)
            for factor in _CFG4_FACTORS:
                d = _binary_tree(p, factor, max_level, tree_id=i)
                if count_leaves(d) <= 2000:
                    break
            trees.append(d)
            rhos.append(_binary_rho(d, p))
            infos.append(dict(p, max_level=max_level, factor=factor,
                              n_leaf=count_leaves(d)))
        desc = concat_trees(trees)
        rho = np.concatenate(rhos, axis=0)
        th = 0.5
        info = dict(trees=infos)
    elif name == "cfg5_small":
        # cfg5's binary refined to level 6 (5129 sub-grids, 641 refined):
        # a small case of the same kernels, for profiler captures
        q = 0.3
        r2 = R1 * q ** (-1.0 / 3.0)
        p = _binary_params(q, R1 + r2 - 0.1 * R1, seed=5)
        desc = _binary_tree(p, 1.2, 6)
        rho = _binary_rho(desc, p)
        th = 0.5
        info = p
    elif name == "cfg5":
        q = 0.3
        r2 = R1 * q ** (-1.0 / 3.0)
        p = _binary_params(q, R1 + r2 - 0.1 * R1, seed=5)
        desc = _binary_tree(p, 0.88, 7)
        rho = _binary_rho(desc, p)
        th = 0.5
        info = p
    else:
        raise ValueError(f"unknown workload {name!r}")
    if theta is not None:
        th = float(theta)
    return dict(name=name, desc=np.ascontiguousarray(desc, dtype=np.int32),
                rho=np.ascontiguousarray(rho.reshape(-1, 512), dtype=np.float64),
                theta=th, G=G, box_lo=box_lo, box_size=box_size,
                n_leaf=count_leaves(desc), info=info)
