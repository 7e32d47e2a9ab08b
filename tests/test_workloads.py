"""The seeded synthetic inputs follow their recipes.

The workloads stand in for the paper's stellar initial model. These checks
pin the generators against textbook facts (Lane-Emden closed forms and
tabulated zero) and against the stated recipes:
- seeded and reproducible;
- a density floor everywhere;
- the binaries' mass ratio q;
- the batch of sixteen trees;
- the sizes the measurements quote.
No GPU is involved.
"""

import numpy as np
import pytest

from workloads import (DENSITY_FLOOR, count_leaves, lane_emden, leaf_cell_centres, leaf_nodes,
                       make_config)


def test_lane_emden_closed_forms():
    """n = 0: theta = 1 - xi^2/6, first zero sqrt(6); n = 1: theta =
    sin(xi)/xi, first zero pi (RK4 with step 1e-4)."""
    xs, th, xi1 = lane_emden(0.0)
    assert abs(xi1 - np.sqrt(6.0)) < 1e-8
    assert np.abs(th[:-1] - (1.0 - xs[:-1] ** 2 / 6.0)).max() < 1e-10
    xs, th, xi1 = lane_emden(1.0)
    assert abs(xi1 - np.pi) < 1e-8
    inner = (xs > 0.0) & (xs < xi1)
    assert np.abs(th[inner] - np.sin(xs[inner]) / xs[inner]).max() < 1e-10


def test_lane_emden_n15_tabulated_zero():
    """n = 1.5 (the workloads' polytropes): first zero xi_1 = 3.65375, the
    standard tabulated value."""
    _, th, xi1 = lane_emden(1.5)
    assert abs(xi1 - 3.65375) < 1e-5
    assert np.all(np.diff(th) < 0.0)          # monotone from the centre outward


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3"])
def test_seeded_and_floored(name):
    a, b = make_config(name), make_config(name)
    assert np.array_equal(a["desc"], b["desc"]) and np.array_equal(a["rho"], b["rho"])
    assert a["rho"].min() >= DENSITY_FLOOR
    assert a["rho"].shape == (count_leaves(a["desc"]), 512)
    # far from every star or blob only the floor is left
    assert np.isclose(a["rho"].min(), DENSITY_FLOOR, rtol=1e-6, atol=0.0)


def _star_masses(c):
    d = c["desc"]
    pos = leaf_cell_centres(d)
    levels = d[leaf_nodes(d), 0]
    h = 1.0 / (8 * 2.0 ** (levels - 1))
    m = c["rho"] * (h ** 3)[:, None]
    i = c["info"]
    in1 = np.linalg.norm(pos - i["c1"], axis=-1) < i["r1"]
    in2 = np.linalg.norm(pos - i["c2"], axis=-1) < i["r2"]
    return m[in1].sum(), m[in2].sum()


@pytest.mark.parametrize("name,tol", [("cfg2", 3e-3), ("cfg3", 3e-3)])
def test_binary_mass_ratio(name, tol):
    """Two n = 1.5 polytropes with rho_c2 = q^2 rho_c1 and R2 = R1 q^(-1/3)
    (equal K): the sampled masses stand in the ratio q = 0.3."""
    c = make_config(name)
    i = c["info"]
    q = 0.3
    assert i["rho_c2"] == pytest.approx(q * q * i["rho_c1"])
    assert i["r2"] == pytest.approx(i["r1"] * q ** (-1.0 / 3.0))
    m1, m2 = _star_masses(c)
    assert abs(m2 / m1 - q) < tol


def test_contact_binary_cfg5():
    """cfg5: the level-7 contact binary the measurements quote (13,369
    sub-grids, 11,698 leaves); the stars overlap, separation about
    R1 + R2 - 0.1 R1 (centres jittered by at most 0.01 per axis)."""
    c = make_config("cfg5")
    d = c["desc"]
    assert len(d) == 13369 and count_leaves(d) == 11698
    assert d[:, 0].max() == 7
    i = c["info"]
    sep = np.linalg.norm(i["c2"] - i["c1"])
    want = i["r1"] + i["r2"] - 0.1 * i["r1"]
    assert abs(sep - want) <= 0.02 * np.sqrt(3.0) + 1e-12
    assert sep < i["r1"] + i["r2"]                       # in contact
    m1, m2 = _star_masses(c)
    assert abs(m2 / m1 - 0.3) < 0.01


def test_cfg5_small_is_cfg5s_binary_at_level_6():
    """cfg5_small, the profiling case: cfg5's binary (same stars, same
    seed) refined to level 6, with more refined nodes than the multipole
    kernel's 456 resident CTAs."""
    c = make_config("cfg5_small")
    big = make_config("cfg5")
    d = c["desc"]
    assert d[:, 0].max() == 6
    assert len(d) == 5129 and count_leaves(d) == 4488
    assert int((d[:, 5] >= 0).sum()) == 641
    for k in ("c1", "c2", "r1", "r2", "rho_c1", "rho_c2"):
        assert np.array_equal(np.asarray(c["info"][k]), np.asarray(big["info"][k]))


def test_batch_of_sixteen_trees():
    """cfg4: sixteen independent trees, q from 0.1 to 1.0, maximum levels
    cycling 4-7, every tree between 100 and 2000 leaves."""
    c = make_config("cfg4")
    d = c["desc"]
    trees = c["info"]["trees"]
    assert len(trees) == 16 and d[:, 13].max() == 15
    qs = np.sqrt([t["rho_c2"] / t["rho_c1"] for t in trees])
    assert np.allclose(qs, np.linspace(0.1, 1.0, 16))
    assert [t["max_level"] for t in trees] == [4, 5, 6, 7] * 4
    for k, t in enumerate(trees):
        n_leaf = int(((d[:, 13] == k) & (d[:, 5] < 0)).sum())
        assert n_leaf == t["n_leaf"] and 100 <= n_leaf <= 2000
        assert d[d[:, 13] == k, 0].max() <= t["max_level"]
    assert count_leaves(d) == sum(t["n_leaf"] for t in trees) == c["rho"].shape[0]
