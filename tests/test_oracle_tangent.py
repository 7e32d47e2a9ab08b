"""Pins of the oracle's time derivative of the solve (oracle.solve_tangent,
complex-step differentiation of the same C source built on complex numbers).

- Its real part is the real build's solve, bit for bit.
- Homogeneity: the solve is homogeneous of degree one in the density (every
  centre of mass is unchanged by scaling), so rho_dot = rho gives
  phi_dot = phi and g_dot = g exactly.
- Linearity in rho_dot.
- Central differences of the real oracle converge to it at second order.
"""

import numpy as np
import pytest

from oracle import oracle as O
from workloads import make_config


def _case():
    c = make_config("cfg1")
    rho = c["rho"]
    x = np.linspace(0.0, 1.0, rho.size).reshape(rho.shape)
    return c, O.Tree.from_config(c), rho, rho * np.sin(7.0 * x), rho * np.cos(3.0 * x) ** 2


def test_real_part_is_the_solve():
    c, tree, rho, rd, _ = _case()
    t = O.solve_tangent(tree, rho, rd)
    ref = O.solve(tree, rho)
    assert np.array_equal(t["phi"], ref["phi"]) and np.array_equal(t["g"], ref["g"])


def test_scaling_gives_the_solve_itself():
    c, tree, rho, _, _ = _case()
    t = O.solve_tangent(tree, rho, rho)
    ref = O.solve(tree, rho)
    assert np.abs(t["phi_dot"] - ref["phi"]).max() <= 1e-13 * np.abs(ref["phi"]).max()
    assert np.abs(t["g_dot"] - ref["g"]).max() <= 1e-13 * np.abs(ref["g"]).max()


def test_linear_in_the_rate():
    c, tree, rho, r1, r2 = _case()
    a = O.solve_tangent(tree, rho, r1)["phi_dot"]
    b = O.solve_tangent(tree, rho, r2)["phi_dot"]
    ab = O.solve_tangent(tree, rho, r1 - 2.0 * r2)["phi_dot"]
    assert np.abs(ab - (a - 2.0 * b)).max() <= 1e-13 * np.abs(ab).max()


def test_central_differences_converge_at_second_order():
    c, tree, rho, rd, _ = _case()
    t = O.solve_tangent(tree, rho, rd)
    errs = []
    for eps in (4e-3, 2e-3):
        fd = (O.solve(tree, rho + eps * rd)["phi"] - O.solve(tree, rho - eps * rd)["phi"]) / (2 * eps)
        errs.append(np.abs(fd - t["phi_dot"]).max() / np.abs(t["phi_dot"]).max())
    assert errs[1] < 2e-10, errs
    assert errs[0] / errs[1] > 3.0, errs          # second order: about 4
