"""fmm_field_time_derivative (four solves, fourth-order central differences)
against the oracle's exact time derivative (complex step), and the
homogeneity case rho_dot = rho, where the derivative is the solve itself."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F
from paper_1908_03121_gb300 import fmm as B
from oracle import oracle as O
from workloads import make_config
from test_gpu_parity import small_case

pytestmark = pytest.mark.gpu


def rate(rho):
    x = np.linspace(0.0, 1.0, rho.size).reshape(rho.shape)
    return rho * np.sin(7.0 * x)


def gpu_derivative(c, rho_dot, precision, eps):
    s = F.Solver(c["desc"], c["theta"], precision=precision)
    s.rho.copy_(torch.from_numpy(np.ascontiguousarray(c["rho"])).cuda())
    phi_dot = torch.empty_like(s.phi)
    g_dot = torch.empty_like(s.g)
    s.time_derivative(torch.from_numpy(np.ascontiguousarray(rho_dot)).cuda(), eps, phi_dot, g_dot)
    torch.cuda.synchronize()
    assert s.status() == 0
    out = phi_dot.cpu().numpy(), g_dot.cpu().numpy()
    s.close()
    return out


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision", ["fp64", "dfloat"])
@pytest.mark.parametrize("name", ["cfg1", "cfg2", "adaptive4"])
def test_matches_the_oracle(name, precision):
    """Truncation O(eps^4) at eps = 1e-3 and rounding 1e-16 / eps (FP64) or
    1e-14 / eps (double-float): 1e-9 and 1e-8 of the largest value."""
    c = small_case(name)
    rd = rate(c["rho"])
    ref = O.solve_tangent(O.Tree.from_config(c), c["rho"], rd)
    phi_dot, g_dot = gpu_derivative(c, rd, precision, 1e-3)
    tol = 1e-9 if precision == "fp64" else 1e-8
    assert rel(phi_dot, ref["phi_dot"]) <= tol
    assert rel(g_dot, ref["g_dot"]) <= tol


def test_scaling_gives_the_solve_itself():
    c = small_case("adaptive4")
    ref = O.solve(O.Tree.from_config(c), c["rho"])
    phi_dot, g_dot = gpu_derivative(c, c["rho"], "fp64", 1e-2)
    assert rel(phi_dot, ref["phi"]) <= 1e-12
    assert rel(g_dot, ref["g"]) <= 1e-12


def test_full_size_sampled_against_the_oracle():
    """cfg3 (adaptive to level 5) in FP64: every leaf cell against the
    oracle's complete complex-step derivative."""
    c = make_config("cfg3")
    rd = rate(c["rho"])
    ref = O.solve_tangent(O.Tree.from_config(c), c["rho"], rd)
    phi_dot, g_dot = gpu_derivative(c, rd, "fp64", 1e-3)
    assert rel(phi_dot, ref["phi_dot"]) <= 1e-9
    assert rel(g_dot, ref["g_dot"]) <= 1e-9


def test_rejects_a_bad_step():
    c = small_case("cfg1")
    s = F.Solver(c["desc"], c["theta"], precision="fp64")
    out = torch.empty_like(s.phi), torch.empty_like(s.g)
    for eps in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(F.FmmError) as ei:
            s.time_derivative(s.rho, eps, *out)
        assert ei.value.code == B.FMM_ERR_INVALID_ARG
    s.close()
