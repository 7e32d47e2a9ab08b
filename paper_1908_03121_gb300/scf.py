"""Self-consistent-field initial models built on the gravity solve.

The paper's initial model comes from Octo-Tiger's self-consistent field
module iterating the FMM solve (Sec. 3, Sec. 4.2; Hachisu's method).  This
driver alternates the library's two calls on one tree: ``fmm_step`` (the
potential of the current density) and ``fmm_scf_update`` (the density in
hydrostatic equilibrium with it), until the iteration's constants settle.
All per-cell work runs in the library's kernels; this loop only decides
when to stop.
"""

import numpy as np

from . import fmm as B


def binary_params(c1, r1, c2, r2, rho_max, h, n=1.5, r_lim_factor=1.6, rho_floor=1e-10):
    """Parameters of a synchronously rotating binary on the x axis: star 1
    centred at ``c1`` with surface points at x = c1 -+ r1, star 2 at ``c2``
    with its inner surface point at x = c2 - r2; the points sit half a cell
    ``h`` off the y = z = const grid planes through the centres so that each
    lies inside one cell; each star's cells lie within ``r_lim_factor`` times
    its radius of its centre, split at the middle of the gap."""
    c1, c2 = np.asarray(c1, dtype=float), np.asarray(c2, dtype=float)
    off = np.array([0.0, 0.5 * h, 0.5 * h])
    return B.scf_params(n, rho_max, point_a=c1 + off - [r1, 0, 0], point_b=c1 + off + [r1, 0, 0],
                        point_c=c2 + off - [r2, 0, 0], centre=(c1, c2),
                        r_lim=(r_lim_factor * r1, r_lim_factor * r2),
                        x_split=0.5 * (c1[0] + r1 + c2[0] - r2), rho_floor=rho_floor, rotate=True)


def single_star_params(centre, radius, h, rho_max=1.0, n=1.5, r_lim_factor=1.5, rho_floor=1e-10):
    """A static single polytrope with its surface point at x = centre + radius."""
    c = np.asarray(centre, dtype=float)
    a = c + np.array([radius - 0.5 * h, 0.5 * h, 0.5 * h])
    return B.scf_params(n, (rho_max, 0.0), point_a=a, point_c=a, centre=(c, c),
                        r_lim=(r_lim_factor * radius, 0.0), x_split=1e30,
                        rho_floor=rho_floor, rotate=False)


def solve(solver, params, iters=100, tol=1e-6, history=None):
    """Iterate from ``solver.rho`` (updated in place) until Omega^2, C_1 and
    C_2 change by at most ``tol`` relative between iterations, or ``iters``
    iterations.  Returns (the last iteration's scalars, iterations done)."""
    prev = None
    res = None
    for k in range(1, iters + 1):
        solver.step()
        res = B.fmm_scf_update(solver.tree, params, solver.phi, solver.rho, solver.rho)
        if history is not None:
            history.append(res)
        cur = np.array([res["omega2"], res["C"][0], res["C"][1]])
        if prev is not None and np.all(np.abs(cur - prev) <= tol * np.maximum(np.abs(cur), 1e-300)):
            return res, k
        prev = cur
    return res, iters
