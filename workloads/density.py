"""Seeded synthetic density fields sampled at leaf-cell centres.

These stand in for the paper's V1309 initial model (a self-consistent-field
binary), which is not available: sums of 3-D Gaussians, and binaries of two
n = 1.5 polytropes whose Lane-Emden profile is integrated here with RK4.
Every field gets a density floor so that every cell mass is positive.
"""

import numpy as np

DENSITY_FLOOR = 1e-10


def lane_emden(n=1.5, dxi=1e-4):
    """Integrate theta'' + 2 theta'/xi + theta**n = 0 with RK4 to the first zero.

    Returns ``(xi, theta, xi1)`` sampled every ``dxi``; theta(0) = 1,
    theta'(0) = 0.  The series theta = 1 - xi**2/6 + n xi**4/120 starts the
    integration at xi = dxi to step over the removable singularity at 0.
    """
    def rhs(xi, th, dth):
        thn = th ** n if th > 0.0 else 0.0
        return dth, -thn - 2.0 * dth / xi

    xi = dxi
    th = 1.0 - xi ** 2 / 6.0 + n * xi ** 4 / 120.0
    dth = -xi / 3.0 + n * xi ** 3 / 30.0
    xs = [0.0, xi]
    ths = [1.0, th]
    h = dxi
    while th > 0.0:
        a1, b1 = rhs(xi, th, dth)
        a2, b2 = rhs(xi + 0.5 * h, th + 0.5 * h * a1, dth + 0.5 * h * b1)
        a3, b3 = rhs(xi + 0.5 * h, th + 0.5 * h * a2, dth + 0.5 * h * b2)
        a4, b4 = rhs(xi + h, th + h * a3, dth + h * b3)
        th_new = th + h / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4)
        dth_new = dth + h / 6.0 * (b1 + 2 * b2 + 2 * b3 + b4)
        if th_new <= 0.0:
            # linear interpolation of the zero crossing
            xi1 = xi + h * th / (th - th_new)
            xs.append(xi1)
            ths.append(0.0)
            return np.asarray(xs), np.asarray(ths), xi1
        xi += h
        th, dth = th_new, dth_new
        xs.append(xi)
        ths.append(th)
    raise RuntimeError("Lane-Emden integration did not cross zero")


_LE_CACHE = {}


def _le_table(n):
    if n not in _LE_CACHE:
        _LE_CACHE[n] = lane_emden(n)
    return _LE_CACHE[n]


def polytrope(pos, centre, radius, rho_c, n=1.5):
    """Density of one polytrope of index ``n`` at points ``pos`` (..., 3)."""
    xi_tab, th_tab, xi1 = _le_table(n)
    r = np.linalg.norm(pos - np.asarray(centre), axis=-1)
    xi = xi1 * r / radius
    th = np.interp(xi, xi_tab, th_tab, right=0.0)
    return rho_c * np.clip(th, 0.0, None) ** n


def gaussian_blobs(pos, centres, sigma=0.1, peak=1.0):
    """Sum of isotropic Gaussians of width ``sigma`` and height ``peak``."""
    rho = np.zeros(pos.shape[:-1])
    for c in centres:
        d2 = np.sum((pos - np.asarray(c)) ** 2, axis=-1)
        rho += peak * np.exp(-0.5 * d2 / sigma ** 2)
    return rho + DENSITY_FLOOR


def polytrope_binary(pos, c1, c2, r1, r2, rho_c1, rho_c2, n=1.5):
    """Two polytropes plus the density floor (overlaps add)."""
    return (polytrope(pos, c1, r1, rho_c1, n) + polytrope(pos, c2, r2, rho_c2, n)
            + DENSITY_FLOOR)
