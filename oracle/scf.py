"""Self-consistent-field (SCF) initial models, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY: the tests are the only callers; the CUDA library
never imports this module and this module never imports it.

The paper builds its V1309 initial model with Octo-Tiger's self-consistent
field module, which iterates the gravity solve (Sec. 3; Sec. 4.2 assembles
the initial scenario "using the Self-Consistent Field technique alongside
the FMM solver"; the method is Hachisu's 1986 SCF for rotating stars and
binaries).  The paper gives no formulas; this is the published method,
restated step by step for polytropes P = K rho^(1 + 1/n) in synchronous
rotation with angular velocity Omega about the z axis through the centre of
mass:

  hydrostatic equilibrium in the rotating frame: inside star i the enthalpy
      H = (n + 1) K_i rho^(1/n) = C_i - Phi + Omega^2 w^2 / 2,
  w the distance from the rotation axis; H = 0 on each star's surface.

One iteration, from a density rho:
  1. Phi: the FMM potential of rho at every leaf cell (``oracle.solve``);
  2. X: the centre of mass of rho (cell masses rho h^3 at cell centres);
  3. from H = 0 at two surface points A, B of star 1 and one point C of
     star 2 (at the centres of the leaf cells containing them, where the
     potential is known; w measured from X):
        Omega^2 = 2 (Phi_A - Phi_B) / (w_A^2 - w_B^2),
        C_1 = Phi_A - Omega^2 w_A^2 / 2,   C_2 = Phi_C - Omega^2 w_C^2 / 2;
     a static model (``rotate`` false) has Omega^2 = 0 and needs A and C only;
  4. H from the equilibrium equation in each star's region: star 1 takes
     the cell centres with x < x_split within distance r_lim[0] of
     centre[0], star 2 those with x >= x_split within r_lim[1] of centre[1]
     (a reading: the method needs each star confined to its own volume,
     because far from the axis the centrifugal term makes H positive again);
  5. each star's maximum density is held fixed:
        rho' = max(rho_floor, rho_max,i (H / H_max,i)^n) where H > 0,
        rho_floor elsewhere
     (which fixes K_i = H_max,i / ((n + 1) rho_max,i^(1/n))).  The floor
     bounds the density from below everywhere (a reading): the new density
     is then continuous in H, so a cell whose H is zero to rounding takes
     the floor whichever sign the rounding gives.  Without it, such a cell
     would switch between the floor and a density of order 1e-24, which
     moves the centre of mass of its near-vacuum parent cells and, through
     the expansions about them, the next potential by about 1e-6 (measured
     on the level-3 binary).
A single star is star 1 alone (rho_max[1] = 0: no cell is assigned to star 2).
"""

import numpy as np

from . import oracle as O


def leaf_cell_geometry(desc, box_lo=(0.0, 0.0, 0.0), box_size=1.0):
    """Cell centres [n_leaf, 512, 3] and volumes [n_leaf] of the leaf cells,
    in leaf-row order (descriptor order of the leaf nodes)."""
    desc = np.asarray(desc)
    leaves = np.nonzero(desc[:, 5] < 0)[0]
    h = box_size / (8.0 * 2.0 ** (desc[leaves, 0].astype(np.float64) - 1))
    c = np.arange(512)
    loc = np.stack([c & 7, (c >> 3) & 7, c >> 6], axis=1).astype(np.float64)
    pos = (8.0 * desc[leaves, 1:4][:, None, :] + loc[None] + 0.5) * h[:, None, None]
    return pos + np.asarray(box_lo, dtype=np.float64), h ** 3


def cell_at(desc, point, box_lo=(0.0, 0.0, 0.0), box_size=1.0):
    """(leaf row, cell) of the leaf cell containing ``point``."""
    desc = np.asarray(desc)
    p = (np.asarray(point, dtype=np.float64) - np.asarray(box_lo)) / box_size
    leaves = np.nonzero(desc[:, 5] < 0)[0]
    for row, node in enumerate(leaves):
        level, ix, iy, iz = desc[node, 0:4]
        n = 2 ** (level - 1)
        q = p * n - np.array([ix, iy, iz])
        if np.all(q >= 0.0) and np.all(q < 1.0):
            k = np.floor(q * 8.0).astype(int)
            return row, int(k[0] + 8 * k[1] + 64 * k[2])
    raise ValueError("point outside every leaf node")


def regions(pos, params):
    """Boolean masks of the cells of star 1 and star 2."""
    left = pos[..., 0] < params["x_split"]
    d1 = np.linalg.norm(pos - np.asarray(params["centre"][0]), axis=-1)
    d2 = np.linalg.norm(pos - np.asarray(params["centre"][1]), axis=-1)
    return left & (d1 < params["r_lim"][0]), ~left & (d2 < params["r_lim"][1])


def iterate(c, rho, params):
    """One SCF iteration of the workload ``c`` (tree and solve parameters)
    from the density ``rho`` [n_leaf, 512].  ``params``: dict with n,
    rho_max (2), point_a, point_b, point_c (3-vectors), x_split, centre
    (two 3-vectors), r_lim (2), rho_floor, rotate.  Returns (rho', info)
    with info = omega2, C (2), com, H_max (2), phi."""
    tree = O.Tree.from_config(c)
    phi = O.solve(tree, rho)["phi"]
    pos, vol = leaf_cell_geometry(c["desc"], c["box_lo"], c["box_size"])
    m = rho * vol[:, None]
    com = (m[..., None] * pos).sum(axis=(0, 1)) / m.sum()
    w2 = (pos[..., 0] - com[0]) ** 2 + (pos[..., 1] - com[1]) ** 2

    def at(point):
        row, cell = cell_at(c["desc"], point, c["box_lo"], c["box_size"])
        return phi[row, cell], w2[row, cell]

    phi_a, w2_a = at(params["point_a"])
    phi_c, w2_c = at(params["point_c"])
    if params["rotate"]:
        phi_b, w2_b = at(params["point_b"])
        omega2 = 2.0 * (phi_a - phi_b) / (w2_a - w2_b)
    else:
        omega2 = 0.0
    C1 = phi_a - 0.5 * omega2 * w2_a
    C2 = phi_c - 0.5 * omega2 * w2_c
    star1, star2 = regions(pos, params)
    H = np.where(star1, C1, C2) - phi + 0.5 * omega2 * w2
    n = params["n"]
    out = np.full_like(rho, params["rho_floor"])
    hmax = [0.0, 0.0]
    for i, sel in enumerate((star1, star2)):
        if params["rho_max"][i] <= 0.0:
            continue
        live = sel & (H > 0.0)
        if not live.any():
            continue
        hmax[i] = H[live].max()
        out[live] = np.maximum(params["rho_floor"],
                               params["rho_max"][i] * (H[live] / hmax[i]) ** n)
    return out, dict(omega2=omega2, C=(C1, C2), com=com, H_max=tuple(hmax), phi=phi)


def solve(c, rho0, params, iters=60, tol=1e-7):
    """Iterate from ``rho0`` until Omega^2 and both C change by less than
    ``tol`` (relative) or ``iters`` iterations.  Returns (rho, info, k)."""
    rho, prev = rho0, None
    for k in range(1, iters + 1):
        rho, info = iterate(c, rho, params)
        cur = np.array([info["omega2"], info["C"][0], info["C"][1]])
        if prev is not None:
            scale = np.maximum(np.abs(cur), 1e-300)
            if np.all(np.abs(cur - prev) <= tol * scale):
                return rho, info, k
        prev = cur
    return rho, info, iters


def virial(c, rho, info, params):
    """Virial-theorem residual |2T + W + 3 Pi| / |W| of an equilibrium:
    T = sum m Omega^2 w^2 / 2 (rigid rotation), W = sum m Phi / 2,
    Pi = sum P dV with P = K_i rho^(1 + 1/n) inside star i."""
    pos, vol = leaf_cell_geometry(c["desc"], c["box_lo"], c["box_size"])
    m = rho * vol[:, None]
    com = info["com"]
    w2 = (pos[..., 0] - com[0]) ** 2 + (pos[..., 1] - com[1]) ** 2
    n = params["n"]
    T = 0.5 * info["omega2"] * (m * w2).sum()
    W = 0.5 * (m * info["phi"]).sum()
    Pi = 0.0
    for i, sel in enumerate(regions(pos, params)):
        if params["rho_max"][i] <= 0.0 or info["H_max"][i] <= 0.0:
            continue
        K = info["H_max"][i] / ((n + 1.0) * params["rho_max"][i] ** (1.0 / n))
        live = sel & (rho > params["rho_floor"])
        Pi += (K * rho[live] ** (1.0 + 1.0 / n) * np.broadcast_to(vol[:, None], rho.shape)[live]).sum()
    return abs(2.0 * T + W + 3.0 * Pi) / abs(W)
