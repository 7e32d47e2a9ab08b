"""Element-wise parity of the whole adaptive level-5 binary (cfg3: 1665
sub-grids, 746k leaf cells) against the complete FP64 oracle solve.

Every leaf cell's field and potential, and every same-level result of every
cell (the orders each node defines), are compared, in the launch
configuration the benchmark times (the fused, overlapped step, autotuned
launch shapes).  This covers every target of the persistent work queues, the
monopole<-multipole pair lists and the fused leaf pass.  Bars: FP64 1e-12;
double-float 1e-11 (the oracle and the library round absolute coordinates
differently, about 1e-12 of the box, which the double-float arithmetic then
carries); mixed force error 1e-6.  Net force and torque: FP64 and
double-float 1e-12.  The mixed precision's net torque is recorded against the
1e-12 target as an expected failure: float contraction at every level of
multipole targets leaves 1e-10 to 2e-9 (per-level measurements in the design
notes).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F
from paper_1908_03121_gb300 import autotune
from oracle import oracle as O
from workloads import make_config

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
DFLOAT_TOL = 1e-11
FORCE_TOL = 1e-6
CONSERVATION = 1e-12
ORDER_SLICES = [slice(0, 1), slice(1, 4), slice(4, 10), slice(10, 20)]
_REF = {}


def reference():
    if not _REF:
        c = make_config("cfg3")
        _REF["c"] = c
        _REF["ref"] = O.solve(O.Tree.from_config(c), c["rho"])
    return _REF["c"], _REF["ref"]


def rel_err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def widths(desc):
    return 1.0 / (8.0 * 2.0 ** (desc[:, 0].astype(np.float64) - 1))


def level_to_phys(Llev, desc):
    h = widths(desc)[:, None, None]
    out = np.empty_like(Llev, dtype=np.float64)
    for n, sl in enumerate(ORDER_SLICES):
        out[:, sl] = Llev[:, sl] * h ** (-(n + 1))
    return out


def run(c, precision):
    s = F.Solver(c["desc"], c["theta"], precision=precision)
    s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
    s.step()
    autotune.tune(s)
    s.capture()
    s.replay()
    torch.cuda.synchronize()
    return s


def net(tot):
    return (np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6],
            np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7])


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("dfloat", DFLOAT_TOL),
                                           ("mixed", FORCE_TOL)])
def test_full_tree_fields(precision, tol):
    c, ref = reference()
    s = run(c, precision)
    g, phi = s.g.cpu().numpy(), s.phi.cpu().numpy()
    assert rel_err(g, ref["g"]) <= tol
    assert rel_err(phi, ref["phi"]) <= tol
    nf, nt = net(s.totals.cpu().numpy())
    if precision != "mixed":
        assert np.all(nf <= CONSERVATION) and np.all(nt <= CONSERVATION), (nf, nt)
    s.close()


# The mixed precision compensates orders 0-1 (potential and field) and the
# correction; orders 2-3 of multipole targets are plain float sums of about
# 260 terms that largely cancel (measured up to 2.1e-6 of the level's largest
# coefficient on cfg3).  They reach the forces only through the downward
# shifts, scaled by the children's offsets, and the field of every leaf cell
# is held to 1e-6 above.
MIXED_L_TOL = (2e-6, 2e-6, 1e-5, 1e-5)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("dfloat", DFLOAT_TOL),
                                           ("mixed", MIXED_L_TOL)])
def test_full_tree_same_level_results(precision, tol):
    """Every cell's same-level result (all 20 orders of refined cells, orders
    0-1 of leaf cells, and the correction) from the oracle's own moments,
    per level and order."""
    tols = tol if isinstance(tol, tuple) else (tol,) * 4
    c, ref = reference()
    desc = c["desc"]
    s = F.Solver(desc, c["theta"], precision=precision)
    s.M.copy_(torch.from_numpy(ref["M"]).cuda())
    s.com.copy_(torch.from_numpy(ref["com"]).cuda())
    s.m2l()
    torch.cuda.synchronize()
    Llev = s.L.cpu().numpy().astype(np.float64)
    if s.Lc is not None:
        Llev = Llev + s.Lc.cpu().numpy().astype(np.float64)
    L = level_to_phys(Llev, desc)
    leaf = desc[:, 5] < 0
    for lev in np.unique(desc[:, 0]):
        for n, sl in enumerate(ORDER_SLICES):
            sel = (desc[:, 0] == lev) & (~leaf if n >= 2 else np.ones_like(leaf))
            if not sel.any() or np.abs(ref["L"][sel][:, sl]).max() == 0:
                continue
            e = rel_err(L[sel][:, sl], ref["L"][sel][:, sl])
            assert e <= tols[n], f"level {lev} order {n}: {e:.3e}"
    h = widths(desc)[:, None, None]
    assert rel_err(s.dL1.cpu().numpy() * h ** -2, ref["dL1"]) <= tols[1]
    s.close()


@pytest.mark.xfail(strict=True, reason="float contraction of the multipole targets: net "
                   "torque 1e-10 to 2e-9 of the total at every level (measured), against "
                   "the 1e-12 target; the double-float precision meets it")
def test_full_tree_mixed_conservation_target():
    c, _ = reference()
    s = run(c, "mixed")
    nf, nt = net(s.totals.cpu().numpy())
    s.close()
    assert np.all(nf <= CONSERVATION) and np.all(nt <= CONSERVATION), (nf, nt)
