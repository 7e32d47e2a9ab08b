"""fmm_forces_noalloc: the leaf-force pass for callers that cannot allocate.

Some callers cannot call cudaMalloc -- a framework that owns all device memory
through its own pool, or a foreign-language host that only passes pointers.
fmm_forces_noalloc gives them the force pass with no tree handle and no
allocation; its scratch is a fixed array inside the library.  This file checks
it against fmm_forces (potential and field bit for bit, conservation sums to
the FP64 tolerance of the other tests) on two calls in a row, which reuse the
same fixed array.  It is named so that pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F
from paper_1908_03121_gb300 import fmm as B
from workloads import make_config, leaf_nodes

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
NORM_TOL = 1e-6


def leaf_table(desc):
    leaves = leaf_nodes(desc)
    t = np.zeros((len(leaves), 6), dtype=np.int32)
    t[:, 0] = leaves
    t[:, 1:5] = desc[leaves, 0:4]
    t[:, 5] = desc[leaves, 13]
    return t


@pytest.mark.parametrize("name,precision", [("cfg3", "mixed"), ("cfg4", "fp64")])
def test_forces_noalloc_matches_fmm_forces(name, precision):
    c = make_config(name)
    s = F.Solver(c["desc"], c["theta"], precision=precision)
    s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
    s.step()
    torch.cuda.synchronize()
    ref_phi, ref_g, ref_tot = s.phi.clone(), s.g.clone(), s.totals.cpu().numpy()
    table = torch.from_numpy(leaf_table(c["desc"])).cuda()
    n_leaf, n_trees = table.shape[0], ref_tot.shape[0]
    for _ in range(2):
        phi = torch.full_like(s.phi, float("nan"))
        g = torch.full_like(s.g, float("nan"))
        tot = torch.full_like(s.totals, float("nan"))
        F.fmm_forces_noalloc(table, n_leaf, len(c["desc"]), n_trees, c["box_size"], s.L64,
                             s.dacc, s.rho, phi, g, tot)
        torch.cuda.synchronize()
        assert torch.equal(phi, ref_phi)
        assert torch.equal(g, ref_g)
        got = tot.cpu().numpy()
        # net force / torque sums relative to their normalisers; the two
        # normalisers are built from float per-cell magnitudes, so they get the
        # float tolerance the other force tests give them
        assert np.all(np.abs(got[:, 0:3] - ref_tot[:, 0:3]) <= FP64_TOL * ref_tot[:, 6:7])
        assert np.all(np.abs(got[:, 3:6] - ref_tot[:, 3:6]) <= FP64_TOL * ref_tot[:, 7:8])
        np.testing.assert_allclose(got[:, 6:8], ref_tot[:, 6:8], rtol=NORM_TOL)
    s.close()


def test_forces_noalloc_rejects_oversize():
    with pytest.raises(F.FmmError) as ei:
        F.fmm_forces_noalloc(1, 65537, 65537, 1, 1.0, 1, 1, 1, 1, 1, 1)
    assert ei.value.code == B.FMM_ERR_INVALID_ARG
    assert "65536" in F.fmm_last_error()


@pytest.mark.parametrize("col,value", [(0, 10 ** 6), (0, -1), (1, 0), (1, 21), (2, 9999),
                                       (5, 7), (5, -2)])
def test_forces_noalloc_flags_bad_rows(col, value):
    """A leaf-table row whose node, level, coordinates or tree lie outside
    the caller's buffers is skipped by the kernels (no access through it):
    its field rows and every tree's totals come out NaN, the good rows are
    untouched."""
    c = make_config("cfg1")
    s = F.Solver(c["desc"], c["theta"], precision="fp64")
    s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
    s.step()
    torch.cuda.synchronize()
    t = leaf_table(c["desc"])
    t[3, col] = value
    table = torch.from_numpy(t).cuda()
    phi = torch.zeros_like(s.phi)
    g = torch.zeros_like(s.g)
    tot = torch.zeros_like(s.totals)
    F.fmm_forces_noalloc(table, t.shape[0], len(c["desc"]), 1, c["box_size"], s.L64, s.dacc,
                         s.rho, phi, g, tot)
    torch.cuda.synchronize()
    assert torch.isnan(phi[3]).all() and torch.isnan(g[3]).all()
    good = [r for r in range(t.shape[0]) if r != 3]
    assert torch.equal(phi[good], s.phi[good]) and torch.equal(g[good], s.g[good])
    assert torch.isnan(tot).all()
    s.close()
