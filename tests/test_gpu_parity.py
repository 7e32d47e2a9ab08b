"""GPU parity of the CUDA library (through its C ABI) against the FP64 oracle.

Small trees are compared element by element, stage by stage and end to end;
the full-size workloads (in the launch configuration the benchmark times) are
compared on sampled cells that the oracle computes one by one.  Bars: the
FP64 path to relative 1e-12, the mixed path to relative force error 1e-6
(max |g - g_ref| / max |g_ref|), the double-float (conserving) path to
relative 1e-12 (1e-11 on the full-size samples) with net force and torque
1e-12 of sum |f| and sum |x cross f|.
"""

import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F
from oracle import oracle as O
from workloads import (make_config, uniform_tree, adaptive_tree, concat_trees,
                       leaf_nodes, leaf_cell_centres)
from workloads.density import gaussian_blobs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FORCE_TOL = 1e-6
# The conservation target (net force and net torque relative to sum |f| and
# sum |x cross f|).  The double-float and FP64 precisions meet it; the mixed
# precision's float contraction does not (1e-10 to 2e-9 measured at every
# level of multipole targets), which the expected-failure tests below record.
CONSERVATION_TARGET = 1e-12
MIXED_XFAIL = ("float contraction rounds the two directions of each pair independently: "
               "net torque 1e-10 to 2e-9 at every level of multipole targets (measured), "
               "against the 1e-12 target; the double-float precision meets it")
# Double-float carries about 48 bits (unit roundoff 2^-48 ~ 3.6e-15 per
# operation); a few hundred terms of a hundred operations each put the
# same-level result near 1e-13 relative (measured up to 1.4e-13 on the small
# trees).  On the full-size workloads the oracle itself rounds absolute
# coordinates at 1e-12 (as for the FP64 path), hence the wider sampled bar.
DFLOAT_TOL = 1e-12
DFLOAT_TOL_FULL = 1e-11
# the conservation target of the conserving precision
DFLOAT_CONSERVATION = 1e-12
ORDER_SLICES = [slice(0, 1), slice(1, 4), slice(4, 10), slice(10, 20)]


# ------------------------------------------------------------------ cases
def _adaptive_desc(max_level=4, centre=(0.31, 0.62, 0.45), r=0.12, tree_id=0):
    c = np.asarray(centre)

    def want(lo, hi):
        d = np.clip(c, lo, hi) - c
        return float(d @ d) < r * r
    return adaptive_tree(want, max_level, tree_id=tree_id)


def small_case(name):
    """Small workloads the oracle solves completely in seconds."""
    if name in ("cfg1", "cfg2"):
        return make_config(name)
    if name == "cfg2_t035":
        return make_config("cfg2", theta=0.35)
    # the other two stencil reaches (theta in (1/2, 1/sqrt 3] gives reach 3,
    # theta in (1/4, 1/3] reach 7); 0.5 and 0.35 both give reach 5
    if name == "cfg2_t055":
        return make_config("cfg2", theta=0.55)
    if name == "adaptive4_t030":
        c = small_case("adaptive4")
        c["theta"] = 0.3
        return c
    rng = np.random.default_rng(7)
    if name == "adaptive4":
        desc = _adaptive_desc()
    elif name == "single":
        # degenerate: one leaf sub-grid, no refined node, no M2M level, every
        # pair on the root level (the root kernel's leaf path only)
        desc = uniform_tree(1)
    elif name == "singles2":
        # two independent single-sub-grid trees solved in one batch
        desc = concat_trees([uniform_tree(1), uniform_tree(1)])
    elif name == "batch3":
        desc = concat_trees([uniform_tree(2), _adaptive_desc(4),
                             _adaptive_desc(3, centre=(0.7, 0.2, 0.5), r=0.2)])
    else:
        raise ValueError(name)
    pos = leaf_cell_centres(desc)
    rho = gaussian_blobs(pos, rng.uniform(0.3, 0.7, size=(3, 3)), 0.08, 1.0)
    return dict(name=name, desc=desc, rho=rho.reshape(-1, 512), theta=0.5, G=1.0,
                box_lo=(0.0, 0.0, 0.0), box_size=1.0)


SMALL = ["cfg1", "cfg2", "cfg2_t035", "cfg2_t055", "adaptive4", "adaptive4_t030", "batch3",
         "single", "singles2"]
_ORACLE = {}


def oracle_solution(name):
    if name not in _ORACLE:
        c = small_case(name)
        _ORACLE[name] = (c, O.solve(O.Tree.from_config(c), c["rho"]))
    return _ORACLE[name]


# ---------------------------------------------------------------- helpers
def widths(desc, box_size=1.0):
    return box_size / (8.0 * 2.0 ** (desc[:, 0].astype(np.float64) - 1))


def level_to_phys(Llev, desc, G=1.0):
    """Level units -> physical: L^(n) * G h^-(n+1)."""
    h = widths(desc)[:, None, None]
    out = np.empty_like(Llev, dtype=np.float64)
    for n, sl in enumerate(ORDER_SLICES):
        out[:, sl] = Llev[:, sl] * G * h ** (-(n + 1))
    return out


def phys_to_level(L, desc, G=1.0):
    h = widths(desc)[:, None, None]
    out = np.empty_like(L)
    for n, sl in enumerate(ORDER_SLICES):
        out[:, sl] = L[:, sl] / (G * h ** (-(n + 1)))
    return out


def rel_err(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def solve_gpu(c, precision):
    s = F.Solver(c["desc"], c["theta"], precision=precision, G=c["G"], box_lo=c["box_lo"],
                 box_size=c["box_size"])
    s.rho.copy_(dev(c["rho"]))
    s.step()
    torch.cuda.synchronize()
    return s


def defined_L_mask(desc):
    """L slots the library defines: all 20 for refined nodes, 0-3 for leaves."""
    m = np.ones((len(desc), 20, 1), dtype=bool)
    m[desc[:, 5] < 0, 4:, :] = False
    return m


def assert_L_close(L, Lref, desc, tol):
    mask = np.broadcast_to(defined_L_mask(desc), L.shape)
    for n, sl in enumerate(ORDER_SLICES):
        for lev in np.unique(desc[:, 0]):
            sel = desc[:, 0] == lev
            a = np.where(mask[sel, sl], L[sel, sl], 0.0)
            b = np.where(mask[sel, sl], Lref[sel, sl], 0.0)
            if np.abs(b).max() == 0:
                continue
            e = rel_err(a, b)
            assert e <= tol, f"order {n} level {lev}: rel err {e:.3e}"


def tree_torque(tot):
    return np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7]


def tree_force(tot):
    return np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6]


# ------------------------------------------------------- stage by stage
@pytest.mark.parametrize("name", SMALL)
def test_upward_parity(name):
    c, ref = oracle_solution(name)
    s = solve_gpu(c, "fp64")
    M, com = host(s.M), host(s.com)
    refined = c["desc"][:, 5] >= 0
    assert rel_err(M[:, 0], ref["M"][:, 0]) <= FP64_TOL
    if refined.any():
        assert rel_err(M[refined][:, 4:10], ref["M"][refined][:, 4:10]) <= FP64_TOL
        assert rel_err(M[refined][:, 10:20], ref["M"][refined][:, 10:20]) <= FP64_TOL
        assert np.all(M[refined][:, 1:4] == 0.0)
        assert np.abs(com[refined] - ref["com"][refined]).max() <= FP64_TOL * 1.0
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_m2l_parity_fp64(name):
    """The oracle's moments in, the GPU same-level pass out, FP64."""
    c, ref = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision="fp64")
    s.M.copy_(dev(ref["M"]))
    s.com.copy_(dev(ref["com"]))
    s.m2l()
    torch.cuda.synchronize()
    L = level_to_phys(host(s.L), c["desc"])
    assert_L_close(L, ref["L"], c["desc"], FP64_TOL)
    h = widths(c["desc"])[:, None, None]
    assert rel_err(host(s.dL1) * h ** -2, ref["dL1"]) <= FP64_TOL
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_m2l_parity_mixed(name):
    """Mixed precision: float contraction with compensated sums."""
    c, ref = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision="mixed")
    s.M.copy_(dev(ref["M"]))
    s.com.copy_(dev(ref["com"]))
    s.m2l()
    torch.cuda.synchronize()
    Llev = host(s.L).astype(np.float64) + host(s.Lc).astype(np.float64)
    assert_L_close(level_to_phys(Llev, c["desc"]), ref["L"], c["desc"], 2e-6)
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_m2l_parity_dfloat(name):
    """Double-float precision: every same-level operation on float pairs."""
    c, ref = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision="dfloat")
    s.M.copy_(dev(ref["M"]))
    s.com.copy_(dev(ref["com"]))
    s.m2l()
    torch.cuda.synchronize()
    Llev = host(s.L).astype(np.float64) + host(s.Lc).astype(np.float64)
    assert_L_close(level_to_phys(Llev, c["desc"]), ref["L"], c["desc"], DFLOAT_TOL)
    h = widths(c["desc"])[:, None, None]
    assert rel_err(host(s.dL1) * h ** -2, ref["dL1"]) <= DFLOAT_TOL
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_downward_and_forces_parity(name):
    """The oracle's same-level result in, GPU downward + forces out (FP64)."""
    c, ref = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision="fp64")
    s.com.copy_(dev(ref["com"]))
    s.L.copy_(dev(phys_to_level(ref["L"], c["desc"])))
    h = widths(c["desc"])[:, None, None]
    s.dL1.copy_(dev(ref["dL1"] * h ** 2))
    s.rho.copy_(dev(c["rho"]))
    s.downward()
    s.forces()
    torch.cuda.synchronize()
    assert_L_close(host(s.L64), ref["L64"], c["desc"], FP64_TOL)
    assert rel_err(host(s.dacc), ref["dL1acc"]) <= FP64_TOL
    assert rel_err(host(s.phi), ref["phi"]) <= FP64_TOL
    assert rel_err(host(s.g), ref["g"]) <= FP64_TOL
    tot, rt = host(s.totals), ref["totals"]
    # sum |f| and sum |x cross f| only normalise the net sums: the library
    # forms the per-cell magnitudes in float (the sums themselves are FP64)
    np.testing.assert_allclose(tot[:, 6:8], rt[:, 6:8], rtol=1e-6)
    assert np.all(np.abs(tot[:, 0:6] - rt[:, 0:6]) <= 1e-13 * rt[:, 6:7].max())
    s.close()


# --------------------------------------------------------- end to end
@pytest.mark.parametrize("name", SMALL)
def test_end_to_end_fp64(name):
    c, ref = oracle_solution(name)
    s = solve_gpu(c, "fp64")
    assert rel_err(host(s.g), ref["g"]) <= FP64_TOL
    assert rel_err(host(s.phi), ref["phi"]) <= FP64_TOL
    tot = host(s.totals)
    assert np.all(tree_force(tot) <= 1e-13)
    assert np.all(tree_torque(tot) <= 1e-13)
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_end_to_end_mixed(name):
    """Force error against the FP64 oracle within the 1e-6 bar."""
    c, ref = oracle_solution(name)
    s = solve_gpu(c, "mixed")
    g, gref = host(s.g), ref["g"]
    assert rel_err(g, gref) <= FORCE_TOL
    assert rel_err(host(s.phi), ref["phi"]) <= FORCE_TOL
    s.close()


@pytest.mark.xfail(reason=MIXED_XFAIL)
@pytest.mark.parametrize("name", ["cfg1", "cfg2", "adaptive4", "batch3"])
def test_mixed_conservation_target(name):
    """The 1e-12 conservation target, on the mixed precision."""
    c, _ = oracle_solution(name)
    s = solve_gpu(c, "mixed")
    tot = host(s.totals)
    s.close()
    assert np.all(tree_force(tot) <= CONSERVATION_TARGET), tree_force(tot)
    assert np.all(tree_torque(tot) <= CONSERVATION_TARGET), tree_torque(tot)


@pytest.mark.parametrize("name", SMALL)
def test_end_to_end_dfloat(name):
    """The conserving precision: oracle field to 1e-11, net force and torque
    to 1e-12 of their normalisers."""
    c, ref = oracle_solution(name)
    s = solve_gpu(c, "dfloat")
    assert rel_err(host(s.g), ref["g"]) <= DFLOAT_TOL
    assert rel_err(host(s.phi), ref["phi"]) <= DFLOAT_TOL
    tot = host(s.totals)
    assert np.all(tree_force(tot) <= DFLOAT_CONSERVATION), tree_force(tot)
    assert np.all(tree_torque(tot) <= DFLOAT_CONSERVATION), tree_torque(tot)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "dfloat"])
def test_deterministic_and_graph_replay(precision):
    c, _ = oracle_solution("adaptive4")
    s = solve_gpu(c, precision)
    g1, t1 = host(s.g).copy(), host(s.totals).copy()
    s.step()
    torch.cuda.synchronize()
    assert np.array_equal(host(s.g), g1) and np.array_equal(host(s.totals), t1)
    s.capture()
    s.g.zero_()
    s.totals.zero_()
    s.replay()
    torch.cuda.synchronize()
    assert np.array_equal(host(s.g), g1) and np.array_equal(host(s.totals), t1)
    s.close()


def test_misaligned_density_is_refused():
    """P2M moves the density and the leaf masses as 16-byte vectors: a
    misaligned pointer is an argument error, found before any launch."""
    c, _ = oracle_solution("cfg1")
    s = F.Solver(c["desc"], c["theta"], precision="mixed")
    buf = torch.zeros(s.rho.numel() + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FmmError):
        F.fmm_upward(s.tree, buf[1:].data_ptr(), s.M, s.com)
    with pytest.raises(F.FmmError):
        s.step(buf[1:])
    torch.cuda.synchronize()
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_reads_pinned_host_density(precision):
    """fmm_step with the density in page-locked host memory (read by the P2M
    kernel over the host link) gives the same bits as with a device copy,
    eagerly and from a captured graph."""
    c, _ = oracle_solution("adaptive4")
    s = F.Solver(c["desc"], c["theta"], precision=precision, G=c["G"], box_lo=c["box_lo"],
                 box_size=c["box_size"])
    rho_host = torch.from_numpy(np.ascontiguousarray(c["rho"])).pin_memory()
    s.rho.copy_(rho_host.cuda())
    s.step()
    torch.cuda.synchronize()
    ref = [host(t).copy() for t in (s.g, s.phi, s.totals)]
    for t in (s.g, s.phi, s.totals):
        t.fill_(float("nan"))
    s.step(rho_host)
    torch.cuda.synchronize()
    for a, b in zip([host(t) for t in (s.g, s.phi, s.totals)], ref):
        assert np.array_equal(a, b)
    s.capture(rho=rho_host)
    for t in (s.g, s.phi, s.totals):
        t.fill_(float("nan"))
    s.replay()
    torch.cuda.synchronize()
    for a, b in zip([host(t) for t in (s.g, s.phi, s.totals)], ref):
        assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan")])
def test_non_positive_density_sets_the_status_word(bad):
    """A leaf density that is zero, negative or NaN sets
    FMM_STATUS_BAD_DENSITY during the step (the calls stay asynchronous);
    fmm_get_status reads and clears it, and a valid density leaves it clear."""
    c, _ = oracle_solution("adaptive4")
    s = F.Solver(c["desc"], c["theta"], precision="mixed", G=c["G"], box_lo=c["box_lo"],
                 box_size=c["box_size"])
    s.rho.copy_(dev(c["rho"]))
    s.step()
    assert s.status() == 0
    s.rho[3, 77] = bad
    s.step()
    assert s.status(clear=False) == F.FMM_STATUS_BAD_DENSITY
    assert s.status() == F.FMM_STATUS_BAD_DENSITY          # read, then cleared
    assert s.status() == 0
    s.upward()                                             # the pass call checks too
    assert s.status() == F.FMM_STATUS_BAD_DENSITY
    s.rho.copy_(dev(c["rho"]))
    s.capture()
    s.replay()
    assert s.status() == 0
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_run_stream_matches_single_steps(precision):
    """Solver.run_stream (next density copied during the current step, two
    device buffers and graphs) gives, for every step, the same totals bits
    as one step() per density, in order, and leaves the last step's field."""
    c, _ = oracle_solution("adaptive4")
    s = F.Solver(c["desc"], c["theta"], precision=precision, G=c["G"], box_lo=c["box_lo"],
                 box_size=c["box_size"])
    base = np.ascontiguousarray(c["rho"])
    rhos = [torch.from_numpy(base * f).pin_memory() for f in (1.0, 1.5, 0.75, 2.0, 1.25)]
    ref_tot, ref_g = [], None
    for r in rhos:
        s.rho.copy_(r.cuda())
        s.step()
        torch.cuda.synchronize()
        ref_tot.append(host(s.totals).copy())
        ref_g = host(s.g).copy()
    s.rho.copy_(rhos[0].cuda())
    got = {}
    before = []
    n = s.run_stream(rhos, lambda k, t: got.__setitem__(k, t.numpy().copy()),
                     lambda: before.append(1))
    assert n == len(rhos) and len(before) == len(rhos)
    assert sorted(got) == list(range(len(rhos)))
    for k in range(len(rhos)):
        assert np.array_equal(got[k], ref_tot[k]), k
    assert np.array_equal(host(s.g), ref_g)
    # a second stream reuses the captured graphs; a wrong input is refused
    got.clear()
    s.run_stream(rhos[::-1], lambda k, t: got.__setitem__(k, t.numpy().copy()))
    for k in range(len(rhos)):
        assert np.array_equal(got[k], ref_tot[len(rhos) - 1 - k]), k
    with pytest.raises(ValueError):
        s.run_stream([torch.from_numpy(base)])           # not page-locked
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "dfloat"])
@pytest.mark.parametrize("name", ["adaptive4", "batch3", "cfg2"])
def test_fused_step_matches_passes(name, precision):
    """fmm_step (passes overlapped on two streams) gives the same bits as the
    four pass calls in sequence."""
    c, _ = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision=precision, G=c["G"], box_lo=c["box_lo"],
                 box_size=c["box_size"])
    s.rho.copy_(dev(c["rho"]))
    s.step_passes()
    torch.cuda.synchronize()
    ref = [host(t).copy() for t in (s.M, s.com, s.dL1, s.L64, s.dacc, s.phi, s.g, s.totals)]
    for t in (s.M, s.com, s.L, s.dL1, s.L64, s.dacc, s.phi, s.g, s.totals):
        t.fill_(float("nan"))
    if s.Lc is not None:
        s.Lc.fill_(float("nan"))
    s.step()
    torch.cuda.synchronize()
    got = [host(t) for t in (s.M, s.com, s.dL1, s.L64, s.dacc, s.phi, s.g, s.totals)]
    refined = c["desc"][:, 5] >= 0
    # slots the library writes: M (refined nodes, and M0 of leaves), com
    # (refined nodes), L64 (orders 0-1 of leaves)
    m_mask = np.broadcast_to(refined[:, None, None] | (np.arange(20) == 0)[None, :, None],
                             got[0].shape)
    com_mask = np.broadcast_to(refined[:, None, None], got[1].shape)
    l_mask = np.broadcast_to(defined_L_mask(c["desc"]), got[3].shape)
    masks = [m_mask, com_mask, None, l_mask, None, None, None, None]
    for a, b, m in zip(got, ref, masks):
        if m is not None:
            a, b = a[m], b[m]
        assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "dfloat"])
def test_tunings_agree_bitwise(precision):
    """Launch shapes change scheduling only: every tuning gives the same bits."""
    c, _ = oracle_solution("adaptive4")
    s = solve_gpu(c, precision)
    ref = None
    for nb, cap, pair, items in itertools.product((1, 2, 4), (0, 1), (0, 1), (1, 2)):
        if precision != "mixed" and (nb == 4 or pair):
            continue
        if pair and items == 2:     # the paired kernel always takes whole sub-grids
            continue
        F.fmm_set_tuning(s.tree, mono_subgrids=nb, ctas_per_sm=cap, mp_pair_targets=pair,
                         mp_items=items)
        got = F.fmm_get_tuning(s.tree)
        assert ((got["mono_subgrids"], got["ctas_per_sm"], got["mp_pair_targets"], got["mp_items"])
                == (nb, cap, pair, items))
        s.L.zero_()
        s.m2l()
        torch.cuda.synchronize()
        got = (host(s.L).copy(), None if s.Lc is None else host(s.Lc).copy(), host(s.dL1).copy())
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert a is None or np.array_equal(a, b)
    s.close()


def test_in_tree_library_is_the_one_loaded():
    F.load()
    maps = open("/proc/self/maps").read()
    assert F.library_path() in maps


# ------------------------------------------------- full-size, sampled
def _sample_cells(c, n, seed):
    rng = np.random.default_rng(seed)
    rho = c["rho"]
    flat = rho.reshape(-1)
    dense = np.argsort(flat)[-max(1, flat.size // 100):]
    pick = np.concatenate([rng.choice(dense, n // 2, replace=False),
                           rng.choice(flat.size, n - n // 2, replace=False)])
    return pick // 512, pick % 512          # leaf rows, cells


def _path_targets(desc, rows, cells):
    leaves = leaf_nodes(desc)
    targets = set()
    for r, cell in zip(rows, cells):
        node = int(leaves[r])
        g = np.array([cell & 7, (cell >> 3) & 7, cell >> 6]) + 8 * desc[node, 1:4]
        while node >= 0:
            loc = g - 8 * desc[node, 1:4]
            targets.add(node * 512 + int(loc[0] + 8 * loc[1] + 64 * loc[2]))
            node = int(desc[node, 4])
            g = g >> 1
    return np.array(sorted(targets), dtype=np.int64)


def sampled_reference(c, n=96, seed=3):
    """Oracle field at sampled leaf cells: same-level results on the sampled
    cells' ancestor paths only, then the full downward pass (the other cells'
    results are zero and never reach the sampled ones)."""
    tree = O.Tree.from_config(c)
    M, com = O.upward(tree, c["rho"])
    rows, cells = _sample_cells(c, n, seed)
    targets = _path_targets(c["desc"], rows, cells)
    L, dL1, _ = O.m2l(tree, M, com, targets=targets)
    L64, acc = O.downward(tree, com, L, dL1)
    phi, g, _ = O.forces(tree, L64, acc, c["rho"])
    return dict(rows=rows, cells=cells, g=g[rows, :, cells], phi=phi[rows, cells],
                targets=targets, L=L, M=M, com=com)


@pytest.mark.parametrize("name", ["cfg3", "cfg4", "cfg5"])
def test_full_size_sampled(name):
    c = make_config(name)
    ref = sampled_reference(c)
    rows, cells = ref["rows"], ref["cells"]
    tnodes, tcells = ref["targets"] // 512, ref["targets"] % 512
    # FP64 path end to end: sampled field
    s = solve_gpu(c, "fp64")
    assert rel_err(host(s.g)[rows, :, cells], ref["g"]) <= FP64_TOL
    assert rel_err(host(s.phi)[rows, cells], ref["phi"]) <= FP64_TOL
    tot64 = host(s.totals)
    assert np.all(tree_force(tot64) <= 1e-13)
    assert np.all(tree_torque(tot64) <= 1e-13)
    # FP64 same-level pass on the oracle's moments: sampled targets
    s.M.copy_(dev(ref["M"]))
    s.com.copy_(dev(ref["com"]))
    s.m2l()
    torch.cuda.synchronize()
    Lgpu = level_to_phys(host(s.L), c["desc"])[tnodes, :, tcells]
    Lref = ref["L"][tnodes, :, tcells]
    for sl in ORDER_SLICES[:2]:
        assert rel_err(Lgpu[:, sl], Lref[:, sl]) <= FP64_TOL
    s.close()
    # mixed path, the benchmark's configuration (its conservation against
    # the target: test_gpu_full_oracle)
    s = solve_gpu(c, "mixed")
    assert rel_err(host(s.g)[rows, :, cells], ref["g"]) <= FORCE_TOL
    s.close()
    # double-float (conserving) path
    s = solve_gpu(c, "dfloat")
    assert rel_err(host(s.g)[rows, :, cells], ref["g"]) <= DFLOAT_TOL_FULL
    tot = host(s.totals)
    assert np.all(tree_force(tot) <= DFLOAT_CONSERVATION), tree_force(tot)
    assert np.all(tree_torque(tot) <= DFLOAT_CONSERVATION), tree_torque(tot)
    s.close()


# ------------------------------------------------- expansion order 2
_ORACLE2 = {}


def oracle_solution_order2(name):
    if name not in _ORACLE2:
        c = dict(small_case(name), order=2)
        _ORACLE2[name] = (c, O.solve(O.Tree.from_config(c), c["rho"]))
    return _ORACLE2[name]


@pytest.mark.parametrize("precision", ["fp64", "dfloat", "mixed"])
@pytest.mark.parametrize("name", ["cfg1", "adaptive4", "batch3", "cfg2"])
def test_order2_end_to_end(name, precision):
    """Order 2 (truncation n + m <= 2, its own correction) against the
    oracle at order 2: FP64 and double-float to 1e-12 with net force and
    torque 1e-12; mixed to force error 1e-6.  The step goes through fmm_step
    and equals the four pass calls bit for bit."""
    c, ref = oracle_solution_order2(name)
    s = F.Solver(c["desc"], c["theta"], precision=precision, order=2)
    s.rho.copy_(dev(c["rho"]))
    s.step()
    torch.cuda.synchronize()
    g, phi, tot = host(s.g).copy(), host(s.phi).copy(), host(s.totals).copy()
    tol = FORCE_TOL if precision == "mixed" else FP64_TOL
    assert rel_err(g, ref["g"]) <= tol
    assert rel_err(phi, ref["phi"]) <= tol
    if precision != "mixed":
        assert np.all(tree_force(tot) <= CONSERVATION_TARGET), tree_force(tot)
        assert np.all(tree_torque(tot) <= CONSERVATION_TARGET), tree_torque(tot)
    s.step_passes()
    torch.cuda.synchronize()
    assert np.array_equal(host(s.g), g) and np.array_equal(host(s.totals), tot)
    s.close()


def test_order2_same_level_fp64():
    """The order-2 same-level pass from the oracle's moments: every order
    each node defines (the third-order slots zero) and the correction."""
    c, ref = oracle_solution_order2("adaptive4")
    s = F.Solver(c["desc"], c["theta"], precision="fp64", order=2)
    s.M.copy_(dev(ref["M"]))
    s.com.copy_(dev(ref["com"]))
    s.m2l()
    torch.cuda.synchronize()
    L = level_to_phys(host(s.L), c["desc"])
    assert_L_close(L, ref["L"], c["desc"], FP64_TOL)
    refined = c["desc"][:, 5] >= 0
    assert np.all(L[refined][:, 10:20] == 0.0) and np.all(ref["L"][:, 10:20] == 0.0)
    h = widths(c["desc"])[:, None, None]
    assert rel_err(host(s.dL1) * h ** -2, ref["dL1"]) <= FP64_TOL
    s.close()


@pytest.mark.parametrize("dataflow", [0, 1])
@pytest.mark.parametrize("name", ["adaptive4", "batch3", "single"])
def test_step_launch_count_matches_stats(name, dataflow):
    """The library kernels one fmm_step launches, as the CUDA profiler
    counts them, equal fmm_get_stats' launches_fused under the same tuning
    (the figure the benchmark reports as gpu_launches)."""
    prof = pytest.importorskip("torch.profiler")
    c = small_case(name)
    s = solve_gpu(c, "mixed")
    F.fmm_set_tuning(s.tree, dataflow=dataflow)
    s.step()
    torch.cuda.synchronize()
    names = []
    for _ in range(2):      # the first session can start its device tracing late
        with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
            s.step()
            torch.cuda.synchronize()
        names = [e.name for e in p.events() if "fmm::" in e.name]
        if names:
            break
    if not names:
        pytest.skip("the profiler recorded no device kernels here")
    assert len(names) == F.fmm_get_stats(s.tree)["launches_fused"], sorted(set(names))
    s.close()
