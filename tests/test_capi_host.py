"""CPU tests of the C ABI: the library loads and exports every declared
symbol, descriptors are validated on the host, and the host planner's
stencils and interaction counts agree with the oracle's brute-force opening
rule.  No GPU compute is called here (trees are planned host-only)."""

import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_1908_03121_gb300 as F
from paper_1908_03121_gb300 import fmm as B
from oracle import oracle as O
from workloads import make_config, uniform_tree, adaptive_tree, leaf_nodes, concat_trees

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmm_gb300.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = F.load()
    names = declared_symbols()
    assert set(B.EXPORTED) == set(names)
    for name in names:
        assert hasattr(lib, name), name
        # every binding declares its C argument types: without them ctypes
        # passes Python ints as 32-bit C ints, and an int64_t parameter would
        # see undefined upper bits
        assert getattr(lib, name).argtypes is not None, name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(B.FmmConfig) == 8 * 6 + 4 * 4
    assert ctypes.sizeof(B.FmmSizes) == 8 * 4 + 4 * 2 + 8 * 11
    assert ctypes.sizeof(B.FmmStats) == 8 * 4 + 8 * 3 + 8 * 4 + 8 * 4 + 8 * 4 + 4 * 6 + 8 * 16 + 8 * 16


def test_struct_sizes_match_the_c_compiler(tmp_path):
    """The binding's structures have the sizes the C compiler gives the
    header's (a layout drift would pass garbage through the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = ["fmm_config", "fmm_node_desc", "fmm_sizes", "fmm_stats", "fmm_tuning",
             "fmm_scf_params", "fmm_scf_result"]
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "fmm_gb300.h"\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({n}));\n' for n in names) + "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    ours = [ctypes.sizeof(B.FmmConfig), 14 * 4, ctypes.sizeof(B.FmmSizes),
            ctypes.sizeof(B.FmmStats), ctypes.sizeof(B.FmmTuning),
            ctypes.sizeof(B.FmmScfParams), ctypes.sizeof(B.FmmScfResult)]
    assert got == ours


def plan(desc, theta):
    return F.fmm_build_tree(desc, theta, host_only=True)


def _adaptive(max_level=4, r=0.12):
    def want(lo, hi):
        c = np.array([0.31, 0.62, 0.45])
        d = np.clip(c, lo, hi) - c
        return float(d @ d) < r * r
    return adaptive_tree(want, max_level)


@pytest.mark.parametrize("case", ["cfg1", "cfg2", "adaptive4", "adaptive4_035", "adaptive4_055",
                                  "adaptive4_030", "single", "singles2"])
def test_planner_counts_match_oracle(case):
    if case.startswith("cfg"):
        c = make_config(case)
        desc, rho, theta = c["desc"], c["rho"], c["theta"]
    elif case.startswith("single"):
        # one leaf sub-grid per tree: every pair on the root level, 512 x 511
        desc = uniform_tree(1) if case == "single" else concat_trees([uniform_tree(1)] * 2)
        rho = np.ones((len(desc), 512))
        theta = 0.5
    else:
        desc = _adaptive()
        rho = np.ones((len(leaf_nodes(desc)), 512))
        # stencil reach 5 (0.5, 0.35), 3 (0.55) and 7 (0.3)
        theta = {"035": 0.35, "055": 0.55, "030": 0.3}.get(case[-3:], 0.5)
    t = plan(desc, theta)
    ot = O.Tree(desc, theta)
    M, com = O.upward(ot, rho)
    _, _, counts = O.m2l(ot, M, com)
    assert list(t.stats["interactions"]) == list(counts)
    assert sum(t.stats["kernel_interactions"]) == sum(counts)
    if case.startswith("single"):
        assert list(counts) == [0, 0, 512 * 511 * len(desc), 0]


def test_planner_stencil_sizes():
    facts = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_facts.json")))
    t = plan(uniform_tree(3), 0.35)
    assert t.stats["stencil_union"] == facts["stencil_neighbours"]["value"]
    assert t.stats["stencil_far"] + t.stats["stencil_near"] == 743
    t = plan(uniform_tree(3), 0.5)
    assert (t.stats["stencil_far"], t.stats["stencil_near"]) == (231, 32)
    assert t.stats["reach"] == 5


def test_sizes_report():
    c = make_config("cfg2")
    t = F.fmm_build_tree(c["desc"], 0.5, precision="mixed", host_only=True)
    s = t.sizes
    assert s["n_nodes"] == 73 and s["n_leaf"] == 64 and s["n_refined"] == 9
    assert s["M_bytes"] == 73 * 20 * 512 * 8
    assert s["L_bytes"] == 73 * 20 * 512 * 4 and s["Lcomp_bytes"] == s["L_bytes"]
    assert s["g_bytes"] == 64 * 3 * 512 * 8 and s["totals_bytes"] == 64
    # the double-float precision keeps the same (hi, lo) float layout of L
    s2 = F.fmm_build_tree(c["desc"], 0.5, precision="dfloat", host_only=True).sizes
    assert s2["precision"] == B.FMM_DFLOAT
    assert s2["L_bytes"] == s["L_bytes"] and s2["Lcomp_bytes"] == s["Lcomp_bytes"]
    s3 = F.fmm_build_tree(c["desc"], 0.5, precision="fp64", host_only=True).sizes
    assert s3["L_bytes"] == 73 * 20 * 512 * 8 and s3["Lcomp_bytes"] == 0


def expect_error(code, desc, theta=0.5, **kw):
    with pytest.raises(F.FmmError) as ei:
        F.fmm_build_tree(desc, theta, host_only=True, **kw)
    assert ei.value.code == code, str(ei.value)


def test_rejects_bad_config():
    d = uniform_tree(2)
    expect_error(B.FMM_ERR_INVALID_ARG, d, theta=0.7)
    expect_error(B.FMM_ERR_INVALID_ARG, d, theta=0.25)
    expect_error(B.FMM_ERR_INVALID_ARG, d, box_size=0.0)
    expect_error(B.FMM_ERR_INVALID_ARG, d, precision=7)
    expect_error(B.FMM_ERR_TREE, uniform_tree(3), max_level=2)


def test_rejects_malformed_trees():
    d = uniform_tree(3)
    bad = d.copy(); bad[5, 1] += 1                       # wrong coordinates
    expect_error(B.FMM_ERR_TREE, bad)
    bad = d.copy(); bad[3, 4] = 2                        # wrong parent
    expect_error(B.FMM_ERR_TREE, bad)
    bad = d.copy(); bad[1, 5 + 3] = -1                   # partially refined
    expect_error(B.FMM_ERR_TREE, bad)
    bad = d.copy(); bad[0, 4] = 3                        # root with a parent
    expect_error(B.FMM_ERR_TREE, bad)
    bad = np.concatenate([d, d[-1:]])                    # duplicate node
    expect_error(B.FMM_ERR_TREE, bad)
    bad = d.copy(); bad[:, 13] = 1                       # tree 0 has no root
    expect_error(B.FMM_ERR_TREE, bad)
    bad = d.copy(); bad[7, 0] = 25                       # level above max_level
    expect_error(B.FMM_ERR_TREE, bad)


def test_rejects_unbalanced_refinement():
    """A refined node whose in-domain same-level neighbour is missing."""
    d = uniform_tree(2)
    # refine only child 0 of the root, then child 0 of that child: the level-3
    # refined node's neighbours at level 3 inside child 0 exist, but the
    # nesting rule also needs its level-3 neighbours across the child-0 faces
    rows = [list(r) for r in d]
    def refine(i):
        lvl, ix, iy, iz = rows[i][:4]
        for k in range(8):
            rows.append([lvl + 1, 2 * ix + (k & 1), 2 * iy + ((k >> 1) & 1),
                         2 * iz + ((k >> 2) & 1), i] + [-1] * 8 + [0])
            rows[i][5 + k] = len(rows) - 1
    refine(1)
    first = rows[1][5 + 7]      # the level-3 child touching the centre
    refine(first)
    bad = np.asarray(rows, dtype=np.int32)
    expect_error(B.FMM_ERR_TREE, bad)


def test_rejects_null_and_host_only_calls():
    t = plan(uniform_tree(2), 0.5)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_upward(t, 0, 0, 0, stream=0)
    assert ei.value.code == B.FMM_ERR_INVALID_ARG
    with pytest.raises(F.FmmError):
        F.fmm_m2l(t, 1, 1, 1, 1, 1, stream=0)
    assert "HOST_ONLY" in F.fmm_last_error()
    # the status word lives on the device: a host-only tree has none
    with pytest.raises(F.FmmError) as ei:
        F.fmm_get_status(t)
    assert ei.value.code == B.FMM_ERR_INVALID_ARG
    assert B.load().fmm_get_status(t.handle, None, 0) == B.FMM_ERR_INVALID_ARG


def test_batched_trees_plan_independently():
    c = make_config("cfg1")
    from workloads import concat_trees
    d = concat_trees([c["desc"], c["desc"], c["desc"]])
    t = plan(d, 0.5)
    one = plan(c["desc"], 0.5)
    assert list(t.stats["interactions"]) == [3 * v for v in one.stats["interactions"]]
    assert t.sizes["n_trees"] == 3


def test_tuning_set_get_and_validation():
    """fmm_set_tuning keeps valid launch shapes, refuses the others and then
    leaves the previous tuning in place (host-only tree: no CUDA)."""
    t = plan(uniform_tree(2), 0.5)
    zero = dict(mono_subgrids=0, ctas_per_sm=0, dataflow=0, wait_budget_us=0,
                drop_first_producer=0, mp_pair_targets=0, mp_items=0)
    assert F.fmm_get_tuning(t) == zero
    good = dict(zero, mono_subgrids=2, ctas_per_sm=1, dataflow=1, wait_budget_us=500,
                mp_pair_targets=1, mp_items=2)
    F.fmm_set_tuning(t, **{k: v for k, v in good.items()})
    assert F.fmm_get_tuning(t) == good
    bad = [dict(mono_subgrids=3), dict(mono_subgrids=5), dict(mono_subgrids=-1),
           dict(ctas_per_sm=33), dict(ctas_per_sm=-1), dict(dataflow=2), dict(dataflow=-1),
           dict(wait_budget_us=-5), dict(drop_first_producer=2), dict(mp_pair_targets=2),
           dict(mp_items=3), dict(mp_items=-1)]
    for b in bad:
        with pytest.raises(F.FmmError) as ei:
            F.fmm_set_tuning(t, **b)
        assert ei.value.code == B.FMM_ERR_INVALID_ARG
        assert F.fmm_get_tuning(t) == good
    for nb in (0, 1, 2, 4):
        F.fmm_set_tuning(t, mono_subgrids=nb, ctas_per_sm=32)
        assert F.fmm_get_tuning(t) == dict(zero, mono_subgrids=nb, ctas_per_sm=32)
