"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of the oracle's C source: a
wrong sign, a dropped term, a wrong factorial or index, a transposed
operand, an off-by-one in the opening rule.  It then compiles that copy
with the oracle's own flags, routes the oracle's calls to it, and runs the
pins listed for it.  At least one of them must fail.  The pins are the
functions of ``test_oracle_pins`` unchanged, so this file checks that the
pins discriminate.  It does not add pins of its own.  No GPU is involved.
"""

import itertools
import os

import pytest

import test_oracle_pins as pins
from oracle import oracle as O

# compiled copies go beside the oracle's own build (git-ignored), removed
# afterwards.  Every case gets a path no earlier case used: the dynamic loader
# hands back an already loaded library for a path it has seen.
_WORK = os.path.join(os.path.dirname(O.build()), "mutants")
_CASE = itertools.count()


@pytest.fixture
def work_so():
    os.makedirs(_WORK, exist_ok=True)
    path = os.path.join(_WORK, f"case_{os.getpid()}_{next(_CASE)}.so")
    yield path
    for f in (path, path + ".c"):
        if os.path.exists(f):
            os.remove(f)

# (name, original text, mutated text, pins expected to catch it)
MUTANTS = [
    # derivative tensors
    ("D3: sign of the R R R term",
     "D3[i + 3 * j + 9 * k] = -15.0 *", "D3[i + 3 * j + 9 * k] = 15.0 *",
     ["dtensors_fd"]),
    ("D4: one delta-delta term dropped",
     "+ 3.0 * (DL(i, j) * DL(k, l) + DL(i, k) * DL(j, l)\n"
     "                                 + DL(i, l) * DL(j, k)) * i5;",
     "+ 3.0 * (DL(i, j) * DL(k, l) + DL(i, k) * DL(j, l)) * i5;",
     ["dtensors_fd"]),
    ("D1: transposed sign",
     "for (int i = 0; i < 3; ++i) D1[i] = -R[i] * i3;",
     "for (int i = 0; i < 3; ++i) D1[i] = R[i] * i3;",
     ["dtensors_first_order", "dtensors_fd"]),
    # the same-level expansion
    ("M2L: (-1)^m dropped",
     "double sgn = (m % 2) ? -1.0 : 1.0;", "double sgn = 1.0;",
     ["multipole_orders", "monopole_fourth_order", "all_near"]),
    ("M2L: 1/m! shifted to 1/(m+1)!",
     "double coef = -G * sgn * INV_FACT[m];", "double coef = -G * sgn * INV_FACT[m + 1];",
     ["multipole_orders", "monopole_fourth_order", "all_near"]),
    ("M2L: truncation n + m < 3 instead of <= 3",
     "for (int m = 0; n + m <= order; ++m) {\n            int nb = ipow3(m);\n            double sgn",
     "for (int m = 0; n + m < order; ++m) {\n            int nb = ipow3(m);\n            double sgn",
     ["monopole_fourth_order", "multipole_orders"]),
    # the angular-momentum correction
    ("correction: sign flipped", "dL1[i] += G / 6.0 * s;", "dL1[i] -= G / 6.0 * s;",
     ["torque_pair", "invariants_cfg1"]),
    ("correction: mass ratio inverted", "real ratio = MB[0] / MA[0];",
     "real ratio = MA[0] / MB[0];", ["torque_pair", "invariants_cfg1"]),
    ("correction: factor 1/2 instead of 1/6", "dL1[i] += G / 6.0 * s;",
     "dL1[i] += G / 2.0 * s;", ["torque_pair", "invariants_cfg1"]),
    ("order-2 correction: the target's share with the order-3 sign",
     "(Mf[2][b] + ratio2 * M2A[b])", "(Mf[2][b] - ratio2 * M2A[b])", ["order2_pair"]),
    ("order-2 correction: sign flipped", "dL1[i] -= G / 2.0 * s;", "dL1[i] += G / 2.0 * s;",
     ["order2_pair"]),
    # the opening rule
    ("opening: well separated at equality", "*far = th2 * o2 > 1.0;",
     "*far = th2 * o2 >= 1.0;", ["stencil_05", "stencil_035"]),
    ("opening: parent offset taken at the child level",
     "po[a] = (gB[a] >> 1) - (gA[a] >> 1);", "po[a] = gB[a] - gA[a];",
     ["coverage", "stencil_05", "stencil_035"]),
    ("opening: refined near pairs evaluated",
     "if (!(*far || a_leaf || b_leaf)) return 0;", "",
     ["coverage", "all_near"]),
    # upward
    ("upward: second moment about the wrong point",
     "for (int a = 0; a < 3; ++a) s[a] = x[a] - com[(node * 3 + a) * NCELL + cell];",
     "for (int a = 0; a < 3; ++a) s[a] = x[a] - com[(node * 3 + a) * NCELL + 0];",
     ["upward_definition"]),
    ("upward: centre of mass without the mass weight",
     "for (int a = 0; a < 3; ++a) mx[(node * 3 + a) * NCELL + cell] += m * x[a];",
     "for (int a = 0; a < 3; ++a) mx[(node * 3 + a) * NCELL + cell] += x[a];",
     ["upward_definition"]),
    # downward
    ("L2L: 1/k! dropped", "s += INV_FACT[k] * part;", "s += part;",
     ["downward_cubic"]),
    ("L2L: shift vector reversed",
     "d[a] = com[(i * 3 + a) * NCELL + c] - com[(pn * 3 + a) * NCELL + pc];",
     "d[a] = com[(pn * 3 + a) * NCELL + pc] - com[(i * 3 + a) * NCELL + c];",
     ["downward_cubic"]),
    ("L2L: correction not carried down",
     "for (int a = 0; a < 3; ++a) corr[a] += dL1acc[(pn * 3 + a) * NCELL + pc];", "",
     ["downward_cubic", "invariants_cfg1"]),
    # forces
    ("forces: correction subtracted",
     "gv[a] = -(L64[(i * NCOMP + 1 + a) * NCELL + c] + dL1acc[(i * 3 + a) * NCELL + c]);",
     "gv[a] = -(L64[(i * NCOMP + 1 + a) * NCELL + c] - dL1acc[(i * 3 + a) * NCELL + c]);",
     ["invariants_cfg1", "mirror"]),
    ("forces: torque with a transposed operand",
     "xf[1] = x[2] * f[0] - x[0] * f[2];", "xf[1] = x[2] * f[0] - x[0] * f[1];",
     ["invariants_cfg1"]),
]

PINS = {
    "order2_pair": pins.test_order2_two_cluster_momentum_and_torque,
    "dtensors_fd": pins.test_dtensors_match_finite_differences,
    "dtensors_first_order": pins.test_dtensors_first_order_closed_form,
    "multipole_orders": pins.test_multipole_source_far_field_orders,
    "monopole_fourth_order": pins.test_monopole_expansion_has_fourth_order_error,
    "all_near": pins.test_all_near_case_equals_direct_sum,
    "torque_pair": pins.test_two_cluster_momentum_and_torque,
    "invariants_cfg1": lambda: pins.test_momentum_invariants("cfg1"),
    "stencil_05": pins.test_paper_stencil_theta_05_counts,
    "stencil_035": pins.test_paper_stencil_size_at_theta_035,
    "coverage": lambda: pins.test_every_leaf_pair_covered_exactly_once(0.5),
    "upward_definition": pins.test_upward_matches_definition,
    "downward_cubic": pins.test_downward_recentres_cubic_exactly,
    "mirror": pins.test_mirror_symmetry,
}


@pytest.mark.parametrize("name,old,new,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, catchers, work_so):
    src = O.source_text()
    assert src.count(old) == 1, f"mutation site not unique or missing: {name}"
    caught = []
    with O.variant(src.replace(old, new), work_so):
        for pin in catchers:
            try:
                PINS[pin]()
            except (AssertionError, FloatingPointError, ValueError):
                caught.append(pin)
                break
    assert caught, f"no pin caught: {name}"


def test_unaltered_copy_passes_every_pin(work_so):
    """The harness itself: a copy compiled the same way passes all the pins
    used above, so a caught mutant is caught for its mistake."""
    with O.variant(O.source_text(), work_so):
        for pin in PINS.values():
            pin()
