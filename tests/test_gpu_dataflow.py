"""The dataflow downward pass (fmm_tuning.dataflow): one persistent launch
in which every refined node's shift and every leaf's shift and forces start
on their parent's readiness counter.  It must give the same bits as the
level-by-level launches, eagerly and from a captured graph, and a wait whose
producer never runs must give up within its budget, report
FMM_STATUS_TIMEOUT / FMM_ERR_TIMEOUT, and leave the tree usable."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1908_03121_gb300 as F
from paper_1908_03121_gb300 import fmm as B
from test_gpu_parity import oracle_solution, defined_L_mask

pytestmark = pytest.mark.gpu

OUTPUTS = ("L64", "dacc", "phi", "g", "totals")


def outputs(s, desc):
    mask = np.broadcast_to(defined_L_mask(desc), s.L64.shape)
    return [s.L64.cpu().numpy()[mask], s.dacc.cpu().numpy(), s.phi.cpu().numpy(),
            s.g.cpu().numpy(), s.totals.cpu().numpy()]


def fill_nan(s):
    for name in OUTPUTS:
        getattr(s, name).fill_(float("nan"))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "dfloat"])
@pytest.mark.parametrize("name", ["adaptive4", "batch3", "cfg2", "single"])
def test_dataflow_step_matches_level_launches(name, precision):
    c, _ = oracle_solution(name)
    s = F.Solver(c["desc"], c["theta"], precision=precision)
    s.rho.copy_(torch.from_numpy(np.ascontiguousarray(c["rho"])).cuda())
    s.step()
    torch.cuda.synchronize()
    ref = outputs(s, c["desc"])
    F.fmm_set_tuning(s.tree, dataflow=1)
    fill_nan(s)
    s.step()
    torch.cuda.synchronize()
    assert s.status() == 0
    for a, b in zip(outputs(s, c["desc"]), ref):
        assert np.array_equal(a, b)
    s.capture()
    fill_nan(s)
    s.replay()
    torch.cuda.synchronize()
    for a, b in zip(outputs(s, c["desc"]), ref):
        assert np.array_equal(a, b)
    s.close()


def test_dataflow_wait_runs_out_and_the_tree_recovers():
    """The host leaves the first refined node's items out of the queue (the
    test injection), so its children's waits can never succeed: the first
    wait gives up after its 20 ms budget, the others at once; the call
    returns, the status word carries FMM_STATUS_TIMEOUT, fmm_get_status
    returns FMM_ERR_TIMEOUT, and the next normal step is exact again."""
    c, _ = oracle_solution("adaptive4")
    s = F.Solver(c["desc"], c["theta"], precision="mixed")
    s.rho.copy_(torch.from_numpy(np.ascontiguousarray(c["rho"])).cuda())
    s.step()
    torch.cuda.synchronize()
    ref = outputs(s, c["desc"])
    F.fmm_set_tuning(s.tree, dataflow=1, wait_budget_us=20000, drop_first_producer=1)
    s.step()
    with pytest.raises(F.FmmError) as ei:
        s.status()
    assert ei.value.code == B.FMM_ERR_TIMEOUT
    assert s.status() == 0                      # read and cleared above
    F.fmm_set_tuning(s.tree, dataflow=1)
    s.step()
    torch.cuda.synchronize()
    assert s.status() == 0
    for a, b in zip(outputs(s, c["desc"]), ref):
        assert np.array_equal(a, b)
    s.close()
