"""No device buffer is read before it is written: contexts created with the
`poison` option (every allocation filled with NaN) give bit-identical
results to ordinary ones, on every precision path, through a full solve, an
inertia-corrected factorization (delta_w > 0: the Z^T Z product and the
right-hand-side correction), the refinement of the mixed path and a warm
start (needs a GPU)."""
import numpy as np
import pytest

from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc", "mixed"])
def test_poisoned_allocations_change_nothing(gpu, precision):
    import torch
    prec = {"fp64": gpu.PREC_FP64, "fp64_tc": gpu.PREC_FP64_TC, "mixed": gpu.PREC_MIXED}[precision]
    net, pd, qd = synth.workload("opf1000_n64", n_scen=4)
    out = []
    for poison in (False, True):
        sol = gpu.Solver(net, pd, qd, precision=prec, poison=poison)
        for _ in range(3):
            sol.ipm_step()
        sol.ipm_eval_derivatives()
        sol.ipm_condense_scenarios()
        assert sol.ipm_factor_schur(0.37)
        step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
        sol.ipm_solve_kkt(step)
        k, e = sol.ipm_solve()
        out.append((step.cpu().numpy(), k, sol.ipm_get_state()))
    assert np.isfinite(out[1][0]).all()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_poisoned_warm_start_changes_nothing(gpu):
    import torch
    net, pd, qd = synth.workload("opf30_n1")
    ref = gpu.Solver(net, pd, qd)
    ref.ipm_solve()
    tgt = torch.empty((1, ref.ipm_warm_dim()), dtype=torch.float32, device="cuda")
    ref.ipm_warm_target(tgt)
    res = []
    for poison in (False, True):
        sol = gpu.Solver(net, pd, qd, poison=poison)
        sol.ipm_warm_start(tgt)
        k, e = sol.ipm_solve()
        res.append((k, sol.ipm_get_state()))
    assert res[0][0] == res[1][0]
    np.testing.assert_array_equal(res[0][1], res[1][1])
