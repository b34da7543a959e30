"""The failure path of the bounded device waits, without a GPU fault (needs a
GPU): a wait on an mbarrier that nothing arrives at gives up after its poll
limit, raises the timeout flag and the call returns IPM_ERR_TIMEOUT; the
device stays usable afterwards (a condensation right after runs and gives a
finite reduced Hessian)."""
import numpy as np
import pytest

from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu
IPM_ERR_ARG, IPM_ERR_TIMEOUT = 1, 8


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


def test_wait_gives_up_and_the_device_stays_usable(gpu):
    assert gpu.selftest_bounded_wait(256) == IPM_ERR_TIMEOUT
    assert gpu.selftest_bounded_wait(1) == IPM_ERR_TIMEOUT
    assert gpu.selftest_bounded_wait(0) == IPM_ERR_ARG
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64_TC)
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    K = sol.ipm_get_quantity(gpu.Q_KHAT)
    assert np.all(np.isfinite(K)) and np.abs(K).max() > 0
