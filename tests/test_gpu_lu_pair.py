"""The batched LU of G_x on a cluster of two CTAs per scenario against the
one-CTA kernel (needs a GPU).

Both factor the same static-pivot LU (Section 3, the batched sparse LU of the
reduction step); they block the dense trailing block differently (the
cluster splits it by 16-column panels between two SMs, the one-CTA kernel
eliminates its first column through the slot map and blocks the rest in
shared memory), so they agree to rounding, not bit for bit.  Checked on the
reduced Hessian and Z after one condensation (normwise relative error
<= 1e-12) and on whole solves (same iteration count, same first-stage
solution to 1e-9), for one scenario and a ragged batch."""
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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n,ng,N", [(118, 19, 1), (300, 40, 7)])
def test_cluster_lu_matches_one_cta(gpu, n, ng, N):
    net = synth.make_network(n, ng, seed=3)
    pd, qd = synth.make_scenarios(net, N, 0.05, seed=4)
    a = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64, lu_pair=True)
    b = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64, lu_pair=False)
    for s in (a, b):
        s.ipm_eval_derivatives()
        s.ipm_condense_scenarios()
    assert rel(a.ipm_get_quantity(gpu.Q_KHAT), b.ipm_get_quantity(gpu.Q_KHAT)) <= 1e-12
    for sc in range(N):
        assert rel(a.ipm_get_quantity(gpu.Q_Z, sc), b.ipm_get_quantity(gpu.Q_Z, sc)) <= 1e-12
    a.ipm_init_state()
    b.ipm_init_state()
    ia, ea = a.ipm_solve()
    ib, eb = b.ipm_solve()
    assert ia == ib and ea <= 1e-8 and eb <= 1e-8
    ua = a.split_state(a.ipm_get_state())["u"]
    ub = b.split_state(b.ipm_get_state())["u"]
    assert rel(ua, ub) <= 1e-9
