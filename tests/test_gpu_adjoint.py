"""The paper's local reduction by adjoint solves (§3.2) on the GPU (needs a
GPU).

With reduction = IPM_REDUCTION_ADJOINT, K_hat is formed as
sum_i (L_u - G_u^T G_x^{-T} L_x) over all n_u unit vectors (one more
multi-RHS solve with G_x^T instead of the Z^T Y contraction).  It must match
the oracle's K_hat (Prop. 2.3) and the oracle's own three-step reduction at
1e-10, give the same solve, and the autotuner (reduction = AUTO) must pick
one of the two reductions and keep results at the same bar."""
import numpy as np
import pytest

from oracle import ipm as oipm
from oracle import kkt, opf
from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


CASES = {"30bus_N1": (30, 6, 1, 0.0, 3), "60bus_N5": (60, 9, 5, 0.05, 4), "1000bus_N4": (1000, 150, 4, 0.05, 5)}
_cache = {}


def case(name):
    if name not in _cache:
        n, ng, N, sigma, iters = CASES[name]
        net = synth.make_network(n, ng, seed=0)
        pd, qd = synth.make_scenarios(net, N, sigma, seed=1)
        M = opf.Model(net, pd, qd)
        st = oipm.initial_state(M)
        for _ in range(iters):
            oipm.iterate(M, st)
        D = kkt.eval_all(M, st)
        C = kkt.condense(M, st, D, st["mu"], 0.0)
        _cache[name] = (net, pd, qd, M, st, D, C)
    return _cache[name]


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_khat(gpu, name, precision):
    net, pd, qd, M, st, D, C = case(name)
    prec = gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC
    sol = gpu.Solver(net, pd, qd, precision=prec, reduction=gpu.REDUCTION_ADJOINT)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    nu = sol.dims.n_u
    K = sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu)
    assert rel(K, C.Khat) <= TOL
    assert rel(K, kkt.reduce_adjoint(M, C, D, n_batch=32)) <= TOL
    assert np.array_equal(K, K.T)
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C.rhs_u) <= TOL
    assert sol.ipm_get_quantity(gpu.Q_INFO)[15] == 1.0


def test_adjoint_solve_same_iterations(gpu):
    net, pd, qd = synth.workload("opf1000_n64", n_scen=4)
    M = opf.Model(net, pd, qd)
    _, k_o, _ = oipm.solve(M)
    sol = gpu.Solver(net, pd, qd, reduction=gpu.REDUCTION_ADJOINT)
    k_g, e_g = sol.ipm_solve()
    assert k_g == k_o and e_g <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_autotuned_reduction(gpu, precision):
    import torch
    net, pd, qd, M, st, D, C = case("1000bus_N4")
    prec = gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = gpu.Solver(net, pd, qd, precision=prec, reduction=gpu.REDUCTION_AUTO, autotune=True, graphs=True)
        sol.ipm_set_state(sol.pack_state(st), stream=stream)
        nu = sol.dims.n_u
        for _ in range(2):  # the first call tunes, the second replays the captured graphs
            sol.ipm_eval_derivatives(stream=stream)
            sol.ipm_condense_scenarios(stream=stream)
            K = sol.ipm_get_quantity(gpu.Q_KHAT, stream=stream).reshape(nu, nu)
            assert rel(K, C.Khat) <= TOL
        info = sol.ipm_get_quantity(gpu.Q_INFO, stream=stream)
    assert info[15] in (0.0, 1.0) and info[16] > 0 and info[17] > 0
    assert info[15] == (1.0 if info[17] < info[16] else 0.0)
