"""Mixed-precision path (FP32 solves, BF16x3 tcgen05 product, FP64 Cholesky and
refinement) against the FP64 oracle (needs a GPU).

Per-quantity bars: Z (FP32 solves) 1e-5 relative, K_hat (BF16x3 products of
FP32 operands, FP32 accumulation per 64-wide block, FP64 across blocks) 1e-5,
the Newton step after conjugate-gradient refinement on the exact FP64
operator 1e-8; the full solve reaches E_0 <= 1e-8 in the same number of
iterations as the FP64 path."""
import numpy as np
import pytest

from oracle import ipm as oipm
from oracle import kkt, opf
from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


@pytest.fixture(scope="module")
def iterate1000():
    net, pd, qd = synth.workload("opf1000_n64", n_scen=6)
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    for _ in range(6):
        oipm.iterate(M, st)
    return net, pd, qd, M, st


def test_mixed_quantities_and_refined_step(gpu, iterate1000):
    import torch
    net, pd, qd, M, st = iterate1000
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_MIXED)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st)
    C, L, delta = oipm.factor_with_inertia_correction(M, dict(st), D, st["mu"])
    C0 = kkt.condense(M, st, D, st["mu"], 0.0)
    nx, nu = sol.dims.n_x, sol.dims.n_u
    errs = {}
    errs["Z"] = max(rel(sol.ipm_get_quantity(gpu.Q_Z, i).reshape(nx, nu), C0.Z[i]) for i in (0, M.N - 1))
    errs["K_hat"] = rel(sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu), C0.Khat)
    errs["rhs_u"] = rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C0.rhs_u)
    assert errs["Z"] <= 1e-5, errs
    assert errs["K_hat"] <= 1e-5, errs
    assert errs["rhs_u"] <= 1e-10, errs
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    res = sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    p = kkt.reduced_step(M, st, D, C, L)
    for k in ("px", "pu", "ps", "py", "pz"):
        errs["step_" + k] = rel(g[k], p[k])
        assert errs["step_" + k] <= 1e-8, errs
    assert res <= 1e-12
    print("mixed-path errors vs FP64 oracle:", {k: f"{v:.1e}" for k, v in errs.items()}, "refine residual", res)


def test_mixed_full_solve_matches_fp64_path(gpu):
    net, pd, qd = synth.workload("opf1000_n64", n_scen=8)
    a = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64)
    k64, e64 = a.ipm_solve()
    b = gpu.Solver(net, pd, qd, precision=gpu.PREC_MIXED)
    kmx, emx = b.ipm_solve()
    assert emx <= 1e-8 and e64 <= 1e-8
    assert kmx == k64
    sa = a.split_state(a.ipm_get_state())
    sb = b.split_state(b.ipm_get_state())
    assert rel(sb["u"], sa["u"]) <= 1e-6


def test_mixed_30bus_same_iterations_as_oracle(gpu):
    net, pd, qd = synth.workload("opf30_n1")
    M = opf.Model(net, pd, qd)
    st_o, k_o, _ = oipm.solve(M)
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_MIXED)
    k_g, e_g = sol.ipm_solve()
    assert e_g <= 1e-8 and k_g == k_o
