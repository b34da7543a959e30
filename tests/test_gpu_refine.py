"""FP64 iterative refinement on the residual of the augmented system eq. (6)
(needs a GPU).

The library forms rho = -r - A p for its step from J, K and the right-hand
sides, solves A dp = rho through the same condensation and reduction, and
stops at a normwise backward error max|rho| / max(|r|, |A_blk p_blk|) <=
1e-12 (a backward-stable FP64 solve starts there).  Checked here:

* on the mixed path with the reduced-system CG switched off, the step from
  the BF16x3 factor alone is far from the oracle's; refinement brings its
  backward error below 1e-12 within the step budget and the step to the
  FP64 step bars of tests/bars.py;
* the residual the library works from is the oracle's: the dense augmented
  matrix of eq. (6) built by the oracle, applied to the returned step,
  leaves a residual within the reported backward error times the scale of
  the products (to the rounding of forming it);
* on the FP64 paths the direct solve is already backward stable (no step);
* with refinement off, the same call returns the unrefined step.
"""
import numpy as np
import pytest

from bars import step_bars
from oracle import ipm as oipm
from oracle import kkt, opf
from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu
EPS = float(np.finfo(np.float64).eps)


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
def iterate60():
    net = synth.make_network(60, 9, seed=0)
    pd, qd = synth.make_scenarios(net, 5, 0.05, seed=1)
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    for _ in range(6):
        oipm.iterate(M, st)
    return net, pd, qd, M, st


def solve_at(gpu, net, pd, qd, st, precision, aug_refine, max_refine=0, delta=0.0):
    import torch
    sol = gpu.Solver(net, pd, qd, precision=precision, aug_refine=aug_refine, max_refine=max_refine)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    res = sol.ipm_solve_kkt(step)
    info = sol.ipm_get_quantity(gpu.Q_INFO)
    g = sol.split_step(step.cpu().numpy())
    sol.close()
    return g, res, info


def flat(g):
    return np.concatenate([g["px"].ravel(), g["pu"], g["ps"].ravel(), g["py"].ravel(), g["pz"].ravel()])


@pytest.mark.parametrize("delta", [0.0, 0.37])
def test_refinement_repairs_the_mixed_precision_step(gpu, iterate60, delta):
    net, pd, qd, M, st = iterate60
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], delta)
    p = kkt.reduced_step(M, st, D, C, kkt.cholesky_pd(C.Khat))
    bars = step_bars(M, st, D, C, p)
    g0, res0, info0 = solve_at(gpu, net, pd, qd, st, gpu.PREC_MIXED, aug_refine=0, delta=delta)
    g1, res1, info1 = solve_at(gpu, net, pd, qd, st, gpu.PREC_MIXED, aug_refine=10, delta=delta)
    e0 = max(rel(g0[k], p[k]) / bars[k] for k in p)
    e1 = {k: rel(g1[k], p[k]) / bars[k] for k in p}
    assert e0 > 1e3, e0  # the BF16x3 factor alone is not FP64-grade
    assert info1[12] >= 1 and info1[13] > 1e-10, info1[12:15]
    assert res1 == info1[14] and res1 <= 1e-12, info1[12:15]
    assert max(e1.values()) <= 1.0, e1  # within each block's bar
    # the oracle's own augmented matrix: the residual of the returned step,
    # over the scale of its products, is a backward error of the same size
    A, rhs, _ = kkt.augmented_dense(M, st, D, st["mu"], delta)
    x = flat(g1)
    r = A @ x - rhs
    scale = max(np.abs(rhs).max(), (np.abs(A) @ np.abs(x)).max())
    assert np.abs(r).max() / scale <= 1e-12 + 64 * EPS, (np.abs(r).max() / scale, info1[14])


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_fp64_paths_report_their_augmented_residual(gpu, iterate60, precision):
    net, pd, qd, M, st = iterate60
    prec = gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC
    D = kkt.eval_all(M, st)
    A, rhs, _ = kkt.augmented_dense(M, st, D, st["mu"], 0.0)
    g, res, info = solve_at(gpu, net, pd, qd, st, prec, aug_refine=10)
    assert res <= 1e-12 and info[14] == res and info[12] == 0, info[12:15]
    x = flat(g)
    r = A @ x - rhs
    scale = max(np.abs(rhs).max(), (np.abs(A) @ np.abs(x)).max())
    assert np.abs(r).max() / scale <= 1e-12 + 64 * EPS
    # refinement off: no residual check, the unrefined step
    g0, res0, info0 = solve_at(gpu, net, pd, qd, st, prec, aug_refine=0)
    assert info0[12] == 0
    assert max(rel(g0[k], g[k]) for k in g) <= 1e-10
