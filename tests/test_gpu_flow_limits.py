"""Line-flow limits (§4.1.1) on the GPU against the oracle (needs a GPU).

With line ratings h gains |S_f|^2 and |S_t|^2 of every line (m = n_g + 1 +
2L).  At the oracle's iterate of a rated network (three limits binding at
the optimum): the flow rows of h, their Jacobian rows, the Lagrangian Hessian
with random multipliers on every row, the condensed blocks, K_hat and the
reduced right-hand side at 1e-10; the Newton step at the step bar
max(1e-10, 10 kappa eps) (kappa: the larger of kappa(K_hat), kappa(G_x)); and the whole solve takes the oracle's
iteration count and ends at a point where the tightened lines sit at their
ratings."""
import numpy as np
import pytest

from bars import step_bars
from oracle import ipm as oipm
from oracle import kkt, opf
from ratings import end_flows, rated

pytestmark = pytest.mark.gpu
TOL = 1e-10
EPS = float(np.finfo(np.float64).eps)


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


CASES = {"30bus_N1": (30, 6, 1, 0.0, 4), "60bus_N3": (60, 9, 3, 0.05, 5)}
_cache = {}


def case(name):
    if name not in _cache:
        n, ng, N, sigma, iters = CASES[name]
        net, pd, qd = rated(n, ng, N, sigma)
        M = opf.Model(net, pd, qd)
        st = oipm.initial_state(M)
        for _ in range(iters):
            oipm.iterate(M, st)
        _cache[name] = (net, pd, qd, M, st)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_flow_rows_and_derivatives(gpu, name):
    net, pd, qd, M, st = case(name)
    sol = gpu.Solver(net, pd, qd)
    d = sol.dims
    nx, nu, m = d.n_x, d.n_u, d.m
    assert m == net.n_gen + 1 + 2 * net.n_line
    st2 = dict(st)
    st2["z"] = np.random.default_rng(4).standard_normal(st["z"].shape)  # weight every row of W
    sol.ipm_set_state(sol.pack_state(st2))
    sol.ipm_eval_derivatives()
    for i in sorted({0, M.N - 1}):
        o = M.derivatives(i, st2["x"][i], st2["u"], st2["y"][i], st2["z"][i])
        fgh = sol.ipm_get_quantity(gpu.Q_FGH, i)
        assert rel(fgh[1 + nx:], o["h"]) <= TOL
        jac = sol.ipm_get_quantity(gpu.Q_JAC, i)
        o2 = nx * nx + nx * nu
        o3 = o2 + m * nx
        assert rel(jac[o2:o3].reshape(m, nx), o["Hx"].toarray()) <= TOL
        assert rel(jac[o3:].reshape(m, nu), o["Hu"].toarray()) <= TOL
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st2)
    C = kkt.condense(M, st2, D, st2["mu"], 0.0)
    for i in sorted({0, M.N - 1}):
        H = sol.ipm_get_quantity(gpu.Q_HESS, i)
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        assert rel(H[:nx * nx].reshape(nx, nx), Kxx.toarray()) <= TOL
        assert rel(H[nx * nx:nx * nx + nx * nu].reshape(nx, nu), Kxu.toarray()) <= TOL
        assert rel(H[nx * nx + nx * nu:].reshape(nu, nu), Kuu.toarray()) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("name", list(CASES))
def test_condensation_and_step(gpu, name, precision):
    import torch
    net, pd, qd, M, st = case(name)
    prec = gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC
    sol = gpu.Solver(net, pd, qd, precision=prec)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st)
    C, L, delta = oipm.factor_with_inertia_correction(M, dict(st), D, st["mu"])
    C0 = kkt.condense(M, st, D, st["mu"], 0.0)
    nu = sol.dims.n_u
    assert rel(sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu), C0.Khat) <= TOL
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C0.rhs_u) <= TOL
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    p = kkt.reduced_step(M, st, D, C, L)
    bars = step_bars(M, st, D, C, p)
    for k in ("px", "pu", "ps", "py", "pz"):
        assert rel(g[k], p[k]) <= bars[k], (k, rel(g[k], p[k]), bars[k])


@pytest.mark.parametrize("name", list(CASES))
def test_rated_solve_same_iterations(gpu, name):
    n, ng, N, sigma, _ = CASES[name]
    net, pd, qd = rated(n, ng, N, sigma)
    M = opf.Model(net, pd, qd)
    st_o, k_o, _ = oipm.solve(M)
    sol = gpu.Solver(net, pd, qd)
    k_g, e_g = sol.ipm_solve()
    assert k_g == k_o and e_g <= 1e-8
    s = sol.split_state(sol.ipm_get_state())
    np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-6)
    fl = end_flows(M, s["x"][0], s["u"])
    assert np.all(fl <= net.rate * (1 + 1e-7))
    assert np.sum(fl >= net.rate * (1 - 1e-5)) >= 1
