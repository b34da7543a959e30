"""GPU FP64 path vs the CPU oracle, through the C ABI (needs a GPU).

Every comparison evaluates both sides at the same iterate (the oracle's,
copied in with ipm_set_state) and checks the normwise relative error
max|gpu - oracle| / max|oracle| per output.  Kernel outputs (derivatives,
condensed blocks, Z, K_hat, the reduced right-hand side) meet the FP64 parity
bar 1e-10.  The Newton step is the solution of a linear system: its bars
(tests/bars.py) follow from the condition numbers of K_hat and G_x at that
iterate and the recovery of Prop. 2.1 (K_hat alone on the 64-scenario
workload, where the dense condition numbers of 64 G_x would dominate the
test's time; the measured errors sit at 0.3 - 3 kappa eps).  Cases span one scenario (30 buses), a ragged small batch
(60 buses, 5 scenarios), and the 1000-bus network with 4 and 64 scenarios."""
import numpy as np
import pytest

from oracle import ipm as oipm
from bars import step_bars
from oracle import kkt, opf
from paper_2301_04869_gb300 import synth

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


CASES = {
    "30bus_N1": (30, 6, 1, 0.0, 3),
    "60bus_N5": (60, 9, 5, 0.05, 4),
    "1000bus_N4": (1000, 150, 4, 0.05, 5),
}
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
        _cache[name] = (net, pd, qd, M, st)
    return _cache[name]


def solver_at(gpu, name, precision="fp64"):
    net, pd, qd, M, st = case(name)
    prec = {"fp64": gpu.PREC_FP64, "fp64_tc": gpu.PREC_FP64_TC}[precision]
    sol = gpu.Solver(net, pd, qd, precision=prec)
    sol.ipm_set_state(sol.pack_state(st))
    return sol


@pytest.mark.parametrize("name", list(CASES))
def test_eval_parity(gpu, name):
    net, pd, qd, M, st = case(name)
    sol = solver_at(gpu, name)
    sol.ipm_eval_derivatives()
    d = sol.dims
    nx, nu, m = d.n_x, d.n_u, d.m
    for i in sorted({0, M.N - 1}):
        o = M.derivatives(i, st["x"][i], st["u"], st["y"][i], st["z"][i])
        fgh = sol.ipm_get_quantity(gpu.Q_FGH, i)
        assert abs(fgh[0] - o["f"]) <= TOL * max(1.0, abs(o["f"]))
        assert rel(fgh[1:1 + nx], o["g"]) <= TOL
        assert rel(fgh[1 + nx:], o["h"]) <= TOL
        jac = sol.ipm_get_quantity(gpu.Q_JAC, i)
        o1 = nx * nx
        o2 = o1 + nx * nu
        o3 = o2 + m * nx
        assert rel(jac[:o1].reshape(nx, nx), o["Gx"].toarray()) <= TOL
        assert rel(jac[o1:o2].reshape(nx, nu), o["Gu"].toarray()) <= TOL
        assert rel(jac[o2:o3].reshape(m, nx), o["Hx"].toarray()) <= TOL
        assert rel(jac[o3:].reshape(m, nu), o["Hu"].toarray()) <= TOL


# fp64_tc: the same FP64 path with the K_hat contraction emulated on the
# tensor cores (exact BF16 slices); it must meet the same FP64 bar
PRECS = ["fp64", "fp64_tc"]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_condense_parity(gpu, name, precision):
    net, pd, qd, M, st = case(name)
    sol = solver_at(gpu, name, precision)
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    d = sol.dims
    nx, nu = d.n_x, d.n_u
    K = sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu)
    assert rel(K, C.Khat) <= TOL
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C.rhs_u) <= TOL
    for i in sorted({0, M.N - 1}):
        Z = sol.ipm_get_quantity(gpu.Q_Z, i).reshape(nx, nu)
        assert rel(Z, C.Z[i]) <= TOL
        H = sol.ipm_get_quantity(gpu.Q_HESS, i)
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        assert rel(H[:nx * nx].reshape(nx, nx), Kxx.toarray()) <= TOL
        assert rel(H[nx * nx:nx * nx + nx * nu].reshape(nx, nu), Kxu.toarray()) <= TOL
        assert rel(H[nx * nx + nx * nu:].reshape(nu, nu), Kuu.toarray()) <= TOL
    # determinism: a second condensation gives the same bits
    sol.ipm_condense_scenarios()
    K2 = sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu)
    assert np.array_equal(K, K2)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("delta", [0.0, 0.37])
def test_newton_step_parity(gpu, name, delta, precision):
    import torch
    net, pd, qd, M, st = case(name)
    sol = solver_at(gpu, name, precision)
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], delta)
    L = kkt.cholesky_pd(C.Khat)
    p = kkt.reduced_step(M, st, D, C, L)
    bars = step_bars(M, st, D, C, p)
    for k in ("px", "pu", "ps", "py", "pz"):
        assert rel(g[k], p[k]) <= bars[k], (k, rel(g[k], p[k]), bars[k])
    # the step the library returns was checked on the augmented system eq. (6):
    # the direct FP64 solve is backward stable (backward error <= 1e-12)
    info = sol.ipm_get_quantity(gpu.Q_INFO)
    assert info[14] <= 1e-12, info[12:15]


@pytest.mark.parametrize("precision", PRECS)
def test_full_solve_same_iterations_30(gpu, precision):
    net, pd, qd = synth.workload("opf30_n1")
    M = opf.Model(net, pd, qd)
    st_o, k_o, log = oipm.solve(M)
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC)
    k_g, e_g = sol.ipm_solve()
    assert k_g == k_o
    assert e_g <= 1e-8
    s = sol.split_state(sol.ipm_get_state())
    np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-8)
    np.testing.assert_allclose(s["x"], st_o["x"], rtol=0, atol=1e-8)


@pytest.mark.parametrize("precision", PRECS)
def test_full_solve_same_iterations_1000_N4(gpu, precision):
    net, pd, qd = synth.workload("opf1000_n64", n_scen=4)
    M = opf.Model(net, pd, qd)
    st_o, k_o, _ = oipm.solve(M)
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC)
    k_g, e_g = sol.ipm_solve()
    assert k_g == k_o
    assert e_g <= 1e-8
    # the GPU's final point judged by the oracle: its own optimality error
    # there must meet the tolerance too
    s = sol.split_state(sol.ipm_get_state())
    st_g = {k: s[k] for k in ("x", "u", "s", "y", "z", "zl_x", "zu_x", "zl_u", "zu_u", "zl_s", "zu_s")}
    errs = oipm.kkt_errors(M, st_g, kkt.eval_all(M, st_g))
    assert oipm.e_mu(errs, 0.0) <= 1e-8, errs
    # near mu -> 0 the iterates agree only to the conditioning of the KKT
    # system (~1e-9 relative at mu = 2.5e-9, kappa(K_hat) ~ 1e7)
    np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-6)


def test_trajectory_matches_per_iteration(gpu):
    """Iterate-by-iterate: after each GPU step the state stays within 1e-8
    (relative) of the oracle's, on a 5-scenario problem."""
    net, pd, qd, M, st0 = case("60bus_N5")
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    sol = gpu.Solver(net, pd, qd)
    for k in range(12):
        conv_o, _ = oipm.iterate(M, st)
        conv_g, _ = sol.ipm_step()
        assert conv_o == conv_g
        if conv_o:
            break
        s = sol.split_state(sol.ipm_get_state())
        for key in ("x", "u", "s", "y", "z"):
            assert rel(s[key], st[key]) <= 1e-8, (k, key)
        assert abs(s["mu"] - st["mu"]) <= 1e-8 * st["mu"]


_n64 = {}


def n64_iterate(k):
    """The 1000-bus / 64-scenario workload at the oracle's k-th iterate, with
    the oracle's condensation (delta = 0), inertia-corrected factor and step."""
    if k not in _n64:
        net, pd, qd = synth.workload("opf1000_n64")
        M = opf.Model(net, pd, qd)
        st = oipm.initial_state(M)
        for _ in range(k):
            oipm.iterate(M, st)
        D = kkt.eval_all(M, st)
        C0 = kkt.condense(M, st, D, st["mu"], 0.0)
        C, L, delta = oipm.factor_with_inertia_correction(M, dict(st), D, st["mu"])
        p = kkt.reduced_step(M, st, D, C, L)
        _n64[k] = (net, pd, qd, M, st, C0, C, delta, p)
    return _n64[k]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("k", [2, 12])
def test_config_1000bus_64_scenarios_components(gpu, precision, k):
    """The full 1000-bus / 64-scenario workload (231 row groups of the
    emulated contraction) at an early (delta > 0) and a late iterate: K_hat,
    Z of the first and last scenario and the reduced right-hand side at 1e-10,
    all five blocks of the Newton step at the step bar."""
    import torch
    net, pd, qd, M, st, C0, C, delta, p = n64_iterate(k)
    sol = solver_for(gpu, net, pd, qd, st, precision)
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    nx, nu = sol.dims.n_x, sol.dims.n_u
    assert rel(sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu), C0.Khat) <= TOL
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C0.rhs_u) <= TOL
    for i in (0, M.N - 1):
        assert rel(sol.ipm_get_quantity(gpu.Q_Z, i).reshape(nx, nu), C0.Z[i]) <= TOL, i
    # the oracle's inertia correction at this iterate (delta may be > 0)
    assert sol.ipm_factor_schur(0.0) == (delta == 0.0)
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    bars = step_bars(M, st, kkt.eval_all(M, st), C, p, with_gx=False)
    for key in ("px", "pu", "ps", "py", "pz"):
        assert rel(g[key], p[key]) <= bars[key], (key, rel(g[key], p[key]), bars[key])


def solver_for(gpu, net, pd, qd, st, precision):
    prec = {"fp64": gpu.PREC_FP64, "fp64_tc": gpu.PREC_FP64_TC, "mixed": gpu.PREC_MIXED}[precision]
    sol = gpu.Solver(net, pd, qd, precision=prec)
    sol.ipm_set_state(sol.pack_state(st))
    return sol


@pytest.mark.parametrize("k", [2, 12])
def test_config_1000bus_64_scenarios_mixed(gpu, k):
    """The mixed path on the same iterates, at its per-quantity bars: Z from
    FP32 solves and K_hat from BF16x3 products 1e-5; the reduced right-hand
    side (FP64 solves) 1e-10; the Newton step after FP64 refinement on the
    augmented system eq. (6) at the FP64 step bar."""
    import torch
    net, pd, qd, M, st, C0, C, delta, p = n64_iterate(k)
    sol = solver_for(gpu, net, pd, qd, st, "mixed")
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    nx, nu = sol.dims.n_x, sol.dims.n_u
    assert rel(sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu), C0.Khat) <= 1e-5
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C0.rhs_u) <= TOL
    for i in (0, M.N - 1):
        assert rel(sol.ipm_get_quantity(gpu.Q_Z, i).reshape(nx, nu), C0.Z[i]) <= 1e-5, i
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    bars = step_bars(M, st, kkt.eval_all(M, st), C, p, with_gx=False)
    for key in ("px", "pu", "ps", "py", "pz"):
        assert rel(g[key], p[key]) <= bars[key], (key, rel(g[key], p[key]), bars[key])


@pytest.mark.slow
def test_full_solve_same_iterations_1000_N64(gpu):
    """The benchmarked workload (1000 buses, 64 scenarios) solved from the cold
    start: the FP64 and FP64_TC paths reach E_0 <= 1e-8 in the same number of
    iterations as the oracle, and the oracle judges their final points."""
    net, pd, qd = synth.workload("opf1000_n64")
    M = opf.Model(net, pd, qd)
    st_o, k_o, _ = oipm.solve(M)
    for prec in (gpu.PREC_FP64, gpu.PREC_FP64_TC):
        sol = gpu.Solver(net, pd, qd, precision=prec)
        k_g, e_g = sol.ipm_solve()
        assert k_g == k_o, (prec, k_g, k_o)
        assert e_g <= 1e-8
        s = sol.split_state(sol.ipm_get_state())
        st_g = {k: s[k] for k in ("x", "u", "s", "y", "z", "zl_x", "zu_x", "zl_u", "zu_u", "zl_s", "zu_s")}
        errs = oipm.kkt_errors(M, st_g, kkt.eval_all(M, st_g))
        assert oipm.e_mu(errs, 0.0) <= 1e-8, (prec, errs)
        np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-6)
        sol.close()


def test_singular_state_jacobian(gpu):
    """A bus with no lines makes G_x singular: the static-pivot LU reports
    IPM_ERR_SINGULAR_GX instead of producing a step."""
    net = synth.make_network(30, 6, seed=0)
    # detach bus 29 (a load bus) by removing its lines and reconnecting the
    # rest through a chord-free copy
    keep = (net.fr != 29) & (net.to != 29)
    net.fr, net.to = net.fr[keep], net.to[keep]
    net.r, net.x, net.b = net.r[keep], net.x[keep], net.b[keep]
    if 29 in set(net.gen_bus.tolist()):
        pytest.skip("bus 29 carries a generator in this draw")
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    sol = gpu.Solver(net, pd, qd)
    sol.ipm_eval_derivatives()
    with pytest.raises(gpu.IPMError) as e:
        sol.ipm_condense_scenarios()
    assert e.value.kind == "IPM_ERR_SINGULAR_GX"


def test_inertia_correction_matches_oracle(gpu):
    """Large random equality multipliers make K_hat indefinite; the GPU
    reports it and takes the same delta_w as the oracle."""
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    st["y"] = 50.0 * np.random.default_rng(3).standard_normal(st["y"].shape)
    sol = gpu.Solver(net, pd, qd)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    assert not sol.ipm_factor_schur(0.0)
    D = kkt.eval_all(M, st)
    _, _, delta = oipm.factor_with_inertia_correction(M, dict(st), D, st["mu"])
    assert delta > 0
    # replay the oracle's delta sequence: every trial before the accepted one
    # must fail on the GPU too, the accepted one must succeed
    trial = 1e-4
    while trial < delta * (1 - 1e-12):
        assert not sol.ipm_factor_schur(trial)
        trial *= 100.0
    assert sol.ipm_factor_schur(delta)
