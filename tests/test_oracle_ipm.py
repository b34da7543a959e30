"""Pins of the oracle IPM (CPU): convergence to a 1e-8 KKT residual with a
zero power-flow residual, a Newton power flow from the converged controls that
reproduces the states, and N identical scenarios behaving like N = 1."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import ipm, kkt, opf
from paper_2301_04869_gb300 import synth


@pytest.fixture(scope="module")
def solved30():
    net, pd, qd = synth.workload("opf30_n1")
    M = opf.Model(net, pd, qd)
    st, k, log = ipm.solve(M)
    return M, st, k, log


def test_converges_with_zero_pf_residual(solved30):
    M, st, k, log = solved30
    D = kkt.eval_all(M, st)
    errs = ipm.kkt_errors(M, st, D)
    assert ipm.e_mu(errs, 0.0) <= 1e-8
    assert np.abs(D[0]["g"]).max() <= 1e-8
    assert 5 <= k <= 60
    # all iterates strictly inside the boxes
    assert np.all(st["u"] > M.ul) and np.all(st["u"] < M.uu)


def test_power_flow_from_controls_reproduces_states(solved30):
    """Fix u at the optimum and solve g(x, u) = 0 by Newton from a flat
    start: the states must coincide with the IPM's x."""
    M, st, k, log = solved30
    u = st["u"]
    x = np.concatenate([np.zeros(M.lay.n - 1), np.ones(M.lay.nx - M.lay.n + 1)])
    for _ in range(30):
        d = M.derivatives(0, x, u, np.zeros(M.lay.nx), np.zeros(M.lay.m))
        if np.abs(d["g"]).max() < 1e-13:
            break
        x = x - spla.spsolve(d["Gx"].tocsc(), d["g"])
    assert np.abs(x - st["x"][0]).max() <= 1e-7


def test_identical_scenarios_match_single():
    """With f_i = cost_i / N, N copies of one scenario have the same
    solution as the single scenario.  (The barrier terms of x_i and s_i are
    repeated N times while the cost is not, so the central paths - and the
    iteration counts - may differ; only the limit is invariant.)"""
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 1, 0.0)
    M1 = opf.Model(net, pd, qd)
    st1, k1, _ = ipm.solve(M1)
    M3 = opf.Model(net, np.repeat(pd, 3, 0), np.repeat(qd, 3, 0))
    st3, k3, _ = ipm.solve(M3)
    np.testing.assert_allclose(st3["u"], st1["u"], rtol=0, atol=1e-6)
    for i in range(3):
        np.testing.assert_allclose(st3["x"][i], st1["x"][0], rtol=0, atol=1e-6)


def test_stochastic_two_stage_small():
    """A 4-scenario problem converges; every scenario's power flow closes and
    the shared controls satisfy their bounds."""
    net = synth.make_network(60, 9, seed=0)
    pd, qd = synth.make_scenarios(net, 4, 0.05, seed=1)
    M = opf.Model(net, pd, qd)
    st, k, _ = ipm.solve(M)
    D = kkt.eval_all(M, st)
    for i in range(4):
        assert np.abs(D[i]["g"]).max() <= 1e-8
    assert ipm.e_mu(ipm.kkt_errors(M, st, D), 0.0) <= 1e-8


def test_line_flow_limits_bind_and_hold():
    """With line ratings (§4.1.1), the oracle converges to a point whose end
    flows respect every rating, the three tightened lines sit at their
    limits, the power flow is satisfied, and the cost is no lower than the
    unconstrained optimum's."""
    from ratings import end_flows, rated
    net, pd, qd = rated(30, 6, 1, 0.0)
    M = opf.Model(net, pd, qd)
    st, k, _ = ipm.solve(M)
    D = kkt.eval_all(M, st)
    assert ipm.e_mu(ipm.kkt_errors(M, st, D), 0.0) <= 1e-8
    assert np.abs(D[0]["g"]).max() <= 1e-8
    fl = end_flows(M, st["x"][0], st["u"])
    assert np.all(fl <= net.rate * (1 + 1e-7))
    assert np.sum(fl >= net.rate * (1 - 1e-5)) >= 3
    plain = synth.make_network(30, 6, seed=0)
    M0 = opf.Model(plain, pd, qd)
    st0, _, _ = ipm.solve(M0)
    f = M.functions(0, st["x"][0], st["u"])[0]
    f0 = M0.functions(0, st0["x"][0], st0["u"])[0]
    assert f >= f0 - 1e-9 * abs(f0)
