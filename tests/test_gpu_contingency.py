"""Line-tripping contingencies (§4.1.1) on the GPU against the oracle (needs a
GPU).

Scenarios share the intact network's sparsity patterns; a tripped line
contributes zeros in its scenario.  At the oracle's iterate of a rated
network whose scenarios each lose a different line (or none): derivatives,
condensed blocks, K_hat and the reduced right-hand side at 1e-10, the Newton
step at the step bar, and the full solve in the oracle's iteration count.
A trip that islands part of the network is refused on the host."""
import numpy as np
import pytest

from bars import step_bars
from oracle import ipm as oipm
from oracle import kkt, opf
from paper_2301_04869_gb300 import synth
from ratings import rated

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


@pytest.fixture(scope="module")
def tripped():
    net, pd, qd = rated(30, 6, 4, 0.05)
    cand = np.flatnonzero(~synth.bridges(net))
    trip = np.array([-1, cand[0], cand[len(cand) // 2], cand[-1]], dtype=np.int32)
    M = opf.Model(net, pd, qd, trip=trip)
    st = oipm.initial_state(M)
    for _ in range(4):
        oipm.iterate(M, st)
    return net, pd, qd, trip, M, st


def make(gpu, net, pd, qd, trip, precision=None):
    sol = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64 if precision is None else precision)
    sol.ipm_set_contingencies(trip)
    return sol


def test_derivatives_and_condensation(gpu, tripped):
    net, pd, qd, trip, M, st = tripped
    sol = make(gpu, net, pd, qd, trip)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    d = sol.dims
    nx, nu, m = d.n_x, d.n_u, d.m
    for i in range(M.N):
        o = M.derivatives(i, st["x"][i], st["u"], st["y"][i], st["z"][i])
        fgh = sol.ipm_get_quantity(gpu.Q_FGH, i)
        assert rel(fgh[1:1 + nx], o["g"]) <= TOL and rel(fgh[1 + nx:], o["h"]) <= TOL
        jac = sol.ipm_get_quantity(gpu.Q_JAC, i)
        o1, o2 = nx * nx, nx * nx + nx * nu
        assert rel(jac[:o1].reshape(nx, nx), o["Gx"].toarray()) <= TOL
        assert rel(jac[o2:o2 + m * nx].reshape(m, nx), o["Hx"].toarray()) <= TOL
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    assert rel(sol.ipm_get_quantity(gpu.Q_KHAT).reshape(nu, nu), C.Khat) <= TOL
    assert rel(sol.ipm_get_quantity(gpu.Q_RHS_U), C.rhs_u) <= TOL
    for i in range(M.N):
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        H = sol.ipm_get_quantity(gpu.Q_HESS, i)
        assert rel(H[:nx * nx].reshape(nx, nx), Kxx.toarray()) <= TOL
        assert rel(sol.ipm_get_quantity(gpu.Q_Z, i).reshape(nx, nu), C.Z[i]) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_step(gpu, tripped, precision):
    import torch
    net, pd, qd, trip, M, st = tripped
    sol = make(gpu, net, pd, qd, trip, gpu.PREC_FP64 if precision == "fp64" else gpu.PREC_FP64_TC)
    sol.ipm_set_state(sol.pack_state(st))
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    D = kkt.eval_all(M, st)
    C, L, delta = oipm.factor_with_inertia_correction(M, dict(st), D, st["mu"])
    assert sol.ipm_factor_schur(delta)
    step = torch.empty(sol.dims.step_len, dtype=torch.float64, device="cuda")
    sol.ipm_solve_kkt(step)
    g = sol.split_step(step.cpu().numpy())
    p = kkt.reduced_step(M, st, D, C, L)
    bars = step_bars(M, st, D, C, p)
    for k in ("px", "pu", "ps", "py", "pz"):
        assert rel(g[k], p[k]) <= bars[k], (k, rel(g[k], p[k]), bars[k])


def test_solve_same_iterations(gpu, tripped):
    net, pd, qd, trip, M, _ = tripped
    st_o, k_o, _ = oipm.solve(M)
    sol = make(gpu, net, pd, qd, trip)
    k_g, e_g = sol.ipm_solve()
    assert k_g == k_o and e_g <= 1e-8
    s = sol.split_state(sol.ipm_get_state())
    np.testing.assert_allclose(s["u"], st_o["u"], rtol=0, atol=1e-6)
    # back to the intact network: the context solves the plain problem again
    sol.ipm_set_contingencies(None)
    M0 = opf.Model(net, pd, qd)
    _, k0, _ = oipm.solve(M0)
    k_g0, e0 = sol.ipm_solve()
    assert k_g0 == k0 and e0 <= 1e-8


def test_islanding_trip_is_refused(gpu, tripped):
    net, pd, qd, trip, M, _ = tripped
    sol = make(gpu, net, pd, qd, trip)
    bad = trip.copy()
    bad[2] = int(np.flatnonzero(synth.bridges(net))[0])
    with pytest.raises(gpu.IPMError) as e:
        sol.ipm_set_contingencies(bad)
    assert e.value.kind == "IPM_ERR_ARG"
    bad[2] = net.n_line
    with pytest.raises(gpu.IPMError):
        sol.ipm_set_contingencies(bad)
