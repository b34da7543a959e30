"""Independent pins of the oracle's optimum and dual point (CPU).

The IPM oracle's convergence test uses its own stationarity formula
(ipm.kkt_errors) fed by its own derivatives.  These tests judge its converged
point on the 30-bus, one-scenario workload with nothing of that machinery:

* an independent NLP solve of the same problem, eq. (2) with the slack form
  of eq. (3) written as the interval h(x, u) in [-s_u, -s_l], by scipy's
  trust-constr method, given only ``Model.functions`` (values: no oracle
  derivative, no oracle residual) with finite-difference Jacobians and a
  quasi-Newton Hessian, must reach the same objective, controls and states;
* the oracle's multipliers (y, z and the bound duals) must make the
  Lagrangian of eq. (4) stationary, eq. (5a)-(5c), with every Jacobian
  formed by central differences of ``Model.functions``, not by the oracle's
  derivative code.
"""
import numpy as np
import pytest
from scipy.optimize import Bounds, NonlinearConstraint, minimize

from oracle import ipm, opf
from paper_2301_04869_gb300 import synth


@pytest.fixture(scope="module")
def problem():
    net, pd, qd = synth.workload("opf30_n1")
    M = opf.Model(net, pd, qd)
    st, k, _ = ipm.solve(M)
    return M, st


def central_jacobian(fun, w, rel=1e-6):
    """Jacobian of fun at w by central differences, step rel * max(1, |w_j|)."""
    cols = []
    for j in range(w.size):
        hj = rel * max(1.0, abs(w[j]))
        e = np.zeros_like(w)
        e[j] = hj
        cols.append((fun(w + e) - fun(w - e)) / (2.0 * hj))
    return np.stack(cols, axis=1)


def _split(M, w):
    nx = M.lay.nx
    return w[:nx], w[nx:]


def test_independent_nlp_solve_reaches_the_oracle_optimum(problem):
    M, st = problem
    nx, nu = M.lay.nx, M.lay.nu
    f = lambda w: M.functions(0, *_split(M, w))[0]
    g = lambda w: M.functions(0, *_split(M, w))[1]
    h = lambda w: M.functions(0, *_split(M, w))[2]
    # start from the flat point (theta = 0, V = 1, Pg at half range): the
    # oracle's optimum is not handed to the independent solve
    x0 = np.concatenate([np.zeros(M.lay.n - 1), np.ones(nx - M.lay.n + 1)])
    u0 = np.concatenate([np.ones(M.lay.ng), 0.5 * M.net.pmax[1:]])
    w0 = np.concatenate([x0, u0])
    lo = np.concatenate([M.xl, M.ul])
    hi = np.concatenate([M.xu, M.uu])
    cons = [NonlinearConstraint(g, 0.0, 0.0, jac="3-point"),
            NonlinearConstraint(h, -M.su, -M.sl, jac="3-point")]
    res = minimize(f, w0, method="trust-constr", jac="3-point", constraints=cons,
                   bounds=Bounds(lo, hi, keep_feasible=False),
                   options=dict(gtol=1e-11, xtol=1e-12, barrier_tol=1e-11, maxiter=3000))
    xs, us = _split(M, res.x)
    assert np.abs(g(res.x)).max() <= 1e-8
    f_o = M.functions(0, st["x"][0], st["u"])[0]
    assert abs(res.fun - f_o) <= 1e-6 * abs(f_o), (res.fun, f_o, res.message)
    np.testing.assert_allclose(us, st["u"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(xs, st["x"][0], rtol=0, atol=1e-5)


def test_oracle_duals_make_the_lagrangian_stationary(problem):
    M, st = problem
    x, u = st["x"][0], st["u"]
    w = np.concatenate([x, u])
    fgh = lambda w: np.concatenate([[M.functions(0, *_split(M, w))[0]],
                                    M.functions(0, *_split(M, w))[1],
                                    M.functions(0, *_split(M, w))[2]])
    J = central_jacobian(fgh, w)
    nx, m = M.lay.nx, M.lay.m
    grad_f, Jg, Jh = J[0], J[1:1 + nx], J[1 + nx:]
    zl = np.concatenate([st["zl_x"][0], st["zl_u"]])
    zu = np.concatenate([st["zu_x"][0], st["zu_u"]])
    # eq. (5a)/(5b): grad f + G^T y + H^T z - (lower duals) + (upper duals) = 0
    r = grad_f + Jg.T @ st["y"][0] + Jh.T @ st["z"][0] - zl + zu
    scale = max(1.0, np.abs(grad_f).max(), np.abs(st["y"]).max())
    assert np.abs(r).max() <= 1e-6 * scale, np.abs(r).max()
    # eq. (5c): z = (slack bound duals), the multiplier of h + s = 0
    assert np.abs(st["z"][0] - st["zl_s"][0] + st["zu_s"][0]).max() <= 1e-7
    # complementarity on every finite bound (eq. (5f)-(5h) at mu -> 0)
    for wv, l, b, a, c in ((w, np.concatenate([M.xl, M.ul]), np.concatenate([M.xu, M.uu]), zl, zu),
                           (st["s"][0], M.sl, M.su, st["zl_s"][0], st["zu_s"][0])):
        fl, fb = np.isfinite(l), np.isfinite(b)
        assert np.all(a[fl] >= 0) and np.all(c[fb] >= 0)
        assert np.abs(a[fl] * (wv[fl] - l[fl])).max(initial=0) <= 1e-7
        assert np.abs(c[fb] * (b[fb] - wv[fb])).max(initial=0) <= 1e-7
