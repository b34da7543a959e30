"""Pins of the oracle model derivatives (CPU).

The Jacobians are checked by complex-step differentiation of the analytic
cos/sin form of the bus injections (exact to rounding), the Hessian of the
Lagrangian by central differences of the Jacobian-transpose products, and the
injections themselves against a per-line branch-flow sum."""
import numpy as np
import pytest

from oracle import opf
from paper_2301_04869_gb300 import synth


@pytest.fixture(scope="module")
def model():
    net = synth.make_network(30, 6, seed=0)
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    return opf.Model(net, pd, qd)


def _point(model, seed=5):
    L = model.lay
    rng = np.random.default_rng(seed)
    x = np.concatenate([0.1 * rng.standard_normal(L.n - 1), 1 + 0.05 * rng.standard_normal(L.nx - L.n + 1)])
    u = np.concatenate([1 + 0.05 * rng.standard_normal(L.ng), rng.uniform(0, 2, L.ng - 1)])
    y = rng.standard_normal(L.nx)
    z = rng.standard_normal(L.m)
    return x, u, y, z


def _cs_jac(fun, w):
    h = 1e-30
    cols = []
    for j in range(w.size):
        wc = w.astype(complex)
        wc[j] += 1j * h
        cols.append(np.imag(fun(wc)) / h)
    return np.array(cols).T


def test_jacobians_complex_step(model):
    x, u, y, z = _point(model)
    nx = model.lay.nx
    d = model.derivatives(1, x, u, y, z)

    def stack(xc, uc):
        f, g, h = model.functions(1, xc, uc, cs=True)
        return np.concatenate([[f], g, h])

    Jx = _cs_jac(lambda xc: stack(xc, u.astype(complex)), x)
    Ju = _cs_jac(lambda uc: stack(x.astype(complex), uc), u)
    scale = max(1.0, np.abs(Jx).max(), np.abs(Ju).max())
    assert np.abs(Jx[0] - d["grad_x"]).max() <= 1e-12 * scale
    assert np.abs(Ju[0] - d["grad_u"]).max() <= 1e-12 * scale
    assert np.abs(Jx[1:1 + nx] - d["Gx"].toarray()).max() <= 1e-12 * scale
    assert np.abs(Ju[1:1 + nx] - d["Gu"].toarray()).max() <= 1e-12 * scale
    assert np.abs(Jx[1 + nx:] - d["Hx"].toarray()).max() <= 1e-12 * scale
    assert np.abs(Ju[1 + nx:] - d["Hu"].toarray()).max() <= 1e-12 * scale


def test_hessian_central_differences(model):
    x, u, y, z = _point(model, 7)
    nx = model.lay.nx
    d = model.derivatives(0, x, u, y, z)

    def lag_grad(w):
        dd = model.derivatives(0, w[:nx], w[nx:], y, z)
        return np.concatenate([dd["grad_x"] + dd["Gx"].T @ y + dd["Hx"].T @ z,
                               dd["grad_u"] + dd["Gu"].T @ y + dd["Hu"].T @ z])

    w = np.concatenate([x, u])
    H = np.zeros((w.size, w.size))
    for j in range(w.size):
        e = 1e-6 * max(1.0, abs(w[j]))
        wp, wm = w.copy(), w.copy()
        wp[j] += e
        wm[j] -= e
        H[:, j] = (lag_grad(wp) - lag_grad(wm)) / (2 * e)
    W = np.block([[d["Wxx"].toarray(), d["Wxu"].toarray()],
                  [d["Wxu"].toarray().T, d["Wuu"].toarray()]])
    assert np.abs(W - W.T).max() <= 1e-12 * np.abs(W).max()
    assert np.abs(H - W).max() <= 1e-6 * np.abs(W).max()


def test_injections_equal_branch_flows(model):
    """S_i from the admittance matrix equals the sum of the pi-model branch
    flows leaving bus i, and sum_i P_i equals the series losses r |I|^2."""
    net = model.net
    x, u, _, _ = _point(model, 9)
    th, v = opf.bus_voltage(model.lay, x, u)
    S = opf.injections(model.Y, th, v)
    V = v * np.exp(1j * th)
    ys = 1.0 / (net.r + 1j * net.x)
    Is = ys * (V[net.fr] - V[net.to])
    If = Is + 0.5j * net.b * V[net.fr]
    It = -Is + 0.5j * net.b * V[net.to]
    S2 = np.zeros(net.n_bus, dtype=complex)
    np.add.at(S2, net.fr, V[net.fr] * np.conj(If))
    np.add.at(S2, net.to, V[net.to] * np.conj(It))
    np.testing.assert_allclose(S, S2, rtol=0, atol=1e-12 * np.abs(S).max())
    assert abs(S.real.sum() - np.sum(net.r * np.abs(Is) ** 2)) <= 1e-11 * np.abs(S).max()


def test_layout_sizes(model):
    L = model.lay
    n, ng = L.n, L.ng
    assert L.nx == 2 * n - 1 - ng and L.nu == 2 * ng - 1 and L.m == ng + 1
    # G_x rows and x columns use the same bus positions (square, diagonal pivots)
    x, u, y, z = _point(model)
    d = model.derivatives(0, x, u, y, z)
    assert d["Gx"].shape == (L.nx, L.nx)
    assert np.all(np.abs(d["Gx"].diagonal()) > 0)
