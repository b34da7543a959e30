"""Pins of the oracle model derivatives (CPU).

The Jacobians are checked by complex-step differentiation of the analytic
cos/sin form of the bus injections (exact to rounding), the Hessian of the
Lagrangian by central differences of the Jacobian-transpose products, and the
injections themselves against a per-line branch-flow sum."""
import numpy as np
import pytest

from oracle import opf
from paper_2301_04869_gb300 import synth


@pytest.fixture(scope="module", params=["plain", "rated", "tripped"])
def model(request):
    """The 30-bus network without and with line ratings (the rated one adds
    the 2L squared apparent-flow rows of §4.1.1 to h), and rated with a line
    out of service in scenario 1 (the scenario the pins evaluate)."""
    net = synth.make_network(30, 6, seed=0)
    if request.param != "plain":
        net = synth.with_ratings(net, np.ones(net.n_line))
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    trip = None
    if request.param == "tripped":
        trip = np.array([-1, int(np.flatnonzero(~synth.bridges(net))[3])])
    return opf.Model(net, pd, qd, trip=trip)


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
    assert L.nx == 2 * n - 1 - ng and L.nu == 2 * ng - 1
    assert L.m == ng + 1 + (2 * model.net.n_line if L.rated else 0)
    # G_x rows and x columns use the same bus positions (square, diagonal pivots)
    x, u, y, z = _point(model)
    d = model.derivatives(0, x, u, y, z)
    assert d["Gx"].shape == (L.nx, L.nx)
    assert np.all(np.abs(d["Gx"].diagonal()) > 0)


def test_flow_rows_equal_line_end_powers(model):
    """With ratings, h holds |V_f conj(I_f)|^2 and |V_t conj(I_t)|^2 of every
    line (pi model: I_f = y (V_f - V_t) + j b/2 V_f), written out here per
    line; the slack box of those rows is s >= -rate^2 only."""
    if not model.lay.rated:
        pytest.skip("no ratings")
    net = model.net
    x, u, _, _ = _point(model, 11)
    _, _, h = model.functions(1, x, u)
    th, v = opf.bus_voltage(model.lay, x, u)
    V = v * np.exp(1j * th)
    ys = 1.0 / (net.r + 1j * net.x)
    If = ys * (V[net.fr] - V[net.to]) + 0.5j * net.b * V[net.fr]
    It = ys * (V[net.to] - V[net.fr]) + 0.5j * net.b * V[net.to]
    ng, L = model.lay.ng, net.n_line
    on = np.ones(L)
    if model.trip is not None and model.trip[1] >= 0:
        on[model.trip[1]] = 0.0  # a line out of service carries nothing
    np.testing.assert_allclose(h[ng + 1:ng + 1 + L], on * np.abs(V[net.fr] * np.conj(If)) ** 2, rtol=1e-13)
    np.testing.assert_allclose(h[ng + 1 + L:], on * np.abs(V[net.to] * np.conj(It)) ** 2, rtol=1e-13)
    assert np.all(model.sl[ng + 1:] == -np.tile(net.rate ** 2, 2)) and np.all(np.isinf(model.su[ng + 1:]))


def test_tripped_scenario_equals_network_without_the_line():
    """A scenario with a line out of service evaluates exactly like a model of
    the network with that line deleted (a separate network object)."""
    import copy
    net = synth.with_ratings(synth.make_network(30, 6, seed=0), np.ones(41))
    pd, qd = synth.make_scenarios(net, 2, 0.05, seed=1)
    l = int(np.flatnonzero(~synth.bridges(net))[5])
    M = opf.Model(net, pd, qd, trip=np.array([-1, l]))
    keep = np.arange(net.n_line) != l
    cut = copy.copy(net)
    for a in ("fr", "to", "r", "x", "b", "rate"):
        setattr(cut, a, getattr(net, a)[keep])
    Mc = opf.Model(cut, pd[1:], qd[1:])
    x, u, y, _ = _point(M, 13)
    z = np.random.default_rng(3).standard_normal(M.lay.m)
    d = M.derivatives(1, x, u, y, z)
    # the cut model has 2 fewer flow rows: drop line l's two rows
    L, ng = net.n_line, M.lay.ng
    rows = np.r_[0:ng + 1, ng + 1 + np.flatnonzero(keep), ng + 1 + L + np.flatnonzero(keep)]
    zc = z[rows]
    dc = Mc.derivatives(0, x, u, y, zc)
    assert abs(d["f"] * 2 - dc["f"]) <= 1e-14 * abs(dc["f"])  # objective weight 1/N
    np.testing.assert_allclose(d["g"], dc["g"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(d["h"][rows], dc["h"], rtol=0, atol=1e-13)
    assert np.all(d["h"][[ng + 1 + l, ng + 1 + L + l]] == 0.0)
    for k in ("Gx", "Gu"):
        np.testing.assert_allclose(d[k].toarray(), dc[k].toarray(), rtol=0, atol=1e-12)
    for k in ("Hx", "Hu"):
        np.testing.assert_allclose(d[k].toarray()[rows], dc[k].toarray(), rtol=0, atol=1e-12)
    # W: the cost term is weighted 1/N in both models (N = 2 vs 1)
    dW = M.derivatives(1, x, u, y, z)["Wxx"] - 0.5 * Mc.derivatives(0, x, u, np.zeros_like(y), np.zeros_like(zc))["Wxx"]
    dWc = dc["Wxx"] - Mc.derivatives(0, x, u, np.zeros_like(y), np.zeros_like(zc))["Wxx"]
    np.testing.assert_allclose(dW.toarray(), dWc.toarray(), rtol=0, atol=1e-11)
