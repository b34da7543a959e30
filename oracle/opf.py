"""Oracle model: two-stage stochastic AC-OPF in the paper's block form.

Test infrastructure only (see ``oracle/__init__``).

Problem (§2, eq. (2)/(3); OPF case study §4.1.1): for scenarios i = 1..N,
  min  sum_i f_i(x_i, u)
  s.t. g_i(x_i, u) = 0            (power balance = state equation)
       h_i(x_i, u) + s_i = 0       (operational constraints, slack form eq. (3))
       bounds on x_i, u, s_i
with
  x_i = (theta at buses 1..n-1, |V| at non-generator buses)      n_x = 2n-1-n_g
  u   = (|V| at generator buses, Pg at non-slack generators)      n_u = 2n_g-1
  g_i = (P-balance at buses 1..n-1, Q-balance at non-generator buses)
  h_i = (Qg of every generator, Pg of the slack generator)        m = n_g+1
  f_i = (1/N) * generation cost (slack Pg is a function of x_i, u)
These sizes reproduce every row of the paper's Table "MATPOWER instances".

Derivatives use complex-matrix notation on the bus admittance matrix
Y = sum over lines of the pi-model stamps.  With V = v*exp(j*theta),
S = diag(V) conj(Y V), and for a multiplier vector mu = lamP - j lamQ,
F = Re(mu^T S) = Re(V^T M conj(V)), M = diag(mu) conj(Y); the product rule
then gives the Hessian of F (derived in ``hess_weighted_S``).  The GPU path
uses a different (real, line-wise) formulation, so agreement between the two
is a real check.  Pins: complex-step / finite differences (tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Layout:
    """Variable / row index maps of one network (no arithmetic of the method).

    Bus-space vector a = (theta_0..theta_{n-1}, v_0..v_{n-1}); rows of the bus
    injections are (P_0..P_{n-1}, Q_0..Q_{n-1}) in the same order."""

    def __init__(self, net):
        n = net.n_bus
        self.n = n
        self.ng = net.n_gen
        gb = np.asarray(net.gen_bus, dtype=np.int64)
        self.gen_bus = gb
        is_gen = np.zeros(n, dtype=bool)
        is_gen[gb] = True
        self.pq = np.flatnonzero(~is_gen)
        # x = (theta_1..theta_{n-1}, v_pq); g rows use the same positions
        self.x_in_a = np.concatenate([np.arange(1, n), n + self.pq])
        self.nx = self.x_in_a.size
        # u = (v at gen buses, Pg_1..Pg_{ng-1})
        self.uv_in_a = n + gb
        self.nu = 2 * self.ng - 1
        self.m = self.ng + 1
        # h rows: Q at gen buses, then P at bus 0
        self.h_in_a = np.concatenate([n + gb, [0]])


def admittance(net):
    """Bus admittance matrix of the pi-model lines (no taps, no shunts):
    Y_ff = Y_tt = y + j b/2, Y_ft = Y_tf = -y with y = 1/(r + j x)."""
    n = net.n_bus
    y = 1.0 / (net.r + 1j * net.x)
    ysh = 0.5j * net.b
    f = np.asarray(net.fr, dtype=np.int64)
    t = np.asarray(net.to, dtype=np.int64)
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([y + ysh, y + ysh, -y, -y])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def bus_voltage(lay, x, u):
    """Full bus (theta, v) vectors from (x, u); theta_0 = 0 (reference)."""
    n = lay.n
    a = np.zeros(2 * n, dtype=np.result_type(x, u))
    a[lay.x_in_a] = x
    a[lay.uv_in_a] = u[: lay.ng]
    return a[:n], a[n:]


def injections(Y, theta, v):
    """Complex power injections S = V * conj(Y V)."""
    V = v * np.exp(1j * theta)
    return V * np.conj(Y @ V)


def injections_cs(Y, theta, v):
    """Complex-step-safe variant: P and Q as analytic functions of (theta, v).

    Writing P and Q out with cos/sin keeps them analytic in each real input,
    so a complex perturbation gives exact first derivatives.  Returns (P, Q)."""
    G = Y.real.tocsr()
    B = Y.imag.tocsr()
    n = theta.shape[0]
    Gc = G.tocoo()
    Bc = B.tocoo()
    P = np.zeros(n, dtype=np.result_type(theta, v))
    Q = np.zeros(n, dtype=np.result_type(theta, v))
    # P_i = v_i sum_k v_k (G_ik cos(th_i - th_k) + B_ik sin(th_i - th_k))
    # Q_i = v_i sum_k v_k (G_ik sin(th_i - th_k) - B_ik cos(th_i - th_k))
    assert np.array_equal(Gc.row, Bc.row) and np.array_equal(Gc.col, Bc.col)
    i, k = Gc.row, Gc.col
    d = theta[i] - theta[k]
    vv = v[i] * v[k]
    np.add.at(P, i, vv * (Gc.data * np.cos(d) + Bc.data * np.sin(d)))
    np.add.at(Q, i, vv * (Gc.data * np.sin(d) - Bc.data * np.cos(d)))
    return P, Q


def dS_da(Y, theta, v):
    """Jacobian of S w.r.t. theta and v (complex sparse n x n each).

    S_i = V_i conj(I_i), I = Y V.  With D_a = diag(dV/da):
      dS/da = diag(conj(I)) D_a + diag(V) conj(Y) conj(D_a),
    D_theta = diag(j V), D_v = diag(V / v)."""
    V = v * np.exp(1j * theta)
    I = Y @ V
    Dth = sp.diags(1j * V)
    Dv = sp.diags(V / v)
    dI = sp.diags(np.conj(I))
    dV = sp.diags(V)
    Yc = Y.conj()
    dS_dth = dI @ Dth + dV @ Yc @ Dth.conj()
    dS_dv = dI @ Dv + dV @ Yc @ Dv.conj()
    return dS_dth.tocsr(), dS_dv.tocsr()


def hess_weighted_S(Y, theta, v, lamP, lamQ):
    """Hessian w.r.t. a = (theta, v) of F = sum_i lamP_i P_i + lamQ_i Q_i.

    F = Re(V^T M conj(V)), M = diag(lamP - j lamQ) conj(Y).  By the product
    rule, with V' = dV/da, V'' = d2V/da db (only on the diagonal):
      H_ab = Re( diag(V''_ab o (M conj V)) + D_a M conj(D_b)
                 + diag(conj(V''_ab) o (M^T V)) + conj(D_a) M^T D_b )
    where dV/dtheta = jV, dV/dv = V/v, d2V/dtheta2 = -V,
    d2V/dtheta dv = jV/v, d2V/dv2 = 0.
    Returns a real sparse (2n x 2n) matrix."""
    V = v * np.exp(1j * theta)
    mu = lamP - 1j * lamQ
    M = sp.diags(mu) @ Y.conj()
    MVc = M @ np.conj(V)
    MtV = M.T @ V
    Dp = {"t": 1j * V, "v": V / v}
    Dpp = {("t", "t"): -V, ("t", "v"): 1j * V / v, ("v", "t"): 1j * V / v,
           ("v", "v"): np.zeros_like(V)}
    blocks = {}
    for a in ("t", "v"):
        for b in ("t", "v"):
            Da = sp.diags(Dp[a])
            Db = sp.diags(Dp[b])
            Vpp = Dpp[(a, b)]
            H = (sp.diags(Vpp * MVc) + Da @ M @ Db.conj()
                 + sp.diags(np.conj(Vpp) * MtV) + Da.conj() @ M.T @ Db)
            blocks[(a, b)] = H.real
    return sp.bmat([[blocks[("t", "t")], blocks[("t", "v")]],
                    [blocks[("v", "t")], blocks[("v", "v")]]]).tocsr()


class Model:
    """Per-scenario functions and derivatives of one network.

    pd, qd: float64[N, n] scenario loads.  Objective weight 1/N per scenario
    (the paper minimises the average cost, §2.1)."""

    def __init__(self, net, pd, qd):
        self.net = net
        self.lay = Layout(net)
        self.Y = admittance(net)
        self.pd = np.atleast_2d(np.asarray(pd, dtype=np.float64))
        self.qd = np.atleast_2d(np.asarray(qd, dtype=np.float64))
        self.N = self.pd.shape[0]
        L = self.lay
        n, ng = L.n, L.ng
        # G_u Pg columns: dP_i/dPg_k = -1 at gen bus of k (k >= 1)
        # bounds
        inf = np.inf
        self.xl = np.concatenate([np.full(n - 1, -inf), net.vmin[L.pq]])
        self.xu = np.concatenate([np.full(n - 1, inf), net.vmax[L.pq]])
        self.ul = np.concatenate([net.vmin[L.gen_bus], np.zeros(ng - 1)])
        self.uu = np.concatenate([net.vmax[L.gen_bus], net.pmax[1:]])
        # h in [hmin, hmax]  ->  s = -h in [-hmax, -hmin]
        hmin = np.concatenate([-net.qmax, [0.0]])
        hmax = np.concatenate([net.qmax, [net.pmax[0]]])
        self.sl = -hmax
        self.su = -hmin

    # -- functions -------------------------------------------------------
    def functions(self, i, x, u, cs=False):
        """(f_i, g_i, h_i) at (x_i, u).  cs=True uses the analytic cos/sin
        form so complex-step differentiation is exact."""
        L, net = self.lay, self.net
        n, ng = L.n, L.ng
        th, v = bus_voltage(L, x, u)
        if cs:
            P, Q = injections_cs(self.Y, th, v)
        else:
            S = injections(self.Y, th, v)
            P, Q = S.real, S.imag
        pd, qd = self.pd[i], self.qd[i]
        Pg = np.zeros(n, dtype=P.dtype)
        Pg[L.gen_bus[1:]] = u[ng:]
        gP = P + pd - Pg
        gQ = Q + qd
        g = np.concatenate([gP[1:], gQ[L.pq]])
        h = np.concatenate([gQ[L.gen_bus], [P[0] + pd[0]]])
        pg0 = h[-1]
        pg = u[ng:]
        cost = (np.sum(net.c2[1:] * pg * pg + net.c1[1:] * pg)
                + net.c2[0] * pg0 * pg0 + net.c1[0] * pg0)
        return cost / self.N, g, h

    # -- first and second derivatives ------------------------------------
    def derivatives(self, i, x, u, y, z):
        """All first/second-order quantities of scenario i at (x_i, u) with
        multipliers y_i (for g_i) and z_i (for h_i + s_i = 0).

        Returns dict with f, g, h, grad_x, grad_u, Gx, Gu, Hx, Hu (sparse),
        Wxx, Wxu, Wuu (sparse): W is the Hessian of
        f_i + y^T g_i + z^T h_i (eq. (4) without the bound terms)."""
        L, net = self.lay, self.net
        n, ng, N = L.n, L.ng, self.N
        f, g, h = self.functions(i, x, u)
        th, v = bus_voltage(L, x, u)
        Sth, Sv = dS_da(self.Y, th, v)
        J = sp.bmat([[Sth.real, Sv.real], [Sth.imag, Sv.imag]]).tocsr()  # 2n x 2n
        # column selectors (bus space -> x / u-voltage parts)
        Jx = J[:, L.x_in_a]
        Juv = J[:, L.uv_in_a]
        # Pg columns of g: -1 at P row of each non-slack gen bus
        gP_rows_of_gen = L.gen_bus[1:]  # bus index = P row in bus space
        Jpg = sp.csr_matrix((-np.ones(ng - 1), (gP_rows_of_gen, np.arange(ng - 1))),
                            shape=(2 * n, ng - 1))
        Ju = sp.hstack([Juv, Jpg]).tocsr()
        Gx = Jx[L.x_in_a, :]
        Gu = Ju[L.x_in_a, :]
        Hx = Jx[L.h_in_a, :]
        Hu = Juv[L.h_in_a, :]
        Hu = sp.hstack([Hu, sp.csr_matrix((L.m, ng - 1))]).tocsr()
        # objective gradient
        pg0 = h[-1]
        dcost0 = (2 * net.c2[0] * pg0 + net.c1[0]) / N
        gradP0 = J[0, :].toarray().ravel()  # dP_0/da
        grad_a = dcost0 * gradP0
        grad_x = grad_a[L.x_in_a]
        pg = u[ng:]
        grad_u = np.concatenate([grad_a[L.uv_in_a],
                                 (2 * net.c2[1:] * pg + net.c1[1:]) / N])
        # Hessian of the Lagrangian: weights on P and Q of every bus
        lamP = np.zeros(n)
        lamQ = np.zeros(n)
        lamP[1:] += y[: n - 1]
        lamQ[L.pq] += y[n - 1:]
        lamQ[L.gen_bus] += z[:ng]
        lamP[0] += z[ng] + dcost0
        Ha = hess_weighted_S(self.Y, th, v, lamP, lamQ)
        # cost curvature through the slack injection: (2 c2_0 / N) dP0 dP0^T
        Ha = Ha + (2 * net.c2[0] / N) * _outer_sparse(gradP0)
        Wxx = Ha[L.x_in_a, :][:, L.x_in_a]
        Wxuv = Ha[L.x_in_a, :][:, L.uv_in_a]
        Wuvuv = Ha[L.uv_in_a, :][:, L.uv_in_a]
        Wxu = sp.hstack([Wxuv, sp.csr_matrix((L.nx, ng - 1))]).tocsr()
        Wpp = sp.diags(2 * net.c2[1:] / N)
        Wuu = sp.bmat([[Wuvuv, None], [None, Wpp]]).tocsr()
        return dict(f=f, g=g, h=h, grad_x=grad_x, grad_u=grad_u, Gx=Gx.tocsr(),
                    Gu=Gu.tocsr(), Hx=Hx.tocsr(), Hu=Hu, Wxx=Wxx.tocsr(),
                    Wxu=Wxu, Wuu=Wuu)


def _outer_sparse(vec):
    nz = np.flatnonzero(vec)
    r = np.repeat(nz, nz.size)
    c = np.tile(nz, nz.size)
    vals = vec[r] * vec[c]
    return sp.csr_matrix((vals, (r, c)), shape=(vec.size, vec.size))


def dimensions(n_bus, n_line, n_gen, N, line_limits=False):
    """(n_x, n_u, m, nvar, ncon) of the block problem: nvar = N n_x + n_u,
    ncon = N (n_x + m) (§2.1), m = n_g + 1 (+ 2L with line-flow limits)."""
    nx = 2 * n_bus - 1 - n_gen
    nu = 2 * n_gen - 1
    m = n_gen + 1 + (2 * n_line if line_limits else 0)
    return nx, nu, m, N * nx + nu, N * (nx + m)
