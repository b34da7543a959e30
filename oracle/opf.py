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
        and, when the network carries line ratings, the line-flow limits
        of §4.1.1 as |S_f,l|^2 and |S_t,l|^2 (apparent power at both ends of
        every line, bounded above by rate_l^2)          m = n_g+1+2L
  f_i = (1/N) * generation cost (slack Pg is a function of x_i, u)
These sizes reproduce every row of the paper's Table "MATPOWER instances" and
the nvar / ncon columns of its Table of instance dimensions (with limits).

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
        # h rows: Q at gen buses, then P at bus 0, then (with ratings) the
        # squared apparent flow at the from end of every line, then at the
        # to end
        self.h_in_a = np.concatenate([n + gb, [0]])
        self.rated = getattr(net, "rate", None) is not None
        self.L = int(np.asarray(net.fr).shape[0])
        self.m = self.ng + 1 + (2 * self.L if self.rated else 0)


def admittance(net, on=None):
    """Bus admittance matrix of the pi-model lines (no taps, no shunts):
    Y_ff = Y_tt = y + j b/2, Y_ft = Y_tf = -y with y = 1/(r + j x).
    on: optional 0/1 status per line (a line out of service stamps nothing)."""
    n = net.n_bus
    y = 1.0 / (net.r + 1j * net.x)
    ysh = 0.5j * net.b
    if on is not None:
        y, ysh = y * on, ysh * on
    f = np.asarray(net.fr, dtype=np.int64)
    t = np.asarray(net.to, dtype=np.int64)
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([y + ysh, y + ysh, -y, -y])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def branch_admittance(net, on=None):
    """From- and to-end branch admittance matrices (L x n) of the pi model:
    I_f = Y_f V with Y_f[l, f] = y + j b/2, Y_f[l, t] = -y (and the mirror for
    the to end), and the end selectors C_f, C_t (L x n).  on: optional 0/1
    status per line (a line out of service carries no current)."""
    n = net.n_bus
    y = 1.0 / (net.r + 1j * net.x)
    ysh = 0.5j * net.b
    if on is not None:
        y, ysh = y * on, ysh * on
    f = np.asarray(net.fr, dtype=np.int64)
    t = np.asarray(net.to, dtype=np.int64)
    L = f.size
    ls = np.arange(L)
    Yf = sp.csr_matrix((np.concatenate([y + ysh, -y]), (np.concatenate([ls, ls]), np.concatenate([f, t]))),
                       shape=(L, n))
    Yt = sp.csr_matrix((np.concatenate([y + ysh, -y]), (np.concatenate([ls, ls]), np.concatenate([t, f]))),
                       shape=(L, n))
    Cf = sp.csr_matrix((np.ones(L), (ls, f)), shape=(L, n))
    Ct = sp.csr_matrix((np.ones(L), (ls, t)), shape=(L, n))
    return Yf, Yt, Cf, Ct


def branch_flows(Yb, Cb, theta, v):
    """Complex power entering the lines at one end: S = (C V) o conj(Y_b V)."""
    V = v * np.exp(1j * theta)
    return (Cb @ V) * np.conj(Yb @ V)


def branch_flows_cs(Yb, Cb, theta, v):
    """(P, Q) of branch_flows written with cos/sin, analytic in (theta, v) for
    complex-step differentiation: with m the end's bus and k = the other,
    S = sum_k v_m v_k conj(Y_lk) e^{j(th_m - th_k)}."""
    Yc = Yb.tocoo()
    mb = Cb.tocsr().indices.astype(np.int64)  # one entry per row: the end's bus
    l, k = Yc.row, Yc.col
    m = mb[l]
    d = theta[m] - theta[k]
    vv = v[m] * v[k]
    G, B = Yc.data.real, Yc.data.imag
    P = np.zeros(Cb.shape[0], dtype=np.result_type(theta, v))
    Q = np.zeros(Cb.shape[0], dtype=np.result_type(theta, v))
    np.add.at(P, l, vv * (G * np.cos(d) + B * np.sin(d)))
    np.add.at(Q, l, vv * (G * np.sin(d) - B * np.cos(d)))
    return P, Q


def dSb_da(Yb, Cb, theta, v):
    """Jacobian of the branch flows S = (C V) o conj(Y_b V) w.r.t. theta and
    v (complex sparse L x n each): with D_a = diag(dV/da),
      dS/da = diag(conj(Y_b V)) C D_a + diag(C V) conj(Y_b) conj(D_a)."""
    V = v * np.exp(1j * theta)
    Ib = Yb @ V
    Dth = sp.diags(1j * V)
    Dv = sp.diags(V / v)
    dI = sp.diags(np.conj(Ib))
    dV = sp.diags(Cb @ V)
    Ybc = Yb.conj()
    return (dI @ Cb @ Dth + dV @ Ybc @ Dth.conj()).tocsr(), (dI @ Cb @ Dv + dV @ Ybc @ Dv.conj()).tocsr()


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
    mu = lamP - 1j * lamQ
    return hess_re_vmv(sp.diags(mu) @ Y.conj(), theta, v)


def hess_re_vmv(M, theta, v):
    """Hessian w.r.t. a = (theta, v) of F = Re(V^T M conj(V)) for a complex
    sparse n x n matrix M, by the product rule of hess_weighted_S."""
    V = v * np.exp(1j * theta)
    M = sp.csr_matrix(M)
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
    (the paper minimises the average cost, §2.1).  trip: optional int[N], the
    line out of service in each scenario or -1 (line-tripping contingencies,
    §4.1.1): that scenario's admittances leave the line out."""

    def __init__(self, net, pd, qd, trip=None):
        self.net = net
        self.lay = Layout(net)
        self.pd = np.atleast_2d(np.asarray(pd, dtype=np.float64))
        N = self.pd.shape[0]
        self.trip = None if trip is None else np.asarray(trip, dtype=np.int64)
        self._Y, self._B = {}, {}
        self.Y = admittance(net)
        if self.lay.rated:
            self.rate = np.asarray(net.rate, dtype=np.float64)
        assert self.trip is None or self.trip.shape == (N,)
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
        # h in [hmin, hmax]  ->  s = -h in [-hmax, -hmin]; a flow row is
        # bounded above only (|S|^2 <= rate^2)
        hmin = np.concatenate([-net.qmax, [0.0]])
        hmax = np.concatenate([net.qmax, [net.pmax[0]]])
        if L.rated:
            hmin = np.concatenate([hmin, np.full(2 * L.L, -inf)])
            hmax = np.concatenate([hmax, np.tile(self.rate ** 2, 2)])
        self.sl = -hmax
        self.su = -hmin

    def _on(self, i):
        if self.trip is None or self.trip[i] < 0:
            return None
        on = np.ones(self.lay.L)
        on[self.trip[i]] = 0.0
        return on

    def Y_of(self, i):
        """Bus admittance matrix of scenario i."""
        t = -1 if self.trip is None else int(self.trip[i])
        if t not in self._Y:
            self._Y[t] = admittance(self.net, self._on(i))
        return self._Y[t]

    def branches_of(self, i):
        """((Y_f, C_f), (Y_t, C_t)) of scenario i."""
        t = -1 if self.trip is None else int(self.trip[i])
        if t not in self._B:
            Yf, Yt, Cf, Ct = branch_admittance(self.net, self._on(i))
            self._B[t] = ((Yf, Cf), (Yt, Ct))
        return self._B[t]

    # -- functions -------------------------------------------------------
    def functions(self, i, x, u, cs=False):
        """(f_i, g_i, h_i) at (x_i, u).  cs=True uses the analytic cos/sin
        form so complex-step differentiation is exact."""
        L, net = self.lay, self.net
        n, ng = L.n, L.ng
        th, v = bus_voltage(L, x, u)
        if cs:
            P, Q = injections_cs(self.Y_of(i), th, v)
        else:
            S = injections(self.Y_of(i), th, v)
            P, Q = S.real, S.imag
        pd, qd = self.pd[i], self.qd[i]
        Pg = np.zeros(n, dtype=P.dtype)
        Pg[L.gen_bus[1:]] = u[ng:]
        gP = P + pd - Pg
        gQ = Q + qd
        g = np.concatenate([gP[1:], gQ[L.pq]])
        pg0 = P[0] + pd[0]
        h = np.concatenate([gQ[L.gen_bus], [pg0]])
        if L.rated:
            flows = []
            for Yb, Cb in self.branches_of(i):
                if cs:
                    Pb, Qb = branch_flows_cs(Yb, Cb, th, v)
                else:
                    Sb = branch_flows(Yb, Cb, th, v)
                    Pb, Qb = Sb.real, Sb.imag
                flows.append(Pb * Pb + Qb * Qb)
            h = np.concatenate([h] + flows)
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
        Sth, Sv = dS_da(self.Y_of(i), th, v)
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
        if L.rated:
            # flow rows: d|S_b|^2 = 2 (P dP + Q dQ) in bus space
            th_, v_ = bus_voltage(L, x, u)
            Hb, Wb = [], None
            zf = z[ng + 1:ng + 1 + L.L]
            zt = z[ng + 1 + L.L:]
            for (Yb, Cb), zb in zip(self.branches_of(i), (zf, zt)):
                Sb = branch_flows(Yb, Cb, th_, v_)
                dth, dv = dSb_da(Yb, Cb, th_, v_)
                dS = sp.hstack([dth, dv]).tocsr()          # L x 2n complex
                dP, dQ = dS.real, dS.imag
                Hb.append(2.0 * (sp.diags(Sb.real) @ dP + sp.diags(Sb.imag) @ dQ))
                # Hessian of sum_l z_l |S_l|^2 = 2 sum z (dP dP^T + dQ dQ^T)
                #   + Hessian of sum_l (2 z_l P_l) P_l + (2 z_l Q_l) Q_l (weights held)
                mu_b = 2.0 * zb * (Sb.real - 1j * Sb.imag)
                Wl = (2.0 * (dP.T @ sp.diags(zb) @ dP + dQ.T @ sp.diags(zb) @ dQ)
                      + hess_re_vmv(Cb.T @ sp.diags(mu_b) @ Yb.conj(), th_, v_))
                Wb = Wl if Wb is None else Wb + Wl
            Hb = sp.vstack(Hb).tocsr()
            Hx = sp.vstack([Hx, Hb[:, L.x_in_a]])
            Hu = sp.vstack([Hu, Hb[:, L.uv_in_a]])
        Hu = sp.hstack([Hu, sp.csr_matrix((L.m, ng - 1))]).tocsr()
        # objective gradient
        pg0 = h[ng]
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
        Ha = hess_weighted_S(self.Y_of(i), th, v, lamP, lamQ)
        # cost curvature through the slack injection: (2 c2_0 / N) dP0 dP0^T
        Ha = Ha + (2 * net.c2[0] / N) * _outer_sparse(gradP0)
        if L.rated:
            Ha = (Ha + Wb).tocsr()
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
