"""Oracle KKT algebra: augmented system, condensation, reduction, Schur.

Test infrastructure only (see ``oracle/__init__``).

Every function follows a plain definition from §2.2-§2.3 of the paper:
  * augmented Newton system, eq. (6) (``augmented_dense``),
  * condensation, Prop. 2.1 and the block form of K, Prop. 2.2
    (``condensed_blocks``),
  * reduction Z = [-(G_x^i)^{-1} G_u^i; I], K_hat = Z^T K Z and the reduced
    right-hand side eq. (11), recovery of p_x, p_y (Prop. 2.3)
    (``reduced_step``),
  * the Schur complement S_uu = A_0 - sum_i B_i A_i^{-1} B_i^T with the
    explicit A_i^{-1} of eq. (15) (``schur_explicit``).
Sparse LU (scipy SuperLU with its own pivoting) and dense Cholesky (LAPACK)
serve as library steps.  Pins: tests/test_oracle_kkt.py.

Conventions.  Bounds are two-sided boxes (infinite entries allowed); the
paper's one-sided x >= 0 form is the special case.  For a primal block w with
bounds l <= w <= b and bound duals (zl, zu):
  Sigma_w = zl / (w - l) + zu / (b - w)          (primal-dual barrier diagonal)
  r1 part = grad + J^T lambda - mu / (w - l) + mu / (b - w)
The inequality rows use h_i(x_i, u) + s_i = 0 exactly as eq. (3); their slack
box is s in [-h_max, -h_min].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _fin(a):
    return np.isfinite(a)


def sigma(w, l, b, zl, zu):
    """Barrier diagonal zl/(w-l) + zu/(b-w), zero on infinite bounds."""
    out = np.zeros_like(w)
    ml, mu_ = _fin(l), _fin(b)
    out[ml] += zl[ml] / (w[ml] - l[ml])
    out[mu_] += zu[mu_] / (b[mu_] - w[mu_])
    return out


def barrier_grad(w, l, b, mu):
    """Gradient of -mu sum log(w-l) - mu sum log(b-w)."""
    out = np.zeros_like(w)
    ml, mu_ = _fin(l), _fin(b)
    out[ml] -= mu / (w[ml] - l[ml])
    out[mu_] += mu / (b[mu_] - w[mu_])
    return out


def barrier_value(w, l, b, mu):
    ml, mu_ = _fin(l), _fin(b)
    return -mu * (np.sum(np.log(w[ml] - l[ml])) + np.sum(np.log(b[mu_] - w[mu_])))


def eval_all(model, st):
    """Derivatives of every scenario at the state (list of dicts)."""
    return [model.derivatives(i, st["x"][i], st["u"], st["y"][i], st["z"][i])
            for i in range(model.N)]


def residuals(model, st, D, mu):
    """Right-hand sides r1..r4 of eq. (6) at barrier parameter mu.

    r1 = grad f + G^T y + H^T z - mu/(w-l) + mu/(b-w)  (x blocks, coupled u)
    r2 = z - mu/(s-l_s) + mu/(b_s-s),  r3 = g,  r4 = h + s."""
    N = model.N
    r1x = np.empty_like(st["x"])
    r1u = barrier_grad(st["u"], model.ul, model.uu, mu)
    r2 = np.empty_like(st["s"])
    r3 = np.empty_like(st["x"])
    r4 = np.empty_like(st["s"])
    for i in range(N):
        d = D[i]
        r1x[i] = (d["grad_x"] + d["Gx"].T @ st["y"][i] + d["Hx"].T @ st["z"][i]
                  + barrier_grad(st["x"][i], model.xl, model.xu, mu))
        r1u += d["grad_u"] + d["Gu"].T @ st["y"][i] + d["Hu"].T @ st["z"][i]
        r2[i] = st["z"][i] + barrier_grad(st["s"][i], model.sl, model.su, mu)
        r3[i] = d["g"]
        r4[i] = d["h"] + st["s"][i]
    return r1x, r1u, r2, r3, r4


def sigmas(model, st):
    N = model.N
    Sx = np.stack([sigma(st["x"][i], model.xl, model.xu, st["zl_x"][i], st["zu_x"][i])
                   for i in range(N)])
    Su = sigma(st["u"], model.ul, model.uu, st["zl_u"], st["zu_u"])
    Ss = np.stack([sigma(st["s"][i], model.sl, model.su, st["zl_s"][i], st["zu_s"][i])
                   for i in range(N)])
    return Sx, Su, Ss


def condensed_blocks(d, Sx_i, Ss_i, r1x_i, r2_i, r4_i, delta):
    """Prop. 2.1/2.2 for one scenario.

    K_xx = W_xx + Sigma_x + H_x^T Sigma_s H_x (+ delta I)
    K_xu = W_xu + H_x^T Sigma_s H_u
    K_uu^i = W_uu^i + H_u^T Sigma_s H_u   (scenario part; Sigma_u, delta I and
                                           the first-stage terms are added once)
    rhat1_x = r1_x + H_x^T (Sigma_s r4 - r2);   rhat_u^i = H_u^T (Sigma_s r4 - r2)
    """
    S = sp.diags(Ss_i)
    nx = Sx_i.size
    Kxx = (d["Wxx"] + sp.diags(Sx_i + delta) + d["Hx"].T @ S @ d["Hx"]).tocsr()
    Kxu = (d["Wxu"] + d["Hx"].T @ S @ d["Hu"]).tocsr()
    Kuu = (d["Wuu"] + d["Hu"].T @ S @ d["Hu"]).tocsr()
    t = Ss_i * r4_i - r2_i
    rh1x = r1x_i + d["Hx"].T @ t
    rhu = d["Hu"].T @ t
    assert Kxx.shape == (nx, nx)
    return Kxx, Kxu, Kuu, rh1x, rhu


class Condensed:
    """Condensed and reduced data of all scenarios at one iterate."""


def condense(model, st, D, mu, delta=0.0, keep_Z=True):
    """Form K_hat = sum_i Z_i^T K_i Z_i + (Sigma_u + delta I), Prop. 2.3, and
    the reduced right-hand side of eq. (11).

    Z_i = -(G_x^i)^{-1} G_u^i by sparse LU; K_hat_i = Z^T K Z expanded as
    Z_x^T K_xx Z_x + Z_x^T K_xu + K_ux Z_x + K_uu^i."""
    N = model.N
    r1x, r1u, r2, r3, r4 = residuals(model, st, D, mu)
    Sx, Su, Ss = sigmas(model, st)
    nu = model.lay.nu
    C = Condensed()
    C.r = (r1x, r1u, r2, r3, r4)
    C.sig = (Sx, Su, Ss)
    C.delta = delta
    C.blocks = []
    C.lu = []
    C.Z = []
    Khat = np.diag(Su + delta)
    rhat2 = r1u.copy()
    for i in range(N):
        d = D[i]
        Kxx, Kxu, Kuu, rh1x, rhu = condensed_blocks(d, Sx[i], Ss[i], r1x[i], r2[i], r4[i], delta)
        rhat2 += rhu
        lu = spla.splu(d["Gx"].tocsc())
        Z = -lu.solve(d["Gu"].toarray())
        KZ = Kxx @ Z
        Khat += Z.T @ KZ + Z.T @ Kxu.toarray() + (Kxu.T @ Z) + Kuu.toarray()
        C.blocks.append((Kxx, Kxu, Kuu, rh1x))
        C.lu.append(lu)
        if keep_Z:
            C.Z.append(Z)
    C.Khat = Khat
    C.rhat2 = rhat2
    # reduced right-hand side, eq. (11):
    #   -rhat2 + sum_i [ Gu^T Gx^{-T} rhat1 + (Kux - Gu^T Gx^{-T} Kxx) Gx^{-1} r3 ]
    rhs = -rhat2.copy()
    for i in range(N):
        d = D[i]
        Kxx, Kxu, Kuu, rh1x = C.blocks[i]
        lu = C.lu[i]
        a = lu.solve(rh1x, trans="T")                # Gx^{-T} rhat1
        b = lu.solve(r3[i])                          # Gx^{-1} r3
        c = lu.solve(Kxx @ b, trans="T")             # Gx^{-T} Kxx Gx^{-1} r3
        rhs += d["Gu"].T @ a + Kxu.T @ b - d["Gu"].T @ c
    C.rhs_u = rhs
    return C


def reduce_adjoint(model, C, D, n_batch=None):
    """K_hat by the paper's local reduction (§3.2, "Local reduction"): for
    blocks V of n_batch Cartesian basis vectors of R^{n_u} (ceil(n_u /
    n_batch) blocks, the reading of the garbled "div(n_u, n_batch) + 1"),
      1. T_x = -(G_x)^{-1} (G_u V)
      2. [L_x; L_u] = [[K_xx, K_xu], [K_ux, K_uu]] [T_x; V]
      3. K_hat V = L_u - G_u^T (G_x)^{-T} L_x   (G_u^T: the transpose the
         printed step omits, fixed by dimensions and Prop. 2.3),
    summed over scenarios, plus Sigma_u + delta I and the first-stage terms
    once.  Uses the condensed blocks of ``condense`` (C) and the scenarios'
    LU factors; returns the n_u x n_u matrix as assembled (not symmetrised)."""
    nu = model.lay.nu
    Sx, Su, Ss = C.sig
    nb = nu if n_batch is None else int(n_batch)
    out = np.diag(Su + C.delta)
    for i in range(model.N):
        d = D[i]
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        lu = C.lu[i]
        Gu = d["Gu"].toarray()
        for j0 in range(0, nu, nb):
            V = np.eye(nu)[:, j0:j0 + nb]
            Tx = -lu.solve(Gu @ V)
            Lx = Kxx @ Tx + Kxu @ V
            Lu = Kxu.T @ Tx + Kuu @ V
            out[:, j0:j0 + nb] += Lu - Gu.T @ lu.solve(Lx, trans="T")
    return out


def cholesky_pd(A):
    """Cholesky factor of a symmetric matrix, or None if not positive definite."""
    try:
        return np.linalg.cholesky(0.5 * (A + A.T))
    except np.linalg.LinAlgError:
        return None


def reduced_step(model, st, D, C, Lchol):
    """Solve K_hat p_u = rhs (eq. (11)), recover p_x, p_y (Prop. 2.3) and
    p_z, p_s (Prop. 2.1).  Returns dict of step blocks."""
    r1x, r1u, r2, r3, r4 = C.r
    Sx, Su, Ss = C.sig
    pu = sla.cho_solve((Lchol, True), C.rhs_u)
    N = model.N
    px = np.empty_like(st["x"])
    py = np.empty_like(st["x"])
    pz = np.empty_like(st["s"])
    ps = np.empty_like(st["s"])
    for i in range(N):
        d = D[i]
        Kxx, Kxu, Kuu, rh1x = C.blocks[i]
        lu = C.lu[i]
        px[i] = -lu.solve(r3[i] + d["Gu"] @ pu)
        py[i] = -lu.solve(rh1x + Kxx @ px[i] + Kxu @ pu, trans="T")
        pz[i] = Ss[i] * (d["Hx"] @ px[i] + d["Hu"] @ pu + r4[i]) - r2[i]
        ps[i] = -(r2[i] + pz[i]) / Ss[i]
    return dict(px=px, pu=pu, ps=ps, py=py, pz=pz)


# ---------------------------------------------------------------------------
# Dense checkers for tiny instances (pins of Props. 2.1-2.4)
# ---------------------------------------------------------------------------

def augmented_dense(model, st, D, mu, delta=0.0):
    """The full augmented matrix of eq. (6) and its right-hand side, dense.

    Unknown order: (p_x1..p_xN, p_u, p_s1..p_sN, p_y1..p_yN, p_z1..p_zN)."""
    lay = model.lay
    N, nx, nu, m = model.N, lay.nx, lay.nu, lay.m
    nd = N * nx + nu
    ns = N * m
    r1x, r1u, r2, r3, r4 = residuals(model, st, D, mu)
    Sx, Su, Ss = sigmas(model, st)
    W = np.zeros((nd, nd))
    G = np.zeros((N * nx, nd))
    H = np.zeros((N * m, nd))
    U = slice(N * nx, nd)
    W[U, U] += np.diag(Su + delta)
    for i in range(N):
        d = D[i]
        X = slice(i * nx, (i + 1) * nx)
        W[X, X] = d["Wxx"].toarray() + np.diag(Sx[i] + delta)
        W[X, U] = d["Wxu"].toarray()
        W[U, X] = d["Wxu"].toarray().T
        W[U, U] += d["Wuu"].toarray()
        G[X, X] = d["Gx"].toarray()
        G[X, U] = d["Gu"].toarray()
        M_ = slice(i * m, (i + 1) * m)
        H[M_, X] = d["Hx"].toarray()
        H[M_, U] = d["Hu"].toarray()
    n_all = nd + ns + N * nx + N * m
    A = np.zeros((n_all, n_all))
    o1, o2, o3 = nd, nd + ns, nd + ns + N * nx
    A[:nd, :nd] = W
    A[:nd, o2:o3] = G.T
    A[:nd, o3:] = H.T
    A[nd:o2, nd:o2] = np.diag(Ss.ravel())
    A[nd:o2, o3:] = np.eye(ns)
    A[o2:o3, :nd] = G
    A[o3:, :nd] = H
    A[o3:, nd:o2] = np.eye(ns)
    rhs = -np.concatenate([r1x.ravel(), r1u, r2.ravel(), r3.ravel(), r4.ravel()])
    return A, rhs, (nd, ns)


def split_augmented(sol, model):
    lay = model.lay
    N, nx, nu, m = model.N, lay.nx, lay.nu, lay.m
    o = 0
    px = sol[o:o + N * nx].reshape(N, nx); o += N * nx
    pu = sol[o:o + nu]; o += nu
    ps = sol[o:o + N * m].reshape(N, m); o += N * m
    py = sol[o:o + N * nx].reshape(N, nx); o += N * nx
    pz = sol[o:o + N * m].reshape(N, m)
    return dict(px=px, pu=pu, ps=ps, py=py, pz=pz)


def schur_explicit(model, C, D):
    """S_uu = A_0 - sum_i B_i A_i^{-1} B_i^T for the condensed block-angular
    system (eq. (14)), with A_i^{-1} written out as in eq. (15):
      A_i^{-1} = [[0, Gx^{-1}], [Gx^{-T}, -Gx^{-T} Kxx Gx^{-1}]].
    A_0 = K_uu (all first-stage terms).  Dense; tiny instances only."""
    lay = model.lay
    Sx, Su, Ss = C.sig
    S = np.diag(Su + C.delta)
    for i in range(model.N):
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        S += Kuu.toarray()
    for i in range(model.N):
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        Gx = D[i]["Gx"].toarray()
        Gu = D[i]["Gu"].toarray()
        Gi = np.linalg.inv(Gx)
        nx = lay.nx
        Ainv = np.zeros((2 * nx, 2 * nx))
        Ainv[:nx, nx:] = Gi
        Ainv[nx:, :nx] = Gi.T
        Ainv[nx:, nx:] = -Gi.T @ Kxx.toarray() @ Gi
        B = np.hstack([Kxu.toarray().T, Gu.T])     # n_u x 2 n_x
        S -= B @ Ainv @ B.T
    return S


def condensed_matrix_dense(model, C, D):
    """The condensed KKT matrix of eq. (8), [[K, G^T], [G, 0]], dense, with
    K = W + Sigma_p + H^T Sigma_s H (+ delta I)."""
    lay = model.lay
    N, nx, nu = model.N, lay.nx, lay.nu
    nd = N * nx + nu
    Sx, Su, Ss = C.sig
    K = np.zeros((nd, nd))
    G = np.zeros((N * nx, nd))
    U = slice(N * nx, nd)
    K[U, U] = np.diag(Su + C.delta)
    for i in range(N):
        Kxx, Kxu, Kuu, _ = C.blocks[i]
        X = slice(i * nx, (i + 1) * nx)
        K[X, X] = Kxx.toarray()
        K[X, U] = Kxu.toarray()
        K[U, X] = Kxu.toarray().T
        K[U, U] += Kuu.toarray()
        G[X, X] = D[i]["Gx"].toarray()
        G[X, U] = D[i]["Gu"].toarray()
    A = np.block([[K, G.T], [G, np.zeros((N * nx, N * nx))]])
    return A, nd
