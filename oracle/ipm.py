"""Oracle interior-point iteration for the block problem (§2.2).

Test infrastructure only (see ``oracle/__init__``).

The paper delegates the outer IPM (line search, barrier update, inertia
handling) to MadNLP and cites Nocedal & Wright ch. 19 (§2.2).  This oracle
fixes one concrete primal-dual barrier method, step by step, and the CUDA
path implements the same rules so that both take the same iterates:

 0. start: theta = 0, V = 1, Pg = Pmax/2, pushed inside the boxes
    (push = min(k1 max(1,|l|), k2 (b-l)), k1 = k2 = 1e-2); s = -h pushed the
    same way; y = z = 0; bound duals 1; mu = 0.1; rho = 1.
 1. evaluate f, g, h and first/second derivatives (opf.Model);
 2. stop if E_0 <= tol; barrier update, adaptive (default): mu = max(tol/10,
    sigma * mean complementarity), sigma = 0.1, at every iteration; or
    monotone: if E_mu <= 10 mu, mu <- max(tol/10, min(0.2 mu, mu^1.5));
 3. condense (Prop. 2.1/2.2), reduce (Prop. 2.3), Cholesky of K_hat; if it
    is not positive definite add delta*I to the (x,u) diagonal of K and retry
    (first delta 1e-4, else max(1e-20, delta_last/3); x100 on the first
    failure sequence, x8 afterwards; > 1e40 -> failure);
 4. recover p_x, p_y, p_z, p_s; bound-dual steps
    dzl = mu/(w-l) - zl - Sigma_l dw,  dzu = mu/(b-w) - zu + Sigma_u dw;
 5. fraction to boundary tau = max(0.99, 1-mu) for primal and dual steps;
 6. backtracking (halving) on phi = f + barrier + rho ||(g, h+s)||_1 with the
    Armijo constant 1e-4 from the largest primal step (merit changes within
    10 eps |phi| count as no increase); rho raised to
    (grad phi^T p + max(q,0)/2) / (0.9 ||c||_1) when below it;
 7. w += a_p dw; (y,z) += a_p (p_y,p_z); bound duals += a_d dz, then kept
    within [mu/(1e10 (w-l)), 1e10 mu/(w-l)].
E_mu = max(||grad L||_inf / s_d, ||c||_inf, ||compl - mu||_inf / s_c) with the
s_max = 100 scaling of Waechter & Biegler (2006).
Pins: tests/test_oracle_ipm.py (zero power-flow residual at convergence, a
Newton power flow from the converged controls reproduces the states,
N identical scenarios give the N = 1 solution).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import kkt

OPTS = dict(tol=1e-8, max_iter=200, mu0=0.1, k1=1e-2, k2=1e-2, tau_min=0.99,
            kappa_eps=10.0, kappa_mu=0.2, theta_mu=1.5, eta=1e-4,
            alpha_min=1e-12, kappa_sigma=1e10, s_max=100.0, rho0=1.0,
            rho_frac=0.1, delta0=1e-4, delta_min=1e-20, delta_max=1e40,
            kw_minus=1.0 / 3.0, kw_plus=8.0, kw_plus_bar=100.0,
            barrier_rule="adaptive", sigma=0.1)


EPS = float(np.finfo(np.float64).eps)


class IPMError(RuntimeError):
    def __init__(self, kind, msg):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


def push(w, l, b, k1, k2):
    """Move w strictly inside [l, b] (bound push of the starting point)."""
    w = w.copy()
    fl, fb = np.isfinite(l), np.isfinite(b)
    both = fl & fb
    pl = np.where(fl, k1 * np.maximum(1.0, np.abs(np.where(fl, l, 0.0))), 0.0)
    pb = np.where(fb, k1 * np.maximum(1.0, np.abs(np.where(fb, b, 0.0))), 0.0)
    width = np.where(both, b - l, np.inf)
    pl = np.where(both, np.minimum(pl, k2 * width), pl)
    pb = np.where(both, np.minimum(pb, k2 * width), pb)
    w = np.where(fl, np.maximum(w, l + pl), w)
    w = np.where(fb, np.minimum(w, b - pb), w)
    return w


def initial_state(model, opts=OPTS):
    lay, net = model.lay, model.net
    N, nx, nu, m = model.N, lay.nx, lay.nu, lay.m
    x0 = np.concatenate([np.zeros(lay.n - 1), np.ones(nx - (lay.n - 1))])
    u0 = np.concatenate([np.ones(lay.ng), 0.5 * net.pmax[1:]])
    x0 = push(x0, model.xl, model.xu, opts["k1"], opts["k2"])
    u0 = push(u0, model.ul, model.uu, opts["k1"], opts["k2"])
    x = np.tile(x0, (N, 1))
    s = np.empty((N, m))
    for i in range(N):
        _, _, h = model.functions(i, x[i], u0)
        s[i] = push(-h, model.sl, model.su, opts["k1"], opts["k2"])
    one = lambda l: np.where(np.isfinite(l), 1.0, 0.0)
    st = dict(x=x, u=u0, s=s, y=np.zeros((N, nx)), z=np.zeros((N, m)),
              zl_x=np.tile(one(model.xl), (N, 1)), zu_x=np.tile(one(model.xu), (N, 1)),
              zl_u=one(model.ul), zu_u=one(model.uu),
              zl_s=np.tile(one(model.sl), (N, 1)), zu_s=np.tile(one(model.su), (N, 1)),
              mu=opts["mu0"], rho=opts["rho0"], delta_last=0.0)
    return st


def _compl(w, l, b, zl, zu):
    fl, fb = np.isfinite(l), np.isfinite(b)
    cl = zl * (w - np.where(fl, l, 0.0))
    cb = zu * (np.where(fb, b, 0.0) - w)
    return np.concatenate([cl[..., fl].ravel(), cb[..., fb].ravel()])


def kkt_errors(model, st, D):
    """Pieces of the optimality error: (dual_inf_inf, primal_inf_inf,
    compl_max, compl_min, s_d, s_c).  E_mu = max(dual/s_d, primal,
    max(cmax - mu, mu - cmin)/s_c)."""
    N = model.N
    dual = 0.0
    gu = -st["zl_u"] + st["zu_u"]
    prim = 0.0
    for i in range(N):
        d = D[i]
        gx = (d["grad_x"] + d["Gx"].T @ st["y"][i] + d["Hx"].T @ st["z"][i]
              - st["zl_x"][i] + st["zu_x"][i])
        gs = st["z"][i] - st["zl_s"][i] + st["zu_s"][i]
        gu = gu + d["grad_u"] + d["Gu"].T @ st["y"][i] + d["Hu"].T @ st["z"][i]
        dual = max(dual, np.abs(gx).max(initial=0.0), np.abs(gs).max(initial=0.0))
        prim = max(prim, np.abs(d["g"]).max(initial=0.0),
                   np.abs(d["h"] + st["s"][i]).max(initial=0.0))
    dual = max(dual, np.abs(gu).max(initial=0.0))
    comp = np.concatenate([
        _compl(st["x"], model.xl, model.xu, st["zl_x"], st["zu_x"]),
        _compl(st["u"], model.ul, model.uu, st["zl_u"], st["zu_u"]),
        _compl(st["s"], model.sl, model.su, st["zl_s"], st["zu_s"])])
    zb = np.concatenate([
        st["zl_x"][:, np.isfinite(model.xl)].ravel(), st["zu_x"][:, np.isfinite(model.xu)].ravel(),
        st["zl_u"][np.isfinite(model.ul)], st["zu_u"][np.isfinite(model.uu)],
        st["zl_s"][:, np.isfinite(model.sl)].ravel(), st["zu_s"][:, np.isfinite(model.su)].ravel()])
    nlam = st["y"].size + st["z"].size
    smax = OPTS["s_max"]
    s_d = max(smax, (np.abs(st["y"]).sum() + np.abs(st["z"]).sum() + np.abs(zb).sum())
              / (nlam + zb.size)) / smax
    s_c = max(smax, np.abs(zb).sum() / zb.size) / smax
    return dual, prim, comp.max(), comp.min(), s_d, s_c


def e_mu(errs, mu):
    dual, prim, cmax, cmin, s_d, s_c = errs
    return max(dual / s_d, prim, max(cmax - mu, mu - cmin) / s_c)


def _ftb(w, dw, l, b, tau):
    """Largest a in (0,1] with l + (1-tau)(w-l) <= w + a dw <= b - (1-tau)(b-w)."""
    a = 1.0
    l = np.broadcast_to(l, w.shape)
    b = np.broadcast_to(b, w.shape)
    fl, fb = np.isfinite(l), np.isfinite(b)
    neg = fl & (dw < 0)
    if np.any(neg):
        a = min(a, np.min(-tau * (w[neg] - l[neg]) / dw[neg]))
    pos = fb & (dw > 0)
    if np.any(pos):
        a = min(a, np.min(tau * (b[pos] - w[pos]) / dw[pos]))
    return a


def _ftb_dual(zv, dz, mask, tau):
    a = 1.0
    neg = mask & (dz < 0)
    if np.any(neg):
        a = min(a, np.min(-tau * zv[neg] / dz[neg]))
    return a


def merit_parts(model, x, u, s, mu):
    """(objective + barrier, ||c||_1) at a primal point."""
    f = 0.0
    c1 = 0.0
    bar = kkt.barrier_value(u, model.ul, model.uu, mu)
    for i in range(model.N):
        fi, g, h = model.functions(i, x[i], u)
        f += fi
        c1 += np.abs(g).sum() + np.abs(h + s[i]).sum()
        bar += kkt.barrier_value(x[i], model.xl, model.xu, mu)
        bar += kkt.barrier_value(s[i], model.sl, model.su, mu)
    return f + bar, c1


def bound_dual_steps(w, dw, l, b, zl, zu, mu):
    fl, fb = np.isfinite(l), np.isfinite(b)
    dzl = np.zeros_like(w)
    dzu = np.zeros_like(w)
    dl = np.where(fl, w - l, 1.0)
    db = np.where(fb, b - w, 1.0)
    dzl = np.where(fl, mu / dl - zl - zl / dl * dw, 0.0)
    dzu = np.where(fb, mu / db - zu + zu / db * dw, 0.0)
    return dzl, dzu


def _safeguard(z, w, l, mu, ks, upper=False):
    f = np.isfinite(l)
    dist = np.where(f, (l - w) if upper else (w - l), 1.0)
    lo = mu / (ks * dist)
    hi = ks * mu / dist
    return np.where(f, np.maximum(np.minimum(z, hi), lo), 0.0)


class Result:
    pass


def factor_with_inertia_correction(model, st, D, mu, opts=OPTS):
    """Step 3: condense/reduce, Cholesky, delta_w retries.  Returns (C, L)."""
    C = kkt.condense(model, st, D, mu, 0.0)
    Lc = kkt.cholesky_pd(C.Khat)
    if Lc is not None:
        return C, Lc, 0.0
    dl = st["delta_last"]
    delta = opts["delta0"] if dl == 0.0 else max(opts["delta_min"], opts["kw_minus"] * dl)
    while True:
        C = kkt.condense(model, st, D, mu, delta)
        Lc = kkt.cholesky_pd(C.Khat)
        if Lc is not None:
            st["delta_last"] = delta
            return C, Lc, delta
        delta *= opts["kw_plus_bar"] if dl == 0.0 else opts["kw_plus"]
        if delta > opts["delta_max"]:
            raise IPMError("NOT_PD", "inertia correction exceeded delta_max")


def iterate(model, st, D=None, opts=OPTS, log=None):
    """One IPM iteration from ``st`` (modified in place).

    Returns (converged, info dict).  When converged, no step is taken."""
    if D is None:
        D = kkt.eval_all(model, st)
    errs = kkt_errors(model, st, D)
    E0 = e_mu(errs, 0.0)
    info = dict(E0=E0, mu=st["mu"])
    if E0 <= opts["tol"]:
        return True, info
    mu = st["mu"]
    mu_min = opts["tol"] / 10.0
    if opts.get("barrier_rule", "adaptive") == "adaptive":
        comp = np.concatenate([
            _compl(st["x"], model.xl, model.xu, st["zl_x"], st["zu_x"]),
            _compl(st["u"], model.ul, model.uu, st["zl_u"], st["zu_u"]),
            _compl(st["s"], model.sl, model.su, st["zl_s"], st["zu_s"])])
        mu = max(mu_min, opts["sigma"] * comp.sum() / comp.size)
        st["mu"] = mu
    elif e_mu(errs, mu) <= opts["kappa_eps"] * mu and mu > mu_min:
        mu = max(mu_min, min(opts["kappa_mu"] * mu, mu ** opts["theta_mu"]))
        st["mu"] = mu
    C, Lc, delta = factor_with_inertia_correction(model, st, D, mu, opts)
    p = kkt.reduced_step(model, st, D, C, Lc)
    # bound-dual steps
    dzlx, dzux = bound_dual_steps(st["x"], p["px"], model.xl, model.xu, st["zl_x"], st["zu_x"], mu)
    dzlu, dzuu = bound_dual_steps(st["u"], p["pu"], model.ul, model.uu, st["zl_u"], st["zu_u"], mu)
    dzls, dzus = bound_dual_steps(st["s"], p["ps"], model.sl, model.su, st["zl_s"], st["zu_s"], mu)
    tau = max(opts["tau_min"], 1.0 - mu)
    amax = min(_ftb(st["x"], p["px"], model.xl[None, :], model.xu[None, :], tau),
               _ftb(st["u"], p["pu"], model.ul, model.uu, tau),
               _ftb(st["s"], p["ps"], model.sl[None, :], model.su[None, :], tau))
    fx_l = np.broadcast_to(np.isfinite(model.xl), st["x"].shape)
    fx_u = np.broadcast_to(np.isfinite(model.xu), st["x"].shape)
    fs_l = np.broadcast_to(np.isfinite(model.sl), st["s"].shape)
    fs_u = np.broadcast_to(np.isfinite(model.su), st["s"].shape)
    az = min(_ftb_dual(st["zl_x"], dzlx, fx_l, tau), _ftb_dual(st["zu_x"], dzux, fx_u, tau),
             _ftb_dual(st["zl_u"], dzlu, np.isfinite(model.ul), tau),
             _ftb_dual(st["zu_u"], dzuu, np.isfinite(model.uu), tau),
             _ftb_dual(st["zl_s"], dzls, fs_l, tau), _ftb_dual(st["zu_s"], dzus, fs_u, tau))
    # merit: directional derivative and penalty update
    r1x, r1u, r2, r3, r4 = C.r
    Sx, Su, Ss = C.sig
    gphi = (p["pu"] @ kkt.barrier_grad(st["u"], model.ul, model.uu, mu))
    q = p["pu"] @ ((Su + delta) * p["pu"])
    c1 = 0.0
    for i in range(model.N):
        d = D[i]
        gphi += d["grad_x"] @ p["px"][i] + d["grad_u"] @ p["pu"]
        gphi += kkt.barrier_grad(st["x"][i], model.xl, model.xu, mu) @ p["px"][i]
        gphi += kkt.barrier_grad(st["s"][i], model.sl, model.su, mu) @ p["ps"][i]
        q += (p["px"][i] @ (d["Wxx"] @ p["px"][i] + (Sx[i] + delta) * p["px"][i])
              + 2.0 * p["px"][i] @ (d["Wxu"] @ p["pu"]) + p["pu"] @ (d["Wuu"] @ p["pu"])
              + p["ps"][i] @ (Ss[i] * p["ps"][i]))
        c1 += np.abs(r3[i]).sum() + np.abs(r4[i]).sum()
    if c1 > 0.0:
        rho_t = (gphi + 0.5 * max(q, 0.0)) / ((1.0 - opts["rho_frac"]) * c1)
        if st["rho"] < rho_t:
            st["rho"] = rho_t
    rho = st["rho"]
    dphi = gphi - rho * c1
    phi0_fb, c10 = merit_parts(model, st["x"], st["u"], st["s"], mu)
    phi0 = phi0_fb + rho * c10
    alpha = amax
    n_trials = 0
    while True:
        n_trials += 1
        xt = st["x"] + alpha * p["px"]
        ut = st["u"] + alpha * p["pu"]
        s_t = st["s"] + alpha * p["ps"]
        pt_fb, ct = merit_parts(model, xt, ut, s_t, mu)
        # Armijo, with a roundoff allowance of 10 eps |phi| (changes below the
        # rounding level of the merit value are accepted, as in IPOPT)
        if pt_fb + rho * ct - phi0 <= opts["eta"] * alpha * dphi + 10.0 * EPS * abs(phi0):
            break
        alpha *= 0.5
        if alpha < opts["alpha_min"]:
            raise IPMError("LINESEARCH", "step size below alpha_min")
    st["x"], st["u"], st["s"] = xt, ut, s_t
    st["y"] = st["y"] + alpha * p["py"]
    st["z"] = st["z"] + alpha * p["pz"]
    ks = opts["kappa_sigma"]
    st["zl_x"] = _safeguard(st["zl_x"] + az * dzlx, st["x"], model.xl[None, :], mu, ks)
    st["zu_x"] = _safeguard(st["zu_x"] + az * dzux, st["x"], model.xu[None, :], mu, ks, upper=True)
    st["zl_u"] = _safeguard(st["zl_u"] + az * dzlu, st["u"], model.ul, mu, ks)
    st["zu_u"] = _safeguard(st["zu_u"] + az * dzuu, st["u"], model.uu, mu, ks, upper=True)
    st["zl_s"] = _safeguard(st["zl_s"] + az * dzls, st["s"], model.sl[None, :], mu, ks)
    st["zu_s"] = _safeguard(st["zu_s"] + az * dzus, st["s"], model.su[None, :], mu, ks, upper=True)
    info.update(alpha=alpha, alpha_max=amax, alpha_z=az, delta=delta, trials=n_trials,
                rho=rho, mu_used=mu)
    if log is not None:
        log.append(info)
    return False, info


def solve(model, opts=OPTS, st=None, verbose=False):
    """Run the IPM to E_0 <= tol.  Returns (state, n_iter, log)."""
    if st is None:
        st = initial_state(model, opts)
    log = []
    for k in range(opts["max_iter"] + 1):
        t0 = time.perf_counter()
        conv, info = iterate(model, st, opts=opts, log=log)
        if verbose:
            print(k, {a: (f"{b:.3e}" if isinstance(b, float) else b) for a, b in info.items()},
                  f"{time.perf_counter() - t0:.2f}s", flush=True)
        if conv:
            return st, k, log
    raise IPMError("MAXITER", "iteration limit reached")
