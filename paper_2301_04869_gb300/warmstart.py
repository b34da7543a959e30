"""Learned warm start of the reduced-space IPM (not in the paper).

A small MLP (libipm.so's ipm_mlp_*, BF16 tensor-core kernels) maps a load
vector [P_d; Q_d] to the warm-start vector of a single-scenario instance: the
primal point (x, u, s) and the log bound duals (ipm_warm_dim / ipm_warm_target
in include/ipm.h).  It is trained on solutions the IPM itself produces, and at
solve time it only picks the starting point: ipm_warm_start recovers the
equality multipliers y and the slack multipliers z from stationarity, and an
instance that fails from the warm point is solved again from the cold start.

Pipeline: ``SolvePool`` (reused single-scenario contexts of one network,
solved together by the multi-instance runner), ``generate`` (load draws ->
solutions -> training pairs), ``fit`` (Adam on minibatches), ``solve_warm``.
Run as a module for the 1000-bus experiment:
``python -m paper_2301_04869_gb300.warmstart --n-train 20000 --n-test 1024``.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ipm, synth


def features(pd, qd):
    """Network input: the load vector [P_d; Q_d] of each draw."""
    return np.concatenate([np.atleast_2d(pd), np.atleast_2d(qd)], axis=1).astype(np.float32)


class SolvePool:
    """n_ctx single-scenario contexts of one network, reused across load draws."""

    def __init__(self, net, n_ctx=32, n_threads=8, **solver_kw):
        pd, qd = synth.make_scenarios(net, 1, 0.0, seed=0)
        self.net = net
        self.ctx = [ipm.Solver(net, pd, qd, **solver_kw) for _ in range(n_ctx)]
        self.n_threads = n_threads
        self.d = self.ctx[0].ipm_warm_dim()

    def solve(self, pd, qd, warm=None, want_targets=True, want_states=False):
        """Solve every draw (rows of pd, qd).  warm: None (cold start) or a
        device FP32 tensor [S][d] of predicted warm-start vectors; a draw that
        fails from its warm point is solved again from the cold start.
        Returns dict(iters, status, fallback, targets [S][d] device tensor,
        states (host state vectors, when asked), wall_s)."""
        import torch
        S = pd.shape[0]
        iters = np.zeros(S, dtype=np.int64)
        status = np.zeros(S, dtype=np.int64)
        fallback = np.zeros(S, dtype=bool)
        targets = torch.empty((S, self.d), dtype=torch.float32, device="cuda") if want_targets else None
        states = [None] * S if want_states else None
        t0 = time.perf_counter()
        n = len(self.ctx)
        for c0 in range(0, S, n):
            k = min(n, S - c0)
            for j in range(k):
                self.ctx[j].ipm_set_loads(pd[c0 + j:c0 + j + 1], qd[c0 + j:c0 + j + 1])
                if warm is not None:
                    try:
                        self.ctx[j].ipm_warm_start(warm[c0 + j:c0 + j + 1])
                    except ipm.IPMError:
                        self.ctx[j].ipm_set_loads(pd[c0 + j:c0 + j + 1], qd[c0 + j:c0 + j + 1])
                        fallback[c0 + j] = True
            it, er, st, _ = ipm.ipm_solve_batch(self.ctx[:k], n_threads=self.n_threads)
            for j in range(k):
                if st[j] != ipm.IPM_OK and warm is not None and not fallback[c0 + j]:
                    # cold start is the fallback of the learned start
                    fallback[c0 + j] = True
                    extra = it[j]
                    self.ctx[j].ipm_set_loads(pd[c0 + j:c0 + j + 1], qd[c0 + j:c0 + j + 1])
                    try:
                        kk, _ = self.ctx[j].ipm_solve()
                        it[j], st[j] = extra + kk, ipm.IPM_OK
                    except ipm.IPMError as e:
                        it[j], st[j] = extra, e.status
                iters[c0 + j] = it[j]
                status[c0 + j] = st[j]
                if want_targets and st[j] == ipm.IPM_OK:
                    self.ctx[j].ipm_warm_target(targets[c0 + j:c0 + j + 1])
                if want_states:
                    states[c0 + j] = self.ctx[j].ipm_get_state()
        torch.cuda.synchronize()
        return dict(iters=iters, status=status, fallback=fallback, targets=targets, states=states,
                    wall_s=time.perf_counter() - t0)


def generate(pool, n, sigma, seed):
    """n load draws of the pool's network (scenario law of synth with noise
    sigma), solved from the cold start; returns (X, T, info) with X host FP32
    [S][2 n_bus] and T a device FP32 tensor [S][d], converged draws only."""
    pd, qd = synth.make_scenarios(pool.net, n, sigma, seed=seed)
    r = pool.solve(pd, qd)
    import torch
    ok = r["status"] == ipm.IPM_OK
    X = features(pd, qd)[ok]
    T = r["targets"].index_select(0, torch.from_numpy(np.flatnonzero(ok)).cuda())
    return X, T, dict(iters=r["iters"][ok], n_failed=int((~ok).sum()), wall_s=r["wall_s"], pd=pd[ok], qd=qd[ok])


def normalization(X, T):
    """Per-feature mean and standard deviation (floored) of inputs and targets."""
    Tn = T.double().cpu().numpy() if hasattr(T, "cpu") else np.asarray(T, dtype=np.float64)
    xm, xs = X.mean(0), X.std(0)
    tm, ts = Tn.mean(0), Tn.std(0)
    xs = np.maximum(xs, 1e-3 * max(1e-12, float(np.abs(xm).max(initial=0.0))) + 1e-6)
    ts = np.maximum(ts, 1e-6 + 1e-4 * np.abs(tm))
    return xm.astype(np.float32), xs.astype(np.float32), tm.astype(np.float32), ts.astype(np.float32)


def fit(mlp, X, T, epochs=30, batch=256, lr=1e-3, lr_final=1e-5, seed=0):
    """Adam on shuffled minibatches with a geometric learning-rate decay.
    X: host FP32 [S][d_in]; T: device FP32 [S][d_out].  Returns per-epoch mean loss."""
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    S = Xd.shape[0]
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, (S + batch - 1) // batch)
    gamma = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    hist = []
    k = 0
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(S)).cuda()
        tot = 0.0
        nb = 0
        for b0 in range(0, S, batch):
            idx = perm[b0:b0 + batch]
            xb = Xd.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            tot += mlp.train_step(xb, tb, lr * gamma ** k)
            nb += 1
            k += 1
        hist.append(tot / nb)
    return hist


def build(net, n_train, sigma=0.1, seed=11, d_hidden=512, epochs=30, batch=256, lr=1e-3, pool=None):
    """Generate training solutions, fit a network; returns (mlp, pool, report)."""
    pool = pool or SolvePool(net)
    X, T, gi = generate(pool, n_train, sigma, seed)
    mlp = ipm.MLP(X.shape[1], d_hidden, pool.d, max_batch=batch, seed=seed)
    mlp.set_normalization(*normalization(X, T))
    t0 = time.perf_counter()
    hist = fit(mlp, X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    rep = dict(n_train=int(X.shape[0]), n_failed=gi["n_failed"], gen_s=gi["wall_s"],
               train_s=time.perf_counter() - t0, loss_first=hist[0], loss_last=hist[-1],
               cold_iters_train=float(gi["iters"].mean()))
    return mlp, pool, rep


def solve_warm(pool, mlp, pd, qd, want_states=False):
    """Warm-started solves of the draws (prediction on the GPU, cold fallback)."""
    import torch
    x = torch.from_numpy(features(pd, qd)).cuda()
    pred = mlp.forward(x)
    return pool.solve(pd, qd, warm=pred, want_targets=False, want_states=want_states)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="opf1000_n64")
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--n-test", type=int, default=1024)
    ap.add_argument("--sigma", type=float, default=0.1)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--ctx", type=int, default=32)
    ap.add_argument("--threads", type=int, default=8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    net, _, _ = synth.workload(a.workload, n_scen=1)
    pool = SolvePool(net, n_ctx=a.ctx, n_threads=a.threads)
    mlp, pool, rep = build(net, a.n_train, a.sigma, d_hidden=a.hidden, epochs=a.epochs, pool=pool)
    pd, qd = synth.make_scenarios(net, a.n_test, a.sigma, seed=977)
    cold = pool.solve(pd, qd, want_targets=False)
    warm = solve_warm(pool, mlp, pd, qd)
    ok = (cold["status"] == 0) & (warm["status"] == 0)
    rep.update(workload=a.workload, n_bus=net.n_bus, d_out=pool.d, n_test=a.n_test,
               cold_iters=float(cold["iters"][ok].mean()), warm_iters=float(warm["iters"][ok].mean()),
               cold_wall_s=cold["wall_s"], warm_wall_s=warm["wall_s"],
               warm_fallbacks=int(warm["fallback"].sum()), test_failed_cold=int((cold["status"] != 0).sum()),
               test_failed_warm=int((warm["status"] != 0).sum()))
    s = json.dumps(rep)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
