"""Learned warm start on the GPU: the network's kernels against the CPU
oracle, the warm-start vectors, and what the trained network gains over the
cold start (needs a GPU)."""
import numpy as np
import pytest

from oracle import ipm as oipm
from oracle import kkt, mlp as omlp, opf
from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    ipm.load()
    return ipm


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def random_net(gpu, d_in=120, d_h=128, d_out=200, max_batch=128, seed=0):
    rng = np.random.default_rng(seed)
    m = gpu.MLP(d_in, d_h, d_out, max_batch=max_batch, seed=seed)
    p = rng.normal(0, 1, m.n_params) * 0.05
    m.set_params(p.astype(np.float32))
    norm = (rng.normal(0, 0.3, d_in).astype(np.float32), rng.uniform(0.5, 2, d_in).astype(np.float32),
            rng.normal(0, 0.3, d_out).astype(np.float32), rng.uniform(0.5, 2, d_out).astype(np.float32))
    m.set_normalization(*norm)
    p32 = m.get_params().astype(np.float64)
    normd = tuple(v.astype(np.float64) for v in norm)
    return m, p32, normd, rng


def blocks(g, d_in, d_h, d_out):
    return omlp.unflatten(g, d_in, d_h, d_out)


@pytest.mark.parametrize("B", [100, 128])
def test_mlp_gradients_match_oracle(gpu, B):
    import torch
    d_in, d_h, d_out = 120, 128, 200
    m, p, norm, rng = random_net(gpu, d_in, d_h, d_out)
    X = rng.normal(0, 1, (B, d_in)).astype(np.float32)
    T = rng.normal(0, 1, (B, d_out)).astype(np.float32)
    loss, g = m.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    Lo, go = omlp.loss_and_grad(p, X.astype(np.float64), T.astype(np.float64), (d_in, d_h, d_out), norm, bf16=True)
    assert abs(loss - Lo) <= 1e-4 * Lo
    for k, (a, b) in enumerate(zip(blocks(g.astype(np.float64), d_in, d_h, d_out), blocks(go, d_in, d_h, d_out))):
        assert nrel(a, b) <= 5e-3, (k, nrel(a, b))


def test_mlp_forward_matches_oracle_and_splits_batches(gpu):
    import torch
    d_in, d_h, d_out = 120, 128, 200
    m, p, norm, rng = random_net(gpu, d_in, d_h, d_out, max_batch=128, seed=1)
    X = rng.normal(0, 1, (300, d_in)).astype(np.float32)  # three internal passes, ragged last
    y = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    yo, _ = omlp.forward(p, X.astype(np.float64), (d_in, d_h, d_out), norm, bf16=True)
    assert nrel(y, norm[2] + norm[3] * yo) <= 2e-3


def test_adam_step_matches_oracle(gpu):
    import torch
    d_in, d_h, d_out = 120, 128, 200
    m, p, norm, rng = random_net(gpu, d_in, d_h, d_out, seed=2)
    X = torch.from_numpy(rng.normal(0, 1, (64, d_in)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(0, 1, (64, d_out)).astype(np.float32)).cuda()
    losses = []
    mm = np.zeros_like(p)
    vv = np.zeros_like(p)
    pw = p.copy()
    for t in range(1, 4):
        _, g = m.gradients(X, T)
        losses.append(m.train_step(X, T, 1e-3))
        pw, mm, vv = omlp.adam_step(pw, g.astype(np.float64), mm, vv, t, 1e-3)
        np.testing.assert_allclose(m.get_params(), pw, rtol=0, atol=2e-6)
        pw = m.get_params().astype(np.float64)
    assert losses[-1] < losses[0]


def test_warm_vectors_roundtrip(gpu):
    import torch
    net, pd, qd = synth.workload("opf30_n1")
    pd3, qd3 = synth.make_scenarios(net, 3, 0.05, seed=5)
    for P, Q in ((pd, qd), (pd3, qd3)):
        sol = gpu.Solver(net, P, Q)
        k0, _ = sol.ipm_solve()
        d = sol.ipm_warm_dim()
        tgt = torch.empty((sol.N, d), dtype=torch.float32, device="cuda")
        sol.ipm_warm_target(tgt)
        s = sol.split_state(sol.ipm_get_state())
        M = opf.Model(net, P, Q)
        lb = [np.isfinite(M.xl), np.isfinite(M.xu), np.isfinite(M.ul), np.isfinite(M.uu), np.isfinite(M.sl),
              np.isfinite(M.su)]
        want = []
        for i in range(sol.N):
            row = [s["x"][i], s["u"], s["s"][i],
                   np.log(np.maximum(s["zl_x"][i][lb[0]], 1e-30)), np.log(np.maximum(s["zu_x"][i][lb[1]], 1e-30)),
                   np.log(np.maximum(s["zl_u"][lb[2]], 1e-30)), np.log(np.maximum(s["zu_u"][lb[3]], 1e-30)),
                   np.log(np.maximum(s["zl_s"][i][lb[4]], 1e-30)), np.log(np.maximum(s["zu_s"][i][lb[5]], 1e-30))]
            want.append(np.concatenate(row).astype(np.float32))
        np.testing.assert_allclose(tgt.cpu().numpy(), np.stack(want), rtol=1e-6, atol=0)
        # starting from the solution's own vectors: y and z are recovered and
        # the IPM stops within a few iterations
        sol2 = gpu.Solver(net, P, Q)
        sol2.ipm_warm_start(tgt)
        s2 = sol2.split_state(sol2.ipm_get_state())
        assert nrel(s2["y"], s["y"]) <= 1e-3
        k2, e2 = sol2.ipm_solve()
        assert e2 <= 1e-8
        assert k2 <= 6 and 2 * k2 < k0


def test_learned_warm_start_cuts_iterations(gpu):
    """Train on the method's own solutions of 512 load draws of the 60-bus
    network (sigma 0.1); on 64 held-out draws the warm start needs fewer
    iterations than the cold start, every draw converges, and the oracle
    confirms the warm-started solutions."""
    from paper_2301_04869_gb300 import warmstart as ws
    net, _, _ = synth.screened_network(60, 9, 1, 0.0, seed=0)
    pool = ws.SolvePool(net, n_ctx=32, n_threads=8)
    mlp, pool, rep = ws.build(net, 512, sigma=0.1, seed=3, d_hidden=128, epochs=80, batch=128, lr=2e-3, pool=pool)
    assert rep["loss_last"] < 0.2 * rep["loss_first"]
    pd, qd = synth.make_scenarios(net, 64, 0.1, seed=99)
    cold = pool.solve(pd, qd, want_targets=False)
    warm = ws.solve_warm(pool, mlp, pd, qd, want_states=True)
    assert (cold["status"] == 0).all() and (warm["status"] == 0).all()
    gain = cold["iters"].mean() - warm["iters"].mean()
    print(f"cold {cold['iters'].mean():.2f} warm {warm['iters'].mean():.2f} iterations, "
          f"fallbacks {int(warm['fallback'].sum())}")
    assert warm["iters"].mean() <= 0.8 * cold["iters"].mean(), gain
    # the FP64 oracle checks converged warm-started points
    for j in (0, 17, 63):
        M = opf.Model(net, pd[j:j + 1], qd[j:j + 1])
        st = pool.ctx[0].split_state(warm["states"][j])
        st = {k: np.array(v, copy=True) for k, v in st.items()}
        errs = oipm.kkt_errors(M, st, kkt.eval_all(M, st))
        assert oipm.e_mu(errs, 0.0) <= 1.01e-8
        st_o, _, _ = oipm.solve(M)
        np.testing.assert_allclose(st["u"], st_o["u"], rtol=0, atol=1e-6)
