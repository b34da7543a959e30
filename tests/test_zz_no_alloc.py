"""The allocation-free entry point ipm_schur_sum_noalloc (for callers that
cannot call cudaMalloc) against the existing path.

A context is condensed with ipm_condense_scenarios (the existing entry
point); its Z_i and condensed blocks K_i are read back, Y_i = K_i [Z_i; I]
is formed on the GPU, and the allocation-free sum must reproduce the same
K_hat to the 1e-10 relative bar of the other parity tests, on two calls in a
row (the second call reuses the scratch the first one left behind)."""
import ctypes

import numpy as np
import pytest

from paper_2301_04869_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_schur_sum_matches_condense():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_04869_gb300 import ipm
    lib = ipm.load()
    f = lib.ipm_schur_sum_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2

    net = synth.make_network(60, 9, seed=0)
    pd, qd = synth.make_scenarios(net, 5, 0.05, seed=1)
    sol = ipm.Solver(net, pd, qd)
    for _ in range(3):
        sol.ipm_step()
    sol.ipm_eval_derivatives()
    sol.ipm_condense_scenarios()
    d = sol.dims
    N, nx, nu, ng = d.n_scen, d.n_x, d.n_u, d.n_gen
    K_ref = sol.ipm_get_quantity(ipm.Q_KHAT).reshape(nu, nu)

    Z = np.stack([sol.ipm_get_quantity(ipm.Q_Z, i).reshape(nx, nu) for i in range(N)])
    Yx = np.empty_like(Z)
    Yu = np.empty((N, nu, nu))
    dev = torch.device("cuda")
    for i in range(N):
        H = sol.ipm_get_quantity(ipm.Q_HESS, i)
        Kxx = torch.tensor(H[:nx * nx].reshape(nx, nx), device=dev)
        Kxu = torch.tensor(H[nx * nx:nx * nx + nx * nu].reshape(nx, nu), device=dev)
        Kuu = torch.tensor(H[nx * nx + nx * nu:].reshape(nu, nu), device=dev)
        Zi = torch.tensor(Z[i], device=dev)
        Yx[i] = (Kxx @ Zi + Kxu).cpu().numpy()
        Yu[i] = (Kxu.T @ Zi + Kuu).cpu().numpy()
    # first-stage diagonal: Sigma_u (the per-scenario Pg curvature is in Kuu)
    s = sol.split_state(sol.ipm_get_state())
    ul = np.concatenate([net.vmin[net.gen_bus], np.zeros(ng - 1)])
    uu = np.concatenate([net.vmax[net.gen_bus], net.pmax[1:]])
    sig_u = s["zl_u"] / (s["u"] - ul) + s["zu_u"] / (uu - s["u"])

    tZ = torch.tensor(Z, device=dev)
    tY = torch.tensor(Yx, device=dev)
    tYu = torch.tensor(Yu, device=dev)
    tD = torch.tensor(sig_u, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((nu, nu), float("nan"), dtype=torch.float64, device=dev)
        st = f(tZ.data_ptr(), tY.data_ptr(), tYu.data_ptr(), tD.data_ptr(), N, nx, nu, out.data_ptr(), stream)
        assert st == 0, ipm.STATUS.get(st)
        torch.cuda.synchronize()
        K = out.cpu().numpy()
        err = np.abs(K - K_ref).max() / np.abs(K_ref).max()
        assert err <= 1e-10, (call, err)

    # sizes beyond the scratch are rejected before anything is launched
    big = 961
    st = f(tZ.data_ptr(), tY.data_ptr(), None, None, 1, 1, big, out.data_ptr(), stream)
    assert st == 1
