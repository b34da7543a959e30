"""Pins of the oracle KKT algebra (Props. 2.1-2.4) on tiny instances (CPU).

Each identity is checked against an independent dense computation:
the reduced step (Props. 2.1 + 2.3) against a dense LU solve of the full
augmented system eq. (6); K_hat against the Schur complement with the
explicit A_i^{-1} of eq. (15); Z against a dense solve; and the inertia of the
condensed matrix eq. (8) by its eigenvalues."""
import numpy as np
import pytest

from oracle import ipm, kkt, opf
from paper_2301_04869_gb300 import synth


def _model(N=3, n=30, ng=6, sigma=0.05):
    net = synth.make_network(n, ng, seed=0)
    pd, qd = synth.make_scenarios(net, N, sigma, seed=1)
    return opf.Model(net, pd, qd)


@pytest.fixture(scope="module", params=["plain", "rated"])
def mid_iterate(request):
    """A non-trivial interior iterate: 4 IPM iterations from the start; the
    rated variant has the 2L line-flow rows of §4.1.1 in h, three of them
    binding at the optimum."""
    if request.param == "rated":
        from ratings import rated
        net, pd, qd = rated(30, 6, 3, 0.05)
        M = opf.Model(net, pd, qd)
    else:
        M = _model()
    st = ipm.initial_state(M)
    for _ in range(4):
        ipm.iterate(M, st)
    return M, st


def test_reduced_step_equals_augmented_solve(mid_iterate):
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    mu = st["mu"]
    C = kkt.condense(M, st, D, mu, 0.0)
    L = kkt.cholesky_pd(C.Khat)
    assert L is not None
    p = kkt.reduced_step(M, st, D, C, L)
    A, rhs, _ = kkt.augmented_dense(M, st, D, mu, 0.0)
    sol = np.linalg.solve(A, rhs)
    q = kkt.split_augmented(sol, M)
    for k in ("px", "pu", "ps", "py", "pz"):
        err = np.abs(p[k] - q[k]).max() / max(1e-300, np.abs(q[k]).max())
        assert err <= 1e-10, (k, err)


def test_reduced_step_with_delta(mid_iterate):
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.37)
    L = kkt.cholesky_pd(C.Khat)
    p = kkt.reduced_step(M, st, D, C, L)
    A, rhs, _ = kkt.augmented_dense(M, st, D, st["mu"], 0.37)
    q = kkt.split_augmented(np.linalg.solve(A, rhs), M)
    assert np.abs(p["pu"] - q["pu"]).max() <= 1e-10 * np.abs(q["pu"]).max()


def test_schur_explicit_equals_reduced(mid_iterate):
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    S = kkt.schur_explicit(M, C, D)
    assert np.abs(S - C.Khat).max() <= 1e-10 * np.abs(C.Khat).max()


def test_Z_dense_and_symmetry(mid_iterate):
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    for i in range(M.N):
        Zd = -np.linalg.solve(D[i]["Gx"].toarray(), D[i]["Gu"].toarray())
        assert np.abs(C.Z[i] - Zd).max() <= 1e-11 * max(1.0, np.abs(Zd).max())
    K = C.Khat
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()


def test_inertia_condensed_matrix(mid_iterate):
    """K_hat positive definite  <=>  the condensed KKT matrix has inertia
    (N n_x + n_u, N n_x, 0)."""
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    A, nd = kkt.condensed_matrix_dense(M, C, D)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    npos, nneg = int(np.sum(ev > 0)), int(np.sum(ev < 0))
    pd_ = bool(np.all(np.linalg.eigvalsh(C.Khat) > 0))
    ncon = A.shape[0] - nd
    assert (npos == nd and nneg == ncon) == pd_
    assert pd_


def test_inertia_correction_on_nonconvex_point():
    """Negative curvature (random multipliers) makes K_hat indefinite; the
    delta_w rule restores positive definiteness and the right inertia."""
    M = _model(N=2)
    st = ipm.initial_state(M)
    rng = np.random.default_rng(3)
    st["y"] = 50.0 * rng.standard_normal(st["y"].shape)
    D = kkt.eval_all(M, st)
    C0 = kkt.condense(M, st, D, st["mu"], 0.0)
    assert kkt.cholesky_pd(C0.Khat) is None
    C, L, delta = ipm.factor_with_inertia_correction(M, st, D, st["mu"])
    assert delta > 0 and L is not None
    A, nd = kkt.condensed_matrix_dense(M, C, D)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert int(np.sum(ev > 0)) == nd and int(np.sum(ev < 0)) == A.shape[0] - nd


def test_condensed_K_block_structure(mid_iterate):
    """Prop. 2.2: the blocks of K = W + H^T Sigma_s H assembled scenario by
    scenario equal the dense product over the whole block-angular matrices."""
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    A_, rhs, (nd, ns) = kkt.augmented_dense(M, st, D, st["mu"], 0.0)
    W = A_[:nd, :nd]
    H = A_[nd + ns + M.N * M.lay.nx:, :nd]
    Ss = np.diag(A_[nd:nd + ns, nd:nd + ns])
    Kd = W + H.T @ np.diag(Ss) @ H
    Kb, _ = kkt.condensed_matrix_dense(M, C, D)
    assert np.abs(Kb[:nd, :nd] - Kd).max() <= 1e-12 * np.abs(Kd).max()


@pytest.mark.parametrize("n_batch", [None, 4])
def test_adjoint_reduction_equals_schur(mid_iterate, n_batch):
    """The paper's three-step local reduction (§3.2) in blocks of n_batch
    unit vectors gives the Schur complement with the explicit A_i^{-1} of
    eq. (15), and its result is symmetric to rounding."""
    M, st = mid_iterate
    D = kkt.eval_all(M, st)
    C = kkt.condense(M, st, D, st["mu"], 0.0)
    R = kkt.reduce_adjoint(M, C, D, n_batch)
    S = kkt.schur_explicit(M, C, D)
    assert np.abs(R - S).max() <= 1e-10 * np.abs(S).max()
    assert np.abs(R - R.T).max() <= 1e-11 * np.abs(R).max()
