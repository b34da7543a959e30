"""The emulated FP64 contraction (IPM_PREC_FP64_TC's K_hat = sum_s Z_s^T Y_s
on the BF16 tensor cores) on arbitrary data, through ipm_schur_sum_tc (needs
a GPU):

* bit for bit against the step-by-step oracle of the splitting algorithm
  (oracle/emu.py), which uses exact integer arithmetic, with the kernel's
  partition of the row groups over CTAs;

and against the plain FP64 definition computed by numpy:

* integer-valued operands: every slice product and sum is exact, so the
  result equals the exact integer product bit for bit;
* operands spanning 16 orders of magnitude with random signs: each entry
  within 2^-48 of sum over 512-row groups of (rows x largest |Z'_ki| x
  largest |Y'_kj| in the group), Z' and Y' the row-balanced operands -- the
  splitting keeps 56 bits relative to every group's largest entry;
* operands whose magnitudes vary by column (16 decades) but not within a
  column, like the reduction matrices: the same bound, and normwise within
  1e-13;
* ragged sizes: n_u not a multiple of the 128 x 64 tiles, N n_x not a
  multiple of the 512-row groups;
* the 1000-bus / 64-scenario solve with FP64_TC takes the same iterations as
  the FP64 path.
"""
import numpy as np
import pytest

from oracle import emu
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


def contract(gpu, Z, Y):
    import ctypes
    import torch
    N, nx, nu = Z.shape
    tZ = torch.tensor(Z, device="cuda")
    tY = torch.tensor(Y, device="cuda")
    K = torch.empty((nu, nu), dtype=torch.float64, device="cuda")
    lib = gpu.load()
    st = lib.ipm_schur_sum_tc(ctypes.c_void_p(tZ.data_ptr()), ctypes.c_void_p(tY.data_ptr()), N, nx, nu,
                              ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return K.cpu().numpy()


def sym_upper(K):
    nu = K.shape[0]
    iu = np.triu_indices(nu)
    Ks = np.zeros_like(K)
    Ks[iu] = K[iu]
    Ks.T[iu] = K[iu]  # the kernel computes the upper triangle and mirrors it
    return Ks


def ilogb(x):
    return np.frexp(x)[1] - 1


def reference(Z, Y):
    """Plain Z^T Y, and the error bound of the splitting: rows balanced by
    2^a_k (a_k = trunc((ilogb max|Y_k.| - ilogb max|Z_k.|) / 2)), then per
    512-row group rows x (largest |Z'| of column i) x (largest |Y'| of column j)."""
    N, nx, nu = Z.shape
    A = Z.reshape(N * nx, nu)
    B = Y.reshape(N * nx, nu)
    mz, my = np.abs(A).max(1), np.abs(B).max(1)
    a = np.where((mz > 0) & (my > 0), np.trunc((ilogb(my) - ilogb(mz)) / 2.0), 0.0)
    Ab, Bb = A * 2.0 ** a[:, None], B * 2.0 ** -a[:, None]
    bnd = np.zeros((nu, nu))
    for g0 in range(0, A.shape[0], 512):
        za = np.abs(Ab[g0:g0 + 512]).max(0)
        yb = np.abs(Bb[g0:g0 + 512]).max(0)
        bnd += min(512, A.shape[0] - g0) * np.outer(za, yb)
    return sym_upper(A.T @ B), sym_upper(bnd)


def kernel_parts(rows, nu):
    """row groups per CTA partition as the kernel plans them (one wave of
    152 CTAs over the 128 x 64 upper tiles)"""
    ntm, ntn = -(-nu // 128), -(-nu // 64)
    ntiles = sum(1 for a in range(ntm) for b in range(ntn) if a * 128 <= b * 64 + 63)
    ngr = -(-rows // 512)
    G = min(max(1, 152 // ntiles), ngr)
    return -(-ngr // G)


@pytest.mark.parametrize("shape,kind", [((1, 53, 11), "normal"), ((3, 333, 40), "wide"), ((2, 700, 70), "normal"),
                                        ((1, 1200, 20), "barrier")])
def test_bit_exact_against_the_oracle(gpu, shape, kind):
    rng = np.random.default_rng(7)
    N, nx, nu = shape
    Z = rng.normal(size=shape)
    Y = rng.normal(size=shape)
    if kind == "wide":
        Z *= 10.0 ** rng.uniform(-8, 8, shape)
        Y *= 10.0 ** rng.uniform(-8, 8, shape)
    if kind == "barrier":  # a few rows of Y scaled by large barrier terms, as near a solution
        Y *= np.where(rng.uniform(size=(N, nx, 1)) < 0.05, 10.0 ** rng.uniform(4, 11, (N, nx, 1)), 1.0)
    K = contract(gpu, Z, Y)
    want = emu.contract(Z.reshape(-1, nu), Y.reshape(-1, nu), parts=kernel_parts(N * nx, nu))
    np.testing.assert_array_equal(K, want)


@pytest.mark.parametrize("shape", [(3, 333, 150), (2, 700, 299), (1, 64, 7)])
def test_integer_operands_exact(gpu, shape):
    rng = np.random.default_rng(1)
    Z = rng.integers(-100, 101, shape).astype(np.float64)
    Y = rng.integers(-1000, 1001, shape).astype(np.float64)
    K = contract(gpu, Z, Y)
    want, _ = reference(Z, Y)
    np.testing.assert_array_equal(K, want)


@pytest.mark.parametrize("shape", [(3, 333, 150), (8, 1849, 299)])
def test_wide_dynamic_range(gpu, shape):
    rng = np.random.default_rng(2)
    mag = lambda: 10.0 ** rng.uniform(-8, 8, shape)
    Z = mag() * rng.choice([-1.0, 1.0], shape)
    Y = mag() * rng.choice([-1.0, 1.0], shape)
    K = contract(gpu, Z, Y)
    want, bnd = reference(Z, Y)
    assert np.all(np.abs(K - want) <= 2.0 ** -48 * bnd)


@pytest.mark.parametrize("shape", [(3, 333, 150), (8, 1849, 299)])
def test_column_scaled_operands(gpu, shape):
    rng = np.random.default_rng(3)
    N, nx, nu = shape
    cz = 10.0 ** rng.uniform(-8, 8, nu)
    cy = 10.0 ** rng.uniform(-8, 8, nu)
    Z = rng.normal(size=shape) * cz
    Y = rng.normal(size=shape) * cy
    K = contract(gpu, Z, Y)
    want, bnd = reference(Z, Y)
    assert np.all(np.abs(K - want) <= 2.0 ** -48 * bnd)
    assert np.linalg.norm(K - want) <= 1e-13 * np.linalg.norm(want)


def test_fp64_tc_same_iterations_as_fp64_at_64_scenarios(gpu):
    net, pd, qd = synth.workload("opf1000_n64")
    a = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64)
    b = gpu.Solver(net, pd, qd, precision=gpu.PREC_FP64_TC)
    ka, ea = a.ipm_solve()
    kb, eb = b.ipm_solve()
    assert kb == ka and eb <= 1e-8
    sa = a.split_state(a.ipm_get_state())
    sb = b.split_state(b.ipm_get_state())
    np.testing.assert_allclose(sb["u"], sa["u"], rtol=0, atol=1e-6)
