"""Oracle of the emulated FP64 contraction K = A^T B (the tensor-core mode of
the reduced-Hessian product; not in the paper, which uses FP64 hardware).

Test infrastructure only (see ``oracle/__init__``).

The algorithm, step by step, in exact integer arithmetic (numpy int64 and
Python integers), so that the CUDA kernel can be compared with it bit for
bit:

Entries below 2^-1022 (subnormal) count as zero throughout.

1. Row balancing: for each contraction row k, a_k = trunc((ilogb max_j
   |B_kj| - ilogb max_j |A_kj|) / 2) (0 if either row is zero);
   A_k <- A_k 2^a_k, B_k <- B_k 2^-a_k (exact: powers of two; a balanced
   entry below 2^-1022 counts as zero).
2. Per group of 512 rows and per column j: e_j = ilogb(max |x_kj|) + 2 (0 for
   an all-zero column), so |x 2^-e| < 1/2; X = round-half-away(|x| 2^(56-e))
   with the sign of x (|X| <= 2^55); then S = 8 digits, the unique
   representation X = sum_t q_t 2^(49-7t) (t = 0..7) with q_t in [-64, 63]
   for t >= 1: with O = 64 sum_{t>=1} 2^(49-7t), q_0 = floor((X + O) / 2^49)
   (|q_0| <= 64) and q_t = (bits 49-7t .. 55-7t of X + O) - 64.
3. Levels: acc_L = sum_{t+u=L} Q_t^T Q'_u (0-based t, u; L = 0..S-1),
   integer matrices (at most 8 * 2^12 * 512 = 2^24 in magnitude).
4. Group value in units of 2^(e_i + e'_j - 49): the exact integers
   V = sum_{L<=5} acc_L 2^(7 (5 - L)) and W = acc_6 2^7 + acc_7 (S = 8),
   t = fl(fl(W) 2^-14 + fl(V)) (fl: round to nearest FP64; one fused
   multiply-add).
5. K_ij = sum over groups, in group order, of t * 2^(e_i + e'_j - 49),
   each an FP64 fused multiply-add into the running sum; summed over the
   CTA partitions of the groups in partition order (``parts``) and mirrored
   from the upper triangle.

Pins (tests/test_oracle_emu.py): integer operands give the exact product;
random operands stay within 2^-50 of sum over groups of rows x (largest |A|
of column i) x (largest |B| of column j) after balancing; the level sums
stay within 2^24; the row balancing leaves the product unchanged.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

GROUP = 512
NS = 8


def fma(a, b, c):
    """a * b + c with one rounding (exact rational arithmetic, then the
    correctly rounded conversion to FP64)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def parts_of(x):
    """FP64 -> (biased exponent E, integer mantissa m with the implicit bit,
    sign); zero and subnormals give m = 0."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float64)).view(np.uint64)
    E = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    m = ((b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)).astype(np.int64)
    m = np.where(E == 0, 0, m)
    neg = (b >> np.uint64(63)) != 0
    return E, m, neg


def balance(A, B):
    """Step 1: the row exponents a_k."""
    EA, mA, _ = parts_of(A)
    EB, mB, _ = parts_of(B)
    ez = np.where(mA > 0, EA, 0).max(axis=1)
    ey = np.where(mB > 0, EB, 0).max(axis=1)
    d = ey - ez
    return np.where((ez > 0) & (ey > 0), np.sign(d) * (np.abs(d) // 2), 0).astype(np.int64)


def split(X, shift=None):
    """Step 2 for one row group of X (rows scaled by 2^shift first):
    (digits [S][rows][cols] int64, exponents [cols])."""
    E, m, neg = parts_of(X)
    if shift is not None:
        E = E + shift[:, None]
    live = (m > 0) & (E > 0)
    key = np.where(live, (np.minimum(E, 2047).astype(np.uint64) << np.uint64(53)) | m.astype(np.uint64),
                   np.uint64(0))
    kmax = key.max(axis=0)
    e = np.where(kmax > 0, (kmax >> np.uint64(53)).astype(np.int64) - 1023 + 2, 0)
    sh = E - 1019 - e[None, :]
    Xi = np.zeros(X.shape, dtype=np.int64)
    up = live & (sh >= 0)
    Xi[up] = m[up] << sh[up]
    dn = live & (sh < 0) & (sh > -63)
    s_ = -sh[dn]
    Xi[dn] = (m[dn] + (np.int64(1) << (s_ - 1))) >> s_
    Xi = np.where(neg, -Xi, Xi)
    offset = sum(64 << (49 - 7 * t) for t in range(1, NS))
    Y = Xi + np.int64(offset)
    qs = [Y >> 49]
    for t in range(1, NS):
        qs.append(((Y >> (49 - 7 * t)) & 127) - 64)
    return np.stack(qs), e


def levels(QA, QB):
    """Step 3: integer level sums acc_L [S][n][n]."""
    S = QA.shape[0]
    out = []
    for L in range(S):
        acc = np.zeros((QA.shape[2], QB.shape[2]), dtype=np.int64)
        for t in range(L + 1):
            acc += QA[t].T @ QB[L - t]
        out.append(acc)
    return np.stack(out)


def group_value(acc):
    """Step 4: t of each (i, j) as FP64."""
    V = np.zeros(acc.shape[1:], dtype=object)
    for L in range(6):
        V = V * 128 + acc[L].astype(object)
    W = acc[6].astype(object) * 128 + acc[7].astype(object)
    f = np.vectorize(lambda v, w: fma(float(w), 2.0 ** -14, float(v)), otypes=[np.float64])
    return f(V, W)


def contract(A, B, parts=None):
    """K = A^T B by steps 1-5.  A, B: FP64 [rows][n].  parts: the number of
    consecutive row groups each CTA partition takes (None: one partition)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    rows, n = A.shape
    a = balance(A, B)
    ng = (rows + GROUP - 1) // GROUP
    gpp = ng if parts is None else parts
    K = np.zeros((n, n))
    for p0 in range(0, ng, gpp):
        acc_p = np.zeros((n, n))
        for g in range(p0, min(ng, p0 + gpp)):
            sl = slice(g * GROUP, min(rows, (g + 1) * GROUP))
            QA, ea = split(A[sl], a[sl])
            QB, eb = split(B[sl], -a[sl])
            Vd = group_value(levels(QA, QB))
            sc = np.ldexp(1.0, (ea[:, None] + eb[None, :] - 49).astype(np.int64))
            for i in range(n):
                for j in range(n):
                    acc_p[i, j] = fma(Vd[i, j], sc[i, j], acc_p[i, j])
        K += acc_p
    iu = np.triu_indices(n)
    Ks = np.zeros_like(K)
    Ks[iu] = K[iu]
    Ks.T[iu] = K[iu]
    return Ks


def level_bound(A, B):
    """max |acc_L| over all groups and levels (must stay within 2^24)."""
    a = balance(A, B)
    m = 0
    for g0 in range(0, A.shape[0], GROUP):
        QA, _ = split(A[g0:g0 + GROUP], a[g0:g0 + GROUP])
        QB, _ = split(B[g0:g0 + GROUP], -a[g0:g0 + GROUP])
        m = max(m, int(np.abs(levels(QA, QB)).max()))
    return m


def error_bound(A, B):
    """sum over groups of rows x (largest |A'| of column i) x (largest |B'| of
    column j), A', B' the balanced operands."""
    a = balance(A, B)
    Ab = np.abs(np.ldexp(A, a[:, None]))
    Bb = np.abs(np.ldexp(B, -a[:, None]))
    n = A.shape[1]
    bnd = np.zeros((n, n))
    for g0 in range(0, A.shape[0], GROUP):
        r = min(GROUP, A.shape[0] - g0)
        bnd += r * np.outer(Ab[g0:g0 + GROUP].max(0), Bb[g0:g0 + GROUP].max(0))
    return bnd
