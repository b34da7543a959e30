"""Host logic of the symbolic analysis (no GPU): the per-panel forward
schedules of the multi-RHS solve Z = -G_x^{-1} G_u and the lists of products
of the sparse pivots into the dense trailing block of the LU, checked against
brute force on the exported LU pattern.

* A panel's scheduled rows are exactly the rows of [0, t0) that its columns
  of G_u reach through L (row i is reached iff G_u has a panel column in
  row i or L(i, k) != 0 for a reached k < i); the others are its zero rows;
  levels respect the dependencies; each scheduled row's products are its
  L entries against reached columns; the trailing rows' products likewise.
  The last panel (b = G_x^{-1} g) schedules every row.
* Every trailing-block entry (i, j) with i, j >= t0 is flushed exactly once,
  after exactly the products L(i, k) U(k, j) over the sparse pivots k < t0
  where both are in the pattern."""
import numpy as np
import pytest

from paper_2301_04869_gb300 import ipm, synth


@pytest.fixture(scope="module", params=[(118, 19, 3, False), (1000, 150, 0, False), (1000, 150, 0, True)])
def sym(request):
    """The structures of a 118-bus and a 1000-bus network, and of the 1000-bus
    network in the large-trailing-block mode (widened dense block)."""
    n, ng, seed, big = request.param
    net = synth.make_network(n, ng, seed=seed)
    return {k: ipm.symbolic_export(net, k, force_big=big) for k in ipm.SYM_NAMES}


def slot_rc(S):
    """(row, col, slot) of every LU pattern entry from the CSC pattern by
    position and the slot map."""
    cp, rw = S["lu_colptr"], S["lu_row"]
    col = np.repeat(np.arange(len(cp) - 1), np.diff(cp))
    return rw, col, S["lu_slot"]


def test_panel_schedules_are_the_reach_of_each_panel(sym):
    S = sym
    nx, nu, t0, nd, nnz, npan, nlists = S["dims"][:7]
    fr_ptr, fr_col, fr_lslot = S["fr_ptr"], S["fr_col"], S["fr_lslot"]
    gu_ptr, gu_col = S["gu_ptr"], S["gu_col"]
    lev_off, lev_ptr, rows, eptr = S["zp_lev_off"], S["zp_lev_ptr"], S["zp_rows"], S["zp_eptr"]
    assert npan == (nu + 31) // 32 + 1
    for p in range(npan):
        c0, c1 = 32 * p, min(32 * p + 32, nu)
        last = p == npan - 1
        nz = np.zeros(nx, dtype=bool)
        for i in range(t0):
            z = last or bool(np.any((gu_col[gu_ptr[i]:gu_ptr[i + 1]] >= c0) & (gu_col[gu_ptr[i]:gu_ptr[i + 1]] < c1)))
            for f in range(fr_ptr[i], fr_ptr[i + 1]):
                z = z or bool(nz[fr_col[f]])
            nz[i] = z
        # scheduled rows, by level, and zero rows
        level_of = {}
        for L in range(lev_off[p], lev_off[p + 1]):
            for e in range(lev_ptr[L], lev_ptr[L + 1]):
                level_of[int(rows[e])] = (L, e)
        assert set(level_of) == set(np.flatnonzero(nz[:t0]).tolist())
        zr = S["zp_zrows"][S["zp_zptr"][p]:S["zp_zptr"][p + 1]]
        assert set(zr.tolist()) == set(np.flatnonzero(~nz[:t0]).tolist())
        for i, (L, e) in level_of.items():
            want = [(int(fr_col[f]), int(fr_lslot[f])) for f in range(fr_ptr[i], fr_ptr[i + 1]) if nz[fr_col[f]]]
            got = list(zip(S["zp_col"][eptr[e]:eptr[e + 1]].tolist(), S["zp_slot"][eptr[e]:eptr[e + 1]].tolist()))
            assert got == want
            for k, _ in want:  # dependencies at earlier levels
                assert level_of[k][0] < L
        tp = S["zp_tptr"]
        for a in range(nd):
            i = t0 + a
            want = [(int(fr_col[f]), int(fr_lslot[f])) for f in range(fr_ptr[i], fr_ptr[i + 1])
                    if fr_col[f] < t0 and nz[fr_col[f]]]
            s0, s1 = tp[p * nd + a], tp[p * nd + a + 1]
            assert list(zip(S["zp_tcol"][s0:s1].tolist(), S["zp_tslot"][s0:s1].tolist())) == want


def test_trailing_block_products(sym):
    S = sym
    nx, nu, t0, nd, nnz, npan, nlists = S["dims"][:7]
    row, col, sl = slot_rc(S)
    lens, tl, tu, te = S["tw_len"], S["tw_l"], S["tw_u"], S["tw_e"]
    assert len(lens) == nlists
    # products per flushed entry, list by list
    got = {}
    for t in range(nlists):
        pending = []
        for q in range(lens[t]):
            at = q * nlists + t
            pending.append((int(tl[at]), int(tu[at])))
            if te[at] >= 0:
                e = int(te[at])
                assert e not in got
                got[e] = pending
                pending = []
        assert not pending  # every list ends with a flush
    # brute force: entries (i, j) of the trailing block, k < t0 with L(i,k) and U(k,j) in the pattern
    slot = {(int(r), int(c)): int(s) for r, c, s in zip(row, col, sl)}
    want = {}
    for (i, j), s in slot.items():
        if i >= t0 and j >= t0:
            ks = [k for k in range(t0) if (i, k) in slot and (k, j) in slot]
            if ks:
                want[s] = sorted((slot[(i, k)], slot[(k, j)]) for k in ks)
    assert set(got) == set(want)
    for s in want:
        assert sorted(got[s]) == want[s]


def test_slot_layout(sym):
    """Every pattern entry has its own slot; the trailing block is stored
    column-major with leading dimension nd at dense_base (a multiple of 4)
    after every other entry, and it is fully dense."""
    S = sym
    nx, nu, t0, nd, nnz, npan, nlists, dense_base, big = S["dims"]
    row, col, sl = slot_rc(S)
    assert len(set(sl.tolist())) == len(sl) and sl.min() >= 0 and sl.max() < nnz
    assert dense_base % 4 == 0 and nnz % 4 == 0 and nnz >= dense_base + nd * nd
    inb = (row >= t0) & (col >= t0)
    assert np.array_equal(sl[inb], dense_base + (col[inb] - t0) * nd + (row[inb] - t0))
    assert np.all(sl[~inb] < dense_base)
    assert inb.sum() == nd * nd  # the block is full
