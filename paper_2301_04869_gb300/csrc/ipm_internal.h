// Internal structures of the reduced-space IPM library (host side).
#pragma once
#include <string>
#include <vector>

#include "../../include/ipm.h"

#ifndef IPM_LU_LISTS_DEFINED
#define IPM_LU_LISTS_DEFINED
constexpr int LU_LISTS = 1024;  // lists of trailing-block products of the LU factorization
#endif

struct HostNet {
  int n = 0, L = 0, ng = 0;
  std::vector<int> fr, to, gen;
  std::vector<double> r, x, b, pmax, qmax, c2, c1, vmin, vmax;
  std::vector<double> rate;  // [L] line ratings, or empty (no line-flow limits)
};

// Symbolic structures built once per network (S1).  Index conventions:
//  * bus variables: theta_i (kind 0) and v_i (kind 1);
//  * x index: (theta_1..theta_{n-1}, v at non-generator buses); a g row has
//    the same index as the x variable it pivots on (P_i <-> theta_i,
//    Q_i <-> v_i);
//  * u index: v at generator k (k = 0..ng-1), then Pg_k (k = 1..ng-1) at
//    ng + k - 1;
//  * position: place of an x variable in the static LU elimination order;
//  * A: bus adjacency (with diagonal); a Jacobian value is stored per A slot
//    as 4 entries e = comp*2 + kind (comp 0 = P, 1 = Q), scenario fastest;
//  * KB: bus-level pattern of the condensed matrix K (A plus the couplings
//    through every h row), 4 entries per block (row kind*2 + col kind).
struct Sym {
  int n = 0, L = 0, ng = 0, N = 0, nx = 0, nu = 0, m = 0;
  std::vector<int> xth, xv, uv, gen_of_bus;  // per bus, -1 if none
  std::vector<int> xbus, xkind;              // per x index
  std::vector<int> lfr, lto;
  std::vector<double> lg, lb, lbh;           // series g, series b, half charging
  int nnzA = 0;
  std::vector<int> a_ptr, a_col, a_diag;
  std::vector<int> a_tslot;                  // per A slot (i, k): the slot of (k, i)
  std::vector<int> inc_ptr, inc_line, inc_other, inc_aslot;
  int nnzKB = 0;
  std::vector<int> kb_ptr, kb_col, kb_row, kb_aslot;
  std::vector<int> kbi_ptr, kbi_r, kbi_ja, kbi_jb;
  // per h row: the bus and component of an injection row (comp 0 = P,
  // 1 = Q), or for a line-flow row the bus of its end and comp 2 (from end)
  // or 3 (to end); line-flow rows are n_g + 1 + e L + l (e = 0 from, 1 to)
  int nflow = 0;                             // 2 L with ratings, else 0
  std::vector<int> hrow_bus, hrow_comp;      // per h row
  std::vector<int> ht_ptr, ht_r, ht_aslot;   // per bus: h rows touching it
  // static-pivot LU of G_x (positions)
  std::vector<int> perm, iperm;
  int nnzLU = 0;
  std::vector<int> lu_colptr, lu_row, lu_diag, lu_init;
  int nlev = 0, nlev_b = 0;
  int nlev_f = 0;          // levels of the sparse (non-tail) pivots
  int t0 = 0, nd = 0;      // dense trailing block: positions [t0, nx), nd = nx - t0
  std::vector<int> tail_slot;  // nd*nd LU slots of the trailing block, row-major
  // LU storage: the entries outside the trailing block in CSC order by
  // position (slots 0 ..), then the trailing block column-major with leading
  // dimension nd at dense_base (a multiple of 4): (t0 + a, t0 + b) at
  // dense_base + b nd + a.  lu_colptr / lu_row describe the whole pattern,
  // lu_slot the storage slot of each of its entries.
  int dense_base = 0;
  bool big = false;        // trailing block factored and solved by the global-memory kernels
  std::vector<int> lu_slot;
  int nlev_fs = 0, nlev_bs = 0;  // forward / backward levels of the sparse rows only
  std::vector<int> fs_lev_ptr, fs_rows, bs_lev_ptr, bs_rows;
  std::vector<int> f_lev_ptr, f_piv_ptr, f_piv, f_tgt, f_op_ptr, f_op_l, f_op_u, f_op_k;
  std::vector<int> lsc_slot, lsc_k;
  // products of the sparse pivots into the dense trailing block, in
  // LU_LISTS lists (symbolic.cpp)
  std::vector<int> tw_len, tw_l, tw_u, tw_e;
  long long n_tail_ops = 0;
  std::vector<int> fw_lev_ptr, fw_rows, fr_ptr, fr_col, fr_lslot, fr_uslot;
  std::vector<int> bw_lev_ptr, bw_rows, br_ptr, br_col, br_uslot, br_lslot;
  // packed single-RHS sweeps (4 ints each): per scheduled row {row, first, end, 0}
  // (fs4: forward sparse rows, bs4: backward), per product {col, slot, transposed slot, 0}
  // (fr4 over fr_*, br4 over br_*)
  std::vector<int> fs4, bs4, fr4, br4;
  // sparse operators by position (x rows) or u rows
  std::vector<int> gu_ptr, gu_col, gu_src;
  std::vector<int> gut_ptr, gut_col, gut_src;
  // forward schedules per 32-column panel of Z (see symbolic.cpp):
  // levels [zp_lev_off[p], zp_lev_off[p+1]) of panel p, rows of level l in
  // zp_rows[zp_lev_ptr[l], zp_lev_ptr[l+1]), products of scheduled row e in
  // [zp_eptr[e], zp_eptr[e+1]); zero rows zp_zrows[zp_zptr[p], zp_zptr[p+1]);
  // products of trailing-block row a in [zp_tptr[p*nd + a], zp_tptr[p*nd + a + 1])
  int zp_npan = 0;
  std::vector<int> zp_lev_off, zp_lev_ptr, zp_rows, zp_eptr, zp_col, zp_slot, zp_zptr, zp_zrows, zp_tptr, zp_tcol,
      zp_tslot;
  std::vector<int> kx_ptr, kx_col, kx_src;
  std::vector<int> ku_ptr, ku_col, ku_src;
  // bounds (+-inf allowed)
  std::vector<double> xl, xu, ul, uu, sl, su;
  std::vector<double> c2, c1, pmax, qmax;
  long long n_ops = 0;
};

// Builds the symbolic structures.  Returns false with a message on invalid
// networks (bad indices, duplicate or self lines, gen_bus[0] != 0, ...).
// big: 0 = the large-trailing-block kernels only when the dense trailing
// block exceeds BIG_ND, 1 = always (the same results through the other
// kernels, for tests on small networks)
constexpr int BIG_ND = 400;
bool build_symbolic(const HostNet &net, int N, Sym &S, std::string &err, int big = 0);
