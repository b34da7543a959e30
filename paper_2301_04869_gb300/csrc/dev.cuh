// Device-side views of the symbolic structures and shared helpers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef IPM_LU_LISTS_DEFINED
#define IPM_LU_LISTS_DEFINED
constexpr int LU_LISTS = 1024;  // lists of trailing-block products of the LU factorization
#endif

struct DevSym {
  int n, L, ng, N, nx, nu, m, nnzA, nnzKB, nnzLU, nlev, nlev_b, nlev_f, t0, nd, nlev_fs, nlev_bs;
  int nflow;  // line-flow rows of h (2 L with ratings, else 0)
  // large trailing block (global-memory kernels): flag, offset of the block
  // in each scenario's LU values (column-major, leading dimension nd), and
  // max |G_x| per scenario (reference of the pivot test) [N]
  int big, dense_base;
  double *lu_amax;
  const int *xth, *xv, *uv, *gen_of_bus, *xbus, *xkind;
  const int *lfr, *lto;
  const double *lg, *lb, *lbh;
  const int *a_ptr, *a_col, *a_diag, *inc_ptr, *inc_line, *inc_other, *inc_aslot;
  const int *a_tslot;  // per A slot (i, k): the slot of (k, i)
  const int *kb_ptr, *kb_col, *kb_row, *kb_aslot, *kbi_ptr, *kbi_r, *kbi_ja, *kbi_jb;
  const int *hrow_bus, *hrow_comp, *ht_ptr, *ht_r, *ht_aslot;
  const int *perm, *iperm;
  const int *lu_diag, *lu_init, *tail_slot;
  const int *f_lev_ptr, *f_piv_ptr, *f_piv, *f_tgt, *f_op_ptr, *f_op_l, *f_op_u, *f_op_k;
  const int *lsc_slot, *lsc_k;
  const int *tw_len, *tw_l, *tw_u, *tw_e;  // trailing-block products per LU thread
  const int *fw_lev_ptr, *fw_rows, *fr_ptr, *fr_col, *fr_lslot, *fr_uslot;
  const int *bw_lev_ptr, *bw_rows, *br_ptr, *br_col, *br_uslot, *br_lslot;
  const int *fs_lev_ptr, *fs_rows, *bs_lev_ptr, *bs_rows;
  const int4 *fs4, *bs4, *fr4, *br4;  // packed single-RHS sweeps (symbolic.cpp)
  const int *gu_ptr, *gu_col, *gu_src, *gut_ptr, *gut_col, *gut_src;
  const int *kx_ptr, *kx_col, *kx_src, *ku_ptr, *ku_col, *ku_src;
  int zp_npan;  // forward schedules per 32-column panel of Z (symbolic.cpp)
  const int *zp_lev_off, *zp_lev_ptr, *zp_rows, *zp_eptr, *zp_col, *zp_slot, *zp_zptr, *zp_zrows, *zp_tptr, *zp_tcol,
      *zp_tslot;
  const double *xl, *xu, *ul, *uu, *sl, *su, *c2, *c1;
  const double *pd, *qd;  // [N][n]
  // line status per (line, scenario), lon[l * N + sc] in {0, 1}, or null
  // (every line in service): line-tripping contingencies
  const double *lon;
};

// Dynamic per-iteration arrays (device).  Vectors are scenario-major
// [N][len]; sparse values (J, W, K) are scenario-fastest [slot*4+e][N];
// LU values are scenario-major [N][nnzLU].
struct DevWork {
  // primal/dual state (views into the state vector)
  double *x, *u, *s, *y, *z, *zlx, *zux, *zlu, *zuu, *zls, *zus, *scal;
  // evaluation
  double *P, *Q, *g, *h, *fs;    // P,Q [N][n]; g [N][nx]; h [N][m]; fs [N]
  double *J, *W, *JTl;           // J,W [4 nnzA][N]; JTl [N][2n]
  // line-flow rows (with ratings): d h / d (theta, v) of the row's own-end bus
  // (w = 0) and other-end bus (w = 1), HF[((f * 2 + w) * 2 + kind) * N + sc]
  // for flow row f = r - (n_g + 1)
  double *HF;
  double *K;                     // [4 nnzKB][N]
  double *Sx, *Su, *Ss;          // barrier diagonals
  double *r1x, *r1u, *r2, *r4, *rh1x, *rh2, *tv;  // right-hand sides
  double *LU, *rd;               // [N][nnzLU], reciprocal pivots [N][nx]
  int *flags;                    // device error / status words
};

// 1/sqrt(d) for d > 0: the single-precision hardware estimate (relative
// error below 2^-22) refined by two Newton-Raphson steps for the reciprocal
// square root, y <- y + y (1/2 - (d/2) y^2), each of which about squares
// the relative error (2^-43, then below FP64 rounding).  Three dependent
// FP64 operations per step instead of a square root and a division (~1,200
// cycles of dependent latency on GB300).  Outside [1e-30, 1e30] (no FP32
// estimate) the plain form is used.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)d));
  double y = (double)yf;
  const double h = 0.5 * d;
  double r = fma(-h * y, y, 0.5);
  y = fma(y, r, y);
  r = fma(-h * y, y, 0.5);
  return fma(y, r, y);
}


__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// bus voltage angle / magnitude of scenario sc
__device__ __forceinline__ double bus_theta(const DevSym &S, const double *x, int sc, int i) {
  return i == 0 ? 0.0 : x[(size_t)sc * S.nx + S.xth[i]];
}
__device__ __forceinline__ double bus_v(const DevSym &S, const double *x, const double *u, int sc, int i) {
  int q = S.xv[i];
  return q >= 0 ? x[(size_t)sc * S.nx + q] : u[S.uv[i]];
}

// other-end bus of line-flow row f (from-end rows first, then to-end rows)
__device__ __forceinline__ int flow_other(const DevSym &S, int f) {
  return f < S.L ? S.lto[f] : S.lfr[f - S.L];
}

// flags
enum { FLAG_SINGULAR = 0, FLAG_NOT_PD = 1, FLAG_NONFINITE = 2, FLAG_TIMEOUT = 3, FLAG_COUNT = 8 };
