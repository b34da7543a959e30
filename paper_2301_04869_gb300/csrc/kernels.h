// Host-side launch wrappers of the CUDA kernels (internal).
#pragma once
#include <atomic>

#include "dev.cuh"

// kernels launched by this library: all threads, and the calling thread
extern std::atomic<long long> g_ipm_launches;
extern thread_local long long t_ipm_launches;
inline void ipm_count_launch() {
  ++g_ipm_launches;
  ++t_ipm_launches;
}

// Raise a kernel's dynamic shared-memory cap to everything the device allows
// next to its static shared memory.  Done once per kernel: setting it per
// launch to that launch's size would race between host threads that launch
// the same kernel for different instances.
template <class K>
inline bool raise_smem_cap(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes) == cudaSuccess;
}

// kernels_eval.cu
void launch_functions(const DevSym &S, const double *x, const double *u, double *P, double *Q, double *g,
                      double *h, double *fs, cudaStream_t st);
void launch_derivatives(const DevSym &S, DevWork &D, cudaStream_t st);
void launch_sigmas(const DevSym &S, DevWork &D, cudaStream_t st);
void launch_condense(const DevSym &S, DevWork &D, cudaStream_t st);
// mu: device pointer to the barrier parameter (read when the kernels run, so
// that a captured graph of the condensation follows the current value)
void launch_rhs(const DevSym &S, DevWork &D, const double *mu, double *gLu, double *HTt_u, cudaStream_t st);
void launch_ugrad(const DevSym &S, DevWork &D, double *gLu, cudaStream_t st);

struct EmuLuPlan;
// kernels_lu.cu (emu_lu: the large-block LU's trailing updates on the tensor
// cores at FP64 grade; null: on the FP64 units)
void launch_lu_factor(const DevSym &S, int nL, const double *J, double *LU, double *rd, int *flags,
                      cudaStream_t st, bool allow_pair = true, const EmuLuPlan *emu_lu = nullptr);
// g, b (optional, [N][n_x]): also b = G_x^{-1} g in position order (g in
// state order), in an extra right-hand-side lane, when zsolve64_folds_b
void launch_zsolve64(const DevSym &S, const double *LU, const double *rd, const double *J, const double *K,
                     double *Z, double *Y, double *Yu, cudaStream_t st, int threads = 256,
                     const double *g = nullptr, double *b = nullptr, int *ezy = nullptr);
bool zsolve64_folds_b(const DevSym &S);
// kernels_big.cu: the large trailing block (S.big) in global memory
void launch_big_lu_dense(const DevSym &S, double *LU, double *rd, const double *amax, int *flags, cudaStream_t st,
                         const EmuLuPlan *emu_lu = nullptr);
void launch_big_trsm64(const DevSym &S, const double *LU, const double *rd, double *Z, cudaStream_t st);
// one vector per scenario (v: [N][n_x], positions) through the block: forward
// then backward, with G_x (trans 0) or G_x^T (trans 1)
void launch_big_trsv(const DevSym &S, const double *LU, const double *rd, double *v, int trans, cudaStream_t st);
struct TcsPlan;
// tcs: the tensor-core variant of the block updates (mixed path), or null
void launch_big_trsm32(const DevSym &S, const double *LU, const double *rd, float *Z, cudaStream_t st,
                       const TcsPlan *tcs = nullptr, int *flags = nullptr);
void launch_zsolve32(const DevSym &S, const double *LU, const double *rd, const double *J, const double *K,
                     float *Z, float *Y, double *Yu, cudaStream_t st, int threads = 256,
                     const TcsPlan *tcs = nullptr, int *flags = nullptr);
void launch_solve1(const DevSym &S, const double *LU, const double *rd, double *v, int trans,
                   cudaStream_t st);
// vps vectors per scenario: v [N * vps][n_x] (position order), one CTA of
// `threads` (a multiple of 32) per vector
void launch_solve1_batched(const DevSym &S, const double *LU, const double *rd, double *v, int trans, int vps,
                           int threads, cudaStream_t st);
// kernels_adjoint.cu: the paper's local reduction by adjoint solves
// (K_hat V = L_u - G_u^T G_x^{-T} L_x, §3.2) on all n_u unit vectors at once
void launch_transpose_rows(int N, int nx, int nu, const double *Y, double *W, cudaStream_t st);
void launch_adjoint_assemble(const DevSym &S, const double *J, const double *Yu, const double *W, const double *diag,
                             double *Khat, cudaStream_t st);

// kernels_dense.cu
void launch_gemm_tn64(long long krows, long long kc, int nu, int ngroups, const double *A, const double *B,
                      const int2 *tiles, int ntiles, double *partial, cudaStream_t st);
// one work item of the grouped multi-instance contraction: the 64 x 64 tile at
// (i0, j0) of A^T B over rows [r0, r1), written to P
struct GemmItem {
  const double *A, *B;
  double *P;
  long long r0, r1;
  int nu, i0, j0, pad;
};
void launch_gemm_grouped(const GemmItem *items, int nitems, int *counter, cudaStream_t st);
void launch_khat_assemble(int nu, int N, int ngroups, int ntiles, int nt1, const double *partial,
                          const int *tile_of, const double *Yu, const double *diag, double *Khat,
                          cudaStream_t st);
void launch_shift(int nu, const double *Khat, const double *M, double delta, double tau, double *F,
                  cudaStream_t st);
void launch_maxdiag(int n, const double *A, double *out, cudaStream_t st);
void launch_cholesky(int n, double *A, int *flags, cudaStream_t st);
void launch_chol_solve(int n, const double *L, double *b, cudaStream_t st);

// kernels_step.cu
void launch_errors(const DevSym &S, DevWork &D, const double *gLu, double *partial, double *out,
                   cudaStream_t st);
void launch_merit(const DevSym &S, const double *x, const double *u, const double *s, const double *g,
                  const double *h, const double *fs, double *partial, double *out, cudaStream_t st);
void launch_dir(const DevSym &S, DevWork &D, const double *px, const double *pu, const double *ps,
                const double *kpx, const double *kpu, const double *Hp, double mu, double delta,
                double *partial, double *out, cudaStream_t st);
void launch_ftb(const DevSym &S, DevWork &D, const double *px, const double *pu, const double *ps,
                const double *const *dz, double tau, double *partial, double *out, cudaStream_t st);
void launch_gather_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale,
                       cudaStream_t st);
void launch_scatter_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale,
                        cudaStream_t st);
void launch_gu_apply(const DevSym &S, const double *J, const double *pu, double *v, cudaStream_t st);
void launch_kapply(const DevSym &S, const double *K, const double *px_pos, const double *pu, double *kpx,
                   double *kpu, cudaStream_t st);
void launch_lincomb(long long n, double *out, double a, const double *x, double b, const double *y,
                    double c, const double *z, cudaStream_t st);
void launch_rhs_reduced(const DevSym &S, const double *J, const double *K, const double *rh2,
                        const double *a, const double *b, double *rhs, cudaStream_t st);
void launch_zt_apply(const DevSym &S, const double *Z, const double *w, const double *K, const double *b,
                     double alpha, double beta, double *out, double *part, cudaStream_t st);
void launch_z_apply(const DevSym &S, const double *Z, const double *pu, double a, double *v, cudaStream_t st);
void launch_gut_sum(const DevSym &S, const double *J, const double *a, double scale, double *out,
                    cudaStream_t st);
void launch_apply_finish(const DevSym &S, const double *kpu, const double *diag, double delta, const double *v,
                         double *out, cudaStream_t st);
void launch_dot2(int n, const double *a, const double *b, const double *c, const double *d, double *out,
                 cudaStream_t st);
void launch_pz_ps(const DevSym &S, DevWork &D, const double *px, const double *pu, double *Hp, double *pz,
                  double *ps, cudaStream_t st);
void launch_bound_steps(long long n, int period, const double *w, const double *dw, const double *l,
                        const double *b, const double *zl, const double *zu, double mu, double *dzl,
                        double *dzu, cudaStream_t st);
void launch_dual_update(long long n, int period, const double *w, const double *l, const double *b,
                        double *zl, double *zu, const double *dzl, const double *dzu, double az, double mu,
                        double ks, cudaStream_t st);
void launch_push(long long n, int period, double *w, const double *l, const double *b, double k1, double k2,
                 cudaStream_t st);
void launch_init_primal(const DevSym &S, double *x, double *u, const double *pmax, cudaStream_t st);
void launch_fill_bound_duals(long long n, int period, const double *l, const double *b, double *zl,
                             double *zu, cudaStream_t st);

// kernels_refine.cu (residual of the augmented system eq. (6) at a step; all
// vectors in state order except kpx_pos, the positions of K p_d; amax[0],
// amax[1] (zeroed by the caller) receive the bit patterns of max |rho| and
// of the largest magnitude among the right-hand side and the block products)
void launch_aug_residual(const DevSym &S, const DevWork &D, double delta, const double *px, const double *pu,
                         const double *ps, const double *py, const double *pz, const double *kpx_pos,
                         const double *kpu, const double *diag1, double *Hp, double *tw, double *rho1x,
                         double *rho1u, double *rho2, double *rho3, double *rho4, double *upart, double *umag,
                         unsigned long long *amax, cudaStream_t st);
// outx = ax + H_x^T v (per scenario), outu = au + sum_i H_u^T v_i
void launch_htv(const DevSym &S, const DevWork &D, const double *ax, const double *au, const double *v, double *outx,
                double *outu, double *upart, cudaStream_t st);
// t = Sigma_s r4 - r2
void launch_tv(long long n, const double *Ss, const double *r2, const double *r4, double *t, cudaStream_t st);
// pz = Sigma_s (H p_d + r4) - r2, ps = -(r2 + pz) / Sigma_s
void launch_pzps_rhs(const DevSym &S, const DevWork &D, const double *px, const double *pu, const double *r2,
                     const double *r4, double *pz, double *ps, cudaStream_t st);
// out[0] = max(out[0], max|a|), out[1] = max(out[1], max|b|) as the bit patterns of the magnitudes
void launch_maxabs2(long long n, const double *a, const double *b, unsigned long long *out, cudaStream_t st);

// warm-start vectors: segment offsets (seg[0] = 0 ... seg[9] = d) and the
// bounded-component lists of the six dual blocks (device, concatenated)
struct WarmSeg {
  int seg[10];
  int nx, m;
  const int *idx;
};
void launch_warm_target(const DevWork &D, const WarmSeg &W, int N, float *out, cudaStream_t st);
void launch_warm_apply(const DevWork &D, const WarmSeg &W, int N, const float *pred, cudaStream_t st);
void launch_warm_z(long long n, const DevWork &D, cudaStream_t st);
void launch_warm_yrhs(const DevSym &S, const DevWork &D, double *r, cudaStream_t st);

// kernels_tc.cu (tcgen05 BF16x3 reduced-Hessian product)
struct TcPlan {
  int nu = 0, nt1 = 0, ntiles = 0, kb_total = 0, kb_per_group = 0, ngroups = 0;
  long long kpad = 0;
  alignas(64) unsigned char maps[6 * 128];  // six CUtensorMap (A planes, B planes)
};
void tc_plan(int nu, long long krows, TcPlan &P);
// tensor map (128 bytes at map) of a BF16 matrix [rows][k] (k contiguous, k a
// multiple of 8), box 64 (k) x 128 (rows), 128-byte swizzle
bool tc_make_kmajor_map(void *map, const void *base, int rows, long long k);
// the same with a box of box_rows rows (64 or 128)
bool tc_make_kmajor_map_box(void *map, const void *base, int rows, long long k, int box_rows, int box_k);

// kernels_emu.cu (FP64-grade K_hat from exact BF16 slices on the tensor cores)
struct EmuPlan {
  int nu = 0, ntm = 0, ntn = 0, ntiles = 0, kb_total = 0, kb_per_group = 0, ngroups = 0;
  long long krows = 0, kpad = 0;
  int2 *tiles = nullptr;
  int *tile_of = nullptr;
  const void *a_planes = nullptr, *b_planes = nullptr;
  int *exp_a = nullptr, *exp_b = nullptr;
  alignas(64) unsigned char maps[16 * 128];  // eight A-plane and eight B-plane CUtensorMap
};
// bytes of the slice planes of one operand; exponents take (kpad / 512) * nu ints
size_t emu_planes_bytes(int nu, long long krows);
long long emu_kpad(long long krows);
// tiles_dev: room for ceil(nu/128) * ceil(nu/64) int2; tile_of_dev: the same count of ints
bool emu_plan(EmuPlan &P, int nu, long long krows, const void *a_planes, const void *b_planes, int *exp_a,
              int *exp_b, int2 *tiles_dev, int *tile_of_dev);
void emu_regroup(EmuPlan &P, int groups);
size_t emu_partial_doubles(const EmuPlan &P, int max_groups);
// power-of-two row balancing of Z, Y (rs: one int per contraction row)
void launch_emu_rowscale(const EmuPlan &P, const double *Z, const double *Y, int *rs, cudaStream_t st);
// split one operand (A: scaled by 2^rs, B: by 2^-rs; rs may be null)
void launch_emu_split(const EmuPlan &P, const double *src, bool b_side, const int *rs, cudaStream_t st,
                      const int *ezy = nullptr);
// both operands of K = Z^T Y in one launch (Z: A side, Y: B side)
void launch_emu_split_pair(const EmuPlan &P, const double *Z, const double *Y, const int *rs, cudaStream_t st,
                           const int *ezy = nullptr);
void launch_emu_schur(const EmuPlan &P, double *partial, int *flags, cudaStream_t st);
void launch_emu_assemble(const EmuPlan &P, int N, const double *partial, const double *Yu, const double *diag,
                         double *Khat, cudaStream_t st);
// the large-block LU's trailing update A22 -= L21 U12 at FP64 grade on the
// tensor cores: slices of the N scenarios' L21 rows and U12 columns stacked
// with stride Mp (nd rounded up to 128), planes [8][N Mp][64] each
struct EmuLuPlan {
  int N = 0, nd = 0, Mp = 0;
  void *a_planes = nullptr, *b_planes = nullptr;
  int *exp_a = nullptr, *exp_b = nullptr;
  alignas(64) unsigned char maps[16 * 128];
};
size_t emu_lu_planes_bytes(int N, int nd);
bool emu_lu_plan(EmuLuPlan &P, int N, int nd, void *a_planes, void *b_planes, int *exp_a, int *exp_b);
void launch_emu_lu_update(const EmuLuPlan &P, double *LU, long long nnzlu, int dense_base, int kb, int ke, int *flags,
                          cudaStream_t st);
// kernels_tcsolve.cu: the mixed path's solve through the large trailing
// block with its updates as BF16x3 products on the tensor cores; planes of
// the factor block [3][N ndp][kpl] then of the finished rows [3][N nup][kpl]
// (ndp = kpl = nd, nup = nu, rounded up to 128), zero-filled once
struct TcsPlan {
  int N = 0, nd = 0, nu = 0, ndp = 0, nup = 0;
  long long kpl = 0;
  void *fpl = nullptr, *xpl = nullptr;
  alignas(64) unsigned char maps[6 * 128];
};
size_t tcs_planes_bytes(int N, int nd, int nu, size_t *f_bytes = nullptr);
bool tcs_plan(TcsPlan &P, int N, int nd, int nu, void *planes);
void launch_tcs_split_f(const TcsPlan &P, const double *LU, long long nnzlu, int dense_base, cudaStream_t st);
void launch_tcs_split_x(const TcsPlan &P, int nx, int t0, const float *Z, int r0, int r1, cudaStream_t st);
// Z_d rows [r0, r1) -= F(rows, [k0, k1)) Z_d([k0, k1), :) (k0 a multiple of 64)
void launch_tcs_update(const TcsPlan &P, int nx, int t0, float *Z, int r0, int r1, int k0, int k1, int *flags,
                       cudaStream_t st);
bool tc_set_operands(TcPlan &P, const void *a_planes, const void *b_planes);
void launch_split_t(long long krows, int nu, long long kpad, const float *src, void *planes, cudaStream_t st);
void launch_tc_schur(const TcPlan &P, double *partial, int *flags, cudaStream_t st);
// re-split the K range of a plan into about `groups` scenario groups
void tc_regroup(TcPlan &P, int groups);
void launch_tc_assemble(const TcPlan &P, int N, const double *partial, const double *Yu, const double *diag,
                        double *Khat, cudaStream_t st);
