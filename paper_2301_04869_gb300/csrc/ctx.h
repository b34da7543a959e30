// The context of one reduced-space IPM instance (internal to libipm.so).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ipm.h"
#include "dev.cuh"
#include "ipm_internal.h"
#include "kernels.h"

// IPM constants (the same rule set as the CPU oracle)
namespace ipmc {
constexpr double MU0 = 0.1;
constexpr double RHO0 = 1.0;
}

struct ipm_ctx {
  Sym S;
  DevSym ds{};
  DevWork dw{};
  ipm_options opt{};
  std::string err;
  std::vector<void *> allocs;
  double *state = nullptr;
  long long state_len = 0, step_len = 0;
  // work buffers
  double *Z = nullptr, *Y = nullptr, *Yu = nullptr, *partial = nullptr;
  int2 *tiles = nullptr;
  int *tile_of = nullptr;
  int ntiles = 0, nt1 = 0, ngroups = 0;
  long long kchunk = 0;
  double *Khat = nullptr, *M = nullptr, *F = nullptr, *diag1 = nullptr, *rhs_u = nullptr;
  double *rhs_corr = nullptr, *cpos = nullptr;  // d(rhs_u)/d(delta); scratch [N][max(nx,nu)]
  double *gLu = nullptr, *HTt_u = nullptr;
  double *pg_curv = nullptr, *pmax_d = nullptr;
  // large-block LU: trailing updates on the tensor cores at FP64 grade
  // (mixed and FP64_TC paths), turned off for good if it ever gives a
  // non-finite value
  bool emu_lu_on = false;
  EmuLuPlan emu_lu;
  bool tcs_on = false;  // mixed, large trailing block: its solve updates on the tensor cores
  TcsPlan tcs;
  // the paper's adjoint-solve reduction (IPM_REDUCTION_ADJOINT / _AUTO):
  // the columns of L_x as vectors [N][n_u][n_x], solved in place with G_x^T
  bool adjoint = false;
  double *Wadj = nullptr;
  // FP64 contraction emulated on the tensor cores (IPM_PREC_FP64_TC)
  bool emu = false;
  EmuPlan emuZY, emuZZ;
  void *zplE = nullptr, *yplE = nullptr;
  int *expZ = nullptr, *expY = nullptr, *emu_rs = nullptr;
  int2 *emu_tiles = nullptr;
  int *emu_tile_of = nullptr;
  double *emupart = nullptr;
  int emu_max_groups = 0;
  long long n_emu_fallback = 0;
  // mixed path
  bool mixed = false;
  float *Z32 = nullptr, *Y32 = nullptr;
  void *zpl = nullptr, *ypl = nullptr;  // BF16x3 planes, K-major [3][nu][kpad]
  double *tcpart = nullptr;
  TcPlan planZY, planZZ;
  double *pcg_b = nullptr, *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr, *pcg_Ap = nullptr;
  int refine_iters = 0;
  double refine_res = 0.0;
  bool neg_curv = false;     // CG met p^T A p <= 0
  double curv_q = 0.0;       // and the Rayleigh quotient p^T A p / p^T p there
  bool exact_iter = false;   // this iteration runs the FP64 condensation (mixed fallback)
  long long n_fallback = 0;  // mixed-path iterations that needed the FP64 condensation
  long long n_curv_raise = 0;  // mixed path: delta_w raised after CG met non-positive curvature
  double *step = nullptr, *px = nullptr, *pu = nullptr, *ps = nullptr, *py = nullptr, *pz = nullptr;
  // iterative refinement on the residual of the augmented system eq. (6):
  // residual blocks (reused as the correction's right-hand side), the
  // correction, its condensed right-hand side, scratch in position order
  double *ar1x = nullptr, *ar1u = nullptr, *ar2 = nullptr, *ar3 = nullptr, *ar4 = nullptr, *atw = nullptr;
  double *dstep = nullptr, *dpx = nullptr, *dpu = nullptr, *dps = nullptr, *dpy = nullptr, *dpz = nullptr;
  double *arh1x = nullptr, *arh2 = nullptr, *arhs = nullptr, *apos2 = nullptr, *bpos2 = nullptr, *vpos2 = nullptr;
  unsigned long long *amax = nullptr, *h_amax = nullptr;
  double *aupart = nullptr, *aumag = nullptr;  // per-(scenario, u row) terms [N][n_u]
  int aug_steps = 0;
  double aug_res0 = 0.0, aug_res = 0.0;
  double *dz[6] = {};
  double *Hp = nullptr, *kpx = nullptr, *kpu = nullptr, *vpos = nullptr, *bpos = nullptr, *apos = nullptr;
  double *xt = nullptr, *ut = nullptr, *st = nullptr, *gt = nullptr, *ht = nullptr, *fst = nullptr,
         *Pt = nullptr, *Qt = nullptr;
  double *red_partial = nullptr, *red_out = nullptr;
  double *h_red = nullptr;  // pinned host mirror of reduction outputs
  int *h_flags = nullptr;
  int nL = 0;
  long long n_bounds = 0;
  // host mirror of the state scalars
  double mu = ipmc::MU0, rho = ipmc::RHO0, delta_last = 0.0;
  double delta_fact = 0.0;
  bool have_eval = false, have_cond = false, have_fact = false, M_valid = false;
  double info[10] = {0};
  double errs[6] = {0};
  double mean_compl = 0.0;
  // phase timers
  bool prof = false;
  cudaEvent_t ev[2 * IPM_N_PHASES] = {};
  // side streams: the transposed solve for p_y (joined before y is
  // updated; it overlaps the line search, which does not need p_y), and the
  // reduced right-hand side beside the split (inside the captured graph)
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;  // reduced right-hand side beside the split
  bool py_pending = false;
  bool ev_pending[IPM_N_PHASES] = {};
  double t_ms[IPM_N_PHASES] = {0};
  double t_cnt[IPM_N_PHASES] = {0};
  // barrier parameter as read by the condensation kernels (pinned host -> device)
  double *h_mu = nullptr, *d_mu = nullptr;
  // CUDA graphs of the condensation: [0] FP64 branch, [1] mixed branch; the
  // part before the reduced-Hessian contraction and the part after it
  cudaGraphExec_t gx_pre[2] = {}, gx_post[2] = {};
  long long gx_pre_n[2] = {}, gx_post_n[2] = {};
  bool graph_failed = false;
  // multi-instance runner: when set, the FP64 contraction is handed to the
  // hook (which may group it with other instances) instead of launched here
  void (*gemm_hook)(void *arg, ipm_ctx *c, cudaStream_t st) = nullptr;
  void *gemm_hook_arg = nullptr;
  // launch parameters chosen by the autotuner
  bool tuned = false;
  int zs_threads = 256;
  int max_groups = 0;      // capacity of `partial` in scenario groups
  int tc_max_groups = 0;   // capacity of `tcpart`
  double tune_ms[8] = {0};
  // warm-start vector layout (built on first use)
  int *warm_idx = nullptr;
  int warm_seg[10] = {};
  bool warm_ready = false;
};
