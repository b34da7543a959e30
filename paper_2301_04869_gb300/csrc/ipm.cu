// C ABI of the reduced-space IPM (include/ipm.h): context management and the
// host-side driver of one interior-point iteration.  Every numerical step of
// the path runs in the kernels of kernels_*.cu; the host only sequences them
// and takes the scalar decisions (barrier update, inertia-correction retries,
// line-search acceptance) on values read back from the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "ctx.h"
#include "dev.cuh"
#include "ipm_internal.h"
#include "kernels.h"

std::atomic<long long> g_ipm_launches{0};
thread_local long long t_ipm_launches = 0;

namespace {

// IPM constants (the same rule set as the CPU oracle)
constexpr double MU0 = 0.1, K1 = 1e-2, K2 = 1e-2, TAU_MIN = 0.99, KAPPA_EPS = 10.0, KAPPA_MU = 0.2,
                 THETA_MU = 1.5, ETA = 1e-4, ALPHA_MIN = 1e-12, KAPPA_SIGMA = 1e10, S_MAX = 100.0,
                 RHO0 = 1.0, RHO_FRAC = 0.1, DELTA0 = 1e-4, DELTA_MIN = 1e-20, DELTA_MAX = 1e40,
                 KW_MINUS = 1.0 / 3.0, KW_PLUS = 8.0, KW_PLUS_BAR = 100.0;
// bound push of a learned warm start (relative, as K1/K2 of the cold start)
constexpr double K1_WARM = 1e-5;

}  // namespace


namespace {

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return fail(c, IPM_ERR_CUDA, #call, e_); \
  } while (0)

ipm_status fail(ipm_ctx *c, ipm_status s, const char *what, cudaError_t e = cudaSuccess) {
  if (c) {
    c->err = what;
    if (e != cudaSuccess) {
      c->err += ": ";
      c->err += cudaGetErrorString(e);
    }
  }
  return s;
}

template <class T>
ipm_status dalloc(ipm_ctx *c, T **p, size_t count) {
  if (count == 0) count = 1;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, IPM_ERR_OOM, "cudaMalloc", e);
  }
  c->allocs.push_back(q);
  *p = (T *)q;
  if (c->opt.poison) cudaMemset(q, 0xFF, count * sizeof(T));  // all-ones bytes: NaN in FP64 and FP32
  return IPM_OK;
}

template <class T>
ipm_status upload(ipm_ctx *c, const T **dst, const std::vector<T> &v) {
  T *p = nullptr;
  ipm_status s = dalloc(c, &p, v.size());
  if (s != IPM_OK) return s;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dst = p;
  return IPM_OK;
}

#define TRY(x)                   \
  do {                           \
    ipm_status s_ = (x);         \
    if (s_ != IPM_OK) return s_; \
  } while (0)

inline cudaStream_t STR(void *s) { return (cudaStream_t)s; }

double emu(const double *e, double mu) {
  return std::max(std::max(e[0] / e[4], e[1]), std::max(e[2] - mu, mu - e[3]) / e[5]);
}

ipm_status upload_symbolic(ipm_ctx *c, const HostNet &net, const double *pd, const double *qd) {
  Sym &S = c->S;
  DevSym &d = c->ds;
  d.n = S.n; d.L = S.L; d.ng = S.ng; d.N = S.N; d.nx = S.nx; d.nu = S.nu; d.m = S.m;
  d.nnzA = S.nnzA; d.nnzKB = S.nnzKB; d.nnzLU = S.nnzLU; d.nlev = S.nlev; d.nlev_b = S.nlev_b;
  d.nlev_f = S.nlev_f; d.t0 = S.t0; d.nd = S.nd; d.nlev_fs = S.nlev_fs; d.nlev_bs = S.nlev_bs;
  d.nflow = S.nflow;
  d.big = S.big ? 1 : 0;
  d.dense_base = S.dense_base;
  d.lu_amax = nullptr;
  if (S.big) TRY(dalloc(c, &d.lu_amax, (size_t)S.N));
  TRY(upload(c, &d.xth, S.xth)); TRY(upload(c, &d.xv, S.xv)); TRY(upload(c, &d.uv, S.uv));
  TRY(upload(c, &d.gen_of_bus, S.gen_of_bus)); TRY(upload(c, &d.xbus, S.xbus)); TRY(upload(c, &d.xkind, S.xkind));
  TRY(upload(c, &d.lfr, S.lfr)); TRY(upload(c, &d.lto, S.lto));
  TRY(upload(c, &d.lg, S.lg)); TRY(upload(c, &d.lb, S.lb)); TRY(upload(c, &d.lbh, S.lbh));
  TRY(upload(c, &d.a_ptr, S.a_ptr)); TRY(upload(c, &d.a_col, S.a_col)); TRY(upload(c, &d.a_diag, S.a_diag));
  TRY(upload(c, &d.a_tslot, S.a_tslot));
  TRY(upload(c, &d.inc_ptr, S.inc_ptr)); TRY(upload(c, &d.inc_line, S.inc_line));
  TRY(upload(c, &d.inc_other, S.inc_other)); TRY(upload(c, &d.inc_aslot, S.inc_aslot));
  TRY(upload(c, &d.kb_ptr, S.kb_ptr)); TRY(upload(c, &d.kb_col, S.kb_col)); TRY(upload(c, &d.kb_row, S.kb_row));
  TRY(upload(c, &d.kb_aslot, S.kb_aslot)); TRY(upload(c, &d.kbi_ptr, S.kbi_ptr)); TRY(upload(c, &d.kbi_r, S.kbi_r));
  TRY(upload(c, &d.kbi_ja, S.kbi_ja)); TRY(upload(c, &d.kbi_jb, S.kbi_jb));
  TRY(upload(c, &d.hrow_bus, S.hrow_bus)); TRY(upload(c, &d.hrow_comp, S.hrow_comp));
  TRY(upload(c, &d.ht_ptr, S.ht_ptr)); TRY(upload(c, &d.ht_r, S.ht_r)); TRY(upload(c, &d.ht_aslot, S.ht_aslot));
  TRY(upload(c, &d.perm, S.perm)); TRY(upload(c, &d.iperm, S.iperm));
  TRY(upload(c, &d.lu_diag, S.lu_diag)); TRY(upload(c, &d.lu_init, S.lu_init));
  TRY(upload(c, &d.tail_slot, S.tail_slot));
  TRY(upload(c, &d.fs_lev_ptr, S.fs_lev_ptr)); TRY(upload(c, &d.fs_rows, S.fs_rows));
  {
    const int *q = nullptr;
    TRY(upload(c, &q, S.fs4)); d.fs4 = reinterpret_cast<const int4 *>(q);
    TRY(upload(c, &q, S.bs4)); d.bs4 = reinterpret_cast<const int4 *>(q);
    TRY(upload(c, &q, S.fr4)); d.fr4 = reinterpret_cast<const int4 *>(q);
    TRY(upload(c, &q, S.br4)); d.br4 = reinterpret_cast<const int4 *>(q);
  }
  TRY(upload(c, &d.bs_lev_ptr, S.bs_lev_ptr)); TRY(upload(c, &d.bs_rows, S.bs_rows));
  TRY(upload(c, &d.f_lev_ptr, S.f_lev_ptr)); TRY(upload(c, &d.f_piv_ptr, S.f_piv_ptr)); TRY(upload(c, &d.f_piv, S.f_piv));
  TRY(upload(c, &d.f_tgt, S.f_tgt)); TRY(upload(c, &d.f_op_ptr, S.f_op_ptr)); TRY(upload(c, &d.f_op_l, S.f_op_l));
  TRY(upload(c, &d.f_op_u, S.f_op_u)); TRY(upload(c, &d.f_op_k, S.f_op_k));
  TRY(upload(c, &d.lsc_slot, S.lsc_slot)); TRY(upload(c, &d.lsc_k, S.lsc_k));
  TRY(upload(c, &d.tw_len, S.tw_len)); TRY(upload(c, &d.tw_l, S.tw_l)); TRY(upload(c, &d.tw_u, S.tw_u));
  TRY(upload(c, &d.tw_e, S.tw_e));
  TRY(upload(c, &d.fw_lev_ptr, S.fw_lev_ptr)); TRY(upload(c, &d.fw_rows, S.fw_rows)); TRY(upload(c, &d.fr_ptr, S.fr_ptr));
  TRY(upload(c, &d.fr_col, S.fr_col)); TRY(upload(c, &d.fr_lslot, S.fr_lslot)); TRY(upload(c, &d.fr_uslot, S.fr_uslot));
  TRY(upload(c, &d.bw_lev_ptr, S.bw_lev_ptr)); TRY(upload(c, &d.bw_rows, S.bw_rows)); TRY(upload(c, &d.br_ptr, S.br_ptr));
  TRY(upload(c, &d.br_col, S.br_col)); TRY(upload(c, &d.br_uslot, S.br_uslot)); TRY(upload(c, &d.br_lslot, S.br_lslot));
  TRY(upload(c, &d.gu_ptr, S.gu_ptr)); TRY(upload(c, &d.gu_col, S.gu_col)); TRY(upload(c, &d.gu_src, S.gu_src));
  TRY(upload(c, &d.gut_ptr, S.gut_ptr)); TRY(upload(c, &d.gut_col, S.gut_col)); TRY(upload(c, &d.gut_src, S.gut_src));
  d.zp_npan = S.zp_npan;
  TRY(upload(c, &d.zp_lev_off, S.zp_lev_off)); TRY(upload(c, &d.zp_lev_ptr, S.zp_lev_ptr));
  TRY(upload(c, &d.zp_rows, S.zp_rows)); TRY(upload(c, &d.zp_eptr, S.zp_eptr)); TRY(upload(c, &d.zp_col, S.zp_col));
  TRY(upload(c, &d.zp_slot, S.zp_slot)); TRY(upload(c, &d.zp_zptr, S.zp_zptr)); TRY(upload(c, &d.zp_zrows, S.zp_zrows));
  TRY(upload(c, &d.zp_tptr, S.zp_tptr)); TRY(upload(c, &d.zp_tcol, S.zp_tcol)); TRY(upload(c, &d.zp_tslot, S.zp_tslot));
  TRY(upload(c, &d.kx_ptr, S.kx_ptr)); TRY(upload(c, &d.kx_col, S.kx_col)); TRY(upload(c, &d.kx_src, S.kx_src));
  TRY(upload(c, &d.ku_ptr, S.ku_ptr)); TRY(upload(c, &d.ku_col, S.ku_col)); TRY(upload(c, &d.ku_src, S.ku_src));
  TRY(upload(c, &d.xl, S.xl)); TRY(upload(c, &d.xu, S.xu)); TRY(upload(c, &d.ul, S.ul)); TRY(upload(c, &d.uu, S.uu));
  TRY(upload(c, &d.sl, S.sl)); TRY(upload(c, &d.su, S.su)); TRY(upload(c, &d.c2, S.c2)); TRY(upload(c, &d.c1, S.c1));
  std::vector<double> vpd(pd, pd + (size_t)S.N * S.n), vqd(qd, qd + (size_t)S.N * S.n);
  TRY(upload(c, &d.pd, vpd)); TRY(upload(c, &d.qd, vqd));
  c->nL = (int)S.lsc_slot.size();
  (void)net;
  return IPM_OK;
}

void set_groups(ipm_ctx *c, long long G);

ipm_status alloc_work(ipm_ctx *c) {
  const Sym &S = c->S;
  const long long N = S.N, nx = S.nx, nu = S.nu, m = S.m, n = S.n;
  c->state_len = 4 * N * nx + 4 * N * m + 3 * nu + 3;
  c->step_len = 2 * N * nx + 2 * N * m + nu;
  TRY(dalloc(c, &c->state, c->state_len));
  CK(cudaMemset(c->state, 0, c->state_len * sizeof(double)));
  DevWork &D = c->dw;
  double *p = c->state;
  D.x = p; p += N * nx;
  D.u = p; p += nu;
  D.s = p; p += N * m;
  D.y = p; p += N * nx;
  D.z = p; p += N * m;
  D.zlx = p; p += N * nx;
  D.zux = p; p += N * nx;
  D.zlu = p; p += nu;
  D.zuu = p; p += nu;
  D.zls = p; p += N * m;
  D.zus = p; p += N * m;
  D.scal = p;
  TRY(dalloc(c, &D.P, N * n)); TRY(dalloc(c, &D.Q, N * n)); TRY(dalloc(c, &D.g, N * nx));
  TRY(dalloc(c, &D.h, N * m)); TRY(dalloc(c, &D.fs, N));
  TRY(dalloc(c, &D.J, 4LL * S.nnzA * N)); TRY(dalloc(c, &D.W, 4LL * S.nnzA * N));
  D.HF = nullptr;
  if (S.nflow > 0) TRY(dalloc(c, &D.HF, 4LL * S.nflow * N));
  TRY(dalloc(c, &D.JTl, 2 * N * n)); TRY(dalloc(c, &D.K, 4LL * S.nnzKB * N));
  TRY(dalloc(c, &D.Sx, N * nx)); TRY(dalloc(c, &D.Su, nu)); TRY(dalloc(c, &D.Ss, N * m));
  TRY(dalloc(c, &D.r1x, N * nx)); TRY(dalloc(c, &D.r1u, nu)); TRY(dalloc(c, &D.r2, N * m));
  TRY(dalloc(c, &D.r4, N * m)); TRY(dalloc(c, &D.rh1x, N * nx)); TRY(dalloc(c, &D.rh2, nu));
  TRY(dalloc(c, &D.tv, N * m));
  TRY(dalloc(c, &D.LU, (long long)S.nnzLU * N)); TRY(dalloc(c, &D.rd, N * nx));
  if (S.big && (c->opt.precision == IPM_PREC_MIXED || c->opt.precision == IPM_PREC_FP64_TC)) {
    const size_t pb = emu_lu_planes_bytes((int)N, S.nd);
    const long long rows = N * (long long)((S.nd + 127) / 128 * 128);
    unsigned char *pa = nullptr, *pbp = nullptr;
    int *ea = nullptr, *eb = nullptr;
    TRY(dalloc(c, &pa, pb)); TRY(dalloc(c, &pbp, pb));
    TRY(dalloc(c, &ea, rows)); TRY(dalloc(c, &eb, rows));
    if (!emu_lu_plan(c->emu_lu, (int)N, S.nd, pa, pbp, ea, eb))
      return fail(c, IPM_ERR_CUDA, "tensor maps of the large-block LU update");
    c->emu_lu_on = true;
  }
  TRY(dalloc(c, &D.flags, FLAG_COUNT));
  CK(cudaMemset(D.flags, 0, FLAG_COUNT * sizeof(int)));
  c->mixed = c->opt.precision == IPM_PREC_MIXED;
  TRY(dalloc(c, &c->Yu, N * nu * nu));
  c->emu = c->opt.precision == IPM_PREC_FP64_TC;
  if (!c->mixed) {
    TRY(dalloc(c, &c->Z, N * nx * nu));
    TRY(dalloc(c, &c->Y, N * nx * nu));
    if (c->opt.reduction != IPM_REDUCTION_DENSE) TRY(dalloc(c, &c->Wadj, N * nx * nu));
    c->adjoint = c->opt.reduction == IPM_REDUCTION_ADJOINT;
    if (c->emu) {
      const long long krows = N * nx;
      const size_t pb = emu_planes_bytes((int)nu, krows);
      const long long ngr = emu_kpad(krows) / 512;
      unsigned char *pz = nullptr, *py = nullptr;
      TRY(dalloc(c, &pz, pb));
      TRY(dalloc(c, &py, pb));
      c->zplE = pz;
      c->yplE = py;
      TRY(dalloc(c, &c->expZ, ngr * nu));
      TRY(dalloc(c, &c->emu_rs, 2 * krows));  // row exponent maxima of Z and Y
      TRY(dalloc(c, &c->expY, ngr * nu));
      const long long nt = ((nu + 127) / 128) * ((nu + 63) / 64);
      TRY(dalloc(c, &c->emu_tiles, nt));
      TRY(dalloc(c, &c->emu_tile_of, nt));
      if (!emu_plan(c->emuZY, (int)nu, krows, c->zplE, c->yplE, c->expZ, c->expY, c->emu_tiles, c->emu_tile_of) ||
          !emu_plan(c->emuZZ, (int)nu, krows, c->zplE, c->zplE, c->expZ, c->expZ, c->emu_tiles, c->emu_tile_of))
        return fail(c, IPM_ERR_CUDA, "tensor maps of the emulated contraction");
      EmuPlan big = c->emuZY;
      emu_regroup(big, 2 * std::max(1, 152 / big.ntiles));
      c->emu_max_groups = std::max(big.ngroups, c->emuZY.ngroups);
      TRY(dalloc(c, &c->emupart, (long long)emu_partial_doubles(c->emuZY, c->emu_max_groups)));
    }
  } else {
    // one region holds either the mixed operands (FP32 Z, Y and the BF16x3
    // planes) or, in an iteration that falls back, the FP64 Z and Y
    tc_plan((int)nu, N * nx, c->planZY);
    c->planZZ = c->planZY;
    const size_t E = (size_t)N * nx * nu;
    const size_t pl = (size_t)3 * nu * c->planZY.kpad;  // bf16 elements per operand
    const size_t mixed_bytes = E * 4 * 2 + pl * 2 * 2;
    const size_t bytes = std::max(mixed_bytes, E * 8 * 2);
    unsigned char *region = nullptr;
    TRY(dalloc(c, &region, (bytes + 255) / 256 * 256));
    c->Z32 = (float *)region;
    c->Y32 = (float *)(region + E * 4);
    c->zpl = region + ((E * 8 + 255) / 256) * 256;
    c->ypl = (unsigned char *)c->zpl + pl * 2;
    c->Z = (double *)region;
    c->Y = (double *)(region + E * 8);
    if ((size_t)((unsigned char *)c->ypl - region) + pl * 2 > (bytes + 255) / 256 * 256)
      return fail(c, IPM_ERR_ARG, "internal: mixed region layout");
    if (!tc_set_operands(c->planZY, c->zpl, c->ypl) || !tc_set_operands(c->planZZ, c->zpl, c->zpl))
      return fail(c, IPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    {
      TcPlan big = c->planZY;
      tc_regroup(big, 2 * std::max(1, 152 / big.ntiles));
      c->tc_max_groups = std::max(big.ngroups, c->planZY.ngroups);
    }
    TRY(dalloc(c, &c->tcpart, (long long)c->tc_max_groups * c->planZY.ntiles * 128 * 128));
    if (S.big && c->opt.tc_solve) {
      // BF16x3 planes of the trailing factor block and of the finished rows
      // of Z_d for the tensor-core block updates; padding stays zero
      const size_t tb = tcs_planes_bytes((int)N, S.nd, (int)nu);
      unsigned char *tp = nullptr;
      TRY(dalloc(c, &tp, (tb + 255) / 256 * 256));
      CK(cudaMemset(tp, 0, tb));
      if (!tcs_plan(c->tcs, (int)N, S.nd, (int)nu, tp))
        return fail(c, IPM_ERR_CUDA, "tensor maps of the tensor-core block solve");
      c->tcs_on = true;
    }
    TRY(dalloc(c, &c->pcg_b, nu)); TRY(dalloc(c, &c->pcg_r, nu)); TRY(dalloc(c, &c->pcg_z, nu));
    TRY(dalloc(c, &c->pcg_p, nu)); TRY(dalloc(c, &c->pcg_Ap, nu));
  }
  // GEMM tiling: upper tiles, scenario groups
  c->nt1 = (int)((nu + 63) / 64);
  std::vector<int2> tl;
  std::vector<int> tof((size_t)c->nt1 * c->nt1, -1);
  for (int i = 0; i < c->nt1; ++i)
    for (int j = i; j < c->nt1; ++j) {
      tof[(size_t)i * c->nt1 + j] = (int)tl.size();
      tl.push_back(make_int2(i, j));
    }
  c->ntiles = (int)tl.size();
  // split the N*nx contraction rows into equal chunks so that tiles x chunks
  // fills one wave (3 CTAs of 256 threads per SM, 152 SMs); the buffer of
  // partial tiles has room for the autotuner's largest candidate (4x)
  {
    const long long G0 = std::max(1, (3 * 152) / c->ntiles);
    set_groups(c, 4 * G0);
    c->max_groups = c->ngroups;
    set_groups(c, G0);
  }
  c->zs_threads = (c->opt.solve_threads == 128 || c->opt.solve_threads == 256) ? c->opt.solve_threads : 256;
  TRY(dalloc(c, &c->tiles, tl.size()));
  CK(cudaMemcpy(c->tiles, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice));
  TRY(dalloc(c, &c->tile_of, tof.size()));
  CK(cudaMemcpy(c->tile_of, tof.data(), tof.size() * sizeof(int), cudaMemcpyHostToDevice));
  TRY(dalloc(c, &c->partial, (long long)c->max_groups * c->ntiles * 4096));
  TRY(dalloc(c, &c->Khat, nu * nu)); TRY(dalloc(c, &c->M, nu * nu)); TRY(dalloc(c, &c->F, nu * nu));
  TRY(dalloc(c, &c->diag1, nu)); TRY(dalloc(c, &c->rhs_u, nu));
  TRY(dalloc(c, &c->rhs_corr, nu)); TRY(dalloc(c, &c->cpos, N * std::max(nx, nu)));
  TRY(dalloc(c, &c->gLu, nu)); TRY(dalloc(c, &c->HTt_u, nu));
  {
    std::vector<double> pgc(nu, 0.0);
    for (int k = 1; k < S.ng; ++k) pgc[S.ng + k - 1] = 2.0 * S.c2[k];
    const double *tmp = nullptr;
    TRY(upload(c, &tmp, pgc));
    c->pg_curv = const_cast<double *>(tmp);
    TRY(upload(c, &tmp, S.pmax));
    c->pmax_d = const_cast<double *>(tmp);
  }
  TRY(dalloc(c, &c->step, c->step_len));
  c->px = c->step;
  c->pu = c->px + N * nx;
  c->ps = c->pu + nu;
  c->py = c->ps + N * m;
  c->pz = c->py + N * nx;
  for (int i = 0; i < 6; ++i) {
    long long len = (i < 2) ? N * nx : (i < 4 ? nu : N * m);
    TRY(dalloc(c, &c->dz[i], len));
  }
  TRY(dalloc(c, &c->Hp, N * m)); TRY(dalloc(c, &c->kpx, N * nx)); TRY(dalloc(c, &c->kpu, N * nu));
  if (c->opt.aug_refine > 0) {
    TRY(dalloc(c, &c->ar1x, N * nx)); TRY(dalloc(c, &c->ar3, N * nx)); TRY(dalloc(c, &c->ar1u, nu));
    TRY(dalloc(c, &c->ar2, N * m)); TRY(dalloc(c, &c->ar4, N * m)); TRY(dalloc(c, &c->atw, N * m));
    TRY(dalloc(c, &c->dstep, c->step_len));
    c->dpx = c->dstep;
    c->dpu = c->dpx + N * nx;
    c->dps = c->dpu + nu;
    c->dpy = c->dps + N * m;
    c->dpz = c->dpy + N * nx;
    TRY(dalloc(c, &c->arh1x, N * nx)); TRY(dalloc(c, &c->arh2, nu)); TRY(dalloc(c, &c->arhs, nu));
    TRY(dalloc(c, &c->apos2, N * nx)); TRY(dalloc(c, &c->bpos2, N * nx)); TRY(dalloc(c, &c->vpos2, N * nx));
    TRY(dalloc(c, &c->amax, 2));
    TRY(dalloc(c, &c->aupart, N * nu)); TRY(dalloc(c, &c->aumag, N * nu));
    CK(cudaMallocHost(&c->h_amax, 2 * sizeof(unsigned long long)));
  }
  TRY(dalloc(c, &c->vpos, N * nx)); TRY(dalloc(c, &c->bpos, N * nx)); TRY(dalloc(c, &c->apos, N * nx));
  TRY(dalloc(c, &c->xt, N * nx)); TRY(dalloc(c, &c->ut, nu)); TRY(dalloc(c, &c->st, N * m));
  TRY(dalloc(c, &c->gt, N * nx)); TRY(dalloc(c, &c->ht, N * m)); TRY(dalloc(c, &c->fst, N));
  TRY(dalloc(c, &c->Pt, N * n)); TRY(dalloc(c, &c->Qt, N * n));
  TRY(dalloc(c, &c->red_partial, 152 * 8)); TRY(dalloc(c, &c->red_out, 16));
  CK(cudaMallocHost(&c->h_red, 16 * sizeof(double)));
  CK(cudaMallocHost(&c->h_flags, FLAG_COUNT * sizeof(int)));
  CK(cudaMallocHost(&c->h_mu, sizeof(double)));
  TRY(dalloc(c, &c->d_mu, 1));
  // first-stage diagonal terms of K_hat that do not depend on the iterate
  // (cost curvature of the non-slack generators); Sigma_u is added per call
  long long nb = 0;
  for (int j = 0; j < S.nx; ++j) nb += (std::isfinite(S.xl[j]) ? 1 : 0) + (std::isfinite(S.xu[j]) ? 1 : 0);
  nb *= N;
  for (int j = 0; j < S.nu; ++j) nb += (std::isfinite(S.ul[j]) ? 1 : 0) + (std::isfinite(S.uu[j]) ? 1 : 0);
  long long nbs = 0;
  for (int j = 0; j < S.m; ++j) nbs += (std::isfinite(S.sl[j]) ? 1 : 0) + (std::isfinite(S.su[j]) ? 1 : 0);
  nb += nbs * N;
  c->n_bounds = nb;
  return IPM_OK;
}

ipm_status read_red(ipm_ctx *c, int nv, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->h_red, c->red_out, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}


// the tensor-core block-solve plan of a mixed context, or null
inline const TcsPlan *tcs_of(const ipm_ctx *c) { return c->tcs_on ? &c->tcs : nullptr; }

enum { PH_EVAL = 0, PH_COND, PH_LU, PH_ZSOLVE, PH_GEMM, PH_RRHS, PH_CHOL, PH_RECOVER, PH_LS, PH_SPLIT,
       PH_FALLBACK, PH_SOLVE1 };

// accumulate one finished phase (waits for its end event)
void ph_take(ipm_ctx *c, int p) {
  if (!c->ev_pending[p]) return;
  float ms = 0.f;
  cudaEventSynchronize(c->ev[2 * p + 1]);
  if (cudaEventElapsedTime(&ms, c->ev[2 * p], c->ev[2 * p + 1]) == cudaSuccess) {
    c->t_ms[p] += ms;
    c->t_cnt[p] += 1;
  }
  c->ev_pending[p] = false;
}
// A mixed-path iteration condensed again in FP64 is timed as one phase of its
// own (fallback); its inner phases are not added to the mixed path's.
inline bool ph_skip(const ipm_ctx *c, int p) { return !c->prof || (c->mixed && c->exact_iter && p != PH_FALLBACK); }
inline void ph_begin(ipm_ctx *c, int p, cudaStream_t st) {
  if (ph_skip(c, p)) return;
  ph_take(c, p);  // a phase met again in the same iteration (inertia trials, solves)
  cudaEventRecord(c->ev[2 * p], st);
}
inline void ph_end(ipm_ctx *c, int p, cudaStream_t st) {
  if (ph_skip(c, p)) return;
  cudaEventRecord(c->ev[2 * p + 1], st);
  c->ev_pending[p] = true;
}
// accumulate finished phases (call after a stream synchronisation)
void ph_collect(ipm_ctx *c) {
  if (!c->prof) return;
  for (int p = 0; p < IPM_N_PHASES; ++p) ph_take(c, p);
}

// one vector per scenario through G_x (trans 0) or G_x^T (trans 1) on the
// main stream, timed as the solve1 phase (nested in the phase it serves)
void solve1(ipm_ctx *c, double *v, int trans, cudaStream_t st) {
  ph_begin(c, PH_SOLVE1, st);
  launch_solve1(c->ds, c->dw.LU, c->dw.rd, v, trans, st);
  ph_end(c, PH_SOLVE1, st);
}

ipm_status read_flags(ipm_ctx *c, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->h_flags, c->dw.flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}

ipm_status write_scalars(ipm_ctx *c, cudaStream_t st) {
  c->h_red[8] = c->mu;
  c->h_red[9] = c->rho;
  c->h_red[10] = c->delta_last;
  CK(cudaMemcpyAsync(c->dw.scal, c->h_red + 8, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}

ipm_status read_scalars(ipm_ctx *c, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->h_red + 8, c->dw.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  c->mu = c->h_red[8];
  c->rho = c->h_red[9];
  c->delta_last = c->h_red[10];
  return IPM_OK;
}

// f, g, h at (x, u); J, W, J^T lambda at (x, u, y, z)
ipm_status do_eval(ipm_ctx *c, cudaStream_t st) {
  DevWork &D = c->dw;
  ph_begin(c, PH_EVAL, st);
  launch_functions(c->ds, D.x, D.u, D.P, D.Q, D.g, D.h, D.fs, st);
  launch_derivatives(c->ds, D, st);
  launch_ugrad(c->ds, D, c->gLu, st);
  ph_end(c, PH_EVAL, st);
  CK(cudaGetLastError());
  c->have_eval = true;
  c->have_cond = c->have_fact = false;
  return IPM_OK;
}

// optimality error pieces -> c->errs (dual, primal, compl max, compl min, s_d, s_c)
ipm_status do_errors(ipm_ctx *c, cudaStream_t st) {
  launch_errors(c->ds, c->dw, c->gLu, c->red_partial, c->red_out, st);
  TRY(read_red(c, 7, st));
  c->mean_compl = c->h_red[6] / std::max(1.0, (double)c->n_bounds);
  const Sym &S = c->S;
  const double nlam = (double)S.N * (S.nx + S.m);
  const double nb = (double)c->n_bounds;
  c->errs[0] = c->h_red[0];
  c->errs[1] = c->h_red[1];
  c->errs[2] = c->h_red[2];
  c->errs[3] = c->h_red[3];
  c->errs[4] = std::max(S_MAX, (c->h_red[4] + c->h_red[5]) / (nlam + nb)) / S_MAX;
  c->errs[5] = std::max(S_MAX, c->h_red[5] / nb) / S_MAX;
  return IPM_OK;
}

// Runs fn (a sequence of launches on st) directly, or as a CUDA graph that
// is captured the first time: every launch parameter of a context is fixed
// after its first condensation (the barrier parameter is read from device
// memory), so one capture per part serves every later iteration.  A capture
// the driver refuses leaves the context on direct launches.
template <class Fn>
ipm_status run_part(ipm_ctx *c, cudaGraphExec_t &gx, long long &gn, Fn fn, cudaStream_t st) {
  if (!c->opt.graphs || c->prof || st == nullptr || c->graph_failed) {
    fn();
    return IPM_OK;
  }
  if (!gx) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      c->graph_failed = true;
      fn();
      return IPM_OK;
    }
    const long long n0 = t_ipm_launches;
    fn();
    const long long n = t_ipm_launches - n0;
    g_ipm_launches -= n;  // captured, not launched
    const cudaError_t le = cudaGetLastError();  // a launch the capture refused
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return fail(c, IPM_ERR_CUDA, "kernel launch while capturing the condensation", le);
    }
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&gx, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || !gx) {
      cudaGetLastError();
      gx = nullptr;
      c->graph_failed = true;
      fn();
      return IPM_OK;
    }
    gn = n;
  }
  CK(cudaGraphLaunch(gx, st));
  g_ipm_launches += gn;
  return IPM_OK;
}

// K_hat by the paper's adjoint solves (after the multi-RHS solve left Y, Y_u):
// the n_u columns of L_x = Y as vectors, G_x^{-T} on each (one CTA per
// vector), then K_hat = sum_i (Y_u,i - G_u^T W_i) + first-stage diagonal
void launch_adjoint_reduce(ipm_ctx *c, cudaStream_t st) {
  const DevSym &S = c->ds;
  launch_transpose_rows(S.N, S.nx, S.nu, c->Y, c->Wadj, st);
  launch_solve1_batched(S, c->dw.LU, c->dw.rd, c->Wadj, 1, S.nu, 128, st);
  launch_adjoint_assemble(S, c->dw.J, c->Yu, c->Wadj, c->diag1, c->Khat, st);
}

// K_hat contraction of the FP64 branch: partial tiles over ngroups scenario
// groups (the multi-instance runner may take it over through the hook)
void fp64_contraction(ipm_ctx *c, cudaStream_t st) {
  const DevSym &S = c->ds;
  if (c->emu) launch_emu_schur(c->emuZY, c->emupart, c->dw.flags, st);
  else if (c->gemm_hook) c->gemm_hook(c->gemm_hook_arg, c, st);
  else launch_gemm_tn64((long long)S.N * S.nx, c->kchunk, S.nu, c->ngroups, c->Z, c->Y, c->tiles, c->ntiles,
                        c->partial, st);
}

// split the N*nx contraction rows into G chunks (a multiple of 16 rows each)
void set_groups(ipm_ctx *c, long long G) {
  const long long krows = (long long)c->S.N * c->S.nx;
  G = std::max(1LL, std::min(G, (krows + 15) / 16));
  long long kc = (krows + G - 1) / G;
  kc = (kc + 15) / 16 * 16;
  c->kchunk = kc;
  c->ngroups = (int)((krows + kc - 1) / kc);
}

struct Tuned {
  int zs_threads;
  long long kchunk;
  int ngroups, tc_groups;
  bool adjoint;
};
void launch_adjoint_reduce(ipm_ctx *c, cudaStream_t st);
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, Tuned> g_tune_cache;

// milliseconds of fn on st (events; fn's outputs are overwritten by the caller's next run)
// (a candidate whose launch fails reports +infinity and is not chosen)
template <class Fn>
double time_ms(Fn fn, cudaStream_t st, int reps = 2) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();  // warm
  cudaEventRecord(a, st);
  for (int r = 0; r < reps; ++r) fn();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaGetLastError() != cudaSuccess) return std::numeric_limits<double>::infinity();
  return ms / reps;
}

// Autotuner: after the first pre-contraction part has run (so LU, J, K hold
// real values), time the candidate launch shapes of the multi-RHS solves and
// of the reduced-Hessian contraction and keep the fastest.  Each candidate
// recomputes the same quantities (the solves are identical for every thread
// count; the contraction's rounding depends on the group split, and the
// chosen split is the one run last).
ipm_status autotune(ipm_ctx *c, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const auto key = std::make_tuple(S.nx, S.nu, S.N, (c->mixed ? 1 : (c->emu ? 2 : 0)) + 4 * c->opt.reduction);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->zs_threads = it->second.zs_threads;
      c->kchunk = it->second.kchunk;
      c->ngroups = it->second.ngroups;
      if (c->opt.reduction == IPM_REDUCTION_AUTO && !c->mixed) {
        c->adjoint = it->second.adjoint;
        if (c->adjoint) launch_adjoint_reduce(c, st);  // K_hat of this first condensation
      }
      if (c->emu) {
        emu_regroup(c->emuZY, it->second.tc_groups);
        emu_regroup(c->emuZZ, it->second.tc_groups);
      }
      if (c->mixed) {
        tc_regroup(c->planZY, it->second.tc_groups);
        tc_regroup(c->planZZ, it->second.tc_groups);
      }
      c->tuned = true;
      return IPM_OK;
    }
  }
  const bool fp64 = !c->mixed;
  double best = 1e300;
  int best_thr = 256;
  for (int thr : {128, 256}) {
    const double ms = fp64 ? time_ms([&] { launch_zsolve64(S, D.LU, D.rd, D.J, D.K, c->Z, c->Y, c->Yu, st, thr); }, st)
                           : time_ms([&] { launch_zsolve32(S, D.LU, D.rd, D.J, D.K, c->Z32, c->Y32, c->Yu, st, thr, tcs_of(c), D.flags); }, st);
    c->tune_ms[thr == 128 ? 0 : 1] = ms;
    if (ms < best) best = ms, best_thr = thr;
  }
  c->zs_threads = best_thr;
  // the solve outputs are identical for every thread count; rerun the winner
  // so that the mixed planes are split from them below
  if (fp64) {
    launch_zsolve64(S, D.LU, D.rd, D.J, D.K, c->Z, c->Y, c->Yu, st, best_thr);
  } else {
    launch_zsolve32(S, D.LU, D.rd, D.J, D.K, c->Z32, c->Y32, c->Yu, st, best_thr, tcs_of(c), D.flags);
    launch_split_t((long long)S.N * S.nx, S.nu, c->planZY.kpad, c->Z32, c->zpl, st);
    launch_split_t((long long)S.N * S.nx, S.nu, c->planZY.kpad, c->Y32, c->ypl, st);
  }
  int tc_groups = 0;
  if (fp64 && c->emu) {
    const int G0 = std::max(1, 152 / c->emuZY.ntiles);
    int bestG = G0;
    best = 1e300;
    int slot = 2;
    for (int G : {G0 / 2, G0, 2 * G0}) {
      if (G < 1) continue;
      EmuPlan trial = c->emuZY;
      emu_regroup(trial, G);
      if (trial.ngroups > c->emu_max_groups) continue;
      c->emuZY = trial;
      const double ms = time_ms([&] { launch_emu_schur(c->emuZY, c->emupart, D.flags, st); }, st);
      if (slot < 8) c->tune_ms[slot++] = ms;
      if (ms < best) best = ms, bestG = G;
    }
    emu_regroup(c->emuZY, bestG);
    emu_regroup(c->emuZZ, bestG);
    tc_groups = bestG;
  } else if (fp64) {
    const long long G0 = std::max(1, (3 * 152) / c->ntiles);
    long long bestG = G0;
    best = 1e300;
    int slot = 2;
    for (long long G : {G0 / 2, G0, 2 * G0, 4 * G0}) {
      if (G < 1 || G > c->max_groups) continue;
      set_groups(c, G);
      if (c->ngroups > c->max_groups) continue;
      const double ms = time_ms([&] {
        launch_gemm_tn64((long long)S.N * S.nx, c->kchunk, S.nu, c->ngroups, c->Z, c->Y, c->tiles, c->ntiles,
                         c->partial, st);
      }, st);
      if (slot < 8) c->tune_ms[slot++] = ms;
      if (ms < best) best = ms, bestG = G;
    }
    set_groups(c, bestG);
  } else {
    const int G0 = std::max(1, 152 / c->planZY.ntiles);
    int bestG = G0;
    best = 1e300;
    int slot = 2;
    for (int G : {G0 / 2, G0, 2 * G0}) {
      if (G < 1 || G > c->tc_max_groups) continue;
      tc_regroup(c->planZY, G);
      const double ms = time_ms([&] { launch_tc_schur(c->planZY, c->tcpart, D.flags, st); }, st);
      if (slot < 8) c->tune_ms[slot++] = ms;
      if (ms < best) best = ms, bestG = G;
    }
    tc_regroup(c->planZY, bestG);
    tc_regroup(c->planZZ, bestG);
    tc_groups = bestG;
  }
  // the paper's adjoint-solve reduction against the dense contraction (split,
  // contraction and assembly of K_hat), both from the same Z, Y, Y_u
  if (fp64 && c->opt.reduction == IPM_REDUCTION_AUTO) {
    const double md = time_ms([&] {
      if (c->emu) {
        launch_emu_split_pair(c->emuZY, c->Z, c->Y, nullptr, st, c->emu_rs);
        launch_emu_schur(c->emuZY, c->emupart, D.flags, st);
        launch_emu_assemble(c->emuZY, S.N, c->emupart, c->Yu, c->diag1, c->Khat, st);
      } else {
        launch_gemm_tn64((long long)S.N * S.nx, c->kchunk, S.nu, c->ngroups, c->Z, c->Y, c->tiles, c->ntiles,
                         c->partial, st);
        launch_khat_assemble(S.nu, S.N, c->ngroups, c->ntiles, c->nt1, c->partial, c->tile_of, c->Yu, c->diag1,
                             c->Khat, st);
      }
    }, st);
    const double ma = time_ms([&] { launch_adjoint_reduce(c, st); }, st);
    c->tune_ms[6] = md;
    c->tune_ms[7] = ma;
    c->adjoint = ma < md;
    // the adjoint K_hat is in place now; the dense one is formed next by
    // the caller's contraction
  }
  CK(cudaGetLastError());
  c->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune_cache[key] = Tuned{c->zs_threads, c->kchunk, c->ngroups, tc_groups, c->adjoint};
  return IPM_OK;
}

// the stream st waits for a p_y solve left on the side stream
void join_py(ipm_ctx *c, cudaStream_t st) {
  if (!c->py_pending) return;
  cudaStreamWaitEvent(st, c->ev_join, 0);
  c->py_pending = false;
}

// Reduced right-hand side, eq. (11), FP64 path: with b = G_x^{-1} r3 and
// Z = -G_x^{-1} G_u,
//   rhs_u = -rhat2 - sum_i Z_i^T (rhat1_i - K_xx b_i) + K_ux b_i
// (b came with Z from the multi-RHS solve when the trailing block fits in
// shared memory).  Needs only the solve's outputs, so it runs on the side
// stream next to the split and the contraction.
void reduced_rhs_fp64(ipm_ctx *c, cudaStream_t s2) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  ph_begin(c, PH_RRHS, s2);
  if (!zsolve64_folds_b(S)) {
    launch_gather_pos(S.N, S.nx, S.iperm, D.g, c->bpos, 1.0, s2);
    launch_solve1(S, D.LU, D.rd, c->bpos, 0, s2);
  }
  launch_kapply(S, D.K, c->bpos, nullptr, c->kpx, nullptr, s2);
  launch_gather_pos(S.N, S.nx, S.iperm, D.rh1x, c->apos, 1.0, s2);
  launch_lincomb((long long)S.N * S.nx, c->apos, 1.0, c->apos, -1.0, c->kpx, 0.0, nullptr, s2);
  launch_lincomb(S.nu, c->rhs_u, -1.0, D.rh2, 0.0, nullptr, 0.0, nullptr, s2);
  launch_zt_apply(S, c->Z, c->apos, D.K, c->bpos, -1.0, 1.0, c->rhs_u, c->cpos, s2);
  ph_end(c, PH_RRHS, s2);
}

// Sigma, K, LU(G_x), Z, Y, K_hat (delta = 0), reduced right-hand side
ipm_status ensure_side(ipm_ctx *c) {
  if (c->side) return IPM_OK;
  CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming));
  return IPM_OK;
}

ipm_status do_condense(ipm_ctx *c, cudaStream_t st) {
  join_py(c, st);
  TRY(ensure_side(c));
  if (!c->have_eval) return fail(c, IPM_ERR_STATE, "condense before eval");
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const bool fp64 = !c->mixed || c->exact_iter;
  const int br = fp64 ? 0 : 1;
  *c->h_mu = c->mu;
  CK(cudaMemcpyAsync(c->d_mu, c->h_mu, sizeof(double), cudaMemcpyHostToDevice, st));
  auto pre = [&] {
    ph_begin(c, PH_COND, st);
    launch_sigmas(S, D, st);
    launch_condense(S, D, st);
    launch_rhs(S, D, c->d_mu, c->gLu, c->HTt_u, st);
    ph_end(c, PH_COND, st);
    cudaMemsetAsync(D.flags, 0, FLAG_COUNT * sizeof(int), st);
    ph_begin(c, PH_LU, st);
    launch_lu_factor(S, c->nL, D.J, D.LU, D.rd, D.flags, st, c->opt.lu_pair != 0, c->emu_lu_on ? &c->emu_lu : nullptr);
    ph_end(c, PH_LU, st);
    // first-stage diagonal of K_hat: Sigma_u + 2 c2_k on the non-slack Pg entries
    launch_lincomb(S.nu, c->diag1, 1.0, D.Su, 1.0, c->pg_curv, 0.0, nullptr, st);
    ph_begin(c, PH_ZSOLVE, st);
    // FP64: b = G_x^{-1} g of eq. (11) rides along as an extra right-hand side
    if (fp64 && c->emu)
      cudaMemsetAsync(c->emu_rs, 0, 2 * (size_t)S.N * S.nx * sizeof(int), st);  // row exponent maxima
    if (fp64)
      launch_zsolve64(S, D.LU, D.rd, D.J, D.K, c->Z, c->Y, c->Yu, st, c->zs_threads, D.g, c->bpos,
                      c->emu ? c->emu_rs : nullptr);
    else launch_zsolve32(S, D.LU, D.rd, D.J, D.K, c->Z32, c->Y32, c->Yu, st, c->zs_threads, tcs_of(c), D.flags);
    ph_end(c, PH_ZSOLVE, st);
    if (fp64) {
      // the reduced right-hand side needs Z and b only: on the side stream,
      // under the split and the contraction's set-up
      cudaEventRecord(c->ev_fork2, st);
      cudaStreamWaitEvent(c->side2, c->ev_fork2, 0);
      reduced_rhs_fp64(c, c->side2);
      cudaEventRecord(c->ev_join2, c->side2);
    }
    if (fp64 && c->adjoint) {
      // §3.2 local reduction, step 3 for V = I: K_hat = sum_i (L_u - G_u^T G_x^{-T} L_x)
      ph_begin(c, PH_GEMM, st);
      launch_adjoint_reduce(c, st);
      ph_end(c, PH_GEMM, st);
      cudaStreamWaitEvent(st, c->ev_join2, 0);
      return;
    }
    ph_begin(c, PH_SPLIT, st);
    if (fp64 && c->emu) {
      // exact BF16 slices of the row-balanced Z and Y for the tensor cores
      // (row shifts from the row exponent maxima the solve left in emu_rs)
      launch_emu_split_pair(c->emuZY, c->Z, c->Y, nullptr, st, c->emu_rs);
    } else if (!fp64) {
      // mixed: BF16x3 planes of the FP32 Z and Y
      launch_split_t((long long)S.N * S.nx, S.nu, c->planZY.kpad, c->Z32, c->zpl, st);
      launch_split_t((long long)S.N * S.nx, S.nu, c->planZY.kpad, c->Y32, c->ypl, st);
    }
    ph_end(c, PH_SPLIT, st);
    if (fp64) cudaStreamWaitEvent(st, c->ev_join2, 0);
  };
  auto post = [&] {
    if (fp64) {
      if (c->emu) launch_emu_assemble(c->emuZY, S.N, c->emupart, c->Yu, c->diag1, c->Khat, st);
      else launch_khat_assemble(S.nu, S.N, c->ngroups, c->ntiles, c->nt1, c->partial, c->tile_of, c->Yu, c->diag1,
                                c->Khat, st);
      ph_end(c, PH_GEMM, st);
    } else {
      launch_tc_assemble(c->planZY, S.N, c->tcpart, c->Yu, c->diag1, c->Khat, st);
      ph_end(c, PH_GEMM, st);
      ph_begin(c, PH_RRHS, st);
      // eq. (11) with FP64 solves: b = G_x^{-1} r3, a = G_x^{-T}(rhat1 - K_xx b)
      launch_gather_pos(S.N, S.nx, S.iperm, D.g, c->bpos, 1.0, st);
      solve1(c, c->bpos, 0, st);
      launch_kapply(S, D.K, c->bpos, nullptr, c->kpx, nullptr, st);
      launch_gather_pos(S.N, S.nx, S.iperm, D.rh1x, c->apos, 1.0, st);
      launch_lincomb((long long)S.N * S.nx, c->apos, 1.0, c->apos, -1.0, c->kpx, 0.0, nullptr, st);
      solve1(c, c->apos, 1, st);
      launch_rhs_reduced(S, D.J, D.K, D.rh2, c->apos, c->bpos, c->rhs_u, st);
      ph_end(c, PH_RRHS, st);
    }
  };
  if (c->opt.autotune && !c->tuned) {
    pre();  // direct launches: the tuned shapes must be fixed before a graph is captured
    TRY(autotune(c, st));
  } else {
    TRY(run_part(c, c->gx_pre[br], c->gx_pre_n[br], pre, st));
  }
  if (!(fp64 && c->adjoint)) {
    ph_begin(c, PH_GEMM, st);
    if (fp64) fp64_contraction(c, st);
    else launch_tc_schur(c->planZY, c->tcpart, D.flags, st);
    TRY(run_part(c, c->gx_post[br], c->gx_post_n[br], post, st));
  }
  CK(cudaGetLastError());
  TRY(read_flags(c, st));
  ph_collect(c);
  if (c->h_flags[FLAG_SINGULAR]) return fail(c, IPM_ERR_SINGULAR_GX, "singular pivot in the LU of G_x");
  if (c->h_flags[FLAG_TIMEOUT]) return fail(c, IPM_ERR_TIMEOUT, "a bounded device wait gave up");
  if (c->emu_lu_on && c->h_flags[FLAG_NONFINITE]) {
    // a non-finite value from the tensor-core LU update (or the contraction):
    // factor on the FP64 units from now on and condense again
    c->emu_lu_on = false;
    for (int b = 0; b < 2; ++b) {
      if (c->gx_pre[b]) cudaGraphExecDestroy(c->gx_pre[b]);
      if (c->gx_post[b]) cudaGraphExecDestroy(c->gx_post[b]);
      c->gx_pre[b] = c->gx_post[b] = nullptr;
    }
    CK(cudaMemsetAsync(D.flags, 0, FLAG_COUNT * sizeof(int), st));
    return do_condense(c, st);
  }
  if (fp64 && c->emu && !c->adjoint && c->h_flags[FLAG_NONFINITE]) {
    // the emulated contraction gave a non-finite value: redo it on the FP64 units
    ++c->n_emu_fallback;
    launch_gemm_tn64((long long)S.N * S.nx, c->kchunk, S.nu, c->ngroups, c->Z, c->Y, c->tiles, c->ntiles,
                     c->partial, st);
    launch_khat_assemble(S.nu, S.N, c->ngroups, c->ntiles, c->nt1, c->partial, c->tile_of, c->Yu, c->diag1,
                         c->Khat, st);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(D.flags + FLAG_NONFINITE, 0, sizeof(int), st));
  }
  c->have_cond = true;
  c->have_fact = false;
  c->M_valid = false;
  return IPM_OK;
}

ipm_status do_factor(ipm_ctx *c, double delta, int *is_pd, cudaStream_t st, double tau = 0.0) {
  if (!c->have_cond) return fail(c, IPM_ERR_STATE, "factor before condense");
  const DevSym &S = c->ds;
  if (delta != 0.0 && !c->M_valid) {
    // M = sum_i Z_i^T Z_i, so that K_hat(K + delta I) = K_hat(K) + delta (M + I);
    // eq. (11) contains K_xx: with K_xx + delta I the reduced right-hand side
    // gains -delta sum_i G_u^T G_x^{-T} b_i = delta sum_i Z_i^T b_i
    if (!c->mixed || c->exact_iter) {
      bool done = false;
      if (c->emu) {
        CK(cudaMemsetAsync(c->dw.flags + FLAG_NONFINITE, 0, sizeof(int), st));
        // Z^T Z: both operands from one unbalanced split of Z (K_hat is done,
        // so the balanced planes are no longer needed)
        launch_emu_split(c->emuZZ, c->Z, false, nullptr, st);
        launch_emu_schur(c->emuZZ, c->emupart, c->dw.flags, st);
        launch_emu_assemble(c->emuZZ, S.N, c->emupart, nullptr, nullptr, c->M, st);
        TRY(read_flags(c, st));
        done = !c->h_flags[FLAG_NONFINITE];
        if (!done) ++c->n_emu_fallback;
      }
      if (!done) {
        launch_gemm_tn64((long long)S.N * S.nx, c->kchunk, S.nu, c->ngroups, c->Z, c->Z, c->tiles, c->ntiles,
                         c->partial, st);
        launch_khat_assemble(S.nu, S.N, c->ngroups, c->ntiles, c->nt1, c->partial, c->tile_of, nullptr, nullptr,
                             c->M, st);
      }
      launch_zt_apply(S, c->Z, c->bpos, nullptr, nullptr, 1.0, 0.0, c->rhs_corr, c->cpos, st);
    } else {
      launch_tc_schur(c->planZZ, c->tcpart, c->dw.flags, st);
      launch_tc_assemble(c->planZZ, S.N, c->tcpart, nullptr, nullptr, c->M, st);
      CK(cudaMemcpyAsync(c->cpos, c->bpos, (size_t)S.N * S.nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
      solve1(c, c->cpos, 1, st);
      launch_gut_sum(S, c->dw.J, c->cpos, -1.0, c->rhs_corr, st);
    }
    c->M_valid = true;
  }
  ph_begin(c, PH_CHOL, st);
  launch_shift(S.nu, c->Khat, c->M, delta, tau, c->F, st);
  CK(cudaMemsetAsync(c->dw.flags + FLAG_NOT_PD, 0, sizeof(int), st));
  launch_cholesky(S.nu, c->F, c->dw.flags, st);
  ph_end(c, PH_CHOL, st);
  CK(cudaGetLastError());
  TRY(read_flags(c, st));
  ph_collect(c);
  *is_pd = c->h_flags[FLAG_NOT_PD] ? 0 : 1;
  c->have_fact = *is_pd != 0;
  c->delta_fact = delta;
  return IPM_OK;
}

// Exact FP64 product of the reduced matrix of K + delta I with v (matrix-free,
// Prop. 2.3): w_i = -G_x^{-1} G_u v, then
// out = sum_i [ -G_u^T G_x^{-T}((K_xx + delta) w_i + K_xu v) + K_ux w_i + K_uu^i v ] + (diag1 + delta) v
ipm_status reduced_apply(ipm_ctx *c, const double *v, double *out, double delta, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const long long NX = (long long)S.N * S.nx;
  CK(cudaMemsetAsync(c->vpos, 0, NX * sizeof(double), st));
  launch_gu_apply(S, D.J, v, c->vpos, st);
  solve1(c, c->vpos, 0, st);
  launch_lincomb(NX, c->vpos, -1.0, c->vpos, 0.0, nullptr, 0.0, nullptr, st);
  launch_kapply(S, D.K, c->vpos, v, c->kpx, c->kpu, st);
  launch_lincomb(NX, c->apos, 1.0, c->kpx, delta, c->vpos, 0.0, nullptr, st);
  solve1(c, c->apos, 1, st);
  launch_gut_sum(S, D.J, c->apos, -1.0, out, st);
  launch_apply_finish(S, c->kpu, c->diag1, delta, v, out, st);
  return IPM_OK;
}

// p_u of the reduced system eq. (11) to FP64 accuracy: conjugate gradients on
// the exact operator, preconditioned by the Cholesky factor of the BF16x3
// K_hat; c->pu holds the right-hand side on entry and the solution on exit.
ipm_status pcg_reduced(ipm_ctx *c, double delta, cudaStream_t st) {
  const int nu = c->ds.nu;
  double *x = c->pu, *b = c->pcg_b, *r = c->pcg_r, *z = c->pcg_z, *p = c->pcg_p, *Ap = c->pcg_Ap;
  c->neg_curv = false;
  CK(cudaMemcpyAsync(b, x, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_chol_solve(nu, c->F, x, st);
  TRY(reduced_apply(c, x, Ap, delta, st));
  launch_lincomb(nu, r, 1.0, b, -1.0, Ap, 0.0, nullptr, st);
  CK(cudaMemcpyAsync(z, r, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_chol_solve(nu, c->F, z, st);
  CK(cudaMemcpyAsync(p, z, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_dot2(nu, r, z, b, b, c->red_out, st);
  TRY(read_red(c, 2, st));
  double rz = c->h_red[0];
  const double bnorm = std::sqrt(std::max(c->h_red[1], 1e-300));
  launch_dot2(nu, r, r, nullptr, nullptr, c->red_out, st);
  TRY(read_red(c, 1, st));
  double res = std::sqrt(c->h_red[0]) / bnorm;
  int it = 0;
  for (; it < c->opt.max_refine && res > 1e-13 && rz > 0.0; ++it) {
    TRY(reduced_apply(c, p, Ap, delta, st));
    launch_dot2(nu, p, Ap, p, p, c->red_out, st);
    TRY(read_red(c, 2, st));
    const double pAp = c->h_red[0];
    if (!(pAp > 0.0)) {
      c->neg_curv = true;
      c->curv_q = c->h_red[1] > 0.0 ? pAp / c->h_red[1] : 0.0;
      break;
    }
    const double alpha = rz / pAp;
    launch_lincomb(nu, x, 1.0, x, alpha, p, 0.0, nullptr, st);
    launch_lincomb(nu, r, 1.0, r, -alpha, Ap, 0.0, nullptr, st);
    CK(cudaMemcpyAsync(z, r, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_chol_solve(nu, c->F, z, st);
    launch_dot2(nu, r, z, r, r, c->red_out, st);
    TRY(read_red(c, 2, st));
    const double rz_new = c->h_red[0];
    res = std::sqrt(c->h_red[1]) / bnorm;
    launch_lincomb(nu, p, 1.0, z, rz_new / rz, p, 0.0, nullptr, st);
    rz = rz_new;
  }
  c->refine_iters = it;
  c->refine_res = res;
  return IPM_OK;
}

// Backward error of the step (c->px .. c->pz) on the augmented system eq. (6):
// rho = -r - A p, returns max|rho| over the largest magnitude among r and
// the block products A_blk p_blk (read back).  Leaves
// kpx, kpu = K p_d (positions) and Hp = H p_d of this step, which the line
// search reads, and rho in ar1x .. ar4.
ipm_status aug_residual(ipm_ctx *c, double delta, double *rel, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  launch_gather_pos(S.N, S.nx, S.iperm, c->px, c->vpos, 1.0, st);
  launch_kapply(S, D.K, c->vpos, c->pu, c->kpx, c->kpu, st);
  CK(cudaMemsetAsync(c->amax, 0, 2 * sizeof(unsigned long long), st));
  launch_aug_residual(S, D, delta, c->px, c->pu, c->ps, c->py, c->pz, c->kpx, c->kpu, c->diag1, c->Hp, c->atw,
                      c->ar1x, c->ar1u, c->ar2, c->ar3, c->ar4, c->aupart, c->aumag, c->amax, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_amax, c->amax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double a, b;
  std::memcpy(&a, &c->h_amax[0], sizeof(double));
  std::memcpy(&b, &c->h_amax[1], sizeof(double));
  *rel = b > 0.0 ? a / b : a;
  return IPM_OK;
}

// FP64 iterative refinement of the step on the augmented system eq. (6):
// with rho the residual of the current step, the correction solves
// A dp = rho, i.e. the Newton system with right-hand side r' = -rho, through
// the same condensation (Prop. 2.1), reduction (eq. (11), Prop. 2.3) and
// factor; then p += dp.  Stops at a backward error <= 1e-12 (a backward-
// stable FP64 solve is already there: no step), when a step does not halve
// it (the better step is kept), or after opt.aug_refine steps.
ipm_status refine_aug(ipm_ctx *c, double delta, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  double rel = 0.0;
  TRY(aug_residual(c, delta, &rel, st));
  c->aug_res0 = rel;
  c->aug_steps = 0;
  for (int it = 0; it < c->opt.aug_refine && rel > 1e-12 && std::isfinite(rel); ++it) {
    // right-hand side r' = -rho (in place)
    launch_lincomb(NX, c->ar1x, -1.0, c->ar1x, 0.0, nullptr, 0.0, nullptr, st);
    launch_lincomb(NX, c->ar3, -1.0, c->ar3, 0.0, nullptr, 0.0, nullptr, st);
    launch_lincomb(S.nu, c->ar1u, -1.0, c->ar1u, 0.0, nullptr, 0.0, nullptr, st);
    launch_lincomb(NM, c->ar2, -1.0, c->ar2, 0.0, nullptr, 0.0, nullptr, st);
    launch_lincomb(NM, c->ar4, -1.0, c->ar4, 0.0, nullptr, 0.0, nullptr, st);
    // condensed right-hand side (Prop. 2.1): rhat1 = r1' + H^T (Sigma_s r4' - r2')
    launch_tv(NM, D.Ss, c->ar2, c->ar4, c->atw, st);
    launch_htv(S, D, c->ar1x, c->ar1u, c->atw, c->arh1x, c->arh2, c->aupart, st);
    // eq. (11): b = G_x^{-1} r3', a = G_x^{-T}(rhat1_x - (K_xx + delta) b)
    launch_gather_pos(S.N, S.nx, S.iperm, c->ar3, c->bpos2, 1.0, st);
    solve1(c, c->bpos2, 0, st);
    launch_kapply(S, D.K, c->bpos2, nullptr, c->kpx, nullptr, st);
    launch_gather_pos(S.N, S.nx, S.iperm, c->arh1x, c->apos2, 1.0, st);
    launch_lincomb(NX, c->apos2, 1.0, c->apos2, -1.0, c->kpx, -delta, c->bpos2, st);
    const bool zfp64 = !c->mixed || c->exact_iter;  // an FP64 Z is at hand
    if (zfp64) {
      // with Z = -G_x^{-1} G_u: G_u^T G_x^{-T} w = -Z^T w, and
      // G_x^{-1}(r3' + G_u dp_u) = b - Z dp_u (no further forward solve)
      launch_lincomb(S.nu, c->dpu, -1.0, c->arh2, 0.0, nullptr, 0.0, nullptr, st);
      launch_zt_apply(S, c->Z, c->apos2, D.K, c->bpos2, -1.0, 1.0, c->dpu, c->cpos, st);
    } else {
      solve1(c, c->apos2, 1, st);
      launch_rhs_reduced(S, D.J, D.K, c->arh2, c->apos2, c->bpos2, c->dpu, st);
    }
    launch_chol_solve(S.nu, c->F, c->dpu, st);
    // Prop. 2.3: dp_x = -G_x^{-1}(r3' + G_u dp_u), dp_y = -G_x^{-T}(rhat1_x + (K_xx + delta) dp_x + K_xu dp_u)
    if (zfp64) {
      CK(cudaMemcpyAsync(c->vpos2, c->bpos2, NX * sizeof(double), cudaMemcpyDeviceToDevice, st));
      launch_z_apply(S, c->Z, c->dpu, -1.0, c->vpos2, st);
    } else {
      launch_gather_pos(S.N, S.nx, S.iperm, c->ar3, c->vpos2, 1.0, st);
      launch_gu_apply(S, D.J, c->dpu, c->vpos2, st);
      solve1(c, c->vpos2, 0, st);
      launch_lincomb(NX, c->vpos2, -1.0, c->vpos2, 0.0, nullptr, 0.0, nullptr, st);
    }
    launch_kapply(S, D.K, c->vpos2, c->dpu, c->kpx, c->kpu, st);
    launch_gather_pos(S.N, S.nx, S.iperm, c->arh1x, c->apos2, 1.0, st);
    launch_lincomb(NX, c->apos2, 1.0, c->apos2, 1.0, c->kpx, delta, c->vpos2, st);
    solve1(c, c->apos2, 1, st);
    launch_scatter_pos(S.N, S.nx, S.iperm, c->apos2, c->dpy, -1.0, st);
    launch_scatter_pos(S.N, S.nx, S.iperm, c->vpos2, c->dpx, 1.0, st);
    // Prop. 2.1: dp_z, dp_s
    launch_pzps_rhs(S, D, c->dpx, c->dpu, c->ar2, c->ar4, c->dpz, c->dps, st);
    launch_lincomb(c->step_len, c->step, 1.0, c->step, 1.0, c->dstep, 0.0, nullptr, st);
    double rel_new = 0.0;
    TRY(aug_residual(c, delta, &rel_new, st));
    ++c->aug_steps;
    if (!(rel_new <= 0.5 * rel)) {
      // stagnation: undo this correction and stop (the residual and the
      // products of the kept step are formed again for the line search)
      launch_lincomb(c->step_len, c->step, 1.0, c->step, -1.0, c->dstep, 0.0, nullptr, st);
      TRY(aug_residual(c, delta, &rel, st));
      break;
    }
    rel = rel_new;
  }
  c->aug_res = rel;
  return IPM_OK;
}

// Newton step: p_u from the Cholesky factor, then p_x, p_y (Prop. 2.3),
// p_z, p_s (Prop. 2.1) and the bound-dual steps.  With defer_py the
// transposed solve for p_y runs on the side stream (join_py before y is
// used).
ipm_status do_solve(ipm_ctx *c, cudaStream_t st, bool defer_py = false) {
  join_py(c, st);
  if (!c->have_fact) return fail(c, IPM_ERR_STATE, "solve before a successful factorization");
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const double delta = c->delta_fact, mu = c->mu;
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  ph_begin(c, PH_RECOVER, st);
  launch_lincomb(S.nu, c->pu, 1.0, c->rhs_u, delta, delta != 0.0 ? c->rhs_corr : nullptr, 0.0, nullptr, st);
  if (!c->mixed || c->exact_iter) {
    launch_chol_solve(S.nu, c->F, c->pu, st);
    // p_x = -G_x^{-1} (r3 + G_u p_u) = Z p_u - b
    CK(cudaMemcpyAsync(c->vpos, c->bpos, NX * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_z_apply(S, c->Z, c->pu, -1.0, c->vpos, st);
  } else {
    if (c->opt.max_refine > 0) {
      TRY(pcg_reduced(c, delta, st));
    } else {
      // the mixed-precision factor alone; refinement on eq. (6) follows
      launch_chol_solve(S.nu, c->F, c->pu, st);
      c->refine_iters = 0;
      c->refine_res = 0.0;
      c->neg_curv = false;
    }
    // p_x = -G_x^{-1} (r3 + G_u p_u) with FP64 solves
    launch_gather_pos(S.N, S.nx, S.iperm, D.g, c->vpos, 1.0, st);
    launch_gu_apply(S, D.J, c->pu, c->vpos, st);
    solve1(c, c->vpos, 0, st);
    launch_lincomb(NX, c->vpos, -1.0, c->vpos, 0.0, nullptr, 0.0, nullptr, st);
  }
  launch_scatter_pos(S.N, S.nx, S.iperm, c->vpos, c->px, 1.0, st);
  // p_y = -G_x^{-T} (rhat1 + (K_xx + delta I) p_x + K_xu p_u)
  launch_kapply(S, D.K, c->vpos, c->pu, c->kpx, c->kpu, st);
  launch_gather_pos(S.N, S.nx, S.iperm, D.rh1x, c->apos, 1.0, st);
  launch_lincomb(NX, c->apos, 1.0, c->apos, 1.0, c->kpx, delta, c->vpos, st);
  const bool refine = c->opt.aug_refine > 0;
  if (defer_py && !refine) {
    TRY(ensure_side(c));
    CK(cudaEventRecord(c->ev_fork, st));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    launch_solve1(S, D.LU, D.rd, c->apos, 1, c->side);
    launch_scatter_pos(S.N, S.nx, S.iperm, c->apos, c->py, -1.0, c->side);
    CK(cudaEventRecord(c->ev_join, c->side));
    c->py_pending = true;
  } else {
    solve1(c, c->apos, 1, st);
    launch_scatter_pos(S.N, S.nx, S.iperm, c->apos, c->py, -1.0, st);
  }
  launch_pz_ps(S, D, c->px, c->pu, c->Hp, c->pz, c->ps, st);
  if (refine) TRY(refine_aug(c, delta, st));
  launch_bound_steps(NX, S.nx, D.x, c->px, S.xl, S.xu, D.zlx, D.zux, mu, c->dz[0], c->dz[1], st);
  launch_bound_steps(S.nu, S.nu, D.u, c->pu, S.ul, S.uu, D.zlu, D.zuu, mu, c->dz[2], c->dz[3], st);
  launch_bound_steps(NM, S.m, D.s, c->ps, S.sl, S.su, D.zls, D.zus, mu, c->dz[4], c->dz[5], st);
  ph_end(c, PH_RECOVER, st);
  CK(cudaGetLastError());
  return IPM_OK;
}

ipm_status do_init(ipm_ctx *c, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  CK(cudaMemsetAsync(c->state, 0, c->state_len * sizeof(double), st));
  launch_init_primal(S, D.x, D.u, c->pmax_d, st);
  launch_push(NX, S.nx, D.x, S.xl, S.xu, K1, K2, st);
  launch_push(S.nu, S.nu, D.u, S.ul, S.uu, K1, K2, st);
  launch_functions(S, D.x, D.u, D.P, D.Q, D.g, D.h, D.fs, st);
  launch_lincomb(NM, D.s, -1.0, D.h, 0.0, nullptr, 0.0, nullptr, st);
  launch_push(NM, S.m, D.s, S.sl, S.su, K1, K2, st);
  launch_fill_bound_duals(NX, S.nx, S.xl, S.xu, D.zlx, D.zux, st);
  launch_fill_bound_duals(S.nu, S.nu, S.ul, S.uu, D.zlu, D.zuu, st);
  launch_fill_bound_duals(NM, S.m, S.sl, S.su, D.zls, D.zus, st);
  CK(cudaGetLastError());
  c->mu = MU0;
  c->rho = RHO0;
  c->delta_last = 0.0;
  c->have_eval = c->have_cond = c->have_fact = false;
  return write_scalars(c, st);
}

// One interior-point iteration, the same rule set as the oracle.
ipm_status do_step(ipm_ctx *c, int *converged, double *kkt_err, cudaStream_t st) {
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  TRY(do_eval(c, st));
  TRY(do_errors(c, st));
  const double E0 = emu(c->errs, 0.0);
  if (kkt_err) *kkt_err = E0;
  if (E0 <= c->opt.tol) {
    *converged = 1;
    return IPM_OK;
  }
  *converged = 0;
  double mu = c->mu;
  const double mu_min = c->opt.tol / 10.0;
  if (c->opt.barrier_rule == IPM_BARRIER_ADAPTIVE) {
    mu = std::max(mu_min, c->opt.sigma * c->mean_compl);
    c->mu = mu;
  } else if (emu(c->errs, mu) <= KAPPA_EPS * mu && mu > mu_min) {
    mu = std::max(mu_min, std::min(KAPPA_MU * mu, std::pow(mu, THETA_MU)));
    c->mu = mu;
  }
  c->exact_iter = false;
  TRY(do_condense(c, st));
  int pd = 0;
  TRY(do_factor(c, 0.0, &pd, st));
  if (c->mixed && !pd) {
    // The BF16x3 K_hat carries errors ~5e-7 of its largest entries; near the
    // solution (Sigma ~ 1/mu) that can make it indefinite although the exact
    // K_hat is positive definite.  Shift only the preconditioner (tau I,
    // tau = 1e-8 .. 1e-5 of its largest diagonal entry); the system keeps
    // delta = 0 and conjugate gradients on the exact operator decide: non-
    // positive curvature sends the iteration to the FP64 condensation.
    launch_maxdiag(S.nu, c->Khat, c->red_out, st);
    TRY(read_red(c, 1, st));
    const double dmax = c->h_red[0];
    for (double f = 1e-8; f <= 1e-5 * 1.0001 && !pd; f *= 10.0) TRY(do_factor(c, 0.0, &pd, st, f * dmax));
    // Still not positive definite: the reduced matrix is indefinite by more
    // than the BF16x3 error, so the delta_w rule below corrects the inertia
    // on it (the refinement on the exact operator at that delta_w checks the
    // decision: non-positive curvature there raises delta_w further).
  }
  double delta = 0.0;
  if (!pd) {
    const double dl = c->delta_last;
    delta = dl == 0.0 ? DELTA0 : std::max(DELTA_MIN, KW_MINUS * dl);
    while (true) {
      TRY(do_factor(c, delta, &pd, st));
      if (pd) {
        c->delta_last = delta;
        break;
      }
      delta *= (dl == 0.0) ? KW_PLUS_BAR : KW_PLUS;
      if (delta > DELTA_MAX) return fail(c, IPM_ERR_NOT_PD, "inertia correction exceeded delta_max");
    }
  }
  TRY(do_solve(c, st, true));
  // Mixed path: CG met non-positive curvature of the exact operator at this
  // delta_w, so the BF16x3 matrix passed a Cholesky test that the exact one
  // fails.  The Rayleigh quotient q = p^T A p / p^T p <= 0 of the direction
  // CG found bounds the smallest eigenvalue of the exact operator from
  // above, so delta_w must grow by at least |q|: take delta + 2 |q| (at
  // least twice delta, at least the rule's first trial) and solve again, a
  // few times at most; the inertia is then decided on the exact operator.
  for (int raise = 0; c->mixed && !c->exact_iter && c->opt.max_refine > 0 && c->neg_curv && raise < 6; ++raise) {
    const double dl = c->delta_last;
    const double first = dl == 0.0 ? DELTA0 : std::max(DELTA_MIN, KW_MINUS * dl);
    delta = std::max({first, 2.0 * delta, delta + 2.0 * std::fabs(c->curv_q)});
    if (delta > DELTA_MAX) break;
    ++c->n_curv_raise;
    join_py(c, st);
    TRY(do_factor(c, delta, &pd, st));
    if (!pd) continue;
    c->delta_last = delta;
    TRY(do_solve(c, st, true));
  }
  // the mixed-precision step is kept when CG (if run) converged without
  // meeting non-positive curvature and, with refinement on eq. (6), its
  // augmented residual reached 1e-10
  const bool cg_bad = c->opt.max_refine > 0 && (c->neg_curv || !(c->refine_res <= 1e-10));
  const bool aug_bad = c->opt.aug_refine > 0 && !(c->aug_res <= 1e-10);
  if (c->mixed && !c->exact_iter && (cg_bad || aug_bad)) {
    join_py(c, st);
    // CG met non-positive curvature or did not converge: redo in FP64
    c->exact_iter = true;
    ++c->n_fallback;
    ph_begin(c, PH_FALLBACK, st);
    TRY(do_condense(c, st));
    pd = 0;
    TRY(do_factor(c, 0.0, &pd, st));
    delta = 0.0;
    if (!pd) {
      const double dl = c->delta_last;
      delta = dl == 0.0 ? DELTA0 : std::max(DELTA_MIN, KW_MINUS * dl);
      while (true) {
        TRY(do_factor(c, delta, &pd, st));
        if (pd) {
          c->delta_last = delta;
          break;
        }
        delta *= (dl == 0.0) ? KW_PLUS_BAR : KW_PLUS;
        if (delta > DELTA_MAX) return fail(c, IPM_ERR_NOT_PD, "inertia correction exceeded delta_max");
      }
    }
    TRY(do_solve(c, st, true));
    ph_end(c, PH_FALLBACK, st);
  }
  // every exit from here on waits for the p_y solve on the side stream
  struct JoinPy {
    ipm_ctx *c;
    cudaStream_t st;
    ~JoinPy() { join_py(c, st); }
  } join_at_exit{c, st};
  ph_begin(c, PH_LS, st);
  const double tau = std::max(TAU_MIN, 1.0 - mu);
  // fraction to the boundary, directional-derivative terms and the merit
  // at the current point: three reductions, one read-back
  launch_ftb(S, D, c->px, c->pu, c->ps, c->dz, tau, c->red_partial, c->red_out, st);
  launch_dir(S, D, c->px, c->pu, c->ps, c->kpx, c->kpu, c->Hp, mu, delta, c->red_partial, c->red_out + 2, st);
  launch_merit(S, D.x, D.u, D.s, D.g, D.h, D.fs, c->red_partial, c->red_out + 5, st);
  TRY(read_red(c, 8, st));
  const double amax = std::min(1.0, c->h_red[0]), az = std::min(1.0, c->h_red[1]);
  const double gphi = c->h_red[2], q = c->h_red[3], c1 = c->h_red[4];
  const double merit0[3] = {c->h_red[5], c->h_red[6], c->h_red[7]};
  if (c1 > 0.0) {
    const double rt = (gphi + 0.5 * std::max(q, 0.0)) / ((1.0 - RHO_FRAC) * c1);
    if (c->rho < rt) c->rho = rt;
  }
  const double rho = c->rho;
  const double dphi = gphi - rho * c1;
  const double phi0 = (merit0[0] - mu * merit0[1]) + rho * merit0[2];
  double alpha = amax;
  int trials = 0;
  while (true) {
    ++trials;
    launch_lincomb(NX, c->xt, 1.0, D.x, alpha, c->px, 0.0, nullptr, st);
    launch_lincomb(S.nu, c->ut, 1.0, D.u, alpha, c->pu, 0.0, nullptr, st);
    launch_lincomb(NM, c->st, 1.0, D.s, alpha, c->ps, 0.0, nullptr, st);
    launch_functions(S, c->xt, c->ut, c->Pt, c->Qt, c->gt, c->ht, c->fst, st);
    launch_merit(S, c->xt, c->ut, c->st, c->gt, c->ht, c->fst, c->red_partial, c->red_out, st);
    TRY(read_red(c, 3, st));
    const double phit = (c->h_red[0] - mu * c->h_red[1]) + rho * c->h_red[2];
    // Armijo with a roundoff allowance: changes below 10 eps |phi| count as none
    if (phit - phi0 <= ETA * alpha * dphi + 10.0 * std::numeric_limits<double>::epsilon() * std::fabs(phi0)) break;
    alpha *= 0.5;
    if (alpha < ALPHA_MIN) return fail(c, IPM_ERR_LINESEARCH, "step size below alpha_min");
  }
  CK(cudaMemcpyAsync(D.x, c->xt, NX * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(D.u, c->ut, S.nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(D.s, c->st, NM * sizeof(double), cudaMemcpyDeviceToDevice, st));
  join_py(c, st);
  launch_lincomb(NX, D.y, 1.0, D.y, alpha, c->py, 0.0, nullptr, st);
  launch_lincomb(NM, D.z, 1.0, D.z, alpha, c->pz, 0.0, nullptr, st);
  launch_dual_update(NX, S.nx, D.x, S.xl, S.xu, D.zlx, D.zux, c->dz[0], c->dz[1], az, mu, KAPPA_SIGMA, st);
  launch_dual_update(S.nu, S.nu, D.u, S.ul, S.uu, D.zlu, D.zuu, c->dz[2], c->dz[3], az, mu, KAPPA_SIGMA, st);
  launch_dual_update(NM, S.m, D.s, S.sl, S.su, D.zls, D.zus, c->dz[4], c->dz[5], az, mu, KAPPA_SIGMA, st);
  ph_end(c, PH_LS, st);
  CK(cudaGetLastError());
  c->info[0] = alpha; c->info[1] = amax; c->info[2] = az; c->info[3] = delta;
  c->info[4] = trials; c->info[5] = rho; c->info[6] = mu; c->info[7] = c->mixed ? c->refine_iters : 0;
  c->info[8] = c->mixed ? c->refine_res : 0.0; c->info[9] = c->exact_iter ? 1.0 : 0.0;
  c->exact_iter = false;
  c->have_eval = c->have_cond = c->have_fact = false;
  ipm_status ws = write_scalars(c, st);
  ph_collect(c);
  return ws;
}

// layout of the warm-start vectors of a context
ipm_status warm_layout(ipm_ctx *c) {
  if (c->warm_ready) return IPM_OK;
  const Sym &S = c->S;
  std::vector<int> idx;
  int *seg = c->warm_seg;
  seg[0] = 0;
  seg[1] = S.nx;
  seg[2] = seg[1] + S.nu;
  seg[3] = seg[2] + S.m;
  const std::vector<double> *bnd[6] = {&S.xl, &S.xu, &S.ul, &S.uu, &S.sl, &S.su};
  for (int b = 0; b < 6; ++b) {
    int cnt = 0;
    for (size_t j = 0; j < bnd[b]->size(); ++j)
      if (std::isfinite((*bnd[b])[j])) {
        idx.push_back((int)j);
        ++cnt;
      }
    seg[4 + b] = seg[3 + b] + cnt;
  }
  const int *p = nullptr;
  TRY(upload(c, &p, idx));
  c->warm_idx = const_cast<int *>(p);
  c->warm_ready = true;
  return IPM_OK;
}

WarmSeg warm_seg(const ipm_ctx *c) {
  WarmSeg W;
  for (int i = 0; i < 10; ++i) W.seg[i] = c->warm_seg[i];
  W.nx = c->S.nx;
  W.m = c->S.m;
  W.idx = c->warm_idx;
  return W;
}

// Start from predicted warm-start vectors (ipm_warm_start in include/ipm.h)
ipm_status do_warm_start(ipm_ctx *c, const float *pred, cudaStream_t st) {
  TRY(warm_layout(c));
  const DevSym &S = c->ds;
  DevWork &D = c->dw;
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  // bound duals of unbounded components stay zero
  CK(cudaMemsetAsync(c->state, 0, c->state_len * sizeof(double), st));
  launch_warm_apply(D, warm_seg(c), S.N, pred, st);
  // interior point: a push much smaller than the cold start's keeps the prediction
  launch_push(NX, S.nx, D.x, S.xl, S.xu, K1_WARM, K1_WARM, st);
  launch_push(S.nu, S.nu, D.u, S.ul, S.uu, K1_WARM, K1_WARM, st);
  launch_push(NM, S.m, D.s, S.sl, S.su, K1_WARM, K1_WARM, st);
  launch_warm_z(NM, D, st);
  // y from the x-stationarity with one transposed solve per scenario
  launch_functions(S, D.x, D.u, D.P, D.Q, D.g, D.h, D.fs, st);
  launch_derivatives(S, D, st);
  CK(cudaMemsetAsync(D.flags, 0, FLAG_COUNT * sizeof(int), st));
  launch_lu_factor(S, c->nL, D.J, D.LU, D.rd, D.flags, st, c->opt.lu_pair != 0);
  launch_warm_yrhs(S, D, c->kpx, st);
  launch_gather_pos(S.N, S.nx, S.iperm, c->kpx, c->apos, 1.0, st);
  solve1(c, c->apos, 1, st);
  launch_scatter_pos(S.N, S.nx, S.iperm, c->apos, D.y, -1.0, st);
  CK(cudaGetLastError());
  TRY(read_flags(c, st));
  if (c->h_flags[FLAG_SINGULAR]) return fail(c, IPM_ERR_SINGULAR_GX, "singular G_x at the warm-start point");
  c->have_eval = c->have_cond = c->have_fact = false;
  TRY(do_eval(c, st));
  TRY(do_errors(c, st));
  c->mu = std::max(1e-6, c->mean_compl);
  c->rho = RHO0;
  c->delta_last = 0.0;
  return write_scalars(c, st);
}

bool finite_nonneg(const double *p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i]) || p[i] < 0) return false;
  return true;
}

}  // namespace

// ===========================================================================
void host_net(const ipm_network *net, HostNet &h) {
  h.n = net->n_bus; h.L = net->n_line; h.ng = net->n_gen;
  h.fr.assign(net->from, net->from + h.L); h.to.assign(net->to, net->to + h.L);
  h.gen.assign(net->gen_bus, net->gen_bus + h.ng);
  h.r.assign(net->r, net->r + h.L); h.x.assign(net->x, net->x + h.L); h.b.assign(net->b, net->b + h.L);
  h.pmax.assign(net->pmax, net->pmax + h.ng); h.qmax.assign(net->qmax, net->qmax + h.ng);
  h.c2.assign(net->c2, net->c2 + h.ng); h.c1.assign(net->c1, net->c1 + h.ng);
  h.vmin.assign(net->vmin, net->vmin + h.n); h.vmax.assign(net->vmax, net->vmax + h.n);
  h.rate.clear();
  if (net->rate) h.rate.assign(net->rate, net->rate + h.L);
}

extern "C" {

ipm_status ipm_default_options(ipm_options *opt) {
  if (!opt) return IPM_ERR_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->tol = 1e-8;
  opt->max_iter = 200;
  opt->precision = IPM_PREC_FP64;
  opt->max_refine = 60;
  opt->solve_threads = 0;
  opt->graphs = 0;
  opt->autotune = 0;
  opt->lu_pair = 1;
  opt->aug_refine = 10;
  opt->barrier_rule = IPM_BARRIER_ADAPTIVE;
  opt->sigma = 0.1;
  opt->tc_solve = 1;
  return IPM_OK;
}

ipm_status ipm_create(const ipm_network *net, int n_scen, const double *pd, const double *qd,
                      const ipm_options *opt, ipm_ctx **out) {
  if (!out) return IPM_ERR_ARG;
  *out = nullptr;
  if (!net || !pd || !qd || n_scen < 1 || net->n_bus < 2 || net->n_line < 1 || net->n_gen < 1)
    return IPM_ERR_ARG;
  if (!net->from || !net->to || !net->gen_bus || !net->r || !net->x || !net->b || !net->pmax ||
      !net->qmax || !net->c2 || !net->c1 || !net->vmin || !net->vmax)
    return IPM_ERR_ARG;
  const size_t nl = (size_t)n_scen * net->n_bus;
  if (!finite_nonneg(pd, nl)) return IPM_ERR_ARG;
  for (size_t i = 0; i < nl; ++i)
    if (!std::isfinite(qd[i])) return IPM_ERR_ARG;
  ipm_ctx *c = new ipm_ctx();
  if (opt) c->opt = *opt;
  else ipm_default_options(&c->opt);
  if ((c->opt.precision != IPM_PREC_FP64 && c->opt.precision != IPM_PREC_MIXED &&
       c->opt.precision != IPM_PREC_FP64_TC) || !(c->opt.tol > 0) ||
      c->opt.max_iter < 0 || c->opt.max_refine < 0 || c->opt.aug_refine < 0 || c->opt.aug_refine > 100 ||
      c->opt.reduction < IPM_REDUCTION_DENSE || c->opt.reduction > IPM_REDUCTION_AUTO ||
      (c->opt.big_block != 0 && c->opt.big_block != 1) ||
      (c->opt.solve_threads != 0 && c->opt.solve_threads != 128 && c->opt.solve_threads != 256) ||
      (c->opt.graphs != 0 && c->opt.graphs != 1) || (c->opt.autotune != 0 && c->opt.autotune != 1) ||
      (c->opt.poison != 0 && c->opt.poison != 1) || (c->opt.lu_pair != 0 && c->opt.lu_pair != 1) ||
      (c->opt.tc_solve != 0 && c->opt.tc_solve != 1) ||
      (c->opt.barrier_rule == IPM_BARRIER_ADAPTIVE && !(c->opt.sigma > 0 && c->opt.sigma < 1))) {
    delete c;
    return IPM_ERR_ARG;
  }
  HostNet h;
  host_net(net, h);
  bool ok = true;
  for (int k = 0; k < h.ng; ++k)
    if (!(h.pmax[k] > 0) || !(h.qmax[k] >= 0) || !std::isfinite(h.c2[k]) || !std::isfinite(h.c1[k])) ok = false;
  for (int i = 0; i < h.n; ++i)
    if (!(h.vmin[i] > 0) || !(h.vmax[i] > h.vmin[i]) || !std::isfinite(h.vmax[i])) ok = false;
  std::string err;
  if (!ok || !build_symbolic(h, n_scen, c->S, err, c->opt.big_block)) {
    delete c;
    return IPM_ERR_ARG;
  }
  ipm_status s = upload_symbolic(c, h, pd, qd);
  if (s == IPM_OK) s = alloc_work(c);
  if (s == IPM_OK) s = do_init(c, 0);
  if (s != IPM_OK) {
    ipm_destroy(c);
    return s;
  }
  *out = c;
  return IPM_OK;
}

ipm_status ipm_destroy(ipm_ctx *c) {
  if (!c) return IPM_ERR_ARG;
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->side2) cudaStreamSynchronize(c->side2);
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->ev_fork, c->ev_join, c->ev_fork2, c->ev_join2})
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  for (void *p : c->allocs) cudaFree(p);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->h_mu) cudaFreeHost(c->h_mu);
  if (c->h_amax) cudaFreeHost(c->h_amax);
  for (int b = 0; b < 2; ++b) {
    if (c->gx_pre[b]) cudaGraphExecDestroy(c->gx_pre[b]);
    if (c->gx_post[b]) cudaGraphExecDestroy(c->gx_post[b]);
  }
  delete c;
  return IPM_OK;
}

ipm_status ipm_get_dims(const ipm_ctx *c, ipm_dims *o) {
  if (!c || !o) return IPM_ERR_ARG;
  o->n_bus = c->S.n; o->n_line = c->S.L; o->n_gen = c->S.ng; o->n_scen = c->S.N;
  o->n_x = c->S.nx; o->n_u = c->S.nu; o->m = c->S.m;
  o->state_len = c->state_len; o->step_len = c->step_len;
  o->nnz_lu = c->S.nnzLU;
  o->lu_levels = c->S.nlev;
  o->nnz_kx = (int)c->S.kx_col.size();
  o->nnz_ku = (int)c->S.ku_col.size();
  o->nd = c->S.nd;
  o->big_block = c->S.big ? 1 : 0;
  o->lu_sparse_ops = c->S.n_ops + c->S.n_tail_ops;
  return IPM_OK;
}

const char *ipm_last_error(const ipm_ctx *c) { return c ? c->err.c_str() : "null context"; }

ipm_status ipm_init_state(ipm_ctx *c, void *stream) {
  if (!c) return IPM_ERR_ARG;
  return do_init(c, STR(stream));
}

ipm_status ipm_set_state(ipm_ctx *c, const double *state, int on_device, void *stream) {
  if (!c || !state) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  CK(cudaMemcpyAsync(c->state, state, c->state_len * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  c->have_eval = c->have_cond = c->have_fact = false;
  return read_scalars(c, st);
}

ipm_status ipm_get_state(ipm_ctx *c, double *state, int on_device, void *stream) {
  if (!c || !state) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  CK(cudaMemcpyAsync(state, c->state, c->state_len * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}

ipm_status ipm_eval_derivatives(ipm_ctx *c, void *stream) {
  if (!c) return IPM_ERR_ARG;
  return do_eval(c, STR(stream));
}

ipm_status ipm_condense_scenarios(ipm_ctx *c, void *stream) {
  if (!c) return IPM_ERR_ARG;
  return do_condense(c, STR(stream));
}

ipm_status ipm_factor_schur(ipm_ctx *c, double delta_w, int *is_pd, void *stream) {
  if (!c || !is_pd || !(delta_w >= 0) || !std::isfinite(delta_w)) return IPM_ERR_ARG;
  return do_factor(c, delta_w, is_pd, STR(stream));
}

ipm_status ipm_solve_kkt(ipm_ctx *c, double *step, double *refine_resid, void *stream) {
  if (!c) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  TRY(do_solve(c, st));
  if (step) CK(cudaMemcpyAsync(step, c->step, c->step_len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (refine_resid) *refine_resid = c->opt.aug_refine > 0 ? c->aug_res : (c->mixed ? c->refine_res : 0.0);
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}

ipm_status ipm_step(ipm_ctx *c, int *converged, double *kkt_err, void *stream) {
  if (!c || !converged) return IPM_ERR_ARG;
  return do_step(c, converged, kkt_err, STR(stream));
}

ipm_status ipm_solve(ipm_ctx *c, int *iters, double *kkt_err, void *stream) {
  if (!c) return IPM_ERR_ARG;
  int conv = 0;
  double e = 0.0;
  for (int k = 0; k <= c->opt.max_iter; ++k) {
    TRY(do_step(c, &conv, &e, STR(stream)));
    if (conv) {
      if (iters) *iters = k;
      if (kkt_err) *kkt_err = e;
      return IPM_OK;
    }
  }
  if (iters) *iters = c->opt.max_iter;
  if (kkt_err) *kkt_err = e;
  return fail(c, IPM_ERR_MAXITER, "iteration limit reached");
}

ipm_status ipm_get_quantity(ipm_ctx *c, int which, int scen, double *out, long long cap, void *stream) {
  if (!c || !out) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  const Sym &S = c->S;
  const int N = S.N, nx = S.nx, nu = S.nu, m = S.m;
  auto need = [&](long long k) { return cap >= k; };
  CK(cudaStreamSynchronize(st));
  if (which == IPM_Q_KHAT) {
    if (!c->have_cond) return fail(c, IPM_ERR_STATE, "no condensed system");
    if (!need((long long)nu * nu)) return IPM_ERR_ARG;
    CK(cudaMemcpy(out, c->Khat, (size_t)nu * nu * sizeof(double), cudaMemcpyDeviceToHost));
    return IPM_OK;
  }
  if (which == IPM_Q_ZTZ) {
    if (!c->have_cond || !c->M_valid) return fail(c, IPM_ERR_STATE, "no inertia-correction product");
    if (!need((long long)nu * nu)) return IPM_ERR_ARG;
    CK(cudaMemcpy(out, c->M, (size_t)nu * nu * sizeof(double), cudaMemcpyDeviceToHost));
    return IPM_OK;
  }
  if (which == IPM_Q_RHS_U) {
    if (!c->have_cond) return fail(c, IPM_ERR_STATE, "no condensed system");
    if (!need(nu)) return IPM_ERR_ARG;
    CK(cudaMemcpy(out, c->rhs_u, nu * sizeof(double), cudaMemcpyDeviceToHost));
    return IPM_OK;
  }
  if (which == IPM_Q_ERRS) {
    if (!need(6)) return IPM_ERR_ARG;
    if (c->have_eval) TRY(do_errors(c, st));
    std::memcpy(out, c->errs, 6 * sizeof(double));
    return IPM_OK;
  }
  if (which == IPM_Q_TIMERS) {
    if (!need(2 * IPM_N_PHASES)) return IPM_ERR_ARG;
    ph_collect(c);
    for (int p = 0; p < IPM_N_PHASES; ++p) {
      out[p] = c->t_ms[p];
      out[IPM_N_PHASES + p] = c->t_cnt[p];
    }
    if (cap >= 2 * IPM_N_PHASES + 1) out[2 * IPM_N_PHASES] = (double)g_ipm_launches;
    return IPM_OK;
  }
  if (which == IPM_Q_INFO) {
    if (!need(10)) return IPM_ERR_ARG;
    std::memcpy(out, c->info, 10 * sizeof(double));
    // optional tail: counts since the context was created
    if (cap >= 11) out[10] = (double)c->n_fallback;       // mixed: iterations condensed again in FP64
    if (cap >= 12) out[11] = (double)c->n_emu_fallback;   // FP64_TC: contractions redone on the FP64 units
    if (cap >= 13) out[12] = (double)c->aug_steps;        // refinement steps on eq. (6), last solve
    if (cap >= 14) out[13] = c->aug_res0;                  // its relative residual before them
    if (cap >= 15) out[14] = c->aug_res;                   // and after
    if (cap >= 16) out[15] = c->adjoint ? 1.0 : 0.0;       // K_hat by the adjoint-solve reduction
    if (cap >= 17) out[16] = c->tune_ms[6];                // autotuner: dense reduction (ms)
    if (cap >= 18) out[17] = c->tune_ms[7];                // autotuner: adjoint reduction (ms)
    if (cap >= 19) out[18] = (double)c->n_curv_raise;      // mixed: delta_w raises after CG curvature
    return IPM_OK;
  }
  if (scen < 0 || scen >= N) return IPM_ERR_ARG;
  if (which == IPM_Q_Z) {
    if (!c->have_cond) return fail(c, IPM_ERR_STATE, "no condensed system");
    if (!need((long long)nx * nu)) return IPM_ERR_ARG;
    std::vector<double> z((size_t)nx * nu);
    if (c->mixed) {
      std::vector<float> zf((size_t)nx * nu);
      CK(cudaMemcpy(zf.data(), c->Z32 + (size_t)scen * nx * nu, zf.size() * sizeof(float), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < zf.size(); ++i) z[i] = zf[i];
    } else {
      CK(cudaMemcpy(z.data(), c->Z + (size_t)scen * nx * nu, z.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    for (int p = 0; p < nx; ++p)
      std::memcpy(out + (size_t)S.iperm[p] * nu, z.data() + (size_t)p * nu, nu * sizeof(double));
    return IPM_OK;
  }
  if (!c->have_eval) return fail(c, IPM_ERR_STATE, "no evaluation");
  if (which == IPM_Q_FGH) {
    if (!need(1 + nx + m)) return IPM_ERR_ARG;
    double fs = 0.0;
    CK(cudaMemcpy(&fs, c->dw.fs + scen, sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> u(nu);
    CK(cudaMemcpy(u.data(), c->dw.u, nu * sizeof(double), cudaMemcpyDeviceToHost));
    double fu = 0.0;
    for (int k = 1; k < S.ng; ++k) fu += S.c2[k] * u[S.ng + k - 1] * u[S.ng + k - 1] + S.c1[k] * u[S.ng + k - 1];
    out[0] = fs + fu / N;
    CK(cudaMemcpy(out + 1, c->dw.g + (size_t)scen * nx, nx * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(out + 1 + nx, c->dw.h + (size_t)scen * m, m * sizeof(double), cudaMemcpyDeviceToHost));
    return IPM_OK;
  }
  auto aslot = [&](int i, int k) -> int {
    for (int p = S.a_ptr[i]; p < S.a_ptr[i + 1]; ++p)
      if (S.a_col[p] == k) return p;
    return -1;
  };
  auto kbslot = [&](int i, int k) -> int {
    for (int p = S.kb_ptr[i]; p < S.kb_ptr[i + 1]; ++p)
      if (S.kb_col[p] == k) return p;
    return -1;
  };
  auto ucol = [&](int j, int &bus, int &kind) {  // kind 1 = voltage, 2 = Pg
    if (j < S.ng) { bus = S.hrow_bus[j]; kind = 1; }
    else { bus = S.hrow_bus[j - S.ng + 1]; kind = 2; }
  };
  if (which == IPM_Q_JAC) {
    const long long tot = (long long)nx * nx + (long long)nx * nu + (long long)m * nx + (long long)m * nu;
    if (!need(tot)) return IPM_ERR_ARG;
    std::vector<double> J((size_t)4 * S.nnzA * N);
    CK(cudaMemcpy(J.data(), c->dw.J, J.size() * sizeof(double), cudaMemcpyDeviceToHost));
    auto jv = [&](int slot, int e) { return J[((size_t)slot * 4 + e) * N + scen]; };
    std::memset(out, 0, tot * sizeof(double));
    double *Gx = out, *Gu = Gx + (size_t)nx * nx, *Hx = Gu + (size_t)nx * nu, *Hu = Hx + (size_t)m * nx;
    for (int r = 0; r < nx; ++r) {
      const int a = S.xbus[r], ka = S.xkind[r];
      for (int cidx = 0; cidx < nx; ++cidx) {
        const int s = aslot(a, S.xbus[cidx]);
        if (s >= 0) Gx[(size_t)r * nx + cidx] = jv(s, ka * 2 + S.xkind[cidx]);
      }
      for (int j = 0; j < nu; ++j) {
        int b, kind;
        ucol(j, b, kind);
        if (kind == 1) {
          const int s = aslot(a, b);
          if (s >= 0) Gu[(size_t)r * nu + j] = jv(s, ka * 2 + 1);
        } else if (ka == 0 && a == b) {
          Gu[(size_t)r * nu + j] = -1.0;
        }
      }
    }
    std::vector<double> HF;
    if (S.nflow > 0) {
      HF.resize((size_t)4 * S.nflow * N);
      CK(cudaMemcpy(HF.data(), c->dw.HF, HF.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    for (int r = 0; r < m; ++r) {
      const int g = S.hrow_bus[r], cp = S.hrow_comp[r];
      if (cp >= 2) {  // line-flow row: its two end buses
        const int f = r - S.ng - 1, l = f % S.L;
        for (int w = 0; w < 2; ++w) {
          const int b = w == 0 ? g : (f < S.L ? S.lto[l] : S.lfr[l]);
          for (int kind = 0; kind < 2; ++kind) {
            const double v = HF[((size_t)(f * 2 + w) * 2 + kind) * N + scen];
            const int xi = kind == 0 ? S.xth[b] : S.xv[b];
            if (xi >= 0) Hx[(size_t)r * nx + xi] = v;
            else if (kind == 1) Hu[(size_t)r * nu + S.uv[b]] = v;
          }
        }
        continue;
      }
      for (int cidx = 0; cidx < nx; ++cidx) {
        const int s = aslot(g, S.xbus[cidx]);
        if (s >= 0) Hx[(size_t)r * nx + cidx] = jv(s, cp * 2 + S.xkind[cidx]);
      }
      for (int j = 0; j < nu; ++j) {
        int b, kind;
        ucol(j, b, kind);
        if (kind == 1) {
          const int s = aslot(g, b);
          if (s >= 0) Hu[(size_t)r * nu + j] = jv(s, cp * 2 + 1);
        }
      }
    }
    return IPM_OK;
  }
  if (which == IPM_Q_HESS) {
    if (!c->have_cond) return fail(c, IPM_ERR_STATE, "no condensed system");
    const long long tot = (long long)nx * nx + (long long)nx * nu + (long long)nu * nu;
    if (!need(tot)) return IPM_ERR_ARG;
    std::vector<double> K((size_t)4 * S.nnzKB * N);
    CK(cudaMemcpy(K.data(), c->dw.K, K.size() * sizeof(double), cudaMemcpyDeviceToHost));
    auto kv = [&](int slot, int e) { return K[((size_t)slot * 4 + e) * N + scen]; };
    std::memset(out, 0, tot * sizeof(double));
    double *Kxx = out, *Kxu = Kxx + (size_t)nx * nx, *Kuu = Kxu + (size_t)nx * nu;
    for (int r = 0; r < nx; ++r) {
      const int a = S.xbus[r], ka = S.xkind[r];
      for (int cidx = 0; cidx < nx; ++cidx) {
        const int s = kbslot(a, S.xbus[cidx]);
        if (s >= 0) Kxx[(size_t)r * nx + cidx] = kv(s, ka * 2 + S.xkind[cidx]);
      }
      for (int j = 0; j < nu; ++j) {
        int b, kind;
        ucol(j, b, kind);
        if (kind == 1) {
          const int s = kbslot(a, b);
          if (s >= 0) Kxu[(size_t)r * nu + j] = kv(s, ka * 2 + 1);
        }
      }
    }
    for (int i = 0; i < nu; ++i) {
      int a, ka;
      ucol(i, a, ka);
      for (int j = 0; j < nu; ++j) {
        int b, kb;
        ucol(j, b, kb);
        if (ka == 1 && kb == 1) {
          const int s = kbslot(a, b);
          if (s >= 0) Kuu[(size_t)i * nu + j] = kv(s, 3);
        } else if (ka == 2 && kb == 2 && i == j) {
          Kuu[(size_t)i * nu + j] = 2.0 * S.c2[j - S.ng + 1] / N;
        }
      }
    }
    return IPM_OK;
  }
  return IPM_ERR_ARG;
}

ipm_status ipm_set_loads(ipm_ctx *c, const double *pd, const double *qd, void *stream) {
  if (!c || !pd || !qd) return IPM_ERR_ARG;
  const size_t nl = (size_t)c->S.N * c->S.n;
  if (!finite_nonneg(pd, nl)) return IPM_ERR_ARG;
  for (size_t i = 0; i < nl; ++i)
    if (!std::isfinite(qd[i])) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  CK(cudaMemcpyAsync(const_cast<double *>(c->ds.pd), pd, nl * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<double *>(c->ds.qd), qd, nl * sizeof(double), cudaMemcpyHostToDevice, st));
  return do_init(c, st);
}

ipm_status ipm_set_contingencies(ipm_ctx *c, const int *trip, void *stream) {
  if (!c) return IPM_ERR_ARG;
  const Sym &S = c->S;
  const int N = S.N, L = S.L, n = S.n;
  std::vector<double> on((size_t)L * N, 1.0);
  if (trip) {
    // bridges of the bus graph (depth-first low-link values): tripping one
    // of them islands part of the network
    std::vector<std::vector<std::pair<int, int>>> adj(n);
    for (int l = 0; l < L; ++l) {
      adj[S.lfr[l]].push_back({S.lto[l], l});
      adj[S.lto[l]].push_back({S.lfr[l], l});
    }
    std::vector<int> disc(n, -1), low(n, 0);
    std::vector<char> bridge(L, 0);
    int t = 0;
    for (int root = 0; root < n; ++root) {
      if (disc[root] >= 0) continue;
      struct Fr { int v, pl; size_t k; };
      std::vector<Fr> stk;
      disc[root] = low[root] = t++;
      stk.push_back({root, -1, 0});
      while (!stk.empty()) {
        Fr &f = stk.back();
        if (f.k == adj[f.v].size()) {
          const int v = f.v, pl = f.pl;
          stk.pop_back();
          if (!stk.empty()) {
            const int p = stk.back().v;
            low[p] = std::min(low[p], low[v]);
            if (low[v] > disc[p]) bridge[pl] = 1;
          }
          continue;
        }
        const auto e = adj[f.v][f.k++];
        if (e.second == f.pl) continue;
        if (disc[e.first] < 0) {
          disc[e.first] = low[e.first] = t++;
          stk.push_back({e.first, e.second, 0});
        } else {
          low[f.v] = std::min(low[f.v], disc[e.first]);
        }
      }
    }
    for (int s = 0; s < N; ++s) {
      const int l = trip[s];
      if (l < -1 || l >= L) return fail(c, IPM_ERR_ARG, "contingency line index out of range");
      if (l >= 0 && bridge[l]) return fail(c, IPM_ERR_ARG, "tripping this line disconnects the network");
      if (l >= 0) on[(size_t)l * N + s] = 0.0;
    }
  }
  cudaStream_t st = STR(stream);
  if (!c->ds.lon) {
    const double *p = nullptr;
    TRY(upload(c, &p, on));
    c->ds.lon = p;
  } else {
    CK(cudaMemcpyAsync(const_cast<double *>(c->ds.lon), on.data(), on.size() * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  return do_init(c, st);
}

ipm_status ipm_warm_dim(const ipm_ctx *c, int *d) {
  if (!c || !d) return IPM_ERR_ARG;
  const Sym &S = c->S;
  int n = S.nx + S.nu + S.m;
  const std::vector<double> *bnd[6] = {&S.xl, &S.xu, &S.ul, &S.uu, &S.sl, &S.su};
  for (auto *b : bnd)
    for (double v : *b) n += std::isfinite(v) ? 1 : 0;
  *d = n;
  return IPM_OK;
}

ipm_status ipm_warm_target(ipm_ctx *c, float *out, void *stream) {
  if (!c || !out) return IPM_ERR_ARG;
  cudaStream_t st = STR(stream);
  TRY(warm_layout(c));
  launch_warm_target(c->dw, warm_seg(c), c->S.N, out, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return IPM_OK;
}

ipm_status ipm_warm_start(ipm_ctx *c, const float *pred, void *stream) {
  if (!c || !pred) return IPM_ERR_ARG;
  return do_warm_start(c, pred, STR(stream));
}

long long ipm_kernel_launches(void) { return g_ipm_launches.load(); }

ipm_status ipm_symbolic_export(const ipm_network *net, int which, int *out, long long cap, long long *len) {
  const int force_big = (which & IPM_SYM_FORCE_BIG) ? 1 : 0;
  which &= ~IPM_SYM_FORCE_BIG;
  if (!net || !len || which < 0 || which >= IPM_SYM_COUNT || cap < 0 || net->n_bus < 2 || net->n_line < 1 ||
      net->n_gen < 1 || !net->from || !net->to || !net->gen_bus || !net->r || !net->x || !net->b ||
      !net->pmax || !net->qmax || !net->c2 || !net->c1 || !net->vmin || !net->vmax)
    return IPM_ERR_ARG;
  HostNet h;
  host_net(net, h);
  Sym S;
  std::string err;
  if (!build_symbolic(h, 1, S, err, force_big)) return IPM_ERR_ARG;
  std::vector<int> v;
  const std::vector<int> *src = &v;
  switch (which) {
    case IPM_SYM_DIMS:
      v = {S.nx, S.nu, S.t0, S.nd, S.nnzLU, S.zp_npan, LU_LISTS, S.dense_base, S.big ? 1 : 0};
      break;
    case IPM_SYM_LU_SLOT: src = &S.lu_slot; break;
    case IPM_SYM_LU_COLPTR: src = &S.lu_colptr; break;
    case IPM_SYM_LU_ROW: src = &S.lu_row; break;
    case IPM_SYM_FR_PTR: src = &S.fr_ptr; break;
    case IPM_SYM_FR_COL: src = &S.fr_col; break;
    case IPM_SYM_FR_LSLOT: src = &S.fr_lslot; break;
    case IPM_SYM_GU_PTR: src = &S.gu_ptr; break;
    case IPM_SYM_GU_COL: src = &S.gu_col; break;
    case IPM_SYM_ZP_LEV_OFF: src = &S.zp_lev_off; break;
    case IPM_SYM_ZP_LEV_PTR: src = &S.zp_lev_ptr; break;
    case IPM_SYM_ZP_ROWS: src = &S.zp_rows; break;
    case IPM_SYM_ZP_EPTR: src = &S.zp_eptr; break;
    case IPM_SYM_ZP_COL: src = &S.zp_col; break;
    case IPM_SYM_ZP_SLOT: src = &S.zp_slot; break;
    case IPM_SYM_ZP_ZPTR: src = &S.zp_zptr; break;
    case IPM_SYM_ZP_ZROWS: src = &S.zp_zrows; break;
    case IPM_SYM_ZP_TPTR: src = &S.zp_tptr; break;
    case IPM_SYM_ZP_TCOL: src = &S.zp_tcol; break;
    case IPM_SYM_ZP_TSLOT: src = &S.zp_tslot; break;
    case IPM_SYM_TW_LEN: src = &S.tw_len; break;
    case IPM_SYM_TW_L: src = &S.tw_l; break;
    case IPM_SYM_TW_U: src = &S.tw_u; break;
    case IPM_SYM_TW_E: src = &S.tw_e; break;
    default: return IPM_ERR_ARG;
  }
  *len = (long long)src->size();
  if (out)
    for (long long i = 0; i < std::min(cap, *len); ++i) out[i] = (*src)[(size_t)i];
  return IPM_OK;
}

ipm_status ipm_set_profiling(ipm_ctx *c, int on) {
  if (!c) return IPM_ERR_ARG;
  if (on && !c->ev[0])
    for (auto &e : c->ev) CK(cudaEventCreate(&e));
  if (on == 2 || !on)
    for (int p = 0; p < IPM_N_PHASES; ++p) {
      c->t_ms[p] = 0;
      c->t_cnt[p] = 0;
      c->ev_pending[p] = false;
    }
  c->prof = on != 0;
  return IPM_OK;
}

}  // extern "C"
