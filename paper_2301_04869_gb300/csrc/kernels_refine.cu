// Residual of the augmented Newton system eq. (6) at a computed step, for
// the FP64 iterative refinement of the KKT solve.
//
// With p = (p_d, p_s, p_y, p_z), p_d = (p_x, p_u), the residual of eq. (6)
// (right-hand side -r) is
//   rho_d = -r1 - (W + Sigma_p + delta I) p_d - G^T p_y - H^T p_z
//   rho_s = -r2 - Sigma_s p_s - p_z
//   rho_y = -r3 - G p_d
//   rho_z = -r4 - H p_d - p_s.
// W is not stored alone: the condensed matrix K = W + Sigma_p + H^T Sigma_s H
// of Prop. 2.1 is (K_xx, K_xu per scenario on the bus pattern; K_uu^i plus
// the first-stage diagonal once), so
//   (W + Sigma_p) p_d = K p_d - H^T (Sigma_s H p_d)
// and rho_d = -r1 - K p_d - delta p_d - G^T p_y - H^T (p_z - Sigma_s H p_d).
// Every product here walks the Jacobian values J stored per bus-adjacency
// slot (and the line-flow rows' HF), in a fixed order: thread per
// (scenario, row).  The refinement is judged by a normwise backward error:
// max |rho| over the largest magnitude among the right-hand side and the
// products A_block p of each row (r, K p_d, G^T p_y + H^T t, G p_d, H p_d,
// Sigma_s p_s, p_z, ...); both maxima are gathered by atomic maxima of the
// magnitudes' bit patterns (order-independent, so the result is
// deterministic).
#include "dev.cuh"
#include "kernels.h"

namespace {

// multiplier of the (bus i, component c) injection row in scenario sc: the g
// row takes ly (y-like vector [N][nx], may be null = 0), the h row lz ([N][m])
__device__ __forceinline__ double row_mult(const DevSym &S, const double *ly, const double *lz, int sc, int i,
                                           int c) {
  if (c == 0) {
    if (i >= 1) return ly ? ly[(size_t)sc * S.nx + S.xth[i]] : 0.0;
    return lz[(size_t)sc * S.m + S.ng];
  }
  const int q = S.xv[i];
  if (q >= 0) return ly ? ly[(size_t)sc * S.nx + q] : 0.0;
  return lz[(size_t)sc * S.m + S.gen_of_bus[i]];
}

// (G^T ly + H^T lz) at bus variable (a, kind) of scenario sc: every row
// (i, c) with i adjacent to a (or a itself) contributes dF_(i,c)/d(a,kind)
// times its multiplier, and so does every line-flow row with an end at a.
// The Pg columns are handled by the callers.
__device__ __forceinline__ double jt_at(const DevSym &S, const DevWork &D, const double *ly, const double *lz,
                                        int sc, int a, int kind) {
  double acc = 0.0;
  for (int q = S.a_ptr[a]; q < S.a_ptr[a + 1]; ++q) {
    const int i = S.a_col[q], tq = S.a_tslot[q];
    acc += D.J[((size_t)tq * 4 + 0 * 2 + kind) * S.N + sc] * row_mult(S, ly, lz, sc, i, 0);
    acc += D.J[((size_t)tq * 4 + 1 * 2 + kind) * S.N + sc] * row_mult(S, ly, lz, sc, i, 1);
  }
  if (S.nflow)
    for (int e = S.ht_ptr[a]; e < S.ht_ptr[a + 1]; ++e) {
      const int r = S.ht_r[e];
      if (S.hrow_comp[r] < 2) continue;
      acc += D.HF[((size_t)S.ht_aslot[e] * 2 + kind) * S.N + sc] * lz[(size_t)sc * S.m + r];
    }
  return acc;
}

// (H p_d) of line-flow row f of scenario sc
__device__ __forceinline__ double flowrow(const DevSym &S, const double *HF, const double *px, const double *pu,
                                          int sc, int f, int own) {
  double acc = 0.0;
  for (int w = 0; w < 2; ++w) {
    const int b = w == 0 ? own : flow_other(S, f);
    const double pth = b >= 1 ? px[(size_t)sc * S.nx + S.xth[b]] : 0.0;
    const double pv = S.xv[b] >= 0 ? px[(size_t)sc * S.nx + S.xv[b]] : pu[S.uv[b]];
    acc += HF[((size_t)(f * 2 + w) * 2 + 0) * S.N + sc] * pth + HF[((size_t)(f * 2 + w) * 2 + 1) * S.N + sc] * pv;
  }
  return acc;
}

// (G p_d) or (H p_d) of row (bus i, component c) of scenario sc
__device__ __forceinline__ double jrow(const DevSym &S, const double *J, const double *px, const double *pu, int sc,
                                       int i, int c) {
  double acc = 0.0;
  for (int q = S.a_ptr[i]; q < S.a_ptr[i + 1]; ++q) {
    const int b = S.a_col[q];
    const double pth = b >= 1 ? px[(size_t)sc * S.nx + S.xth[b]] : 0.0;
    const double pv = S.xv[b] >= 0 ? px[(size_t)sc * S.nx + S.xv[b]] : pu[S.uv[b]];
    acc += J[((size_t)q * 4 + c * 2 + 0) * S.N + sc] * pth + J[((size_t)q * 4 + c * 2 + 1) * S.N + sc] * pv;
  }
  const int gk = S.gen_of_bus[i];
  if (c == 0 && i >= 1 && gk >= 1) acc -= pu[S.ng + gk - 1];  // dP_i/dPg = -1 in the g row
  return acc;
}

// out[0] = max(out[0], max |a| over the warp), out[1] likewise for b; every
// lane of the warp calls it (out-of-range lanes with zeros)
__device__ __forceinline__ void warp_max2(double a, double b, unsigned long long *out) {
  unsigned long long ma = __double_as_longlong(fabs(a)), mb = __double_as_longlong(fabs(b));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oa = __shfl_down_sync(0xffffffffu, ma, o);
    const unsigned long long ob = __shfl_down_sync(0xffffffffu, mb, o);
    ma = oa > ma ? oa : ma;
    mb = ob > mb ? ob : mb;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], ma);
    atomicMax(&out[1], mb);
  }
}

// h rows: Hp, rho_s, rho_z and tw = p_z - Sigma_s Hp
__global__ void k_res_h(DevSym S, DevWork D, const double *px, const double *pu, const double *ps,
                        const double *pz, double *Hp, double *rho2, double *rho4, double *tw,
                        unsigned long long *amax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double res = 0.0, scl = 0.0;
  if (t < (long long)S.N * S.m) {
    const int sc = (int)(t / S.m), r = (int)(t - (long long)sc * S.m);
    const double hp = S.hrow_comp[r] < 2 ? jrow(S, D.J, px, pu, sc, S.hrow_bus[r], S.hrow_comp[r])
                                         : flowrow(S, D.HF, px, pu, sc, r - S.ng - 1, S.hrow_bus[r]);
    Hp[t] = hp;
    const double sps = D.Ss[t] * ps[t];
    const double r2 = -D.r2[t] - sps - pz[t], r4 = -D.r4[t] - hp - ps[t];
    rho2[t] = r2;
    rho4[t] = r4;
    tw[t] = pz[t] - D.Ss[t] * hp;
    res = fmax(fabs(r2), fabs(r4));
    scl = fmax(fmax(fmax(fabs(D.r2[t]), fabs(sps)), fmax(fabs(pz[t]), fabs(D.r4[t]))), fmax(fabs(hp), fabs(ps[t])));
  }
  warp_max2(res, scl, amax);
}

// x rows (state order): rho_y = -g - G p_d and
// rho_1x = -r1x - K p_d - delta p_x - G_x^T p_y - H_x^T tw; the threads past
// the x rows form the per-scenario terms of the u rows, upart[s][j] =
// kpu_s,j + (G_u^T p_y,s + H_u^T tw_s)_j and the largest magnitude of its
// terms umag[s][j] (summed over scenarios by k_res_u)
__global__ void k_res_x(DevSym S, DevWork D, double delta, const double *px, const double *pu, const double *py,
                        const double *tw, const double *kpx_pos, const double *kpu, double *rho1x, double *rho3,
                        double *upart, double *umag, unsigned long long *amax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long NX = (long long)S.N * S.nx;
  double res = 0.0, scl = 0.0;
  if (t >= NX && t < NX + (long long)S.N * S.nu) {
    const long long q = t - NX;
    const int sc = (int)(q / S.nu), j = (int)(q - (long long)sc * S.nu);
    const double kq = kpu[q];
    double jt;
    if (j < S.ng) jt = jt_at(S, D, py, tw, sc, S.hrow_bus[j], 1);   // v at generator j's bus
    else jt = -row_mult(S, py, tw, sc, S.hrow_bus[j - S.ng + 1], 0);  // Pg: -1 in the P row
    upart[q] = kq + jt;
    umag[q] = fmax(fabs(kq), fabs(jt));
  }
  if (t < NX) {
    const int sc = (int)(t / S.nx), j = (int)(t - (long long)sc * S.nx);
    const int a = S.xbus[j], kind = S.xkind[j];
    const double gp = jrow(S, D.J, px, pu, sc, a, kind);
    const double r3 = -D.g[t] - gp;
    rho3[t] = r3;
    const double kp = kpx_pos[(size_t)sc * S.nx + S.perm[j]];
    const double jt = jt_at(S, D, py, tw, sc, a, kind);
    const double r1 = -D.r1x[t] - kp - delta * px[t] - jt;
    rho1x[t] = r1;
    res = fmax(fabs(r1), fabs(r3));
    scl = fmax(fmax(fmax(fabs(D.r1x[t]), fabs(kp)), fmax(fabs(delta * px[t]), fabs(jt))),
               fmax(fabs(D.g[t]), fabs(gp)));
  }
  warp_max2(res, scl, amax);
}

// u rows (scenarios summed in index order):
// rho_1u = -r1u - (sum_i kpu_i + diag1 p_u) - delta p_u - sum_i (G_u^T p_y,i + H_u^T tw_i)
__global__ void k_res_u(DevSym S, DevWork D, double delta, const double *pu, const double *upart,
                        const double *umag, const double *diag1, double *rho1u, unsigned long long *amax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double res = 0.0, scl = 0.0;
  if (j < S.nu) {
    double acc = 0.0, mag = 0.0;
    for (int sc = 0; sc < S.N; ++sc) {
      acc += upart[(size_t)sc * S.nu + j];
      mag = fmax(mag, umag[(size_t)sc * S.nu + j]);
    }
    const double dp = (diag1[j] + delta) * pu[j];
    const double r1 = -D.r1u[j] - acc - dp;
    rho1u[j] = r1;
    res = fabs(r1);
    scl = fmax(fmax(fabs(D.r1u[j]), mag), fmax(fabs(acc), fabs(dp)));
  }
  warp_max2(res, scl, amax);
}

// x rows of H^T v (state order): out = a + H_x^T v   (v [N][m])
__global__ void k_htv_x(DevSym S, DevWork D, const double *a, const double *v, double *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.N * S.nx) return;
  const int sc = (int)(t / S.nx), j = (int)(t - (long long)sc * S.nx);
  out[t] = a[t] + jt_at(S, D, nullptr, v, sc, S.xbus[j], S.xkind[j]);
}

// u rows of the same: part[s][j] = (H_u^T v_s)_j (thread per (scenario, u
// row)), then out = a + sum_s part[s] (scenarios in index order)
__global__ void k_htv_upart(DevSym S, DevWork D, const double *v, double *part) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)S.N * S.nu) return;
  const int sc = (int)(q / S.nu), j = (int)(q - (long long)sc * S.nu);
  part[q] = j < S.ng ? jt_at(S, D, nullptr, v, sc, S.hrow_bus[j], 1)
                     : -row_mult(S, nullptr, v, sc, S.hrow_bus[j - S.ng + 1], 0);
}
__global__ void k_htv_u(DevSym S, const double *a, const double *part, double *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = 0.0;
  for (int sc = 0; sc < S.N; ++sc) acc += part[(size_t)sc * S.nu + j];
  out[j] = a[j] + acc;
}

// slack rows of a correction: t = Sigma_s r4 - r2 (condensed right-hand side)
__global__ void k_tv(long long n, const double *Ss, const double *r2, const double *r4, double *t) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = Ss[i] * r4[i] - r2[i];
}

// recovery of a correction's slack blocks (Prop. 2.1 with right-hand side r):
// pz = Sigma_s (H p_d + r4) - r2, ps = -(r2 + pz) / Sigma_s
__global__ void k_pzps_rhs(DevSym S, DevWork D, const double *px, const double *pu, const double *r2,
                           const double *r4, double *pz, double *ps) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.N * S.m) return;
  const int sc = (int)(t / S.m), r = (int)(t - (long long)sc * S.m);
  const double hp = S.hrow_comp[r] < 2 ? jrow(S, D.J, px, pu, sc, S.hrow_bus[r], S.hrow_comp[r])
                                       : flowrow(S, D.HF, px, pu, sc, r - S.ng - 1, S.hrow_bus[r]);
  const double z = D.Ss[t] * (hp + r4[t]) - r2[t];
  pz[t] = z;
  ps[t] = -(r2[t] + z) / D.Ss[t];
}

// out[0] = max |a|, out[1] = max |b| over n elements (non-negative doubles
// compare like their bit patterns; a NaN orders above every finite value)
__global__ void k_maxabs2(long long n, const double *a, const double *b, unsigned long long *out) {
  unsigned long long ma = 0, mb = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long va = __double_as_longlong(fabs(a[i]));
    const unsigned long long vb = __double_as_longlong(fabs(b[i]));
    ma = va > ma ? va : ma;
    mb = vb > mb ? vb : mb;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oa = __shfl_down_sync(0xffffffffu, ma, o);
    const unsigned long long ob = __shfl_down_sync(0xffffffffu, mb, o);
    ma = oa > ma ? oa : ma;
    mb = ob > mb ? ob : mb;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], ma);
    atomicMax(&out[1], mb);
  }
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_aug_residual(const DevSym &S, const DevWork &D, double delta, const double *px, const double *pu,
                         const double *ps, const double *py, const double *pz, const double *kpx_pos,
                         const double *kpu, const double *diag1, double *Hp, double *tw, double *rho1x,
                         double *rho1u, double *rho2, double *rho3, double *rho4, double *upart, double *umag,
                         unsigned long long *amax, cudaStream_t st) {
  const long long NX = (long long)S.N * S.nx, NM = (long long)S.N * S.m;
  k_res_h<<<nblk(NM, 256), 256, 0, st>>>(S, D, px, pu, ps, pz, Hp, rho2, rho4, tw, amax); ipm_count_launch();
  const long long NU = (long long)S.N * S.nu;
  k_res_x<<<nblk(NX + NU, 256), 256, 0, st>>>(S, D, delta, px, pu, py, tw, kpx_pos, kpu, rho1x, rho3, upart, umag,
                                               amax);
  ipm_count_launch();
  k_res_u<<<nblk(S.nu, 128), 128, 0, st>>>(S, D, delta, pu, upart, umag, diag1, rho1u, amax); ipm_count_launch();
}

void launch_htv(const DevSym &S, const DevWork &D, const double *ax, const double *au, const double *v, double *outx,
                double *outu, double *upart, cudaStream_t st) {
  const long long NX = (long long)S.N * S.nx, NU = (long long)S.N * S.nu;
  k_htv_x<<<nblk(NX, 256), 256, 0, st>>>(S, D, ax, v, outx); ipm_count_launch();
  k_htv_upart<<<nblk(NU, 256), 256, 0, st>>>(S, D, v, upart); ipm_count_launch();
  k_htv_u<<<nblk(S.nu, 128), 128, 0, st>>>(S, au, upart, outu); ipm_count_launch();
}

void launch_tv(long long n, const double *Ss, const double *r2, const double *r4, double *t, cudaStream_t st) {
  k_tv<<<nblk(n, 256), 256, 0, st>>>(n, Ss, r2, r4, t); ipm_count_launch();
}

void launch_pzps_rhs(const DevSym &S, const DevWork &D, const double *px, const double *pu, const double *r2,
                     const double *r4, double *pz, double *ps, cudaStream_t st) {
  const long long NM = (long long)S.N * S.m;
  k_pzps_rhs<<<nblk(NM, 256), 256, 0, st>>>(S, D, px, pu, r2, r4, pz, ps); ipm_count_launch();
}

void launch_maxabs2(long long n, const double *a, const double *b, unsigned long long *out, cudaStream_t st) {
  const int blocks = (int)std::min<long long>(nblk(n, 256), 152 * 4);
  k_maxabs2<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(n, a, b, out); ipm_count_launch();
}
