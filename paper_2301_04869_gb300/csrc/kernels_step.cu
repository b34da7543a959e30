// K8/K9: step recovery (Props. 2.1, 2.3), bound-dual steps, and the scalar
// reductions of one interior-point iteration (optimality error, merit value,
// directional derivative, fraction to boundary).
//
// All reductions run on a fixed grid with a fixed assignment of indices to
// threads and a fixed combination tree, so repeated runs give identical bits.
#include <atomic>

#include "dev.cuh"
#include "kernels.h"


namespace {

enum { OP_SUM = 0, OP_MAX = 1, OP_MIN = 2 };
constexpr int RED_BLOCKS = 152;

__device__ __forceinline__ double op_init(int op) {
  return op == OP_SUM ? 0.0 : (op == OP_MAX ? -INFINITY : INFINITY);
}
__device__ __forceinline__ double op_comb(int op, double a, double b) {
  return op == OP_SUM ? a + b : (op == OP_MAX ? fmax(a, b) : fmin(a, b));
}
__device__ __forceinline__ double warp_op(int op, double v) {
  for (int o = 16; o > 0; o >>= 1) v = op_comb(op, v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

template <class F>
__global__ void __launch_bounds__(256) k_reduce(F f, long long n, double *partial) {
  double acc[F::NV];
#pragma unroll
  for (int i = 0; i < F::NV; ++i) acc[i] = op_init(F::op(i));
  for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < n; t += (long long)gridDim.x * 256)
    f(t, acc);
  __shared__ double sh[F::NV][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < F::NV; ++i) {
    const double v = warp_op(F::op(i), acc[i]);
    if (lane == 0) sh[i][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < F::NV) {
    const int i = threadIdx.x;
    double v = sh[i][0];
    for (int q = 1; q < 8; ++q) v = op_comb(F::op(i), v, sh[i][q]);
    partial[(size_t)blockIdx.x * F::NV + i] = v;
  }
}

template <class F>
__global__ void k_reduce_final(int nb, const double *partial, double *out) {
  const int i = threadIdx.x;
  if (i >= F::NV) return;
  double v = partial[i];
  for (int b = 1; b < nb; ++b) v = op_comb(F::op(i), v, partial[(size_t)b * F::NV + i]);
  out[i] = v;
}

template <class F>
void run_reduce(const F &f, long long n, double *partial, double *out, cudaStream_t st) {
  k_reduce<F><<<RED_BLOCKS, 256, 0, st>>>(f, n, partial); ipm_count_launch();
  k_reduce_final<F><<<1, 32, 0, st>>>(RED_BLOCKS, partial, out); ipm_count_launch();
}

__device__ __forceinline__ double bgrad(double w, double l, double b, double mu) {
  double r = 0.0;
  if (isfinite(l)) r -= mu / (w - l);
  if (isfinite(b)) r += mu / (b - w);
  return r;
}
__device__ __forceinline__ double blog(double w, double l, double b) {
  double r = 0.0;
  if (isfinite(l)) r += log(w - l);
  if (isfinite(b)) r += log(b - w);
  return r;
}

// optimality error pieces: dual max, primal max, compl max, compl min,
// sum |y|+|z|, sum |bound duals|, sum of complementarity products
struct ErrF {
  static constexpr int NV = 7;
  __device__ static int op(int i) { return i == 3 ? OP_MIN : (i >= 4 ? OP_SUM : OP_MAX); }
  DevSym S;
  DevWork D;
  const double *gLu;
  __device__ void compl_of(double w, double l, double b, double zl, double zu, double *acc) const {
    if (isfinite(l)) { const double c = zl * (w - l); acc[2] = fmax(acc[2], c); acc[3] = fmin(acc[3], c); acc[5] += fabs(zl); acc[6] += c; }
    if (isfinite(b)) { const double c = zu * (b - w); acc[2] = fmax(acc[2], c); acc[3] = fmin(acc[3], c); acc[5] += fabs(zu); acc[6] += c; }
  }
  __device__ void operator()(long long t, double *acc) const {
    const long long nX = (long long)S.N * S.nx, nS = (long long)S.N * S.m;
    if (t < nX) {
      const int sc = (int)(t / S.nx), j = (int)(t - (long long)sc * S.nx);
      const double gl = D.JTl[(size_t)sc * 2 * S.n + S.xkind[j] * S.n + S.xbus[j]] - D.zlx[t] + D.zux[t];
      acc[0] = fmax(acc[0], fabs(gl));
      acc[1] = fmax(acc[1], fabs(D.g[t]));
      acc[4] += fabs(D.y[t]);
      compl_of(D.x[t], S.xl[j], S.xu[j], D.zlx[t], D.zux[t], acc);
    } else if (t < nX + nS) {
      const long long q = t - nX;
      const int j = (int)(q % S.m);
      acc[0] = fmax(acc[0], fabs(D.z[q] - D.zls[q] + D.zus[q]));
      acc[1] = fmax(acc[1], fabs(D.h[q] + D.s[q]));
      acc[4] += fabs(D.z[q]);
      compl_of(D.s[q], S.sl[j], S.su[j], D.zls[q], D.zus[q], acc);
    } else {
      const int j = (int)(t - nX - nS);
      acc[0] = fmax(acc[0], fabs(gLu[j] - D.zlu[j] + D.zuu[j]));
      compl_of(D.u[j], S.ul[j], S.uu[j], D.zlu[j], D.zuu[j], acc);
    }
  }
};

// merit pieces at a primal point (x, u, s) whose g, h, fs were evaluated:
// objective, sum of logs (barrier / -mu), ||c||_1
struct MeritF {
  static constexpr int NV = 3;
  __device__ static int op(int) { return OP_SUM; }
  DevSym S;
  const double *x, *u, *s, *g, *h, *fs;
  __device__ void operator()(long long t, double *acc) const {
    const long long nX = (long long)S.N * S.nx, nS = (long long)S.N * S.m;
    if (t < nX) {
      const int j = (int)(t % S.nx);
      acc[1] += blog(x[t], S.xl[j], S.xu[j]);
      acc[2] += fabs(g[t]);
    } else if (t < nX + nS) {
      const long long q = t - nX;
      const int j = (int)(q % S.m);
      acc[1] += blog(s[q], S.sl[j], S.su[j]);
      acc[2] += fabs(h[q] + s[q]);
    } else if (t < nX + nS + S.nu) {
      const int j = (int)(t - nX - nS);
      acc[1] += blog(u[j], S.ul[j], S.uu[j]);
      if (j >= S.ng) {
        const int k = j - S.ng + 1;
        acc[0] += S.c2[k] * u[j] * u[j] + S.c1[k] * u[j];
      }
    } else {
      acc[0] += fs[t - nX - nS - S.nu];
    }
  }
};

// directional derivative pieces after a step: grad(phi_mu)^T p, the
// curvature q = p^T (W + Sigma + delta I) p (+ slacks), ||c||_1 of the
// linearised constraints (r3, r4)
struct DirF {
  static constexpr int NV = 3;
  __device__ static int op(int) { return OP_SUM; }
  DevSym S;
  DevWork D;
  const double *px, *pu, *ps, *kpx, *kpu, *Hp;  // px x-order; kpx position order
  double mu, delta;
  __device__ void operator()(long long t, double *acc) const {
    const long long nX = (long long)S.N * S.nx, nS = (long long)S.N * S.m, nUS = (long long)S.N * S.nu;
    if (t < nX) {
      const int sc = (int)(t / S.nx), p = (int)(t - (long long)sc * S.nx);
      const int j = S.iperm[p];
      const size_t xi = (size_t)sc * S.nx + j;
      acc[0] += bgrad(D.x[xi], S.xl[j], S.xu[j], mu) * px[xi];
      acc[1] += px[xi] * (kpx[t] + delta * px[xi]);
      acc[2] += fabs(D.g[xi]);
    } else if (t < nX + nS) {
      const long long q = t - nX;
      const int sc = (int)(q / S.m), r = (int)(q % S.m);
      acc[0] += bgrad(D.s[q], S.sl[r], S.su[r], mu) * ps[q];
      if (r == S.ng) {
        const double pg0 = D.h[q];
        acc[0] += (2.0 * S.c2[0] * pg0 + S.c1[0]) / S.N * Hp[q];
      }
      acc[1] += D.Ss[q] * (ps[q] * ps[q] - Hp[q] * Hp[q]);
      acc[2] += fabs(D.r4[q]);
      (void)sc;
    } else if (t < nX + nS + nUS) {
      const long long q = t - nX - nS;
      const int j = (int)(q % S.nu);
      acc[1] += pu[j] * kpu[q];
    } else {
      const int j = (int)(t - nX - nS - nUS);
      acc[0] += bgrad(D.u[j], S.ul[j], S.uu[j], mu) * pu[j];
      double d = D.Su[j] + delta;
      if (j >= S.ng) {
        const int k = j - S.ng + 1;
        acc[0] += (2.0 * S.c2[k] * D.u[j] + S.c1[k]) * pu[j];
        d += 2.0 * S.c2[k];
      }
      acc[1] += pu[j] * d * pu[j];
    }
  }
};

// largest primal / dual steps keeping tau of the distance to the bounds
struct FtbF {
  static constexpr int NV = 2;
  __device__ static int op(int) { return OP_MIN; }
  DevSym S;
  DevWork D;
  const double *px, *pu, *ps, *dzlx, *dzux, *dzlu, *dzuu, *dzls, *dzus;
  double tau;
  __device__ void prim(double w, double dw, double l, double b, double *acc) const {
    if (isfinite(l) && dw < 0) acc[0] = fmin(acc[0], -tau * (w - l) / dw);
    if (isfinite(b) && dw > 0) acc[0] = fmin(acc[0], tau * (b - w) / dw);
  }
  __device__ void dual(double z, double dz, bool fin, double *acc) const {
    if (fin && dz < 0) acc[1] = fmin(acc[1], -tau * z / dz);
  }
  __device__ void operator()(long long t, double *acc) const {
    const long long nX = (long long)S.N * S.nx, nS = (long long)S.N * S.m;
    if (t < nX) {
      const int j = (int)(t % S.nx);
      prim(D.x[t], px[t], S.xl[j], S.xu[j], acc);
      dual(D.zlx[t], dzlx[t], isfinite(S.xl[j]), acc);
      dual(D.zux[t], dzux[t], isfinite(S.xu[j]), acc);
    } else if (t < nX + nS) {
      const long long q = t - nX;
      const int j = (int)(q % S.m);
      prim(D.s[q], ps[q], S.sl[j], S.su[j], acc);
      dual(D.zls[q], dzls[q], isfinite(S.sl[j]), acc);
      dual(D.zus[q], dzus[q], isfinite(S.su[j]), acc);
    } else {
      const int j = (int)(t - nX - nS);
      prim(D.u[j], pu[j], S.ul[j], S.uu[j], acc);
      dual(D.zlu[j], dzlu[j], isfinite(S.ul[j]), acc);
      dual(D.zuu[j], dzuu[j], isfinite(S.uu[j]), acc);
    }
  }
};

__global__ void k_gather_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * nx) return;
  const int sc = (int)(t / nx), p = (int)(t - (long long)sc * nx);
  dst[t] = scale * src[(size_t)sc * nx + iperm[p]];
}
__global__ void k_scatter_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * nx) return;
  const int sc = (int)(t / nx), p = (int)(t - (long long)sc * nx);
  dst[(size_t)sc * nx + iperm[p]] = scale * src[t];
}

// v[s][p] += sum_j G_u[p, j] pu[j]     (position rows)
__global__ void k_gu_apply(DevSym S, const double *J, const double *pu, double *v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.N * S.nx) return;
  const int sc = (int)(t / S.nx), p = (int)(t - (long long)sc * S.nx);
  double acc = v[t];
  for (int e = S.gu_ptr[p]; e < S.gu_ptr[p + 1]; ++e) {
    const int src = S.gu_src[e];
    acc += (src >= 0 ? J[(size_t)src * S.N + sc] : -1.0) * pu[S.gu_col[e]];
  }
  v[t] = acc;
}

// kpx = K_xx px (+ K_xu pu);  kpu = K_ux px + K_uu pu  (position rows, u rows)
__global__ void k_kapply(DevSym S, const double *K, const double *px_pos, const double *pu,
                         double *kpx, double *kpu) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nX = (long long)S.N * S.nx;
  if (t < nX) {
    const int sc = (int)(t / S.nx), p = (int)(t - (long long)sc * S.nx);
    double acc = 0.0;
    for (int e = S.kx_ptr[p]; e < S.kx_ptr[p + 1]; ++e) {
      const int col = S.kx_col[e];
      const double v = K[(size_t)S.kx_src[e] * S.N + sc];
      if (col < S.nx) acc += v * px_pos[(size_t)sc * S.nx + col];
      else if (pu) acc += v * pu[col - S.nx];
    }
    kpx[t] = acc;
  } else if (kpu && t < nX + (long long)S.N * S.nu) {
    const long long q = t - nX;
    const int sc = (int)(q / S.nu), j = (int)(q - (long long)sc * S.nu);
    double acc = 0.0;
    for (int e = S.ku_ptr[j]; e < S.ku_ptr[j + 1]; ++e) {
      const int col = S.ku_col[e];
      const double v = K[(size_t)S.ku_src[e] * S.N + sc];
      acc += v * (col < S.nx ? px_pos[(size_t)sc * S.nx + col] : pu[col - S.nx]);
    }
    kpu[q] = acc;
  }
}

__global__ void k_lincomb(long long n, double *out, double a, const double *x, double b,
                          const double *y, double c, const double *z) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v = 0.0;
  if (x) v += a * x[t];
  if (y) v += b * y[t];
  if (z) v += c * z[t];
  out[t] = v;
}

// reduced right-hand side, eq. (11):
//   rhs_u = -rhat2 + sum_s [ G_u^T G_x^{-T}(rhat1 - K_xx G_x^{-1} r3) + K_ux G_x^{-1} r3 ]
// with a = G_x^{-T}(rhat1 - K_xx b), b = G_x^{-1} r3 (position order)
__global__ void k_rhs_reduced(DevSym S, const double *J, const double *K, const double *rh2,
                              const double *a, const double *b, double *rhs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = -rh2[j];
  for (int sc = 0; sc < S.N; ++sc) {
    for (int e = S.gut_ptr[j]; e < S.gut_ptr[j + 1]; ++e) {
      const int src = S.gut_src[e];
      acc += (src >= 0 ? J[(size_t)src * S.N + sc] : -1.0) * a[(size_t)sc * S.nx + S.gut_col[e]];
    }
    for (int e = S.ku_ptr[j]; e < S.ku_ptr[j + 1]; ++e) {
      const int col = S.ku_col[e];
      if (col < S.nx) acc += K[(size_t)S.ku_src[e] * S.N + sc] * b[(size_t)sc * S.nx + col];
    }
  }
  rhs[j] = acc;
}

// part[s][j] = alpha (Z_s^T w_s)[j] (+ (K_ux,s b_s)[j] when b != null).
// CTA per (scenario, 32 columns): lane = column (coalesced row segments of
// Z), the 8 warps take every 8th row, a fixed-order shared-memory sum joins
// them.
__global__ void __launch_bounds__(256) k_zt_part(DevSym S, const double *__restrict__ Z,
                                                 const double *__restrict__ w, const double *__restrict__ K,
                                                 const double *__restrict__ b, double alpha, double *part) {
  __shared__ double red[8][33];
  const int sc = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const double *Zs = Z + (size_t)sc * S.nx * S.nu;
  const double *ws = w + (size_t)sc * S.nx;
  double acc = 0.0;
  if (j < S.nu)
    for (int p = warp; p < S.nx; p += 8) acc += Zs[(size_t)p * S.nu + j] * ws[p];
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && j < S.nu) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    t *= alpha;
    if (b)
      for (int e = S.ku_ptr[j]; e < S.ku_ptr[j + 1]; ++e) {
        const int col = S.ku_col[e];
        if (col < S.nx) t += K[(size_t)S.ku_src[e] * S.N + sc] * b[(size_t)sc * S.nx + col];
      }
    part[(size_t)sc * S.nu + j] = t;
  }
}

// out[j] = beta*out[j] + sum_s part[s][j]  (scenarios in index order);
// beta = 0 does not read out (it may hold anything, NaN included)
__global__ void k_zt_sum(DevSym S, const double *part, double beta, double *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = 0.0;
  for (int sc = 0; sc < S.N; ++sc) acc += part[(size_t)sc * S.nu + j];
  out[j] = beta == 0.0 ? acc : beta * out[j] + acc;
}

// v[s][p] = a * v[s][p] + (Z_s pu)[p]   (position rows)
__global__ void k_z_apply(DevSym S, const double *__restrict__ Z, const double *__restrict__ pu, double a,
                          double *v) {
  const int lane = threadIdx.x & 31;
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= (long long)S.N * S.nx) return;
  const double *Zr = Z + (size_t)row * S.nu;
  double part = 0.0;
  for (int j = lane; j < S.nu; j += 32) part += Zr[j] * pu[j];
  part = warp_sum(part);
  if (lane == 0) v[row] = (a == 0.0 ? 0.0 : a * v[row]) + part;
}

// out[j] = scale * sum_s (G_u^T a_s)[j]   (a in position order)
__global__ void k_gut_sum(DevSym S, const double *J, const double *a, double scale, double *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = 0.0;
  for (int sc = 0; sc < S.N; ++sc)
    for (int e = S.gut_ptr[j]; e < S.gut_ptr[j + 1]; ++e) {
      const int src = S.gut_src[e];
      acc += (src >= 0 ? J[(size_t)src * S.N + sc] : -1.0) * a[(size_t)sc * S.nx + S.gut_col[e]];
    }
  out[j] = scale * acc;
}

// out[j] += sum_s kpu[s][j] + (diag[j] + delta) v[j]   (scenarios in index order)
__global__ void k_apply_finish(DevSym S, const double *kpu, const double *diag, double delta, const double *v,
                               double *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = out[j];
  for (int sc = 0; sc < S.N; ++sc) acc += kpu[(size_t)sc * S.nu + j];
  out[j] = acc + (diag[j] + delta) * v[j];
}

// out[0] = a.b, out[1] = c.d (one block, fixed partition and tree)
__global__ void k_dot2(int n, const double *a, const double *b, const double *c, const double *d, double *out) {
  __shared__ double sh[2][32];
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s0 += a[i] * b[i];
    if (c) s1 += c[i] * d[i];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sh[0][w] = s0; sh[1][w] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { t0 += sh[0][q]; t1 += sh[1][q]; }
    out[0] = t0;
    out[1] = t1;
  }
}

// Hp = H_x p_x + H_u p_u; p_z = Sigma_s (Hp + r4) - r2; p_s = -(r2 + p_z)/Sigma_s
__global__ void k_pz_ps(DevSym S, DevWork D, const double *px, const double *pu, double *Hp,
                        double *pz, double *ps) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.N * S.m) return;
  const int sc = (int)(t / S.m), r = (int)(t - (long long)sc * S.m);
  const int gb = S.hrow_bus[r], c = S.hrow_comp[r];
  double acc = 0.0;
  if (c < 2) {
    for (int q = S.a_ptr[gb]; q < S.a_ptr[gb + 1]; ++q) {
      const int b = S.a_col[q];
      const double pth = b >= 1 ? px[(size_t)sc * S.nx + S.xth[b]] : 0.0;
      const double pv = S.xv[b] >= 0 ? px[(size_t)sc * S.nx + S.xv[b]] : pu[S.uv[b]];
      acc += D.J[((size_t)q * 4 + c * 2 + 0) * S.N + sc] * pth + D.J[((size_t)q * 4 + c * 2 + 1) * S.N + sc] * pv;
    }
  } else {  // line-flow row: its two end buses
    const int f = r - S.ng - 1;
    for (int w = 0; w < 2; ++w) {
      const int b = w == 0 ? gb : flow_other(S, f);
      const double pth = b >= 1 ? px[(size_t)sc * S.nx + S.xth[b]] : 0.0;
      const double pv = S.xv[b] >= 0 ? px[(size_t)sc * S.nx + S.xv[b]] : pu[S.uv[b]];
      acc += D.HF[((size_t)(f * 2 + w) * 2 + 0) * S.N + sc] * pth + D.HF[((size_t)(f * 2 + w) * 2 + 1) * S.N + sc] * pv;
    }
  }
  Hp[t] = acc;
  const double z = D.Ss[t] * (acc + D.r4[t]) - D.r2[t];
  pz[t] = z;
  ps[t] = -(D.r2[t] + z) / D.Ss[t];
}

// bound-dual steps dzl = mu/(w-l) - zl - Sigma_l dw, dzu = mu/(b-w) - zu + Sigma_u dw
__global__ void k_bound_steps(long long n, int period, const double *w, const double *dw, const double *l,
                              const double *b, const double *zl, const double *zu, double mu,
                              double *dzl, double *dzu) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = (int)(t % period);
  if (isfinite(l[j])) {
    const double d = w[t] - l[j];
    dzl[t] = mu / d - zl[t] - zl[t] / d * dw[t];
  } else {
    dzl[t] = 0.0;
  }
  if (isfinite(b[j])) {
    const double d = b[j] - w[t];
    dzu[t] = mu / d - zu[t] + zu[t] / d * dw[t];
  } else {
    dzu[t] = 0.0;
  }
}

// bound duals after the step, kept within [mu/(ks d), ks mu/d]
__global__ void k_dual_update(long long n, int period, const double *w, const double *l, const double *b,
                              double *zl, double *zu, const double *dzl, const double *dzu, double az,
                              double mu, double ks) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = (int)(t % period);
  if (isfinite(l[j])) {
    const double d = w[t] - l[j];
    zl[t] = fmax(fmin(zl[t] + az * dzl[t], ks * mu / d), mu / (ks * d));
  } else {
    zl[t] = 0.0;
  }
  if (isfinite(b[j])) {
    const double d = b[j] - w[t];
    zu[t] = fmax(fmin(zu[t] + az * dzu[t], ks * mu / d), mu / (ks * d));
  } else {
    zu[t] = 0.0;
  }
}

// w = clip(w, l + push_l, b - push_b) with the starting-point push rule
__global__ void k_push(long long n, int period, double *w, const double *l, const double *b, double k1,
                       double k2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = (int)(t % period);
  const double lj = l[j], bj = b[j];
  const bool fl = isfinite(lj), fb = isfinite(bj);
  double pl = fl ? k1 * fmax(1.0, fabs(lj)) : 0.0;
  double pb = fb ? k1 * fmax(1.0, fabs(bj)) : 0.0;
  if (fl && fb) {
    pl = fmin(pl, k2 * (bj - lj));
    pb = fmin(pb, k2 * (bj - lj));
  }
  double v = w[t];
  if (fl) v = fmax(v, lj + pl);
  if (fb) v = fmin(v, bj - pb);
  w[t] = v;
}

__global__ void k_init_primal(DevSym S, double *x, double *u, const double *pmax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nX = (long long)S.N * S.nx;
  if (t < nX) {
    const int j = (int)(t % S.nx);
    x[t] = S.xkind[j] == 0 ? 0.0 : 1.0;
  } else if (t < nX + S.nu) {
    const int j = (int)(t - nX);
    u[j] = j < S.ng ? 1.0 : 0.5 * pmax[j - S.ng + 1];
  }
}

__global__ void k_fill_bound_duals(long long n, int period, const double *l, const double *b, double *zl,
                                   double *zu) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = (int)(t % period);
  zl[t] = isfinite(l[j]) ? 1.0 : 0.0;
  zu[t] = isfinite(b[j]) ? 1.0 : 0.0;
}

}  // namespace

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

void launch_errors(const DevSym &S, DevWork &D, const double *gLu, double *partial, double *out,
                   cudaStream_t st) {
  ErrF f{S, D, gLu};
  run_reduce(f, (long long)S.N * S.nx + (long long)S.N * S.m + S.nu, partial, out, st);
}
void launch_merit(const DevSym &S, const double *x, const double *u, const double *s, const double *g,
                  const double *h, const double *fs, double *partial, double *out, cudaStream_t st) {
  MeritF f{S, x, u, s, g, h, fs};
  run_reduce(f, (long long)S.N * S.nx + (long long)S.N * S.m + S.nu + S.N, partial, out, st);
}
void launch_dir(const DevSym &S, DevWork &D, const double *px, const double *pu, const double *ps,
                const double *kpx, const double *kpu, const double *Hp, double mu, double delta,
                double *partial, double *out, cudaStream_t st) {
  DirF f{S, D, px, pu, ps, kpx, kpu, Hp, mu, delta};
  run_reduce(f, (long long)S.N * S.nx + (long long)S.N * S.m + (long long)S.N * S.nu + S.nu, partial,
             out, st);
}
void launch_ftb(const DevSym &S, DevWork &D, const double *px, const double *pu, const double *ps,
                const double *const *dz, double tau, double *partial, double *out, cudaStream_t st) {
  FtbF f{S, D, px, pu, ps, dz[0], dz[1], dz[2], dz[3], dz[4], dz[5], tau};
  run_reduce(f, (long long)S.N * S.nx + (long long)S.N * S.m + S.nu, partial, out, st);
}
void launch_gather_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale,
                       cudaStream_t st) {
  k_gather_pos<<<nblk((long long)N * nx, 256), 256, 0, st>>>(N, nx, iperm, src, dst, scale); ipm_count_launch();
}
void launch_scatter_pos(int N, int nx, const int *iperm, const double *src, double *dst, double scale,
                        cudaStream_t st) {
  k_scatter_pos<<<nblk((long long)N * nx, 256), 256, 0, st>>>(N, nx, iperm, src, dst, scale); ipm_count_launch();
}
void launch_gu_apply(const DevSym &S, const double *J, const double *pu, double *v, cudaStream_t st) {
  k_gu_apply<<<nblk((long long)S.N * S.nx, 256), 256, 0, st>>>(S, J, pu, v); ipm_count_launch();
}
void launch_kapply(const DevSym &S, const double *K, const double *px_pos, const double *pu, double *kpx,
                   double *kpu, cudaStream_t st) {
  long long n = (long long)S.N * S.nx + (kpu ? (long long)S.N * S.nu : 0);
  k_kapply<<<nblk(n, 256), 256, 0, st>>>(S, K, px_pos, pu, kpx, kpu); ipm_count_launch();
}
void launch_lincomb(long long n, double *out, double a, const double *x, double b, const double *y,
                    double c, const double *z, cudaStream_t st) {
  if (n <= 0) return;
  k_lincomb<<<nblk(n, 256), 256, 0, st>>>(n, out, a, x, b, y, c, z); ipm_count_launch();
}
void launch_rhs_reduced(const DevSym &S, const double *J, const double *K, const double *rh2,
                        const double *a, const double *b, double *rhs, cudaStream_t st) {
  k_rhs_reduced<<<nblk(S.nu, 64), 64, 0, st>>>(S, J, K, rh2, a, b, rhs); ipm_count_launch();
}
void launch_zt_apply(const DevSym &S, const double *Z, const double *w, const double *K, const double *b,
                     double alpha, double beta, double *out, double *part, cudaStream_t st) {
  k_zt_part<<<dim3((S.nu + 31) / 32, S.N), 256, 0, st>>>(S, Z, w, K, b, alpha, part); ipm_count_launch();
  k_zt_sum<<<nblk(S.nu, 64), 64, 0, st>>>(S, part, beta, out); ipm_count_launch();
}
void launch_z_apply(const DevSym &S, const double *Z, const double *pu, double a, double *v, cudaStream_t st) {
  k_z_apply<<<nblk((long long)S.N * S.nx * 32, 256), 256, 0, st>>>(S, Z, pu, a, v); ipm_count_launch();
}
void launch_gut_sum(const DevSym &S, const double *J, const double *a, double scale, double *out,
                    cudaStream_t st) {
  k_gut_sum<<<nblk(S.nu, 64), 64, 0, st>>>(S, J, a, scale, out); ipm_count_launch();
}
void launch_apply_finish(const DevSym &S, const double *kpu, const double *diag, double delta, const double *v,
                         double *out, cudaStream_t st) {
  k_apply_finish<<<nblk(S.nu, 128), 128, 0, st>>>(S, kpu, diag, delta, v, out); ipm_count_launch();
}
void launch_dot2(int n, const double *a, const double *b, const double *c, const double *d, double *out,
                 cudaStream_t st) {
  k_dot2<<<1, 256, 0, st>>>(n, a, b, c, d, out); ipm_count_launch();
}
void launch_pz_ps(const DevSym &S, DevWork &D, const double *px, const double *pu, double *Hp, double *pz,
                  double *ps, cudaStream_t st) {
  k_pz_ps<<<nblk((long long)S.N * S.m, 128), 128, 0, st>>>(S, D, px, pu, Hp, pz, ps); ipm_count_launch();
}
void launch_bound_steps(long long n, int period, const double *w, const double *dw, const double *l,
                        const double *b, const double *zl, const double *zu, double mu, double *dzl,
                        double *dzu, cudaStream_t st) {
  if (n <= 0) return;
  k_bound_steps<<<nblk(n, 256), 256, 0, st>>>(n, period, w, dw, l, b, zl, zu, mu, dzl, dzu); ipm_count_launch();
}
void launch_dual_update(long long n, int period, const double *w, const double *l, const double *b,
                        double *zl, double *zu, const double *dzl, const double *dzu, double az, double mu,
                        double ks, cudaStream_t st) {
  if (n <= 0) return;
  k_dual_update<<<nblk(n, 256), 256, 0, st>>>(n, period, w, l, b, zl, zu, dzl, dzu, az, mu, ks); ipm_count_launch();
}
void launch_push(long long n, int period, double *w, const double *l, const double *b, double k1, double k2,
                 cudaStream_t st) {
  if (n <= 0) return;
  k_push<<<nblk(n, 256), 256, 0, st>>>(n, period, w, l, b, k1, k2); ipm_count_launch();
}
void launch_init_primal(const DevSym &S, double *x, double *u, const double *pmax, cudaStream_t st) {
  k_init_primal<<<nblk((long long)S.N * S.nx + S.nu, 256), 256, 0, st>>>(S, x, u, pmax); ipm_count_launch();
}
void launch_fill_bound_duals(long long n, int period, const double *l, const double *b, double *zl, double *zu,
                             cudaStream_t st) {
  if (n <= 0) return;
  k_fill_bound_duals<<<nblk(n, 256), 256, 0, st>>>(n, period, l, b, zl, zu); ipm_count_launch();
}

// ---------------------------------------------------------------------------
// Warm-start vectors (learned warm start).  Per scenario, d = seg[8]:
//   [0, seg1) x | [seg1, seg2) u | [seg2, seg3) s | [seg3, seg4) log zl_x |
//   [seg4, seg5) log zu_x | [seg5, seg6) log zl_u | [seg6, seg7) log zu_u |
//   [seg7, seg8) log zl_s | [seg8, seg9) log zu_s
// idx lists the bounded components of each dual block, concatenated.
namespace {

__device__ __forceinline__ const double *warm_dual_src(const DevWork &D, int b, int sc, const WarmSeg &W, int i,
                                                       int &off) {
  const int k = W.idx[W.seg[3 + b] - W.seg[3] + i];
  switch (b) {
    case 0: off = sc * W.nx + k; return D.zlx;
    case 1: off = sc * W.nx + k; return D.zux;
    case 2: off = k; return D.zlu;
    case 3: off = k; return D.zuu;
    case 4: off = sc * W.m + k; return D.zls;
    default: off = sc * W.m + k; return D.zus;
  }
}

__global__ void k_warm_target(DevWork D, WarmSeg W, int N, float *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = W.seg[9];
  if (t >= (long long)N * d) return;
  const int sc = (int)(t / d), k = (int)(t - (long long)sc * d);
  double v;
  if (k < W.seg[1]) v = D.x[(size_t)sc * W.nx + k];
  else if (k < W.seg[2]) v = D.u[k - W.seg[1]];
  else if (k < W.seg[3]) v = D.s[(size_t)sc * W.m + k - W.seg[2]];
  else {
    int b = 0;
    while (k >= W.seg[4 + b]) ++b;
    int off = 0;
    const double *src = warm_dual_src(D, b, sc, W, k - W.seg[3 + b], off);
    v = log(fmax(src[off], 1e-30));
  }
  out[t] = (float)v;
}

// primal rows and bound duals of each scenario (u and its duals: next kernel)
__global__ void k_warm_apply(DevWork D, WarmSeg W, int N, const float *pred) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = W.seg[9];
  if (t >= (long long)N * d) return;
  const int sc = (int)(t / d), k = (int)(t - (long long)sc * d);
  const double v = pred[t];
  if (k < W.seg[1]) D.x[(size_t)sc * W.nx + k] = v;
  else if (k < W.seg[2]) return;
  else if (k < W.seg[3]) D.s[(size_t)sc * W.m + k - W.seg[2]] = v;
  else {
    int b = 0;
    while (k >= W.seg[4 + b]) ++b;
    if (b == 2 || b == 3) return;
    int off = 0;
    double *dst = const_cast<double *>(warm_dual_src(D, b, sc, W, k - W.seg[3 + b], off));
    dst[off] = exp(fmin(fmax(v, -27.631021115928547), 27.631021115928547));  // [1e-12, 1e12]
  }
}

// u = mean over scenarios; first-stage bound duals: geometric mean
__global__ void k_warm_u(DevWork D, WarmSeg W, int N, const float *pred) {
  const int d = W.seg[9];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = W.seg[2] - W.seg[1];
  const int nl = W.seg[6] - W.seg[5], nb = W.seg[7] - W.seg[6];
  if (k < nu) {
    double s = 0.0;
    for (int sc = 0; sc < N; ++sc) s += pred[(size_t)sc * d + W.seg[1] + k];
    D.u[k] = s / N;
  } else if (k < nu + nl + nb) {
    const int i = k - nu;
    const int b = i < nl ? 2 : 3;
    const int c = W.seg[3 + b] + (b == 2 ? i : i - nl);
    double s = 0.0;
    for (int sc = 0; sc < N; ++sc) s += pred[(size_t)sc * d + c];
    int off = 0;
    double *dst = const_cast<double *>(warm_dual_src(D, b, 0, W, c - W.seg[3 + b], off));
    dst[off] = exp(fmin(fmax(s / N, -27.631021115928547), 27.631021115928547));
  }
}

// slack stationarity: z = zl_s - zu_s
__global__ void k_warm_z(long long n, DevWork D) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) D.z[t] = D.zls[t] - D.zus[t];
}

// x-gradient of the Lagrangian without the y terms (y = 0 when JTl was formed)
__global__ void k_warm_yrhs(DevSym S, DevWork D, double *r) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)S.N * S.nx) return;
  const int sc = (int)(t / S.nx), j = (int)(t - (long long)sc * S.nx);
  r[t] = D.JTl[(size_t)sc * 2 * S.n + S.xkind[j] * S.n + S.xbus[j]] - D.zlx[t] + D.zux[t];
}

}  // namespace

void launch_warm_target(const DevWork &D, const WarmSeg &W, int N, float *out, cudaStream_t st) {
  k_warm_target<<<nblk((long long)N * W.seg[9], 256), 256, 0, st>>>(D, W, N, out); ipm_count_launch();
}
void launch_warm_apply(const DevWork &D, const WarmSeg &W, int N, const float *pred, cudaStream_t st) {
  k_warm_apply<<<nblk((long long)N * W.seg[9], 256), 256, 0, st>>>(D, W, N, pred); ipm_count_launch();
  const int n = (W.seg[2] - W.seg[1]) + (W.seg[7] - W.seg[5]);
  k_warm_u<<<nblk(n, 128), 128, 0, st>>>(D, W, N, pred); ipm_count_launch();
}
void launch_warm_z(long long n, const DevWork &D, cudaStream_t st) {
  k_warm_z<<<nblk(n, 256), 256, 0, st>>>(n, D); ipm_count_launch();
}
void launch_warm_yrhs(const DevSym &S, const DevWork &D, double *r, cudaStream_t st) {
  k_warm_yrhs<<<nblk((long long)S.N * S.nx, 256), 256, 0, st>>>(S, D, r); ipm_count_launch();
}
