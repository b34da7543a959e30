// K6 (FP64 path) and K7: the dense reduced Hessian
//   K_hat = sum_i (Z_i^T Y_i + Y_u,i) + Sigma_u + (first-stage cost curvature)
// (Prop. 2.3, K_hat = Z^T K Z, summed over scenarios as the global reduction of
// §3.2 does with MPI_Allreduce), and its dense Cholesky factorization
// (§4: the Schur complement is factorized with dense LAPACK on the GPU).
//
// The scenario sum is part of the contraction: K runs over (scenario, row)
// pairs.  CTAs split that range into fixed groups of scenarios and write
// partial tiles; one pass then adds the groups in index order (deterministic).
// Only upper tiles (i <= j) are computed; the symmetric result is mirrored.
#include <atomic>

#include <cooperative_groups.h>

#include "dev.cuh"
#include "kernels.h"


namespace {

constexpr int TB = 64;   // output tile
constexpr int TK = 16;   // k chunk

// One 64 x 64 tile of A^T B over the rows [r0, r1) of the (rows x nu)
// matrices A, B (scenario-major storage makes the scenario sum one
// contraction over the concatenated rows); the tile goes to P (row-major).
__device__ __forceinline__ void tile_tn64(long long r0, long long r1, int nu, int i0, int j0,
                                          const double *__restrict__ A, const double *__restrict__ B,
                                          double *P, double (*As)[TB], double (*Bs)[TB]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (long long k0 = r0; k0 < r1; k0 += TK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256, kk = e >> 6, cc = e & 63;
      const long long k = k0 + kk;
      As[kk][cc] = (k < r1 && i0 + cc < nu) ? A[k * nu + i0 + cc] : 0.0;
      Bs[kk][cc] = (k < r1 && j0 + cc < nu) ? B[k * nu + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) P[(ty * 4 + a) * TB + tx * 4 + b] = acc[a][b];
}

// partial[g][tile t][64*64] = A^T B on tile t over the rows [g*kc, (g+1)*kc)
__global__ void __launch_bounds__(256) k_gemm_tn64(long long krows, long long kc, int nu,
                                                   const double *__restrict__ A,
                                                   const double *__restrict__ B,
                                                   const int2 *__restrict__ tiles, double *partial) {
  __shared__ double As[TK][TB];
  __shared__ double Bs[TK][TB];
  const int t = blockIdx.x, g = blockIdx.y;
  const long long r0 = (long long)g * kc, r1 = min(krows, r0 + kc);
  tile_tn64(r0, r1, nu, tiles[t].x * TB, tiles[t].y * TB, A, B,
            partial + ((size_t)g * gridDim.x + t) * TB * TB, As, Bs);
}

// The same contraction for many independent instances in one persistent
// launch: every (instance, tile, scenario group) is a work item; CTAs take
// items from an atomic counter (items are sorted by decreasing length, so
// the long ones start first).  Each item writes the partial tile that the
// instance's own launch would write, so the result does not depend on which
// CTA ran it.
__global__ void __launch_bounds__(256) k_gemm_grouped(const GemmItem *__restrict__ items, int nitems,
                                                      int *counter) {
  __shared__ double As[TK][TB];
  __shared__ double Bs[TK][TB];
  __shared__ int w;
  for (;;) {
    if (threadIdx.x == 0) w = atomicAdd(counter, 1);
    __syncthreads();
    const int it = w;
    __syncthreads();
    if (it >= nitems) break;
    const GemmItem g = items[it];
    tile_tn64(g.r0, g.r1, g.nu, g.i0, g.j0, g.A, g.B, g.P, As, Bs);
  }
}

// K_hat[i][j] = K_hat[j][i] = sum_g partial + sum_s Yu[s][i][j] + diag  (i <= j)
__global__ void k_khat_assemble(int nu, int N, int ngroups, int ntiles, int nt1,
                                const double *__restrict__ partial, const int *__restrict__ tile_of,
                                const double *__restrict__ Yu, const double *__restrict__ diag,
                                double *Khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int i = (int)(t / nu), j = (int)(t % nu);
  if (i > j) return;
  const int ti = i / TB, tj = j / TB;
  const int tt = tile_of[ti * nt1 + tj];
  double v = 0.0;
  for (int g = 0; g < ngroups; ++g)
    v += partial[((size_t)g * ntiles + tt) * TB * TB + (i - ti * TB) * TB + (j - tj * TB)];
  if (Yu)
    for (int s = 0; s < N; ++s) v += Yu[(size_t)s * nu * nu + (size_t)i * nu + j];
  if (diag && i == j) v += diag[i];
  Khat[(size_t)i * nu + j] = v;
  Khat[(size_t)j * nu + i] = v;
}

// F = Khat + delta (M + I) + tau I   (tau: shift of a preconditioner only)
__global__ void k_shift(int nu, const double *Khat, const double *M, double delta, double tau, double *F) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int i = (int)(t / nu), j = (int)(t % nu);
  double v = Khat[t];
  if (delta != 0.0) v += delta * (M[t] + (i == j ? 1.0 : 0.0));
  if (i == j) v += tau;
  F[t] = v;
}

// out[0] = max_i |A_ii|
__global__ void k_maxdiag(int n, const double *A, double *out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(A[(size_t)i * n + i]));
  m = warp_max(m);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    out[0] = r;
  }
}

constexpr int CB = 32;  // Cholesky block

// factor the CB x CB diagonal block at (k0, k0) in place (lower), unblocked

// Right-looking Cholesky of the nb x nb block a (lower part, in shared
// memory) by the calling CTA: thread 0 takes each pivot's reciprocal square
// root, then warps 0-3 scale the column and update the trailing columns
// (warp w: columns j = w mod 4; lane = row; column entries by shuffles).  A
// non-positive or non-finite pivot raises FLAG_NOT_PD and is replaced by 1.
__device__ void potrf_block(int nb, int *flags, double (*a)[CB + 1], double *rs_sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      double d = a[k][k];
      if (!(d > 0.0) || !isfinite(d)) {
        flags[FLAG_NOT_PD] = 1;
        d = 1.0;
      }
      const double rs = rsqrt_newton(d);
      *rs_sh = rs;
      a[k][k] = d * rs;
    }
    __syncthreads();
    double lik = 0.0;
    if (warp < 4) {
      lik = (lane > k && lane < nb) ? a[lane][k] * *rs_sh : 0.0;
      for (int j = k + 1 + ((warp - (k + 1)) & 3); j < nb; j += 4) {
        const double ljk = __shfl_sync(0xffffffffu, lik, j);
        if (lane >= j && lane < nb) a[lane][j] -= lik * ljk;
      }
    }
    __syncthreads();
    // column k is read by no later step: written after the barrier
    if (warp == 0 && lane > k && lane < nb) a[lane][k] = lik;
  }
  __syncthreads();
}

// Load, factor and store the diagonal block at (k0, k0) (upper part of the
// block set to zero).
__device__ void potrf_tile(int n, int k0, double *A, int *flags, double (*a)[CB + 1], double *rs_sh) {
  const int nb = min(CB, n - k0), tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) a[e / nb][e % nb] = A[(size_t)(k0 + e / nb) * n + k0 + e % nb];
  __syncthreads();
  potrf_block(nb, flags, a, rs_sh);
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    A[(size_t)(k0 + i) * n + k0 + j] = (j <= i) ? a[i][j] : 0.0;
  }
  __syncthreads();
}

__global__ void k_potrf_diag(int n, int k0, double *A, int *flags) {
  __shared__ double a[CB][CB + 1];
  __shared__ double rs_sh;
  potrf_tile(n, k0, A, flags, a, &rs_sh);
}

// rows below the diagonal block: L_ik = A_ik L_kk^{-T}
__global__ void k_trsm_panel(int n, int k0, double *A) {
  __shared__ double Lk[CB][CB + 1];
  const int nb = min(CB, n - k0), tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) Lk[e / nb][e % nb] = A[(size_t)(k0 + e / nb) * n + k0 + e % nb];
  __syncthreads();
  const int i = k0 + nb + blockIdx.x * blockDim.x + tid;
  if (i >= n) return;
  double x[CB];
  for (int j = 0; j < nb; ++j) {
    double v = A[(size_t)i * n + k0 + j];
    for (int t = 0; t < j; ++t) v -= x[t] * Lk[j][t];
    x[j] = v / Lk[j][j];
  }
  for (int j = 0; j < nb; ++j) A[(size_t)i * n + k0 + j] = x[j];
}

// trailing update of the lower part: A_ij -= sum_t L_it L_jt (tiles CB x CB)
__global__ void k_syrk_trail(int n, int k0, double *A) {
  const int nb = min(CB, n - k0);
  const int r0 = k0 + nb;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ double Li[CB][CB + 1], Lj[CB][CB + 1];
  const int tid = threadIdx.x;
  const int i0 = r0 + bi * CB, j0 = r0 + bj * CB;
  for (int e = tid; e < CB * nb; e += blockDim.x) {
    const int rr = e / nb, t = e % nb;
    Li[rr][t] = (i0 + rr < n) ? A[(size_t)(i0 + rr) * n + k0 + t] : 0.0;
    Lj[rr][t] = (j0 + rr < n) ? A[(size_t)(j0 + rr) * n + k0 + t] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int ii = e / CB, jj = e % CB, i = i0 + ii, j = j0 + jj;
    if (i >= n || j >= n || j > i) continue;
    double v = 0.0;
    for (int t = 0; t < nb; ++t) v += Li[ii][t] * Lj[jj][t];
    A[(size_t)i * n + j] -= v;
  }
}

// The same blocked factorization as one cooperative launch (grid-wide
// barriers between the steps instead of three launches per block column).
// Per block column k0 (32 wide): (a) every CTA with panel rows loads L_kk and
// solves its rows x L_kk^T = a (a warp per row, lane = column, shuffles; the
// multipliers L_jt / L_tt are formed once per CTA so each step is one
// shuffle and one multiply-add); (b) the trailing matrix is updated: CTA 0
// forms the next diagonal block in one pass straight into shared memory and
// factors it right away, the other lower 16 x 16 tiles go round-robin to
// the remaining CTAs.
constexpr int CT = 16;  // trailing-update tile

__device__ void syrk_tile16(int n, int k0, int nb, int i0, int j0, double *A, double (*Li)[CB + 1],
                            double (*Lj)[CB + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < CT * nb; e += blockDim.x) {
    const int rr = e / nb, t = e % nb;
    Li[rr][t] = (i0 + rr < n) ? A[(size_t)(i0 + rr) * n + k0 + t] : 0.0;
    Lj[rr][t] = (j0 + rr < n) ? A[(size_t)(j0 + rr) * n + k0 + t] : 0.0;
  }
  __syncthreads();
  if (tid < CT * CT) {
    const int ii = tid / CT, jj = tid % CT, i = i0 + ii, j = j0 + jj;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int t = 0;
    for (; t + 4 <= nb; t += 4) {
      s0 = fma(Li[ii][t], Lj[jj][t], s0);
      s1 = fma(Li[ii][t + 1], Lj[jj][t + 1], s1);
      s2 = fma(Li[ii][t + 2], Lj[jj][t + 2], s2);
      s3 = fma(Li[ii][t + 3], Lj[jj][t + 3], s3);
    }
    for (; t < nb; ++t) s0 = fma(Li[ii][t], Lj[jj][t], s0);
    if (i < n && j < n && j <= i) A[(size_t)i * n + j] -= (s0 + s1) + (s2 + s3);
  }
}

__global__ void __launch_bounds__(256) k_chol_coop(int n, double *A, int *flags) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ double a[CB][CB + 1], b2[CB][CB + 1];
  __shared__ double rinv[CB], rs_sh;
  const int G = gridDim.x, bk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (bk == 0) potrf_tile(n, 0, A, flags, a, &rs_sh);
  grid.sync();
  for (int k0 = 0; k0 < n; k0 += CB) {
    const int nb = min(CB, n - k0), r0 = k0 + nb, rest = n - r0;
    if (rest <= 0) break;
    // (a) panel rows
    if (r0 + bk * 8 < n) {
      for (int e = tid; e < CB * CB; e += blockDim.x) {
        const int rr = e / CB, cc = e % CB;
        a[rr][cc] = (rr < nb && cc <= rr) ? A[(size_t)(k0 + rr) * n + k0 + cc] : 0.0;
      }
      __syncthreads();
      if (tid < CB) rinv[tid] = tid < nb ? 1.0 / a[tid][tid] : 0.0;
      __syncthreads();
      for (int e = tid; e < CB * CB; e += blockDim.x) {
        const int rr = e / CB, cc = e % CB;
        b2[rr][cc] = cc < rr ? a[rr][cc] * rinv[cc] : 0.0;  // L_jt / L_tt (j = rr, t = cc)
      }
      __syncthreads();
      for (int i = r0 + bk * 8 + warp; i < n; i += G * 8) {
        double v = lane < nb ? A[(size_t)i * n + k0 + lane] : 0.0;
        for (int t = 0; t < nb; ++t) {
          const double vt = __shfl_sync(0xffffffffu, v, t);
          if (lane > t) v = fma(-b2[lane][t], vt, v);
        }
        if (lane < nb) A[(size_t)i * n + k0 + lane] = v * rinv[lane];
      }
    }
    grid.sync();
    // (b) trailing update; tiles with bi, bj < 2 form the next diagonal block
    const int nt = (rest + CT - 1) / CT;
    const int ndt = nt >= 2 ? 3 : 1;
    const int ntl = nt * (nt + 1) / 2 - ndt;
    if (bk == 0) {
      if (G == 1)
        for (int t = 0; t < ntl; ++t) {
          int bi = 2, rem = t;
          while (rem > bi) { rem -= bi + 1; ++bi; }
          syrk_tile16(n, k0, nb, r0 + bi * CT, r0 + rem * CT, A, a, b2);
        }
      // the next diagonal block, A_dd - L_d L_d^T, straight into shared
      // memory (one pass over its lower part), then factored and stored
      const int nb2 = min(CB, rest);
      __syncthreads();
      for (int e = tid; e < CB * nb; e += blockDim.x) {
        const int rr = e / nb, t = e % nb;
        b2[rr][t] = rr < nb2 ? A[(size_t)(r0 + rr) * n + k0 + t] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < nb2 * nb2; e += blockDim.x) {
        const int i = e / nb2, j = e % nb2;
        if (j > i) continue;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int t = 0;
        for (; t + 4 <= nb; t += 4) {
          s0 = fma(b2[i][t], b2[j][t], s0);
          s1 = fma(b2[i][t + 1], b2[j][t + 1], s1);
          s2 = fma(b2[i][t + 2], b2[j][t + 2], s2);
          s3 = fma(b2[i][t + 3], b2[j][t + 3], s3);
        }
        for (; t < nb; ++t) s0 = fma(b2[i][t], b2[j][t], s0);
        a[i][j] = A[(size_t)(r0 + i) * n + r0 + j] - ((s0 + s1) + (s2 + s3));
      }
      __syncthreads();
      potrf_block(nb2, flags, a, &rs_sh);
      for (int e = tid; e < nb2 * nb2; e += blockDim.x) {
        const int i = e / nb2, j = e % nb2;
        A[(size_t)(r0 + i) * n + r0 + j] = (j <= i) ? a[i][j] : 0.0;
      }
      __syncthreads();
    } else {
      for (int t = bk - 1; t < ntl; t += G - 1) {
        // t-th lower tile in rows bi >= 2: row bi holds bi + 1 tiles
        int bi = 2, rem = t;
        while (rem > bi) { rem -= bi + 1; ++bi; }
        syrk_tile16(n, k0, nb, r0 + bi * CT, r0 + rem * CT, A, a, b2);
      }
    }
    grid.sync();
  }
}

// solve L L^T x = b in place (one CTA; x in shared memory).  Blocked by 32:
// one warp solves each 32 x 32 diagonal block with shuffles, then all
// threads apply the block's columns to the remaining rows (forward: rows of
// L, contiguous per thread; backward: rows of L read across threads).
// L L^T x = b for one right-hand side, one CTA (x in shared memory).
// Blocked by 32: one warp solves each 32 x 32 diagonal
// block (lane = row, shuffles), multiplying by reciprocal pivots that all
// lanes form at once (a dependent FP64 division costs ~9 multiply-adds of
// latency); then a thread per remaining row applies the block's 32 columns
// with four partial sums (the dependent FP64 chain is 8 long instead of 32).
__global__ void __launch_bounds__(512) k_chol_solve(int n, const double *__restrict__ L, double *b) {
  extern __shared__ double x[];
  __shared__ double blk[32][33];
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += bd) x[i] = b[i];
  __syncthreads();
  for (int kb = 0; kb < n; kb += 32) {
    const int w = min(32, n - kb);
    for (int e = tid; e < 32 * 32; e += bd) {
      const int r = e >> 5, c = e & 31;
      blk[r][c] = (r < w && c <= r) ? L[(size_t)(kb + r) * n + kb + c] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      const double ri = lane < w ? 1.0 / blk[lane][lane] : 0.0;
      double v = lane < w ? x[kb + lane] : 0.0;
      for (int jj = 0; jj < w; ++jj) {
        if (lane == jj) v *= ri;
        const double xj = __shfl_sync(0xffffffffu, v, jj);
        if (lane > jj) v -= blk[lane][jj] * xj;
      }
      if (lane < w) x[kb + lane] = v;
    }
    __syncthreads();
    for (int i = kb + w + tid; i < n; i += bd) {
      const double *row = L + (size_t)i * n + kb;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 4 <= w; j += 4) {
        s0 = fma(row[j], x[kb + j], s0);
        s1 = fma(row[j + 1], x[kb + j + 1], s1);
        s2 = fma(row[j + 2], x[kb + j + 2], s2);
        s3 = fma(row[j + 3], x[kb + j + 3], s3);
      }
      for (; j < w; ++j) s0 = fma(row[j], x[kb + j], s0);
      x[i] -= (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
  }
  for (int kb = ((n - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int w = min(32, n - kb);
    for (int e = tid; e < 32 * 32; e += bd) {
      const int r = e >> 5, c = e & 31;
      blk[r][c] = (r < w && c <= r) ? L[(size_t)(kb + r) * n + kb + c] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      const double ri = lane < w ? 1.0 / blk[lane][lane] : 0.0;
      double v = lane < w ? x[kb + lane] : 0.0;
      for (int jj = w - 1; jj >= 0; --jj) {
        if (lane == jj) v *= ri;
        const double xj = __shfl_sync(0xffffffffu, v, jj);
        if (lane < jj) v -= blk[jj][lane] * xj;  // (L^T)[lane][jj] = L[jj][lane]
      }
      if (lane < w) x[kb + lane] = v;
    }
    __syncthreads();
    for (int i = tid; i < kb; i += bd) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 4 <= w; j += 4) {
        s0 = fma(L[(size_t)(kb + j) * n + i], x[kb + j], s0);
        s1 = fma(L[(size_t)(kb + j + 1) * n + i], x[kb + j + 1], s1);
        s2 = fma(L[(size_t)(kb + j + 2) * n + i], x[kb + j + 2], s2);
        s3 = fma(L[(size_t)(kb + j + 3) * n + i], x[kb + j + 3], s3);
      }
      for (; j < w; ++j) s0 = fma(L[(size_t)(kb + j) * n + i], x[kb + j], s0);
      x[i] -= (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += bd) b[i] = x[i];
}

}  // namespace

void launch_gemm_tn64(long long krows, long long kc, int nu, int ngroups, const double *A, const double *B,
                      const int2 *tiles, int ntiles, double *partial, cudaStream_t st) {
  dim3 grid(ntiles, ngroups);
  k_gemm_tn64<<<grid, 256, 0, st>>>(krows, kc, nu, A, B, tiles, partial); ipm_count_launch();
}
void launch_gemm_grouped(const GemmItem *items, int nitems, int *counter, cudaStream_t st) {
  static const int ctas = [] {
    int per_sm = 0, dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_grouped, 256, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    return sms * per_sm;
  }();
  cudaMemsetAsync(counter, 0, sizeof(int), st);
  const int grid = nitems < ctas ? nitems : ctas;
  if (grid > 0) {
    k_gemm_grouped<<<grid, 256, 0, st>>>(items, nitems, counter);
    ipm_count_launch();
  }
}

void launch_khat_assemble(int nu, int N, int ngroups, int ntiles, int nt1, const double *partial,
                          const int *tile_of, const double *Yu, const double *diag, double *Khat,
                          cudaStream_t st) {
  long long tot = (long long)nu * nu;
  k_khat_assemble<<<(int)((tot + 255) / 256), 256, 0, st>>>(nu, N, ngroups, ntiles, nt1, partial,
                                                             tile_of, Yu, diag, Khat); ipm_count_launch();
}
void launch_shift(int nu, const double *Khat, const double *M, double delta, double tau, double *F,
                  cudaStream_t st) {
  long long tot = (long long)nu * nu;
  k_shift<<<(int)((tot + 255) / 256), 256, 0, st>>>(nu, Khat, M, delta, tau, F); ipm_count_launch();
}
void launch_maxdiag(int n, const double *A, double *out, cudaStream_t st) {
  k_maxdiag<<<1, 256, 0, st>>>(n, A, out); ipm_count_launch();
}
void launch_cholesky(int n, double *A, int *flags, cudaStream_t st) {
  // one cooperative launch when the device allows it (all CTAs resident)
  static const int coop_ctas = [] {
    int dev = 0, ok = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ok, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!ok || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_coop, 256, 0) != cudaSuccess || per < 1)
      return 0;
    return sms;  // one CTA per SM
  }();
  if (coop_ctas > 0) {
    const int nt = (n + CT - 1) / CT;
    int G = 1 + nt * (nt + 1) / 2;  // CTA 0 plus one per lower tile of the first trailing update
    G = G < coop_ctas ? G : coop_ctas;
    if (G < 1) G = 1;
    void *args[] = {(void *)&n, (void *)&A, (void *)&flags};
    if (cudaLaunchCooperativeKernel((const void *)k_chol_coop, dim3(G), dim3(256), args, 0, st) == cudaSuccess) {
      ipm_count_launch();
      return;
    }
    cudaGetLastError();
  }
  for (int k0 = 0; k0 < n; k0 += CB) {
    k_potrf_diag<<<1, 256, 0, st>>>(n, k0, A, flags); ipm_count_launch();
    const int nb = n - k0 < CB ? n - k0 : CB;
    const int rest = n - k0 - nb;
    if (rest > 0) {
      k_trsm_panel<<<(rest + 127) / 128, 128, 0, st>>>(n, k0, A); ipm_count_launch();
      const int nt = (rest + CB - 1) / CB;
      k_syrk_trail<<<dim3(nt, nt), 256, 0, st>>>(n, k0, A); ipm_count_launch();
    }
  }
}
void launch_chol_solve(int n, const double *L, double *b, cudaStream_t st) {
  const size_t bytes = (size_t)n * sizeof(double);
  static const bool cap = raise_smem_cap(k_chol_solve);
  (void)cap;
  k_chol_solve<<<1, 512, bytes, st>>>(n, L, b); ipm_count_launch();
}
