// K3-K5: batched static-pivot sparse LU of G_x (one pattern for all
// scenarios), the multi-RHS reduction solves Z = -G_x^{-1} G_u fused with the
// products Y = K [Z; I], and single-vector solves with G_x and G_x^T.
//
// Paper: §3.2 "Assembling the sparse matrices" (batched LU sharing one
// pattern, G_x^{-1} b = Q U^{-1} L^{-1} P b) and "Local reduction" (steps
// 1-2: T_x = -G_x^{-1} G_u V, [L_x; L_u] = K [T_x; V]).  Here V runs over
// all Cartesian vectors at once, split into RHS panels of 32 columns.
//
// Scheduling: every CTA owns one scenario (LU, single-vector solves) or one
// (scenario, RHS panel) pair (multi-RHS solves) and walks the level schedule
// of the shared pattern with __syncthreads() between levels; no grid-wide
// synchronisation and no inter-CTA waits.
#include "dev.cuh"
#include "kernels.h"

extern long long g_ipm_launches;

namespace {

__device__ __forceinline__ double block_max(double v, double *sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (blockDim.x >> 5)) ? sh[lane] : 0.0;
    v = warp_max(v);
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_lu_factor(DevSym S, int nL, const double *__restrict__ J, double *LU, double *rd,
                            int *flags, double piv_tol) {
  __shared__ double sh[32];
  const int sc = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  double *A = LU + (size_t)sc * S.nnzLU;
  double *r = rd + (size_t)sc * S.nx;
  double amax = 0.0;
  for (int p = tid; p < S.nnzLU; p += bd) {
    const int src = S.lu_init[p];
    const double v = src >= 0 ? J[(size_t)src * S.N + sc] : 0.0;
    A[p] = v;
    amax = fmax(amax, fabs(v));
  }
  amax = block_max(amax, sh);
  for (int l = 0; l < S.nlev; ++l) {
    for (int e = S.f_piv_ptr[l] + tid; e < S.f_piv_ptr[l + 1]; e += bd) {
      const int k = S.f_piv[e];
      const double d = A[S.lu_diag[k]];
      if (!(fabs(d) > piv_tol * amax)) flags[FLAG_SINGULAR] = 1;
      r[k] = 1.0 / d;
    }
    __syncthreads();
    for (int t = S.f_lev_ptr[l] + tid; t < S.f_lev_ptr[l + 1]; t += bd) {
      const int slot = S.f_tgt[t];
      double acc = A[slot];
      for (int o = S.f_op_ptr[t]; o < S.f_op_ptr[t + 1]; ++o)
        acc -= A[S.f_op_l[o]] * (A[S.f_op_u[o]] * r[S.f_op_k[o]]);
      A[slot] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < nL; e += bd) A[S.lsc_slot[e]] *= r[S.lsc_k[e]];
}

// Z = -U^{-1} L^{-1} (P G_u) for one scenario and one panel of 32 RHS
// columns (lane = column), then Y = K_x [Z; I] and Y_u = K_u [Z; I].
// Rows of Z and Y are in LU position order.
__global__ void __launch_bounds__(256) k_zsolve64(DevSym S, const double *__restrict__ LU,
                                                  const double *__restrict__ rd,
                                                  const double *__restrict__ J,
                                                  const double *__restrict__ K, double *Z,
                                                  double *Y, double *Yu) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sc = blockIdx.y, c = blockIdx.x * 32 + lane, nu = S.nu, nx = S.nx, N = S.N;
  const bool valid = c < nu;
  const int cc = valid ? c : nu - 1;
  const double *A = LU + (size_t)sc * S.nnzLU;
  const double *r = rd + (size_t)sc * nx;
  double *Zs = Z + (size_t)sc * nx * nu;
  double *Ys = Y + (size_t)sc * nx * nu;
  double *Yus = Yu + (size_t)sc * nu * nu;
  for (int l = 0; l < S.nlev; ++l) {
    for (int e = S.fw_lev_ptr[l] + warp; e < S.fw_lev_ptr[l + 1]; e += nw) {
      const int row = S.fw_rows[e];
      double acc = 0.0;
      for (int g = S.gu_ptr[row]; g < S.gu_ptr[row + 1]; ++g)
        if (S.gu_col[g] == cc) {
          const int src = S.gu_src[g];
          acc -= src >= 0 ? J[(size_t)src * N + sc] : -1.0;
        }
      for (int f = S.fr_ptr[row]; f < S.fr_ptr[row + 1]; ++f)
        acc -= A[S.fr_lslot[f]] * Zs[(size_t)S.fr_col[f] * nu + cc];
      if (valid) Zs[(size_t)row * nu + c] = acc;
    }
    __syncthreads();
  }
  for (int l = 0; l < S.nlev_b; ++l) {
    for (int e = S.bw_lev_ptr[l] + warp; e < S.bw_lev_ptr[l + 1]; e += nw) {
      const int row = S.bw_rows[e];
      double acc = Zs[(size_t)row * nu + cc];
      for (int f = S.br_ptr[row]; f < S.br_ptr[row + 1]; ++f)
        acc -= A[S.br_uslot[f]] * Zs[(size_t)S.br_col[f] * nu + cc];
      if (valid) Zs[(size_t)row * nu + c] = acc * r[row];
    }
    __syncthreads();
  }
  for (int row = warp; row < nx; row += nw) {
    double acc = 0.0;
    for (int e = S.kx_ptr[row]; e < S.kx_ptr[row + 1]; ++e) {
      const int col = S.kx_col[e];
      const double v = K[(size_t)S.kx_src[e] * N + sc];
      if (col < nx) acc += v * Zs[(size_t)col * nu + cc];
      else if (col - nx == cc) acc += v;
    }
    if (valid) Ys[(size_t)row * nu + c] = acc;
  }
  for (int j = warp; j < nu; j += nw) {
    double acc = 0.0;
    for (int e = S.ku_ptr[j]; e < S.ku_ptr[j + 1]; ++e) {
      const int col = S.ku_col[e];
      const double v = K[(size_t)S.ku_src[e] * N + sc];
      if (col < nx) acc += v * Zs[(size_t)col * nu + cc];
      else if (col - nx == cc) acc += v;
    }
    if (valid) Yus[(size_t)j * nu + c] = acc;
  }
}

// In-place solve of G_x v = b (trans = 0) or G_x^T v = b (trans = 1) for every
// scenario; v is [N][nx] in LU position order.
__global__ void k_solve1(DevSym S, const double *__restrict__ LU, const double *__restrict__ rd,
                         double *v, int trans) {
  const int sc = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const double *A = LU + (size_t)sc * S.nnzLU;
  const double *r = rd + (size_t)sc * S.nx;
  double *vs = v + (size_t)sc * S.nx;
  for (int l = 0; l < S.nlev; ++l) {
    for (int e = S.fw_lev_ptr[l] + tid; e < S.fw_lev_ptr[l + 1]; e += bd) {
      const int row = S.fw_rows[e];
      double acc = vs[row];
      if (trans) {
        for (int f = S.fr_ptr[row]; f < S.fr_ptr[row + 1]; ++f) acc -= A[S.fr_uslot[f]] * vs[S.fr_col[f]];
        vs[row] = acc * r[row];
      } else {
        for (int f = S.fr_ptr[row]; f < S.fr_ptr[row + 1]; ++f) acc -= A[S.fr_lslot[f]] * vs[S.fr_col[f]];
        vs[row] = acc;
      }
    }
    __syncthreads();
  }
  for (int l = 0; l < S.nlev_b; ++l) {
    for (int e = S.bw_lev_ptr[l] + tid; e < S.bw_lev_ptr[l + 1]; e += bd) {
      const int row = S.bw_rows[e];
      double acc = vs[row];
      if (trans) {
        for (int f = S.br_ptr[row]; f < S.br_ptr[row + 1]; ++f) acc -= A[S.br_lslot[f]] * vs[S.br_col[f]];
        vs[row] = acc;
      } else {
        for (int f = S.br_ptr[row]; f < S.br_ptr[row + 1]; ++f) acc -= A[S.br_uslot[f]] * vs[S.br_col[f]];
        vs[row] = acc * r[row];
      }
    }
    __syncthreads();
  }
}

}  // namespace

void launch_lu_factor(const DevSym &S, int nL, const double *J, double *LU, double *rd, int *flags,
                      cudaStream_t st) {
  k_lu_factor<<<S.N, 256, 0, st>>>(S, nL, J, LU, rd, flags, 1e-14); ++g_ipm_launches;
}
void launch_zsolve64(const DevSym &S, const double *LU, const double *rd, const double *J,
                     const double *K, double *Z, double *Y, double *Yu, cudaStream_t st) {
  dim3 grid((S.nu + 31) / 32, S.N);
  k_zsolve64<<<grid, 256, 0, st>>>(S, LU, rd, J, K, Z, Y, Yu); ++g_ipm_launches;
}
void launch_solve1(const DevSym &S, const double *LU, const double *rd, double *v, int trans,
                   cudaStream_t st) {
  k_solve1<<<S.N, 256, 0, st>>>(S, LU, rd, v, trans); ++g_ipm_launches;
}
