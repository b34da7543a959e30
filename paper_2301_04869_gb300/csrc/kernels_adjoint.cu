// The paper's local reduction by adjoint solves (§3.2, "Local reduction"):
// for a block V of unit vectors,
//   1. T_x = -G_x^{-1} (G_u V)                (the columns of Z)
//   2. [L_x; L_u] = [K_xx K_xu; K_ux K_uu] [T_x; V]   (Y and Y_u)
//   3. K_hat V = L_u - G_u^T G_x^{-T} L_x     (transpose read as in
//      Prop. 2.3: the G_u of step 3 is G_u^T by dimensions)
// Steps 1-2 are the multi-RHS solve of the dense route (V = I, all n_u
// columns at once); here step 3 replaces the dense contraction Z^T Y by one
// more multi-RHS solve, with G_x^T, on the columns of L_x.  These kernels
// lay L_x out as vectors for that solve and assemble K_hat from its result.
#include "dev.cuh"
#include "kernels.h"

namespace {

// W[s][j][p] = Y[s][p][j]: the n_u columns of L_x (rows of Y in position
// order) as vectors, 32 x 32 tiles through shared memory
__global__ void k_transpose_rows(int nx, int nu, const double *__restrict__ Y, double *__restrict__ W) {
  __shared__ double t[32][33];
  const int s = blockIdx.z, p0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const double *Ys = Y + (size_t)s * nx * nu;
  double *Ws = W + (size_t)s * nu * nx;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = p0 + r, j = j0 + threadIdx.x;
    t[r][threadIdx.x] = (p < nx && j < nu) ? Ys[(size_t)p * nu + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, p = p0 + threadIdx.x;
    if (j < nu && p < nx) Ws[(size_t)j * nx + p] = t[threadIdx.x][r];
  }
}

// (K_hat)_kj = sum_s [ (Y_u,s)_kj - (G_u^T W_s[j])_k ] + diag_k delta_kj for
// k <= j, and the same with k, j exchanged; both are averaged into the two
// symmetric entries (the exact K_hat is symmetric; the two orders of the
// adjoint route round differently).  Scenarios in index order.
__global__ void k_adjoint_assemble(DevSym S, const double *__restrict__ J, const double *__restrict__ Yu,
                                   const double *__restrict__ W, const double *__restrict__ diag, double *Khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = S.nu, nx = S.nx, N = S.N;
  if (t >= (long long)nu * nu) return;
  const int k = (int)(t / nu), j = (int)(t % nu);
  if (k > j) return;
  double a = 0.0, b = 0.0;  // (k, j) and (j, k)
  for (int s = 0; s < N; ++s) {
    const double *Ws = W + (size_t)s * nu * nx;
    double gk = 0.0, gj = 0.0;
    for (int e = S.gut_ptr[k]; e < S.gut_ptr[k + 1]; ++e) {
      const int src = S.gut_src[e];
      gk += (src >= 0 ? J[(size_t)src * N + s] : -1.0) * Ws[(size_t)j * nx + S.gut_col[e]];
    }
    for (int e = S.gut_ptr[j]; e < S.gut_ptr[j + 1]; ++e) {
      const int src = S.gut_src[e];
      gj += (src >= 0 ? J[(size_t)src * N + s] : -1.0) * Ws[(size_t)k * nx + S.gut_col[e]];
    }
    const double *Ys = Yu + (size_t)s * nu * nu;
    a += Ys[(size_t)k * nu + j] - gk;
    b += Ys[(size_t)j * nu + k] - gj;
  }
  double v = 0.5 * (a + b);
  if (k == j && diag) v += diag[k];
  Khat[(size_t)k * nu + j] = v;
  Khat[(size_t)j * nu + k] = v;
}

}  // namespace

void launch_transpose_rows(int N, int nx, int nu, const double *Y, double *W, cudaStream_t st) {
  dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((nu + 31) / 32), (unsigned)N);
  k_transpose_rows<<<grid, dim3(32, 8), 0, st>>>(nx, nu, Y, W); ipm_count_launch();
}

void launch_adjoint_assemble(const DevSym &S, const double *J, const double *Yu, const double *W, const double *diag,
                             double *Khat, cudaStream_t st) {
  const long long tot = (long long)S.nu * S.nu;
  k_adjoint_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(S, J, Yu, W, diag, Khat); ipm_count_launch();
}
