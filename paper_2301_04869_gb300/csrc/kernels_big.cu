// Large dense trailing block of the static-pivot LU of G_x (global memory).
//
// On the 10,000-bus networks the minimum-degree order ends in a dense block
// of about 1,800 states; it cannot live in one SM's shared memory as the
// smaller blocks do.  Here it is stored per scenario column-major with
// leading dimension nd (its entry (a, b) at LU + dense_base + b nd + a) and
// factored and solved by batched blocked kernels over all scenarios:
//
//  * LU (right-looking, panels of PB columns, static diagonal pivots as in
//    the rest of the factorization): per panel, the panel itself (one CTA
//    per scenario), U12 = L11^{-1} A12 (a warp per column), and the trailing
//    update A22 -= L21 U12 as 64 x 64 FP64 tiles over (tile, scenario);
//  * the multi-RHS solve of Z through the block: Z_d (the block's n_u
//    right-hand sides, row-major with leading dimension n_u in Z) is solved
//    with the unit-lower L_dd and then with U_dd, each blocked by PB rows:
//    a triangular solve of the diagonal block (a thread per column), then a
//    tile product updating the remaining rows; T = double on the FP64 path,
//    float on the mixed path (products accumulated in T, factors read in
//    FP64 and rounded to T).
//
// §3.2, "Assembling the sparse matrices": the paper factors G_x^{1:M} with a
// batched sparse LU sharing one pattern; the dense trailing block is the part
// of that factorization where every entry is filled.
#include "dev.cuh"
#include "kernels.h"

namespace {

constexpr int PB = 64;   // panel / block width
constexpr int TT = 64;   // tile of the updates

// ---- LU ----------------------------------------------------------------

// Factor the panel: columns [kb, ke) of rows [kb, nd) of scenario blockIdx.x.
__global__ void __launch_bounds__(256) k_blu_panel(int nd, int nx, int t0, long long nnzlu, int dense_base,
                                                   double *LU, double *rd, const double *amax, double piv_tol,
                                                   int *flags, int kb, int ke) {
  __shared__ double rowk[PB];
  __shared__ double rk_s;
  const int sc = blockIdx.x, tid = threadIdx.x;
  double *A = LU + (size_t)sc * nnzlu + dense_base;
  double *r = rd + (size_t)sc * nx + t0;
  const double ref = amax[sc];
  for (int k = kb; k < ke; ++k) {
    if (tid == 0) {
      const double d = A[(size_t)k * nd + k];
      if (!(fabs(d) > piv_tol * ref)) flags[FLAG_SINGULAR] = 1;
      rk_s = 1.0 / d;
      r[k] = rk_s;
    }
    for (int j = k + 1 + tid; j < ke; j += blockDim.x) rowk[j - kb] = A[(size_t)j * nd + k];
    __syncthreads();
    const double rk = rk_s;
    for (int i = k + 1 + tid; i < nd; i += blockDim.x) {
      const double l = A[(size_t)k * nd + i] * rk;
      A[(size_t)k * nd + i] = l;
      for (int j = k + 1; j < ke; ++j) A[(size_t)j * nd + i] -= l * rowk[j - kb];
    }
    __syncthreads();
  }
}

// U12 = L11^{-1} A12: columns [ke, nd) of rows [kb, ke); a warp per column,
// lane l holding rows kb + l and kb + 32 + l; L11 staged in shared memory.
__global__ void __launch_bounds__(256) k_blu_trsm(int nd, long long nnzlu, int dense_base, double *LU, int kb,
                                                  int ke) {
  __shared__ double L11[PB][PB + 1];
  const int sc = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double *A = LU + (size_t)sc * nnzlu + dense_base;
  const int pb = ke - kb;
  for (int e = tid; e < pb * pb; e += blockDim.x) {
    const int i = e % pb, k = e / pb;  // column k of L11 is contiguous in i
    L11[i][k] = A[(size_t)(kb + k) * nd + kb + i];
  }
  __syncthreads();
  const int j = ke + blockIdx.x * 8 + warp;
  if (j >= nd) return;
  double *col = A + (size_t)j * nd + kb;
  double x0 = lane < pb ? col[lane] : 0.0;
  double x1 = lane + 32 < pb ? col[lane + 32] : 0.0;
  for (int k = 0; k < pb; ++k) {
    const double xk = __shfl_sync(0xffffffffu, k < 32 ? x0 : x1, k & 31);
    if (lane > k && lane < pb) x0 = fma(-L11[lane][k], xk, x0);
    if (lane + 32 > k && lane + 32 < pb) x1 = fma(-L11[lane + 32][k], xk, x1);
  }
  if (lane < pb) col[lane] = x0;
  if (lane + 32 < pb) col[lane + 32] = x1;
}

// A22 -= L21 U12 over rows and columns [ke, nd), K = [kb, ke): 64 x 64 tiles,
// each thread a 4 x 4 block (rows m0 + 4 (t % 16) .., columns n0 + 4 (t / 16) ..,
// so a warp's stores of one column are 64 consecutive rows).
__global__ void __launch_bounds__(256) k_blu_gemm(int nd, long long nnzlu, int dense_base, double *LU, int kb,
                                                  int ke, int ntn) {
  // dynamic shared memory (above the 48 KB of static shared memory)
  extern __shared__ double smem_g[];
  double(*As)[TT] = reinterpret_cast<double(*)[TT]>(smem_g);                    // As[k][m] = L21(m, k)
  double(*Bs)[TT + 1] = reinterpret_cast<double(*)[TT + 1]>(smem_g + PB * TT);  // Bs[k][n] = U12(k, n)
  const int sc = blockIdx.y, tid = threadIdx.x;
  const int tm = blockIdx.x / ntn, tn = blockIdx.x % ntn;
  const int m0 = ke + tm * TT, n0 = ke + tn * TT, pb = ke - kb;
  double *A = LU + (size_t)sc * nnzlu + dense_base;
  for (int e = tid; e < PB * TT; e += blockDim.x) {
    const int m = e % TT, k = e / TT;
    As[k][m] = (k < pb && m0 + m < nd) ? A[(size_t)(kb + k) * nd + m0 + m] : 0.0;
    const int kk = e % PB, n = e / PB;
    Bs[kk][n] = (kk < pb && n0 + n < nd) ? A[(size_t)(n0 + n) * nd + kb + kk] : 0.0;
  }
  __syncthreads();
  const int mi = (tid % 16) * 4, ni = (tid / 16) * 4;
  double c[4][4] = {};
  for (int k = 0; k < pb; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[k][mi + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[k][ni + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) c[i][j] = fma(a[i], b[j], c[i][j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + ni + j;
    if (n >= nd) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + mi + i;
      if (m < nd) A[(size_t)n * nd + m] -= c[i][j];
    }
  }
}

// ---- multi-RHS solve through the block ------------------------------------

// Diagonal block [kb, ke) of X = Z[t0 + .][0 .. nu) (row-major, ld nu):
// lower: x = L11^{-1} x (unit diagonal); upper: x = U11^{-1} x with the
// reciprocal pivots.  A thread per right-hand-side column.
template <typename T, bool UPPER>
__global__ void __launch_bounds__(128) k_btrsm_diag(int nd, int nx, int t0, int nu, long long nnzlu, int dense_base,
                                                    const double *__restrict__ LU, const double *__restrict__ rd,
                                                    T *Z, int kb, int ke) {
  __shared__ T F[PB][PB + 1];
  __shared__ T rpiv[PB];
  const int sc = blockIdx.y, tid = threadIdx.x, pb = ke - kb;
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  for (int e = tid; e < pb * pb; e += blockDim.x) {
    const int i = e % pb, k = e / pb;
    F[i][k] = (T)A[(size_t)(kb + k) * nd + kb + i];
  }
  if (UPPER)
    for (int i = tid; i < pb; i += blockDim.x) rpiv[i] = (T)rd[(size_t)sc * nx + t0 + kb + i];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + tid;
  if (j >= nu) return;
  T *X = Z + (size_t)sc * nx * nu + (size_t)(t0 + kb) * nu + j;
  T x[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i) x[i] = i < pb ? X[(size_t)i * nu] : (T)0;
  if (!UPPER) {
#pragma unroll
    for (int i = 1; i < PB; ++i) {
      T acc = x[i];
#pragma unroll
      for (int k = 0; k < i; ++k) acc -= F[i][k] * x[k];
      x[i] = acc;
    }
  } else {
#pragma unroll
    for (int i = PB - 1; i >= 0; --i) {
      if (i < pb) {
        T acc = x[i];
#pragma unroll
        for (int k = i + 1; k < PB; ++k)
          if (k < pb) acc -= F[i][k] * x[k];
        x[i] = acc * rpiv[i];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < PB; ++i)
    if (i < pb) X[(size_t)i * nu] = x[i];
}

// X[rows] -= F[rows][kb:ke) X[kb:ke), rows = [ke, nd) (lower) or [0, kb)
// (upper): 64 x 64 tiles of X over (tile, scenario), each thread a 4 x 4
// block (columns 4 (t % 16) .., rows 4 (t / 16) ..: a warp's loads and
// stores of one row are 64 consecutive columns).
template <typename T, bool UPPER>
__global__ void __launch_bounds__(256) k_btrsm_update(int nd, int nx, int t0, int nu, long long nnzlu, int dense_base,
                                                      const double *__restrict__ LU, T *Z, int kb, int ke, int ntn) {
  extern __shared__ __align__(16) unsigned char smem_u[];
  T(*Fs)[TT + 1] = reinterpret_cast<T(*)[TT + 1]>(smem_u);                           // Fs[k][m] = F(m0 + m, kb + k)
  T(*Xs)[TT] = reinterpret_cast<T(*)[TT]>(smem_u + sizeof(T) * PB * (TT + 1));        // Xs[k][n] = X(kb + k, n0 + n)
  const int sc = blockIdx.y, tid = threadIdx.x;
  const int tm = blockIdx.x / ntn, tn = blockIdx.x % ntn;
  const int r0 = UPPER ? 0 : ke, r1 = UPPER ? kb : nd;
  const int m0 = r0 + tm * TT, n0 = tn * TT, pb = ke - kb;
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  T *X = Z + (size_t)sc * nx * nu + (size_t)t0 * nu;
  for (int e = tid; e < PB * TT; e += blockDim.x) {
    const int m = e % TT, k = e / TT;
    Fs[k][m] = (k < pb && m0 + m < r1) ? (T)A[(size_t)(kb + k) * nd + m0 + m] : (T)0;
    const int n = e % TT, kk = e / TT;
    Xs[kk][n] = (kk < pb && n0 + n < nu) ? X[(size_t)(kb + kk) * nu + n0 + n] : (T)0;
  }
  __syncthreads();
  const int ni = (tid % 16) * 4, mi = (tid / 16) * 4;
  T c[4][4] = {};
  for (int k = 0; k < pb; ++k) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Fs[k][mi + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Xs[k][ni + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) c[i][j] = fma(a[i], b[j], c[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + mi + i;
    if (m >= r1) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + ni + j;
      if (n < nu) X[(size_t)m * nu + n] -= c[i][j];
    }
  }
}

template <typename T>
constexpr size_t update_smem() { return sizeof(T) * PB * (TT + 1) + sizeof(T) * PB * TT; }
constexpr size_t gemm_smem() { return sizeof(double) * PB * TT + sizeof(double) * PB * (TT + 1); }

template <typename T>
void btrsm(const DevSym &S, const double *LU, const double *rd, T *Z, cudaStream_t st) {
  static const bool cap_l = cudaFuncSetAttribute(k_btrsm_update<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)update_smem<T>()) == cudaSuccess;
  static const bool cap_u = cudaFuncSetAttribute(k_btrsm_update<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)update_smem<T>()) == cudaSuccess;
  (void)cap_l;
  (void)cap_u;
  const int nd = S.nd, nu = S.nu, ntn = (nu + TT - 1) / TT;
  const dim3 gdiag((nu + 127) / 128, S.N);
  for (int kb = 0; kb < nd; kb += PB) {
    const int ke = kb + PB < nd ? kb + PB : nd;
    k_btrsm_diag<T, false><<<gdiag, 128, 0, st>>>(nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU, rd, Z, kb, ke);
    ipm_count_launch();
    if (ke < nd) {
      const int ntm = (nd - ke + TT - 1) / TT;
      k_btrsm_update<T, false><<<dim3(ntm * ntn, S.N), 256, update_smem<T>(), st>>>(nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU,
                                                                     Z, kb, ke, ntn);
      ipm_count_launch();
    }
  }
  for (int kb = ((nd - 1) / PB) * PB; kb >= 0; kb -= PB) {
    const int ke = kb + PB < nd ? kb + PB : nd;
    k_btrsm_diag<T, true><<<gdiag, 128, 0, st>>>(nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU, rd, Z, kb, ke);
    ipm_count_launch();
    if (kb > 0) {
      const int ntm = (kb + TT - 1) / TT;
      k_btrsm_update<T, true><<<dim3(ntm * ntn, S.N), 256, update_smem<T>(), st>>>(nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU, Z,
                                                                    kb, ke, ntn);
      ipm_count_launch();
    }
  }
}

}  // namespace

void launch_big_lu_dense(const DevSym &S, double *LU, double *rd, const double *amax, int *flags, cudaStream_t st,
                         const EmuLuPlan *emu_lu) {
  static const bool cap = cudaFuncSetAttribute(k_blu_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)gemm_smem()) == cudaSuccess;
  (void)cap;
  const int nd = S.nd;
  for (int kb = 0; kb < nd; kb += PB) {
    const int ke = kb + PB < nd ? kb + PB : nd;
    k_blu_panel<<<S.N, 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, amax, 1e-14, flags, kb, ke);
    ipm_count_launch();
    if (ke >= nd) break;
    k_blu_trsm<<<dim3((nd - ke + 7) / 8, S.N), 256, 0, st>>>(nd, S.nnzLU, S.dense_base, LU, kb, ke);
    ipm_count_launch();
    if (emu_lu) {
      // FP64-grade on the tensor cores (exact 7-bit slices of L21, U12)
      launch_emu_lu_update(*emu_lu, LU, S.nnzLU, S.dense_base, kb, ke, flags, st);
    } else {
      const int nt = (nd - ke + TT - 1) / TT;
      k_blu_gemm<<<dim3(nt * nt, S.N), 256, gemm_smem(), st>>>(nd, S.nnzLU, S.dense_base, LU, kb, ke, nt);
      ipm_count_launch();
    }
  }
}

void launch_big_trsm64(const DevSym &S, const double *LU, const double *rd, double *Z, cudaStream_t st) {
  btrsm<double>(S, LU, rd, Z, st);
}
void launch_big_trsm32(const DevSym &S, const double *LU, const double *rd, float *Z, cudaStream_t st) {
  btrsm<float>(S, LU, rd, Z, st);
}
