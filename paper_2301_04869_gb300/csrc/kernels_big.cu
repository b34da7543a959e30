// Large dense trailing block of the static-pivot LU of G_x (global memory).
//
// On the 10,000-bus networks the minimum-degree order ends in a dense block
// of about 1,800 states; it cannot live in one SM's shared memory as the
// smaller blocks do.  Here it is stored per scenario column-major with
// leading dimension nd (its entry (a, b) at LU + dense_base + b nd + a) and
// factored and solved by batched blocked kernels over all scenarios:
//
//  * LU (right-looking, panels of PB columns, static diagonal pivots as in
//    the rest of the factorization): per panel, its diagonal block (one CTA
//    per scenario, in shared memory), L21 = A21 U11^{-1} (a thread per row),
//    U12 = L11^{-1} A12 (a warp per column), and the trailing update
//    A22 -= L21 U12 as 64 x 64 FP64 tiles over (tile, scenario) or on the
//    tensor cores;
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

// The panel (columns [kb, ke) of rows [kb, nd)) in two kernels, so that its
// rows are worked on by many CTAs at once rather than by one CTA walking the
// 64 columns over all nd rows in global memory.  First the 64 x 64 diagonal
// block of scenario blockIdx.x in shared memory: L11 (unit lower,
// multipliers scaled by the reciprocal pivots) and U11, the reciprocal
// pivots to rd.
__global__ void __launch_bounds__(256) k_blu_diag(int nd, int nx, int t0, long long nnzlu, int dense_base, double *LU,
                                                  double *rd, const double *amax, double piv_tol, int *flags, int kb,
                                                  int ke) {
  __shared__ double D[PB][PB + 1];
  __shared__ double rk_s;
  const int sc = blockIdx.x, tid = threadIdx.x, bd = blockDim.x, pb = ke - kb;
  double *A = LU + (size_t)sc * nnzlu + dense_base;
  for (int e = tid; e < pb * pb; e += bd) {
    const int i = e % pb, j = e / pb;  // column j contiguous in i
    D[i][j] = A[(size_t)(kb + j) * nd + kb + i];
  }
  __syncthreads();
  const double ref = amax[sc];
  for (int k = 0; k < pb; ++k) {
    if (tid == 0) {
      const double d = D[k][k];
      if (!(fabs(d) > piv_tol * ref)) flags[FLAG_SINGULAR] = 1;
      rk_s = 1.0 / d;
      rd[(size_t)sc * nx + t0 + kb + k] = rk_s;
    }
    __syncthreads();
    const int w = pb - k - 1;
    for (int i = k + 1 + tid; i < pb; i += bd) D[i][k] *= rk_s;
    __syncthreads();
    for (int e = tid; e < w * w; e += bd) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      D[i][j] -= D[i][k] * D[k][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < pb * pb; e += bd) {
    const int i = e % pb, j = e / pb;
    A[(size_t)(kb + j) * nd + kb + i] = D[i][j];
  }
}

// Then L21 = A21 U11^{-1} for the rows [ke, nd): a thread per row, the row's
// panel entries in registers, U11 and the reciprocal pivots in shared memory
// (read as broadcasts).  Each row goes through the same multiply-adds in the
// same order as in the one-CTA panel.  Grid (ceil((nd - ke) / 128), N).
__global__ void __launch_bounds__(128) k_blu_l21(int nd, int nx, int t0, long long nnzlu, int dense_base, double *LU,
                                                 const double *__restrict__ rd, int kb, int ke) {
  __shared__ double U[PB][PB];
  __shared__ double rk[PB];
  const int sc = blockIdx.y, tid = threadIdx.x, pb = ke - kb;
  double *A = LU + (size_t)sc * nnzlu + dense_base;
  for (int e = tid; e < PB * PB; e += blockDim.x) {
    const int k = e % PB, m = e / PB;  // column m of U11 contiguous in k
    U[k][m] = (k < pb && m < pb && k < m) ? A[(size_t)(kb + m) * nd + kb + k] : 0.0;
  }
  for (int k = tid; k < PB; k += blockDim.x) rk[k] = k < pb ? rd[(size_t)sc * nx + t0 + kb + k] : 0.0;
  __syncthreads();
  const int i = ke + blockIdx.x * 128 + tid;
  if (i >= nd) return;
  double a[PB];
#pragma unroll
  for (int c = 0; c < PB; ++c) a[c] = c < pb ? A[(size_t)(kb + c) * nd + i] : 0.0;
#pragma unroll
  for (int k = 0; k < PB; ++k) {
    if (k < pb) {
      const double x = a[k] * rk[k];
      a[k] = x;
#pragma unroll
      for (int m = k + 1; m < PB; ++m) a[m] -= x * U[k][m];
    }
  }
#pragma unroll
  for (int c = 0; c < PB; ++c)
    if (c < pb) A[(size_t)(kb + c) * nd + i] = a[c];
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

// X[rows] -= F[rows][kb:ke) X[kb:ke), rows = [r0, r1) (below ke for lower,
// above kb for upper): 64 x 64 tiles of X over (tile, scenario), each thread
// a 4 x 4 block (columns 4 (t % 16) .., rows 4 (t / 16) ..: a warp's loads
// and stores of one row are 64 consecutive columns).
template <typename T, bool UPPER>
__global__ void __launch_bounds__(256) k_btrsm_update(int nd, int nx, int t0, int nu, long long nnzlu, int dense_base,
                                                      const double *__restrict__ LU, T *Z, int kb, int ke, int ntn,
                                                      int r0, int r1) {
  extern __shared__ __align__(16) unsigned char smem_u[];
  T(*Fs)[TT + 1] = reinterpret_cast<T(*)[TT + 1]>(smem_u);                           // Fs[k][m] = F(m0 + m, kb + k)
  T(*Xs)[TT] = reinterpret_cast<T(*)[TT]>(smem_u + sizeof(T) * PB * (TT + 1));        // Xs[k][n] = X(kb + k, n0 + n)
  const int sc = blockIdx.y, tid = threadIdx.x;
  const int tm = blockIdx.x / ntn, tn = blockIdx.x % ntn;
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
void btrsm_caps() {
  static const bool cap_l = cudaFuncSetAttribute(k_btrsm_update<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)update_smem<T>()) == cudaSuccess;
  static const bool cap_u = cudaFuncSetAttribute(k_btrsm_update<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)update_smem<T>()) == cudaSuccess;
  (void)cap_l;
  (void)cap_u;
}

// the diagonal block [kb, ke) of the lower (upper) solve, then the update of
// the rows [r0, r1) by it
template <typename T, bool UPPER>
void btrsm_step(const DevSym &S, const double *LU, const double *rd, T *Z, int kb, int ke, int r0, int r1,
                cudaStream_t st) {
  const int nu = S.nu, ntn = (nu + TT - 1) / TT;
  const dim3 gdiag((nu + 127) / 128, S.N);
  k_btrsm_diag<T, UPPER><<<gdiag, 128, 0, st>>>(S.nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU, rd, Z, kb, ke);
  ipm_count_launch();
  if (r1 > r0) {
    const int ntm = (r1 - r0 + TT - 1) / TT;
    k_btrsm_update<T, UPPER><<<dim3(ntm * ntn, S.N), 256, update_smem<T>(), st>>>(
        S.nd, S.nx, S.t0, nu, S.nnzLU, S.dense_base, LU, Z, kb, ke, ntn, r0, r1);
    ipm_count_launch();
  }
}

template <typename T>
void btrsm(const DevSym &S, const double *LU, const double *rd, T *Z, cudaStream_t st) {
  btrsm_caps<T>();
  const int nd = S.nd;
  for (int kb = 0; kb < nd; kb += PB) {
    const int ke = kb + PB < nd ? kb + PB : nd;
    btrsm_step<T, false>(S, LU, rd, Z, kb, ke, ke, nd, st);
  }
  for (int kb = ((nd - 1) / PB) * PB; kb >= 0; kb -= PB) {
    const int ke = kb + PB < nd ? kb + PB : nd;
    btrsm_step<T, true>(S, LU, rd, Z, kb, ke, 0, kb, st);
  }
}

// The same solve, left-looking by row blocks of RB = 128 with the products of
// each block against every finished row on the tensor cores (BF16x3, FP32
// accumulation; kernels_tcsolve.cu); the 128 x 128 diagonal blocks by the
// SIMT kernels above, two 64-row steps each.
constexpr int RB = 128;
void btrsm_tc(const DevSym &S, const double *LU, const double *rd, float *Z, const TcsPlan &P, int *flags,
              cudaStream_t st) {
  btrsm_caps<float>();
  const int nd = S.nd, nb = (nd + RB - 1) / RB;
  launch_tcs_split_f(P, LU, S.nnzLU, S.dense_base, st);
  for (int b = 0; b < nb; ++b) {
    const int r0 = b * RB, r1 = r0 + RB < nd ? r0 + RB : nd, rm = r0 + PB < r1 ? r0 + PB : r1;
    launch_tcs_update(P, S.nx, S.t0, Z, r0, r1, 0, r0, flags, st);  // rows above, through L_dd
    btrsm_step<float, false>(S, LU, rd, Z, r0, rm, rm, r1, st);
    if (rm < r1) btrsm_step<float, false>(S, LU, rd, Z, rm, r1, r1, r1, st);
    if (b + 1 < nb) launch_tcs_split_x(P, S.nx, S.t0, Z, r0, r1, st);
  }
  for (int b = nb - 1; b >= 0; --b) {
    const int r0 = b * RB, r1 = r0 + RB < nd ? r0 + RB : nd, rm = r0 + PB < r1 ? r0 + PB : r1;
    launch_tcs_update(P, S.nx, S.t0, Z, r0, r1, r1, nd, flags, st);  // rows below, through U_dd
    if (rm < r1) btrsm_step<float, true>(S, LU, rd, Z, rm, r1, r0, rm, st);
    btrsm_step<float, true>(S, LU, rd, Z, r0, rm, r0, r0, st);
    if (b > 0) launch_tcs_split_x(P, S.nx, S.t0, Z, r0, r1, st);
  }
}

// ---- one vector per scenario through the block ------------------------------
//
// T(i, k) is the entry of the triangular factor a sweep applies: forward
// (lower) T = L, or U^T with trans; backward (upper) T = U, or L^T with
// trans.  In the column-major block T(i, k) = LU[k nd + i] without trans and
// LU[i nd + k] with it; the sweeps that apply U or U^T multiply by the
// reciprocal pivots.  Blocked by VB rows: a launch per block applies the
// block's solved values to every later row, 64 rows per CTA over (chunk,
// scenario), so the factor streams through many SMs at once; the CTA holding
// the next block's rows then solves that diagonal block (a warp, in shared
// memory).
constexpr int VB = 64;

template <bool TRANS>
__device__ __forceinline__ double tval(const double *A, int nd, int i, int k) {
  return TRANS ? A[(size_t)i * nd + k] : A[(size_t)k * nd + i];
}

// the diagonal block [b0, b1) (at most VB rows) in place on xs (indexed from
// b0); called by the whole CTA
template <bool TRANS, bool UPPER>
__device__ void trsv_diag(const double *A, const double *r, int nd, int b0, int b1, double *xs,
                          double (*Dg)[VB + 1]) {
  const int tid = threadIdx.x, w = b1 - b0;
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e % w, k = e / w;
    Dg[i][k] = tval<TRANS>(A, nd, b0 + i, b0 + k);
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    constexpr bool scale = TRANS != UPPER;  // U^T going down or U coming up
    double y0 = lane < w ? xs[lane] : 0.0, y1 = lane + 32 < w ? xs[lane + 32] : 0.0;
    for (int s = 0; s < w; ++s) {
      const int k = UPPER ? w - 1 - s : s;
      double own = k < 32 ? y0 : y1;
      if (scale) own *= r[b0 + k];
      const double xk = __shfl_sync(0xffffffffu, own, k & 31);
      if ((k & 31) == lane) {
        if (k < 32) y0 = xk;
        else y1 = xk;
      }
      if (UPPER) {
        if (lane < k) y0 = fma(-Dg[lane][k], xk, y0);
        if (lane + 32 < k) y1 = fma(-Dg[lane + 32][k], xk, y1);
      } else {
        if (lane > k && lane < w) y0 = fma(-Dg[lane][k], xk, y0);
        if (lane + 32 > k && lane + 32 < w) y1 = fma(-Dg[lane + 32][k], xk, y1);
      }
    }
    if (lane < w) xs[lane] = y0;
    if (lane + 32 < w) xs[lane + 32] = y1;
  }
  __syncthreads();
}

// the first diagonal block of a sweep (lower: [0, VB), upper: the last one)
template <bool TRANS, bool UPPER>
__global__ void __launch_bounds__(256) k_trsv_first(int nd, int nx, int t0, long long nnzlu, int dense_base,
                                                    const double *__restrict__ LU, const double *__restrict__ rd,
                                                    double *v) {
  __shared__ double xs[VB];
  __shared__ double Dg[VB][VB + 1];
  const int sc = blockIdx.x, tid = threadIdx.x;
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  const double *r = rd + (size_t)sc * nx + t0;
  double *x = v + (size_t)sc * nx + t0;
  const int b0 = UPPER ? ((nd - 1) / VB) * VB : 0, b1 = UPPER ? nd : min(nd, VB);
  if (tid < b1 - b0) xs[tid] = x[b0 + tid];
  __syncthreads();
  trsv_diag<TRANS, UPPER>(A, r, nd, b0, b1, xs, Dg);
  if (tid < b1 - b0) x[b0 + tid] = xs[tid];
}

// rows of chunk blockIdx.x minus T(rows, [kb, ke)) x([kb, ke)); chunk 0 is
// the next diagonal block (lower: [ke, ke + VB), upper: [kb - VB, kb)),
// solved after its update.  Grid (chunks, N), 256 threads.
template <bool TRANS, bool UPPER>
__global__ void __launch_bounds__(256) k_trsv_step(int nd, int nx, int t0, long long nnzlu, int dense_base,
                                                   const double *__restrict__ LU, const double *__restrict__ rd,
                                                   double *v, int kb, int ke) {
  __shared__ double xk[VB];
  __shared__ double part[4][VB];
  __shared__ double xs[VB];
  __shared__ double Dg[VB][VB + 1];
  const int sc = blockIdx.y, tid = threadIdx.x, c = blockIdx.x;
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  const double *r = rd + (size_t)sc * nx + t0;
  double *x = v + (size_t)sc * nx + t0;
  int c0, c1;
  if (UPPER) {
    c1 = kb - VB * c;
    c0 = c1 - VB > 0 ? c1 - VB : 0;
  } else {
    c0 = ke + VB * c;
    c1 = c0 + VB < nd ? c0 + VB : nd;
  }
  const int w = ke - kb, h = c1 - c0;
  if (tid < VB) xk[tid] = tid < w ? x[kb + tid] : 0.0;
  __syncthreads();
  if (!TRANS) {
    // T(i, k) = LU[k nd + i]: a thread per (row, 16 columns), loads along the rows
    const int rr = tid & (VB - 1), g = tid >> 6;
    double s = 0.0;
    if (rr < h)
      for (int j = 16 * g; j < 16 * g + 16 && j < w; ++j) s = fma(A[(size_t)(kb + j) * nd + c0 + rr], xk[j], s);
    part[g][rr] = s;
  } else {
    // T(i, k) = LU[i nd + k]: a warp per (row group, 32 columns), lanes along the columns
    const int wp = tid >> 5, lane = tid & 31, rg = wp >> 1, hf = wp & 1, j = 32 * hf + lane;
    const double xj = xk[j];
    for (int m = 0; m < VB / 4; ++m) {
      const int rr = rg + 4 * m;
      double p = (rr < h && j < w) ? A[(size_t)(c0 + rr) * nd + kb + j] * xj : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == 0) part[hf][rr] = p;
    }
    if (tid < VB) part[2][tid] = part[3][tid] = 0.0;
  }
  __syncthreads();
  if (tid < h) {
    const double nv = x[c0 + tid] - ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]));
    xs[tid] = nv;
    if (c != 0) x[c0 + tid] = nv;
  }
  __syncthreads();
  if (c == 0) {
    trsv_diag<TRANS, UPPER>(A, r, nd, c0, c1, xs, Dg);
    if (tid < h) x[c0 + tid] = xs[tid];
  }
}

template <bool TRANS>
void trsv_sweeps(const DevSym &S, const double *LU, const double *rd, double *v, cudaStream_t st) {
  const int nd = S.nd;
  k_trsv_first<TRANS, false><<<S.N, 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, v);
  ipm_count_launch();
  for (int kb = 0; kb + VB < nd; kb += VB) {
    const int ke = kb + VB;
    k_trsv_step<TRANS, false><<<dim3((nd - ke + VB - 1) / VB, S.N), 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU,
                                                                                 S.dense_base, LU, rd, v, kb, ke);
    ipm_count_launch();
  }
  const int lb = ((nd - 1) / VB) * VB;
  k_trsv_first<TRANS, true><<<S.N, 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, v);
  ipm_count_launch();
  for (int kb = lb; kb > 0; kb -= VB) {
    const int ke = kb + VB < nd ? kb + VB : nd;
    k_trsv_step<TRANS, true><<<dim3(kb / VB, S.N), 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, v,
                                                                kb, ke);
    ipm_count_launch();
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
    k_blu_diag<<<S.N, 256, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, amax, 1e-14, flags, kb, ke);
    ipm_count_launch();
    if (ke >= nd) break;
    k_blu_l21<<<dim3((nd - ke + 127) / 128, S.N), 128, 0, st>>>(nd, S.nx, S.t0, S.nnzLU, S.dense_base, LU, rd, kb,
                                                                 ke);
    ipm_count_launch();
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
void launch_big_trsm32(const DevSym &S, const double *LU, const double *rd, float *Z, cudaStream_t st,
                       const TcsPlan *tcs, int *flags) {
  if (tcs && flags) {
    btrsm_tc(S, LU, rd, Z, *tcs, flags, st);
    return;
  }
  btrsm<float>(S, LU, rd, Z, st);
}

void launch_big_trsv(const DevSym &S, const double *LU, const double *rd, double *v, int trans, cudaStream_t st) {
  if (trans) trsv_sweeps<true>(S, LU, rd, v, st);
  else trsv_sweeps<false>(S, LU, rd, v, st);
}
