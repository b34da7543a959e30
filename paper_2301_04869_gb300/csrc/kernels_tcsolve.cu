// Multi-RHS solve through the large dense trailing block on the tensor cores
// (mixed path): the block updates of Z_d = U_dd^{-1} L_dd^{-1} R_d as
// three-term BF16 split products (tcgen05, FP32 accumulation).
//
// Z_d (the block's n_u right-hand sides, FP32, row-major with leading
// dimension n_u) is solved left-looking in row blocks of 128: for the rows R
// of a block, first R -= F(R, K) Z_d(K) with K every row already final (the
// rows above R going down through L_dd, the rows below R coming back up
// through U_dd) -- one product on the tensor cores -- then the 128 x 128
// diagonal block of R by the SIMT triangular kernels, then the three BF16
// terms of the finished rows are written for the products of the later
// blocks.  Both operands are split as a = a1 + a2 + a3 (round to nearest of
// successive remainders) and the six products a_i b_j with i + j <= 4 are
// accumulated, which reproduces the FP32 product to about 2^-24 relative;
// the factor is split once per factorization from FP64.
//
// Operand layout (K-major, the contraction index contiguous, so one TMA box
// row is 64 BF16 = 128 bytes, 128-byte swizzle):
//  * F planes [3][N ndp][kpl]: row s ndp + m holds row m of scenario s's
//    factor block, F(m, k) = LU(m, k) (L below the diagonal, U above);
//  * X planes [3][N nup][kpl]: row s nup + j holds column j of Z_d, X(k, j)
//    at position k;
// with ndp = kpl = nd rounded up to 128 and nup = n_u rounded up to 128; the
// padding is zero from the allocation on and never written, so a tile that
// passes the block's edge reads zeros.
//
// §3.2 "Local reduction": Z = -G_x^{-1} G_u by a batched sparse LU sharing
// one pattern; the dense trailing block is the part of that solve where every
// entry is filled, and its updates are the dense products the tensor cores
// are for.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "dev.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace tcs {

using namespace tcx;

constexpr int BM = 128, BN = 128, BK = 64;  // output tile (rows of R x columns of Z_d), K block
constexpr int STAGES = 2;
constexpr int PLANE_BYTES = BM * BK * 2;     // 16 KB: one operand plane of one K block
constexpr int STAGE_BYTES = 6 * PLANE_BYTES;  // 3 F planes + 3 X planes
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

struct Maps {
  CUtensorMap a[3], b[3];
};

// Z_d(r0 + i, n0 + j) -= sum_k F(r0 + i, k) X(k, n0 + j) over the K blocks
// [kb0, kb0 + nkb) of 64, for r0 + i < r1, n0 + j < nu.  Grid (n tiles, N).
// Roles: warp 0 issues the TMA loads, warp 1 allocates TMEM and issues the
// MMAs, warps 2-5 drain each K block's accumulator into FP32 registers (the
// tensor core's FP32 accumulation is kept to one K block) and finally
// subtract the tile from Z_d.  Every mbarrier wait is bounded: past the limit
// the kernel raises FLAG_TIMEOUT, stops issuing, lets its copies land and
// frees its TMEM; the tile is then left unchanged.
__global__ void __launch_bounds__(192, 1) k_tcs_update(const __grid_constant__ Maps maps, int ndp, int nup, int nx,
                                                       int t0, int nu, int r0, int r1, int kb0, int nkb, float *Z,
                                                       int *flags) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;  // [2]
  uint64_t *acc_empty = acc_full + 2;   // [2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sc = blockIdx.y, n0 = blockIdx.x * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // TMEM: two 128-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    const int ya = sc * ndp + r0, yb = sc * nup + n0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) - 1) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t *st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int kx = (kb0 + i) * BK;
      for (int p = 0; p < 3; ++p) tma_load_2d(st + p * PLANE_BYTES, &maps.a[p], &full[s], kx, ya);
      for (int p = 0; p < 3; ++p) tma_load_2d(st + (3 + p) * PLANE_BYTES, &maps.b[p], &full[s], kx, yb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: per K block, 4 steps of 16 x 6 split products into buffer i & 1
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    const int pa[6] = {0, 0, 1, 0, 1, 2};
    const int pb[6] = {0, 1, 0, 2, 1, 0};
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES, b = i & 1;
      if (!mbar_wait(&full[s], (i / STAGES) & 1) ||
          (i >= 2 && !mbar_wait(&acc_empty[b], ((i >> 1) - 1) & 1))) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = sdesc(base + pa[q] * PLANE_BYTES + kk * 32);
          const uint64_t db = sdesc(base + (3 + pb[q]) * PLANE_BYTES + kk * 32);
          mma_bf16(d, da, db, idesc, (kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
      mma_commit(&acc_full[b]);
    }
  } else if (warp >= 2) {
    // epilogue: a thread per output row (the warp's TMEM lane quarter)
    const int q = warp & 3;
    const int row = q * 32 + lane;
    float acc[BN];
#pragma unroll
    for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
    for (int i = 0; i < nkb; ++i) {
      const int b = i & 1;
      if (!mbar_wait(&acc_full[b], (i >> 1) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[c0 + e] += __uint_as_float(v[e]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
    }
    // the stage buffers are idle once the last accumulator has been drained:
    // the tile goes through shared memory so that the subtraction from Z_d
    // reads and writes whole rows (a warp per row, lanes along the columns)
    asm volatile("bar.sync 1, 128;" ::: "memory");
    float *T = reinterpret_cast<float *>(smem);  // [BM][BN + 1]
#pragma unroll
    for (int c = 0; c < BN; ++c) T[row * (BN + 1) + c] = acc[c];
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (!*abort_flag) {
      const int ew = warp - 2;  // 0..3
      for (int rr = ew; rr < BM; rr += 4) {
        const int r = r0 + rr;
        if (r >= r1) break;
        float *X = Z + (size_t)sc * nx * nu + (size_t)(t0 + r) * nu + n0;
        for (int c = lane; c < BN && n0 + c < nu; c += 32) X[c] -= T[rr * (BN + 1) + c];
      }
    }
  }
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int s = 0; s < STAGES; ++s) (void)mbar_wait(&full[s], 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

__device__ __forceinline__ void split3(double a, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __double2bfloat16(a);
  const double r1 = a - (double)__bfloat162float(h);
  m = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(m);
  l = __double2bfloat16(r2);
}

// F planes of the factor block: F(m, k) = LU(m, k) for m, k < nd, read
// column-major (m contiguous) and written K-major through 32 x 32 shared
// transposes.  Grid (ceil(nd/32) m tiles, ceil(nd/32) k tiles, N).
__global__ void k_tcs_split_f(int nd, int ndp, long long kpl, long long nnzlu, int dense_base,
                              const double *__restrict__ LU, __nv_bfloat16 *planes, size_t plane) {
  __shared__ double t[32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32, sc = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, m = m0 + tx;
    t[r][tx] = (k < nd && m < nd) ? A[(size_t)k * nd + m] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int m = m0 + r, k = k0 + tx;
    if (m < nd && k < nd) {
      __nv_bfloat16 h, mi, l;
      split3(t[tx][r], h, mi, l);
      const size_t o = ((size_t)sc * ndp + m) * (size_t)kpl + k;
      planes[o] = h;
      planes[plane + o] = mi;
      planes[2 * plane + o] = l;
    }
  }
}

// X planes of the finished rows [r0, r1) of Z_d: X(k, j) = Z_d(k, j), read
// row-major (j contiguous) and written K-major.  Grid (ceil((r1-r0)/32),
// ceil(nu/32), N).
__global__ void k_tcs_split_x(int nx, int t0, int nu, int nup, long long kpl, int r0, int r1,
                              const float *__restrict__ Z, __nv_bfloat16 *planes, size_t plane) {
  __shared__ float t[32][33];
  const int k0 = r0 + blockIdx.x * 32, j0 = blockIdx.y * 32, sc = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float *X = Z + (size_t)sc * nx * nu + (size_t)t0 * nu;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, j = j0 + tx;
    t[r][tx] = (k < r1 && j < nu) ? X[(size_t)k * nu + j] : 0.0f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, k = k0 + tx;
    if (j < nu && k < r1) {
      __nv_bfloat16 h, mi, l;
      split3((double)t[tx][r], h, mi, l);
      const size_t o = ((size_t)sc * nup + j) * (size_t)kpl + k;
      planes[o] = h;
      planes[plane + o] = mi;
      planes[2 * plane + o] = l;
    }
  }
}

}  // namespace tcs

size_t tcs_planes_bytes(int N, int nd, int nu, size_t *f_bytes) {
  const long long ndp = (nd + 127) / 128 * 128, nup = (nu + 127) / 128 * 128;
  const size_t f = (size_t)3 * N * ndp * ndp * 2, x = (size_t)3 * N * nup * ndp * 2;
  if (f_bytes) *f_bytes = f;
  return f + x;
}

bool tcs_plan(TcsPlan &P, int N, int nd, int nu, void *planes) {
  P.N = N;
  P.nd = nd;
  P.nu = nu;
  P.ndp = (nd + 127) / 128 * 128;
  P.nup = (nu + 127) / 128 * 128;
  P.kpl = P.ndp;
  size_t fb = 0;
  tcs_planes_bytes(N, nd, nu, &fb);
  P.fpl = planes;
  P.xpl = (unsigned char *)planes + fb;
  tcs::Maps m;
  const size_t fplane = (size_t)N * P.ndp * P.kpl * 2, xplane = (size_t)N * P.nup * P.kpl * 2;
  for (int p = 0; p < 3; ++p) {
    if (!tc_make_kmajor_map(&m.a[p], (const char *)P.fpl + p * fplane, N * P.ndp, P.kpl)) return false;
    if (!tc_make_kmajor_map(&m.b[p], (const char *)P.xpl + p * xplane, N * P.nup, P.kpl)) return false;
  }
  static_assert(sizeof(tcs::Maps) <= sizeof(P.maps), "map storage");
  memcpy(P.maps, &m, sizeof(m));
  return true;
}

void launch_tcs_split_f(const TcsPlan &P, const double *LU, long long nnzlu, int dense_base, cudaStream_t st) {
  const size_t plane = (size_t)P.N * P.ndp * P.kpl;
  dim3 grid((P.nd + 31) / 32, (P.nd + 31) / 32, P.N);
  tcs::k_tcs_split_f<<<grid, dim3(32, 8), 0, st>>>(P.nd, P.ndp, P.kpl, nnzlu, dense_base, LU,
                                                   (__nv_bfloat16 *)P.fpl, plane);
  ipm_count_launch();
}

void launch_tcs_split_x(const TcsPlan &P, int nx, int t0, const float *Z, int r0, int r1, cudaStream_t st) {
  if (r1 <= r0) return;
  const size_t plane = (size_t)P.N * P.nup * P.kpl;
  dim3 grid((r1 - r0 + 31) / 32, (P.nu + 31) / 32, P.N);
  tcs::k_tcs_split_x<<<grid, dim3(32, 8), 0, st>>>(nx, t0, P.nu, P.nup, P.kpl, r0, r1, Z,
                                                   (__nv_bfloat16 *)P.xpl, plane);
  ipm_count_launch();
}

void launch_tcs_update(const TcsPlan &P, int nx, int t0, float *Z, int r0, int r1, int k0, int k1, int *flags,
                       cudaStream_t st) {
  if (r1 <= r0 || k1 <= k0) return;
  static const bool attr = cudaFuncSetAttribute(tcs::k_tcs_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                tcs::SMEM_BYTES) == cudaSuccess;
  (void)attr;
  tcs::Maps m;
  memcpy(&m, P.maps, sizeof(m));
  const int kb0 = k0 / tcs::BK, kb1 = (k1 + tcs::BK - 1) / tcs::BK;
  dim3 grid((P.nu + tcs::BN - 1) / tcs::BN, P.N);
  tcs::k_tcs_update<<<grid, 192, tcs::SMEM_BYTES, st>>>(m, P.ndp, P.nup, nx, t0, P.nu, r0, r1, kb0, kb1 - kb0, Z,
                                                        flags);
  ipm_count_launch();
}
