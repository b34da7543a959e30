// K6 (mixed path): the reduced Hessian sum_s Z_s^T Y_s on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators, TMA-staged operands).
//
// Each FP32 operand is split into three BF16 terms a = a1 + a2 + a3 (round to
// nearest of successive remainders).  The six products a_i b_j with
// i + j <= 4 -- (1,1) (1,2) (2,1) (1,3) (2,2) (3,1) -- accumulate into one
// FP32 accumulator in tensor memory, which reproduces a*b to about 2^-24
// relative (FP32 grade).  Operands arrive K-major: the multi-RHS solve writes
// the planes transposed, Zt[p][j][kappa] with kappa = s*n_x + row running over
// scenarios and rows, so the scenario sum of §3.2 (the MPI_Allreduce of the
// paper) is part of the contraction.  Tiles are 128 x 128 (one CTA, cta_group
// ::1), the K range is split into groups for one full wave, and each CTA
// writes its FP32 partial tile; a fixed-order pass adds the groups in FP64.
//
// Roles: warp 0 issues TMA loads (one elected lane), warp 1 allocates TMEM and
// issues tcgen05.mma (one elected lane), warps 2-5 drain the accumulator.
// Every mbarrier wait is bounded: past the limit the kernel records
// FLAG_TIMEOUT, stops issuing, lets its in-flight copies land (bounded) and
// frees its TMEM before returning.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "dev.cuh"
#include "kernels.h"
#include "tcgen05.cuh"


namespace tc {

using namespace tcx;

constexpr int BM = 128, BN = 128, BK = 64;              // tile; BK bf16 = one 128-byte swizzle row
constexpr int STAGES = 2;
constexpr int PLANE_BYTES = BM * BK * 2;                 // 16 KB per operand plane per stage
constexpr int STAGE_BYTES = 6 * PLANE_BYTES;             // 3 A planes + 3 B planes
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;  // + barriers, TMEM slot
// upper-triangle tile t -> (ti, tj), row-major over ti
__device__ __forceinline__ void tile_ij(int t, int nt1, int &ti, int &tj) {
  int i = 0, rem = t;
  while (rem >= nt1 - i) {
    rem -= nt1 - i;
    ++i;
  }
  ti = i;
  tj = i + rem;
}

struct Maps {
  CUtensorMap a[3], b[3];
};

// Accumulation: the tensor core's FP32 accumulation loses precision over long
// K, so every 64-wide K block (its 24 split products) accumulates into a fresh
// TMEM buffer (two buffers, double-buffered); the epilogue warps drain each
// buffer into round-to-nearest FP32 registers and flush those into this CTA's
// FP64 partial tile every FLUSH blocks.
constexpr int FLUSH = 16;

__global__ void __launch_bounds__(192, 1) k_tc_schur(const __grid_constant__ Maps maps, int nt1, int kb_total,
                                                     int kb_per_group, double *partial, int *flags) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;   // [2]
  uint64_t *acc_empty = acc_full + 2;    // [2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti, tj;
  tile_ij(blockIdx.x, nt1, ti, tj);
  const int kb0 = blockIdx.y * kb_per_group;
  const int kb1 = min(kb_total, kb0 + kb_per_group);
  const int nkb = kb1 - kb0;

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
  if (warp == 1) {  // TMEM: two 128-column FP32 accumulators (128 lanes each)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
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
      for (int p = 0; p < 3; ++p) tma_load_2d(st + p * PLANE_BYTES, &maps.a[p], &full[s], kx, ti * BM);
      for (int p = 0; p < 3; ++p) tma_load_2d(st + (3 + p) * PLANE_BYTES, &maps.b[p], &full[s], kx, tj * BN);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
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
      mma_commit(&empty[s]);     // stage reusable once these MMAs complete
      mma_commit(&acc_full[b]);  // accumulator b holds this block's sum
    }
  } else if (warp >= 2) {
    // epilogue: drain every block's accumulator into FP32 registers
    const int q = warp & 3;  // lane quarter this warp may access
    const int row = q * 32 + lane;
    double *out = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * BM * BN + (size_t)row * BN;
    float acc[BN];
#pragma unroll
    for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
    for (int c = 0; c < BN; ++c) out[c] = 0.0;
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
      if ((i + 1) % FLUSH == 0 || i + 1 == nkb) {
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          out[c] += (double)acc[c];
          acc[c] = 0.0f;
        }
      }
    }
  }
  // drain: if we aborted, let issued copies land before the CTA exits
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

}  // namespace tc

// ---------------------------------------------------------------------------
// FP32 [krows][nu] (row-major) -> three BF16 planes, transposed to [nu][kpad]
// (K-major for the MMA).  a1 = bf16(a), a2 = bf16(a - a1), a3 = bf16(a - a1 - a2).
namespace tc {

__device__ __forceinline__ void split3(float a, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

__global__ void k_split_t(long long krows, int nu, long long kpad, const float *__restrict__ src,
                          __nv_bfloat16 *planes) {
  // 32 x 32 transpose tiles through shared memory
  __shared__ float t[32][33];
  const long long k0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const long long k = k0 + r;
    const int j = j0 + tx;
    t[r][tx] = (k < krows && j < nu) ? src[k * nu + j] : 0.0f;
  }
  __syncthreads();
  const size_t plane = (size_t)nu * kpad;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r;
    const long long k = k0 + tx;
    if (j < nu && k < kpad) {
      __nv_bfloat16 h, m, l;
      split3(t[tx][r], h, m, l);
      const size_t o = (size_t)j * kpad + k;
      planes[o] = h;
      planes[plane + o] = m;
      planes[2 * plane + o] = l;
    }
  }
}

// K_hat (FP64, upper tiles mirrored) = sum over groups of the FP32 partial
// tiles (+ sum_s Yu_s + diag), groups added in index order
__global__ void k_tc_assemble(int nu, int N, int ngroups, int ntiles, int nt1, const double *__restrict__ partial,
                              const double *__restrict__ Yu, const double *__restrict__ diag, double *Khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int i = (int)(t / nu), j = (int)(t % nu);
  if (i > j) return;
  const int ti = i / BM, tj = j / BN;
  const int tt = ti * nt1 - ti * (ti - 1) / 2 + (tj - ti);
  double v = 0.0;
  for (int g = 0; g < ngroups; ++g)
    v += partial[((size_t)g * ntiles + tt) * BM * BN + (size_t)(i - ti * BM) * BN + (j - tj * BN)];
  if (Yu)
    for (int s = 0; s < N; ++s) v += Yu[(size_t)s * nu * nu + (size_t)i * nu + j];
  if (diag && i == j) v += diag[i];
  Khat[(size_t)i * nu + j] = v;
  Khat[(size_t)j * nu + i] = v;
}

}  // namespace tc

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

// tensor map of one BF16 plane [rows][kpad], box 64 (K) x box_rows, 128-byte swizzle
static bool make_map(CUtensorMap *m, const void *base, int rows, long long kpad, int box_rows = tc::BM,
                     int box_k = tc::BK) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  // 128-byte rows (64 BF16) take the 128-byte swizzle, 64-byte rows the 64-byte one
  const CUtensorMapSwizzle sw = box_k * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_make_kmajor_map(void *map, const void *base, int rows, long long k) {
  return make_map(reinterpret_cast<CUtensorMap *>(map), base, rows, k);
}

bool tc_make_kmajor_map_box(void *map, const void *base, int rows, long long k, int box_rows, int box_k) {
  if (box_k != 32 && box_k != 64) return false;
  return make_map(reinterpret_cast<CUtensorMap *>(map), base, rows, k, box_rows, box_k);
}

void tc_plan(int nu, long long krows, TcPlan &P) {
  P.nu = nu;
  P.kpad = (krows + tc::BK - 1) / tc::BK * tc::BK;
  P.nt1 = (nu + tc::BM - 1) / tc::BM;
  P.ntiles = P.nt1 * (P.nt1 + 1) / 2;
  P.kb_total = (int)(P.kpad / tc::BK);
  tc_regroup(P, 152 / P.ntiles);  // one CTA per SM (the stage buffers take ~193 KB of shared memory)
}

void tc_regroup(TcPlan &P, int G) {
  if (G < 1) G = 1;
  if (G > P.kb_total) G = P.kb_total;
  P.kb_per_group = (P.kb_total + G - 1) / G;
  P.ngroups = (P.kb_total + P.kb_per_group - 1) / P.kb_per_group;
}

bool tc_set_operands(TcPlan &P, const void *a_planes, const void *b_planes) {
  tc::Maps m;
  const size_t plane = (size_t)P.nu * P.kpad * 2;
  for (int p = 0; p < 3; ++p) {
    if (!make_map(&m.a[p], (const char *)a_planes + p * plane, P.nu, P.kpad)) return false;
    if (!make_map(&m.b[p], (const char *)b_planes + p * plane, P.nu, P.kpad)) return false;
  }
  static_assert(sizeof(tc::Maps) <= sizeof(P.maps), "map storage");
  memcpy(P.maps, &m, sizeof(m));
  return true;
}

void launch_split_t(long long krows, int nu, long long kpad, const float *src, void *planes, cudaStream_t st) {
  dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((nu + 31) / 32));
  tc::k_split_t<<<grid, dim3(32, 8), 0, st>>>(krows, nu, kpad, src, (__nv_bfloat16 *)planes); ipm_count_launch();
}

void launch_tc_schur(const TcPlan &P, double *partial, int *flags, cudaStream_t st) {
  static const bool attr =
      cudaFuncSetAttribute(tc::k_tc_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES) ==
      cudaSuccess;
  (void)attr;
  tc::Maps m;
  memcpy(&m, P.maps, sizeof(m));
  dim3 grid(P.ntiles, P.ngroups);
  tc::k_tc_schur<<<grid, 192, tc::SMEM_BYTES, st>>>(m, P.nt1, P.kb_total, P.kb_per_group, partial, flags);
  ipm_count_launch();
}

void launch_tc_assemble(const TcPlan &P, int N, const double *partial, const double *Yu, const double *diag,
                        double *Khat, cudaStream_t st) {
  const long long tot = (long long)P.nu * P.nu;
  tc::k_tc_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P.nu, N, P.ngroups, P.ntiles, P.nt1, partial,
                                                                    Yu, diag, Khat);
  ipm_count_launch();
}
