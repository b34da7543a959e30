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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "dev.cuh"
#include "kernels.h"

extern long long g_ipm_launches;

namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;              // tile; BK bf16 = one 128-byte swizzle row
constexpr int STAGES = 2;
constexpr int PLANE_BYTES = BM * BK * 2;                 // 16 KB per operand plane per stage
constexpr int STAGE_BYTES = 6 * PLANE_BYTES;             // 3 A planes + 3 B planes
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;  // + barriers, TMEM slot
constexpr long long WAIT_LIMIT = 1LL << 22;              // bounded spin (well under a second)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bounded wait on phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                      // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;            // SBO
  d |= (uint64_t)1 << 46;                      // version
  d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
  return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4)            // D = F32
         | (1u << 7)          // A = BF16
         | (1u << 10)         // B = BF16
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

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
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// tensor map of one BF16 plane [rows][kpad], box 64 (K) x 128 (rows), 128-byte swizzle
static bool make_map(CUtensorMap *m, const void *base, int rows, long long kpad) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {tc::BK, tc::BM};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void tc_plan(int nu, long long krows, TcPlan &P) {
  P.nu = nu;
  P.kpad = (krows + tc::BK - 1) / tc::BK * tc::BK;
  P.nt1 = (nu + tc::BM - 1) / tc::BM;
  P.ntiles = P.nt1 * (P.nt1 + 1) / 2;
  P.kb_total = (int)(P.kpad / tc::BK);
  int G = 152 / P.ntiles;  // one CTA per SM (the stage buffers take ~193 KB of shared memory)
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
  tc::k_split_t<<<grid, dim3(32, 8), 0, st>>>(krows, nu, kpad, src, (__nv_bfloat16 *)planes); ++g_ipm_launches;
}

void launch_tc_schur(const TcPlan &P, double *partial, int *flags, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_tc_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    attr = true;
  }
  tc::Maps m;
  memcpy(&m, P.maps, sizeof(m));
  dim3 grid(P.ntiles, P.ngroups);
  tc::k_tc_schur<<<grid, 192, tc::SMEM_BYTES, st>>>(m, P.nt1, P.kb_total, P.kb_per_group, partial, flags);
  ++g_ipm_launches;
}

void launch_tc_assemble(const TcPlan &P, int N, const double *partial, const double *Yu, const double *diag,
                        double *Khat, cudaStream_t st) {
  const long long tot = (long long)P.nu * P.nu;
  tc::k_tc_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P.nu, N, P.ngroups, P.ntiles, P.nt1, partial,
                                                                    Yu, diag, Khat);
  ++g_ipm_launches;
}
