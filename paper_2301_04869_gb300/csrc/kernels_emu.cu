// K6 on the tensor cores at FP64 grade: K_hat = sum_i Z_i^T Y_i with FP64
// operands, computed by BF16 tcgen05 products of exact integer slices.
//
// GB300 runs FP64 at ~1.25 TFLOP/s but BF16 at ~2 PFLOP/s, so the FP64
// contraction is emulated (an Ozaki-type error-free splitting).  For every
// group of 512 contraction rows and every column j, an operand column is
// scaled by a power of two 2^-e (e = ilogb(max |.|) + 2, so |x| 2^-e < 1/2),
// rounded to a multiple of 2^-56 and written as eight 7-bit integer slices,
//     x 2^-e = sum_{t=1..8} q_t 2^-7t + r,   q_t integer, |q_t| <= 64
//     (q_2..q_8 in [-64, 63]),  |r| <= 2^-57,
// each exact in BF16.  A product of slices q_t q'_u is an integer of at most
// 2^12; the pairs with t + u = L + 2 (L = 0..7, 36 pairs in all) accumulate
// in their own FP32 TMEM accumulator ("level" L), whose partial sums over
// 512 rows stay integers of at most 8 * 2^12 * 512 = 2^24 and are therefore
// exact.  The dropped pairs and the remainders weigh about 2^-52 of the
// product of the group's largest entries of the two columns, per row; rows
// are balanced first (row shifts from the rows' largest exponents of Z and
// Y: taken by the multi-RHS solve on the IPM path, by k_emu_rowscale on
// caller data) so that those largest entries belong to the same rows as far
// as a power-of-two row scaling can arrange.  After
// each group the epilogue combines the eight levels into two exact 64-bit
// integers (levels 0-5 and levels 6-7), converts their sum to FP64 (two
// roundings) and accumulates it, scaled by 2^(e_A + e_B - 49), in FP64.
//
// Tiles are 128 (rows of K_hat) x 64 (columns), upper part only; two
// stages of operands, 32 rows of the contraction each (8 x 8 KB + 8 x 4 KB,
// 64-byte rows with the 64-byte swizzle), so the TMA loads of one stage run
// under the MMAs of the other; TMEM holds the eight 64-column level
// accumulators (all 512 columns).  Warp 0 issues the TMA loads, warp 1 the MMAs, warps 2-9
// drain the levels (lane quarter x column half); every wait is bounded as in
// the BF16x3 kernel (kernels_tc.cu).  A non-finite sum raises FLAG_NONFINITE and
// the caller redoes the contraction on the FP64 units.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/ipm.h"
#include "dev.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace emu {

using namespace tcx;

constexpr int NS = 8;                      // slices per operand
constexpr int BM = 128, BN = 64, BK = 32;  // tile; K per stage (64-byte rows, 64-byte swizzle)
constexpr int GROUP = 512;                 // rows per exact level sum
constexpr int KB_PER_GROUP = GROUP / BK;
constexpr int A_PLANE = BM * BK * 2;  // 8 KB
constexpr int B_PLANE = BN * BK * 2;  // 4 KB
constexpr int STAGE_BYTES = NS * (A_PLANE + B_PLANE);  // 96 KB
constexpr int NSTAGE = 2;                               // TMA of one stage under the MMAs of the other
// stages, alignment slack, barriers, and 8 KB of slack after the last
// plane (no descriptor can address past the allocation)
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 + 256 + 8192;

struct Maps {
  CUtensorMap a[NS], b[NS];
};

// ---------------------------------------------------------------------------
// Splitting, in integer arithmetic on the FP64 bit patterns (the FP64 units
// of GB300 are too slow for ~30 operations per element).  Inputs below
// 2^-1022 (subnormal) count as zero.
//
// FP64 bits -> (biased exponent E, 53-bit integer mantissa m), |x| = m 2^(E-1075)
__device__ __forceinline__ void dsplit_bits(double x, int &E, long long &m, bool &neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (b >> 63) != 0;
  E = (int)((b >> 52) & 0x7FF);
  m = (long long)(b & 0xFFFFFFFFFFFFFull) | (1ll << 52);
  if (E == 0) m = 0;  // zero and subnormals
}

// The group-and-column scaled operand as a fixed-point integer:
// X = round-half-away(|x| 2^(56 - e)) with the sign of x, |X| <= 2^55, where
// the balanced biased exponent is E + shift_rows.
__device__ __forceinline__ long long fixed56(int E, long long m, bool neg, int e) {
  if (m == 0) return 0;
  const int sh = E - 1019 - e;  // (E - 1075) + 56 - e
  long long X;
  if (sh >= 0) X = m << sh;     // sh <= 2 because |x| < 2^(e - 1)
  else if (sh <= -63) X = 0;
  else X = (m + (1ll << (-sh - 1))) >> (-sh);
  return neg ? -X : X;
}

// FP64 [krows][nu] -> NS BF16 slice planes [NS][nu][kpad] (K-major) and the
// exponents [kpad / GROUP][nu].  Row k is first scaled by 2^(rsign rs[k])
// (row balancing; rs may be null).  Column exponent of a row group:
// e = ilogb(max |x|) + 2.  Digits of X in base 2^7 with
//   X = sum_t q_t 2^(49 - 7t)  (t = 0..7),  q_t in [-64, 63] for t >= 1,
// the unique such representation: with O = 64 sum_{t>=1} 2^(49 - 7t),
// q_0 = (X + O) >> 49 (|q_0| <= 64) and q_t = bits [s, s+7) of X + O minus
// 64 (s = 49 - 7t), so x 2^-e = sum_t q_t 2^-7(t+1) up to the rounding of X
// (2^-57).  A digit becomes BF16 bits through the FP32 pattern of
// 1.5 2^23 + q (exact for |q| < 2^22; the low 16 bits are zero).
//
// CTA: one row group (512 rows) x 8 columns.  The group is copied into
// shared memory once with asynchronous 8-byte copies (all 32 KB in flight,
// no second read of global memory); the column maxima and the digits are
// taken from there.  Digits of 256 rows at a time go through a staging
// buffer and leave as 512-byte runs of each plane and column (streaming
// stores).  Column blocks are the fast grid index, so the CTAs that share
// the cache lines of the same rows run together.
constexpr long long DIGIT_OFFSET = (64ll << 42) + (64ll << 35) + (64ll << 28) + (64ll << 21) + (64ll << 14) +
                                   (64ll << 7) + 64ll;
constexpr int SPLIT_COLS = 8;                  // columns per CTA
constexpr int SPLIT_SLOTS = 256 / SPLIT_COLS;  // row slots (threads per column)
constexpr int SPLIT_CHUNK = SPLIT_SLOTS * 8;   // rows split per pass (8 per thread)
constexpr int SPLIT_ROW = SPLIT_CHUNK + 8;     // bf16 per (plane, column) row of the staging buffer
constexpr size_t SPLIT_SMEM = (size_t)GROUP * SPLIT_COLS * sizeof(double) + (size_t)NS * SPLIT_COLS * SPLIT_ROW * 2;

__device__ __forceinline__ uint32_t digit_bf16(int q) {
  return __float_as_uint(__int_as_float(0x4B400000 + q) - 12582912.0f) >> 16;
}

// One or two operands per launch (blockIdx.z selects src[z], planes[z],
// exps[z]; the second is the B side, its rows scaled by 2^-rs).
struct SplitOps {
  const double *src[2];
  __nv_bfloat16 *planes[2];
  int *exps[2];
};

__global__ void __launch_bounds__(256, 3) k_emu_split(long long krows, int nu, long long kpad, SplitOps ops,
                                                      const int *__restrict__ rs, int rsign0,
                                                      const int *__restrict__ ezy) {
  const double *__restrict__ src = ops.src[blockIdx.z];
  __nv_bfloat16 *planes = ops.planes[blockIdx.z];
  int *exps = ops.exps[blockIdx.z];
  const int rsign = blockIdx.z == 0 ? rsign0 : -1;
  extern __shared__ __align__(16) uint8_t split_smem[];
  double *tile = reinterpret_cast<double *>(split_smem);  // [GROUP][SPLIT_COLS]
  uint16_t *buf = reinterpret_cast<uint16_t *>(split_smem + (size_t)GROUP * SPLIT_COLS * sizeof(double));
  __shared__ int es[SPLIT_COLS];
  __shared__ int shf[GROUP];
  __shared__ unsigned long long kred[SPLIT_SLOTS][SPLIT_COLS];
  const int j0 = blockIdx.x * SPLIT_COLS;
  const long long g = blockIdx.y, rg = g * GROUP;
  const int tid = threadIdx.x, c = tid % SPLIT_COLS, o = tid / SPLIT_COLS;  // column, row slot
  const int j = j0 + c;
  const bool jv = j < nu;
  // (1) the group into shared memory; row shifts alongside
  for (int r = o; r < GROUP; r += SPLIT_SLOTS) {
    const long long k = rg + r;
    double *d = tile + r * SPLIT_COLS + c;
    if (k < krows && jv) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(d)),
                   "l"(src + k * nu + j));
    } else {
      *d = 0.0;
    }
  }
  // row shifts: given, or from the rows' largest biased exponents of Z
  // (ezy[k]) and Y (ezy[krows + k]) as k_emu_rowscale forms them
  for (int r = tid; r < GROUP; r += 256) {
    const long long k = rg + r;
    int sh = 0;
    if (k < krows) {
      if (rs) {
        sh = rs[k];
      } else if (ezy) {
        const int ez = ezy[k], ey = ezy[krows + k];
        sh = (ez > 0 && ey > 0) ? (ey - ez) / 2 : 0;
      }
    }
    shf[r] = rsign * sh;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // (2) largest balanced magnitude per column: compare (biased exponent,
  // mantissa) as one unsigned key; balanced exponents outside 1..2047 count
  // as zero / clamp
  unsigned long long key = 0;
  for (int r = o; r < GROUP; r += SPLIT_SLOTS) {
    int E;
    long long m;
    bool neg;
    dsplit_bits(tile[r * SPLIT_COLS + c], E, m, neg);
    if (m) {
      E += shf[r];
      if (E > 0) key = max(key, ((unsigned long long)min(E, 2047) << 53) | (unsigned long long)m);
    }
  }
  kred[o][c] = key;
  __syncthreads();
  if (tid < SPLIT_COLS) {
    unsigned long long kk = kred[0][tid];
    for (int q = 1; q < SPLIT_SLOTS; ++q) kk = max(kk, kred[q][tid]);
    const int e = kk > 0 ? (int)(kk >> 53) - 1023 + 2 : 0;
    es[tid] = e;
    if (j0 + tid < nu) exps[g * nu + j0 + tid] = e;
  }
  __syncthreads();
  const int e = es[c];
  const size_t plane = (size_t)nu * kpad;
  const int ncol = min(SPLIT_COLS, nu - j0);
  for (int cb = 0; cb < GROUP; cb += SPLIT_CHUNK) {
    // (3) digits of rows cb + 8 o .. + 7 of column c
    uint32_t w[NS][4];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int rr = cb + o * 8 + r;
      int E;
      long long m;
      bool neg;
      dsplit_bits(tile[rr * SPLIT_COLS + c], E, m, neg);
      const long long X = m ? fixed56(E + shf[rr], m, neg, e) : 0;
      const unsigned long long Y = (unsigned long long)(X + DIGIT_OFFSET);
      const uint32_t lo = (uint32_t)Y, hi = (uint32_t)(Y >> 32);
      uint32_t d[NS];
      d[0] = digit_bf16((int)hi >> 17);
      d[1] = digit_bf16((int)((hi >> 10) & 127) - 64);
      d[2] = digit_bf16((int)((hi >> 3) & 127) - 64);
      d[3] = digit_bf16((int)(__funnelshift_r(lo, hi, 28) & 127) - 64);
      d[4] = digit_bf16((int)((lo >> 21) & 127) - 64);
      d[5] = digit_bf16((int)((lo >> 14) & 127) - 64);
      d[6] = digit_bf16((int)((lo >> 7) & 127) - 64);
      d[7] = digit_bf16((int)(lo & 127) - 64);
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        if (r & 1) w[t][r >> 1] |= d[t] << 16;
        else w[t][r >> 1] = d[t];
      }
    }
#pragma unroll
    for (int t = 0; t < NS; ++t)
      *reinterpret_cast<uint4 *>(buf + (t * SPLIT_COLS + c) * SPLIT_ROW + o * 8) =
          make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    __syncthreads();
    // (4) 16-byte pieces (plane, column, piece of 8 rows), pieces fastest
    for (int p = tid; p < NS * SPLIT_COLS * (SPLIT_CHUNK / 8); p += 256) {
      const int seg = p % (SPLIT_CHUNK / 8), jj = (p / (SPLIT_CHUNK / 8)) % SPLIT_COLS,
                t = p / (SPLIT_CHUNK / 8 * SPLIT_COLS);
      if (jj < ncol) {
        const uint4 v = *reinterpret_cast<const uint4 *>(buf + (t * SPLIT_COLS + jj) * SPLIT_ROW + seg * 8);
        __stcs(reinterpret_cast<uint4 *>(planes + t * plane + (size_t)(j0 + jj) * kpad + rg + cb + seg * 8), v);
      }
    }
    __syncthreads();
  }
}

// Row balancing: Z^T Y = (D Z)^T (D^-1 Y) for any diagonal D; with
// D_kk = 2^a_k, a_k = (ilogb max_j |Y_kj| - ilogb max_j |Z_kj|) / 2 (C
// division), the two operands' rows meet halfway, so a row whose Y is large
// because of a large barrier term no longer sets the scale of the whole row
// group of Y alone.  One warp per row; exponents from the bit patterns.
__global__ void k_emu_rowscale(long long krows, int nu, const double *__restrict__ Z, const double *__restrict__ Y,
                               int *rs) {
  const long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= krows) return;
  int ez = 0, ey = 0;  // largest biased exponents (0: no normal entry)
  for (int j = lane; j < nu; j += 32) {
    ez = max(ez, (int)(((unsigned long long)__double_as_longlong(Z[k * nu + j]) >> 52) & 0x7FF));
    ey = max(ey, (int)(((unsigned long long)__double_as_longlong(Y[k * nu + j]) >> 52) & 0x7FF));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ez = max(ez, __shfl_down_sync(0xffffffffu, ez, o));
    ey = max(ey, __shfl_down_sync(0xffffffffu, ey, o));
  }
  if (lane == 0) rs[k] = (ez > 0 && ey > 0) ? (ey - ez) / 2 : 0;
}

__device__ __forceinline__ void tile_of_index(const int2 *tiles, int t, int &ti, int &tj) {
  const int2 v = tiles[t];
  ti = v.x;
  tj = v.y;
}

// Batched updates C -= A B (MODE 1, 2): the operands are the scenarios' A
// rows and B columns stacked with fixed strides mpa, mpb (multiples of 128)
// per scenario, the contraction is one 64-wide block (KPG = 2: one group),
// and the epilogue subtracts the tile from the scenario's output instead of
// writing a partial tile: MODE 1 a column-major FP64 block (the large-block
// LU's trailing update), MODE 2 a row-major FP32 block (the multi-RHS
// solve's block updates on the mixed path).  Rows m < M and columns n < ncol
// of a scenario are written, at out + s stride + (roff + m) rs + (coff + n) cs.
struct TileOut {
  void *out;
  long long stride;
  long long rs, cs;
  int roff, coff, M, ncol, mpa, mpb, na, nb;
};

template <int KPG, int MODE>
__global__ void __launch_bounds__(320, 1) k_emu_mma(const __grid_constant__ Maps maps, const int2 *tiles,
                                                    int nu, int kb_total, int kb_per_group,
                                                    const int *__restrict__ expA, const int *__restrict__ expB,
                                                    double *partial, int *flags, TileOut lo) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NSTAGE * STAGE_BYTES);  // [NSTAGE]
  uint64_t *empty = full + NSTAGE;                                               // [NSTAGE]
  uint64_t *acc_full = empty + NSTAGE;
  uint64_t *acc_empty = acc_full + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti, tj, lsc = 0;
  if (MODE != 0) {
    const int per = lo.na * lo.nb, r = blockIdx.x % per;
    lsc = blockIdx.x / per;
    ti = lsc * (lo.mpa / BM) + r / lo.nb;
    tj = lsc * (lo.mpb / BN) + r % lo.nb;
  } else {
    tile_of_index(tiles, blockIdx.x, ti, tj);
  }
  const int kb0 = blockIdx.y * kb_per_group;
  const int kb1 = min(kb_total, kb0 + kb_per_group);
  const int nkb = kb1 - kb0;               // a multiple of KPG
  const int ngr = nkb / KPG;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSTAGE; ++q) {
      mbar_init(full + q, 1);
      mbar_init(empty + q, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // TMEM: eight 64-column FP32 level accumulators (all 512 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb; ++i) {
      const int s = i % NSTAGE;
      // stage s is free once the MMAs of load i - NSTAGE have completed
      if (i >= NSTAGE && !mbar_wait(empty + s, ((i - NSTAGE) / NSTAGE) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t *st = smem + s * STAGE_BYTES;
      mbar_expect_tx(full + s, STAGE_BYTES);
      const int kx = (kb0 + i) * BK;
      for (int p = 0; p < NS; ++p) tma_load_2d(st + p * A_PLANE, &maps.a[p], full + s, kx, ti * BM);
      for (int p = 0; p < NS; ++p) tma_load_2d(st + NS * A_PLANE + p * B_PLANE, &maps.b[p], full + s, kx, tj * BN);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % NSTAGE;
      const int d = i / KPG, kbi = i % KPG;
      if (kbi == 0 && d >= 1 && !mbar_wait(acc_empty, (d - 1) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      if (!mbar_wait(full + s, (i / NSTAGE) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // descriptors of the stage's first A and B planes; the others differ
      // only in the start-address field (16-byte units, no carry: the
      // stage lies below 256 KB of shared memory)
      const uint32_t abase = smem_u32(smem + s * STAGE_BYTES), bbase = abase + NS * A_PLANE;
      const uint64_t da0 = sdesc_sw64(abase), db0 = sdesc_sw64(bbase);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
        for (int L = 0; L < NS; ++L) {
#pragma unroll
          for (int t = 0; t <= L; ++t) {
            const int u = L - t;
            const uint32_t acc = (kbi > 0 || kk > 0 || t > 0) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(L * BN), da0 + (uint64_t)((t * A_PLANE + kk * 32) >> 4),
                     db0 + (uint64_t)((u * B_PLANE + kk * 32) >> 4), idesc, acc);
          }
        }
      }
      mma_commit(empty + s);
      if (kbi == KPG - 1) mma_commit(acc_full);
    }
  } else if (warp >= 2) {
    // eight epilogue warps: lane quarter q (the TMEM lanes a warp may read)
    // and column half h of the 64-column tile
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const int gi = ti * BM + row;  // row of K_hat
    constexpr int HC = BN / 2;
    double acc[HC];
#pragma unroll
    for (int c = 0; c < HC; ++c) acc[c] = 0.0;
    bool bad = false;
    for (int d = 0; d < ngr; ++d) {
      if (!mbar_wait(acc_full, d & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long g = (kb0 / KPG) + d;
      const int ea = gi < nu ? expA[g * nu + gi] : 0;
#pragma unroll
      for (int c0 = 0; c0 < HC; c0 += 16) {
        // the group's value in units of 2^(e_A + e_B - 49):
        // V = sum_{L <= 5} acc_L 2^(7 (5 - L)) (an exact integer of at most
        // 2^60) plus W 2^-14, W = acc_6 2^7 + acc_7 (exact)
        long long V[16], W[16];
#pragma unroll
        for (int L = 0; L < NS; ++L) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(L * BN + h * HC + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            // exact: an integer of at most 2^24 in magnitude (a 32-bit
            // conversion; the 64-bit one runs on the FP64 units)
            const long long a = (long long)__float2int_rn(__uint_as_float(v[e]));
            if (L == 0) V[e] = a;
            else if (L <= 5) V[e] = (V[e] << 7) + a;
            else if (L == 6) W[e] = a << 7;
            else W[e] += a;
          }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int gj = tj * BN + h * HC + c0 + e;
          const int eb = gj < nu ? expB[g * nu + gj] : 0;
          // V + W 2^-14 with one rounding of V and one of the sum
          const double t = fma(__ll2double_rn(W[e]), 0x1p-14, __ll2double_rn(V[e]));
          const int x = ea + eb - 49;
          const double sc = (x > -1023 && x < 1024) ? __hiloint2double((x + 1023) << 20, 0) : ldexp(1.0, x);
          acc[c0 + e] = fma(t, sc, acc[c0 + e]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acc_empty)) : "memory");
    }
    if (MODE != 0) {
      // out -= tile on the valid rows and columns
      const int m = ti * BM - lsc * lo.mpa + row, n0 = tj * BN - lsc * lo.mpb + h * HC;
      if (m < lo.M) {
        const size_t rbase = (size_t)lsc * lo.stride + (size_t)(lo.roff + m) * lo.rs;
#pragma unroll
        for (int c = 0; c < HC; ++c)
          if (n0 + c < lo.ncol) {
            bad |= !isfinite(acc[c]);
            const size_t at = rbase + (size_t)(lo.coff + n0 + c) * lo.cs;
            if (MODE == 1) static_cast<double *>(lo.out)[at] -= acc[c];
            else static_cast<float *>(lo.out)[at] -= (float)acc[c];
          }
      }
    } else {
      double *out = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * BM * BN + (size_t)row * BN + h * HC;
#pragma unroll
      for (int c = 0; c < HC; ++c) {
        bad |= !isfinite(acc[c]);
        out[c] = acc[c];
      }
    }
    if (bad) flags[FLAG_NONFINITE] = 1;
  }
  // after an abort, let the loads in flight land before the CTA exits
  if (warp == 0 && lane == 0 && *abort_flag)
    for (int i = max(0, issued - NSTAGE); i < issued; ++i) (void)mbar_wait(full + i % NSTAGE, (i / NSTAGE) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// Slices of the trailing update's operands for one panel [kb, ke) of the
// large-block LU: stacked row r = s Mp + m (m < M = nd - ke) is row m of
// L21 (side 0: L(ke + m, kb + k)) or column m of U12 (side 1:
// U(kb + k, ke + m)), k = 0 .. ke - kb - 1 (at most 64); a warp per row: its
// exponent e = ilogb(max |x|) + 2 and eight 7-bit digits per entry as in
// k_emu_split, planes [NS][N Mp][64] (K-major); rows m >= M are zero.
__global__ void __launch_bounds__(256) k_emu_lu_split(const double *__restrict__ LU, long long nnzlu, int dense_base,
                                                      int nd, int kb, int ke, int Mp, int N,
                                                      __nv_bfloat16 *pa, __nv_bfloat16 *pb, int *ea, int *eb) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, side = blockIdx.y;
  if (r >= (long long)N * Mp) return;
  const int sc = (int)(r / Mp), m = (int)(r - (long long)sc * Mp), M = nd - ke, pbw = ke - kb;
  const double *A = LU + (size_t)sc * nnzlu + dense_base;
  double x[2] = {0.0, 0.0};
  if (m < M)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      if (k < pbw) x[h] = side == 0 ? A[(size_t)(kb + k) * nd + ke + m] : A[(size_t)(ke + m) * nd + kb + k];
    }
  unsigned long long key = 0;
  int E[2];
  long long mt[2];
  bool neg[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    dsplit_bits(x[h], E[h], mt[h], neg[h]);
    if (mt[h]) key = max(key, ((unsigned long long)E[h] << 53) | (unsigned long long)mt[h]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
    key = max(key, ok);
  }
  const int e = key > 0 ? (int)(key >> 53) - 1023 + 2 : 0;
  __nv_bfloat16 *planes = side == 0 ? pa : pb;
  if (lane == 0) (side == 0 ? ea : eb)[r] = e;
  const size_t plane = (size_t)N * Mp * 64;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const long long X = mt[h] ? fixed56(E[h], mt[h], neg[h], e) : 0;
    const unsigned long long Y = (unsigned long long)(X + DIGIT_OFFSET);
    const uint32_t lo = (uint32_t)Y, hi = (uint32_t)(Y >> 32);
    uint32_t d[NS];
    d[0] = digit_bf16((int)hi >> 17);
    d[1] = digit_bf16((int)((hi >> 10) & 127) - 64);
    d[2] = digit_bf16((int)((hi >> 3) & 127) - 64);
    d[3] = digit_bf16((int)(__funnelshift_r(lo, hi, 28) & 127) - 64);
    d[4] = digit_bf16((int)((lo >> 21) & 127) - 64);
    d[5] = digit_bf16((int)((lo >> 14) & 127) - 64);
    d[6] = digit_bf16((int)((lo >> 7) & 127) - 64);
    d[7] = digit_bf16((int)(lo & 127) - 64);
    uint16_t *dst = reinterpret_cast<uint16_t *>(planes) + (size_t)r * 64 + lane + 32 * h;
#pragma unroll
    for (int t = 0; t < NS; ++t) dst[t * plane] = (uint16_t)d[t];
  }
}

// K_hat[i][j] = K_hat[j][i] = sum_g partial + sum_s Yu[s] + diag  (i <= j)
__global__ void k_emu_assemble(int nu, int N, int ngroups, int ntiles, int ntn, const double *__restrict__ partial,
                               const int *__restrict__ tile_of, const double *__restrict__ Yu,
                               const double *__restrict__ diag, double *Khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int i = (int)(t / nu), j = (int)(t % nu);
  if (i > j) return;
  const int ti = i / BM, tj = j / BN;
  const int tt = tile_of[ti * ntn + tj];
  double v = 0.0;
  for (int g = 0; g < ngroups; ++g) v += partial[((size_t)g * ntiles + tt) * BM * BN + (i - ti * BM) * BN + (j - tj * BN)];
  if (Yu)
    for (int s = 0; s < N; ++s) v += Yu[(size_t)s * nu * nu + (size_t)i * nu + j];
  if (diag && i == j) v += diag[i];
  Khat[(size_t)i * nu + j] = v;
  Khat[(size_t)j * nu + i] = v;
}

}  // namespace emu

size_t emu_planes_bytes(int nu, long long krows) {
  const long long kpad = (krows + emu::GROUP - 1) / emu::GROUP * emu::GROUP;
  return (size_t)emu::NS * nu * kpad * 2;
}

bool emu_plan(EmuPlan &P, int nu, long long krows, const void *a_planes, const void *b_planes, int *exp_a,
              int *exp_b, int2 *tiles_dev, int *tile_of_dev) {
  P.nu = nu;
  P.krows = krows;
  P.kpad = (krows + emu::GROUP - 1) / emu::GROUP * emu::GROUP;
  P.kb_total = (int)(P.kpad / emu::BK);
  P.ntm = (nu + emu::BM - 1) / emu::BM;
  P.ntn = (nu + emu::BN - 1) / emu::BN;
  std::vector<int2> tl;
  std::vector<int> tof((size_t)P.ntm * P.ntn, -1);
  for (int a = 0; a < P.ntm; ++a)
    for (int b = 0; b < P.ntn; ++b)
      if (a * emu::BM <= b * emu::BN + emu::BN - 1) {
        tof[(size_t)a * P.ntn + b] = (int)tl.size();
        tl.push_back(make_int2(a, b));
      }
  P.ntiles = (int)tl.size();
  P.tiles = tiles_dev;
  P.tile_of = tile_of_dev;
  if (cudaMemcpy(tiles_dev, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) return false;
  if (cudaMemcpy(tile_of_dev, tof.data(), tof.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  emu_regroup(P, 152 / P.ntiles);
  P.a_planes = a_planes;
  P.b_planes = b_planes;
  P.exp_a = exp_a;
  P.exp_b = exp_b;
  emu::Maps m;
  const size_t plane = (size_t)nu * P.kpad * 2;
  for (int p = 0; p < emu::NS; ++p) {
    if (!tc_make_kmajor_map_box(&m.a[p], (const char *)a_planes + p * plane, nu, P.kpad, emu::BM, emu::BK))
      return false;
    if (!tc_make_kmajor_map_box(&m.b[p], (const char *)b_planes + p * plane, nu, P.kpad, emu::BN, emu::BK))
      return false;
  }
  static_assert(sizeof(emu::Maps) <= sizeof(P.maps), "map storage");
  memcpy(P.maps, &m, sizeof(m));
  return true;
}

void emu_regroup(EmuPlan &P, int G) {
  const int ngr = P.kb_total / emu::KB_PER_GROUP;  // row groups
  if (G < 1) G = 1;
  if (G > ngr) G = ngr;
  const int gpg = (ngr + G - 1) / G;  // row groups per CTA
  P.kb_per_group = gpg * emu::KB_PER_GROUP;
  P.ngroups = (ngr + gpg - 1) / gpg;
}

long long emu_kpad(long long krows) { return (krows + emu::GROUP - 1) / emu::GROUP * emu::GROUP; }

void launch_emu_rowscale(const EmuPlan &P, const double *Z, const double *Y, int *rs, cudaStream_t st) {
  const long long thr = P.krows * 32;
  emu::k_emu_rowscale<<<(unsigned)((thr + 255) / 256), 256, 0, st>>>(P.krows, P.nu, Z, Y, rs);
  ipm_count_launch();
}

static void split_launch(const EmuPlan &P, emu::SplitOps ops, int nz, int rsign0, const int *rs, const int *ezy,
                         cudaStream_t st) {
  static const bool cap = cudaFuncSetAttribute(emu::k_emu_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)emu::SPLIT_SMEM) == cudaSuccess;
  (void)cap;
  dim3 grid((unsigned)((P.nu + emu::SPLIT_COLS - 1) / emu::SPLIT_COLS), (unsigned)(P.kpad / emu::GROUP),
            (unsigned)nz);
  emu::k_emu_split<<<grid, 256, emu::SPLIT_SMEM, st>>>(P.krows, P.nu, P.kpad, ops, rs, rsign0, ezy);
  ipm_count_launch();
}

void launch_emu_split(const EmuPlan &P, const double *src, bool b_side, const int *rs, cudaStream_t st,
                      const int *ezy) {
  emu::SplitOps ops{};
  ops.src[0] = src;
  ops.planes[0] = (__nv_bfloat16 *)(b_side ? P.b_planes : P.a_planes);
  ops.exps[0] = b_side ? P.exp_b : P.exp_a;
  split_launch(P, ops, 1, b_side ? -1 : 1, rs, ezy, st);
}

void launch_emu_split_pair(const EmuPlan &P, const double *Z, const double *Y, const int *rs, cudaStream_t st,
                           const int *ezy) {
  emu::SplitOps ops{};
  ops.src[0] = Z;
  ops.src[1] = Y;
  ops.planes[0] = (__nv_bfloat16 *)P.a_planes;
  ops.planes[1] = (__nv_bfloat16 *)P.b_planes;
  ops.exps[0] = P.exp_a;
  ops.exps[1] = P.exp_b;
  split_launch(P, ops, 2, 1, rs, ezy, st);
}

void launch_emu_schur(const EmuPlan &P, double *partial, int *flags, cudaStream_t st) {
  auto kern = emu::k_emu_mma<emu::KB_PER_GROUP, 0>;
  static const bool attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, emu::SMEM_BYTES) == cudaSuccess;
  (void)attr;
  emu::Maps m;
  memcpy(&m, P.maps, sizeof(m));
  dim3 grid(P.ntiles, P.ngroups);
  kern<<<grid, 320, emu::SMEM_BYTES, st>>>(m, P.tiles, P.nu, P.kb_total, P.kb_per_group, P.exp_a, P.exp_b, partial,
                                           flags, emu::TileOut{});
  ipm_count_launch();
}

void launch_emu_assemble(const EmuPlan &P, int N, const double *partial, const double *Yu, const double *diag,
                         double *Khat, cudaStream_t st) {
  const long long tot = (long long)P.nu * P.nu;
  emu::k_emu_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P.nu, N, P.ngroups, P.ntiles, P.ntn, partial,
                                                                      P.tile_of, Yu, diag, Khat);
  ipm_count_launch();
}

size_t emu_partial_doubles(const EmuPlan &P, int max_groups) {
  return (size_t)max_groups * P.ntiles * emu::BM * emu::BN;
}

// ---------------------------------------------------------------------------
// The failure path of the bounded device waits, exercised without a fault:
// one thread waits on an mbarrier that nothing arrives at, gives up after
// `polls` polls and raises FLAG_TIMEOUT, as every wait of the tcgen05 kernels
// does (they use the same wait with a larger limit).
namespace emu {
__global__ void k_wait_selftest(long long polls, int *flags) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_limit(&bar, 0, polls)) flags[FLAG_TIMEOUT] = 1;
}
}  // namespace emu

extern "C" ipm_status ipm_selftest_bounded_wait(long long polls, void *stream) {
  if (polls < 1 || polls > (1LL << 22)) return IPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int *flags = nullptr;
  int hf[FLAG_COUNT] = {0};
  if (cudaMalloc(&flags, FLAG_COUNT * sizeof(int)) != cudaSuccess) return IPM_ERR_OOM;
  ipm_status rc = IPM_OK;
  if (cudaMemsetAsync(flags, 0, FLAG_COUNT * sizeof(int), st) != cudaSuccess) rc = IPM_ERR_CUDA;
  if (rc == IPM_OK) {
    emu::k_wait_selftest<<<1, 32, 0, st>>>(polls, flags);
    ipm_count_launch();
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = IPM_ERR_CUDA;
    else if (hf[FLAG_TIMEOUT])
      rc = IPM_ERR_TIMEOUT;
  }
  cudaFree(flags);
  return rc;
}

// ---------------------------------------------------------------------------
// Stand-alone entry point (include/ipm.h): the emulated contraction on
// caller-owned device matrices, for checking the kernel on arbitrary data.
extern "C" ipm_status ipm_schur_sum_tc(const double *Z, const double *Y, int n_scen, int n_x, int n_u,
                                       double *Khat, void *stream) {
  if (!Z || !Y || !Khat || n_scen < 1 || n_x < 1 || n_u < 1) return IPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long krows = (long long)n_scen * n_x;
  const size_t pb = emu_planes_bytes(n_u, krows);
  const long long ngr = emu_kpad(krows) / emu::GROUP;
  const long long nt = (long long)((n_u + emu::BM - 1) / emu::BM) * ((n_u + emu::BN - 1) / emu::BN);
  void *pa = nullptr, *pbp = nullptr, *part = nullptr;
  int *ea = nullptr, *eb = nullptr, *tof = nullptr, *flags = nullptr, *rsd = nullptr;
  int2 *tiles = nullptr;
  ipm_status rc = IPM_OK;
  EmuPlan P;
  int hf[FLAG_COUNT] = {0};
  if (cudaMalloc(&pa, pb) != cudaSuccess || cudaMalloc(&pbp, pb) != cudaSuccess ||
      cudaMalloc(&ea, ngr * n_u * sizeof(int)) != cudaSuccess || cudaMalloc(&eb, ngr * n_u * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&tiles, nt * sizeof(int2)) != cudaSuccess || cudaMalloc(&tof, nt * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&flags, FLAG_COUNT * sizeof(int)) != cudaSuccess) {
    rc = IPM_ERR_OOM;
    goto done;
  }
  if (!emu_plan(P, n_u, krows, pa, pbp, ea, eb, tiles, tof)) {
    rc = IPM_ERR_CUDA;
    goto done;
  }
  if (cudaMalloc(&part, emu_partial_doubles(P, P.ngroups) * sizeof(double)) != cudaSuccess) {
    rc = IPM_ERR_OOM;
    goto done;
  }
  if (cudaMalloc(&rsd, krows * sizeof(int)) != cudaSuccess) {
    rc = IPM_ERR_OOM;
    goto done;
  }
  cudaMemsetAsync(flags, 0, FLAG_COUNT * sizeof(int), st);
  launch_emu_rowscale(P, Z, Y, rsd, st);
  launch_emu_split_pair(P, Z, Y, rsd, st);
  launch_emu_schur(P, (double *)part, flags, st);
  launch_emu_assemble(P, n_scen, (const double *)part, nullptr, nullptr, Khat, st);
  if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    rc = IPM_ERR_CUDA;
    goto done;
  }
  if (hf[FLAG_TIMEOUT]) rc = IPM_ERR_TIMEOUT;
  else if (hf[FLAG_NONFINITE]) rc = IPM_ERR_ARG;
done:
  cudaStreamSynchronize(st);
  for (void *p : {pa, pbp, part, (void *)ea, (void *)eb, (void *)tof, (void *)flags, (void *)tiles, (void *)rsd})
    if (p) cudaFree(p);
  return rc;
}

// ---------------------------------------------------------------------------
// The trailing update A22 -= L21 U12 of the large-block LU at FP64 grade on
// the tensor cores (the emulated product above with one 64-row group).
bool emu_lu_plan(EmuLuPlan &P, int N, int nd, void *a_planes, void *b_planes, int *exp_a, int *exp_b) {
  P.N = N;
  P.nd = nd;
  P.Mp = (nd + emu::BM - 1) / emu::BM * emu::BM;
  P.a_planes = a_planes;
  P.b_planes = b_planes;
  P.exp_a = exp_a;
  P.exp_b = exp_b;
  const long long rows = (long long)N * P.Mp;
  if (rows > 0x7fffffffLL) return false;
  emu::Maps m;
  const size_t plane = (size_t)rows * 64 * 2;
  for (int p = 0; p < emu::NS; ++p) {
    if (!tc_make_kmajor_map_box(&m.a[p], (const char *)a_planes + p * plane, (int)rows, 64, emu::BM, emu::BK))
      return false;
    if (!tc_make_kmajor_map_box(&m.b[p], (const char *)b_planes + p * plane, (int)rows, 64, emu::BN, emu::BK))
      return false;
  }
  static_assert(sizeof(emu::Maps) <= sizeof(P.maps), "map storage");
  memcpy(P.maps, &m, sizeof(m));
  return true;
}

size_t emu_lu_planes_bytes(int N, int nd) {
  const long long Mp = (nd + emu::BM - 1) / emu::BM * emu::BM;
  return (size_t)emu::NS * N * Mp * 64 * 2;
}

void launch_emu_lu_update(const EmuLuPlan &P, double *LU, long long nnzlu, int dense_base, int kb, int ke, int *flags,
                          cudaStream_t st) {
  const int M = P.nd - ke;
  if (M <= 0) return;
  const long long rows = (long long)P.N * P.Mp;
  emu::k_emu_lu_split<<<dim3((unsigned)((rows * 32 + 255) / 256), 2), 256, 0, st>>>(
      LU, nnzlu, dense_base, P.nd, kb, ke, P.Mp, P.N, (__nv_bfloat16 *)P.a_planes, (__nv_bfloat16 *)P.b_planes,
      P.exp_a, P.exp_b);
  ipm_count_launch();
  auto kern = emu::k_emu_mma<2, 1>;
  static const bool attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, emu::SMEM_BYTES) == cudaSuccess;
  (void)attr;
  emu::Maps m;
  memcpy(&m, P.maps, sizeof(m));
  // C = the dense block, column-major: (ke + m, ke + n) at dense_base + (ke + n) nd + ke + m
  emu::TileOut lo{LU + dense_base, nnzlu, 1, P.nd, ke, ke, M, M, P.Mp, P.Mp,
                  (M + emu::BM - 1) / emu::BM, (M + emu::BN - 1) / emu::BN};
  const long long grid = (long long)P.N * lo.na * lo.nb;
  kern<<<dim3((unsigned)grid, 1), 320, emu::SMEM_BYTES, st>>>(m, nullptr, (int)rows, 2, 2, P.exp_a, P.exp_b, nullptr,
                                                             flags, lo);
  ipm_count_launch();
}
