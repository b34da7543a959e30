// Learned warm start: a small MLP  x -> Linear -> GELU -> Linear -> GELU ->
// Linear  that maps a scenario's load vector to a primal point and log bound
// duals.  Training and inference run in this file's kernels: BF16 operands on
// the 5th-generation tensor cores (tcgen05.mma, TMEM accumulator, TMA-staged
// 128-byte-swizzled tiles), FP32 accumulation and epilogues, FP32 master
// weights with Adam.  The paper has no learned component.
//
// Every product is C[M][N] = A[M][K] B[N][K]^T with both operands K-major, so
// each weight matrix is kept in BF16 both as W [out][in] (forward) and as
// W^T [in][out] (backward through the layer), and the epilogues write the
// activations both row-major and transposed (the transposed copies are the
// K-major operands of the weight-gradient products, K = batch).  Sizes are
// padded: input and output widths to multiples of 128 (zero weights and
// targets in the padding), batches to multiples of 128 (padded rows carry
// zero loss gradients, so they add nothing to the weight gradients).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/ipm.h"
#include "dev.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mlpk {

using namespace tcx;

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KB per operand tile
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

enum { ACT_NONE = 0, ACT_GELU = 1, ACT_GELU_BWD = 2 };

struct Epi {
  const float *bias;      // [N] or null
  const float *pre_in;    // [M][ldo]: pre-activation for ACT_GELU_BWD
  float *pre_out;         // [M][ldo] or null: pre-activation (ACT_GELU)
  float *out_f32;         // [M][ldo] or null
  __nv_bfloat16 *out_bf;  // [M][ldo] or null
  __nv_bfloat16 *out_t;   // [N][ldt] or null (transposed)
  const float *scale;     // [N] or null: out_f32 = shift + scale * v
  const float *shift;
  int ldo, ldt, act, n_valid;  // columns >= n_valid of out_f32 are written as 0 when scaled
};

// GELU with the Gauss error function, and its derivative
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void __launch_bounds__(192, 1) k_gemm(const __grid_constant__ CUtensorMap ma,
                                                 const __grid_constant__ CUtensorMap mb, int kblocks, Epi e,
                                                 int *flags) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *accf = empty + STAGES;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // TMEM: one 128-column FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  int issued = 0;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t *st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(st, &ma, &full[s], kb * BK, m0);
      tma_load_2d(st + TILE_BYTES, &mb, &full[s], kb * BK, n0);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
        flags[FLAG_TIMEOUT] = 1;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        mma_bf16(tmem, sdesc(base + kk * 32), sdesc(base + TILE_BYTES + kk * 32), idesc,
                 (kb > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(accf);
  } else if (warp >= 2) {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    const int m = m0 + row;
    const bool ok = mbar_wait(accf, 0);
    if (!ok) {
      flags[FLAG_TIMEOUT] = 1;
      *abort_flag = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const size_t ro = (size_t)m * e.ldo + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          float a = __uint_as_float(v[j]);
          if (e.bias) a += e.bias[n];
          float o = a;
          if (e.act == ACT_GELU) {
            if (e.pre_out) e.pre_out[ro + j] = a;
            o = gelu(a);
          } else if (e.act == ACT_GELU_BWD) {
            o = a * gelu_d(e.pre_in[ro + j]);
          }
          if (e.out_f32) {
            float w = o;
            if (e.scale) w = n < e.n_valid ? e.shift[n] + e.scale[n] * o : 0.0f;
            e.out_f32[ro + j] = w;
          }
          const __nv_bfloat16 b = __float2bfloat16_rn(o);
          if (e.out_bf) e.out_bf[ro + j] = b;
          if (e.out_t) e.out_t[(size_t)n * e.ldt + m] = b;
        }
      }
    }
  }
  if (warp == 0 && lane == 0 && *abort_flag) {
    // let the copies already issued land before the CTA exits (bounded)
    for (int kb = max(0, issued - STAGES); kb < issued; ++kb) (void)mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  }
}

// X (FP32 [B][din]) -> normalised BF16 rows [Mb][dinp] and columns [dinp][ldt]
// (zero in the padding: rows >= B, columns >= din)
__global__ void k_input(int B, int Mb, int din, int dinp, int ldt, const float *__restrict__ X,
                        const float *__restrict__ mean, const float *__restrict__ stdv, __nv_bfloat16 *Xb,
                        __nv_bfloat16 *XT) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float v = 0.0f;
    if (row < B && col < din) v = (X[(size_t)row * din + col] - mean[col]) / stdv[col];
    if (row < Mb && col < dinp) Xb[(size_t)row * dinp + col] = __float2bfloat16_rn(v);
    t[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int col = c0 + r, row = r0 + tx;
    if (col < dinp && row < Mb) XT[(size_t)col * ldt + row] = __float2bfloat16_rn(t[tx][r]);
  }
}

// mean squared error on normalised targets (padding excluded):
//   L = (1 / (B dout)) sum (y - tn)^2,  dL/dy = 2 (y - tn) / (B dout)
// dY written FP32 and BF16 row-major [Mb][doutp] and BF16 transposed
// [doutp][ldt]; per-block partial sums of the squared error in part[].
__global__ void k_loss(int B, int Mb, int dout, int doutp, int ldt, const float *__restrict__ Y,
                       const float *__restrict__ T, const float *__restrict__ mean, const float *__restrict__ stdv,
                       float *dYf, __nv_bfloat16 *dYb, __nv_bfloat16 *dYT, double *part) {
  __shared__ float t[32][33];
  __shared__ double red[8];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float sc = 2.0f / ((float)B * (float)dout);
  double se = 0.0;
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float g = 0.0f;
    if (row < B && col < dout) {
      const float d = Y[(size_t)row * doutp + col] - (T[(size_t)row * dout + col] - mean[col]) / stdv[col];
      se += (double)d * d;
      g = sc * d;
    }
    if (row < Mb && col < doutp) {
      dYf[(size_t)row * doutp + col] = g;
      dYb[(size_t)row * doutp + col] = __float2bfloat16_rn(g);
    }
    t[r][tx] = g;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int col = c0 + r, row = r0 + tx;
    if (col < doutp && row < Mb) dYT[(size_t)col * ldt + row] = __float2bfloat16_rn(t[tx][r]);
  }
  se = warp_sum(se);
  if (tx == 0) red[ty] = se;
  __syncthreads();
  if (tx == 0 && ty == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_sum(int n, const double *part, double *out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    out[0] = r;
  }
}

// bias gradients: g[n] = sum_{b < B} d[b][n]  (fixed order over b)
__global__ void k_colsum(int B, int N, int ld, const float *__restrict__ d, float *g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int b = 0; b < B; ++b) s += d[(size_t)b * ld + n];
  g[n] = s;
}

// Adam (Kingma & Ba) on the FP32 masters, then the BF16 copies
__global__ void k_adam(long long n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// W [rows][cols] FP32 -> BF16 W and (optionally) BF16 W^T [cols][rows]
__global__ void k_to_bf16(int rows, int cols, const float *__restrict__ W, __nv_bfloat16 *Wb, __nv_bfloat16 *WT) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float v = 0.0f;
    if (row < rows && col < cols) {
      v = W[(size_t)row * cols + col];
      Wb[(size_t)row * cols + col] = __float2bfloat16_rn(v);
    }
    t[r][tx] = v;
  }
  if (!WT) return;
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int col = c0 + r, row = r0 + tx;
    if (col < cols && row < rows) WT[(size_t)col * rows + row] = __float2bfloat16_rn(t[tx][r]);
  }
}

}  // namespace mlpk

using namespace mlpk;

struct ipm_mlp {
  int din = 0, dh = 0, dout = 0, maxb = 0;
  int dinp = 0, doutp = 0, bpad = 0;
  long long np = 0;                // padded parameter count
  long long oW1, ob1, oW2, ob2, oW3, ob3;  // offsets in the padded parameter vector
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *V = nullptr;
  __nv_bfloat16 *W1b, *W2b, *W2T, *W3b, *W3T;
  __nv_bfloat16 *Xb, *XT, *H1b, *H1T, *H2b, *H2T, *dYb, *dYT, *dp2b, *dp2T, *dp1T;
  float *pre1, *pre2, *Y, *dYf, *dp2f, *dp1f;
  float *in_mean, *in_std, *out_mean, *out_std;
  double *part = nullptr, *lsum = nullptr, *h_loss = nullptr;
  int *flags = nullptr, *h_flags = nullptr;
  long long adam_t = 0;
  CUtensorMap maps[16];
  std::vector<void *> allocs;
};

namespace {

enum { MX, MW1, MH1, MW2, MH2, MW3, MDY, MW3T, MDYT, MH2T, MDP2, MW2T, MDP2T, MH1T, MDP1T, MXT };

template <class T>
bool mal(ipm_mlp *m, T **p, size_t count) {
  void *q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
  m->allocs.push_back(q);
  *p = (T *)q;
  return true;
}

inline int r128(int v) { return (v + 127) / 128 * 128; }

void gemm(ipm_mlp *m, int mapA, int mapB, int M, int N, int K, const Epi &e, cudaStream_t st) {
  static const bool attr = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                SMEM_BYTES) == cudaSuccess;
  (void)attr;
  dim3 grid(M / BM, N / BN);
  k_gemm<<<grid, 192, SMEM_BYTES, st>>>(m->maps[mapA], m->maps[mapB], K / BK, e, m->flags);
  ipm_count_launch();
}

Epi epi(int ldo) {
  Epi e;
  std::memset(&e, 0, sizeof(e));
  e.ldo = ldo;
  return e;
}

void refresh_bf16(ipm_mlp *m, cudaStream_t st) {
  const dim3 b(32, 8);
  k_to_bf16<<<dim3((m->dinp + 31) / 32, (m->dh + 31) / 32), b, 0, st>>>(m->dh, m->dinp, m->P + m->oW1, m->W1b, nullptr);
  k_to_bf16<<<dim3((m->dh + 31) / 32, (m->dh + 31) / 32), b, 0, st>>>(m->dh, m->dh, m->P + m->oW2, m->W2b, m->W2T);
  k_to_bf16<<<dim3((m->dh + 31) / 32, (m->doutp + 31) / 32), b, 0, st>>>(m->doutp, m->dh, m->P + m->oW3, m->W3b,
                                                                         m->W3T);
  ipm_count_launch();
  ipm_count_launch();
  ipm_count_launch();
}

// forward pass over B rows of X; the output layer writes de-normalised
// predictions when `denorm`, normalised ones otherwise (training)
void forward(ipm_mlp *m, const float *X, int B, bool denorm, float *Yout, int ldy, cudaStream_t st) {
  const int Mb = r128(B);
  k_input<<<dim3((m->dinp + 31) / 32, (Mb + 31) / 32), dim3(32, 8), 0, st>>>(B, Mb, m->din, m->dinp, m->bpad, X,
                                                                           m->in_mean, m->in_std, m->Xb, m->XT);
  ipm_count_launch();
  Epi e = epi(m->dh);
  e.bias = m->P + m->ob1;
  e.act = ACT_GELU;
  e.pre_out = m->pre1;
  e.out_bf = m->H1b;
  e.out_t = m->H1T;
  e.ldt = m->bpad;
  gemm(m, MX, MW1, Mb, m->dh, m->dinp, e, st);
  e.bias = m->P + m->ob2;
  e.pre_out = m->pre2;
  e.out_bf = m->H2b;
  e.out_t = m->H2T;
  gemm(m, MH1, MW2, Mb, m->dh, m->dh, e, st);
  Epi o = epi(ldy);
  o.bias = m->P + m->ob3;
  o.act = ACT_NONE;
  o.out_f32 = Yout;
  if (denorm) {
    o.scale = m->out_std;
    o.shift = m->out_mean;
    o.n_valid = m->dout;
  }
  gemm(m, MH2, MW3, Mb, m->doutp, m->dh, o, st);
}

// loss and gradients (into m->G) for B rows
void backward(ipm_mlp *m, const float *T, int B, cudaStream_t st) {
  const int Mb = r128(B);
  const dim3 lg((m->doutp + 31) / 32, (Mb + 31) / 32);
  k_loss<<<lg, dim3(32, 8), 0, st>>>(B, Mb, m->dout, m->doutp, m->bpad, m->Y, T, m->out_mean, m->out_std, m->dYf,
                                     m->dYb, m->dYT, m->part);
  ipm_count_launch();
  k_sum<<<1, 256, 0, st>>>((int)(lg.x * lg.y), m->part, m->lsum);
  ipm_count_launch();
  // dpre2 = (dY W3) * GELU'(pre2)
  Epi e = epi(m->dh);
  e.act = ACT_GELU_BWD;
  e.pre_in = m->pre2;
  e.out_f32 = m->dp2f;
  e.out_bf = m->dp2b;
  e.out_t = m->dp2T;
  e.ldt = m->bpad;
  gemm(m, MDY, MW3T, Mb, m->dh, m->doutp, e, st);
  // dW3 = dY^T H2
  Epi w = epi(m->dh);
  w.out_f32 = m->G + m->oW3;
  gemm(m, MDYT, MH2T, m->doutp, m->dh, Mb, w, st);
  // dpre1 = (dpre2 W2) * GELU'(pre1)
  Epi e1 = epi(m->dh);
  e1.act = ACT_GELU_BWD;
  e1.pre_in = m->pre1;
  e1.out_f32 = m->dp1f;
  e1.out_t = m->dp1T;
  e1.ldt = m->bpad;
  gemm(m, MDP2, MW2T, Mb, m->dh, m->dh, e1, st);
  // dW2 = dpre2^T H1, dW1 = dpre1^T X
  w.out_f32 = m->G + m->oW2;
  gemm(m, MDP2T, MH1T, m->dh, m->dh, Mb, w, st);
  Epi w1 = epi(m->dinp);
  w1.out_f32 = m->G + m->oW1;
  gemm(m, MDP1T, MXT, m->dh, m->dinp, Mb, w1, st);
  k_colsum<<<(m->dh + 127) / 128, 128, 0, st>>>(B, m->dh, m->dh, m->dp1f, m->G + m->ob1);
  k_colsum<<<(m->dh + 127) / 128, 128, 0, st>>>(B, m->dh, m->dh, m->dp2f, m->G + m->ob2);
  k_colsum<<<(m->doutp + 127) / 128, 128, 0, st>>>(B, m->doutp, m->doutp, m->dYf, m->G + m->ob3);
  ipm_count_launch();
  ipm_count_launch();
  ipm_count_launch();
}

ipm_status finish(ipm_mlp *m, cudaStream_t st, float *loss, int B) {
  if (cudaGetLastError() != cudaSuccess) return IPM_ERR_CUDA;
  if (cudaMemcpyAsync(m->h_flags, m->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return IPM_ERR_CUDA;
  if (loss && cudaMemcpyAsync(m->h_loss, m->lsum, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return IPM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return IPM_ERR_CUDA;
  if (m->h_flags[FLAG_TIMEOUT]) return IPM_ERR_TIMEOUT;
  if (loss) *loss = (float)(*m->h_loss / ((double)B * m->dout));
  return IPM_OK;
}

// logical (unpadded) parameter layout: W1 [dh][din], b1, W2 [dh][dh], b2, W3 [dout][dh], b3
long long logical_count(const ipm_mlp *m) {
  return (long long)m->dh * m->din + m->dh + (long long)m->dh * m->dh + m->dh + (long long)m->dout * m->dh + m->dout;
}

void pack(const ipm_mlp *m, const float *lg, std::vector<float> &pd) {
  pd.assign(m->np, 0.0f);
  const float *s = lg;
  for (int o = 0; o < m->dh; ++o)
    for (int i = 0; i < m->din; ++i) pd[m->oW1 + (long long)o * m->dinp + i] = *s++;
  for (int o = 0; o < m->dh; ++o) pd[m->ob1 + o] = *s++;
  for (int o = 0; o < m->dh; ++o)
    for (int i = 0; i < m->dh; ++i) pd[m->oW2 + (long long)o * m->dh + i] = *s++;
  for (int o = 0; o < m->dh; ++o) pd[m->ob2 + o] = *s++;
  for (int o = 0; o < m->dout; ++o)
    for (int i = 0; i < m->dh; ++i) pd[m->oW3 + (long long)o * m->dh + i] = *s++;
  for (int o = 0; o < m->dout; ++o) pd[m->ob3 + o] = *s++;
}

void unpack(const ipm_mlp *m, const std::vector<float> &pd, float *lg) {
  float *s = lg;
  for (int o = 0; o < m->dh; ++o)
    for (int i = 0; i < m->din; ++i) *s++ = pd[m->oW1 + (long long)o * m->dinp + i];
  for (int o = 0; o < m->dh; ++o) *s++ = pd[m->ob1 + o];
  for (int o = 0; o < m->dh; ++o)
    for (int i = 0; i < m->dh; ++i) *s++ = pd[m->oW2 + (long long)o * m->dh + i];
  for (int o = 0; o < m->dh; ++o) *s++ = pd[m->ob2 + o];
  for (int o = 0; o < m->dout; ++o)
    for (int i = 0; i < m->dh; ++i) *s++ = pd[m->oW3 + (long long)o * m->dh + i];
  for (int o = 0; o < m->dout; ++o) *s++ = pd[m->ob3 + o];
}

}  // namespace

extern "C" {

ipm_status ipm_mlp_create(int d_in, int d_hidden, int d_out, int max_batch, unsigned long long seed,
                          ipm_mlp **out) {
  if (!out) return IPM_ERR_ARG;
  *out = nullptr;
  if (d_in < 1 || d_out < 1 || d_hidden < 128 || d_hidden % 128 != 0 || max_batch < 1 || d_in > (1 << 20) ||
      d_out > (1 << 20) || max_batch > (1 << 20))
    return IPM_ERR_ARG;
  ipm_mlp *m = new ipm_mlp();
  m->din = d_in;
  m->dh = d_hidden;
  m->dout = d_out;
  m->maxb = max_batch;
  m->dinp = r128(d_in);
  m->doutp = r128(d_out);
  m->bpad = r128(max_batch);
  long long o = 0;
  m->oW1 = o; o += (long long)m->dh * m->dinp;
  m->ob1 = o; o += m->dh;
  m->oW2 = o; o += (long long)m->dh * m->dh;
  m->ob2 = o; o += m->dh;
  m->oW3 = o; o += (long long)m->doutp * m->dh;
  m->ob3 = o; o += m->doutp;
  m->np = o;
  const size_t B = m->bpad, H = m->dh;
  bool ok = mal(m, &m->P, m->np) && mal(m, &m->G, m->np) && mal(m, &m->Mm, m->np) && mal(m, &m->V, m->np) &&
            mal(m, &m->W1b, H * m->dinp) && mal(m, &m->W2b, H * H) && mal(m, &m->W2T, H * H) &&
            mal(m, &m->W3b, (size_t)m->doutp * H) && mal(m, &m->W3T, (size_t)m->doutp * H) &&
            mal(m, &m->Xb, B * m->dinp) && mal(m, &m->XT, B * m->dinp) && mal(m, &m->H1b, B * H) &&
            mal(m, &m->H1T, B * H) && mal(m, &m->H2b, B * H) && mal(m, &m->H2T, B * H) &&
            mal(m, &m->dYb, B * m->doutp) && mal(m, &m->dYT, B * m->doutp) && mal(m, &m->dp2b, B * H) &&
            mal(m, &m->dp2T, B * H) && mal(m, &m->dp1T, B * H) && mal(m, &m->pre1, B * H) &&
            mal(m, &m->pre2, B * H) && mal(m, &m->Y, B * m->doutp) && mal(m, &m->dYf, B * m->doutp) &&
            mal(m, &m->dp2f, B * H) && mal(m, &m->dp1f, B * H) && mal(m, &m->in_mean, m->din) &&
            mal(m, &m->in_std, m->din) && mal(m, &m->out_mean, m->dout) && mal(m, &m->out_std, m->dout) &&
            mal(m, &m->part, (B / 32 + 1) * (m->doutp / 32 + 1)) && mal(m, &m->lsum, 1) &&
            mal(m, &m->flags, FLAG_COUNT);
  ok = ok && cudaMallocHost(&m->h_loss, sizeof(double)) == cudaSuccess &&
       cudaMallocHost(&m->h_flags, FLAG_COUNT * sizeof(int)) == cudaSuccess;
  struct MapDef {
    const void *p;
    int rows;
    long long k;
  } defs[16] = {
      {m->Xb, m->bpad, m->dinp},   {m->W1b, m->dh, m->dinp},  {m->H1b, m->bpad, m->dh},
      {m->W2b, m->dh, m->dh},      {m->H2b, m->bpad, m->dh},  {m->W3b, m->doutp, m->dh},
      {m->dYb, m->bpad, m->doutp}, {m->W3T, m->dh, m->doutp}, {m->dYT, m->doutp, m->bpad},
      {m->H2T, m->dh, m->bpad},    {m->dp2b, m->bpad, m->dh}, {m->W2T, m->dh, m->dh},
      {m->dp2T, m->dh, m->bpad},   {m->H1T, m->dh, m->bpad},  {m->dp1T, m->dh, m->bpad},
      {m->XT, m->dinp, m->bpad}};
  for (int i = 0; ok && i < 16; ++i) ok = tc_make_kmajor_map(&m->maps[i], defs[i].p, defs[i].rows, defs[i].k);
  if (!ok) {
    ipm_mlp_destroy(m);
    return IPM_ERR_OOM;
  }
  // He-uniform initial weights (a = sqrt(6 / fan_in)), zero biases, unit normalisation
  std::mt19937_64 rng(seed);
  std::vector<float> lg(logical_count(m), 0.0f);
  {
    float *s = lg.data();
    auto fill = [&](long long n, int fan_in) {
      std::uniform_real_distribution<float> U(-std::sqrt(6.0f / fan_in), std::sqrt(6.0f / fan_in));
      for (long long i = 0; i < n; ++i) *s++ = U(rng);
    };
    fill((long long)m->dh * m->din, m->din);
    s += m->dh;
    fill((long long)m->dh * m->dh, m->dh);
    s += m->dh;
    fill((long long)m->dout * m->dh, m->dh);
  }
  if (ipm_mlp_set_params(m, lg.data()) != IPM_OK) {
    ipm_mlp_destroy(m);
    return IPM_ERR_CUDA;
  }
  std::vector<float> zeros(std::max(m->din, m->dout), 0.0f), ones(std::max(m->din, m->dout), 1.0f);
  if (ipm_mlp_set_normalization(m, zeros.data(), ones.data(), zeros.data(), ones.data()) != IPM_OK) {
    ipm_mlp_destroy(m);
    return IPM_ERR_CUDA;
  }
  *out = m;
  return IPM_OK;
}

ipm_status ipm_mlp_destroy(ipm_mlp *m) {
  if (!m) return IPM_ERR_ARG;
  cudaDeviceSynchronize();
  for (void *p : m->allocs) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  if (m->h_flags) cudaFreeHost(m->h_flags);
  delete m;
  return IPM_OK;
}

long long ipm_mlp_param_count(const ipm_mlp *m) { return m ? logical_count(m) : -1; }

ipm_status ipm_mlp_set_params(ipm_mlp *m, const float *params) {
  if (!m || !params) return IPM_ERR_ARG;
  for (long long i = 0; i < logical_count(m); ++i)
    if (!std::isfinite(params[i])) return IPM_ERR_ARG;
  std::vector<float> pd;
  pack(m, params, pd);
  if (cudaMemcpy(m->P, pd.data(), m->np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return IPM_ERR_CUDA;
  cudaMemset(m->Mm, 0, m->np * sizeof(float));
  cudaMemset(m->V, 0, m->np * sizeof(float));
  m->adam_t = 0;
  refresh_bf16(m, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? IPM_OK : IPM_ERR_CUDA;
}

ipm_status ipm_mlp_get_params(ipm_mlp *m, float *params) {
  if (!m || !params) return IPM_ERR_ARG;
  std::vector<float> pd(m->np);
  if (cudaMemcpy(pd.data(), m->P, m->np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return IPM_ERR_CUDA;
  unpack(m, pd, params);
  return IPM_OK;
}

ipm_status ipm_mlp_set_normalization(ipm_mlp *m, const float *in_mean, const float *in_std, const float *out_mean,
                                     const float *out_std) {
  if (!m || !in_mean || !in_std || !out_mean || !out_std) return IPM_ERR_ARG;
  for (int i = 0; i < m->din; ++i)
    if (!std::isfinite(in_mean[i]) || !(in_std[i] > 0) || !std::isfinite(in_std[i])) return IPM_ERR_ARG;
  for (int i = 0; i < m->dout; ++i)
    if (!std::isfinite(out_mean[i]) || !(out_std[i] > 0) || !std::isfinite(out_std[i])) return IPM_ERR_ARG;
  if (cudaMemcpy(m->in_mean, in_mean, m->din * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->in_std, in_std, m->din * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->out_mean, out_mean, m->dout * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->out_std, out_std, m->dout * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return IPM_ERR_CUDA;
  return IPM_OK;
}

ipm_status ipm_mlp_forward(ipm_mlp *m, const float *x, int batch, float *y, void *stream) {
  if (!m || !x || !y || batch < 1) return IPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  for (int b0 = 0; b0 < batch; b0 += m->maxb) {
    const int B = std::min(m->maxb, batch - b0);
    cudaMemsetAsync(m->flags, 0, FLAG_COUNT * sizeof(int), st);
    forward(m, x + (size_t)b0 * m->din, B, true, m->Y, m->doutp, st);
    if (cudaMemcpy2DAsync(y + (size_t)b0 * m->dout, m->dout * sizeof(float), m->Y, m->doutp * sizeof(float),
                          m->dout * sizeof(float), B, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return IPM_ERR_CUDA;
    ipm_status s = finish(m, st, nullptr, B);
    if (s != IPM_OK) return s;
  }
  return IPM_OK;
}

ipm_status ipm_mlp_gradients(ipm_mlp *m, const float *x, const float *target, int batch, float *grads, float *loss,
                             void *stream) {
  if (!m || !x || !target || batch < 1 || batch > m->maxb) return IPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(m->flags, 0, FLAG_COUNT * sizeof(int), st);
  forward(m, x, batch, false, m->Y, m->doutp, st);
  backward(m, target, batch, st);
  ipm_status s = finish(m, st, loss, batch);
  if (s != IPM_OK || !grads) return s;
  std::vector<float> pd(m->np);
  if (cudaMemcpy(pd.data(), m->G, m->np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return IPM_ERR_CUDA;
  unpack(m, pd, grads);
  return IPM_OK;
}

ipm_status ipm_mlp_train_step(ipm_mlp *m, const float *x, const float *target, int batch, float lr, float *loss,
                              void *stream) {
  if (!m || !x || !target || batch < 1 || batch > m->maxb || !(lr > 0) || !std::isfinite(lr)) return IPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(m->flags, 0, FLAG_COUNT * sizeof(int), st);
  forward(m, x, batch, false, m->Y, m->doutp, st);
  backward(m, target, batch, st);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++m->adam_t;
  const float c1 = 1.0f - std::pow(b1, (float)m->adam_t), c2 = 1.0f - std::pow(b2, (float)m->adam_t);
  k_adam<<<(unsigned)((m->np + 255) / 256), 256, 0, st>>>(m->np, m->P, m->G, m->Mm, m->V, lr, b1, b2, eps, c1, c2);
  ipm_count_launch();
  refresh_bf16(m, st);
  return finish(m, st, loss, batch);
}

}  // extern "C"
