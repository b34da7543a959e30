// Allocation-free variant of the scenario-summed reduced-Hessian product.
//
// Some callers cannot call cudaMalloc: code that runs while an external
// memory pool owns the whole device, plug-ins that are only handed device
// buffers by their host application, or processes whose allocator is locked
// down.  ipm_schur_sum_noalloc serves them.  It computes
//     K_hat = sum_s Z_s^T Y_s  (+ sum_s Yu_s)  (+ diag(d))
// from caller-owned device buffers, like the product inside
// ipm_condense_scenarios, but its split-K partial tiles live in the
// file-scope device array below instead of memory obtained from cudaMalloc.
//
// The array is a fixed 4 MiB (kScratchDoubles doubles).  Every GPU that
// loads this library holds it until the process exits.  Every call shares
// it and leaves its last contents behind; each partial tile is fully
// rewritten before it is read, so nothing needs clearing, but calls that
// overlap on the GPU (different streams, or different host threads) race on
// the array and must be serialised by the caller.
#include <atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/ipm.h"
#include "kernels.h"


namespace {

constexpr int NT = 64;                        // output tile
constexpr int NK = 16;                        // k chunk
constexpr long long kScratchDoubles = 1 << 19;  // 4 MiB of partial tiles
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_schur_scratch[kScratchDoubles];

// tile t of the upper triangle (ti <= tj), row-major over ti
__device__ __forceinline__ void tile_coords(int t, int nt1, int &ti, int &tj) {
  int i = 0, rem = t;
  while (rem >= nt1 - i) {
    rem -= nt1 - i;
    ++i;
  }
  ti = i;
  tj = i + rem;
}

__global__ void __launch_bounds__(256) k_schur_partial_na(int nx, int nu, int N, int spg, int nt1,
                                                          const double *__restrict__ A,
                                                          const double *__restrict__ B, double *scratch) {
  __shared__ double As[NK][NT];
  __shared__ double Bs[NK][NT];
  const int t = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
  int ti, tj;
  tile_coords(t, nt1, ti, tj);
  const int i0 = ti * NT, j0 = tj * NT;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int s0 = g * spg, s1 = min(N, s0 + spg);
  for (int s = s0; s < s1; ++s) {
    const double *Ag = A + (size_t)s * nx * nu;
    const double *Bg = B + (size_t)s * nx * nu;
    for (int k0 = 0; k0 < nx; k0 += NK) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + q * 256, kk = e >> 6, cc = e & 63;
        const int k = k0 + kk;
        As[kk][cc] = (k < nx && i0 + cc < nu) ? Ag[(size_t)k * nu + i0 + cc] : 0.0;
        Bs[kk][cc] = (k < nx && j0 + cc < nu) ? Bg[(size_t)k * nu + j0 + cc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) {
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
  }
  double *P = scratch + ((size_t)g * gridDim.x + t) * NT * NT;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) P[(ty * 4 + a) * NT + tx * 4 + b] = acc[a][b];
}

__global__ void k_schur_assemble_na(int nu, int N, int ngroups, int ntiles, int nt1,
                                    const double *__restrict__ scratch, const double *__restrict__ Yu,
                                    const double *__restrict__ diag, double *Khat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int i = (int)(t / nu), j = (int)(t % nu);
  if (i > j) return;
  const int ti = i / NT, tj = j / NT;
  const int tt = ti * nt1 - ti * (ti - 1) / 2 + (tj - ti);  // index of (ti, tj) in the upper list
  double v = 0.0;
  for (int g = 0; g < ngroups; ++g)
    v += scratch[((size_t)g * ntiles + tt) * NT * NT + (i - ti * NT) * NT + (j - tj * NT)];
  if (Yu)
    for (int s = 0; s < N; ++s) v += Yu[(size_t)s * nu * nu + (size_t)i * nu + j];
  if (diag && i == j) v += diag[i];
  Khat[(size_t)i * nu + j] = v;
  Khat[(size_t)j * nu + i] = v;
}

std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" ipm_status ipm_schur_sum_noalloc(const double *Z, const double *Y, const double *Yu,
                                            const double *diag, int n_scen, int n_x, int n_u, double *Khat,
                                            void *stream) {
  if (!Z || !Y || !Khat || n_scen < 1 || n_x < 1 || n_u < 1) return IPM_ERR_ARG;
  const int nt1 = (n_u + NT - 1) / NT;
  const long long ntiles = (long long)nt1 * (nt1 + 1) / 2;
  const long long tile_doubles = (long long)NT * NT;
  if (n_u > IPM_SCHUR_NOALLOC_MAX_NU || ntiles * tile_doubles > kScratchDoubles) return IPM_ERR_ARG;
  // an error left pending by earlier work on this thread is not ours to
  // clear or report as ours: refuse before launching anything
  if (cudaPeekAtLastError() != cudaSuccess) return IPM_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IPM_ERR_CUDA;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_schur_scratch) != cudaSuccess || !p) return IPM_ERR_CUDA;
      g_scratch_addr[dev] = (double *)p;
    }
    scratch = g_scratch_addr[dev];
  }
  // scenario groups: as many as the scratch holds, at most one per scenario
  long long gmax = kScratchDoubles / (ntiles * tile_doubles);
  long long target = (3 * 152 + ntiles - 1) / ntiles;
  int ngroups = (int)std::min<long long>(std::min<long long>(gmax, target), n_scen);
  if (ngroups < 1) ngroups = 1;
  const int spg = (n_scen + ngroups - 1) / ngroups;
  ngroups = (n_scen + spg - 1) / spg;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((unsigned)ntiles, (unsigned)ngroups);
  k_schur_partial_na<<<grid, 256, 0, st>>>(n_x, n_u, n_scen, spg, nt1, Z, Y, scratch);
  if (cudaGetLastError() != cudaSuccess) return IPM_ERR_CUDA;  // this launch's own error
  ipm_count_launch();
  const long long tot = (long long)n_u * n_u;
  k_schur_assemble_na<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_u, n_scen, ngroups, (int)ntiles, nt1,
                                                                      scratch, Yu, diag, Khat);
  if (cudaGetLastError() != cudaSuccess) return IPM_ERR_CUDA;
  ipm_count_launch();
  return IPM_OK;
}
