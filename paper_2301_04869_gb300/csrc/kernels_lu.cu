// K3-K5: batched static-pivot sparse LU of G_x (one pattern for all
// scenarios), the multi-RHS reduction solves Z = -G_x^{-1} G_u fused with the
// products Y = K [Z; I], and single-vector solves with G_x and G_x^T.
//
// Paper: §3.2 "Assembling the sparse matrices" (batched LU sharing one
// pattern, G_x^{-1} b = Q U^{-1} L^{-1} P b) and "Local reduction" (steps
// 1-2: T_x = -G_x^{-1} G_u V, [L_x; L_u] = K [T_x; V]).  Here V runs over
// all Cartesian vectors at once, split into RHS panels of 32 columns.
//
// Scheduling: the LU runs on a cluster of two CTAs per scenario (cluster
// barriers between its steps; a one-CTA kernel when the trailing block does
// not fit the pair's shared memory), the single-vector solves on one CTA per
// scenario, the multi-RHS solves on one CTA per (scenario, RHS panel) pair
// plus one per scenario for b; each walks a level schedule of the shared
// pattern with __syncthreads() between levels.  No grid-wide
// synchronisation and no waits between CTAs other than the cluster
// barriers.
#include <atomic>

#include "dev.cuh"
#include "kernels.h"


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

// Batched LU: the sparse pivots follow the level schedule (gather-form
// updates), then the dense trailing block [t0, nx) is factorized right-looking
// in shared memory when it fits (dynamic shared memory of nd*nd doubles),
// else in place through the slot map.
// Cluster helpers: rank in the cluster, a barrier over both CTAs with
// release/acquire ordering (shared and global memory), and a load from the
// peer CTA's shared memory.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ double ld_peer(const double *local, unsigned peer) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local));
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(peer));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

// Sparse part of the factorization of one scenario: values of G_x into the
// LU pattern, the level-scheduled sparse pivots (gather form), the scaling
// of L, and the products of the sparse pivots into the dense trailing
// block.  One CTA, or (PAIR) the two CTAs of a cluster sharing every step
// by index parity with cluster barriers between the steps.  Returns
// max |G_x| (the reference of the pivot test).
template <bool PAIR>
__device__ double lu_sparse_part(const DevSym &S, int nL, const double *__restrict__ J, double *A, double *r,
                                 int *flags, double piv_tol, int sc, double *sh, unsigned rank) {
  const int tid = threadIdx.x, bd = blockDim.x;
  const int t0i = PAIR ? tid + (int)rank * bd : tid, step = PAIR ? 2 * bd : bd;
  auto sync = [] {
    if (PAIR) cluster_sync_all();
    else __syncthreads();
  };
  double amax = 0.0;
  for (int p = t0i; p < S.nnzLU; p += step) {
    const int src = S.lu_init[p];
    const double v = src >= 0 ? J[(size_t)src * S.N + sc] : 0.0;
    A[p] = v;
    amax = fmax(amax, fabs(v));
  }
  amax = block_max(amax, sh);
  if (PAIR) {
    if (tid == 0) sh[16] = amax;
    cluster_sync_all();
    amax = fmax(amax, ld_peer(&sh[16], rank ^ 1u));
  }
  for (int l = 0; l < S.nlev_f; ++l) {
    for (int e = S.f_piv_ptr[l] + t0i; e < S.f_piv_ptr[l + 1]; e += step) {
      const int k = S.f_piv[e];
      const double d = A[S.lu_diag[k]];
      if (!(fabs(d) > piv_tol * amax)) flags[FLAG_SINGULAR] = 1;
      r[k] = 1.0 / d;
    }
    sync();
    for (int t = S.f_lev_ptr[l] + t0i; t < S.f_lev_ptr[l + 1]; t += step) {
      const int slot = S.f_tgt[t];
      double acc = A[slot];
      for (int o = S.f_op_ptr[t]; o < S.f_op_ptr[t + 1]; ++o)
        acc -= A[S.f_op_l[o]] * (A[S.f_op_u[o]] * r[S.f_op_k[o]]);
      A[slot] = acc;
    }
    sync();
  }
  for (int e = t0i; e < nL; e += step) A[S.lsc_slot[e]] *= r[S.lsc_k[e]];
  sync();
  if (S.nd == 0) return amax;
  // Products of the sparse pivots into the trailing block (L already
  // scaled): each entry owned by one of LU_LISTS lists, its products summed
  // and subtracted once; lists interleaved (coalesced), list q taken by
  // thread q of the cluster (or q mod blockDim.x of one CTA).  The products
  // read sparse L and U slots only, never a trailing-block slot, so batches
  // of eight have all their loads issued before the multiply-adds and
  // stores.
  const double *__restrict__ Ar = A;
  for (int q = t0i; q < LU_LISTS; q += step) {
    const int len = S.tw_len[q];
    double acc = 0.0;
    for (int q0 = 0; q0 < len; q0 += 8) {
      double lv[8], uv[8];
      int ev[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        lv[b] = 0.0;
        uv[b] = 0.0;
        ev[b] = -1;
        if (q0 + b < len) {
          const size_t at = (size_t)(q0 + b) * LU_LISTS + q;
          lv[b] = Ar[S.tw_l[at]];
          uv[b] = Ar[S.tw_u[at]];
          ev[b] = S.tw_e[at];
        }
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (q0 + b < len) {
          acc = fma(lv[b], uv[b], acc);
          if (ev[b] >= 0) {
            A[ev[b]] -= acc;
            acc = 0.0;
          }
        }
      }
    }
  }
  sync();
  return amax;
}

__global__ void k_lu_factor(DevSym S, int nL, const double *__restrict__ J, double *LU, double *rd,
                            int *flags, double piv_tol, int ns) {
  __shared__ double sh[32];
  extern __shared__ double T[];
  const int sc = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  double *A = LU + (size_t)sc * S.nnzLU;
  double *r = rd + (size_t)sc * S.nx;
  const double amax = lu_sparse_part<false>(S, nL, J, A, r, flags, piv_tol, sc, sh, 0u);
  const int nd = S.nd, t0 = S.t0;
  if (S.big) {  // the block is factored by the batched kernels
    if (tid == 0) S.lu_amax[sc] = amax;
    return;
  }
  if (nd == 0) return;
  const int *ts = S.tail_slot;
  // dense trailing block: columns [0, k0) in place through the slot map,
  // then the remaining (nd-k0)^2 block in shared memory (k0 = nd - ns)
  const int k0 = nd - ns;
  // columns [0, k0 - 1) through the slot map; the last of them is fused
  // into the load of the shared-memory block
  for (int k = 0; k < k0; ++k) {
    if (tid == 0) {
      const double d = A[ts[k * nd + k]];
      if (!(fabs(d) > piv_tol * amax)) flags[FLAG_SINGULAR] = 1;
      r[t0 + k] = 1.0 / d;
      sh[0] = r[t0 + k];
    }
    __syncthreads();
    const double rk = sh[0];
    const int m = nd - k - 1;
    if (k + 1 == k0) {
      // T = A22 - (A21 / d) A12, and L21 = A21 / d written back
      for (int e = tid; e < ns * ns; e += bd) {
        const int a = k0 + e / ns, b = k0 + e % ns;
        T[e] = A[ts[a * nd + b]] - (A[ts[a * nd + k]] * rk) * A[ts[k * nd + b]];
      }
      __syncthreads();
      for (int e = tid; e < m; e += bd) A[ts[(k + 1 + e) * nd + k]] *= rk;
      break;
    }
    for (int e = tid; e < m; e += bd) A[ts[(k + 1 + e) * nd + k]] *= rk;
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
      const int a = k + 1 + e / m, b = k + 1 + e % m;
      A[ts[a * nd + b]] -= A[ts[a * nd + k]] * A[ts[k * nd + b]];
    }
    __syncthreads();
  }
  if (ns == 0) return;
  if (k0 == 0)
    for (int e = tid; e < ns * ns; e += bd) T[e] = A[ts[(k0 + e / ns) * nd + k0 + e % ns]];
  __syncthreads();
  // Blocked right-looking LU of the ns x ns block in shared memory (static
  // diagonal pivots): per panel of PB columns, (a) the panel column by
  // column, (b) U12 = L11^{-1} A12 (thread per column), (c) the trailing
  // update A22 -= L21 U12 with 4 x 4 register tiles (one shared-memory read
  // per 4 multiply-adds instead of three per multiply-add).
  constexpr int PB = 16;
  for (int kb = 0; kb < ns; kb += PB) {
    const int pb = min(PB, ns - kb), ke = kb + pb;
    for (int k = kb; k < ke; ++k) {
      // one thread forms the pivot's reciprocal (a dependent FP64 division
      // is ~9 multiply-adds of FP64 work: not once per thread)
      if (tid == 0) {
        const double d = T[k * ns + k];
        if (!(fabs(d) > piv_tol * amax)) flags[FLAG_SINGULAR] = 1;
        r[t0 + k0 + k] = 1.0 / d;
        sh[0] = r[t0 + k0 + k];
      }
      __syncthreads();
      const double rk = sh[0];
      // thread per row: scale L(i, k), update the rest of the panel row
      for (int i = k + 1 + tid; i < ns; i += bd) {
        const double l = T[i * ns + k] * rk;
        T[i * ns + k] = l;
        for (int j = k + 1; j < ke; ++j) T[i * ns + j] -= l * T[k * ns + j];
      }
      __syncthreads();
    }
    if (ke >= ns) break;
    for (int j = ke + tid; j < ns; j += bd)
      for (int k = kb; k < ke; ++k) {
        const double x = T[k * ns + j];
        for (int i = k + 1; i < ke; ++i) T[i * ns + j] -= T[i * ns + k] * x;
      }
    __syncthreads();
    const int m = ns - ke, nt4 = (m + 3) / 4;
    for (int e = tid; e < nt4 * nt4; e += bd) {
      const int i0 = ke + (e / nt4) * 4, j0 = ke + (e % nt4) * 4;
      double c[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) c[a][b] = 0.0;
      for (int k = kb; k < ke; ++k) {
        double lv[4], uv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = i0 + a < ns ? T[(i0 + a) * ns + k] : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) uv[b] = j0 + b < ns ? T[k * ns + j0 + b] : 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) c[a][b] = fma(lv[a], uv[b], c[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (i0 + a < ns && j0 + b < ns) T[(i0 + a) * ns + j0 + b] -= c[a][b];
    }
    __syncthreads();
  }
  for (int e = tid; e < ns * ns; e += bd) A[ts[(k0 + e / ns) * nd + k0 + e % ns]] = T[e];
}

// Multi-RHS reduction solve for one scenario and one panel of 32 RHS columns
// (lane = column): Z = -U^{-1} L^{-1} (P G_u) (rows in LU position order),
// then Y = K_x [Z; I] and Y_u = K_u [Z; I].  The sparse rows follow the level
// schedule (one warp per row); the dense trailing block [t0, nx) is solved
// column by column by the whole CTA, in shared memory when it fits
// (tail_smem), else in place in Z.  T is the storage/arithmetic type of Z, Y
// (double on the FP64 path, float on the mixed path); Y_u accumulates in FP64.
// phase (large trailing block, S.big): 1 = the forward sparse rows and the
// trailing rows' right-hand sides only (left in Z for the batched block
// solves), 2 = the backward sparse rows and the products only; 0 = all.
template <typename T>
__device__ void zsolve_body(const DevSym &S, const double *__restrict__ LU, const double *__restrict__ rd,
                            const double *__restrict__ J, const double *__restrict__ K, T *Z, T *Y, double *Yu,
                            bool tail_smem, T *sh, const double *__restrict__ gvec, T *bvec, int *ezy,
                            int phase = 0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, bd = blockDim.x;
  const int nu = S.nu, nx = S.nx, N = S.N;
  // the CTA after the panels of Z (when bvec is given) solves b alone
  const bool bpanel = bvec != nullptr && (int)blockIdx.x == (nu + 31) / 32;
  const int sc = blockIdx.y, c0 = blockIdx.x * 32, c = bpanel ? nu + lane : c0 + lane;
  const int t0 = S.t0, nd = S.nd;
  const bool valid = c < nu;
  const int cc = valid ? c : nu - 1;
  const double *A = LU + (size_t)sc * S.nnzLU;
  const double *r = rd + (size_t)sc * nx;
  T *Zs = Z + (size_t)sc * nx * nu;
  T *Ys = Y + (size_t)sc * nx * nu;
  double *Yus = Yu + (size_t)sc * nu * nu;
  // Optional extra column n_u (when bvec is given): b = G_x^{-1} g of the
  // reduced right-hand side, solved by lane 0 of an extra CTA per scenario
  // (its forward sweep is dense, unlike those of the columns of G_u, so it
  // gets a CTA of its own instead of slowing one panel of Z), stored in
  // bvec [N][n_x] (position order).  zb/zst read a lane's own column, zw
  // writes it.
  const bool xb = bpanel && lane == 0;
  T *bs = bvec ? bvec + (size_t)sc * nx : nullptr;
  const T *zb = xb ? bs : Zs + cc;
  T *zw = xb ? bs : Zs + c;
  const size_t zst = xb ? 1 : (size_t)nu;
  const bool wr = valid || xb;
  // forward, sparse rows: this panel's schedule (rows its columns of G_u
  // reach, products against such rows only); the other rows are zero
  const int pan = blockIdx.x;
  if (phase != 2) {
  for (int e = S.zp_zptr[pan] + warp; e < S.zp_zptr[pan + 1]; e += nw)
    if (wr) zw[(size_t)S.zp_zrows[e] * zst] = (T)0;
  for (int l = S.zp_lev_off[pan]; l < S.zp_lev_off[pan + 1]; ++l) {
    for (int e = S.zp_lev_ptr[l] + warp; e < S.zp_lev_ptr[l + 1]; e += nw) {
      const int row = S.zp_rows[e];
      T acc = 0;
      if (xb) acc = (T)gvec[(size_t)sc * nx + S.iperm[row]];
      else
        for (int g = S.gu_ptr[row]; g < S.gu_ptr[row + 1]; ++g)
          if (S.gu_col[g] == cc) {
            const int src = S.gu_src[g];
            acc -= src >= 0 ? (T)J[(size_t)src * N + sc] : (T)-1.0;
          }
      for (int f = S.zp_eptr[e]; f < S.zp_eptr[e + 1]; ++f)
        acc -= (T)A[S.zp_slot[f]] * zb[(size_t)S.zp_col[f] * zst];
      if (wr) zw[(size_t)row * zst] = acc;
    }
    __syncthreads();
  }
  if (nd > 0) {
    // trailing block: right-hand side and the sparse part of each row
    for (int i = warp; i < nd; i += nw) {
      const int row = t0 + i;
      T acc = 0;
      if (xb) acc = (T)gvec[(size_t)sc * nx + S.iperm[row]];
      else
        for (int g = S.gu_ptr[row]; g < S.gu_ptr[row + 1]; ++g)
          if (S.gu_col[g] == cc) {
            const int src = S.gu_src[g];
            acc -= src >= 0 ? (T)J[(size_t)src * N + sc] : (T)-1.0;
          }
      for (int f = S.zp_tptr[pan * nd + i]; f < S.zp_tptr[pan * nd + i + 1]; ++f)
        acc -= (T)A[S.zp_tslot[f]] * zb[(size_t)S.zp_tcol[f] * zst];
      if (tail_smem) sh[i * 32 + lane] = acc;
      else if (valid) Zs[(size_t)row * nu + c] = acc;
    }
    __syncthreads();
    if (phase == 1) return;  // the block is solved by the batched kernels
    const int *ts = S.tail_slot;
    if (tail_smem) {
      // Blocked by 32 in shared memory: one warp solves each 32 x 32
      // diagonal block (lane = RHS column), then every warp applies the
      // block's columns to the remaining rows (warp = row, lane = column).
      // Column c of the block is contiguous in LU storage: (a, c) sits at
      // tail_slot[c] + a (read straight from the LU values, the same address
      // for all lanes).  Backward values are scaled as they are found.
      for (int kb = 0; kb < nd; kb += 32) {
        const int w = min(32, nd - kb);
        if (warp == 0) {
          for (int jj = 0; jj < w; ++jj) {
            const T xj = sh[(kb + jj) * 32 + lane];
            const double *col = A + ts[kb + jj] + kb;  // L(kb + i2, kb + jj) = col[i2]
            for (int i2 = jj + 1; i2 < w; ++i2) sh[(kb + i2) * 32 + lane] -= (T)col[i2] * xj;
          }
        }
        __syncthreads();
        for (int i = kb + w + warp; i < nd; i += nw) {
          T acc = sh[i * 32 + lane];
          for (int j = 0; j < w; ++j) acc -= (T)A[ts[kb + j] + i] * sh[(kb + j) * 32 + lane];
          sh[i * 32 + lane] = acc;
        }
        __syncthreads();
      }
      for (int kb = ((nd - 1) / 32) * 32; kb >= 0; kb -= 32) {
        const int w = min(32, nd - kb);
        if (warp == 0) {
          for (int jj = w - 1; jj >= 0; --jj) {
            const T xj = sh[(kb + jj) * 32 + lane] * (T)r[t0 + kb + jj];
            sh[(kb + jj) * 32 + lane] = xj;
            const double *col = A + ts[kb + jj] + kb;  // U(kb + i2, kb + jj) = col[i2]
            for (int i2 = 0; i2 < jj; ++i2) sh[(kb + i2) * 32 + lane] -= (T)col[i2] * xj;
          }
        }
        __syncthreads();
        for (int i = warp; i < kb; i += nw) {
          T acc = sh[i * 32 + lane];
          for (int j = 0; j < w; ++j) acc -= (T)A[ts[kb + j] + i] * sh[(kb + j) * 32 + lane];
          sh[i * 32 + lane] = acc;
        }
        __syncthreads();
      }
      for (int e = tid; e < nd * 32; e += bd) {
        const int i = e >> 5, q = e & 31;
        if (bpanel) {
          if (q == 0) bs[t0 + i] = sh[i * 32];
        } else if (c0 + q < nu) {
          Zs[(size_t)(t0 + i) * nu + c0 + q] = sh[i * 32 + q];
        }
      }
      __syncthreads();
    } else {
      // in place in Z (trailing block too large for shared memory):
      // forward, dense unit-lower part, column by column
      for (int k = 0; k < nd - 1; ++k) {
        const int m = (nd - k - 1) * 32;
        for (int e = tid; e < m; e += bd) {
          const int i = k + 1 + (e >> 5), q = e & 31;
          const T l = (T)A[ts[i * nd + k]];
          if (c0 + q < nu) Zs[(size_t)(t0 + i) * nu + c0 + q] -= l * Zs[(size_t)(t0 + k) * nu + c0 + q];
        }
        __syncthreads();
      }
      // backward, dense upper part (unscaled accumulators; x_k = acc_k / u_kk)
      for (int k = nd - 1; k > 0; --k) {
        const T rk = (T)r[t0 + k];
        const int m = k * 32;
        for (int e = tid; e < m; e += bd) {
          const int i = e >> 5, q = e & 31;
          const T u = (T)A[ts[i * nd + k]];
          if (c0 + q < nu) Zs[(size_t)(t0 + i) * nu + c0 + q] -= u * (Zs[(size_t)(t0 + k) * nu + c0 + q] * rk);
        }
        __syncthreads();
      }
      for (int e = tid; e < nd * 32; e += bd) {
        const int i = e >> 5, q = e & 31;
        if (c0 + q < nu) {
          T *dst = &Zs[(size_t)(t0 + i) * nu + c0 + q];
          *dst = *dst * (T)r[t0 + i];
        }
      }
      __syncthreads();
    }
  }
  }  // phase != 2
  if (phase == 1) return;
  // backward, sparse rows
  for (int l = 0; l < S.nlev_bs; ++l) {
    for (int e = S.bs_lev_ptr[l] + warp; e < S.bs_lev_ptr[l + 1]; e += nw) {
      const int row = S.bs_rows[e];
      T acc = zb[(size_t)row * zst];
      for (int f = S.br_ptr[row]; f < S.br_ptr[row + 1]; ++f)
        acc -= (T)A[S.br_uslot[f]] * zb[(size_t)S.br_col[f] * zst];
      if (wr) zw[(size_t)row * zst] = acc * (T)r[row];
    }
    __syncthreads();
  }
  if (bpanel) return;  // b needs no product with K
  for (int row = warp; row < nx; row += nw) {
    T acc = 0;
    for (int e = S.kx_ptr[row]; e < S.kx_ptr[row + 1]; ++e) {
      const int col = S.kx_col[e];
      const T v = (T)K[(size_t)S.kx_src[e] * N + sc];
      if (col < nx) acc += v * Zs[(size_t)col * nu + cc];
      else if (col - nx == cc) acc += v;
    }
    if (valid) Ys[(size_t)row * nu + c] = acc;
    if (ezy) {
      // largest biased exponents of the row of Z and of Y (the row balancing
      // of the emulated contraction), over the panels by atomic maximum;
      // ezy[k] for Z and ezy[N nx + k] for Y, k = sc nx + row
      unsigned ez = 0, ey = 0;
      if (valid) {
        ez = (unsigned)(((unsigned long long)__double_as_longlong((double)Zs[(size_t)row * nu + c]) >> 52) & 0x7FF);
        ey = (unsigned)(((unsigned long long)__double_as_longlong((double)acc) >> 52) & 0x7FF);
      }
      ez = __reduce_max_sync(0xffffffffu, ez);
      ey = __reduce_max_sync(0xffffffffu, ey);
      if (lane == 0) {
        const size_t k = (size_t)sc * nx + row;
        if (ez) atomicMax(&ezy[k], (int)ez);
        if (ey) atomicMax(&ezy[(size_t)N * nx + k], (int)ey);
      }
    }
  }
  for (int j = warp; j < nu; j += nw) {
    double acc = 0.0;
    for (int e = S.ku_ptr[j]; e < S.ku_ptr[j + 1]; ++e) {
      const int col = S.ku_col[e];
      const double v = K[(size_t)S.ku_src[e] * N + sc];
      if (col < nx) acc += v * (double)Zs[(size_t)col * nu + cc];
      else if (col - nx == cc) acc += v;
    }
    if (valid) Yus[(size_t)j * nu + c] = acc;
  }
}

// 5 CTAs per SM (shared memory and registers sized for it): the 640 CTAs of
// 64 scenarios x 10 panels then run in one wave on 152 SMs instead of 1.05
__global__ void __launch_bounds__(256, 5) k_zsolve64(DevSym S, const double *__restrict__ LU,
                                                  const double *__restrict__ rd,
                                                  const double *__restrict__ J,
                                                  const double *__restrict__ K, double *Z, double *Y,
                                                  double *Yu, int tail_smem, const double *__restrict__ gvec,
                                                  double *bvec, int *ezy, int phase) {
  extern __shared__ double shd[];
  zsolve_body<double>(S, LU, rd, J, K, Z, Y, Yu, tail_smem != 0, shd, gvec, bvec, ezy, phase);
}

__global__ void __launch_bounds__(256, 5) k_zsolve32(DevSym S, const double *__restrict__ LU,
                                                  const double *__restrict__ rd,
                                                  const double *__restrict__ J,
                                                  const double *__restrict__ K, float *Z, float *Y,
                                                  double *Yu, int tail_smem, int phase) {
  extern __shared__ float shf[];
  zsolve_body<float>(S, LU, rd, J, K, Z, Y, Yu, tail_smem != 0, shf, nullptr, (float *)nullptr, nullptr, phase);
}

// In-place solve of G_x v = b (trans = 0) or G_x^T v = b (trans = 1) for every
// scenario; v is [N][nx] in LU position order.  One CTA per scenario: sparse
// rows by levels (one warp per row, lanes over the row's entries), the dense
// trailing block column by column in shared memory.
// Sum over a group of GS consecutive lanes (GS a power of two <= 32).
template <int GS>
__device__ __forceinline__ double group_sum(double p) {
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  return p;
}

// One level of sparse rows, GS lanes per row: x[row] = (x[row] - sum_f
// A[slot_f] x[col_f]) * (scale ? r[row] : 1) over the row's products.  A
// scheduled row is one 16-byte record {row, first, end} and a product one
// {col, slot, transposed slot}, so each row costs three dependent loads
// (record, product, value).  Rows of a level are independent; the loop
// bounds are uniform over the CTA (shuffles).
template <int GS>
__device__ __forceinline__ void solve_level(const int4 *__restrict__ rows, int e0, int e1,
                                            const int4 *__restrict__ prod, bool trans_slot,
                                            const double *__restrict__ A, const double *__restrict__ r, bool scale,
                                            double *x) {
  const int grp = threadIdx.x / GS, sub = threadIdx.x % GS, ngrp = blockDim.x / GS;
  for (int eb = e0; eb < e1; eb += ngrp) {
    const int e = eb + grp;
    double part = 0.0;
    int row = -1;
    if (e < e1) {
      const int4 R = rows[e];
      row = R.x;
      for (int f = R.y + sub; f < R.z; f += GS) {
        const int4 P = prod[f];
        part = fma(A[trans_slot ? P.z : P.y], x[P.x], part);
      }
    }
    part = group_sum<GS>(part);
    if (sub == 0 && row >= 0) x[row] = scale ? (x[row] - part) * r[row] : x[row] - part;
  }
}

// One CTA per vector: vector b of v ([N * vps][n_x], position order) belongs
// to scenario b / vps (vps vectors per scenario share its factors).
// phase (large trailing block, S.big): 1 = the forward sparse rows and the
// sparse part of the trailing rows only, 2 = the backward sparse rows only
// (the dense block between them by the batched kernels of kernels_big.cu);
// 0 = all.
__global__ void __launch_bounds__(1024) k_solve1(DevSym S, const double *__restrict__ LU, const double *__restrict__ rd,
                                                double *v, int trans, int in_smem, int vps, int phase) {
  extern __shared__ double xsm[];
  __shared__ double blk[32][33];
  const int sc = blockIdx.x / vps, tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nx = S.nx, t0 = S.t0, nd = S.nd;
  const double *A = LU + (size_t)sc * S.nnzLU;
  const double *r = rd + (size_t)sc * nx;
  double *vs = v + (size_t)blockIdx.x * nx;
  // the solution vector of this scenario lives in shared memory when it fits
  double *x = in_smem ? xsm : vs;
  if (in_smem) {
    for (int i = tid; i < nx; i += bd) x[i] = vs[i];
    __syncthreads();
  }
  // forward sparse rows (few entries each): four lanes per row
  for (int l = 0; l < (phase == 2 ? 0 : S.nlev_fs); ++l) {
    solve_level<4>(S.fs4, S.fs_lev_ptr[l], S.fs_lev_ptr[l + 1], S.fr4, trans != 0, A, r, trans != 0, x);
    __syncthreads();
  }
  if (nd > 0 && phase != 2) {
    const int *ts = S.tail_slot;
    double *tv = x + t0;
    // sparse part of the trailing rows (their columns < t0), eight lanes per row
    {
      const int grp = tid / 8, sub = tid % 8, ngrp = bd / 8;
      for (int ib = 0; ib < nd; ib += ngrp) {
        const int i = ib + grp;
        double part = 0.0;
        if (i < nd) {
          const int row = t0 + i;
          for (int f = S.fr_ptr[row] + sub; f < S.fr_ptr[row + 1]; f += 8) {
            const int4 P = S.fr4[f];
            if (P.x < t0) part = fma(A[trans ? P.z : P.y], x[P.x], part);
          }
        }
        part = group_sum<8>(part);
        if (sub == 0 && i < nd) tv[i] -= part;
      }
    }
    __syncthreads();
    if (phase == 1) {
      if (in_smem)
        for (int i = tid; i < nx; i += bd) vs[i] = x[i];
      return;
    }
    // Dense trailing block, blocked by 32: one warp per 32 x 32 diagonal
    // block (lane = row, shuffles), all threads for the off-diagonal updates
    // (four partial sums).  Column c of the block is contiguous in LU
    // storage: entry (a, c) sits at tail_slot[c] + a.  Forward: T = L (unit)
    // or U^T (diagonal u_kk); backward: T = U or L^T.  Where T has the
    // diagonal u_kk the block multipliers are pre-scaled by 1/u_kk, so each
    // step of the diagonal solve is one shuffle and one multiply-add.
    for (int kb = 0; kb < nd; kb += 32) {
      const int w = min(32, nd - kb);
      for (int e = tid; e < 32 * 32; e += bd) {
        const int rr = e >> 5, cc = e & 31;
        double bv = 0.0;
        if (rr < w && cc < rr) bv = trans ? A[ts[kb + rr] + kb + cc] * r[t0 + kb + cc] : A[ts[kb + cc] + kb + rr];
        blk[rr][cc] = bv;
      }
      __syncthreads();
      if (warp == 0) {
        double xv = lane < w ? tv[kb + lane] : 0.0;
        for (int jj = 0; jj < w; ++jj) {
          const double xj = __shfl_sync(0xffffffffu, xv, jj);
          if (lane > jj) xv = fma(-blk[lane][jj], xj, xv);
        }
        if (lane < w) tv[kb + lane] = trans ? xv * r[t0 + kb + lane] : xv;
      }
      __syncthreads();
      for (int i = kb + w + tid; i < nd; i += bd) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = 0;
        if (trans) {
          const double *col = A + ts[i] + kb;  // U(kb + j, i), j = 0..w-1
          for (; j + 4 <= w; j += 4) {
            s0 = fma(col[j], tv[kb + j], s0);
            s1 = fma(col[j + 1], tv[kb + j + 1], s1);
            s2 = fma(col[j + 2], tv[kb + j + 2], s2);
            s3 = fma(col[j + 3], tv[kb + j + 3], s3);
          }
          for (; j < w; ++j) s0 = fma(col[j], tv[kb + j], s0);
        } else {
          for (; j + 4 <= w; j += 4) {
            s0 = fma(A[ts[kb + j] + i], tv[kb + j], s0);
            s1 = fma(A[ts[kb + j + 1] + i], tv[kb + j + 1], s1);
            s2 = fma(A[ts[kb + j + 2] + i], tv[kb + j + 2], s2);
            s3 = fma(A[ts[kb + j + 3] + i], tv[kb + j + 3], s3);
          }
          for (; j < w; ++j) s0 = fma(A[ts[kb + j] + i], tv[kb + j], s0);
        }
        tv[i] -= (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
    }
    for (int kb = ((nd - 1) / 32) * 32; kb >= 0; kb -= 32) {
      const int w = min(32, nd - kb);
      for (int e = tid; e < 32 * 32; e += bd) {
        const int rr = e >> 5, cc = e & 31;
        double bv = 0.0;
        if (rr < w && cc < w && cc > rr) bv = trans ? A[ts[kb + rr] + kb + cc] : A[ts[kb + cc] + kb + rr] * r[t0 + kb + cc];
        blk[rr][cc] = bv;
      }
      __syncthreads();
      if (warp == 0) {
        double xv = lane < w ? tv[kb + lane] : 0.0;
        for (int jj = w - 1; jj >= 0; --jj) {
          const double xj = __shfl_sync(0xffffffffu, xv, jj);
          if (lane < jj) xv = fma(-blk[lane][jj], xj, xv);
        }
        if (lane < w) tv[kb + lane] = trans ? xv : xv * r[t0 + kb + lane];
      }
      __syncthreads();
      for (int i = tid; i < kb; i += bd) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = 0;
        if (trans) {
          const double *col = A + ts[i] + kb;  // L(kb + j, i), j = 0..w-1
          for (; j + 4 <= w; j += 4) {
            s0 = fma(col[j], tv[kb + j], s0);
            s1 = fma(col[j + 1], tv[kb + j + 1], s1);
            s2 = fma(col[j + 2], tv[kb + j + 2], s2);
            s3 = fma(col[j + 3], tv[kb + j + 3], s3);
          }
          for (; j < w; ++j) s0 = fma(col[j], tv[kb + j], s0);
        } else {
          for (; j + 4 <= w; j += 4) {
            s0 = fma(A[ts[kb + j] + i], tv[kb + j], s0);
            s1 = fma(A[ts[kb + j + 1] + i], tv[kb + j + 1], s1);
            s2 = fma(A[ts[kb + j + 2] + i], tv[kb + j + 2], s2);
            s3 = fma(A[ts[kb + j + 3] + i], tv[kb + j + 3], s3);
          }
          for (; j < w; ++j) s0 = fma(A[ts[kb + j] + i], tv[kb + j], s0);
        }
        tv[i] -= (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
    }
  }
  if (phase == 1) {  // (no trailing block)
    if (in_smem)
      for (int i = tid; i < nx; i += bd) vs[i] = x[i];
    return;
  }
  // backward sparse rows: eight lanes per row
  for (int l = 0; l < S.nlev_bs; ++l) {
    solve_level<8>(S.bs4, S.bs_lev_ptr[l], S.bs_lev_ptr[l + 1], S.br4, trans != 0, A, r, trans == 0, x);
    __syncthreads();
  }
  if (in_smem)
    for (int i = tid; i < nx; i += bd) vs[i] = x[i];
}


// The same factorization by a cluster of two CTAs per scenario (two SMs'
// FP64 units): the sparse part shared by index parity; the nd x nd
// trailing block is then split by column panels of 16, panel q
// held by CTA q mod 2 in its shared memory.  Per panel: its owner factors
// it (pivots, L column scaling, the rest of the panel), both CTAs meet at a
// cluster barrier, the other CTA copies the panel from the owner's shared
// memory, and each CTA solves U12 = L11^{-1} A12 and updates A22 -= L21 U12
// on its own columns (4 x 4 register tiles).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 1)
    k_lu_factor_pair(DevSym S, int nL, const double *__restrict__ J, double *LU, double *rd, int *flags,
                     double piv_tol) {
  constexpr int PB = 16;
  __shared__ double sh[32];
  extern __shared__ double Tl[];
  const unsigned rank = cluster_rank();
  const int sc = blockIdx.x >> 1, tid = threadIdx.x, bd = blockDim.x;
  double *A = LU + (size_t)sc * S.nnzLU;
  double *r = rd + (size_t)sc * S.nx;
  const int nd = S.nd, t0 = S.t0, ns = nd;
  const double amax = lu_sparse_part<true>(S, nL, J, A, r, flags, piv_tol, sc, sh, rank);
  if (nd == 0) return;  // the same on both CTAs
  const int np = (ns + PB - 1) / PB, LDL = ((np + 1) / 2) * PB;
  double *Pb = Tl + (size_t)ns * LDL;  // the other CTA's panel [ns][PB]
  const int *ts = S.tail_slot;
  // own local column lc <-> block column (2 (lc / PB) + rank) PB + lc % PB
  for (int e = tid; e < ns * LDL; e += bd) {
    const int i = e / LDL, lc = e % LDL;
    const int c = (2 * (lc / PB) + (int)rank) * PB + lc % PB;
    Tl[e] = c < ns ? A[ts[i * nd + c]] : 0.0;
  }
  __syncthreads();
  for (int p = 0; p < np; ++p) {
    const int kb = p * PB, ke = min(kb + PB, ns), pb = ke - kb;
    const bool own = (p & 1) == (int)rank;
    const int lc0 = (p >> 1) * PB;  // the panel's first local column in its owner
    if (own) {
      for (int k = kb; k < ke; ++k) {
        const int lk = lc0 + (k - kb);
        if (tid == 0) {
          const double d = Tl[k * LDL + lk];
          if (!(fabs(d) > piv_tol * amax)) flags[FLAG_SINGULAR] = 1;
          r[t0 + k] = 1.0 / d;
          sh[17] = r[t0 + k];
        }
        __syncthreads();
        const double rk = sh[17];
        for (int i = k + 1 + tid; i < ns; i += bd) {
          const double l = Tl[i * LDL + lk] * rk;
          Tl[i * LDL + lk] = l;
          for (int j = k + 1; j < ke; ++j) Tl[i * LDL + lc0 + (j - kb)] -= l * Tl[k * LDL + lc0 + (j - kb)];
        }
        __syncthreads();
      }
    }
    cluster_sync_all();  // panel p factored
    if (p == np - 1) break;
    const double *Lp;
    int ldp, cp0;
    if (own) {
      Lp = Tl;
      ldp = LDL;
      cp0 = lc0;
    } else {
      for (int e = tid; e < (ns - kb) * pb; e += bd) {
        const int i = kb + e / pb, j = e % pb;
        Pb[i * PB + j] = ld_peer(&Tl[i * LDL + lc0 + j], rank ^ 1u);
      }
      __syncthreads();
      Lp = Pb;
      ldp = PB;
      cp0 = 0;
    }
    // own columns right of the panel: local panels from lps on
    const int lcs = ((p + 2 - (int)rank) / 2) * PB;
    for (int lj = lcs + tid; lj < LDL; lj += bd)
      for (int k = kb; k < ke; ++k) {
        const double x = Tl[k * LDL + lj];
        for (int i = k + 1; i < ke; ++i) Tl[i * LDL + lj] -= Lp[i * ldp + cp0 + (k - kb)] * x;
      }
    __syncthreads();
    const int m = ns - ke, nc = LDL - lcs, nt4r = (m + 3) / 4, nt4c = (nc + 3) / 4;
    for (int e = tid; e < nt4r * nt4c; e += bd) {
      const int i0 = ke + (e / nt4c) * 4, j0 = lcs + (e % nt4c) * 4;
      double c[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) c[a][b] = 0.0;
      for (int k = kb; k < ke; ++k) {
        double lv[4], uv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = i0 + a < ns ? Lp[(i0 + a) * ldp + cp0 + (k - kb)] : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) uv[b] = j0 + b < LDL ? Tl[k * LDL + j0 + b] : 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) c[a][b] = fma(lv[a], uv[b], c[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (i0 + a < ns && j0 + b < LDL) Tl[(i0 + a) * LDL + j0 + b] -= c[a][b];
    }
    __syncthreads();
  }
  cluster_sync_all();  // no CTA leaves while the other may still read its panels
  for (int e = tid; e < ns * LDL; e += bd) {
    const int i = e / LDL, lc = e % LDL;
    const int c = (2 * (lc / PB) + (int)rank) * PB + lc % PB;
    if (c < ns) A[ts[i * nd + c]] = Tl[e];
  }
}
}  // namespace

void launch_lu_factor(const DevSym &S, int nL, const double *J, double *LU, double *rd, int *flags,
                      cudaStream_t st, bool allow_pair, const EmuLuPlan *emu_lu) {
  // trailing sub-block held in shared memory: as large as fits next to the
  // kernel's static shared memory (170 x 170 doubles on GB300)
  static const int ns_max = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_lu_factor);
    int n = 1;
    while ((size_t)(n + 1) * (n + 1) * sizeof(double) + fa.sharedSizeBytes <= (size_t)optin) ++n;
    return n;
  }();
  // a cluster of two CTAs per scenario when the trailing block fits their
  // shared memory (own columns plus one panel of the other CTA)
  static const size_t pair_cap = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_lu_factor_pair) != cudaSuccess) return (size_t)0;
    return raise_smem_cap(k_lu_factor_pair) ? (size_t)optin - fa.sharedSizeBytes : (size_t)0;
  }();
  if (S.big) {
    // sparse part (one CTA per scenario), then the block by the batched kernels
    k_lu_factor<<<S.N, 512, 0, st>>>(S, nL, J, LU, rd, flags, 1e-14, 0); ipm_count_launch();
    launch_big_lu_dense(S, LU, rd, S.lu_amax, flags, st, emu_lu);
    return;
  }
  const int np = (S.nd + 15) / 16, ldl = ((np + 1) / 2) * 16;
  const size_t pair_smem = (size_t)S.nd * (ldl + 16) * sizeof(double);
  if (allow_pair && S.nd > 0 && pair_smem <= pair_cap) {
    k_lu_factor_pair<<<2 * S.N, 512, pair_smem, st>>>(S, nL, J, LU, rd, flags, 1e-14);
    ipm_count_launch();
    return;
  }
  const int ns = S.nd < ns_max ? S.nd : ns_max;
  const size_t smem = (size_t)ns * ns * sizeof(double);
  static const bool cap = raise_smem_cap(k_lu_factor);
  (void)cap;
  k_lu_factor<<<S.N, 512, smem, st>>>(S, nL, J, LU, rd, flags, 1e-14, ns); ipm_count_launch();
}
static int zsolve_smem_ok(const DevSym &S, size_t elem) {
  return (S.nd > 0 && (size_t)S.nd * 32 * elem <= 100 * 1024) ? 1 : 0;
}
bool zsolve64_folds_b(const DevSym &S) { return !S.big && (S.nd == 0 || zsolve_smem_ok(S, sizeof(double))); }

void launch_zsolve64(const DevSym &S, const double *LU, const double *rd, const double *J,
                     const double *K, double *Z, double *Y, double *Yu, cudaStream_t st, int threads,
                     const double *g, double *b, int *ezy) {
  const int sm = zsolve_smem_ok(S, sizeof(double));
  if (!zsolve64_folds_b(S)) b = nullptr;
  dim3 grid((S.nu + 31) / 32 + (b ? 1 : 0), S.N);
  const size_t bytes = sm ? (size_t)S.nd * 32 * sizeof(double) : 0;
  // dynamic plus static shared memory may pass the 48 KB default
  static const bool cap = raise_smem_cap(k_zsolve64);
  (void)cap;
  if (S.big) {
    // forward sparse rows and the block's right-hand sides, the block by the
    // batched triangular solves, then the backward sparse rows and products
    k_zsolve64<<<grid, threads, 0, st>>>(S, LU, rd, J, K, Z, Y, Yu, 0, g, b, ezy, 1); ipm_count_launch();
    launch_big_trsm64(S, LU, rd, Z, st);
    k_zsolve64<<<grid, threads, 0, st>>>(S, LU, rd, J, K, Z, Y, Yu, 0, g, b, ezy, 2); ipm_count_launch();
    return;
  }
  k_zsolve64<<<grid, threads, bytes, st>>>(S, LU, rd, J, K, Z, Y, Yu, sm, g, b, ezy, 0); ipm_count_launch();
}
void launch_zsolve32(const DevSym &S, const double *LU, const double *rd, const double *J,
                     const double *K, float *Z, float *Y, double *Yu, cudaStream_t st, int threads,
                     const TcsPlan *tcs, int *flags) {
  dim3 grid((S.nu + 31) / 32, S.N);
  const int sm = zsolve_smem_ok(S, sizeof(float));
  const size_t bytes = sm ? (size_t)S.nd * 32 * sizeof(float) : 0;
  static const bool cap = raise_smem_cap(k_zsolve32);
  (void)cap;
  if (S.big) {
    k_zsolve32<<<grid, threads, 0, st>>>(S, LU, rd, J, K, Z, Y, Yu, 0, 1); ipm_count_launch();
    launch_big_trsm32(S, LU, rd, Z, st, tcs, flags);
    k_zsolve32<<<grid, threads, 0, st>>>(S, LU, rd, J, K, Z, Y, Yu, 0, 2); ipm_count_launch();
    return;
  }
  k_zsolve32<<<grid, threads, bytes, st>>>(S, LU, rd, J, K, Z, Y, Yu, sm, 0); ipm_count_launch();
}
void launch_solve1(const DevSym &S, const double *LU, const double *rd, double *v, int trans,
                   cudaStream_t st) {
  // the scenario's vector in shared memory when it fits next to the
  // kernel's static shared memory
  static const size_t cap = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_solve1);
    return raise_smem_cap(k_solve1) ? (size_t)optin - fa.sharedSizeBytes : (size_t)0;
  }();
  const int sm = (size_t)S.nx * sizeof(double) <= cap ? 1 : 0;
  const size_t bytes = sm ? (size_t)S.nx * sizeof(double) : 0;
  if (S.big) {
    // sparse rows in one CTA of 1,024 threads per scenario (the level sweeps
    // of the large networks are long: more rows in flight per round); the
    // dense block by the batched single-vector kernels (many CTAs per scenario)
    k_solve1<<<S.N, 1024, bytes, st>>>(S, LU, rd, v, trans, sm, 1, 1); ipm_count_launch();
    launch_big_trsv(S, LU, rd, v, trans, st);
    k_solve1<<<S.N, 1024, bytes, st>>>(S, LU, rd, v, trans, sm, 1, 2); ipm_count_launch();
    return;
  }
  k_solve1<<<S.N, 512, bytes, st>>>(S, LU, rd, v, trans, sm, 1, 0); ipm_count_launch();
}

void launch_solve1_batched(const DevSym &S, const double *LU, const double *rd, double *v, int trans, int vps,
                           int threads, cudaStream_t st) {
  static const size_t cap = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_solve1);
    return raise_smem_cap(k_solve1) ? (size_t)optin - fa.sharedSizeBytes : (size_t)0;
  }();
  const int sm = (size_t)S.nx * sizeof(double) <= cap ? 1 : 0;
  const size_t bytes = sm ? (size_t)S.nx * sizeof(double) : 0;
  const long long nb = (long long)S.N * vps;
  k_solve1<<<(unsigned)nb, threads, bytes, st>>>(S, LU, rd, v, trans, sm, vps, 0); ipm_count_launch();
}
