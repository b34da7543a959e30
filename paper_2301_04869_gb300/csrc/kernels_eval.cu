// K1/K2: line-wise evaluation of the OPF model and condensation of the KKT
// blocks (Props. 2.1, 2.2), plus the right-hand sides of eq. (6).
//
// Evaluation is organised by bus: thread (bus i, scenario) walks the lines
// incident to i and owns row i of every bus-level block (no atomics, fixed
// summation order).  Each pi-model line end contributes
//   P = g v_m^2 - v_m v_o (g cos d + b sin d)
//   Q = -(b + b_c/2) v_m^2 - v_m v_o (g sin d - b cos d),   d = th_m - th_o
// to the injections of its bus; derivatives below are those of these two
// closed forms (the CPU oracle instead differentiates S = V conj(Y V) in
// complex-matrix form).  With line ratings, the line-flow rows of h
// (§4.1.1) are h = P^2 + Q^2 of one line end, owned by the thread of that
// end's bus: its first derivatives 2 (P dP + Q dQ) and the Hessian
// 2 (dP dP^T + dQ dQ^T + P d2P + Q d2Q) come from the same closed forms.
#include <atomic>

#include "dev.cuh"
#include "kernels.h"


namespace {

struct LineEnd {
  double P, Q;
  double dPtm, dPto, dPvm, dPvo, dQtm, dQto, dQvm, dQvo;
  double A, B, vm, vo, g, bb;
};

__device__ __forceinline__ void line_end(double vm, double vo, double c, double s, double g,
                                         double b, double bh, LineEnd &e) {
  const double A = g * c + b * s, B = g * s - b * c, vv = vm * vo;
  e.P = g * vm * vm - vv * A;
  e.Q = -(b + bh) * vm * vm - vv * B;
  e.dPtm = vv * B;
  e.dPto = -vv * B;
  e.dPvm = 2.0 * g * vm - vo * A;
  e.dPvo = -vm * A;
  e.dQtm = -vv * A;
  e.dQto = vv * A;
  e.dQvm = -2.0 * (b + bh) * vm - vo * B;
  e.dQvo = -vm * B;
  e.A = A; e.B = B; e.vm = vm; e.vo = vo; e.g = g; e.bb = b + bh;
}
// second derivatives of P and Q of one line end (m = own bus, o = other bus)
__device__ __forceinline__ double Ptmtm(const LineEnd &e) { return e.vm * e.vo * e.A; }
__device__ __forceinline__ double Ptmto(const LineEnd &e) { return -e.vm * e.vo * e.A; }
__device__ __forceinline__ double Ptoto(const LineEnd &e) { return e.vm * e.vo * e.A; }
__device__ __forceinline__ double Ptmvm(const LineEnd &e) { return e.vo * e.B; }
__device__ __forceinline__ double Ptmvo(const LineEnd &e) { return e.vm * e.B; }
__device__ __forceinline__ double Ptovm(const LineEnd &e) { return -e.vo * e.B; }
__device__ __forceinline__ double Ptovo(const LineEnd &e) { return -e.vm * e.B; }
__device__ __forceinline__ double Pvmvm(const LineEnd &e) { return 2.0 * e.g; }
__device__ __forceinline__ double Pvmvo(const LineEnd &e) { return -e.A; }
__device__ __forceinline__ double Qtmtm(const LineEnd &e) { return e.vm * e.vo * e.B; }
__device__ __forceinline__ double Qtmto(const LineEnd &e) { return -e.vm * e.vo * e.B; }
__device__ __forceinline__ double Qtoto(const LineEnd &e) { return e.vm * e.vo * e.B; }
__device__ __forceinline__ double Qtmvm(const LineEnd &e) { return -e.vo * e.A; }
__device__ __forceinline__ double Qtmvo(const LineEnd &e) { return -e.vm * e.A; }
__device__ __forceinline__ double Qtovm(const LineEnd &e) { return e.vo * e.A; }
__device__ __forceinline__ double Qtovo(const LineEnd &e) { return e.vm * e.A; }
__device__ __forceinline__ double Qvmvm(const LineEnd &e) { return -2.0 * e.bb; }
__device__ __forceinline__ double Qvmvo(const LineEnd &e) { return -e.B; }

// d2 P and d2 Q of a line end w.r.t. two of its variables, indexed
// 0 = theta_m, 1 = v_m, 2 = theta_o, 3 = v_o (m: the end's bus, o: the other)
__device__ __forceinline__ void d2PQ(const LineEnd &e, int a, int b, double &p, double &q) {
  if (a > b) { const int t = a; a = b; b = t; }
  const int k = a * 4 + b;
  switch (k) {
    case 0: p = Ptmtm(e); q = Qtmtm(e); break;   // tm tm
    case 1: p = Ptmvm(e); q = Qtmvm(e); break;   // tm vm
    case 2: p = Ptmto(e); q = Qtmto(e); break;   // tm to
    case 3: p = Ptmvo(e); q = Qtmvo(e); break;   // tm vo
    case 5: p = Pvmvm(e); q = Qvmvm(e); break;   // vm vm
    case 6: p = Ptovm(e); q = Qtovm(e); break;   // vm to
    case 7: p = Pvmvo(e); q = Qvmvo(e); break;   // vm vo
    case 10: p = Ptoto(e); q = Qtoto(e); break;  // to to
    case 11: p = Ptovo(e); q = Qtovo(e); break;  // to vo
    default: p = 0.0; q = 0.0; break;            // vo vo: P, Q are linear in v_o
  }
}
__device__ __forceinline__ double d1P(const LineEnd &e, int a) {
  return a == 0 ? e.dPtm : a == 1 ? e.dPvm : a == 2 ? e.dPto : e.dPvo;
}
__device__ __forceinline__ double d1Q(const LineEnd &e, int a) {
  return a == 0 ? e.dQtm : a == 1 ? e.dQvm : a == 2 ? e.dQto : e.dQvo;
}
// second derivative of h = P^2 + Q^2 of a line end
__device__ __forceinline__ double d2flow(const LineEnd &e, int a, int b) {
  double p2, q2;
  d2PQ(e, a, b, p2, q2);
  return 2.0 * (d1P(e, a) * d1P(e, b) + d1Q(e, a) * d1Q(e, b) + e.P * p2 + e.Q * q2);
}
// flow row of the end of line l at bus i (from-end rows first, then to-end rows)
__device__ __forceinline__ int flow_row(const DevSym &S, int l, int i) {
  return S.ng + 1 + (i == S.lfr[l] ? 0 : S.L) + l;
}

// multipliers of the P and Q injections of bus k in scenario sc: the g row
// multiplier y, the h row multiplier z, and for the slack bus the cost slope
// (f_i = cost/N depends on x through Pg_0 = P_0 + Pd_0).
__device__ __forceinline__ double lam_P(const DevSym &S, const double *y, const double *z,
                                        const double *h, int sc, int k) {
  if (k >= 1) return y[(size_t)sc * S.nx + S.xth[k]];
  const double pg0 = h[(size_t)sc * S.m + S.ng];
  return z[(size_t)sc * S.m + S.ng] + (2.0 * S.c2[0] * pg0 + S.c1[0]) / S.N;
}
__device__ __forceinline__ double lam_Q(const DevSym &S, const double *y, const double *z, int sc,
                                        int k) {
  const int q = S.xv[k];
  return q >= 0 ? y[(size_t)sc * S.nx + q] : z[(size_t)sc * S.m + S.gen_of_bus[k]];
}

__global__ void k_functions(DevSym S, const double *__restrict__ x, const double *__restrict__ u,
                            double *P, double *Q, double *g, double *h, double *fs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.n * S.N) return;
  const int i = t / S.N, sc = t - i * S.N;
  const double thi = bus_theta(S, x, sc, i), vi = bus_v(S, x, u, sc, i);
  double p = 0.0, q = 0.0;
  for (int e = S.inc_ptr[i]; e < S.inc_ptr[i + 1]; ++e) {
    const int l = S.inc_line[e], k = S.inc_other[e];
    double sn, cs;
    sincos(thi - bus_theta(S, x, sc, k), &sn, &cs);
    LineEnd le;
    const double on = S.lon ? S.lon[(size_t)l * S.N + sc] : 1.0;  // 0: line out of service
    line_end(vi, bus_v(S, x, u, sc, k), cs, sn, on * S.lg[l], on * S.lb[l], on * S.lbh[l], le);
    p += le.P;
    q += le.Q;
    if (S.nflow) h[(size_t)sc * S.m + flow_row(S, l, i)] = le.P * le.P + le.Q * le.Q;
  }
  const size_t bi = (size_t)sc * S.n + i;
  P[bi] = p;
  Q[bi] = q;
  const double pd = S.pd[bi], qd = S.qd[bi];
  const int gk = S.gen_of_bus[i];
  if (i >= 1) g[(size_t)sc * S.nx + S.xth[i]] = p + pd - (gk >= 1 ? u[S.ng + gk - 1] : 0.0);
  if (S.xv[i] >= 0) g[(size_t)sc * S.nx + S.xv[i]] = q + qd;
  if (gk >= 0) h[(size_t)sc * S.m + gk] = q + qd;
  if (i == 0) {
    const double pg0 = p + pd;
    h[(size_t)sc * S.m + S.ng] = pg0;
    fs[sc] = (S.c2[0] * pg0 * pg0 + S.c1[0] * pg0) / S.N;
  }
}

__global__ void k_derivatives(DevSym S, const double *__restrict__ x, const double *__restrict__ u,
                              const double *__restrict__ y, const double *__restrict__ z,
                              const double *__restrict__ h, double *J, double *W, double *JTl, double *HF) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.n * S.N) return;
  const int i = t / S.N, sc = t - i * S.N, N = S.N;
  const double thi = bus_theta(S, x, sc, i), vi = bus_v(S, x, u, sc, i);
  const double lPi = lam_P(S, y, z, h, sc, i), lQi = lam_Q(S, y, z, sc, i);
  double jd0 = 0, jd1 = 0, jd2 = 0, jd3 = 0;   // dP/dth, dP/dv, dQ/dth, dQ/dv (own bus)
  double wtt = 0, wtv = 0, wvv = 0;            // diagonal Hessian block
  double gt = 0, gv = 0;                       // (J^T lambda) at (th_i, v_i)
  for (int e = S.inc_ptr[i]; e < S.inc_ptr[i + 1]; ++e) {
    const int l = S.inc_line[e], k = S.inc_other[e], q = S.inc_aslot[e];
    const double vk = bus_v(S, x, u, sc, k);
    double sn, cs;
    sincos(thi - bus_theta(S, x, sc, k), &sn, &cs);
    LineEnd own, oth;
    // a line out of service (contingency) stamps nothing: every quantity of a
    // line end is linear in its admittances g, b, b_c/2
    const double on = S.lon ? S.lon[(size_t)l * N + sc] : 1.0;
    const double lg = on * S.lg[l], lb = on * S.lb[l], lbh = on * S.lbh[l];
    line_end(vi, vk, cs, sn, lg, lb, lbh, own);
    line_end(vk, vi, cs, -sn, lg, lb, lbh, oth);
    const double lPk = lam_P(S, y, z, h, sc, k), lQk = lam_Q(S, y, z, sc, k);
    jd0 += own.dPtm; jd1 += own.dPvm; jd2 += own.dQtm; jd3 += own.dQvm;
    J[((size_t)q * 4 + 0) * N + sc] = own.dPto;
    J[((size_t)q * 4 + 1) * N + sc] = own.dPvo;
    J[((size_t)q * 4 + 2) * N + sc] = own.dQto;
    J[((size_t)q * 4 + 3) * N + sc] = own.dQvo;
    wtt += lPi * Ptmtm(own) + lQi * Qtmtm(own) + lPk * Ptoto(oth) + lQk * Qtoto(oth);
    wtv += lPi * Ptmvm(own) + lQi * Qtmvm(own) + lPk * Ptovo(oth) + lQk * Qtovo(oth);
    wvv += lPi * Pvmvm(own) + lQi * Qvmvm(own);
    W[((size_t)q * 4 + 0) * N + sc] = lPi * Ptmto(own) + lQi * Qtmto(own) + lPk * Ptmto(oth) + lQk * Qtmto(oth);
    W[((size_t)q * 4 + 1) * N + sc] = lPi * Ptmvo(own) + lQi * Qtmvo(own) + lPk * Ptovm(oth) + lQk * Qtovm(oth);
    W[((size_t)q * 4 + 2) * N + sc] = lPi * Ptovm(own) + lQi * Qtovm(own) + lPk * Ptmvo(oth) + lQk * Qtmvo(oth);
    W[((size_t)q * 4 + 3) * N + sc] = lPi * Pvmvo(own) + lQi * Qvmvo(own) + lPk * Pvmvo(oth) + lQk * Qvmvo(oth);
    gt += lPi * own.dPtm + lQi * own.dQtm + lPk * oth.dPto + lQk * oth.dQto;
    gv += lPi * own.dPvm + lQi * own.dQvm + lPk * oth.dPvo + lQk * oth.dQvo;
    if (S.nflow) {
      // flow rows of both ends of line l: h_own (this thread's row) and h_oth;
      // row i of W and of J^T lambda gets the terms in (theta_i, v_i)
      const int ro = flow_row(S, l, i), rk = flow_row(S, l, k);
      const double zo = z[(size_t)sc * S.m + ro], zk = z[(size_t)sc * S.m + rk];
      const int fo = ro - S.ng - 1;
      for (int a = 0; a < 4; ++a)
        HF[((size_t)(fo * 2 + (a >> 1)) * 2 + (a & 1)) * N + sc] =
            2.0 * (own.P * d1P(own, a) + own.Q * d1Q(own, a));
      // own end: i is m (0, 1), k is o (2, 3); other end: i is o, k is m
      gt += zo * 2.0 * (own.P * own.dPtm + own.Q * own.dQtm) + zk * 2.0 * (oth.P * oth.dPto + oth.Q * oth.dQto);
      gv += zo * 2.0 * (own.P * own.dPvm + own.Q * own.dQvm) + zk * 2.0 * (oth.P * oth.dPvo + oth.Q * oth.dQvo);
      wtt += zo * d2flow(own, 0, 0) + zk * d2flow(oth, 2, 2);
      wtv += zo * d2flow(own, 0, 1) + zk * d2flow(oth, 2, 3);
      wvv += zo * d2flow(own, 1, 1) + zk * d2flow(oth, 3, 3);
      W[((size_t)q * 4 + 0) * N + sc] += zo * d2flow(own, 0, 2) + zk * d2flow(oth, 2, 0);
      W[((size_t)q * 4 + 1) * N + sc] += zo * d2flow(own, 0, 3) + zk * d2flow(oth, 2, 1);
      W[((size_t)q * 4 + 2) * N + sc] += zo * d2flow(own, 1, 2) + zk * d2flow(oth, 3, 0);
      W[((size_t)q * 4 + 3) * N + sc] += zo * d2flow(own, 1, 3) + zk * d2flow(oth, 3, 1);
    }
  }
  const int d = S.a_diag[i];
  J[((size_t)d * 4 + 0) * N + sc] = jd0;
  J[((size_t)d * 4 + 1) * N + sc] = jd1;
  J[((size_t)d * 4 + 2) * N + sc] = jd2;
  J[((size_t)d * 4 + 3) * N + sc] = jd3;
  W[((size_t)d * 4 + 0) * N + sc] = wtt;
  W[((size_t)d * 4 + 1) * N + sc] = wtv;
  W[((size_t)d * 4 + 2) * N + sc] = wtv;
  W[((size_t)d * 4 + 3) * N + sc] = wvv;
  JTl[(size_t)sc * 2 * S.n + i] = gt;
  JTl[(size_t)sc * 2 * S.n + S.n + i] = gv;
}

__device__ __forceinline__ double sigma_of(double w, double l, double b, double zl, double zu) {
  double r = 0.0;
  if (isfinite(l)) r += zl / (w - l);
  if (isfinite(b)) r += zu / (b - w);
  return r;
}
__device__ __forceinline__ double bgrad_of(double w, double l, double b, double mu) {
  double r = 0.0;
  if (isfinite(l)) r -= mu / (w - l);
  if (isfinite(b)) r += mu / (b - w);
  return r;
}

__global__ void k_sigmas(DevSym S, DevWork D) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nX = S.N * S.nx, nS = S.N * S.m;
  if (t < nX) {
    const int j = t % S.nx;
    D.Sx[t] = sigma_of(D.x[t], S.xl[j], S.xu[j], D.zlx[t], D.zux[t]);
  } else if (t < nX + nS) {
    const int q = t - nX, j = q % S.m;
    D.Ss[q] = sigma_of(D.s[q], S.sl[j], S.su[j], D.zls[q], D.zus[q]);
  } else if (t < nX + nS + S.nu) {
    const int j = t - nX - nS;
    D.Su[j] = sigma_of(D.u[j], S.ul[j], S.uu[j], D.zlu[j], D.zuu[j]);
  }
}

// K = W + Sigma_x + H^T Sigma_s H (+ the cost curvature (2 c2_0/N) dP0 dP0^T,
// which shares the P_0 row with the slack h row) on the KB pattern.
__global__ void k_condense(DevSym S, DevWork D) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.nnzKB * S.N) return;
  const int q = t / S.N, sc = t - q * S.N, N = S.N;
  const int a = S.kb_row[q], b = S.kb_col[q], as = S.kb_aslot[q];
  double k0 = 0, k1 = 0, k2 = 0, k3 = 0;
  if (as >= 0) {
    k0 = D.W[((size_t)as * 4 + 0) * N + sc];
    k1 = D.W[((size_t)as * 4 + 1) * N + sc];
    k2 = D.W[((size_t)as * 4 + 2) * N + sc];
    k3 = D.W[((size_t)as * 4 + 3) * N + sc];
  }
  for (int e = S.kbi_ptr[q]; e < S.kbi_ptr[q + 1]; ++e) {
    const int r = S.kbi_r[e], c = S.hrow_comp[r], ja = S.kbi_ja[e], jb = S.kbi_jb[e];
    double w = D.Ss[(size_t)sc * S.m + r];
    if (r == S.ng) w += 2.0 * S.c2[0] / N;
    double ha0, ha1, hb0, hb1;
    if (c < 2) {
      ha0 = D.J[((size_t)ja * 4 + c * 2 + 0) * N + sc];
      ha1 = D.J[((size_t)ja * 4 + c * 2 + 1) * N + sc];
      hb0 = D.J[((size_t)jb * 4 + c * 2 + 0) * N + sc];
      hb1 = D.J[((size_t)jb * 4 + c * 2 + 1) * N + sc];
    } else {  // line-flow row: ja, jb index HF
      ha0 = D.HF[((size_t)ja * 2 + 0) * N + sc];
      ha1 = D.HF[((size_t)ja * 2 + 1) * N + sc];
      hb0 = D.HF[((size_t)jb * 2 + 0) * N + sc];
      hb1 = D.HF[((size_t)jb * 2 + 1) * N + sc];
    }
    k0 += w * ha0 * hb0;
    k1 += w * ha0 * hb1;
    k2 += w * ha1 * hb0;
    k3 += w * ha1 * hb1;
  }
  if (a == b) {
    if (S.xth[a] >= 0) k0 += D.Sx[(size_t)sc * S.nx + S.xth[a]];
    if (S.xv[a] >= 0) k3 += D.Sx[(size_t)sc * S.nx + S.xv[a]];
  }
  D.K[((size_t)q * 4 + 0) * N + sc] = k0;
  D.K[((size_t)q * 4 + 1) * N + sc] = k1;
  D.K[((size_t)q * 4 + 2) * N + sc] = k2;
  D.K[((size_t)q * 4 + 3) * N + sc] = k3;
}

// slack rows: r2 = z - mu/(s-l) + mu/(b-s); r4 = h + s; t = Sigma_s r4 - r2
__global__ void k_rhs_s(DevSym S, DevWork D, const double *mu_d) {
  const double mu = *mu_d;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.N * S.m) return;
  const int j = t % S.m;
  const double r2 = D.z[t] + bgrad_of(D.s[t], S.sl[j], S.su[j], mu);
  const double r4 = D.h[t] + D.s[t];
  D.r2[t] = r2;
  D.r4[t] = r4;
  D.tv[t] = D.Ss[t] * r4 - r2;
}

// (H^T v) at bus variable (a, kind) of scenario sc
__device__ __forceinline__ double HT_at(const DevSym &S, const double *J, const double *HF, const double *v,
                                        int sc, int a, int kind) {
  double acc = 0.0;
  for (int e = S.ht_ptr[a]; e < S.ht_ptr[a + 1]; ++e) {
    const int r = S.ht_r[e], c = S.hrow_comp[r];
    const double hv = c < 2 ? J[((size_t)S.ht_aslot[e] * 4 + c * 2 + kind) * S.N + sc]
                            : HF[((size_t)S.ht_aslot[e] * 2 + kind) * S.N + sc];
    acc += v[(size_t)sc * S.m + r] * hv;
  }
  return acc;
}

// x rows: r1_x = grad f + G^T y + H^T z + barrier gradient; rhat1 = r1_x + H_x^T t
__global__ void k_rhs_x(DevSym S, DevWork D, const double *mu_d) {
  const double mu = *mu_d;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.N * S.nx) return;
  const int sc = t / S.nx, j = t - sc * S.nx;
  const int a = S.xbus[j], kind = S.xkind[j];
  const double r1 = D.JTl[(size_t)sc * 2 * S.n + kind * S.n + a] + bgrad_of(D.x[t], S.xl[j], S.xu[j], mu);
  D.r1x[t] = r1;
  D.rh1x[t] = r1 + HT_at(S, D.J, D.HF, D.tv, sc, a, kind);
}

// u gradient of sum_i (f_i + y_i^T g_i + z_i^T h_i), summed over scenarios in
// index order (first-stage coupling row of eq. (5)).
__global__ void k_ugrad(DevSym S, DevWork D, double *gLu, double *HTt_u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  double acc = 0.0, acc2 = 0.0;
  if (j < S.ng) {
    const int a = S.hrow_bus[j];
    for (int sc = 0; sc < S.N; ++sc) {
      acc += D.JTl[(size_t)sc * 2 * S.n + S.n + a];
      if (HTt_u) acc2 += HT_at(S, D.J, D.HF, D.tv, sc, a, 1);
    }
  } else {
    const int k = j - S.ng + 1, a = S.hrow_bus[k];
    const double pg = D.u[j];
    for (int sc = 0; sc < S.N; ++sc)
      acc += (2.0 * S.c2[k] * pg + S.c1[k]) / S.N - D.y[(size_t)sc * S.nx + S.xth[a]];
  }
  gLu[j] = acc;
  if (HTt_u) HTt_u[j] = acc2;
}

__global__ void k_rhs_u(DevSym S, DevWork D, const double *gLu, const double *HTt_u, const double *mu_d) {
  const double mu = *mu_d;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nu) return;
  const double r1 = gLu[j] + bgrad_of(D.u[j], S.ul[j], S.uu[j], mu);
  D.r1u[j] = r1;
  D.rh2[j] = r1 + HTt_u[j];
}

}  // namespace

// ---------------------------------------------------------------------------
static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

void launch_functions(const DevSym &S, const double *x, const double *u, double *P, double *Q,
                      double *g, double *h, double *fs, cudaStream_t st) {
  k_functions<<<nblk((long long)S.n * S.N, 128), 128, 0, st>>>(S, x, u, P, Q, g, h, fs); ipm_count_launch();
}
void launch_derivatives(const DevSym &S, DevWork &D, cudaStream_t st) {
  k_derivatives<<<nblk((long long)S.n * S.N, 128), 128, 0, st>>>(S, D.x, D.u, D.y, D.z, D.h, D.J, D.W, D.JTl, D.HF); ipm_count_launch();
}
void launch_sigmas(const DevSym &S, DevWork &D, cudaStream_t st) {
  long long tot = (long long)S.N * S.nx + (long long)S.N * S.m + S.nu;
  k_sigmas<<<nblk(tot, 256), 256, 0, st>>>(S, D); ipm_count_launch();
}
void launch_condense(const DevSym &S, DevWork &D, cudaStream_t st) {
  k_condense<<<nblk((long long)S.nnzKB * S.N, 128), 128, 0, st>>>(S, D); ipm_count_launch();
}
void launch_rhs(const DevSym &S, DevWork &D, const double *mu, double *gLu, double *HTt_u, cudaStream_t st) {
  k_rhs_s<<<nblk((long long)S.N * S.m, 256), 256, 0, st>>>(S, D, mu); ipm_count_launch();
  k_rhs_x<<<nblk((long long)S.N * S.nx, 256), 256, 0, st>>>(S, D, mu); ipm_count_launch();
  k_ugrad<<<nblk(S.nu, 64), 64, 0, st>>>(S, D, gLu, HTt_u); ipm_count_launch();
  k_rhs_u<<<nblk(S.nu, 64), 64, 0, st>>>(S, D, gLu, HTt_u, mu); ipm_count_launch();
}
void launch_ugrad(const DevSym &S, DevWork &D, double *gLu, cudaStream_t st) {
  k_ugrad<<<nblk(S.nu, 64), 64, 0, st>>>(S, D, gLu, nullptr); ipm_count_launch();
}
