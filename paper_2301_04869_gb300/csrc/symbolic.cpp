// Symbolic setup (S1): index maps, sparsity patterns, the fill-reducing
// ordering and static-pivot LU schedule of G_x shared by all scenarios.
//
// The paper factorizes G_x^{1:M} with a sparse LU that can run in batch
// because every scenario shares one sparsity pattern (§3.2, "Assembling the
// sparse matrices": P G_x Q = L U, G_x^{-1} b = Q U^{-1} L^{-1} P b).  Here
// P = Q^T is one symmetric permutation chosen once by minimum degree on the
// bus graph, with pivots on the diagonal (dP_i/dtheta_i, dQ_i/dv_i); the
// numeric factorization then replays a fixed, level-scheduled list of
// operations for every scenario.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <limits>
#include <map>
#include <set>
#include <unordered_map>

#include "ipm_internal.h"

namespace {

inline int64_t key2(int a, int b) { return (int64_t)a * 2147483647LL + b; }

// Minimum-degree elimination on an undirected graph (explicit elimination
// graph; ties broken by the smaller vertex index).  Returns the order and,
// for every vertex, its uneliminated neighbours at elimination (the
// structure of its L column).  Once the remaining graph is complete, the
// rest is appended in index order.
void min_degree(int nv, std::vector<std::vector<int>> adj, std::vector<int> &order,
                std::vector<std::vector<int>> &lpat) {
  order.clear();
  lpat.assign(nv, {});
  std::vector<char> done(nv, 0);
  std::set<std::pair<int, int>> pq;
  for (int v = 0; v < nv; ++v) {
    std::sort(adj[v].begin(), adj[v].end());
    adj[v].erase(std::unique(adj[v].begin(), adj[v].end()), adj[v].end());
    pq.insert({(int)adj[v].size(), v});
  }
  int remaining = nv;
  std::vector<int> tmp;
  while (remaining > 0) {
    auto it = pq.begin();
    int d = it->first, p = it->second;
    if (d == remaining - 1) {
      // remaining graph is a clique
      std::vector<int> rest;
      for (auto &e : pq) rest.push_back(e.second);
      std::sort(rest.begin(), rest.end());
      for (size_t i = 0; i < rest.size(); ++i) {
        order.push_back(rest[i]);
        lpat[rest[i]].assign(rest.begin() + i + 1, rest.end());
        done[rest[i]] = 1;
      }
      break;
    }
    pq.erase(it);
    done[p] = 1;
    order.push_back(p);
    const std::vector<int> nb = adj[p];
    lpat[p] = nb;
    for (int q : nb) {
      pq.erase({(int)adj[q].size(), q});
      tmp.clear();
      std::set_union(adj[q].begin(), adj[q].end(), nb.begin(), nb.end(), std::back_inserter(tmp));
      std::vector<int> nq;
      nq.reserve(tmp.size());
      for (int w : tmp)
        if (w != q && w != p) nq.push_back(w);
      adj[q].swap(nq);
      pq.insert({(int)adj[q].size(), q});
    }
    adj[p].clear();
    --remaining;
  }
}

}  // namespace

bool build_symbolic(const HostNet &net, int N, Sym &S, std::string &err, int big) {
  const int n = net.n, L = net.L, ng = net.ng;
  if (n < 2 || L < 1 || ng < 1 || N < 1) { err = "bad sizes"; return false; }
  if ((int)net.fr.size() != L || (int)net.to.size() != L || (int)net.gen.size() != ng) {
    err = "bad array sizes"; return false;
  }
  if (net.gen[0] != 0) { err = "gen_bus[0] must be 0 (slack)"; return false; }
  S.n = n; S.L = L; S.ng = ng; S.N = N;
  S.gen_of_bus.assign(n, -1);
  for (int k = 0; k < ng; ++k) {
    int g = net.gen[k];
    if (g < 0 || g >= n) { err = "gen_bus out of range"; return false; }
    if (S.gen_of_bus[g] >= 0) { err = "two generators on one bus"; return false; }
    S.gen_of_bus[g] = k;
  }
  if (!net.rate.empty() && (int)net.rate.size() != L) { err = "bad rate array size"; return false; }
  for (int l = 0; l < L; ++l) {
    int a = net.fr[l], b = net.to[l];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) { err = "bad line endpoints"; return false; }
    if (!net.rate.empty() && !(net.rate[l] > 0 && std::isfinite(net.rate[l]))) { err = "bad line rating"; return false; }
    double z2 = net.r[l] * net.r[l] + net.x[l] * net.x[l];
    if (!(z2 > 0) || !std::isfinite(z2) || !std::isfinite(net.b[l])) { err = "bad line impedance"; return false; }
  }
  // ---- variable maps ----
  S.xth.assign(n, -1); S.xv.assign(n, -1); S.uv.assign(n, -1);
  int nx = 0;
  for (int i = 1; i < n; ++i) S.xth[i] = nx++;
  for (int i = 0; i < n; ++i)
    if (S.gen_of_bus[i] < 0) S.xv[i] = nx++;
  S.nx = nx;
  S.nu = 2 * ng - 1;
  S.nflow = net.rate.empty() ? 0 : 2 * L;
  S.m = ng + 1 + S.nflow;
  for (int k = 0; k < ng; ++k) S.uv[net.gen[k]] = k;
  S.xbus.assign(nx, -1); S.xkind.assign(nx, -1);
  for (int i = 0; i < n; ++i) {
    if (S.xth[i] >= 0) { S.xbus[S.xth[i]] = i; S.xkind[S.xth[i]] = 0; }
    if (S.xv[i] >= 0) { S.xbus[S.xv[i]] = i; S.xkind[S.xv[i]] = 1; }
  }
  // ---- line parameters (pi model) ----
  S.lfr = net.fr; S.lto = net.to;
  S.lg.resize(L); S.lb.resize(L); S.lbh.resize(L);
  for (int l = 0; l < L; ++l) {
    double z2 = net.r[l] * net.r[l] + net.x[l] * net.x[l];
    S.lg[l] = net.r[l] / z2;
    S.lb[l] = -net.x[l] / z2;
    S.lbh[l] = 0.5 * net.b[l];
  }
  // ---- adjacency A (with diagonal) ----
  std::vector<std::vector<int>> nbr(n);
  {
    std::set<int64_t> seen;
    for (int l = 0; l < L; ++l) {
      int a = std::min(net.fr[l], net.to[l]), b = std::max(net.fr[l], net.to[l]);
      if (!seen.insert(key2(a, b)).second) { err = "duplicate (parallel) line"; return false; }
      nbr[a].push_back(b);
      nbr[b].push_back(a);
    }
  }
  S.a_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    std::vector<int> row = nbr[i];
    row.push_back(i);
    std::sort(row.begin(), row.end());
    S.a_ptr[i + 1] = S.a_ptr[i] + (int)row.size();
    for (int c : row) S.a_col.push_back(c);
  }
  S.nnzA = S.a_ptr[n];
  auto aslot = [&](int i, int k) -> int {
    auto b = S.a_col.begin() + S.a_ptr[i], e = S.a_col.begin() + S.a_ptr[i + 1];
    auto it = std::lower_bound(b, e, k);
    if (it == e || *it != k) return -1;
    return (int)(it - S.a_col.begin());
  };
  S.a_diag.resize(n);
  for (int i = 0; i < n; ++i) S.a_diag[i] = aslot(i, i);
  S.a_tslot.resize(S.nnzA);
  for (int i = 0; i < n; ++i)
    for (int q = S.a_ptr[i]; q < S.a_ptr[i + 1]; ++q) S.a_tslot[q] = aslot(S.a_col[q], i);
  // incidence lists
  S.inc_ptr.assign(n + 1, 0);
  {
    std::vector<std::vector<std::pair<int, int>>> inc(n);
    for (int l = 0; l < L; ++l) {
      inc[net.fr[l]].push_back({l, net.to[l]});
      inc[net.to[l]].push_back({l, net.fr[l]});
    }
    for (int i = 0; i < n; ++i) {
      S.inc_ptr[i + 1] = S.inc_ptr[i] + (int)inc[i].size();
      for (auto &p : inc[i]) {
        S.inc_line.push_back(p.first);
        S.inc_other.push_back(p.second);
        S.inc_aslot.push_back(aslot(i, p.second));
      }
    }
  }
  // ---- h rows: Qg of every generator, then Pg of the slack ----
  S.hrow_bus.resize(S.m); S.hrow_comp.resize(S.m);
  for (int k = 0; k < ng; ++k) { S.hrow_bus[k] = net.gen[k]; S.hrow_comp[k] = 1; }
  S.hrow_bus[ng] = 0; S.hrow_comp[ng] = 0;
  // line-flow rows (§4.1.1): |S|^2 at the from end of every line, then at the to end
  for (int f = 0; f < S.nflow; ++f) {
    const int l = f % L;
    S.hrow_bus[ng + 1 + f] = f < L ? net.fr[l] : net.to[l];
    S.hrow_comp[ng + 1 + f] = f < L ? 2 : 3;
  }
  // buses an h row depends on, and the H-value index of each: an injection
  // row touches the A row of its bus (index: the A slot), a flow row its two
  // end buses (index f * 2 + w, w = 0 own end, 1 other end)
  auto hrow_touch = [&](int r, std::vector<std::pair<int, int>> &tb) {
    tb.clear();
    if (r <= ng) {
      const int g = S.hrow_bus[r];
      for (int p = S.a_ptr[g]; p < S.a_ptr[g + 1]; ++p) tb.push_back({S.a_col[p], p});
    } else {
      const int f = r - ng - 1, l = f % L;
      const int own = f < L ? net.fr[l] : net.to[l], oth = f < L ? net.to[l] : net.fr[l];
      tb.push_back({own, f * 2 + 0});
      tb.push_back({oth, f * 2 + 1});
    }
  };
  std::vector<std::pair<int, int>> tb;
  // nbhd(g) = {g} u nbr(g), i.e. A row g
  // ---- KB pattern ----
  std::vector<std::map<int, std::vector<int>>> kb(n);  // row bus -> col bus -> h rows
  for (int i = 0; i < n; ++i)
    for (int p = S.a_ptr[i]; p < S.a_ptr[i + 1]; ++p) kb[i][S.a_col[p]];
  for (int r = 0; r < S.m; ++r) {
    hrow_touch(r, tb);
    for (auto &pa : tb)
      for (auto &pb : tb) kb[pa.first][pb.first].push_back(r);
  }
  S.kb_ptr.assign(n + 1, 0);
  S.kbi_ptr.push_back(0);
  for (int i = 0; i < n; ++i) {
    for (auto &kv : kb[i]) {
      int j = kv.first;
      S.kb_col.push_back(j);
      S.kb_row.push_back(i);
      S.kb_aslot.push_back(aslot(i, j));
      for (int r : kv.second) {
        hrow_touch(r, tb);
        int ja = -1, jb = -1;
        for (auto &pa : tb) {
          if (pa.first == i) ja = pa.second;
          if (pa.first == j) jb = pa.second;
        }
        S.kbi_r.push_back(r);
        S.kbi_ja.push_back(ja);
        S.kbi_jb.push_back(jb);
      }
      S.kbi_ptr.push_back((int)S.kbi_r.size());
    }
    S.kb_ptr[i + 1] = (int)S.kb_col.size();
  }
  S.nnzKB = (int)S.kb_col.size();
  auto kbslot = [&](int i, int k) -> int {
    auto b = S.kb_col.begin() + S.kb_ptr[i], e = S.kb_col.begin() + S.kb_ptr[i + 1];
    auto it = std::lower_bound(b, e, k);
    if (it == e || *it != k) return -1;
    return (int)(it - S.kb_col.begin());
  };
  // H^T lists per bus
  {
    std::vector<std::vector<std::pair<int, int>>> ht(n);
    for (int r = 0; r < S.m; ++r) {
      hrow_touch(r, tb);
      for (auto &pa : tb) ht[pa.first].push_back({r, pa.second});
    }
    S.ht_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      S.ht_ptr[i + 1] = S.ht_ptr[i] + (int)ht[i].size();
      for (auto &p : ht[i]) { S.ht_r.push_back(p.first); S.ht_aslot.push_back(p.second); }
    }
  }
  // ---- ordering: minimum degree on buses 1..n-1 ----
  std::vector<std::vector<int>> badj(n - 1);
  for (int i = 1; i < n; ++i)
    for (int k : nbr[i])
      if (k != 0) badj[i - 1].push_back(k - 1);
  std::vector<int> border;
  std::vector<std::vector<int>> blpat;
  min_degree(n - 1, badj, border, blpat);
  // x positions: theta then v of each bus, in elimination order
  S.perm.assign(nx, -1);
  S.iperm.assign(nx, -1);
  std::vector<int> bus_pos0(n, -1);
  {
    int pos = 0;
    for (int bb : border) {
      int i = bb + 1;
      bus_pos0[i] = pos;
      if (S.xth[i] >= 0) { S.perm[S.xth[i]] = pos; S.iperm[pos] = S.xth[i]; ++pos; }
      if (S.xv[i] >= 0) { S.perm[S.xv[i]] = pos; S.iperm[pos] = S.xv[i]; ++pos; }
    }
    if (pos != nx) { err = "internal: ordering size"; return false; }
  }
  // x-level pattern of L columns (rows below the pivot), sorted
  std::vector<std::vector<int>> pat(nx);
  for (int bb : border) {
    int i = bb + 1;
    std::vector<int> rows;
    for (int q : blpat[bb]) {
      int qb = q + 1;
      if (S.xth[qb] >= 0) rows.push_back(S.perm[S.xth[qb]]);
      if (S.xv[qb] >= 0) rows.push_back(S.perm[S.xv[qb]]);
    }
    std::sort(rows.begin(), rows.end());
    int pth = S.perm[S.xth[i]];
    if (S.xv[i] >= 0) {
      int pv = S.perm[S.xv[i]];
      pat[pth].push_back(pv);
      for (int r : rows) pat[pth].push_back(r);
      pat[pv] = rows;
    } else {
      pat[pth] = rows;
    }
  }
  // ---- levels: lev(p) = 1 + max over pivots k with p in pat(k) ----
  // (computed on the minimum-degree pattern; a widened trailing block below
  // only adds fill inside itself, which the dense kernels handle)
  std::vector<int> lev(nx, 0), blev(nx, 0);
  for (int k = 0; k < nx; ++k)
    for (int p : pat[k]) lev[p] = std::max(lev[p], lev[k] + 1);
  for (int i = nx - 1; i >= 0; --i)
    for (int k : pat[i]) blev[i] = std::max(blev[i], blev[k] + 1);
  int nlev = 0, nlevb = 0;
  for (int k = 0; k < nx; ++k) { nlev = std::max(nlev, lev[k] + 1); nlevb = std::max(nlevb, blev[k] + 1); }
  S.nlev = nlev; S.nlev_b = nlevb;
  // dense trailing block: the largest suffix [t0, nx) whose L columns are full
  int t0 = nx;
  while (t0 > 0 && (int)pat[t0 - 1].size() == nx - t0) --t0;
  if (nx - t0 < 2) t0 = nx;  // nothing worth a dense phase
  // A large trailing block goes to the global-memory kernels.  The sparse
  // pivots just before it that reach a sizable part of it (a few hundred on
  // the 10,000-bus networks, each coupled to most of the block) then join it:
  // their products into the block become part of its dense factorization
  // instead of millions of gather operations.
  S.big = (nx - t0) > 0 && (big != 0 || nx - t0 > BIG_ND);
  if (S.big) {
    const int nd0 = nx - t0, thr = std::max(8, nd0 / 6);
    int tp = t0;
    for (int k = 0; k < t0; ++k) {
      int ck = 0;
      for (int i : pat[k]) ck += i >= t0;
      if (ck >= thr) { tp = k; break; }
    }
    for (int k = tp; k < nx; ++k) {
      pat[k].clear();
      for (int i = k + 1; i < nx; ++i) pat[k].push_back(i);
    }
    t0 = tp;
  }
  S.t0 = t0;
  S.nd = nx - t0;
  const int nd = S.nd;
  // ---- LU pattern (CSC by position): U part, diagonal, L part ----
  std::vector<std::vector<int>> ucols(nx);  // rows r < c with U(r,c) != 0
  for (int r = 0; r < nx; ++r)
    for (int c : pat[r]) ucols[c].push_back(r);
  S.lu_colptr.assign(nx + 1, 0);
  std::vector<int> diag_at(nx, -1);
  for (int c = 0; c < nx; ++c) {
    for (int r : ucols[c]) S.lu_row.push_back(r);
    diag_at[c] = (int)S.lu_row.size();
    S.lu_row.push_back(c);
    for (int r : pat[c]) S.lu_row.push_back(r);
    S.lu_colptr[c + 1] = (int)S.lu_row.size();
  }
  // storage slots: entries outside the trailing block first, then the block
  S.lu_slot.assign(S.lu_row.size(), -1);
  {
    int q = 0;
    for (int c = 0; c < nx; ++c)
      for (int p = S.lu_colptr[c]; p < S.lu_colptr[c + 1]; ++p)
        if (!(c >= t0 && S.lu_row[p] >= t0)) S.lu_slot[p] = q++;
    S.dense_base = (q + 3) / 4 * 4;
    for (int c = t0; c < nx; ++c)
      for (int p = S.lu_colptr[c]; p < S.lu_colptr[c + 1]; ++p)
        if (S.lu_row[p] >= t0) S.lu_slot[p] = S.dense_base + (c - t0) * nd + (S.lu_row[p] - t0);
    S.nnzLU = (int)(((long long)S.dense_base + (long long)nd * nd + 3) / 4 * 4);
  }
  S.lu_diag.assign(nx, -1);
  for (int c = 0; c < nx; ++c) S.lu_diag[c] = S.lu_slot[diag_at[c]];
  auto luslot = [&](int r, int c) -> int {
    if (r >= t0 && c >= t0) return S.dense_base + (c - t0) * nd + (r - t0);
    auto b = S.lu_row.begin() + S.lu_colptr[c];
    auto e = S.lu_row.begin() + S.lu_colptr[c + 1];
    // U part sorted, then diag, then L part sorted; rows < c precede c
    if (r < c) {
      auto ee = S.lu_row.begin() + diag_at[c];
      auto it = std::lower_bound(b, ee, r);
      if (it == ee || *it != r) return -1;
      return S.lu_slot[it - S.lu_row.begin()];
    }
    if (r == c) return S.lu_diag[c];
    auto bb = S.lu_row.begin() + diag_at[c] + 1;
    auto it = std::lower_bound(bb, e, r);
    if (it == e || *it != r) return -1;
    return S.lu_slot[it - S.lu_row.begin()];
  };
  // row and column of every slot (-1 for padding)
  std::vector<int> slot_row(S.nnzLU, -1), slot_col(S.nnzLU, -1);
  for (int c = 0; c < nx; ++c)
    for (int p = S.lu_colptr[c]; p < S.lu_colptr[c + 1]; ++p) {
      slot_row[S.lu_slot[p]] = S.lu_row[p];
      slot_col[S.lu_slot[p]] = c;
    }
  // initial values: G_x entry = J[aslot(bus_r, bus_c)][kind_r*2 + kind_c]
  S.lu_init.assign(S.nnzLU, -1);
  for (int c = 0; c < nx; ++c) {
    int xc = S.iperm[c];
    int bc = S.xbus[xc], kc = S.xkind[xc];
    for (int p = S.lu_colptr[c]; p < S.lu_colptr[c + 1]; ++p) {
      int xr = S.iperm[S.lu_row[p]];
      int br = S.xbus[xr], kr = S.xkind[xr];
      int a = aslot(br, bc);
      if (a >= 0) S.lu_init[S.lu_slot[p]] = a * 4 + kr * 2 + kc;
    }
  }
  S.tail_slot.assign((size_t)S.nd * S.nd, -1);
  for (int a = 0; a < S.nd; ++a)
    for (int b = 0; b < S.nd; ++b) S.tail_slot[(size_t)a * S.nd + b] = luslot(t0 + a, t0 + b);
  // factorization levels of the sparse pivots only (the trailing block is
  // factorized densely afterwards; sparse pivots never depend on it)
  int nlevf = 0;
  for (int k = 0; k < t0; ++k) nlevf = std::max(nlevf, lev[k] + 1);
  S.nlev_f = nlevf;
  std::vector<std::vector<int>> piv_of_lev(nlevf);
  for (int k = 0; k < t0; ++k) piv_of_lev[lev[k]].push_back(k);
  S.f_lev_ptr.assign(nlevf + 1, 0);
  S.f_piv_ptr.assign(nlevf + 1, 0);
  for (int l = 0; l < nlevf; ++l) {
    for (int k : piv_of_lev[l]) S.f_piv.push_back(k);
    S.f_piv_ptr[l + 1] = (int)S.f_piv.size();
  }
  S.f_op_ptr.push_back(0);
  // updates of the dense trailing block by the sparse pivots (L(i,k) U(k,j),
  // i, j >= t0, k < t0) are kept out of the level lists: per trailing-block
  // entry, all its products, applied after the sparse phase (see below)
  struct TailOp { int t, k, l, u; };
  std::vector<TailOp> tail_ops;
  std::vector<std::pair<int, int>> tk;  // (target slot, pivot) of one level
  for (int l = 0; l < nlevf; ++l) {
    tk.clear();
    for (int k : piv_of_lev[l])
      for (int i : pat[k])
        for (int j : pat[k]) {
          const int t = luslot(i, j);
          if (t < 0) { err = "internal: fill pattern not closed"; return false; }
          if (i >= t0 && j >= t0) tail_ops.push_back({t, k, luslot(i, k), luslot(k, j)});
          else tk.push_back({t, k});
        }
    std::sort(tk.begin(), tk.end());
    for (size_t e = 0; e < tk.size();) {
      const int t = tk[e].first, i = slot_row[t], j = slot_col[t];
      S.f_tgt.push_back(t);
      for (; e < tk.size() && tk[e].first == t; ++e) {
        const int k = tk[e].second;
        S.f_op_l.push_back(luslot(i, k));
        S.f_op_u.push_back(luslot(k, j));
        S.f_op_k.push_back(k);
      }
      S.f_op_ptr.push_back((int)S.f_op_l.size());
    }
    S.f_lev_ptr[l + 1] = (int)S.f_tgt.size();
  }
  S.n_ops = (long long)S.f_op_l.size();
  for (int k = 0; k < t0; ++k)
    for (int i : pat[k]) { S.lsc_slot.push_back(luslot(i, k)); S.lsc_k.push_back(k); }
  // Trailing-block products in LU_LISTS lists (one per thread of a
  // two-CTA cluster): entries dealt to the least-loaded list, longest first;
  // op s of list t at s * LU_LISTS + t (coalesced); tw_e names the entry
  // slot after its last product, else -1.
  {
    std::sort(tail_ops.begin(), tail_ops.end(),
              [](const TailOp &a, const TailOp &b) { return a.t != b.t ? a.t < b.t : a.k < b.k; });
    std::vector<std::array<int, 3>> ents;  // (op count, slot, first op)
    for (size_t e = 0; e < tail_ops.size();) {
      size_t f = e;
      while (f < tail_ops.size() && tail_ops[f].t == tail_ops[e].t) ++f;
      ents.push_back({(int)(f - e), tail_ops[e].t, (int)e});
      e = f;
    }
    std::sort(ents.begin(), ents.end(), [](const std::array<int, 3> &a, const std::array<int, 3> &b) {
      return a[0] != b[0] ? a[0] > b[0] : a[1] < b[1];
    });
    std::vector<std::vector<int>> own(LU_LISTS);  // entries (index into ents) per list
    std::vector<long long> load(LU_LISTS, 0);
    // least-loaded list first (ties: the lower list)
    std::set<std::pair<long long, int>> heap;
    for (int q = 0; q < LU_LISTS; ++q) heap.insert({0LL, q});
    for (size_t e = 0; e < ents.size(); ++e) {
      const auto top = *heap.begin();
      heap.erase(heap.begin());
      own[top.second].push_back((int)e);
      heap.insert({top.first + ents[e][0], top.second});
      load[top.second] += ents[e][0];
    }
    long long M = 0;
    for (int q = 0; q < LU_LISTS; ++q) M = std::max(M, load[q]);
    S.tw_len.assign(LU_LISTS, 0);
    S.tw_l.assign((size_t)M * LU_LISTS, 0);
    S.tw_u.assign((size_t)M * LU_LISTS, 0);
    S.tw_e.assign((size_t)M * LU_LISTS, -1);
    for (int q = 0; q < LU_LISTS; ++q) {
      int s_ = 0;
      for (int ei : own[q]) {
        const auto &en = ents[ei];
        for (int o = 0; o < en[0]; ++o, ++s_) {
          const size_t at = (size_t)s_ * LU_LISTS + q;
          const TailOp &op = tail_ops[(size_t)en[2] + o];
          S.tw_l[at] = op.l;
          S.tw_u[at] = op.u;
          if (o + 1 == en[0]) S.tw_e[at] = en[1];
        }
      }
      S.tw_len[q] = s_;
    }
    S.n_tail_ops = (long long)tail_ops.size();
  }
  // forward rows (L rows, k < i) with the matching U(k,i) slots
  {
    std::vector<std::vector<int>> frow(nx);
    for (int k = 0; k < nx; ++k)
      for (int i : pat[k]) frow[i].push_back(k);
    S.fr_ptr.assign(nx + 1, 0);
    for (int i = 0; i < nx; ++i) {
      for (int k : frow[i]) {
        S.fr_col.push_back(k);
        S.fr_lslot.push_back(luslot(i, k));
        S.fr_uslot.push_back(luslot(k, i));
      }
      S.fr_ptr[i + 1] = (int)S.fr_col.size();
    }
    S.br_ptr.assign(nx + 1, 0);
    for (int i = 0; i < nx; ++i) {
      for (int k : pat[i]) {
        S.br_col.push_back(k);
        S.br_uslot.push_back(luslot(i, k));
        S.br_lslot.push_back(luslot(k, i));
      }
      S.br_ptr[i + 1] = (int)S.br_col.size();
    }
    std::vector<std::vector<int>> fl(nlev), bl(nlevb);
    for (int i = 0; i < nx; ++i) { fl[lev[i]].push_back(i); bl[blev[i]].push_back(i); }
    S.fw_lev_ptr.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
      for (int i : fl[l]) S.fw_rows.push_back(i);
      S.fw_lev_ptr[l + 1] = (int)S.fw_rows.size();
    }
    S.bw_lev_ptr.assign(nlevb + 1, 0);
    for (int l = 0; l < nlevb; ++l) {
      for (int i : bl[l]) S.bw_rows.push_back(i);
      S.bw_lev_ptr[l + 1] = (int)S.bw_rows.size();
    }
    // the same schedules over the sparse rows only (the dense trailing block
    // [t0, nx) is solved separately); empty levels dropped
    S.fs_lev_ptr.assign(1, 0);
    for (int l = 0; l < nlev; ++l) {
      bool any = false;
      for (int i : fl[l])
        if (i < S.t0) { S.fs_rows.push_back(i); any = true; }
      if (any) S.fs_lev_ptr.push_back((int)S.fs_rows.size());
    }
    S.nlev_fs = (int)S.fs_lev_ptr.size() - 1;
    S.bs_lev_ptr.assign(1, 0);
    for (int l = 0; l < nlevb; ++l) {
      bool any = false;
      for (int i : bl[l])
        if (i < S.t0) { S.bs_rows.push_back(i); any = true; }
      if (any) S.bs_lev_ptr.push_back((int)S.bs_rows.size());
    }
    S.nlev_bs = (int)S.bs_lev_ptr.size() - 1;
    for (int i : S.fs_rows) S.fs4.insert(S.fs4.end(), {i, S.fr_ptr[i], S.fr_ptr[i + 1], 0});
    for (int i : S.bs_rows) S.bs4.insert(S.bs4.end(), {i, S.br_ptr[i], S.br_ptr[i + 1], 0});
    for (size_t f = 0; f < S.fr_col.size(); ++f) S.fr4.insert(S.fr4.end(), {S.fr_col[f], S.fr_lslot[f], S.fr_uslot[f], 0});
    for (size_t f = 0; f < S.br_col.size(); ++f) S.br4.insert(S.br4.end(), {S.br_col[f], S.br_uslot[f], S.br_lslot[f], 0});
  }
  // ---- G_u (rows: positions) and its transpose (rows: u) ----
  const int nu = S.nu;
  {
    std::vector<std::vector<std::pair<int, int>>> gut(nu);
    S.gu_ptr.assign(nx + 1, 0);
    for (int p = 0; p < nx; ++p) {
      int xi = S.iperm[p];
      int a = S.xbus[xi], ka = S.xkind[xi];
      std::vector<std::pair<int, int>> row;
      for (int q = S.a_ptr[a]; q < S.a_ptr[a + 1]; ++q) {
        int b = S.a_col[q];
        if (S.uv[b] >= 0) row.push_back({S.uv[b], q * 4 + ka * 2 + 1});
      }
      if (ka == 0 && S.gen_of_bus[a] >= 1) row.push_back({ng + S.gen_of_bus[a] - 1, -1});
      std::sort(row.begin(), row.end());
      for (auto &e : row) {
        S.gu_col.push_back(e.first);
        S.gu_src.push_back(e.second);
        gut[e.first].push_back({p, e.second});
      }
      S.gu_ptr[p + 1] = (int)S.gu_col.size();
    }
    S.gut_ptr.assign(nu + 1, 0);
    for (int j = 0; j < nu; ++j) {
      for (auto &e : gut[j]) { S.gut_col.push_back(e.first); S.gut_src.push_back(e.second); }
      S.gut_ptr[j + 1] = (int)S.gut_col.size();
    }
  }
  // ---- forward schedules per 32-column panel of the multi-RHS solve ----
  // A column of G_u reaches few rows of the forward sweep L^{-1} G_u: row i
  // is structurally nonzero for a panel iff G_u has an entry of a panel
  // column in row i, or L(i, k) != 0 for a nonzero row k < i.  Panels
  // 0 .. ceil(n_u/32) - 1 hold the columns of Z; the last one holds
  // b = G_x^{-1} g alone and keeps every row.
  // Per panel: the nonzero sparse rows by level of the reduced sweep with
  // their products against nonzero rows only, the zero rows, and for each
  // trailing-block row its products against nonzero sparse rows.
  {
    const int np = (nu + 31) / 32 + 1, t0 = S.t0, nd = S.nd;
    S.zp_npan = np;
    S.zp_lev_off.assign(1, 0);
    S.zp_lev_ptr.assign(1, 0);
    S.zp_eptr.assign(1, 0);
    S.zp_zptr.assign(1, 0);
    S.zp_tptr.assign(1, 0);
    std::vector<char> nz(nx);
    std::vector<int> zl(nx);
    for (int p = 0; p < np; ++p) {
      const int c0 = 32 * p, c1 = std::min(32 * p + 32, nu);
      const bool all = p == np - 1;  // the panel of b
      int nl = 0;
      for (int i = 0; i < t0; ++i) {
        bool z = all;
        for (int g = S.gu_ptr[i]; !z && g < S.gu_ptr[i + 1]; ++g) z = S.gu_col[g] >= c0 && S.gu_col[g] < c1;
        int lv = 0;
        for (int f = S.fr_ptr[i]; f < S.fr_ptr[i + 1]; ++f) {
          const int k = S.fr_col[f];
          if (nz[k]) { z = true; lv = std::max(lv, zl[k] + 1); }
        }
        nz[i] = z;
        zl[i] = lv;
        if (z) nl = std::max(nl, lv + 1);
      }
      std::vector<std::vector<int>> byl(nl);
      for (int i = 0; i < t0; ++i) {
        if (nz[i]) byl[zl[i]].push_back(i);
        else S.zp_zrows.push_back(i);
      }
      S.zp_zptr.push_back((int)S.zp_zrows.size());
      for (int l = 0; l < nl; ++l) {
        for (int i : byl[l]) {
          S.zp_rows.push_back(i);
          for (int f = S.fr_ptr[i]; f < S.fr_ptr[i + 1]; ++f)
            if (nz[S.fr_col[f]]) { S.zp_col.push_back(S.fr_col[f]); S.zp_slot.push_back(S.fr_lslot[f]); }
          S.zp_eptr.push_back((int)S.zp_col.size());
        }
        S.zp_lev_ptr.push_back((int)S.zp_rows.size());
      }
      S.zp_lev_off.push_back(S.zp_lev_off.back() + nl);
      for (int a = 0; a < nd; ++a) {
        const int i = t0 + a;
        for (int f = S.fr_ptr[i]; f < S.fr_ptr[i + 1] && S.fr_col[f] < t0; ++f)
          if (nz[S.fr_col[f]]) { S.zp_tcol.push_back(S.fr_col[f]); S.zp_tslot.push_back(S.fr_lslot[f]); }
        S.zp_tptr.push_back((int)S.zp_tcol.size());
      }
    }
  }
  // ---- K_x (rows: positions) and K_u (rows: u) ----
  auto var_col = [&](int b, int kind) -> int {  // column id: position or nx + u
    if (kind == 0) return S.xth[b] >= 0 ? S.perm[S.xth[b]] : -1;
    if (S.xv[b] >= 0) return S.perm[S.xv[b]];
    return nx + S.uv[b];
  };
  S.kx_ptr.assign(nx + 1, 0);
  for (int p = 0; p < nx; ++p) {
    int xi = S.iperm[p];
    int a = S.xbus[xi], ka = S.xkind[xi];
    std::vector<std::pair<int, int>> row;
    for (int q = S.kb_ptr[a]; q < S.kb_ptr[a + 1]; ++q) {
      int b = S.kb_col[q];
      for (int kb2 = 0; kb2 < 2; ++kb2) {
        int c = var_col(b, kb2);
        if (c >= 0) row.push_back({c, q * 4 + ka * 2 + kb2});
      }
    }
    std::sort(row.begin(), row.end());
    for (auto &e : row) { S.kx_col.push_back(e.first); S.kx_src.push_back(e.second); }
    S.kx_ptr[p + 1] = (int)S.kx_col.size();
  }
  S.ku_ptr.assign(nu + 1, 0);
  for (int j = 0; j < nu; ++j) {
    std::vector<std::pair<int, int>> row;
    if (j < ng) {
      int a = net.gen[j];
      for (int q = S.kb_ptr[a]; q < S.kb_ptr[a + 1]; ++q) {
        int b = S.kb_col[q];
        for (int kb2 = 0; kb2 < 2; ++kb2) {
          int c = var_col(b, kb2);
          if (c >= 0) row.push_back({c, q * 4 + 1 * 2 + kb2});
        }
      }
    }
    std::sort(row.begin(), row.end());
    for (auto &e : row) { S.ku_col.push_back(e.first); S.ku_src.push_back(e.second); }
    S.ku_ptr[j + 1] = (int)S.ku_col.size();
  }
  (void)kbslot;
  // ---- bounds ----
  const double inf = std::numeric_limits<double>::infinity();
  S.xl.assign(nx, -inf); S.xu.assign(nx, inf);
  for (int i = 0; i < n; ++i)
    if (S.xv[i] >= 0) { S.xl[S.xv[i]] = net.vmin[i]; S.xu[S.xv[i]] = net.vmax[i]; }
  S.ul.assign(nu, 0.0); S.uu.assign(nu, 0.0);
  for (int k = 0; k < ng; ++k) { S.ul[k] = net.vmin[net.gen[k]]; S.uu[k] = net.vmax[net.gen[k]]; }
  for (int k = 1; k < ng; ++k) { S.ul[ng + k - 1] = 0.0; S.uu[ng + k - 1] = net.pmax[k]; }
  S.sl.assign(S.m, 0.0); S.su.assign(S.m, 0.0);
  for (int k = 0; k < ng; ++k) { S.sl[k] = -net.qmax[k]; S.su[k] = net.qmax[k]; }
  S.sl[ng] = -net.pmax[0]; S.su[ng] = -0.0;
  // flow rows: h = |S|^2 <= rate^2 only, so s = -h in [-rate^2, +inf)
  for (int f = 0; f < S.nflow; ++f) {
    const double rt = net.rate[f % L];
    S.sl[ng + 1 + f] = -rt * rt;
    S.su[ng + 1 + f] = inf;
  }
  S.c2 = net.c2; S.c1 = net.c1; S.pmax = net.pmax; S.qmax = net.qmax;
  return true;
}
