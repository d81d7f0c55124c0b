// Symbolic analysis of the fixed pattern of G_k (host, once per circuit).
//
// The paper factors G_k once per time step and never C or C/h + G (Alg. 2, Sec. IV-A);
// the pattern of G_k = G_lin + G_dev(x_k) is fixed by the netlist, so everything that
// depends only on the pattern is computed here:
//   1. fill-reducing ordering: nested dissection with level-structure vertex separators
//      (George's method) on the symmetrised pattern, exact minimum degree on small parts;
//   2. elimination tree (Liu), postorder, column counts by row subtrees;
//   3. fundamental supernodes (width-capped) and their row structures;
//   4. the multifrontal refactor plan (front arena, assembly/extend-add maps, tiles);
//   5. the task lists of the warp-granular sync-free triangular solves.
#include "symbolic.h"

#include <algorithm>
#include <functional>
#include <climits>
#include <map>
#include <set>
#include <cstring>
#include <numeric>

namespace ers {
namespace {

struct Graph {  // symmetric adjacency without the diagonal
  int n = 0;
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
};

Graph symmetrize(int n, const int32_t* ptr, const int32_t* idx) {
  std::vector<int64_t> cnt(n + 1, 0);
  for (int i = 0; i < n; ++i)
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) {
      int j = idx[e];
      if (j == i) continue;
      cnt[i + 1]++;
      cnt[j + 1]++;
    }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int32_t> tmp(cnt[n]);
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) {
      int j = idx[e];
      if (j == i) continue;
      tmp[pos[i]++] = j;
      tmp[pos[j]++] = i;
    }
  Graph g;
  g.n = n;
  g.xadj.assign(n + 1, 0);
  g.adj.reserve(tmp.size());
  for (int i = 0; i < n; ++i) {
    std::sort(tmp.begin() + cnt[i], tmp.begin() + cnt[i + 1]);
    int last = -1;
    for (int64_t e = cnt[i]; e < cnt[i + 1]; ++e)
      if (tmp[e] != last) { g.adj.push_back(tmp[e]); last = tmp[e]; }
    g.xadj[i + 1] = (int64_t)g.adj.size();
  }
  return g;
}

// ---- nested dissection --------------------------------------------------------------
class Dissector {
 public:
  Dissector(const Graph& g, int leaf, int window_pct, int roots)
      : g_(g), leaf_(leaf), window_pct_(window_pct), roots_(roots), mark_(g.n, -1),
        lev_(g.n, -1), loc_(g.n, -1) {}

  // returns new -> old
  std::vector<int32_t> run() {
    int n = g_.n;
    buf_.resize(n);
    std::iota(buf_.begin(), buf_.end(), 0);
    std::vector<std::pair<int, int>> stack;
    if (n) stack.push_back({0, n});
    while (!stack.empty()) {
      auto [lo, hi] = stack.back();
      stack.pop_back();
      split(lo, hi, stack);
    }
    return buf_;
  }

 private:
  const Graph& g_;
  int leaf_, window_pct_, roots_;
  std::vector<int32_t> buf_, mark_, lev_, loc_;
  int stamp_ = 0;
  std::vector<int32_t> queue_, tmp_;

  void stamp_range(int lo, int hi) {
    ++stamp_;
    for (int k = lo; k < hi; ++k) mark_[buf_[k]] = stamp_;
  }

  // BFS inside the stamped part; fills lev_ and returns (#levels, last vertex visited)
  int bfs(int root, int& far) {
    queue_.clear();
    queue_.push_back(root);
    lev_[root] = 0;
    mark_[root] = -stamp_;  // visited marker: negative stamp
    size_t h = 0;
    int maxl = 0;
    while (h < queue_.size()) {
      int v = queue_[h++];
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int u = g_.adj[e];
        if (mark_[u] == stamp_) {
          mark_[u] = -stamp_;
          lev_[u] = lev_[v] + 1;
          maxl = std::max(maxl, lev_[u]);
          queue_.push_back(u);
        }
      }
    }
    far = queue_.back();
    return maxl + 1;
  }

  void unvisit() {
    for (int v : queue_) mark_[v] = stamp_;
  }

  int degree_in_part(int v) {
    int d = 0;
    for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
      int u = g_.adj[e];
      if (mark_[u] == stamp_ || mark_[u] == -stamp_) ++d;
    }
    return d;
  }

  void min_degree(int lo, int hi) {
    // exact minimum degree on the induced subgraph (<= 64 vertices) with bit masks
    int m = hi - lo;
    uint64_t adjm[64];
    for (int a = 0; a < m; ++a) loc_[buf_[lo + a]] = a;
    for (int a = 0; a < m; ++a) {
      int v = buf_[lo + a];
      uint64_t mk = 0;
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int u = g_.adj[e];
        if (mark_[u] == stamp_) mk |= (uint64_t)1 << loc_[u];
      }
      adjm[a] = mk;
    }
    uint64_t alive = (m == 64) ? ~(uint64_t)0 : (((uint64_t)1 << m) - 1);
    tmp_.assign(m, 0);
    for (int step = 0; step < m; ++step) {
      int best = -1, bd = 1 << 30;
      for (int a = 0; a < m; ++a)
        if (alive >> a & 1) {
          int d = __builtin_popcountll(adjm[a] & alive);
          if (d < bd) { bd = d; best = a; }
        }
      uint64_t nb = adjm[best] & alive & ~((uint64_t)1 << best);
      for (int a = 0; a < m; ++a)
        if (nb >> a & 1) adjm[a] |= nb & ~((uint64_t)1 << a);
      alive &= ~((uint64_t)1 << best);
      tmp_[step] = buf_[lo + best];
    }
    for (int a = 0; a < m; ++a) {
      buf_[lo + a] = tmp_[a];
      loc_[tmp_[a]] = -1;
    }
  }

  void by_degree(int lo, int hi) {
    // fallback for parts of diameter < 3: low degree first, high degree last
    std::vector<std::pair<int, int>> dv;
    for (int k = lo; k < hi; ++k) dv.push_back({degree_in_part(buf_[k]), buf_[k]});
    std::sort(dv.begin(), dv.end());
    for (int k = lo; k < hi; ++k) buf_[k] = dv[k - lo].second;
  }

  // Separator level of a BFS level structure with cnt[l] vertices on level l: the level where
  // the cumulative count crosses half, or (window_pct_ > 0) the smallest level that leaves at
  // least (50 - window_pct_)% of the part on each side (ties: the first).
  int separator_level(const std::vector<int>& cnt, int size) const {
    int nlev = (int)cnt.size();
    int k = 1, acc = cnt[0];
    while (k < nlev - 1 && acc + cnt[k] <= size / 2) { acc += cnt[k]; ++k; }
    if (k >= nlev - 1) k = nlev - 2;
    if (window_pct_ <= 0) return k;
    int best = -1;
    int64_t below = cnt[0];
    const int64_t need = (int64_t)(50 - window_pct_) * size;
    for (int j = 1; j < nlev - 1; ++j) {
      int64_t above = size - below - cnt[j];
      if (100 * below >= need && 100 * above >= need && (best < 0 || cnt[j] < cnt[best])) best = j;
      below += cnt[j];
    }
    return best >= 0 ? best : k;
  }

  void split(int lo, int hi, std::vector<std::pair<int, int>>& stack) {
    int size = hi - lo;
    stamp_range(lo, hi);
    if (size <= leaf_ && size <= 64) {
      min_degree(lo, hi);
      return;
    }
    // connected components
    int far;
    bfs(buf_[lo], far);
    if ((int)queue_.size() < size) {
      // label all components, regroup the range component by component
      std::vector<int32_t> comp_vertices;
      comp_vertices.reserve(size);
      std::vector<int> bounds{0};
      for (int v : queue_) comp_vertices.push_back(v);
      bounds.push_back((int)comp_vertices.size());
      for (int k = lo; k < hi; ++k) {
        int v = buf_[k];
        if (mark_[v] == stamp_) {
          bfs(v, far);
          for (int u : queue_) comp_vertices.push_back(u);
          bounds.push_back((int)comp_vertices.size());
        }
      }
      std::copy(comp_vertices.begin(), comp_vertices.end(), buf_.begin() + lo);
      for (size_t c = 0; c + 1 < bounds.size(); ++c)
        stack.push_back({lo + bounds[c], lo + bounds[c + 1]});
      return;
    }
    // pseudo-peripheral root
    int root = buf_[lo];
    unvisit();
    int nlev = bfs(root, far);
    for (int it = 0; it < 5; ++it) {
      // candidate: minimum-degree vertex of the last level
      int cand = far, cd = 1 << 30;
      for (int v : queue_)
        if (lev_[v] == nlev - 1) {
          int d = degree_in_part(v);
          if (d < cd) { cd = d; cand = v; }
        }
      unvisit();
      int f2;
      int nl2 = bfs(cand, f2);
      if (nl2 <= nlev) {
        unvisit();
        nlev = bfs(root, far);
        break;
      }
      root = cand;
      nlev = nl2;
      far = f2;
    }
    if (nlev < 3) {
      unvisit();
      if (size <= 64) min_degree(lo, hi); else by_degree(lo, hi);
      return;
    }
    std::vector<int> cnt(nlev, 0);
    for (int v : queue_) cnt[lev_[v]]++;
    int k = separator_level(cnt, size);
    if (roots_ > 1) {
      // the same choice on the level structure from the other end; keep the smaller level
      int f2;
      unvisit();
      int nl2 = bfs(far, f2);
      std::vector<int> cnt2(nl2, 0);
      for (int v : queue_) cnt2[lev_[v]]++;
      int k2 = nl2 >= 3 ? separator_level(cnt2, size) : -1;
      if (k2 >= 0 && cnt2[k2] < cnt[k]) {
        k = k2;
        nlev = nl2;
      } else {
        unvisit();
        nlev = bfs(root, far);
      }
    }
    // classify: 0 = A (lev < k), 1 = B (lev > k), 2 = S
    tmp_.clear();
    std::vector<int32_t> A, B, S;
    for (int v : queue_) {
      int l = lev_[v];
      if (l < k) A.push_back(v);
      else if (l > k) B.push_back(v);
      else S.push_back(v);
    }
    // refine: separator vertices with no neighbour in B move to A
    std::vector<int32_t> S2;
    for (int v : S) {
      bool touchB = false;
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int u = g_.adj[e];
        if ((mark_[u] == -stamp_) && lev_[u] == k + 1) { touchB = true; break; }
      }
      if (touchB) S2.push_back(v); else A.push_back(v);
    }
    unvisit();
    int p = lo;
    for (int v : A) buf_[p++] = v;
    for (int v : B) buf_[p++] = v;
    for (int v : S2) buf_[p++] = v;
    if (!A.empty()) stack.push_back({lo, lo + (int)A.size()});
    if (!B.empty()) stack.push_back({lo + (int)A.size(), lo + (int)(A.size() + B.size())});
  }
};

// Merged blocks for the triangular solves.  A chain of consecutive supernodes s, s+1, ...,
// each the parent of the previous, whose row structures nest -- R(s) is the columns of s+1
// followed by R(s+1) -- is one dense triangle of the factor cut at the supernode width cap (a
// nested-dissection separator).  Solving it piece by piece is a chain of dependent hand-offs;
// through the explicit inverse M of the merged triangle (L_G^-1 forward, U_G^-1 backward) it
// is a GEMV that many CTAs share.  M is computed after each refactor by recursive block
// inversion of the pieces (inv [A 0; B C] = [A^-1 0; -C^-1 B A^-1  C^-1], and the upper-
// triangular mirror) as phases of 64 x 64-tiled copies and GEMMs over the existing factor.
static bool nests(const Symbolic& S, int a) {
  const int b = a + 1;
  if (S.sn_parent[a] != b) return false;
  const int64_t ra = S.rptr[a + 1] - S.rptr[a], rb = S.rptr[b + 1] - S.rptr[b];
  const int wb = S.sn_start[b + 1] - S.sn_start[b];
  if (ra != wb + rb) return false;
  const int32_t* Ra = S.rows.data() + S.rptr[a];
  const int32_t* Rb = S.rows.data() + S.rptr[b];
  for (int q = 0; q < wb; ++q)
    if (Ra[q] != S.sn_start[b] + q) return false;
  for (int64_t q = 0; q < rb; ++q)
    if (Ra[wb + q] != Rb[q]) return false;
  return true;
}

static void plan_merged_blocks(Symbolic& S, const SymbolicOptions& opt) {
  const int nsn = S.nsn;
  S.sn_grp.assign(nsn, -1);
  S.grp_first.clear(); S.grp_last.clear(); S.grp_c0.clear(); S.grp_W.clear();
  S.grp_moff.clear();
  S.m_total = 0;
  S.mjobs.clear(); S.mphase_ptr.assign(1, 0); S.mtile.clear();
  S.mscratch = 0;
  S.minv_flops = 0.0;
  if (opt.merge_min_width <= 0) return;
  for (int s = 0; s < nsn;) {
    int e = s;
    while (e + 1 < nsn && nests(S, e) &&
           S.sn_start[e + 2] - S.sn_start[s] <= opt.merge_max_width)
      ++e;
    const int W = S.sn_start[e + 1] - S.sn_start[s];
    if (e > s && W >= opt.merge_min_width) {
      const int g = (int)S.grp_first.size();
      S.grp_first.push_back(s);
      S.grp_last.push_back(e);
      S.grp_c0.push_back(S.sn_start[s]);
      S.grp_W.push_back(W);
      S.grp_moff.push_back(S.m_total);
      S.m_total += (int64_t)W * W;
      for (int q = s; q <= e; ++q) S.sn_grp[q] = g;
    }
    s = e > s ? e + 1 : s + 1;
  }
  // inversion plan: recursion nodes by height (leaves 0), phases 0 (leaf copies) then, per
  // height h >= 1, the copies of B, T = B X, and the off-diagonal block -X T
  struct Node { int g, lo, mid, hi; };
  std::vector<std::vector<Node>> by_h;
  std::vector<MJob> leaf_jobs;
  std::function<int(int, int, int)> rec = [&](int g, int lo, int hi) -> int {
    const int f = S.grp_first[g];
    if (lo == hi) {
      const int sp = f + lo;
      const int w = S.sn_start[sp + 1] - S.sn_start[sp];
      const int W = S.grp_W[g];
      const int64_t o = S.sn_start[sp] - S.grp_c0[g];
      for (int side = 0; side < 2; ++side) {
        MJob j{};
        j.kind = MJOB_COPY; j.m = w; j.n = w; j.k = 0;
        j.a_arr = side == 0 ? MARR_LDI : MARR_UDI; j.a_off = S.d_off[sp]; j.lda = w;
        j.c_arr = side == 0 ? MARR_ML : MARR_MU; j.c_off = S.grp_moff[g] + o + o * W;
        j.ldc = W; j.alpha = 1.0;
        leaf_jobs.push_back(j);
      }
      return 0;
    }
    const int mid = (lo + hi + 1) / 2;
    const int h = std::max(rec(g, lo, mid - 1), rec(g, mid, hi)) + 1;
    if ((int)by_h.size() <= h) by_h.resize(h + 1);
    by_h[h].push_back({g, lo, mid, hi});
    return h;
  };
  for (int g = 0; g < (int)S.grp_first.size(); ++g)
    rec(g, 0, S.grp_last[g] - S.grp_first[g]);
  std::vector<std::vector<MJob>> phases(1, leaf_jobs);
  for (size_t h = 1; h < by_h.size(); ++h) {
    std::vector<MJob> pa, pb, pc;
    int64_t scr = 0;
    for (const Node& nd : by_h[h]) {
      const int f = S.grp_first[nd.g], W = S.grp_W[nd.g], c0 = S.grp_c0[nd.g];
      const int64_t moff = S.grp_moff[nd.g];
      auto o = [&](int i) -> int64_t { return S.sn_start[f + i] - c0; };
      const int WA = (int)(o(nd.mid) - o(nd.lo)), WC = (int)(o(nd.hi + 1) - o(nd.mid));
      const int64_t bdL = scr, tL = scr + (int64_t)WA * WC, bdU = scr + 2 * (int64_t)WA * WC,
                    tU = scr + 3 * (int64_t)WA * WC;
      scr += 4 * (int64_t)WA * WC;
      for (int p = nd.lo; p < nd.mid; ++p) {
        const int sp = f + p;
        const int wp = S.sn_start[sp + 1] - S.sn_start[sp];
        const int rp = (int)(S.rptr[sp + 1] - S.rptr[sp]);
        const int64_t roff = o(nd.mid) - o(p + 1);   // first row of the C block in R(sp)
        MJob a{};
        a.kind = MJOB_COPY; a.m = WC; a.n = wp;
        a.a_arr = MARR_LO; a.a_off = S.o_off[sp] + roff; a.lda = rp;
        a.c_arr = MARR_SCR; a.c_off = bdL + (o(p) - o(nd.lo)) * WC; a.ldc = WC; a.alpha = 1.0;
        pa.push_back(a);
        MJob u{};
        u.kind = MJOB_COPYT; u.m = wp; u.n = WC;
        u.a_arr = MARR_UO; u.a_off = S.o_off[sp] + roff; u.lda = rp;
        u.c_arr = MARR_SCR; u.c_off = bdU + (o(p) - o(nd.lo)); u.ldc = WA; u.alpha = 1.0;
        pa.push_back(u);
      }
      MJob b1{};   // T_L = B_L X_A (X_A lower)
      b1.kind = MJOB_GEMM; b1.m = WC; b1.n = WA; b1.k = WA; b1.tri = MTRI_B_LOWER;
      b1.a_arr = MARR_SCR; b1.a_off = bdL; b1.lda = WC;
      b1.b_arr = MARR_ML; b1.b_off = moff + o(nd.lo) + o(nd.lo) * W; b1.ldb = W;
      b1.c_arr = MARR_SCR; b1.c_off = tL; b1.ldc = WC; b1.alpha = 1.0;
      pb.push_back(b1);
      MJob b2{};   // T_U = B_U X_C (X_C upper)
      b2.kind = MJOB_GEMM; b2.m = WA; b2.n = WC; b2.k = WC; b2.tri = MTRI_B_UPPER;
      b2.a_arr = MARR_SCR; b2.a_off = bdU; b2.lda = WA;
      b2.b_arr = MARR_MU; b2.b_off = moff + o(nd.mid) + o(nd.mid) * W; b2.ldb = W;
      b2.c_arr = MARR_SCR; b2.c_off = tU; b2.ldc = WA; b2.alpha = 1.0;
      pb.push_back(b2);
      MJob c1{};   // M_L[C, A] = -X_C T_L (X_C lower)
      c1.kind = MJOB_GEMM; c1.m = WC; c1.n = WA; c1.k = WC; c1.tri = MTRI_A_LOWER;
      c1.a_arr = MARR_ML; c1.a_off = moff + o(nd.mid) + o(nd.mid) * W; c1.lda = W;
      c1.b_arr = MARR_SCR; c1.b_off = tL; c1.ldb = WC;
      c1.c_arr = MARR_ML; c1.c_off = moff + o(nd.mid) + o(nd.lo) * W; c1.ldc = W;
      c1.alpha = -1.0;
      pc.push_back(c1);
      MJob c2{};   // M_U[A, C] = -X_A T_U (X_A upper)
      c2.kind = MJOB_GEMM; c2.m = WA; c2.n = WC; c2.k = WA; c2.tri = MTRI_A_UPPER;
      c2.a_arr = MARR_MU; c2.a_off = moff + o(nd.lo) + o(nd.lo) * W; c2.lda = W;
      c2.b_arr = MARR_SCR; c2.b_off = tU; c2.ldb = WA;
      c2.c_arr = MARR_MU; c2.c_off = moff + o(nd.lo) + o(nd.mid) * W; c2.ldc = W;
      c2.alpha = -1.0;
      pc.push_back(c2);
      // about half of each GEMM's products are skipped by its triangular operand
      S.minv_flops += 2.0 * ((double)WC * WA * WA + (double)WA * WC * WC);
    }
    S.mscratch = std::max(S.mscratch, scr);
    phases.push_back(pa);
    phases.push_back(pb);
    phases.push_back(pc);
  }
  for (const auto& ph : phases) {
    for (const MJob& j : ph) {
      const int jid = (int)S.mjobs.size();
      S.mjobs.push_back(j);
      for (int ti = 0; ti < (j.m + 63) / 64; ++ti)
        for (int tj = 0; tj < (j.n + 63) / 64; ++tj) {
          S.mtile.push_back(jid);
          S.mtile.push_back((ti << 16) | tj);
        }
    }
    S.mphase_ptr.push_back((int32_t)(S.mtile.size() / 2));
  }
}

}  // namespace

std::string analyze(int n, const int32_t* ptr, const int32_t* idx, const SymbolicOptions& opt,
                    Symbolic& S) {
  if (n <= 0) return "empty matrix";
  for (int i = 0; i < n; ++i) {
    if (ptr[i + 1] < ptr[i]) return "row pointer not monotone";
    bool diag = false;
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e) {
      if (idx[e] < 0 || idx[e] >= n) return "column index out of range";
      if (e > ptr[i] && idx[e] <= idx[e - 1]) return "columns not sorted/unique";
      if (idx[e] == i) diag = true;
    }
    if (!diag) return "missing diagonal entry in row " + std::to_string(i);
  }
  S = Symbolic();
  S.n = n;
  Graph g = symmetrize(n, ptr, idx);

  // 1. ordering
  Dissector nd(g, std::min(opt.leaf_size, 64), opt.sep_window_pct, opt.sep_roots);
  std::vector<int32_t> perm = nd.run();
  std::vector<int32_t> iperm(n);
  for (int k = 0; k < n; ++k) iperm[perm[k]] = k;

  // permuted symmetric adjacency (for etree and counts)
  auto permuted_adj = [&](const std::vector<int32_t>& iper, std::vector<int64_t>& px,
                          std::vector<int32_t>& pa) {
    px.assign(n + 1, 0);
    for (int k = 0; k < n; ++k) {
      int v = perm[k];
      px[k + 1] = px[k] + (g.xadj[v + 1] - g.xadj[v]);
    }
    pa.resize(px[n]);
    for (int k = 0; k < n; ++k) {
      int v = perm[k];
      int64_t o = px[k];
      for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) pa[o++] = iper[g.adj[e]];
      std::sort(pa.begin() + px[k], pa.begin() + px[k + 1]);
    }
  };
  std::vector<int64_t> px;
  std::vector<int32_t> pa;
  permuted_adj(iperm, px, pa);

  // 2. elimination tree (Liu), then postorder and re-permute
  auto etree = [&](std::vector<int32_t>& par) {
    par.assign(n, -1);
    std::vector<int32_t> anc(n, -1);
    for (int j = 0; j < n; ++j)
      for (int64_t e = px[j]; e < px[j + 1]; ++e) {
        int i = pa[e];
        if (i >= j) break;
        int r = i;
        while (anc[r] != -1 && anc[r] != j) {
          int t = anc[r];
          anc[r] = j;
          r = t;
        }
        if (anc[r] == -1) { anc[r] = j; par[r] = j; }
      }
  };
  std::vector<int32_t> par;
  etree(par);
  {
    // postorder (children in increasing order)
    std::vector<int32_t> head(n, -1), next(n, -1), post;
    post.reserve(n);
    for (int j = n - 1; j >= 0; --j)
      if (par[j] >= 0) { next[j] = head[par[j]]; head[par[j]] = j; }
    std::vector<int32_t> st;
    for (int r = 0; r < n; ++r) {
      if (par[r] != -1) continue;
      st.push_back(r);
      while (!st.empty()) {
        int v = st.back();
        if (head[v] != -1) {
          int c = head[v];
          head[v] = next[c];
          st.push_back(c);
        } else {
          st.pop_back();
          post.push_back(v);
        }
      }
    }
    std::vector<int32_t> perm2(n);
    for (int k = 0; k < n; ++k) perm2[k] = perm[post[k]];
    perm = perm2;
    for (int k = 0; k < n; ++k) iperm[perm[k]] = k;
    permuted_adj(iperm, px, pa);
    etree(par);
  }
  S.perm = perm;
  S.iperm = iperm;
  S.parent = par;

  // permuted A pattern (not symmetrised) with the source slot of each entry
  {
    S.a_ptr.assign(n + 1, 0);
    for (int k = 0; k < n; ++k) {
      int v = perm[k];
      S.a_ptr[k + 1] = S.a_ptr[k] + (ptr[v + 1] - ptr[v]);
    }
    S.a_idx.resize(S.a_ptr[n]);
    S.a_src.resize(S.a_ptr[n]);
    std::vector<std::pair<int32_t, int32_t>> rowbuf;
    for (int k = 0; k < n; ++k) {
      int v = perm[k];
      rowbuf.clear();
      for (int32_t e = ptr[v]; e < ptr[v + 1]; ++e) rowbuf.push_back({iperm[idx[e]], e});
      std::sort(rowbuf.begin(), rowbuf.end());
      int32_t o = S.a_ptr[k];
      for (auto& pr : rowbuf) { S.a_idx[o] = pr.first; S.a_src[o] = pr.second; ++o; }
    }
  }

  // column counts by row subtrees (counts include the diagonal)
  std::vector<int64_t> cc(n, 1);
  {
    std::vector<int32_t> mk(n, -1);
    for (int i = 0; i < n; ++i) {
      mk[i] = i;
      for (int64_t e = px[i]; e < px[i + 1]; ++e) {
        int j = pa[e];
        if (j >= i) break;
        while (mk[j] != i) { mk[j] = i; cc[j]++; j = par[j]; }
      }
    }
  }
  S.colcount = cc;
  S.nnz_L = 0;
  for (int j = 0; j < n; ++j) S.nnz_L += cc[j];
  {
    std::vector<int32_t> depth(n, 0);
    int h = 0;
    for (int j = n - 1; j >= 0; --j) {
      depth[j] = par[j] >= 0 ? depth[par[j]] + 1 : 1;
      h = std::max(h, depth[j]);
    }
    S.etree_height = h;
  }

  // 3. fundamental supernodes (width-capped)
  std::vector<int32_t> nchild(n, 0);
  for (int j = 0; j < n; ++j)
    if (par[j] >= 0) nchild[par[j]]++;
  S.sn_start.clear();
  S.sn_start.push_back(0);
  for (int j = 1; j < n; ++j) {
    bool merge = par[j - 1] == j && cc[j - 1] == cc[j] + 1 && nchild[j] == 1 &&
                 (j - S.sn_start.back()) < opt.max_width;
    if (!merge) S.sn_start.push_back(j);
  }
  S.sn_start.push_back(n);
  // relaxed amalgamation: fold a supernode into its parent when it is the parent's last
  // child (so the columns stay contiguous), the merged width stays within max_width and
  // the explicit zeros it adds stay small.  Long chains of narrow supernodes in the
  // nested-dissection leaves otherwise make the elimination tree (and the number of
  // dependent levels of the solves and the refactor) needlessly deep.
  if (opt.relax_zeros > 0) {
    int nf = (int)S.sn_start.size() - 1;
    std::vector<int32_t> first(nf), width(nf), offr(nf), par_sn(nf, -1), snf(n);
    for (int s = 0; s < nf; ++s) {
      first[s] = S.sn_start[s];
      width[s] = S.sn_start[s + 1] - S.sn_start[s];
      offr[s] = (int32_t)(cc[first[s]] - width[s]);
      for (int j = S.sn_start[s]; j < S.sn_start[s + 1]; ++j) snf[j] = s;
    }
    for (int s = 0; s < nf; ++s) {
      int last = S.sn_start[s + 1] - 1;
      if (par[last] >= 0) par_sn[s] = snf[par[last]];
    }
    // group g (start supernode) accumulates merged width, true nnz of its columns
    std::vector<int32_t> gstart(nf);
    std::vector<int64_t> gtrue(nf);
    std::vector<int32_t> gwidth(nf);
    std::vector<char> merged_into_next(nf, 0);
    for (int s = 0; s < nf; ++s) {
      gstart[s] = s;
      gwidth[s] = width[s];
      int64_t t = 0;
      for (int j = S.sn_start[s]; j < S.sn_start[s + 1]; ++j) t += cc[j];
      gtrue[s] = t;
    }
    for (int s = 0; s < nf; ++s) {
      int p = par_sn[s];
      if (p < 0 || p != s + 1) continue;                 // last child only (contiguous)
      if (S.sn_start[s + 1] != first[p]) continue;
      int64_t W = gwidth[s] + width[p];
      if (W > opt.max_width) continue;
      int64_t rp = offr[p];
      int64_t stored = W * rp + W * (W + 1) / 2;
      int64_t truth = gtrue[s];
      for (int j = S.sn_start[p]; j < S.sn_start[p + 1]; ++j) truth += cc[j];
      if (W > opt.relax_width && (stored - truth) * 100 > (int64_t)opt.relax_zeros * stored)
        continue;
      // merge group of s into p: p's group now starts where s's group started
      merged_into_next[s] = 1;
      gstart[p] = gstart[s];
      gwidth[p] = (int32_t)W;
      gtrue[p] = truth;
    }
    std::vector<int32_t> ns{0};
    for (int s = 0; s < nf; ++s)
      if (!merged_into_next[s]) ns.push_back(S.sn_start[s + 1]);
    S.sn_start = ns;
  }
  S.nsn = (int)S.sn_start.size() - 1;
  int nsn = S.nsn;
  S.sn_of.assign(n, 0);
  for (int s = 0; s < nsn; ++s)
    for (int j = S.sn_start[s]; j < S.sn_start[s + 1]; ++j) S.sn_of[j] = s;

  // row structures: pattern rows of the supernode's columns plus children's structures
  S.rptr.assign(nsn + 1, 0);
  S.rows.clear();
  S.sn_parent.assign(nsn, -1);
  std::vector<std::vector<int32_t>> children(nsn);
  {
    std::vector<int32_t> mk(n, -1), lst;
    for (int s = 0; s < nsn; ++s) {
      int c0 = S.sn_start[s], c1 = S.sn_start[s + 1];
      lst.clear();
      for (int j = c0; j < c1; ++j)
        for (int64_t e = px[j]; e < px[j + 1]; ++e) {
          int i = pa[e];
          if (i >= c1 && mk[i] != s) { mk[i] = s; lst.push_back(i); }
        }
      for (int c : children[s])
        for (int64_t e = S.rptr[c]; e < S.rptr[c + 1]; ++e) {
          int i = S.rows[e];
          if (i >= c1 && mk[i] != s) { mk[i] = s; lst.push_back(i); }
        }
      std::sort(lst.begin(), lst.end());
      if ((int64_t)lst.size() + (c1 - c0) < cc[c0])
        return "internal: supernode structure smaller than its column count";
      S.rows.insert(S.rows.end(), lst.begin(), lst.end());
      S.rptr[s + 1] = (int64_t)S.rows.size();
      if (!lst.empty()) {
        int p = S.sn_of[lst[0]];
        S.sn_parent[s] = p;
        children[p].push_back(s);
      }
    }
  }

  // padding for merged solve blocks: when supernode a's parent is a + 1 and R(a) is a strict
  // subset of the columns of a + 1 followed by R(a + 1) (always a superset, the parent's
  // structure absorbs its child's), R(a) takes that superset with explicit zeros if they
  // cost at most merge_pad_pct % of a's own off-diagonal panel; the two then nest and can be
  // solved as one dense triangle.  Top-down, so a parent is padded before its child reads it.
  if (opt.merge_min_width > 0 && opt.merge_pad_pct > 0) {
    std::vector<std::vector<int32_t>> padded(nsn);
    std::vector<char> has(nsn, 0);
    auto rows_of = [&](int s) -> std::vector<int32_t> {
      if (has[s]) return padded[s];
      return std::vector<int32_t>(S.rows.begin() + S.rptr[s], S.rows.begin() + S.rptr[s + 1]);
    };
    auto large_sn = [&](int s, int64_t r) {
      const int64_t w = S.sn_start[s + 1] - S.sn_start[s];
      return w * (w + r) > opt.fused_limit;
    };
    int64_t grown = 0;
    for (int a = nsn - 2; a >= 0; --a) {
      const int b = a + 1;
      if (S.sn_parent[a] != b) continue;
      std::vector<int32_t> Rb = rows_of(b);
      const int64_t ra = S.rptr[a + 1] - S.rptr[a];
      const int64_t wa = S.sn_start[a + 1] - S.sn_start[a], wb = S.sn_start[b + 1] - S.sn_start[b];
      const int64_t need = wb + (int64_t)Rb.size();
      if (need == ra || !large_sn(a, ra) || !large_sn(b, (int64_t)Rb.size())) continue;
      if ((need - ra) * 100 > (int64_t)opt.merge_pad_pct * ra) continue;
      std::vector<int32_t> R;
      R.reserve(need);
      for (int q = 0; q < wb; ++q) R.push_back(S.sn_start[b] + q);
      R.insert(R.end(), Rb.begin(), Rb.end());
      // R(a) must be contained in R (the parent's columns and structure)
      std::vector<int32_t> Ra(S.rows.begin() + S.rptr[a], S.rows.begin() + S.rptr[a + 1]);
      if (!std::includes(R.begin(), R.end(), Ra.begin(), Ra.end())) continue;
      grown += (need - ra) * wa;
      padded[a] = std::move(R);
      has[a] = 1;
    }
    if (grown > 0) {
      std::vector<int64_t> nptr(nsn + 1, 0);
      std::vector<int32_t> nrows;
      nrows.reserve(S.rows.size() + grown);
      for (int s2 = 0; s2 < nsn; ++s2) {
        if (has[s2]) nrows.insert(nrows.end(), padded[s2].begin(), padded[s2].end());
        else nrows.insert(nrows.end(), S.rows.begin() + S.rptr[s2], S.rows.begin() + S.rptr[s2 + 1]);
        nptr[s2 + 1] = (int64_t)nrows.size();
      }
      S.rows.swap(nrows);
      S.rptr.swap(nptr);
    }
  }

  // levels (leaves 0) and storage
  S.level.assign(nsn, 0);
  for (int s = 0; s < nsn; ++s)
    if (S.sn_parent[s] >= 0) S.level[S.sn_parent[s]] = std::max(S.level[S.sn_parent[s]], S.level[s] + 1);
  S.nlevels = 0;
  for (int s = 0; s < nsn; ++s) S.nlevels = std::max(S.nlevels, S.level[s] + 1);
  S.d_off.assign(nsn, 0);
  S.o_off.assign(nsn, 0);
  S.d_total = S.o_total = 0;
  S.flops = 0.0;
  S.max_front = 0;
  for (int s = 0; s < nsn; ++s) {
    int64_t w = S.sn_start[s + 1] - S.sn_start[s];
    int64_t r = S.rptr[s + 1] - S.rptr[s];
    S.d_off[s] = S.d_total;
    S.d_total += w * w;
    S.o_off[s] = S.o_total;
    S.o_total += r * w;
    S.max_front = std::max<int>(S.max_front, (int)(w + r));
    double wd = (double)w, rd = (double)r;
    S.flops += 2.0 / 3.0 * wd * wd * wd + 2.0 * wd * wd * rd + 2.0 * wd * rd * rd;
  }

  // 4. multifrontal plan ------------------------------------------------------------
  // relative indices of each child's rows in the parent's front
  S.rel.assign(S.rows.size(), 0);
  for (int s = 0; s < nsn; ++s) {
    int p = S.sn_parent[s];
    if (p < 0) continue;
    int pc0 = S.sn_start[p], pw = S.sn_start[p + 1] - pc0;
    const int32_t* prow = S.rows.data() + S.rptr[p];
    int64_t pr = S.rptr[p + 1] - S.rptr[p];
    for (int64_t e = S.rptr[s]; e < S.rptr[s + 1]; ++e) {
      int i = S.rows[e];
      int pos;
      if (i < pc0 + pw) pos = i - pc0;
      else {
        const int32_t* it = std::lower_bound(prow, prow + pr, i);
        if (it == prow + pr || *it != i) return "internal: child row missing from parent";
        pos = pw + (int)(it - prow);
      }
      S.rel[e] = pos;
    }
  }
  // supernodes by level
  S.lvl_sn_ptr.assign(S.nlevels + 1, 0);
  for (int s = 0; s < nsn; ++s) S.lvl_sn_ptr[S.level[s] + 1]++;
  for (int l = 0; l < S.nlevels; ++l) S.lvl_sn_ptr[l + 1] += S.lvl_sn_ptr[l];
  S.lvl_sn.resize(nsn);
  {
    std::vector<int32_t> pos(S.lvl_sn_ptr.begin(), S.lvl_sn_ptr.end() - 1);
    for (int s = 0; s < nsn; ++s) S.lvl_sn[pos[S.level[s]]++] = s;
  }
  // arena: an allocator simulated level by level (best fit, ties to the lowest offset; free
  // blocks indexed by offset for coalescing and by (length, offset) for the fit: O(log n) per
  // operation, since a batch of many circuits has millions of fronts)
  {
    std::map<int64_t, int64_t> by_off;               // offset -> length
    std::set<std::pair<int64_t, int64_t>> by_len;    // (length, offset)
    int64_t top = 0;
    auto take = [&](std::map<int64_t, int64_t>::iterator it) {
      by_len.erase({it->second, it->first});
      by_off.erase(it);
    };
    auto put = [&](int64_t off, int64_t len) {
      by_off[off] = len;
      by_len.insert({len, off});
    };
    auto alloc = [&](int64_t len) -> int64_t {
      len = (len + 31) & ~(int64_t)31;
      auto f = by_len.lower_bound({len, INT64_MIN});
      if (f != by_len.end()) {
        int64_t o = f->second, l = f->first;
        take(by_off.find(o));
        if (l > len) put(o + len, l - len);
        return o;
      }
      int64_t o = top;
      top += len;
      return o;
    };
    auto release = [&](int64_t off, int64_t len) {
      len = (len + 31) & ~(int64_t)31;
      auto nx = by_off.lower_bound(off);
      if (nx != by_off.end() && off + len == nx->first) {   // merge with the next block
        len += nx->second;
        take(nx);
      }
      auto it = by_off.lower_bound(off);
      if (it != by_off.begin()) {                              // merge with the previous block
        auto pv = std::prev(it);
        if (pv->first + pv->second == off) {
          off = pv->first;
          len += pv->second;
          take(pv);
        }
      }
      if (off + len == top) top = off;                         // the block ends the arena
      else put(off, len);
    };
    S.front_off.assign(nsn, 0);
    int64_t peak = 0;
    for (int l = 0; l < S.nlevels; ++l) {
      for (int k = S.lvl_sn_ptr[l]; k < S.lvl_sn_ptr[l + 1]; ++k) {
        int s = S.lvl_sn[k];
        int64_t f = (S.sn_start[s + 1] - S.sn_start[s]) + (S.rptr[s + 1] - S.rptr[s]);
        S.front_off[s] = alloc(f * f);
        peak = std::max(peak, top);
      }
      for (int k = S.lvl_sn_ptr[l]; k < S.lvl_sn_ptr[l + 1]; ++k) {
        int s = S.lvl_sn[k];
        for (int c : children[s]) {
          int64_t f = (S.sn_start[c + 1] - S.sn_start[c]) + (S.rptr[c + 1] - S.rptr[c]);
          release(S.front_off[c], f * f);
        }
        if (S.sn_parent[s] < 0) {
          int64_t f = (S.sn_start[s + 1] - S.sn_start[s]) + (S.rptr[s + 1] - S.rptr[s]);
          release(S.front_off[s], f * f);
        }
      }
    }
    S.arena_size = std::max<int64_t>(peak, 32);
  }
  // assembly map of A's entries into fronts
  {
    int64_t nnzA = S.a_ptr[n];
    S.asm_dst.assign(nnzA, 0);
    std::vector<int32_t> slot_level(nnzA);
    for (int i = 0; i < n; ++i)
      for (int32_t e = S.a_ptr[i]; e < S.a_ptr[i + 1]; ++e) {
        int j = S.a_idx[e];
        int lo = std::min(i, j), hi = std::max(i, j);
        int s = S.sn_of[lo];
        int c0 = S.sn_start[s], w = S.sn_start[s + 1] - c0;
        int64_t f = w + (S.rptr[s + 1] - S.rptr[s]);
        auto pos = [&](int x) -> int64_t {
          if (x < c0 + w) return x - c0;
          const int32_t* b = S.rows.data() + S.rptr[s];
          const int32_t* en = S.rows.data() + S.rptr[s + 1];
          const int32_t* it = std::lower_bound(b, en, x);
          return w + (it - b);
        };
        (void)hi;
        S.asm_dst[e] = S.front_off[s] + pos(i) + pos(j) * f;
        slot_level[e] = S.level[s];
      }
    S.lvl_slot_ptr.assign(S.nlevels + 1, 0);
    for (int64_t e = 0; e < nnzA; ++e) S.lvl_slot_ptr[slot_level[e] + 1]++;
    for (int l = 0; l < S.nlevels; ++l) S.lvl_slot_ptr[l + 1] += S.lvl_slot_ptr[l];
    S.lvl_slot.resize(nnzA);
    std::vector<int32_t> pos(S.lvl_slot_ptr.begin(), S.lvl_slot_ptr.end() - 1);
    for (int64_t e = 0; e < nnzA; ++e) S.lvl_slot[pos[slot_level[e]]++] = (int32_t)e;
  }
  // extend-add pairs grouped by (parent level, child rank)
  {
    S.ch_ptr.assign(nsn + 1, 0);
    S.ch_list.clear();
    for (int s = 0; s < nsn; ++s) {
      S.ch_list.insert(S.ch_list.end(), children[s].begin(), children[s].end());
      S.ch_ptr[s + 1] = (int32_t)S.ch_list.size();
    }
    int maxrank = 1;
    for (int s = 0; s < nsn; ++s) maxrank = std::max<int>(maxrank, (int)children[s].size());
    S.ea_maxrank = maxrank;
    std::vector<std::vector<int32_t>> groups((size_t)S.nlevels * maxrank);
    for (int s = 0; s < nsn; ++s)
      for (size_t r = 0; r < children[s].size(); ++r)
        groups[(size_t)S.level[s] * maxrank + r].push_back(children[s][r]);
    S.ea_ptr.assign(groups.size() + 1, 0);
    S.ea_child.clear();
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      S.ea_child.insert(S.ea_child.end(), groups[gi].begin(), groups[gi].end());
      S.ea_ptr[gi + 1] = (int32_t)S.ea_child.size();
    }
  }
  // Schur-update tiles (64 x 64) and panel tasks (128 rows) per level
  {
    const int TB = 64, PB = 128;
    S.tile_ptr.assign(S.nlevels + 1, 0);
    S.ptask_ptr.assign(S.nlevels + 1, 0);
    S.tile_sn.clear(); S.tile_ij.clear(); S.ptask_sn.clear(); S.ptask_r0.clear();
    for (int l = 0; l < S.nlevels; ++l) {
      for (int k = S.lvl_sn_ptr[l]; k < S.lvl_sn_ptr[l + 1]; ++k) {
        int s = S.lvl_sn[k];
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        int nt = (r + TB - 1) / TB;
        for (int ti = 0; ti < nt; ++ti)
          for (int tj = 0; tj < nt; ++tj) {
            S.tile_sn.push_back(s);
            S.tile_ij.push_back((ti << 16) | tj);
          }
        for (int r0 = 0; r0 < r; r0 += PB) {
          S.ptask_sn.push_back(s);
          S.ptask_r0.push_back(r0);
        }
      }
      S.tile_ptr[l + 1] = (int32_t)S.tile_sn.size();
      S.ptask_ptr[l + 1] = (int32_t)S.ptask_sn.size();
    }
  }

  // merged blocks of the solves and their inversion plan
  plan_merged_blocks(S, opt);

  // 5. triangular-solve work lists ---------------------------------------------------
  {
    S.fwd.clear(); S.bwd.clear(); S.fwd_small.clear(); S.bwd_small.clear(); S.fwd_tgt.clear();
    S.fwd_lane.clear(); S.bwd_lane.clear();
    S.fwd_expect.assign(nsn, 0);
    S.bwd_nchunk.assign(nsn, 0);
    const int CH = opt.solve_chunk;
    auto add_targets = [&](int s, int r0, int r1, SolveTask& t) {
      t.tgt0 = (int32_t)S.fwd_tgt.size();
      int last = -1;
      for (int e = r0; e < r1; ++e) {
        int tg = S.sn_of[S.rows[S.rptr[s] + e]];
        if (tg != last) {
          S.fwd_tgt.push_back(tg);
          S.fwd_expect[tg]++;
          last = tg;
        }
      }
      t.ntgt = (int32_t)S.fwd_tgt.size() - t.tgt0;
    };
    auto small = [&](int s) {
      int64_t w = S.sn_start[s + 1] - S.sn_start[s];
      int64_t r = S.rptr[s + 1] - S.rptr[s];
      return S.sn_grp[s] < 0 && w * (w + r) <= opt.fused_limit;
    };
    // narrow supernodes with few rows: one lane each (a warp task holds 32)
    auto lane_item = [&](int s) {
      return S.sn_grp[s] < 0 && opt.lane_rows > 0 &&
             S.sn_start[s + 1] - S.sn_start[s] <= opt.lane_width &&
             S.rptr[s + 1] - S.rptr[s] <= opt.lane_rows;
    };
    // a large supernode with its own DIAG entry (not a piece of a merged block)
    auto large = [&](int s) { return S.sn_grp[s] < 0 && !small(s); };
    // first row of a merged piece outside its block: the rows before it are the columns of
    // the later pieces, folded into the block's inverse
    auto ext_row0 = [&](int s) -> int {
      const int g = S.sn_grp[s];
      return S.sn_start[S.grp_last[g] + 1] - S.sn_start[s + 1];
    };
    // a column block of an MGEMV task holds at most 512 columns (the kernel's staging)
    const int CB = std::max(1, std::min(opt.merge_col_block, 512 / std::max(1, opt.max_width)));
    int32_t slot_f = 0, slot_b = 0;
    // the MGEMV entries of merged block g: row tile i times column pieces [j0, j1) in blocks
    // of CB pieces (forward: pieces first..i of M_L; backward: pieces i..last of M_U)
    auto mgemv = [&](std::vector<SolveTask>& list, int g, bool fwd, int32_t& slot) {
      const int f = S.grp_first[g], l = S.grp_last[g], W = S.grp_W[g], c0 = S.grp_c0[g];
      for (int i = f; i <= l; ++i) {
        const int lo = fwd ? f : i, hi = fwd ? i + 1 : l + 1;
        const int ntask = (hi - lo + CB - 1) / CB;
        const int32_t first_slot = slot;
        for (int j0 = lo; j0 < hi; j0 += CB) {
          const int j1 = std::min(hi, j0 + CB);
          SolveTask t{};
          t.kind = TASK_MGEMV; t.sn = i; t.r0 = j0; t.r1 = j1;
          t.tgt0 = slot++; t.ntgt = 0; t.wait_sn = first_slot; t.wait_cnt = ntask;
          t.c0 = S.sn_start[i]; t.w = S.sn_start[i + 1] - S.sn_start[i]; t.r = W; t.grp = g;
          t.d_off = S.grp_moff[g] + (S.sn_start[i] - c0) + (int64_t)(S.sn_start[j0] - c0) * W;
          t.o_off = S.sn_start[j0];
          t.row_off = S.sn_start[j1];
          list.push_back(t);
        }
      }
    };

    // warp tasks (small supernodes, far chunks) live in fwd_small / bwd_small; a CTA entry
    // GROUP/BULK refers to up to 8 consecutive warp tasks of one level
    auto flush = [](std::vector<SolveTask>& list, std::vector<SolveTask>& smalls, int& first,
                    int kind) {
      int cnt = (int)smalls.size() - first;
      if (cnt <= 0) return;
      list.push_back(SolveTask{kind, first, cnt, 0, 0, 0, -1, 0});
      first = (int)smalls.size();
    };
    const int WC = opt.warp_chunk;
    const int BWC = opt.bwd_chunk;
    // Forward entries by level (height: leaves first), backward entries by decreasing level
    // (roots first): entries of one level are independent, so the CTAs holding consecutive
    // entries can all make progress and the critical path is the tree height, not the list
    // length.
    std::vector<int32_t> ford(nsn), bord(nsn);
    std::iota(ford.begin(), ford.end(), 0);
    std::iota(bord.begin(), bord.end(), 0);
    std::stable_sort(ford.begin(), ford.end(), [&](int a, int b) { return S.level[a] < S.level[b]; });
    // backward: by decreasing level (height), the forward levels reversed -- a parent's level
    // exceeds its children's, and the narrow leaves gather on the last levels, where lane
    // tasks take them 32 per warp (ordered by depth they spread over many thin levels)
    std::vector<int32_t> bkey(nsn);
    for (int s = 0; s < nsn; ++s) bkey[s] = S.nlevels - 1 - S.level[s];
    std::stable_sort(bord.begin(), bord.end(), [&](int a, int b) { return bkey[a] < bkey[b]; });
    // forward: per level, narrow supernodes (one per lane) and small ones (one per warp) in
    // GROUP entries, DIAG entries, then far chunks (BULK)
    for (size_t k0 = 0; k0 < ford.size();) {
      size_t k1 = k0;
      while (k1 < ford.size() && S.level[ford[k1]] == S.level[ford[k0]]) ++k1;
      int first = (int)S.fwd_small.size();
      bool lane_level = false;
      {
        // lane tasks of this level: 32 narrow supernodes per warp task
        std::vector<int> items;
        for (size_t k = k0; k < k1; ++k) {
          int s = ford[k];
          if (!lane_item(s)) continue;
          items.push_back(s);
        }
        // a level too narrow to fill the GPU's warps is latency-bound: a warp per supernode
        if ((int)items.size() < opt.lane_min_level) items.clear();
        lane_level = !items.empty();
        for (size_t a = 0; a < items.size(); a += 32) {
          int cnt = (int)std::min<size_t>(32, items.size() - a);
          SolveTask t{TASK_LANES, (int32_t)(S.fwd_lane.size() / 4), cnt, 0, 0, 0, -1, 0};
          for (int b = 0; b < cnt; ++b) {
            int s = items[a + b];
            SolveTask u{};
            add_targets(s, 0, (int)(S.rptr[s + 1] - S.rptr[s]), u);
            S.fwd_lane.insert(S.fwd_lane.end(), {s, u.tgt0, u.ntgt, 0});
          }
          S.fwd_small.push_back(t);
          if ((int)S.fwd_small.size() - first == 8) flush(S.fwd, S.fwd_small, first, TASK_GROUP);
        }
      }
      for (size_t k = k0; k < k1; ++k) {
        int s = ford[k];
        if (!small(s) || (lane_level && lane_item(s))) continue;
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        SolveTask t{TASK_FUSED, s, 0, r, 0, 0, -1, 0};
        add_targets(s, 0, r, t);
        S.fwd_small.push_back(t);
        if ((int)S.fwd_small.size() - first == 8) flush(S.fwd, S.fwd_small, first, TASK_GROUP);
      }
      flush(S.fwd, S.fwd_small, first, TASK_GROUP);
      for (size_t k = k0; k < k1; ++k) {
        int s = ford[k];
        if (!large(s)) continue;
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        SolveTask d{TASK_DIAG, s, 0, std::min(r, CH), 0, 0, -1, 0};
        add_targets(s, 0, d.r1, d);
        S.fwd.push_back(d);
      }
      // merged blocks whose last (highest) piece is on this level: every contribution from
      // outside the block comes from lower levels
      std::vector<int> done_grp;
      for (size_t k = k0; k < k1; ++k) {
        int s = ford[k];
        if (S.sn_grp[s] >= 0 && S.grp_last[S.sn_grp[s]] == s) done_grp.push_back(S.sn_grp[s]);
      }
      for (int g : done_grp) mgemv(S.fwd, g, true, slot_f);
      first = (int)S.fwd_small.size();
      auto far_chunks = [&](int s, int r_begin) {
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        for (int r0 = r_begin; r0 < r; r0 += WC) {
          SolveTask t{TASK_OFF, s, r0, std::min(r, r0 + WC), 0, 0, -1, 0};
          add_targets(s, t.r0, t.r1, t);
          S.fwd_small.push_back(t);
          if ((int)S.fwd_small.size() - first == 8) flush(S.fwd, S.fwd_small, first, TASK_BULK);
        }
      };
      for (size_t k = k0; k < k1; ++k) {
        int s = ford[k];
        if (large(s)) far_chunks(s, CH);
      }
      for (int g : done_grp)
        for (int s = S.grp_first[g]; s <= S.grp_last[g]; ++s) far_chunks(s, ext_row0(s));
      flush(S.fwd, S.fwd_small, first, TASK_BULK);
      k0 = k1;
    }
    // backward: per level (decreasing), far chunks (BULK; they wait for ancestors only), then small
    // supernodes (GROUP) and DIAG entries
    for (size_t k0 = 0; k0 < bord.size();) {
      size_t k1 = k0;
      while (k1 < bord.size() && bkey[bord[k1]] == bkey[bord[k0]]) ++k1;
      int first = (int)S.bwd_small.size();
      auto far_chunks = [&](int s, int r_begin) {
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        for (int r0 = r_begin; r0 < r; r0 += BWC) {
          int ws = S.sn_of[S.rows[S.rptr[s] + r0]];
          S.bwd_small.push_back(SolveTask{TASK_OFF, s, r0, std::min(r, r0 + BWC), 0, 0, ws, 0});
          S.bwd_nchunk[s]++;
          if ((int)S.bwd_small.size() - first == 8) flush(S.bwd, S.bwd_small, first, TASK_BULK);
        }
      };
      for (size_t k = k0; k < k1; ++k) {
        int s = bord[k];
        if (large(s)) far_chunks(s, CH);
      }
      // merged blocks whose last (top) piece is on this level: their far chunks wait for
      // ancestors only, their MGEMV entries (below) for those chunks
      std::vector<int> done_grp;
      for (size_t k = k0; k < k1; ++k) {
        int s = bord[k];
        if (S.sn_grp[s] >= 0 && S.grp_last[S.sn_grp[s]] == s) done_grp.push_back(S.sn_grp[s]);
      }
      for (int g : done_grp)
        for (int s = S.grp_first[g]; s <= S.grp_last[g]; ++s) far_chunks(s, ext_row0(s));
      flush(S.bwd, S.bwd_small, first, TASK_BULK);
      bool lane_level = false;
      {
        std::vector<int> items;
        for (size_t k = k0; k < k1; ++k) {
          int s = bord[k];
          if (!lane_item(s)) continue;
          items.push_back(s);
        }
        if ((int)items.size() < opt.lane_min_level) items.clear();
        lane_level = !items.empty();
        for (size_t a = 0; a < items.size(); a += 32) {
          int cnt = (int)std::min<size_t>(32, items.size() - a);
          SolveTask t{TASK_LANES, (int32_t)(S.bwd_lane.size() / 4), cnt, 0, 0, 0, -1, 0};
          for (int b = 0; b < cnt; ++b) {
            int s = items[a + b];
            S.bwd_lane.insert(S.bwd_lane.end(), {s, S.sn_parent[s], 0, 0});
          }
          S.bwd_small.push_back(t);
          if ((int)S.bwd_small.size() - first == 8) flush(S.bwd, S.bwd_small, first, TASK_GROUP);
        }
      }
      for (size_t k = k0; k < k1; ++k) {
        int s = bord[k];
        if (!small(s) || (lane_level && lane_item(s))) continue;
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        S.bwd_small.push_back(SolveTask{TASK_FUSED, s, 0, r, 0, 0, S.sn_parent[s], 0});
        if ((int)S.bwd_small.size() - first == 8) flush(S.bwd, S.bwd_small, first, TASK_GROUP);
      }
      flush(S.bwd, S.bwd_small, first, TASK_GROUP);
      for (size_t k = k0; k < k1; ++k) {
        int s = bord[k];
        if (!large(s)) continue;
        int r = (int)(S.rptr[s + 1] - S.rptr[s]);
        S.bwd.push_back(SolveTask{TASK_DIAG, s, 0, std::min(r, CH), 0, 0, S.sn_parent[s], 0});
      }
      for (int g : done_grp) mgemv(S.bwd, g, false, slot_b);
      k0 = k1;
    }
    S.nslots = std::max(slot_f, slot_b);
    // descriptors: everything a task needs in one record
    auto fill = [&](SolveTask& t, bool fwd) {
      if (t.kind == TASK_MGEMV) return;
      t.grp = -1;
      if (t.kind == TASK_GROUP || t.kind == TASK_BULK) return;
      if (t.kind == TASK_LANES) return;
      int s = t.sn;
      t.grp = S.sn_grp[s];
      t.c0 = S.sn_start[s];
      t.w = S.sn_start[s + 1] - t.c0;
      t.r = (int32_t)(S.rptr[s + 1] - S.rptr[s]);
      t.d_off = S.d_off[s];
      t.o_off = S.o_off[s];
      t.row_off = S.rptr[s];
      if (fwd) t.wait_cnt = (t.kind == TASK_OFF) ? 1 : S.fwd_expect[s];
      else t.wait_cnt = (t.kind == TASK_DIAG) ? S.bwd_nchunk[s] : 0;
    };
    for (size_t q = 0; q < S.fwd_lane.size(); q += 4) S.fwd_lane[q + 3] = S.fwd_expect[S.fwd_lane[q]];
    for (auto& t : S.fwd) fill(t, true);
    for (auto& t : S.fwd_small) fill(t, true);
    for (auto& t : S.bwd) fill(t, false);
    for (auto& t : S.bwd_small) fill(t, false);
  }
  return "";
}


// The multifrontal refactor plan: front s lives from the allocation phase of its level to
// the release phase of its parent's level (its own, for a root), so every two fronts whose
// lives overlap must occupy disjoint arena ranges; every front lies inside the arena; no two
// entries of A assembled at one level go to one arena position; every relative index of a
// child's rows points inside its parent's front.
static std::string check_refactor_plan(const Symbolic& S) {
  const int nsn = S.nsn;
  auto fsize = [&](int s) -> int64_t {
    return (S.sn_start[s + 1] - S.sn_start[s]) + (S.rptr[s + 1] - S.rptr[s]);
  };
  auto padded = [](int64_t len) { return (len + 31) & ~(int64_t)31; };
  std::vector<std::vector<int32_t>> born(S.nlevels), dies(S.nlevels);
  for (int s = 0; s < nsn; ++s) {
    if (S.level[s] < 0 || S.level[s] >= S.nlevels) return "front level out of range";
    int p = S.sn_parent[s];
    int last = p < 0 ? S.level[s] : S.level[p];
    if (p >= 0 && S.level[p] <= S.level[s]) return "a parent front is not above its child";
    if (S.front_off[s] < 0 || S.front_off[s] + fsize(s) * fsize(s) > S.arena_size)
      return "front " + std::to_string(s) + " outside the arena";
    born[S.level[s]].push_back(s);
    dies[last].push_back(s);
  }
  std::map<int64_t, std::pair<int64_t, int32_t>> live;   // offset -> (end, front)
  for (int l = 0; l < S.nlevels; ++l) {
    for (int s : born[l]) {
      int64_t a = S.front_off[s], b = a + padded(fsize(s) * fsize(s));
      auto it = live.lower_bound(a);
      if (it != live.end() && it->first < b)
        return "fronts " + std::to_string(s) + " and " + std::to_string(it->second.second) +
               " overlap in the arena";
      if (it != live.begin() && std::prev(it)->second.first > a)
        return "fronts " + std::to_string(s) + " and " +
               std::to_string(std::prev(it)->second.second) + " overlap in the arena";
      live[a] = {b, s};
    }
    for (int s : dies[l]) live.erase(S.front_off[s]);
  }
  // entries are assembled level by level (fronts of different levels may reuse memory)
  for (int l = 0; l < S.nlevels; ++l) {
    std::vector<int64_t> dst;
    for (int32_t k = S.lvl_slot_ptr[l]; k < S.lvl_slot_ptr[l + 1]; ++k)
      dst.push_back(S.asm_dst[S.lvl_slot[k]]);
    std::sort(dst.begin(), dst.end());
    for (size_t e = 0; e < dst.size(); ++e) {
      if (dst[e] < 0 || dst[e] >= S.arena_size) return "assembly target outside the arena";
      if (e > 0 && dst[e] == dst[e - 1])
        return "two entries of A assemble into one position at level " + std::to_string(l);
    }
  }
  if (S.lvl_slot_ptr[S.nlevels] != (int32_t)S.asm_dst.size()) return "assembly slots not covered";
  for (int s = 0; s < nsn; ++s) {
    int p = S.sn_parent[s];
    if (p < 0) continue;
    for (int64_t e = S.rptr[s]; e < S.rptr[s + 1]; ++e)
      if (S.rel[e] < 0 || S.rel[e] >= fsize(p))
        return "relative index of front " + std::to_string(s) + " outside its parent";
  }
  return "";
}

std::string check_minv_plan(const Symbolic& S) {
  const int64_t size[7] = {S.d_total, S.d_total, S.o_total, S.o_total, S.m_total, S.m_total,
                           S.mscratch};
  auto inside = [&](int arr, int64_t off, int64_t rows, int64_t cols, int64_t ld) {
    if (arr < 0 || arr > 6) return false;
    if (rows <= 0 || cols <= 0) return true;
    if (off < 0 || ld < rows) return false;
    return off + (cols - 1) * ld + rows <= size[arr];
  };
  for (size_t q = 0; q < S.mjobs.size(); ++q) {
    const MJob& j = S.mjobs[q];
    bool ok = true;
    if (j.kind == MJOB_COPY) {
      ok = inside(j.a_arr, j.a_off, j.m, j.n, j.lda) && inside(j.c_arr, j.c_off, j.m, j.n, j.ldc);
    } else if (j.kind == MJOB_COPYT) {
      ok = inside(j.a_arr, j.a_off, j.n, j.m, j.lda) && inside(j.c_arr, j.c_off, j.m, j.n, j.ldc);
    } else if (j.kind == MJOB_GEMM) {
      ok = inside(j.a_arr, j.a_off, j.m, j.k, j.lda) && inside(j.b_arr, j.b_off, j.k, j.n, j.ldb) &&
           inside(j.c_arr, j.c_off, j.m, j.n, j.ldc);
      if ((j.tri & (MTRI_A_LOWER | MTRI_A_UPPER)) && j.m != j.k) ok = false;
      if ((j.tri & (MTRI_B_LOWER | MTRI_B_UPPER)) && j.k != j.n) ok = false;
    } else {
      ok = false;
    }
    if (!ok) return "inversion job " + std::to_string(q) + " reaches outside its arrays";
  }
  // the tiles of every job cover its output grid exactly once, within one phase
  std::vector<int64_t> seen(S.mjobs.size(), 0), phase_of(S.mjobs.size(), -1);
  for (size_t ph = 0; ph + 1 < S.mphase_ptr.size(); ++ph)
    for (int32_t t = S.mphase_ptr[ph]; t < S.mphase_ptr[ph + 1]; ++t) {
      const int jid = S.mtile[2 * t], ti = S.mtile[2 * t + 1] >> 16, tj = S.mtile[2 * t + 1] & 0xffff;
      if (jid < 0 || jid >= (int)S.mjobs.size()) return "inversion tile of an unknown job";
      const MJob& j = S.mjobs[jid];
      if (ti * 64 >= j.m || tj * 64 >= j.n) return "inversion tile outside its job";
      if (phase_of[jid] >= 0 && phase_of[jid] != (int64_t)ph) return "inversion job split over phases";
      phase_of[jid] = (int64_t)ph;
      seen[jid]++;
    }
  for (size_t q = 0; q < S.mjobs.size(); ++q) {
    const MJob& j = S.mjobs[q];
    if (seen[q] != (int64_t)((j.m + 63) / 64) * ((j.n + 63) / 64))
      return "inversion job " + std::to_string(q) + " not covered by its tiles once";
  }
  return "";
}

std::string check_solve_plan(const Symbolic& S, int64_t counts[8]) {
  const int nsn = S.nsn;
  {
    std::string err = check_refactor_plan(S);
    if (!err.empty()) return "refactor plan: " + err;
    err = check_minv_plan(S);
    if (!err.empty()) return "merged-block plan: " + err;
  }
  for (int q = 0; q < 8; ++q) counts[q] = 0;
  counts[0] = (int64_t)S.fwd.size();
  counts[1] = (int64_t)S.bwd.size();
  auto nrows = [&](int s) { return (int)(S.rptr[s + 1] - S.rptr[s]); };
  // a forward unit updating rows [a, b) of supernode s must arrive at exactly the supernodes
  // that own those rows (else one could start before the update lands)
  std::vector<int32_t> owners, targets;
  auto targets_match = [&](int s, int a, int b, int32_t tgt0, int32_t ntgt) {
    owners.clear();
    for (int i = a; i < b; ++i) owners.push_back(S.sn_of[S.rows[S.rptr[s] + i]]);
    std::sort(owners.begin(), owners.end());
    owners.erase(std::unique(owners.begin(), owners.end()), owners.end());
    targets.assign(S.fwd_tgt.begin() + tgt0, S.fwd_tgt.begin() + tgt0 + ntgt);
    std::sort(targets.begin(), targets.end());
    return owners == targets;
  };
  // the row ranges of a supernode solved by a DIAG entry and far chunks, per direction
  std::vector<std::vector<std::pair<int, int>>> franges(nsn), branges(nsn);
  // rows of a merged piece before ext0(s) are the columns of the later pieces of its block
  auto ext0 = [&](int s) -> int {
    const int g = S.sn_grp[s];
    return g < 0 ? 0 : S.sn_start[S.grp_last[g] + 1] - S.sn_start[s + 1];
  };
  for (int g = 0; g < (int)S.grp_first.size(); ++g)
    for (int s = S.grp_first[g]; s < S.grp_last[g]; ++s)
      if (!nests(S, s)) return "merged block " + std::to_string(g) + " is not one triangle";
  auto partitions = [&](std::vector<std::pair<int, int>>& rg, int r, int at = 0) {
    std::sort(rg.begin(), rg.end());
    for (auto& q : rg) {
      if (q.second == q.first) continue;           // an empty range (a root without rows)
      if (q.first != at || q.second < q.first) return false;
      at = q.second;
    }
    return at == r;
  };
  // ---- forward: the entry computing each supernode, and the entries of every arrival
  std::vector<int64_t> fpos(nsn, -1);
  std::vector<int64_t> arrive_last(nsn, -1), arrive_cnt(nsn, 0);
  std::vector<int64_t> chunk_entry;   // entries holding far chunks, with their supernode
  std::vector<int32_t> chunk_sn;
  // merged pieces: column pieces covered by the MGEMV entries of each row tile, and the first
  // MGEMV entry that reads a piece's values
  std::vector<std::vector<int>> fcols(nsn), bcols(nsn);
  std::vector<int64_t> fread(nsn, INT64_MAX), bread(nsn, INT64_MAX), bgrp_last(S.grp_first.size(), -1);
  std::vector<int> fslots, bslots;
  auto mgemv_ok = [&](const SolveTask& T, bool fwd) -> std::string {
    const int g = T.grp;
    if (g < 0 || g >= (int)S.grp_first.size() || S.sn_grp[T.sn] != g) return "bad block";
    if (T.r0 >= T.r1 || S.sn_grp[T.r0] != g || S.sn_grp[T.r1 - 1] != g) return "columns outside the block";
    if (fwd ? (T.r1 - 1 > T.sn) : (T.r0 < T.sn)) return "columns outside the triangle";
    const int64_t W = S.grp_W[g], c0 = S.grp_c0[g];
    if (T.r != W || T.c0 != S.sn_start[T.sn] || T.w != S.sn_start[T.sn + 1] - S.sn_start[T.sn] ||
        T.o_off != S.sn_start[T.r0] || T.row_off != S.sn_start[T.r1] ||
        T.d_off != S.grp_moff[g] + (S.sn_start[T.sn] - c0) + (S.sn_start[T.r0] - c0) * W)
      return "descriptor";
    if (T.tgt0 < 0 || T.tgt0 >= S.nslots || T.wait_sn < 0 || T.wait_sn > T.tgt0 ||
        T.tgt0 >= T.wait_sn + T.wait_cnt)
      return "partial-sum slot";
    return "";
  };
  auto arrive = [&](int32_t tgt0, int32_t ntgt, int64_t e) {
    for (int q = 0; q < ntgt; ++q) {
      int t = S.fwd_tgt[tgt0 + q];
      arrive_last[t] = std::max(arrive_last[t], e);
      arrive_cnt[t]++;
    }
  };
  for (int64_t e = 0; e < (int64_t)S.fwd.size(); ++e) {
    const SolveTask& T = S.fwd[e];
    if (T.kind == TASK_DIAG) {
      if (fpos[T.sn] >= 0) return "forward: supernode computed twice";
      fpos[T.sn] = e;
      counts[6]++;
      arrive(T.tgt0, T.ntgt, e);
      franges[T.sn].push_back({T.r0, T.r1});
      if (!targets_match(T.sn, T.r0, T.r1, T.tgt0, T.ntgt))
        return "forward: targets of a DIAG entry differ from the owners of its rows";
    } else if (T.kind == TASK_GROUP || T.kind == TASK_BULK) {
      for (int w = 0; w < T.r0; ++w) {
        const SolveTask& U = S.fwd_small[T.sn + w];
        if (U.kind == TASK_FUSED) {
          if (fpos[U.sn] >= 0) return "forward: supernode computed twice";
          fpos[U.sn] = e;
          counts[4]++;
          arrive(U.tgt0, U.ntgt, e);
          if (!targets_match(U.sn, 0, nrows(U.sn), U.tgt0, U.ntgt))
            return "forward: targets of a warp task differ from the owners of its rows";
        } else if (U.kind == TASK_LANES) {
          for (int l = 0; l < U.r0; ++l) {
            const int32_t* it = S.fwd_lane.data() + 4 * ((int64_t)U.sn + l);
            if (fpos[it[0]] >= 0) return "forward: supernode computed twice";
            fpos[it[0]] = e;
            counts[2]++;
            arrive(it[1], it[2], e);
            if (!targets_match(it[0], 0, nrows(it[0]), it[1], it[2]))
              return "forward: targets of a lane item differ from the owners of its rows";
          }
        } else if (U.kind == TASK_OFF) {
          chunk_entry.push_back(e);
          chunk_sn.push_back(U.sn);
          arrive(U.tgt0, U.ntgt, e);
          franges[U.sn].push_back({U.r0, U.r1});
          if (!targets_match(U.sn, U.r0, U.r1, U.tgt0, U.ntgt))
            return "forward: targets of a far chunk differ from the owners of its rows";
        } else {
          return "forward: unknown warp task";
        }
      }
    } else if (T.kind == TASK_MGEMV) {
      std::string err = mgemv_ok(T, true);
      if (!err.empty()) return "forward: MGEMV " + err;
      fpos[T.sn] = std::max(fpos[T.sn], e);
      for (int j = T.r0; j < T.r1; ++j) {
        fcols[T.sn].push_back(j);
        fread[j] = std::min(fread[j], e);
      }
      fslots.push_back(T.tgt0);
    } else {
      return "forward: unknown entry";
    }
  }
  for (int s = 0; s < nsn; ++s) {
    const int g = S.sn_grp[s];
    if (g < 0) {
      if (!fcols[s].empty()) return "forward: MGEMV for a supernode outside a block";
      continue;
    }
    counts[6]++;    // a merged piece is solved by CTA entries (its row tile's MGEMV tasks)
    std::sort(fcols[s].begin(), fcols[s].end());
    for (int j = S.grp_first[g]; j <= s; ++j)
      if (fcols[s].size() != (size_t)(s - S.grp_first[g] + 1) || fcols[s][j - S.grp_first[g]] != j)
        return "forward: row tile " + std::to_string(s) + " does not cover its columns once";
    if (arrive_last[s] >= fread[s]) return "forward: an arrival comes after an MGEMV read";
  }
  std::sort(fslots.begin(), fslots.end());
  for (size_t q = 1; q < fslots.size(); ++q)
    if (fslots[q] == fslots[q - 1]) return "forward: two MGEMV entries share a slot";
  for (int s = 0; s < nsn; ++s) {
    if (fpos[s] < 0) return "forward: supernode " + std::to_string(s) + " never computed";
    if (arrive_cnt[s] != S.fwd_expect[s]) return "forward: arrival count mismatch";
    if (arrive_last[s] >= fpos[s]) return "forward: an arrival comes after the wait";
  }
  for (size_t q = 0; q < chunk_entry.size(); ++q)
    if (fpos[chunk_sn[q]] >= chunk_entry[q]) return "forward: far chunk before its DIAG";
  for (int s = 0; s < nsn; ++s)
    if ((!franges[s].empty() || (S.sn_grp[s] >= 0 && ext0(s) < nrows(s))) &&
        !partitions(franges[s], nrows(s), ext0(s)))
      return "forward: the row chunks of supernode " + std::to_string(s) +
             " do not cover its rows exactly once";
  // ---- backward
  // a backward unit reading x over rows [a, b) of supernode s must wait for the owner of the
  // smallest of those rows: its nearest ancestor among them (each supernode completes only
  // after its parent, so that owner's completion implies every higher owner's)
  auto wait_matches = [&](int s, int a, int b, int32_t wait_sn) {
    if (a >= b) return true;
    return wait_sn == S.sn_of[S.rows[S.rptr[s] + a]];
  };
  std::vector<int64_t> bpos(nsn, -1), chunks_last(nsn, -1), chunks_cnt(nsn, 0);
  struct Wait { int64_t e; int32_t on; };
  std::vector<Wait> waits;
  for (int64_t e = 0; e < (int64_t)S.bwd.size(); ++e) {
    const SolveTask& T = S.bwd[e];
    if (T.kind == TASK_DIAG) {
      if (bpos[T.sn] >= 0) return "backward: supernode computed twice";
      bpos[T.sn] = e;
      counts[7]++;
      branges[T.sn].push_back({T.r0, T.r1});
      if (!wait_matches(T.sn, T.r0, T.r1, T.wait_sn))
        return "backward: a DIAG entry waits on the wrong supernode";
      if (T.wait_sn >= 0) waits.push_back({e, T.wait_sn});
    } else if (T.kind == TASK_GROUP || T.kind == TASK_BULK) {
      for (int w = 0; w < T.r0; ++w) {
        const SolveTask& U = S.bwd_small[T.sn + w];
        if (U.kind == TASK_FUSED) {
          if (bpos[U.sn] >= 0) return "backward: supernode computed twice";
          bpos[U.sn] = e;
          counts[5]++;
          if (!wait_matches(U.sn, 0, nrows(U.sn), U.wait_sn))
            return "backward: a warp task waits on the wrong supernode";
          if (U.wait_sn >= 0) waits.push_back({e, U.wait_sn});
        } else if (U.kind == TASK_LANES) {
          for (int l = 0; l < U.r0; ++l) {
            const int32_t* it = S.bwd_lane.data() + 4 * ((int64_t)U.sn + l);
            if (bpos[it[0]] >= 0) return "backward: supernode computed twice";
            bpos[it[0]] = e;
            counts[3]++;
            if (!wait_matches(it[0], 0, nrows(it[0]), it[1]))
              return "backward: a lane item waits on the wrong supernode";
            if (it[1] >= 0) waits.push_back({e, it[1]});
          }
        } else if (U.kind == TASK_OFF) {
          chunks_last[U.sn] = std::max(chunks_last[U.sn], e);
          chunks_cnt[U.sn]++;
          branges[U.sn].push_back({U.r0, U.r1});
          if (!wait_matches(U.sn, U.r0, U.r1, U.wait_sn))
            return "backward: a far chunk waits on the wrong supernode";
          if (U.wait_sn >= 0) waits.push_back({e, U.wait_sn});
        } else {
          return "backward: unknown warp task";
        }
      }
    } else if (T.kind == TASK_MGEMV) {
      std::string err = mgemv_ok(T, false);
      if (!err.empty()) return "backward: MGEMV " + err;
      bgrp_last[T.grp] = std::max(bgrp_last[T.grp], e);
      for (int j = T.r0; j < T.r1; ++j) {
        bcols[T.sn].push_back(j);
        bread[j] = std::min(bread[j], e);
      }
      bslots.push_back(T.tgt0);
    } else {
      return "backward: unknown entry";
    }
  }
  // a merged block's pieces complete together, with its last MGEMV entry
  for (int s = 0; s < nsn; ++s) {
    const int g = S.sn_grp[s];
    if (g < 0) {
      if (!bcols[s].empty()) return "backward: MGEMV for a supernode outside a block";
      continue;
    }
    if (bpos[s] >= 0) return "backward: a merged piece has its own entry";
    bpos[s] = bgrp_last[g];
    counts[7]++;
    std::sort(bcols[s].begin(), bcols[s].end());
    if (bcols[s].size() != (size_t)(S.grp_last[g] - s + 1))
      return "backward: row tile " + std::to_string(s) + " does not cover its columns once";
    for (size_t q = 0; q < bcols[s].size(); ++q)
      if (bcols[s][q] != s + (int)q)
        return "backward: row tile " + std::to_string(s) + " does not cover its columns once";
    if (chunks_last[s] >= bread[s]) return "backward: a far chunk comes after an MGEMV read";
  }
  std::sort(bslots.begin(), bslots.end());
  for (size_t q = 1; q < bslots.size(); ++q)
    if (bslots[q] == bslots[q - 1]) return "backward: two MGEMV entries share a slot";
  for (int s = 0; s < nsn; ++s) {
    if (bpos[s] < 0) return "backward: supernode " + std::to_string(s) + " never computed";
    if (chunks_cnt[s] != S.bwd_nchunk[s]) return "backward: chunk count mismatch";
    if (chunks_last[s] >= bpos[s]) return "backward: a far chunk comes after its DIAG";
    if ((!branges[s].empty() || (S.sn_grp[s] >= 0 && ext0(s) < nrows(s))) &&
        !partitions(branges[s], nrows(s), ext0(s)))
      return "backward: the row chunks of supernode " + std::to_string(s) +
             " do not cover its rows exactly once";
  }
  for (const Wait& w : waits)
    if (bpos[w.on] >= w.e) return "backward: a wait refers to a later entry";
  return "";
}
}  // namespace ers
