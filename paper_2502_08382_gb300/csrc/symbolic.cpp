// Host symbolic analysis: ordering, elimination tree, supernodes and the
// multifrontal / pruned-RHS / SYRK-tile plans.  See symbolic.h.
#include "symbolic.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <stdexcept>

namespace feti {

namespace {

// ------------------------------------------------------------------ graph

struct Graph {  // compressed (node-level) adjacency without self loops
  int nv = 0;
  std::vector<int> off, adj;
  std::vector<int> dof0, ndof;  // first DOF and DOF count of each node
};

bool same_row(const int64_t* rp, const int32_t* col, int a, int b) {
  int64_t la = rp[a + 1] - rp[a], lb = rp[b + 1] - rp[b];
  if (la != lb) return false;
  return std::memcmp(col + rp[a], col + rp[b], sizeof(int32_t) * la) == 0;
}

Graph compress(int n, const int64_t* rp, const int32_t* col) {
  Graph g;
  std::vector<int> node_of(n);
  for (int d = 0; d < n; ++d) {
    if (d > 0 && same_row(rp, col, d, d - 1)) {
      node_of[d] = node_of[d - 1];
      g.ndof.back()++;
    } else {
      node_of[d] = g.nv++;
      g.dof0.push_back(d);
      g.ndof.push_back(1);
    }
  }
  g.off.assign(g.nv + 1, 0);
  std::vector<int> tmp;
  std::vector<std::vector<int>> nb(g.nv);
  for (int v = 0; v < g.nv; ++v) {
    int d = g.dof0[v];
    tmp.clear();
    for (int64_t k = rp[d]; k < rp[d + 1]; ++k) {
      int u = node_of[col[k]];
      if (u != v) tmp.push_back(u);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    nb[v] = tmp;
    g.off[v + 1] = g.off[v] + (int)tmp.size();
  }
  g.adj.reserve(g.off[g.nv]);
  for (int v = 0; v < g.nv; ++v) g.adj.insert(g.adj.end(), nb[v].begin(), nb[v].end());
  return g;
}

// ------------------------------------------------------------------ nested dissection

struct ND {
  const Graph& g;
  const double* xyz;  // per node, 3 coords (may be null)
  int leaf;
  std::vector<int> stamp;
  int cur = 0;
  std::vector<int> order;
  std::vector<int> level;

  ND(const Graph& g_, const double* xyz_, int leaf_) : g(g_), xyz(xyz_), leaf(leaf_) {
    stamp.assign(g.nv, -1);
    level.assign(g.nv, -1);
  }

  // BFS inside the vertex set marked with `mark`; returns vertices in BFS order and fills level[].
  void bfs(int src, int mark, std::vector<int>& q) {
    q.clear();
    q.push_back(src);
    level[src] = 0;
    int stamp_id = ++cur;  // visited marker (separate from set mark)
    std::vector<int>& vis = visited_;
    if ((int)vis.size() < g.nv) vis.assign(g.nv, -1);
    vis[src] = stamp_id;
    for (size_t h = 0; h < q.size(); ++h) {
      int v = q[h];
      for (int k = g.off[v]; k < g.off[v + 1]; ++k) {
        int u = g.adj[k];
        if (stamp[u] == mark && vis[u] != stamp_id) {
          vis[u] = stamp_id;
          level[u] = level[v] + 1;
          q.push_back(u);
        }
      }
    }
  }
  std::vector<int> visited_;

  // Split V into (A, B, S) with no edge between A and B.  Returns false if no useful split.
  bool split(const std::vector<int>& V, std::vector<int>& A, std::vector<int>& B, std::vector<int>& S) {
    int mark = ++cur;
    for (int v : V) stamp[v] = mark;
    A.clear(); B.clear(); S.clear();
    if (xyz) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int v : V)
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], xyz[3 * v + a]);
          hi[a] = std::max(hi[a], xyz[3 * v + a]);
        }
      int ax = 0;
      for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
      if (hi[ax] > lo[ax]) {
        std::vector<double> vals;
        vals.reserve(V.size());
        for (int v : V) vals.push_back(xyz[3 * v + ax]);
        std::nth_element(vals.begin(), vals.begin() + vals.size() / 2, vals.end());
        double cm = vals[vals.size() / 2];
        int markA = ++cur;
        std::vector<int> Bs;
        for (int v : V) {
          if (xyz[3 * v + ax] < cm) { A.push_back(v); stamp[v] = markA; }
          else Bs.push_back(v);
        }
        if (!A.empty() && !Bs.empty()) {
          for (int v : Bs) {
            bool touch = false;
            for (int k = g.off[v]; k < g.off[v + 1] && !touch; ++k) touch = stamp[g.adj[k]] == markA;
            (touch ? S : B).push_back(v);
          }
          for (int v : V) stamp[v] = -1;
          return true;
        }
        A.clear();
        for (int v : V) stamp[v] = mark;
      }
    }
    // BFS level structure from a pseudo-peripheral vertex
    std::vector<int> q;
    int src = V[0];
    bfs(src, mark, q);
    if (q.size() < V.size()) {
      // disconnected: first component vs the rest, empty separator
      int mk = ++cur;
      for (int v : q) stamp[v] = mk;
      for (int v : V) (stamp[v] == mk ? A : B).push_back(v);
      for (int v : V) stamp[v] = -1;
      return true;
    }
    for (int it = 0; it < 4; ++it) {
      int far = q.back();
      int ecc = level[far];
      bfs(far, mark, q);
      if (level[q.back()] <= ecc) break;
    }
    int nlev = level[q.back()] + 1;
    if (nlev < 3) {
      for (int v : V) stamp[v] = -1;
      return false;
    }
    std::vector<int> cnt(nlev, 0);
    for (int v : q) cnt[level[v]]++;
    int half = (int)V.size() / 2, acc = 0, k = 0;
    for (k = 0; k < nlev; ++k) {
      acc += cnt[k];
      if (acc >= half) break;
    }
    k = std::max(1, std::min(k, nlev - 2));
    for (int v : q) {
      if (level[v] < k) A.push_back(v);
      else if (level[v] == k) S.push_back(v);
      else B.push_back(v);
    }
    for (int v : V) stamp[v] = -1;
    return true;
  }

  int dofs(const std::vector<int>& V) const {
    int s = 0;
    for (int v : V) s += g.ndof[v];
    return s;
  }

  void run(std::vector<int> V) {
    if (V.empty()) return;
    if (dofs(V) <= leaf || V.size() <= 2) {
      std::sort(V.begin(), V.end());
      order.insert(order.end(), V.begin(), V.end());
      return;
    }
    std::vector<int> A, B, S;
    if (!split(V, A, B, S)) {
      std::sort(V.begin(), V.end());
      order.insert(order.end(), V.begin(), V.end());
      return;
    }
    run(std::move(A));
    run(std::move(B));
    std::sort(S.begin(), S.end());
    order.insert(order.end(), S.begin(), S.end());
  }
};

}  // namespace

uint64_t hash_ints(const int32_t* a, int64_t n, uint64_t h) {
  h ^= 0x9E3779B97F4A7C15ull + (uint64_t)n;
  for (int64_t i = 0; i < n; ++i) {
    h ^= (uint64_t)(uint32_t)a[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  }
  return h;
}

uint64_t hash_pattern(int n, const int64_t* rowptr, const int32_t* col) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)n;
  for (int i = 0; i <= n; ++i) h = (h ^ (uint64_t)rowptr[i]) * 1099511628211ull;
  return hash_ints(col, rowptr[n], h);
}

void analyse_pattern(int n, const int64_t* rp, const int32_t* col, const double* coords,
                     const SymbolicOptions& opt, PatternPlan& P, const int32_t* last, int nlast) {
  P = PatternPlan();
  P.n = n;
  // ---------------- ordering on the compressed graph
  Graph g = compress(n, rp, col);
  std::vector<double> xyz;
  if (coords && opt.use_coords) {
    xyz.resize(3 * (size_t)g.nv);
    for (int v = 0; v < g.nv; ++v)
      for (int a = 0; a < 3; ++a) xyz[3 * v + a] = coords[3 * (size_t)g.dof0[v] + a];
  }
  ND nd(g, xyz.empty() ? nullptr : xyz.data(), opt.leaf_dofs);
  std::vector<char> is_last(g.nv, 0);
  if (last && nlast > 0) {
    std::vector<int> node_of(n);
    for (int v = 0; v < g.nv; ++v)
      for (int k = 0; k < g.ndof[v]; ++k) node_of[g.dof0[v] + k] = v;
    for (int k = 0; k < nlast; ++k) {
      if (last[k] < 0 || last[k] >= n) throw std::runtime_error("a DOF to order last is out of range");
      is_last[node_of[last[k]]] = 1;
    }
  }
  {
    std::vector<int> rest, tail;
    for (int v = 0; v < g.nv; ++v) (is_last[v] ? tail : rest).push_back(v);
    nd.run(std::move(rest));
    nd.order.insert(nd.order.end(), tail.begin(), tail.end());
  }
  std::vector<int> perm0;
  perm0.reserve(n);
  int n_tail = 0;
  for (int v : nd.order)
    for (int k = 0; k < g.ndof[v]; ++k) {
      perm0.push_back(g.dof0[v] + k);
      n_tail += is_last[v] ? 1 : 0;
    }
  if ((int)perm0.size() != n) throw std::runtime_error("ordering lost DOFs");
  P.nlast = n_tail;

  // ---------------- elimination tree (Liu) in perm0 numbering
  auto etree_of = [&](const std::vector<int>& perm, const std::vector<int>& iperm, std::vector<int>& parent) {
    parent.assign(n, -1);
    std::vector<int> anc(n, -1);
    for (int j = 0; j < n; ++j) {
      int r = perm[j];
      for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
        int i = iperm[col[k]];
        if (i >= j) continue;
        // walk from i to the root of its current subtree
        while (i != -1 && i < j) {
          int nx = anc[i];
          anc[i] = j;
          if (nx == -1) {
            parent[i] = j;
            break;
          }
          i = nx;
        }
      }
    }
  };
  std::vector<int> iperm0(n);
  for (int j = 0; j < n; ++j) iperm0[perm0[j]] = j;
  std::vector<int> par0;
  etree_of(perm0, iperm0, par0);

  // ---------------- postorder
  std::vector<int> head(n, -1), next(n, -1), post;
  post.reserve(n);
  for (int j = n - 1; j >= 0; --j) {
    if (par0[j] != -1) {
      next[j] = head[par0[j]];
      head[par0[j]] = j;
    }
  }
  {
    std::vector<int> stk;
    for (int j = 0; j < n; ++j) {
      if (par0[j] != -1) continue;
      stk.push_back(j);
      while (!stk.empty()) {
        int v = stk.back();
        int c = head[v];
        if (c == -1) {
          post.push_back(v);
          stk.pop_back();
        } else {
          head[v] = next[c];
          stk.push_back(c);
        }
      }
    }
  }
  P.perm.resize(n);
  for (int k = 0; k < n; ++k) P.perm[k] = perm0[post[k]];
  P.iperm.resize(n);
  for (int k = 0; k < n; ++k) P.iperm[P.perm[k]] = k;
  std::vector<int> parent;
  etree_of(P.perm, P.iperm, parent);

  // ---------------- column counts (row subtrees)
  std::vector<int> cc(n, 1), mark(n, -1), nchild(n, 0);
  for (int j = 0; j < n; ++j)
    if (parent[j] != -1) nchild[parent[j]]++;
  for (int i = 0; i < n; ++i) {
    int r = P.perm[i];
    mark[i] = i;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
      int j = P.iperm[col[k]];
      if (j >= i) continue;
      while (j != -1 && mark[j] != i) {
        cc[j]++;
        mark[j] = i;
        j = parent[j];
      }
    }
  }

  // ---------------- fundamental supernodes
  // (the trailing n_tail columns, the DOFs ordered last, are the etree's top: one supernode)
  std::vector<int> sc0;  // first column of each supernode
  for (int j = 0; j < n; ++j) {
    bool merge = j > 0 && parent[j - 1] == j && cc[j - 1] == cc[j] + 1 && nchild[j] == 1;
    if (n_tail > 0 && j >= n - n_tail) merge = j > n - n_tail;
    if (!merge) sc0.push_back(j);
  }
  if (n_tail > 0)
    for (int j = n - n_tail; j + 1 < n; ++j)
      if (parent[j] != j + 1) throw std::runtime_error("the DOFs ordered last do not form the top of the tree");
  int ns0 = (int)sc0.size();
  std::vector<int> w0(ns0), f0(ns0), col2sn0(n), spar0(ns0, -1);
  for (int s = 0; s < ns0; ++s) {
    int c1 = (s + 1 < ns0) ? sc0[s + 1] : n;
    w0[s] = c1 - sc0[s];
    f0[s] = cc[sc0[s]];
    for (int j = sc0[s]; j < c1; ++j) col2sn0[j] = s;
  }
  for (int s = 0; s < ns0; ++s) {
    int last = sc0[s] + w0[s] - 1;
    if (parent[last] != -1) spar0[s] = col2sn0[parent[last]];
  }

  // ---------------- relaxed amalgamation (merge a supernode into its parent
  // when it is the parent's contiguous last child and few zeros are added)
  std::vector<int> rep(ns0);  // union-find: merged supernode -> surviving parent
  std::iota(rep.begin(), rep.end(), 0);
  auto find = [&](int x) {
    int r = x;
    while (rep[r] != r) r = rep[r];
    while (rep[x] != r) {
      int nx = rep[x];
      rep[x] = r;
      x = nx;
    }
    return r;
  };
  std::vector<int> gw(w0), gf(f0), gc0(sc0);
  std::vector<double> gnz(ns0);
  auto nzof = [](double w, double f) { return w * f - w * (w - 1) / 2.0; };
  for (int s = 0; s < ns0; ++s) gnz[s] = nzof(w0[s], f0[s]);
  std::vector<char> alive(ns0, 1);
  for (int p = 0; p < ns0; ++p) {
    // candidate: the supernode ending right before p's first column (p's last child in postorder)
    while (gc0[p] > 0) {
      if (n_tail > 0 && gc0[p] >= n - n_tail) break;  // nothing is merged into the forced root
      int s = find(col2sn0[gc0[p] - 1]);
      if (!alive[s] || s == p) break;
      if (spar0[s] < 0 || find(spar0[s]) != p) break;
      double wm = gw[s] + gw[p];
      double fm = gw[s] + gf[p];
      double nzm = nzof(wm, fm);
      double zeros = nzm - gnz[s] - gnz[p];
      double frac = zeros / nzm;
      bool ok = (wm <= 4) || (wm <= 16 && frac < 0.8) || (wm <= 48 && frac < 0.1) || (frac < 0.05);
      if (!ok) break;
      alive[s] = 0;
      rep[s] = p;
      gc0[p] = gc0[s];
      gw[p] = (int)wm;
      gf[p] = (int)fm;
      gnz[p] = nzm;
    }
  }
  // final supernodes in column order (postorder preserved)
  std::vector<int> fin;
  for (int s = 0; s < ns0; ++s)
    if (alive[s]) fin.push_back(s);
  std::sort(fin.begin(), fin.end(), [&](int a, int b) { return gc0[a] < gc0[b]; });
  int ns = (int)fin.size();
  P.nsn = ns;
  P.sn_c0.resize(ns);
  P.sn_w.resize(ns);
  P.col2sn.resize(n);
  for (int s = 0; s < ns; ++s) {
    P.sn_c0[s] = gc0[fin[s]];
    P.sn_w[s] = gw[fin[s]];
    for (int j = P.sn_c0[s]; j < P.sn_c0[s] + P.sn_w[s]; ++j) P.col2sn[j] = s;
  }
  for (int s = 0; s + 1 < ns; ++s)
    if (P.sn_c0[s] + P.sn_w[s] != P.sn_c0[s + 1]) throw std::runtime_error("supernodes not contiguous");

  // ---------------- supernodal row structures (below the diagonal block)
  std::vector<std::vector<int>> below(ns);
  std::vector<std::vector<int>> kids(ns);
  P.sn_parent.assign(ns, -1);
  {
    std::vector<int> buf;
    for (int s = 0; s < ns; ++s) {
      int c0 = P.sn_c0[s], c1 = c0 + P.sn_w[s];
      buf.clear();
      for (int j = c0; j < c1; ++j) {
        int r = P.perm[j];
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
          int i = P.iperm[col[k]];
          if (i >= c1) buf.push_back(i);
        }
      }
      for (int c : kids[s])
        for (int i : below[c])
          if (i >= c1) buf.push_back(i);
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      below[s] = buf;
      if (!buf.empty()) {
        int p = P.col2sn[buf[0]];
        P.sn_parent[s] = p;
        kids[p].push_back(s);
      }
    }
  }
  P.sn_r.resize(ns);
  P.sn_rows_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) {
    P.sn_r[s] = (int)below[s].size();
    P.sn_rows_off[s + 1] = P.sn_rows_off[s] + P.sn_r[s];
  }
  P.rows.reserve(P.sn_rows_off[ns]);
  for (int s = 0; s < ns; ++s) P.rows.insert(P.rows.end(), below[s].begin(), below[s].end());
  P.ch_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) P.ch_off[s + 1] = P.ch_off[s] + (int)kids[s].size();
  for (int s = 0; s < ns; ++s) P.ch_list.insert(P.ch_list.end(), kids[s].begin(), kids[s].end());
  // first descendant (postorder: subtree = [first_desc, s])
  P.sn_first_desc.resize(ns);
  for (int s = 0; s < ns; ++s) {
    int fd = s;
    for (int c : kids[s]) fd = std::min(fd, P.sn_first_desc[c]);
    P.sn_first_desc[s] = fd;
  }
  // position of a row inside the front of supernode s
  auto front_pos = [&](int s, int i) -> int {
    int c0 = P.sn_c0[s], w = P.sn_w[s];
    if (i >= c0 && i < c0 + w) return i - c0;
    const int* b = P.rows.data() + P.sn_rows_off[s];
    const int* e = P.rows.data() + P.sn_rows_off[s + 1];
    const int* it = std::lower_bound(b, e, i);
    if (it == e || *it != i) throw std::runtime_error("row missing from parent front");
    return w + (int)(it - b);
  };
  // extend-add maps
  P.rel_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) P.rel_off[s + 1] = P.rel_off[s] + (P.sn_parent[s] >= 0 ? P.sn_r[s] : 0);
  P.rel.resize(P.rel_off[ns]);
  for (int s = 0; s < ns; ++s) {
    int p = P.sn_parent[s];
    if (p < 0) continue;
    for (int k = 0; k < P.sn_r[s]; ++k) P.rel[P.rel_off[s] + k] = front_pos(p, below[s][k]);
  }
  // L storage and statistics
  P.Lofs.resize(ns);
  int64_t L = 0;
  double fl = 0;
  for (int s = 0; s < ns; ++s) {
    int w = P.sn_w[s], f = w + P.sn_r[s];
    P.Lofs[s] = L;
    L += (int64_t)f * w;
    P.max_f = std::max(P.max_f, f);
    P.max_w = std::max(P.max_w, w);
    P.nnzL += (double)w * f - (double)w * (w - 1) / 2;
    for (int k = 0; k < w; ++k) {
      double rem = f - k - 1;
      fl += 1 + rem + rem * (rem + 1);
    }
  }
  P.Lsize = L;
  P.chol_flops = fl;
  // K assembly map
  P.kmap_off.assign(ns + 1, 0);
  {
    std::vector<std::vector<std::pair<int, int>>> per(ns);
    for (int j = 0; j < n; ++j) {
      int s = P.col2sn[j];
      int r = P.perm[j];
      int f = P.sn_w[s] + P.sn_r[s];
      for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
        int i = P.iperm[col[k]];
        if (i < j) continue;
        int pos = front_pos(s, i);
        int64_t dst = P.Lofs[s] + (int64_t)(j - P.sn_c0[s]) * f + pos;
        per[s].push_back({(int)k, (int)dst});
      }
    }
    for (int s = 0; s < ns; ++s) {
      std::sort(per[s].begin(), per[s].end(), [](auto a, auto b) { return a.second < b.second; });
      P.kmap_off[s + 1] = P.kmap_off[s] + (int64_t)per[s].size();
      for (auto& e : per[s]) {
        P.kmap_src.push_back(e.first);
        P.kmap_dst.push_back(e.second);
      }
    }
  }
  P.diag_src.resize(n);
  for (int r = 0; r < n; ++r) {
    P.diag_src[r] = -1;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
      if (col[k] == r) P.diag_src[r] = (int)k;
    if (P.diag_src[r] < 0) throw std::runtime_error("K has a structurally zero diagonal");
  }
  // level schedule (height: leaves 0, parent = 1 + max child) and update vectors
  {
    std::vector<int> ht(ns, 0);
    for (int s = 0; s < ns; ++s)
      for (int c : kids[s]) ht[s] = std::max(ht[s], ht[c] + 1);
    P.nlev = 0;
    for (int s = 0; s < ns; ++s) P.nlev = std::max(P.nlev, ht[s] + 1);
    std::vector<std::vector<int>> lv(P.nlev);
    for (int s = 0; s < ns; ++s) lv[ht[s]].push_back(s);
    P.lvl_off.assign(P.nlev + 1, 0);
    for (int l = 0; l < P.nlev; ++l) {
      std::stable_sort(lv[l].begin(), lv[l].end(), [&](int a, int b) {
        return (int64_t)P.sn_w[a] * (P.sn_w[a] + P.sn_r[a]) < (int64_t)P.sn_w[b] * (P.sn_w[b] + P.sn_r[b]);
      });
      P.lvl_off[l + 1] = P.lvl_off[l] + (int)lv[l].size();
      P.lvl_sn.insert(P.lvl_sn.end(), lv[l].begin(), lv[l].end());
    }
    P.uofs.assign(ns, 0);
    int64_t u = 0;
    for (int s = 0; s < ns; ++s) {
      P.uofs[s] = u;
      u += P.sn_r[s];
    }
    P.usize = u;
  }
  // multifrontal update stack (postorder => children's blocks sit on top)
  P.upd_stack_ofs.assign(ns, 0);
  {
    int64_t top = 0, peak = 0, fr = 0;
    std::vector<int64_t> size(ns);
    for (int s = 0; s < ns; ++s) {
      int64_t base = top;
      for (int c : kids[s]) base -= size[c];
      int r = P.sn_r[s];
      size[s] = (P.sn_parent[s] >= 0) ? (int64_t)r * r : 0;
      fr = std::max(fr, (int64_t)r * r);
      P.upd_stack_ofs[s] = base;
      top = base + size[s];
      peak = std::max(peak, top);
    }
    P.chol_stack = peak;
    P.chol_front = fr;
  }
  // small subtrees: factored level by level, one warp per front, so an update block cannot live on the
  // postorder stack.  A block is written at its supernode's level and read at its parent's (levels are
  // separated by a CTA barrier), or in phase 2 when the parent is not small; slots are assigned first-fit at
  // the level a block is written, reusing the space of blocks whose readers ran at an earlier level, so the
  // small region holds the live blocks only (and stays in L2)
  P.sn_small.assign(ns, 0);
  P.usm_ofs.assign(ns, 0);
  {
    for (int s = 0; s < ns; ++s) {  // postorder: children first
      bool sm = P.sn_w[s] + P.sn_r[s] <= kSmallFront;
      for (int c : kids[s]) sm = sm && P.sn_small[c] != 0;
      P.sn_small[s] = sm ? 1 : 0;
    }
    std::vector<int> ht(ns, 0);
    for (int s = 0; s < ns; ++s)
      for (int c : kids[s]) ht[s] = std::max(ht[s], ht[c] + 1);
    const int nl = P.nlev;
    std::vector<std::vector<int>> born(nl), dies(nl + 1);
    for (int s = 0; s < ns; ++s)
      if (P.sn_small[s] && P.sn_parent[s] >= 0) {
        born[ht[s]].push_back(s);
        const int pr = P.sn_parent[s];
        dies[P.sn_small[pr] ? ht[pr] : nl].push_back(s);  // nl: read in phase 2, never freed
      }
    std::map<int64_t, int64_t> freel;  // offset -> size of free intervals
    int64_t top = 0;
    auto release = [&](int64_t o, int64_t sz) {
      auto it = freel.emplace(o, sz).first;
      auto nx = std::next(it);
      if (nx != freel.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        freel.erase(nx);
      }
      if (it != freel.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
          pv->second += it->second;
          freel.erase(it);
        }
      }
    };
    for (int l = 0; l < nl; ++l) {
      if (l > 0)
        for (int s : dies[l - 1]) release(P.usm_ofs[s], (int64_t)P.sn_r[s] * P.sn_r[s]);
      for (int s : born[l]) {
        const int64_t sz = (int64_t)P.sn_r[s] * P.sn_r[s];
        auto it = freel.begin();
        while (it != freel.end() && it->second < sz) ++it;
        if (it != freel.end()) {
          P.usm_ofs[s] = it->first;
          const int64_t o = it->first + sz, rest = it->second - sz;
          freel.erase(it);
          if (rest > 0) freel.emplace(o, rest);
        } else {
          P.usm_ofs[s] = top;
          top += sz;
        }
      }
    }
    P.usm_size = top;
  }
}

void plan_tasks(PatternPlan& P, double target, int big_f) {
  const int ns = P.nsn;
  std::vector<double> own(ns, 0.0), sub(ns, 0.0);
  for (int s = 0; s < ns; ++s) {
    const double w = P.sn_w[s], f = w + P.sn_r[s];
    double fl = 0;
    for (int k = 0; k < (int)w; ++k) {
      const double rem = f - k - 1;
      fl += 1 + rem + rem * (rem + 1);
    }
    own[s] = fl;
  }
  for (int s = 0; s < ns; ++s) {  // postorder: children first
    sub[s] += own[s];
    if (P.sn_parent[s] >= 0) sub[P.sn_parent[s]] += sub[s];
  }
  // the large fronts (at least big_f wide) and all their ancestors: the top of the tree, factored by the
  // tensor-core kernel after everything below it
  P.sn_big.assign(ns, 0);
  P.has_big = false;
  if (big_f > 0) {
    for (int s = 0; s < ns; ++s) {  // postorder: a supernode is seen before its parent
      if (!P.sn_small[s] && P.sn_w[s] + P.sn_r[s] >= big_f) P.sn_big[s] = 1;
      if (P.sn_big[s] && P.sn_parent[s] >= 0) P.sn_big[P.sn_parent[s]] = 1;
    }
    for (int s = 0; s < ns; ++s) P.has_big = P.has_big || P.sn_big[s];
  }
  P.sn_task.assign(ns, 0);
  P.sn_hoff.assign(ns, -1);
  P.task_parent.assign(1, -1);
  P.task_cost.assign(1, 0.0);
  P.hsize = 0;
  // from the roots down (reverse postorder): a non-small supernode with a heavy subtree and a parent starts a
  // task of its own below its parent's task, and so does every supernode outside the large set whose parent
  // is in it (the large set's tasks are factored by another kernel, after the others: their children hand their
  // update blocks over); everything else joins its parent's task.  A task is large if its root is.
  for (int s = ns - 1; s >= 0; --s) {
    const int p = P.sn_parent[s];
    if (p < 0) {
      P.sn_task[s] = 0;
    } else if ((P.sn_big[p] && !P.sn_big[s]) ||
               (target > 0 && !P.sn_small[s] && sub[s] > target && P.sn_r[s] > 0)) {
      const int t = (int)P.task_parent.size();
      P.task_parent.push_back(P.sn_task[p]);
      P.task_cost.push_back(0.0);
      P.sn_task[s] = t;
      P.sn_hoff[s] = P.hsize;
      P.hsize += (int64_t)P.sn_r[s] * P.sn_r[s];
    } else {
      P.sn_task[s] = P.sn_task[p];
    }
    P.task_cost[P.sn_task[s]] += own[s];
  }
  P.ntask = (int)P.task_parent.size();
  P.task_nchild.assign(P.ntask, 0);
  P.task_height.assign(P.ntask, 0);
  P.task_big.assign(P.ntask, 0);
  P.task_nbig.assign(P.ntask, 0);
  for (int s = 0; s < ns; ++s)
    if (P.sn_big[s]) P.task_big[P.sn_task[s]] = 1;  // a task holds large supernodes only or none
  for (int t = 1; t < P.ntask; ++t) {
    P.task_nchild[P.task_parent[t]]++;
    if (P.task_big[t]) P.task_nbig[P.task_parent[t]]++;
  }
  // tasks are numbered parents first, so heights follow from the highest numbers down
  for (int t = P.ntask - 1; t >= 1; --t)
    P.task_height[P.task_parent[t]] = std::max(P.task_height[P.task_parent[t]], P.task_height[t] + 1);
}

void plan_rhs(const PatternPlan& P, int m, const int32_t* B_dof, BPlan& Bp) {
  Bp = BPlan();
  Bp.m = m;
  Bp.nb = (m + kTile - 1) / kTile;
  Bp.m_pad = Bp.nb * kTile;
  int ns = P.nsn;
  // sort columns by (supernode of s_j, s_j, original row)
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<int> sp(m);
  for (int r = 0; r < m; ++r) {
    if (B_dof[r] < 0 || B_dof[r] >= P.n) throw std::runtime_error("B row touches a DOF out of range");
    sp[r] = P.iperm[B_dof[r]];
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    int sa = P.col2sn[sp[a]], sb = P.col2sn[sp[b]];
    if (sa != sb) return sa < sb;
    if (sp[a] != sp[b]) return sp[a] < sp[b];
    return a < b;
  });
  Bp.colperm = idx;
  Bp.spos.resize(m);
  std::vector<int> csn(m);
  for (int j = 0; j < m; ++j) {
    Bp.spos[j] = sp[idx[j]];
    csn[j] = P.col2sn[Bp.spos[j]];
  }
  Bp.jb.resize(ns);
  Bp.je.resize(ns);
  Bp.jo.resize(ns);
  for (int s = 0; s < ns; ++s) {
    int fd = P.sn_first_desc[s];
    Bp.jb[s] = (int)(std::lower_bound(csn.begin(), csn.end(), fd) - csn.begin());
    Bp.je[s] = (int)(std::upper_bound(csn.begin(), csn.end(), s) - csn.begin());
    Bp.jo[s] = (int)(std::lower_bound(csn.begin(), csn.end(), s) - csn.begin());
  }
  Bp.Xofs.assign(ns, 0);
  int64_t X = 0;
  double tf = 0, sf = 0, sfe = 0;
  for (int s = 0; s < ns; ++s) {
    int J = Bp.je[s] - Bp.jb[s];
    if (J <= 0) continue;
    Bp.act.push_back(s);
    Bp.Xofs[s] = X;
    int w = P.sn_w[s], r = P.sn_r[s];
    X += (int64_t)xpad(w) * J;
    tf += (double)J * ((double)w * w + 2.0 * w * r);
    sf += (double)J * (J + 1) * w;
  }
  Bp.Xsize = X;
  // RHS update stack over the active supernodes
  Bp.rhs_stack_ofs.assign(ns, 0);
  {
    int64_t top = 0, peak = 0, fr = 0;
    std::vector<int64_t> size(ns, 0);
    for (int s : Bp.act) {
      int64_t base = top;
      for (int k = P.ch_off[s]; k < P.ch_off[s + 1]; ++k) base -= size[P.ch_list[k]];
      int J = Bp.je[s] - Bp.jb[s];
      int r = P.sn_r[s];
      size[s] = (P.sn_parent[s] >= 0) ? (int64_t)r * J : 0;
      fr = std::max(fr, (int64_t)r * J);
      Bp.rhs_stack_ofs[s] = base;
      top = base + size[s];
      peak = std::max(peak, top);
    }
    Bp.rhs_stack = peak;
    Bp.rhs_front = fr;
  }
  // SYRK tile contributions: supernode s feeds every lower tile inside J_s x J_s
  int nb = Bp.nb;
  int ntile = nb * (nb + 1) / 2;
  std::vector<std::vector<int>> per(ntile);
  for (int s : Bp.act) {
    int t0 = Bp.jb[s] / kTile, t1 = (Bp.je[s] - 1) / kTile;
    for (int bi = t0; bi <= t1; ++bi)
      for (int bj = t0; bj <= bi; ++bj) {
        per[bi * (bi + 1) / 2 + bj].push_back(s);
        sfe += 2.0 * kTile * kTile * P.sn_w[s];
      }
  }
  Bp.tile_off.assign(ntile + 1, 0);
  for (int t = 0; t < ntile; ++t) Bp.tile_off[t + 1] = Bp.tile_off[t] + (int)per[t].size();
  Bp.tile_sn.reserve(Bp.tile_off[ntile]);
  for (int t = 0; t < ntile; ++t) Bp.tile_sn.insert(Bp.tile_sn.end(), per[t].begin(), per[t].end());
  // the same lists for 128 x 128 tiles
  Bp.nb2 = (Bp.m_pad + 127) / 128;
  int nt2 = Bp.nb2 * (Bp.nb2 + 1) / 2;
  std::vector<std::vector<int>> per2(nt2);
  for (int s : Bp.act) {
    int t0 = Bp.jb[s] / 128, t1 = (Bp.je[s] - 1) / 128;
    for (int bi = t0; bi <= t1; ++bi)
      for (int bj = t0; bj <= bi; ++bj) per2[bi * (bi + 1) / 2 + bj].push_back(s);
  }
  Bp.t2_off.assign(nt2 + 1, 0);
  for (int t = 0; t < nt2; ++t) Bp.t2_off[t + 1] = Bp.t2_off[t] + (int)per2[t].size();
  for (int t = 0; t < nt2; ++t) Bp.t2_sn.insert(Bp.t2_sn.end(), per2[t].begin(), per2[t].end());
  Bp.trsm_flops = tf;
  Bp.syrk_flops = sf;
  Bp.syrk_exec_flops = sfe;
}

}  // namespace feti
