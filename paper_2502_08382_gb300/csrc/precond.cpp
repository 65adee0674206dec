// Host set-up of the lumped FETI preconditioner (the M of Algorithm 1, which
// the paper leaves open):
//
//   M = W (sum_i B_i K_i B_i^T) W,   W = (B B^T)^{-1}.
//
// B B^T couples the multipliers that some subdomain puts on one DOF (gluing
// rows of a node shared by several subdomains, chained at cross points, and
// Dirichlet rows), so it is block diagonal with a block per node component:
// W is formed block by block on the host once per B.  M_core = sum_i
// B_i K_i B_i^T is the subdomain stiffness on its B-touched DOFs, signed: its
// pattern and, per entry, the list of (K value, sign product) contributions
// depend only on the patterns of K_i and B_i, so they are planned here once
// and the values are summed on the device at every feti_assemble.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <stdexcept>
#include <tuple>

#include "context.h"
#include "precond.h"

namespace feti {

namespace {

int uf_find(std::vector<int>& p, int a) {
  while (p[a] != a) {
    p[a] = p[p[a]];
    a = p[a];
  }
  return a;
}

// inverse of a small SPD block (Gauss-Jordan with partial pivoting)
bool invert_block(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (std::fabs(a[(size_t)piv * n + col]) == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= d;
      inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

}  // namespace

void plan_lumped(const feti_ctx* c, LumpedPlan& out) {
  const int nl = c->nlam;
  // ---- B B^T: entries (a, b, s_a s_b) for rows of one subdomain on one DOF
  std::vector<std::tuple<int, int, double>> bb;
  for (const auto& s : c->subs) {
    std::vector<int> rows(s.m);
    std::iota(rows.begin(), rows.end(), 0);
    std::stable_sort(rows.begin(), rows.end(), [&](int x, int y) { return s.bdof[x] < s.bdof[y]; });
    for (size_t i = 0; i < rows.size();) {
      size_t j = i;
      while (j < rows.size() && s.bdof[rows[j]] == s.bdof[rows[i]]) ++j;
      for (size_t a = i; a < j; ++a)
        for (size_t b = i; b < j; ++b)
          bb.emplace_back(s.blam[rows[a]], s.blam[rows[b]], s.bsign[rows[a]] * s.bsign[rows[b]]);
      i = j;
    }
  }
  std::vector<int> parent(nl);
  std::iota(parent.begin(), parent.end(), 0);
  for (auto& e : bb) {
    const int a = uf_find(parent, std::get<0>(e)), b = uf_find(parent, std::get<1>(e));
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
  std::vector<std::vector<int>> comp(nl);
  for (int l = 0; l < nl; ++l) comp[uf_find(parent, l)].push_back(l);  // ascending multipliers
  std::vector<int> pos(nl, -1), root(nl, -1);
  for (int r = 0; r < nl; ++r)
    for (size_t k = 0; k < comp[r].size(); ++k) {
      pos[comp[r][k]] = (int)k;
      root[comp[r][k]] = r;
    }
  std::map<int, std::vector<double>> blocks;  // root -> dense block of B B^T, then its inverse
  for (int r = 0; r < nl; ++r)
    if (!comp[r].empty()) blocks[r].assign(comp[r].size() * comp[r].size(), 0.0);
  for (auto& e : bb) {
    const int a = std::get<0>(e), b = std::get<1>(e), r = root[a];
    const int n = (int)comp[r].size();
    blocks[r][(size_t)pos[a] * n + pos[b]] += std::get<2>(e);
  }
  out.w_off.assign(nl + 1, 0);
  for (int l = 0; l < nl; ++l) out.w_off[l + 1] = out.w_off[l] + (int)comp[root[l]].size();
  out.w_col.resize(out.w_off[nl]);
  out.w_val.resize(out.w_off[nl]);
  for (auto& kv : blocks) {
    const int r = kv.first, n = (int)comp[r].size();
    std::vector<double> a = kv.second;
    if (!invert_block(a, n)) throw std::runtime_error("B B^T has a singular block (redundant multipliers)");
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const int l = comp[r][i];
        out.w_col[out.w_off[l] + j] = comp[r][j];
        out.w_val[out.w_off[l] + j] = a[(size_t)i * n + j];
      }
  }
  // ---- M_core = sum_i B_i K_i B_i^T: per row multiplier, (column multiplier, K value index, sign)
  std::vector<std::vector<std::tuple<int, int64_t, double>>> rowc(nl);
  for (size_t i = 0; i < c->subs.size(); ++i) {
    const auto& s = c->subs[i];
    const int64_t kofs = c->info[i].Kval;
    std::vector<int> head(s.n, -1), next(s.m, -1);  // DOF -> its B rows (linked list)
    for (int r = s.m - 1; r >= 0; --r) {
      next[r] = head[s.bdof[r]];
      head[s.bdof[r]] = r;
    }
    for (int r = 0; r < s.m; ++r) {
      const int x = s.bdof[r];
      for (int64_t k = s.rowptr[x]; k < s.rowptr[x + 1]; ++k)
        for (int r2 = head[s.col[k]]; r2 >= 0; r2 = next[r2])
          rowc[s.blam[r]].emplace_back(s.blam[r2], kofs + k, s.bsign[r] * s.bsign[r2]);
    }
  }
  out.m_off.assign(nl + 1, 0);
  out.c_off.assign(1, 0);
  for (int l = 0; l < nl; ++l) {
    auto& v = rowc[l];
    std::sort(v.begin(), v.end());  // by column, then K index: a fixed summation order
    for (size_t k = 0; k < v.size();) {
      size_t j = k;
      while (j < v.size() && std::get<0>(v[j]) == std::get<0>(v[k])) {
        out.c_kidx.push_back(std::get<1>(v[j]));
        out.c_sign.push_back(std::get<2>(v[j]));
        ++j;
      }
      out.m_col.push_back(std::get<0>(v[k]));
      out.c_off.push_back((int64_t)out.c_kidx.size());
      k = j;
    }
    out.m_off[l + 1] = (int)out.m_col.size();
    std::vector<std::tuple<int, int64_t, double>>().swap(v);
  }
}

}  // namespace feti
