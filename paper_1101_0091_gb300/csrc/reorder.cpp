// Reverse Cuthill-McKee reordering (Sec. 1.3.1 applies RCM to the Hamiltonian
// matrix to make the accesses to B more local) and the symmetric permutation
// of a CRS matrix.  One-time host work, like the other format builders.
//
// Tie-breaking (fixed, so the permutation is unique):
//  - graph: pattern of A + A^T without self loops; degree = distinct neighbours;
//  - components in order of their smallest node; start node by the
//    pseudo-peripheral search: r = node of minimum (degree, index); repeat:
//    level structure from r, candidate = minimum (degree, index) of its last
//    level; if the candidate's level structure is deeper, r = candidate;
//  - Cuthill-McKee breadth-first search from r, each node appending its
//    unvisited neighbours in ascending (degree, index);
//  - perm = the reversed order (perm[new] = old).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace spmv {

namespace {

struct Graph {
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
  int64_t deg(int64_t u) const { return ptr[u + 1] - ptr[u]; }
};

Graph build_graph(int64_t n, const int32_t* rp, const int32_t* col) {
  Graph g;
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
      if (col[j] != i) {
        ++cnt[i + 1];
        ++cnt[col[j] + 1];
      }
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int32_t> raw((size_t)cnt[n]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
      if (col[j] != i) {
        raw[fill[i]++] = col[j];
        raw[fill[col[j]]++] = (int32_t)i;
      }
  g.ptr.assign(n + 1, 0);
  g.adj.reserve(raw.size());
  for (int64_t i = 0; i < n; ++i) {
    auto b = raw.begin() + cnt[i], e = raw.begin() + cnt[i + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    g.adj.insert(g.adj.end(), b, e);
    g.ptr[i + 1] = (int64_t)g.adj.size();
  }
  return g;
}

// Breadth-first level structure from r: returns the depth and leaves the last
// level in `last`.  mark/stamp avoid clearing between searches.
int64_t level_structure(const Graph& g, int32_t r, std::vector<uint32_t>& mark, uint32_t stamp,
                        std::vector<int32_t>& cur, std::vector<int32_t>& nxt, std::vector<int32_t>& last) {
  cur.assign(1, r);
  mark[r] = stamp;
  int64_t depth = 1;
  for (;;) {
    nxt.clear();
    for (int32_t u : cur)
      for (int64_t p = g.ptr[u]; p < g.ptr[u + 1]; ++p) {
        const int32_t v = g.adj[p];
        if (mark[v] != stamp) {
          mark[v] = stamp;
          nxt.push_back(v);
        }
      }
    if (nxt.empty()) {
      last = cur;
      return depth;
    }
    cur.swap(nxt);
    ++depth;
  }
}

}  // namespace

bool rcm_permutation(int64_t n, const int32_t* rp, const int32_t* col, int32_t* perm) {
  const Graph g = build_graph(n, rp, col);
  auto less = [&](int32_t a, int32_t b) {
    const int64_t da = g.deg(a), db = g.deg(b);
    return da != db ? da < db : a < b;
  };
  std::vector<uint8_t> visited((size_t)n, 0);
  std::vector<uint32_t> mark((size_t)n, 0);
  uint32_t stamp = 0;
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  std::vector<int32_t> comp, cur, nxt, last, nb;
  for (int64_t s = 0; s < n; ++s) {
    if (visited[s]) continue;
    // the component of s (its smallest node: every smaller node is already ordered)
    ++stamp;
    comp.assign(1, (int32_t)s);
    mark[s] = stamp;
    for (size_t h = 0; h < comp.size(); ++h) {
      const int32_t u = comp[h];
      for (int64_t p = g.ptr[u]; p < g.ptr[u + 1]; ++p)
        if (mark[g.adj[p]] != stamp) {
          mark[g.adj[p]] = stamp;
          comp.push_back(g.adj[p]);
        }
    }
    int32_t r = *std::min_element(comp.begin(), comp.end(), less);
    int64_t depth = level_structure(g, r, mark, ++stamp, cur, nxt, last);
    for (;;) {
      const int32_t cand = *std::min_element(last.begin(), last.end(), less);
      std::vector<int32_t> cand_last;
      const int64_t d = level_structure(g, cand, mark, ++stamp, cur, nxt, cand_last);
      if (d > depth) {
        r = cand;
        depth = d;
        last.swap(cand_last);
      } else {
        break;
      }
    }
    // Cuthill-McKee from r
    size_t head = order.size();
    visited[r] = 1;
    order.push_back(r);
    while (head < order.size()) {
      const int32_t u = order[head++];
      nb.clear();
      for (int64_t p = g.ptr[u]; p < g.ptr[u + 1]; ++p)
        if (!visited[g.adj[p]]) nb.push_back(g.adj[p]);
      std::sort(nb.begin(), nb.end(), less);
      for (int32_t v : nb) {
        visited[v] = 1;
        order.push_back(v);
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) perm[i] = order[(size_t)(n - 1 - i)];
  return true;
}

bool validate_permutation(int64_t n, const int32_t* perm, std::vector<int32_t>* inv, std::string* why) {
  inv->assign((size_t)n, -1);
  for (int64_t r = 0; r < n; ++r) {
    const int32_t o = perm[r];
    if (o < 0 || o >= n) {
      *why = "perm[" + std::to_string(r) + "] = " + std::to_string(o) + " is out of range";
      return false;
    }
    if ((*inv)[o] >= 0) {
      *why = "perm repeats " + std::to_string(o);
      return false;
    }
    (*inv)[o] = (int32_t)r;
  }
  return true;
}

void permute_csr(int64_t n, const int32_t* rp, const int32_t* col, const double* val, const int32_t* perm,
                 const std::vector<int32_t>& inv, int32_t* out_rp, int32_t* out_col, double* out_val) {
  std::vector<std::pair<int32_t, int32_t>> row;  // (new column, position in the row)
  int64_t p = 0;
  out_rp[0] = 0;
  for (int64_t r = 0; r < n; ++r) {
    const int64_t o = perm[r];
    const int64_t b = rp[o], e = rp[o + 1];
    row.clear();
    for (int64_t j = b; j < e; ++j) row.emplace_back(inv[col[j]], (int32_t)(j - b));
    std::sort(row.begin(), row.end());  // by new column, then by position: stable
    for (const auto& c : row) {
      out_col[p] = c.first;
      out_val[p++] = val[b + c.second];
    }
    out_rp[r + 1] = (int32_t)p;
  }
}

}  // namespace spmv
