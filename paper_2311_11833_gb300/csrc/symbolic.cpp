// Host-side symbolic analysis: ordering, elimination tree, supernodes,
// assembly-tree levels and the index maps the GPU kernels use.
//
// The pivot sequence is fixed here once per sparsity pattern (Sec. II-C:
// static pivoting "computed once, and perpetually reused"); the perturbation
// A + t_k D of Sec. III-A changes values only, so every perturbation and
// every later set of values reuses this structure.
#include "symbolic.h"

#include <algorithm>
#include <system_error>
#include <thread>
#include <functional>
#include <atomic>
#include <climits>
#include <cstdio>
#include <numeric>
#include <queue>
#include <utility>

namespace pisp {

// --------------------------------------------------------------------------
// Minimum degree on the quotient graph.  Eliminated nodes become "elements"
// (cliques of their remaining neighbours); a variable's degree is bounded by
// |Lp| - 1 + |its variable neighbours| + sum over its other elements of the
// part not already in Lp (an upper bound on the exact external degree, as in
// approximate minimum degree).  Elements whose variables all lie in the new
// element are absorbed.  Ties go to the lowest index, so the ordering is
// deterministic.
// --------------------------------------------------------------------------
std::vector<int32_t> minimum_degree(int32_t n, const std::vector<int32_t>& xadj,
                                    const std::vector<int32_t>& adj) {
  std::vector<std::vector<int32_t>> vadj(n), eadj(n), le(n);
  std::vector<char> state(n, 0);  // 0 variable, 1 live element, 2 absorbed
  std::vector<int32_t> deg(n), mark(n, -1), w(n, 0), wstamp(n, -1);
  // (degree, index) min-heap with lazy deletion: every variable has an entry
  // with its current degree; entries left behind by a degree update, or by
  // an elimination, are skipped when they reach the top.  The next pivot is
  // the lowest index among the smallest degrees.
  using Entry = std::pair<int32_t, int32_t>;
  std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
  for (int32_t i = 0; i < n; ++i) {
    vadj[i].assign(adj.begin() + xadj[i], adj.begin() + xadj[i + 1]);
    deg[i] = (int32_t)vadj[i].size();
    pq.push({deg[i], i});
  }
  std::vector<int32_t> perm;
  perm.reserve(n);
  int32_t live = n;
  std::vector<int32_t> Lp, nv, ne;
  for (int32_t step = 0; step < n; ++step) {
    while (state[pq.top().second] != 0 || deg[pq.top().second] != pq.top().first) pq.pop();
    const int32_t p = pq.top().second;
    pq.pop();
    perm.push_back(p);
    --live;
    Lp.clear();
    mark[p] = step;
    for (int32_t v : vadj[p])
      if (state[v] == 0 && mark[v] != step) { mark[v] = step; Lp.push_back(v); }
    for (int32_t e : eadj[p]) {
      if (state[e] != 1) continue;
      for (int32_t v : le[e])
        if (state[v] == 0 && mark[v] != step) { mark[v] = step; Lp.push_back(v); }
      state[e] = 2;
      std::vector<int32_t>().swap(le[e]);
    }
    state[p] = 1;
    le[p] = Lp;
    std::vector<int32_t>().swap(vadj[p]);
    std::vector<int32_t>().swap(eadj[p]);
    // |Le \ Lp| for every live element touching Lp
    for (int32_t i : Lp)
      for (int32_t e : eadj[i]) {
        if (state[e] != 1 || e == p) continue;
        if (wstamp[e] != step) { wstamp[e] = step; w[e] = (int32_t)le[e].size(); }
        --w[e];
      }
    for (int32_t i : Lp)
      for (int32_t e : eadj[i])
        if (state[e] == 1 && e != p && wstamp[e] == step && w[e] == 0) {
          state[e] = 2;  // aggressive absorption: Le is inside Lp
          std::vector<int32_t>().swap(le[e]);
        }
    const int32_t lp = (int32_t)Lp.size();
    for (int32_t i : Lp) {
      nv.clear();
      for (int32_t v : vadj[i])
        if (state[v] == 0 && mark[v] != step) nv.push_back(v);
      vadj[i].swap(nv);
      ne.clear();
      int64_t d = (int64_t)lp - 1 + (int64_t)vadj[i].size();
      for (int32_t e : eadj[i])
        if (state[e] == 1 && e != p) {
          ne.push_back(e);
          d += (wstamp[e] == step) ? w[e] : (int64_t)le[e].size();
        }
      ne.push_back(p);
      eadj[i].swap(ne);
      if (d > live - 1) d = live - 1;
      if (deg[i] != (int32_t)d) {
        deg[i] = (int32_t)d;
        pq.push({deg[i], i});
      }
    }
  }
  return perm;
}

namespace {

struct LocalSn {
  int32_t c0, c1;
  std::vector<int32_t> rows;  // local permuted rows > c1-1, ascending
  int64_t zeros = 0;
  int32_t level = 0;
};

int32_t pos_in_front(const Supernode& s, const int32_t* rows, int32_t x) {
  if (x >= s.c0 && x < s.c1) return x - s.c0;
  const int32_t* b = rows + s.row_off;
  const int32_t* e = b + s.ms;
  const int32_t* f = std::lower_bound(b, e, x);
  if (f == e || *f != x) return -1;
  return s.ns() + (int32_t)(f - b);
}

}  // namespace

// Maximum matching of rows to columns in the bipartite graph of the pattern
// (Hopcroft-Karp: breadth-first layering from the free rows, then
// vertex-disjoint shortest augmenting paths by depth-first search along the
// layers, repeated until no augmenting path is left).  The depth-first search
// keeps an explicit stack, so path length is not bounded by the call stack.
std::string match_rows(int32_t n, const int64_t* row_ptr, const int32_t* col,
                       std::vector<int32_t>& row_of_col) {
  const int32_t kNil = -1, kInf = INT32_MAX;
  std::vector<int32_t> col_of_row(n, kNil), dist(n), queue(n), stack;
  std::vector<int64_t> it(n);
  row_of_col.assign(n, kNil);
  for (int32_t r = 0; r < n; ++r)  // greedy start
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
      if (row_of_col[col[e]] == kNil) {
        row_of_col[col[e]] = r;
        col_of_row[r] = col[e];
        break;
      }
  for (;;) {
    int32_t qh = 0, qt = 0;
    bool reach_free = false;
    for (int32_t r = 0; r < n; ++r) {
      if (col_of_row[r] == kNil) {
        dist[r] = 0;
        queue[qt++] = r;
      } else {
        dist[r] = kInf;
      }
    }
    while (qh < qt) {
      const int32_t r = queue[qh++];
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        const int32_t r2 = row_of_col[col[e]];
        if (r2 == kNil) {
          reach_free = true;
        } else if (dist[r2] == kInf) {
          dist[r2] = dist[r] + 1;
          queue[qt++] = r2;
        }
      }
    }
    if (!reach_free) break;
    for (int32_t r = 0; r < n; ++r) it[r] = row_ptr[r];
    int32_t augmented = 0;
    for (int32_t r0 = 0; r0 < n; ++r0) {
      if (col_of_row[r0] != kNil || dist[r0] != 0) continue;
      stack.assign(1, r0);
      while (!stack.empty()) {
        const int32_t r = stack.back();
        int32_t next = kNil;
        bool free_col = false;
        for (; it[r] < row_ptr[r + 1]; ++it[r]) {
          const int32_t r2 = row_of_col[col[it[r]]];
          if (r2 == kNil) {
            free_col = true;
            break;
          }
          if (dist[r2] == dist[r] + 1) {
            next = r2;
            break;
          }
        }
        if (free_col) {
          // each row on the stack takes the column it points at; the column
          // of a row was held by the row above it on the stack
          for (size_t i = 0; i < stack.size(); ++i) {
            const int32_t rr = stack[i], cc = col[it[rr]];
            col_of_row[rr] = cc;
            row_of_col[cc] = rr;
            dist[rr] = kInf;  // off the layered graph for the rest of the phase
          }
          ++augmented;
          break;
        }
        if (next != kNil) {
          stack.push_back(next);
        } else {
          dist[r] = kInf;  // dead end for this phase
          stack.pop_back();
          if (!stack.empty()) ++it[stack.back()];
        }
      }
    }
    if (augmented == 0) break;
  }
  for (int32_t c = 0; c < n; ++c)
    if (row_of_col[c] == kNil) return "structurally singular: no matching covers every column";
  return std::string();
}

namespace {

// Ordering, elimination tree, column structures and relaxed supernodes of one
// instance (local indices).  Instances are independent, so they can be
// analysed concurrently; `analyze` merges them in instance order.
struct InstanceResult {
  std::string err;
  std::vector<int32_t> pf;         // [ng] local permutation, new -> old
  std::vector<LocalSn> merged;     // supernodes, children before parents
  std::vector<int32_t> sn_parent;  // local parent supernode, or -1
  std::vector<int32_t> lsn;        // [ng] local supernode of each permuted column
  int64_t nnzL = 0;
  int32_t height = 0;              // elimination-tree height
};

std::string analyze_instance(int32_t ng, int64_t off, const int64_t* row_ptr, const int32_t* col,
                             const SymbolicOptions& opt, InstanceResult& R) {
  // symmetric adjacency of A + A^T without the diagonal (local indices)
  std::vector<int32_t> cnt(ng + 1, 0);
  for (int32_t i = 0; i < ng; ++i)
    for (int64_t e = row_ptr[off + i]; e < row_ptr[off + i + 1]; ++e) {
      const int64_t j = (int64_t)col[e] - off;
      if (j < 0 || j >= ng) return "column index outside its instance block";
      if (j != i) { ++cnt[i + 1]; ++cnt[j + 1]; }
    }
  std::vector<int32_t> xadj(ng + 1, 0);
  for (int32_t i = 0; i < ng; ++i) xadj[i + 1] = xadj[i] + cnt[i + 1];
  std::vector<int32_t> adj(xadj[ng]);
  std::vector<int32_t> fill(xadj.begin(), xadj.end() - 1);
  for (int32_t i = 0; i < ng; ++i)
    for (int64_t e = row_ptr[off + i]; e < row_ptr[off + i + 1]; ++e) {
      const int32_t j = (int32_t)(col[e] - off);
      if (j != i) { adj[fill[i]++] = j; adj[fill[j]++] = i; }
    }
  // sort + unique each list
  {
    std::vector<int32_t> x2(ng + 1, 0), a2;
    a2.reserve(adj.size());
    for (int32_t i = 0; i < ng; ++i) {
      auto b = adj.begin() + xadj[i], e = adj.begin() + xadj[i + 1];
      std::sort(b, e);
      auto u = std::unique(b, e);
      a2.insert(a2.end(), b, u);
      x2[i + 1] = (int32_t)a2.size();
    }
    xadj.swap(x2);
    adj.swap(a2);
  }
  std::vector<int32_t> pl;
  if (opt.ordering == 0) {
    pl = minimum_degree(ng, xadj, adj);
  } else {
    pl.resize(ng);
    std::iota(pl.begin(), pl.end(), 0);
  }
  std::vector<int32_t> ipl(ng);
  for (int32_t i = 0; i < ng; ++i) ipl[pl[i]] = i;
  // elimination tree of the permuted pattern
  std::vector<int32_t> parent(ng, -1), anc(ng, -1);
  for (int32_t j = 0; j < ng; ++j) {
    const int32_t o = pl[j];
    for (int32_t q = xadj[o]; q < xadj[o + 1]; ++q) {
      int32_t r = ipl[adj[q]];
      if (r >= j) continue;
      while (anc[r] != -1 && anc[r] != j) { const int32_t t = anc[r]; anc[r] = j; r = t; }
      if (anc[r] == -1) { anc[r] = j; parent[r] = j; }
    }
  }
  // postorder (children visited in ascending order)
  std::vector<int32_t> head(ng, -1), next(ng, -1);
  for (int32_t j = ng - 1; j >= 0; --j)
    if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
  std::vector<int32_t> post;
  post.reserve(ng);
  std::vector<int32_t> stack;
  for (int32_t r = 0; r < ng; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      const int32_t v = stack.back();
      if (head[v] >= 0) {
        const int32_t c = head[v];
        head[v] = next[c];
        stack.push_back(c);
      } else {
        stack.pop_back();
        post.push_back(v);
      }
    }
  }
  std::vector<int32_t> ipost(ng);
  for (int32_t k = 0; k < ng; ++k) ipost[post[k]] = k;
  std::vector<int32_t> pf(ng), ipf(ng), par(ng);
  for (int32_t k = 0; k < ng; ++k) {
    pf[k] = pl[post[k]];
    par[k] = parent[post[k]] >= 0 ? ipost[parent[post[k]]] : -1;
  }
  for (int32_t k = 0; k < ng; ++k) ipf[pf[k]] = k;
  // column structures of L (rows > j) by merging children
  std::vector<std::vector<int32_t>> st(ng);
  std::vector<int32_t> mk(ng, -1), height(ng, 0);
  std::vector<std::vector<int32_t>> kids(ng);
  for (int32_t j = 0; j < ng; ++j)
    if (par[j] >= 0) kids[par[j]].push_back(j);
  for (int32_t j = 0; j < ng; ++j) {
    std::vector<int32_t>& s = st[j];
    mk[j] = j;
    const int32_t o = pf[j];
    for (int32_t q = xadj[o]; q < xadj[o + 1]; ++q) {
      const int32_t i = ipf[adj[q]];
      if (i > j && mk[i] != j) { mk[i] = j; s.push_back(i); }
    }
    for (int32_t c : kids[j]) {
      height[j] = std::max(height[j], height[c] + 1);
      for (int32_t i : st[c])
        if (i > j && mk[i] != j) { mk[i] = j; s.push_back(i); }
    }
    std::sort(s.begin(), s.end());
    R.nnzL += (int64_t)s.size();
    R.height = std::max(R.height, height[j] + 1);
  }
  // maximal supernodes: j-1 joins j when struct(j-1) = {j} u struct(j)
  std::vector<LocalSn> fund;
  for (int32_t j = 0; j < ng; ++j) {
    const bool join = j > 0 && par[j - 1] == j && st[j - 1].size() == st[j].size() + 1;
    if (join) {
      fund.back().c1 = j + 1;
    } else {
      LocalSn s;
      s.c0 = j;
      s.c1 = j + 1;
      fund.push_back(std::move(s));
    }
  }
  for (auto& s : fund) s.rows = st[s.c1 - 1];
  std::vector<std::vector<int32_t>>().swap(st);
  // relaxed amalgamation of last-child chains
  std::vector<LocalSn> merged;
  for (auto& p : fund) {
    LocalSn cur = std::move(p);
    while (!merged.empty()) {
      LocalSn& c = merged.back();
      if (c.c1 != cur.c0) break;
      const int32_t pc = par[c.c1 - 1];
      if (pc < cur.c0 || pc >= cur.c1) break;
      const int64_t nsc = c.c1 - c.c0, nsp = cur.c1 - cur.c0;
      const int64_t msc = (int64_t)c.rows.size(), msp = (int64_t)cur.rows.size();
      const int64_t z = c.zeros + cur.zeros + nsc * (nsp + msp - msc);
      const int64_t ns = nsc + nsp;
      const double E = (double)ns * (ns + 1) / 2.0 + (double)ns * msp;
      if (!(ns <= opt.relax_small || (double)z <= opt.relax_zeros * E)) break;
      cur.c0 = c.c0;
      cur.zeros = z;
      merged.pop_back();
    }
    merged.push_back(std::move(cur));
  }
  // supernode parents and levels (children precede parents)
  std::vector<int32_t> lsn(ng, -1);
  for (int32_t s = 0; s < (int32_t)merged.size(); ++s)
    for (int32_t j = merged[s].c0; j < merged[s].c1; ++j) lsn[j] = s;
  R.sn_parent.resize(merged.size());
  for (size_t s = 0; s < merged.size(); ++s) {
    const int32_t pc = par[merged[s].c1 - 1];
    R.sn_parent[s] = pc >= 0 ? lsn[pc] : -1;
  }
  R.pf.swap(pf);
  R.merged.swap(merged);
  R.lsn.swap(lsn);
  return std::string();
}

// Runs body(g) for g = 0..G-1, on up to `threads` host threads (0 = the
// hardware concurrency, at most 16) when there are several instances; each g
// is run exactly once.  If a worker thread cannot be started, the instances
// nobody has taken run on the calling thread.
void for_each_instance(int32_t G, int threads, const std::function<void(int32_t)>& body) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned cap = threads > 0 ? (unsigned)threads : std::min(hw, 16u);
  const int32_t T = (int32_t)std::min<unsigned>(cap, (unsigned)std::max<int32_t>(G, 1));
  if (T <= 1) {
    for (int32_t g = 0; g < G; ++g) body(g);
    return;
  }
  std::atomic<int32_t> next(0);
  auto work = [&]() {
    for (int32_t g = next.fetch_add(1); g < G; g = next.fetch_add(1)) body(g);
  };
  std::vector<std::thread> pool;
  pool.reserve(T);
  try {
    for (int32_t t = 0; t < T; ++t) pool.emplace_back(work);
  } catch (const std::system_error&) {
    // fewer threads than asked for: the ones running and this thread share the rest
  }
  work();
  for (auto& th : pool) th.join();
}

}  // namespace

std::string analyze(int32_t G, const int32_t* n, const int64_t* row_ptr,
                    const int32_t* col, const SymbolicOptions& opt, Symbolic& S) {
  S = Symbolic();
  if (G < 1) return "G must be >= 1";
  S.G = G;
  S.inst_off.assign(G + 1, 0);
  for (int32_t g = 0; g < G; ++g) {
    if (n[g] < 0) return "negative instance size";
    S.inst_off[g + 1] = S.inst_off[g] + n[g];
  }
  S.N = S.inst_off[G];
  if (S.N >= (int64_t)1 << 31) return "too many unknowns (limit 2^31-1)";
  if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
  for (int64_t i = 0; i < S.N; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return "row_ptr must be non-decreasing";
  S.nnzA = row_ptr[S.N];
  if (S.nnzA >= (int64_t)1 << 31) return "too many nonzeros (limit 2^31-1)";
  S.inst_nnz_off.assign(G + 1, 0);
  for (int32_t g = 0; g <= G; ++g) S.inst_nnz_off[g] = row_ptr[S.inst_off[g]];
  S.perm.assign(S.N, 0);
  S.iperm.assign(S.N, 0);
  S.col_sn.assign(S.N, -1);

  std::vector<InstanceResult> res(G);
  for_each_instance(G, opt.threads, [&](int32_t g) {
    if (n[g] <= 0) return;
    // an exception must not leave a worker thread (that would terminate the
    // process): it becomes this instance's error message
    try {
      res[g].err = analyze_instance(n[g], S.inst_off[g], row_ptr, col, opt, res[g]);
    } catch (const std::bad_alloc&) {
      res[g].err = "out of host memory in the symbolic analysis";
    } catch (const std::exception& e) {
      res[g].err = std::string("symbolic analysis failed: ") + e.what();
    }
  });
  for (int32_t g = 0; g < G; ++g)
    if (!res[g].err.empty()) return res[g].err;
  for (int32_t g = 0; g < G; ++g) {
    const int32_t ng = n[g];
    const int64_t off = S.inst_off[g];
    if (ng == 0) continue;
    InstanceResult& R = res[g];
    S.nnzL += R.nnzL;
    S.etree_height = std::max(S.etree_height, R.height);
    const int32_t base = (int32_t)S.sn.size();
    for (size_t s = 0; s < R.merged.size(); ++s) {
      const LocalSn& L = R.merged[s];
      Supernode sn;
      sn.c0 = (int32_t)(L.c0 + off);
      sn.c1 = (int32_t)(L.c1 + off);
      sn.instance = g;
      sn.ms = (int32_t)L.rows.size();
      sn.row_off = (int64_t)S.rows.size();
      for (int32_t r : L.rows) S.rows.push_back((int32_t)(r + off));
      sn.parent = R.sn_parent[s] >= 0 ? base + R.sn_parent[s] : -1;
      S.sn.push_back(sn);
    }
    for (int32_t s = base; s < (int32_t)S.sn.size(); ++s) {
      const int32_t p = S.sn[s].parent;
      if (p >= 0) S.sn[p].level = std::max(S.sn[p].level, S.sn[s].level + 1);
    }
    for (int32_t k = 0; k < ng; ++k) {
      S.perm[off + k] = (int32_t)(R.pf[k] + off);
      S.iperm[off + R.pf[k]] = (int32_t)(k + off);
      S.col_sn[off + k] = base + R.lsn[k];
    }
    R = InstanceResult();  // release this instance's buffers
  }

  const int32_t nS = (int32_t)S.sn.size();
  S.emap.assign(S.rows.size(), 0);
  S.front_off.assign(nS + 1, 0);
  S.vec_off.assign(nS + 1, 0);
  S.child_off.assign(nS + 1, 0);
  for (int32_t s = 0; s < nS; ++s) {
    const Supernode& sn = S.sn[s];
    const int64_t F = sn.F(), ns = sn.ns(), ms = sn.ms;
    S.front_off[s + 1] = S.front_off[s] + F * F;
    S.vec_off[s + 1] = S.vec_off[s] + F;
    S.max_front = std::max<int32_t>(S.max_front, (int32_t)F);
    S.nnzF_stored += ns * (ns + 2 * ms);
    for (int64_t p = 0; p < ns; ++p) {
      const double r = (double)(F - p - 1);
      S.flops_factor += r + 2.0 * r * r;
    }
    S.flops_solve += 2.0 * ((double)ns * ns + 2.0 * ns * ms);
    if (sn.parent >= 0) {
      ++S.child_off[sn.parent + 1];
      const Supernode& P = S.sn[sn.parent];
      for (int32_t a = 0; a < sn.ms; ++a) {
        const int32_t pos = pos_in_front(P, S.rows.data(), S.rows[sn.row_off + a]);
        if (pos < 0) return "internal error: child row missing from parent front";
        S.emap[sn.row_off + a] = pos;
      }
    }
  }
  S.front_elems = S.front_off[nS];
  // inverse of the extend-add maps (children visited in increasing id, so the
  // contributions of each position are in child order)
  S.inv_off.assign(S.vec_off[nS] + 1, 0);
  for (int32_t c = 0; c < nS; ++c) {
    const Supernode& sn = S.sn[c];
    if (sn.parent < 0) continue;
    for (int32_t a = 0; a < sn.ms; ++a) ++S.inv_off[S.vec_off[sn.parent] + S.emap[sn.row_off + a] + 1];
  }
  for (size_t q = 1; q < S.inv_off.size(); ++q) S.inv_off[q] += S.inv_off[q - 1];
  S.inv_child.assign(S.inv_off.back(), 0);
  S.inv_a.assign(S.inv_off.back(), 0);
  {
    std::vector<int64_t> f(S.inv_off.begin(), S.inv_off.end() - 1);
    for (int32_t c = 0; c < nS; ++c) {
      const Supernode& sn = S.sn[c];
      if (sn.parent < 0) continue;
      for (int32_t a = 0; a < sn.ms; ++a) {
        const int64_t q = f[S.vec_off[sn.parent] + S.emap[sn.row_off + a]]++;
        S.inv_child[q] = c;
        S.inv_a[q] = a;
      }
    }
    S.inv_vbase.resize(S.inv_child.size());
    S.inv_cF.resize(S.inv_child.size());
    S.inv_col.resize(S.inv_child.size());
    for (size_t q = 0; q < S.inv_child.size(); ++q) {
      const Supernode& c = S.sn[S.inv_child[q]];
      S.inv_vbase[q] = S.vec_off[S.inv_child[q]];
      S.inv_cF[q] = c.F();
      S.inv_col[q] = c.ns() + S.inv_a[q];
    }
  }
  for (int32_t s = 0; s < nS; ++s) S.child_off[s + 1] += S.child_off[s];
  S.child.assign(S.child_off[nS], 0);
  {
    std::vector<int64_t> f(S.child_off.begin(), S.child_off.end() - 1);
    for (int32_t s = 0; s < nS; ++s)
      if (S.sn[s].parent >= 0) S.child[f[S.sn[s].parent]++] = s;
  }
  // levels
  int32_t L = 0;
  for (const auto& sn : S.sn) L = std::max(L, sn.level + 1);
  S.n_levels = L;
  S.level_off.assign(L + 1, 0);
  for (const auto& sn : S.sn) ++S.level_off[sn.level + 1];
  for (int32_t l = 0; l < L; ++l) S.level_off[l + 1] += S.level_off[l];
  S.level_sn.assign(nS, 0);
  {
    std::vector<int64_t> f(S.level_off.begin(), S.level_off.end() - 1);
    for (int32_t s = 0; s < nS; ++s) S.level_sn[f[S.sn[s].level]++] = s;
  }
  // assembly map: every entry of A lands in the front of the supernode that
  // owns column min(pi, pj); sorted by (supernode, front column, front row)
  std::vector<int32_t> dst_of(S.nnzA);
  std::vector<int32_t> sn_of(S.nnzA);
  for (int64_t i = 0; i < S.N; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t pi = S.iperm[i], pj = S.iperm[col[e]];
      const int32_t s = S.col_sn[std::min(pi, pj)];
      const Supernode& sn = S.sn[s];
      const int32_t r = pos_in_front(sn, S.rows.data(), pi);
      const int32_t c = pos_in_front(sn, S.rows.data(), pj);
      if (r < 0 || c < 0) return "internal error: entry outside its front";
      sn_of[e] = s;
      dst_of[e] = r + c * sn.F();
    }
  }
  S.amap_off.assign(nS + 1, 0);
  for (int64_t e = 0; e < S.nnzA; ++e) ++S.amap_off[sn_of[e] + 1];
  for (int32_t s = 0; s < nS; ++s) S.amap_off[s + 1] += S.amap_off[s];
  S.amap_src.assign(S.nnzA, 0);
  S.amap_dst.assign(S.nnzA, 0);
  {
    std::vector<int64_t> f(S.amap_off.begin(), S.amap_off.end() - 1);
    for (int64_t e = 0; e < S.nnzA; ++e) {
      const int64_t q = f[sn_of[e]]++;
      S.amap_src[q] = (int32_t)e;
      S.amap_dst[q] = dst_of[e];
    }
    // order each supernode's entries by (column, row) of the front
    std::vector<std::pair<int32_t, int32_t>> tmp;
    for (int32_t s = 0; s < nS; ++s) {
      const int32_t F = S.sn[s].F();
      tmp.clear();
      for (int64_t q = S.amap_off[s]; q < S.amap_off[s + 1]; ++q)
        tmp.push_back({S.amap_dst[q], S.amap_src[q]});
      std::sort(tmp.begin(), tmp.end(), [F](const std::pair<int32_t, int32_t>& a,
                                             const std::pair<int32_t, int32_t>& b) {
        const int32_t ca = a.first / F, cb = b.first / F;
        if (ca != cb) return ca < cb;
        if (a.first != b.first) return a.first < b.first;
        return a.second < b.second;
      });
      for (int64_t q = S.amap_off[s], k = 0; q < S.amap_off[s + 1]; ++q, ++k) {
        S.amap_dst[q] = tmp[k].first;
        S.amap_src[q] = tmp[k].second;
      }
    }
  }
  // first entry of every front column: column c of front s starts at
  // amap_coff[vec_off[s] + c]; the entry after a front's last column is the
  // next front's first, so consecutive fronts share it
  S.amap_coff.assign(S.vec_off[nS] + 1, 0);
  for (int32_t s = 0; s < nS; ++s) {
    const int32_t F = S.sn[s].F();
    int64_t q = S.amap_off[s];
    for (int32_t c = 0; c <= F; ++c) {
      while (q < S.amap_off[s + 1] && S.amap_dst[q] / F < c) ++q;
      S.amap_coff[S.vec_off[s] + c] = q;
    }
  }
  S.amap_coff[S.vec_off[nS]] = S.amap_off[nS];
  return std::string();
}

// Every index the kernels follow, checked against the sizes they assume.
std::string validate(const Symbolic& S) {
  const int64_t N = S.N, nS = (int64_t)S.sn.size();
  auto bad = [](const char* what) { return std::string("structure check failed: ") + what; };
  auto prefix_ok = [](const std::vector<int64_t>& off, size_t len, int64_t last) {
    if (off.size() != len || off[0] != 0 || off.back() != last) return false;
    for (size_t i = 1; i < off.size(); ++i)
      if (off[i] < off[i - 1]) return false;
    return true;
  };
  if (S.G < 1 || !prefix_ok(S.inst_off, (size_t)S.G + 1, N) ||
      !prefix_ok(S.inst_nnz_off, (size_t)S.G + 1, S.nnzA))
    return bad("instance offsets");
  if ((int64_t)S.perm.size() != N || (int64_t)S.iperm.size() != N || (int64_t)S.col_sn.size() != N)
    return bad("permutation sizes");
  for (int64_t i = 0; i < N; ++i)
    if (S.perm[i] < 0 || S.perm[i] >= N || S.iperm[S.perm[i]] != i) return bad("permutation");
  if (!prefix_ok(S.front_off, nS + 1, S.front_elems) || !prefix_ok(S.vec_off, nS + 1, S.vec_off.back()))
    return bad("front offsets");
  int32_t maxF = 0;
  int64_t next_col = 0;
  for (int64_t s = 0; s < nS; ++s) {
    const Supernode& sn = S.sn[s];
    const int64_t F = sn.F();
    if (sn.c0 != next_col || sn.c1 <= sn.c0 || sn.ms < 0) return bad("supernode column ranges");
    next_col = sn.c1;
    if (sn.instance < 0 || sn.instance >= S.G || sn.c0 < S.inst_off[sn.instance] ||
        sn.c1 > S.inst_off[sn.instance + 1])
      return bad("supernode instance");
    if (sn.parent != -1 && (sn.parent <= s || sn.parent >= nS)) return bad("parent");
    if (sn.row_off < 0 || sn.row_off + sn.ms > (int64_t)S.rows.size()) return bad("row list range");
    for (int32_t a = 0; a < sn.ms; ++a) {
      const int32_t r = S.rows[sn.row_off + a];
      if (r < sn.c1 || r >= S.inst_off[sn.instance + 1] || (a > 0 && r <= S.rows[sn.row_off + a - 1]))
        return bad("update rows");
    }
    for (int32_t c = sn.c0; c < sn.c1; ++c)
      if (S.col_sn[c] != s) return bad("column owner");
    if (S.front_off[s + 1] - S.front_off[s] != F * F || S.vec_off[s + 1] - S.vec_off[s] != F)
      return bad("front sizes");
    maxF = std::max<int32_t>(maxF, (int32_t)F);
    if (sn.parent >= 0) {  // extend-add positions: the row's place in the parent's index list
      const Supernode& P = S.sn[sn.parent];
      if (S.sn[sn.parent].level <= sn.level) return bad("levels");
      for (int32_t a = 0; a < sn.ms; ++a) {
        const int32_t pos = S.emap[sn.row_off + a], r = S.rows[sn.row_off + a];
        if (pos < 0 || pos >= P.F()) return bad("extend-add map range");
        const int32_t at = pos < P.ns() ? P.c0 + pos : S.rows[P.row_off + pos - P.ns()];
        if (at != r) return bad("extend-add map target");
      }
    }
  }
  if (next_col != N || maxF != S.max_front || S.emap.size() != S.rows.size()) return bad("supernode cover");
  const int64_t V = S.vec_off[nS];
  // assembly map
  if (!prefix_ok(S.amap_off, nS + 1, S.nnzA) || (int64_t)S.amap_src.size() != S.nnzA ||
      (int64_t)S.amap_dst.size() != S.nnzA || (int64_t)S.amap_coff.size() != V + 1 ||
      S.amap_coff[V] != S.nnzA)
    return bad("assembly map sizes");
  for (int64_t s = 0; s < nS; ++s) {
    const int64_t F = S.sn[s].F();
    if (S.amap_coff[S.vec_off[s]] != S.amap_off[s]) return bad("assembly column offsets");
    for (int64_t c = 0; c < F; ++c) {
      const int64_t q0 = S.amap_coff[S.vec_off[s] + c], q1 = S.amap_coff[S.vec_off[s] + c + 1];
      if (q0 > q1 || q1 > S.amap_off[s + 1]) return bad("assembly column offsets");
      for (int64_t q = q0; q < q1; ++q)
        if (S.amap_src[q] < 0 || S.amap_src[q] >= S.nnzA || S.amap_dst[q] < 0 || S.amap_dst[q] >= F * F ||
            S.amap_dst[q] / F != c)
          return bad("assembly map entries");
    }
  }
  // inverse extend-add map
  if (!prefix_ok(S.inv_off, (size_t)V + 1, (int64_t)S.inv_child.size())) return bad("inverse map offsets");
  const size_t nI = S.inv_child.size();
  if (S.inv_a.size() != nI || S.inv_vbase.size() != nI || S.inv_cF.size() != nI || S.inv_col.size() != nI)
    return bad("inverse map sizes");
  for (int64_t p = 0; p < nS; ++p)
    for (int64_t j = 0; j < S.sn[p].F(); ++j)
      for (int64_t q = S.inv_off[S.vec_off[p] + j]; q < S.inv_off[S.vec_off[p] + j + 1]; ++q) {
        const int32_t c = S.inv_child[q];
        if (c < 0 || c >= nS || S.sn[c].parent != p || S.inv_a[q] < 0 || S.inv_a[q] >= S.sn[c].ms ||
            S.emap[S.sn[c].row_off + S.inv_a[q]] != j || S.inv_vbase[q] != S.vec_off[c] ||
            S.inv_cF[q] != S.sn[c].F() || S.inv_col[q] != S.sn[c].ns() + S.inv_a[q])
          return bad("inverse map entries");
      }
  // children and levels
  if (!prefix_ok(S.child_off, nS + 1, (int64_t)S.child.size())) return bad("child offsets");
  for (int64_t s = 0; s < nS; ++s)
    for (int64_t q = S.child_off[s]; q < S.child_off[s + 1]; ++q)
      if (S.child[q] < 0 || S.child[q] >= nS || S.sn[S.child[q]].parent != s ||
          (q > S.child_off[s] && S.child[q] <= S.child[q - 1]))
        return bad("children");
  if (!prefix_ok(S.level_off, (size_t)S.n_levels + 1, nS) || (int64_t)S.level_sn.size() != nS)
    return bad("level offsets");
  std::vector<char> seen(nS, 0);
  for (int32_t l = 0; l < S.n_levels; ++l)
    for (int64_t q = S.level_off[l]; q < S.level_off[l + 1]; ++q) {
      const int32_t s = S.level_sn[q];
      if (s < 0 || s >= nS || seen[s] || S.sn[s].level != l) return bad("level schedule");
      seen[s] = 1;
    }
  return std::string();
}

}  // namespace pisp
