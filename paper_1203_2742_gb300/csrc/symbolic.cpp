// Host symbolic phase: ordering, elimination fill, elimination tree,
// supernode partition and clique tree (Algorithm 6.1), relaxed amalgamation,
// relative index maps for E_{J_p A_k}, workspace offsets and the launch
// schedule.
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
// cones": §2 (filled patterns, elimination tree, Eq. (e-filled),
// Eq. (e-etree-ch)), §6.1 (representative vertices, Eq. (e-repr-test)),
// §6.2 (supernodes, Eq. (e-new2)), §6.3 (clique tree), §6.4 (Algorithm 6.1),
// §1.5 (index sets and E_IJ), §8 (relaxed supernodes, tree parallelism).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <set>
#include <utility>
#include <vector>

#include "chd_internal.h"

namespace {

using std::vector;

// Off-diagonal adjacency lists (both directions) of the user's pattern.
bool build_adjacency(int64_t n, const int64_t* colptr, const int32_t* rowind,
                     vector<vector<int32_t>>& adj) {
  adj.assign(n, {});
  if (colptr[0] != 0) return false;
  for (int64_t j = 0; j < n; ++j) {
    if (colptr[j + 1] < colptr[j]) return false;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      int64_t i = rowind[p];
      if (i < j || i >= n) return false;
      if (i == j) continue;
      adj[j].push_back((int32_t)i);
      adj[i].push_back((int32_t)j);
    }
  }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  return true;
}

// Minimum-degree ordering on the quotient graph (eliminated vertices become
// "elements", cliques of their uneliminated neighbours; adjacent elements are
// absorbed).  The vertex of least exact external degree is eliminated next,
// smallest index on ties; once the least degree equals the number of
// remaining vertices minus one, the rest is a clique and is appended in
// index order.  Returns perm[new] = old.
vector<int64_t> minimum_degree(int64_t n, const vector<vector<int32_t>>& adj0) {
  vector<vector<int32_t>> vadj = adj0, eadj(n), evars(n);
  vector<char> state(n, 0);  // 0 variable, 1 element, 2 absorbed
  vector<int64_t> deg(n), mark(n, -1);
  int64_t stamp = 0;
  auto degree = [&](int64_t u) {
    ++stamp;
    mark[u] = stamp;
    int64_t cnt = 0;
    for (int32_t w : vadj[u])
      if (state[w] == 0 && mark[w] != stamp) { mark[w] = stamp; ++cnt; }
    for (int32_t e : eadj[u])
      for (int32_t w : evars[e])
        if (state[w] == 0 && mark[w] != stamp) { mark[w] = stamp; ++cnt; }
    return cnt;
  };
  std::set<std::pair<int64_t, int64_t>> pq;
  for (int64_t v = 0; v < n; ++v) { deg[v] = (int64_t)vadj[v].size(); pq.insert({deg[v], v}); }
  vector<int64_t> perm;
  perm.reserve(n);
  vector<int32_t> Lv;
  while (!pq.empty()) {
    auto it = pq.begin();
    int64_t v = it->second;
    if (it->first == (int64_t)pq.size() - 1) {  // remaining vertices form a clique
      vector<int64_t> rest;
      for (auto& q : pq) rest.push_back(q.second);
      std::sort(rest.begin(), rest.end());
      for (int64_t r : rest) perm.push_back(r);
      break;
    }
    pq.erase(it);
    // Lv = variables adjacent to v directly or through its elements
    ++stamp;
    mark[v] = stamp;
    Lv.clear();
    for (int32_t w : vadj[v])
      if (state[w] == 0 && mark[w] != stamp) { mark[w] = stamp; Lv.push_back(w); }
    for (int32_t e : eadj[v]) {
      for (int32_t w : evars[e])
        if (state[w] == 0 && mark[w] != stamp) { mark[w] = stamp; Lv.push_back(w); }
      state[e] = 2;
      vector<int32_t>().swap(evars[e]);
    }
    state[v] = 1;
    perm.push_back(v);
    evars[v] = Lv;
    vector<int32_t>().swap(vadj[v]);
    vector<int32_t>().swap(eadj[v]);
    const int64_t inL = stamp;  // mark[w] == inL  <=>  w in Lv ∪ {v}
    for (int32_t u : Lv) {
      vector<int32_t> ne;
      for (int32_t e : eadj[u])
        if (state[e] == 1) ne.push_back(e);
      ne.push_back((int32_t)v);
      eadj[u].swap(ne);
      vector<int32_t> nv;
      for (int32_t w : vadj[u])
        if (state[w] == 0 && mark[w] != inL) nv.push_back(w);
      vadj[u].swap(nv);
    }
    for (int32_t u : Lv) {
      pq.erase({deg[u], u});
      deg[u] = degree(u);
      pq.insert({deg[u], u});
    }
  }
  return perm;
}

// Lower pattern (strictly below the diagonal) of P A P^T, perm[new] = old.
void permuted_lower(int64_t n, const vector<vector<int32_t>>& adj, const vector<int64_t>& perm,
                    vector<vector<int32_t>>& low) {
  vector<int64_t> inv(n);
  for (int64_t i = 0; i < n; ++i) inv[perm[i]] = i;
  low.assign(n, {});
  for (int64_t jn = 0; jn < n; ++jn) {
    int64_t jo = perm[jn];
    for (int32_t io : adj[jo]) {
      int64_t in = inv[io];
      if (in > jn) low[jn].push_back((int32_t)in);
    }
    std::sort(low[jn].begin(), low[jn].end());
  }
}

// Filled pattern I_k of L: column k of L holds the rows of column k of the
// matrix below the diagonal together with I_c \ {k} for the children c of
// k in the elimination tree, whose parent is min I_c (§2; Eq. (e-etree-ch)).
void row_merge_fill(int64_t n, const vector<vector<int32_t>>& low, vector<vector<int32_t>>& I,
                    vector<int64_t>& parent) {
  I.assign(n, {});
  parent.assign(n, -1);
  vector<vector<int32_t>> kids(n);
  vector<int64_t> mark(n, -1);
  for (int64_t k = 0; k < n; ++k) {
    vector<int32_t>& s = I[k];
    for (int32_t r : low[k])
      if (mark[r] != k) { mark[r] = k; s.push_back(r); }
    for (int32_t c : kids[k])
      for (int32_t r : I[c])
        if (r != k && mark[r] != k) { mark[r] = k; s.push_back(r); }
    std::sort(s.begin(), s.end());
    if (!s.empty()) {
      parent[k] = s[0];
      kids[s[0]].push_back((int32_t)k);
    }
  }
}

// Algorithm 6.1, step 1: chain child of each vertex (the child whose
// supernode it joins) or -1 when the vertex is representative
// (Eq. (e-repr-test)).  Children are scanned in increasing index order;
// tie_last picks the eligible child of largest index, otherwise smallest.
vector<int64_t> chain_children(int64_t n, const vector<vector<int32_t>>& I, const vector<int64_t>& parent,
                               bool tie_last) {
  vector<int64_t> chain(n, -1);
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = parent[j];
    if (p < 0) continue;
    if ((int64_t)I[j].size() == (int64_t)I[p].size() + 1) {
      if (chain[p] < 0) chain[p] = j;
      else if (tie_last) chain[p] = std::max(chain[p], j);
      else chain[p] = std::min(chain[p], j);
    }
  }
  return chain;
}

// Postorder of the elimination forest in which each vertex's chain child
// is visited last among its children, so supernodes become contiguous.
vector<int64_t> chain_postorder(int64_t n, const vector<int64_t>& parent, const vector<int64_t>& chain) {
  vector<vector<int64_t>> kids(n);
  vector<int64_t> roots;
  for (int64_t j = 0; j < n; ++j) {
    if (parent[j] < 0) roots.push_back(j);
    else kids[parent[j]].push_back(j);
  }
  for (int64_t v = 0; v < n; ++v) {
    if (chain[v] >= 0) {
      auto& k = kids[v];
      auto it = std::find(k.begin(), k.end(), chain[v]);
      if (it != k.end()) { k.erase(it); k.push_back(chain[v]); }
    }
  }
  vector<int64_t> post;
  post.reserve(n);
  vector<std::pair<int64_t, size_t>> st;
  for (int64_t r : roots) {
    st.push_back({r, 0});
    while (!st.empty()) {
      auto& top = st.back();
      if (top.second < kids[top.first].size()) {
        int64_t c = kids[top.first][top.second++];
        st.push_back({c, 0});
      } else {
        post.push_back(top.first);
        st.pop_back();
      }
    }
  }
  return post;  // post[new] = old (in the current numbering)
}

}  // namespace

namespace {

// Lexicographic order (x fastest) of the box [lo, hi).
void lex_box(const int64_t* dims, const int64_t* lo, const int64_t* hi, vector<int64_t>& out) {
  for (int64_t z = lo[2]; z < hi[2]; ++z)
    for (int64_t y = lo[1]; y < hi[1]; ++y)
      for (int64_t x = lo[0]; x < hi[0]; ++x) out.push_back(x + dims[0] * (y + dims[1] * z));
}

// Geometric nested dissection of a grid whose vertex (x, y, z) has index
// x + dims[0] (y + dims[1] z): the box is cut along its longest side (the
// first such axis on ties) by the plane through its middle; both halves are
// ordered first, the lower one before the upper one, then the plane
// (lexicographically).  Boxes of at most `leaf` vertices, or whose longest
// side is shorter than 3, are ordered lexicographically.  The separators are
// eliminated last, so the fill stays inside the halves and the separators.
void nd_box(const int64_t* dims, const int64_t* lo, const int64_t* hi, int64_t leaf, vector<int64_t>& out) {
  int64_t ext[3], size = 1;
  for (int d = 0; d < 3; ++d) {
    ext[d] = hi[d] - lo[d];
    size *= ext[d];
  }
  if (size == 0) return;
  int ax = 0;
  for (int d = 1; d < 3; ++d)
    if (ext[d] > ext[ax]) ax = d;
  if (size <= leaf || ext[ax] < 3) {
    lex_box(dims, lo, hi, out);
    return;
  }
  const int64_t mid = lo[ax] + ext[ax] / 2;
  int64_t h1[3] = {hi[0], hi[1], hi[2]}, l2[3] = {lo[0], lo[1], lo[2]};
  int64_t sl[3] = {lo[0], lo[1], lo[2]}, sh[3] = {hi[0], hi[1], hi[2]};
  h1[ax] = mid;
  l2[ax] = mid + 1;
  sl[ax] = mid;
  sh[ax] = mid + 1;
  nd_box(dims, lo, h1, leaf, out);
  nd_box(dims, l2, hi, leaf, out);
  lex_box(dims, sl, sh, out);
}

// Ordering of a pattern by its options; perm[new] = old.
chd_status order_of(int64_t n, const vector<vector<int32_t>>& adj, const chd_opts& opts, vector<int64_t>& perm) {
  perm.assign(n, 0);
  if (opts.ordering == CHD_ORDER_NATURAL) {
    std::iota(perm.begin(), perm.end(), 0);
  } else if (opts.ordering == CHD_ORDER_USER) {
    if (!opts.user_perm) return CHD_ERR_INVALID;
    vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
      int64_t v = opts.user_perm[i];
      if (v < 0 || v >= n || seen[v]) return CHD_ERR_INVALID;
      seen[v] = 1;
      perm[i] = v;
    }
  } else if (opts.ordering == CHD_ORDER_MINDEG) {
    perm = minimum_degree(n, adj);
  } else if (opts.ordering == CHD_ORDER_ND_GEOMETRIC) {
    const int64_t dims[3] = {opts.nd_dims[0], opts.nd_dims[1], opts.nd_dims[2]};
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || dims[0] * dims[1] * dims[2] != n) return CHD_ERR_INVALID;
    const int64_t lo[3] = {0, 0, 0};
    perm.clear();
    perm.reserve(n);
    nd_box(dims, lo, dims, opts.nd_leaf > 0 ? opts.nd_leaf : 8, perm);
  } else {
    return CHD_ERR_INVALID;
  }
  return CHD_OK;
}

}  // namespace

// Ordering of one pattern by its options; validates the pattern.
// perm[new] = old.
chd_status chd_order_pattern(int64_t n, const int64_t* colptr, const int32_t* rowind, const chd_opts& opts,
                             std::vector<int64_t>& perm) {
  if (n < 1 || !colptr || !rowind) return CHD_ERR_INVALID;
  vector<vector<int32_t>> adj;
  if (!build_adjacency(n, colptr, rowind, adj)) return CHD_ERR_INVALID;
  return order_of(n, adj, opts, perm);
}

void chd_opts_default(chd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->ordering = CHD_ORDER_NATURAL;
  o->user_perm = nullptr;
  o->relax = 0;
  o->tie_last = 1;
  o->chain_runs = 1;
}

// Plan of the completion with factored update matrices (Algorithm 4.3 in the
// supernodal form of §7.2): V_k = R_k R_k^T is propagated from the parent p
// of k.  Of A_k, the q_k rows in A_p (positions >= n_p of J_p) take their
// factor from rows of R_p, re-triangularised by Householder reflections; the
// p_k = a_k - q_k rows in N_p are added by a triangular solve and a Cholesky
// factorisation.  Held reversed (G_k = P R_k P lower, P the order reversal),
// row t < q_k of G_k comes from row rho_t = J_p - 1 - pos(A_k[a_k - 1 - t])
// of G_p; the reduction works on the q_k x w_k rows, w_k = rho_{q_k - 1} + 1.
// Fronts are grouped by depth in the clique tree (parents first); a leaf
// group's members share one A_k and are handled by its first member.  Per
// depth level the scratch of the reductions is laid out front after front.
// Flop counts: the independent form's Cholesky of every V_k (a^3/3) against
// the factored form (reflections, solve, update and Cholesky of the p_k
// block).
void factored_completion_plan(chd_symbolic* s) {
  const int64_t nsn = s->nsn;
  s->fc_off.assign(nsn, 0);
  s->fc_fronts.clear();
  s->fc_lvl.assign(1, 0);
  s->fc_big.clear();
  s->fc_big_lvl.assign(1, 0);
  s->fc_total = 0;
  s->fc_flops[0] = s->fc_flops[1] = 0.0;
  vector<int32_t> depth(nsn, 0);
  int32_t maxd = 0;
  for (int64_t k = nsn - 1; k >= 0; --k) {
    const int64_t p = s->sn_par[k];
    depth[k] = p >= 0 ? depth[p] + 1 : 0;
    maxd = std::max(maxd, depth[k]);
  }
  vector<vector<int32_t>> by_depth(maxd + 1);
  for (int64_t k = 0; k < nsn; ++k) {
    const int64_t nk = s->sn_ptr[k + 1] - s->sn_ptr[k];
    const int64_t a = s->rows_ptr[k + 1] - s->rows_ptr[k] - nk;
    const bool member = s->grp_of[k] >= 0 && s->grp_first[s->grp_of[k]] != k;
    if (a == 0 || member) continue;
    by_depth[depth[k]].push_back((int32_t)k);
  }
  for (int32_t d = 0; d <= maxd; ++d) {
    int64_t used = 0;
    for (int32_t k : by_depth[d]) {
      const int64_t nk = s->sn_ptr[k + 1] - s->sn_ptr[k];
      const int64_t a = s->rows_ptr[k + 1] - s->rows_ptr[k] - nk;
      const int64_t p = s->sn_par[k];
      const int64_t np = s->sn_ptr[p + 1] - s->sn_ptr[p];
      const int64_t Jp = s->rows_ptr[p + 1] - s->rows_ptr[p];
      const int32_t* rel = s->rel.data() + s->rows_ptr[k] + nk;
      int64_t q = 0;
      for (int64_t r = 0; r < a; ++r) q += rel[r] >= np ? 1 : 0;
      const int64_t w = q > 0 ? Jp - rel[a - q] : 0;
      // the reflections are a sequential chain: the dense tier takes fronts
      // with a large reduction or a large p-block, in panels of 32 rows
      // (scratch: X, then the panel's reflectors V, its T, V T and the
      // trailing rows' product)
      const bool big = s->is_big[k] || a > 256;
      s->fc_off[k] = used;
      used += (q * w + 3) & ~int64_t(3);
      if (big && q > 0) used += 32 * (2 * w + q + 32);
      const double da = (double)a, dq = (double)q, dp = (double)(a - q);
      double hh = 0.0;
      for (int64_t t = 0; t < q; ++t) {
        const int64_t rho = Jp - 1 - rel[a - 1 - t];
        if (rho > t) hh += 4.0 * (double)(rho - t + 1) * (double)(q - t);
      }
      s->fc_flops[0] += da * da * da / 3;
      s->fc_flops[1] += hh + dp * dq * dq + dp * dp * dq + dp * dp * dp / 3;
      if (big)
        s->fc_big.push_back(k);
      else
        s->fc_fronts.push_back(k);
    }
    s->fc_total = std::max(s->fc_total, used);
    s->fc_lvl.push_back((int32_t)s->fc_fronts.size());
    s->fc_big_lvl.push_back((int32_t)s->fc_big.size());
  }
}

chd_status chd_symbolic_build(int64_t n, const int64_t* colptr, const int32_t* rowind,
                              const chd_opts& opts, chd_symbolic* s) {
  if (n < 1 || !colptr || !rowind) return CHD_ERR_INVALID;
  vector<vector<int32_t>> adj;
  if (!build_adjacency(n, colptr, rowind, adj)) return CHD_ERR_INVALID;
  s->tc_mode = opts.tc_products < 0 ? -1 : (opts.tc_products > 0 ? 1 : 0);
  if (opts.completion < 0 || opts.completion > 1) return CHD_ERR_INVALID;
  s->completion_mode = opts.completion;

  // ---- ordering -----------------------------------------------------------
  vector<int64_t> perm0;
  if (chd_status rc = order_of(n, adj, opts, perm0)) return rc;

  // ---- pass 1: fill + Algorithm 6.1 chains -> contiguous postorder --------
  vector<vector<int32_t>> low, I;
  vector<int64_t> parent;
  permuted_lower(n, adj, perm0, low);
  row_merge_fill(n, low, I, parent);
  vector<int64_t> chain = chain_children(n, I, parent, opts.tie_last != 0);
  vector<int64_t> post = chain_postorder(n, parent, chain);
  vector<int64_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = perm0[post[i]];

  // ---- pass 2: final numbering ---------------------------------------------
  permuted_lower(n, adj, perm, low);
  row_merge_fill(n, low, I, parent);
  low.clear();
  low.shrink_to_fit();
  // In the postorder the chain child of i is i-1 (the largest child index).
  chain = chain_children(n, I, parent, true);

  // Supernodes: maximal runs j0..j1 where chain[j] == j-1 for j in (j0, j1].
  vector<int64_t> first;  // first column of each fundamental supernode
  for (int64_t j = 0; j < n; ++j)
    if (!(chain[j] == j - 1 && j > 0)) first.push_back(j);
  int64_t ns = (int64_t)first.size();
  vector<int64_t> last(ns);
  for (int64_t k = 0; k < ns; ++k) last[k] = (k + 1 < ns ? first[k + 1] : n) - 1;
  // A_k = I_{last} (the clique's ancestor set, Eq. (e-new2)); n_k, a_k.
  vector<int64_t> nk(ns), ak(ns);
  vector<int64_t> snode_of(n);
  for (int64_t k = 0; k < ns; ++k) {
    nk[k] = last[k] - first[k] + 1;
    ak[k] = (int64_t)I[last[k]].size();
    for (int64_t j = first[k]; j <= last[k]; ++j) snode_of[j] = k;
  }
  // Each supernode's structure: I_first = N_k \ {first} ∪ A_k must hold.
  for (int64_t k = 0; k < ns; ++k) {
    if ((int64_t)I[first[k]].size() != nk[k] - 1 + ak[k]) return CHD_ERR_INVALID;
  }
  vector<vector<int32_t>> A(ns);
  for (int64_t k = 0; k < ns; ++k) A[k] = I[last[k]];
  I.clear();
  I.shrink_to_fit();

  // ---- relaxed amalgamation -------------------------------------------------
  // Merge the child supernode c whose columns end right before p's first
  // column (c is then a clique-tree child of p: min A_c = first(p)) when the
  // merge adds at most `relax` explicit zeros: the merged node has
  // N = N_c ∪ N_p and A = A_p, so each column of N_c gains
  // |J_p| - |A_c| new entries.
  vector<char> alive(ns, 1);
  if (opts.relax > 0) {
    vector<int64_t> owner(n);  // column -> current supernode id
    for (int64_t j = 0; j < n; ++j) owner[j] = snode_of[j];
    for (int64_t p = 0; p < ns; ++p) {
      bool merged = true;
      while (merged) {
        merged = false;
        int64_t f = first[p];
        if (f == 0) break;
        int64_t c = owner[f - 1];
        if (!alive[c] || c == p) break;
        if (A[c].empty() || A[c][0] != f) break;
        int64_t zeros = nk[c] * (nk[p] + ak[p] - ak[c]);
        if (zeros <= opts.relax) {
          alive[c] = 0;
          first[p] = first[c];
          nk[p] += nk[c];
          for (int64_t j = first[c]; j <= last[c]; ++j) owner[j] = p;
          A[c].clear();
          merged = true;
        }
      }
    }
  }

  // ---- supernode splitting ---------------------------------------------------
  // A supernode wider than split_cols columns becomes a chain of supernodes of
  // at most split_cols columns: piece i keeps its own columns as N and the
  // later columns of the original N together with A as its ancestor set, so
  // every column keeps its structure and V is unchanged (it is the same
  // clique, partitioned more finely; §6.2 allows any such path partition).
  // The parent of a piece is the next piece, the last piece keeps the
  // original parent.  Wide dense fronts then cost ~2n^3 per Hessian
  // right-hand side instead of the ~3n^3 of products with a dense D_NN^{-1}.
  {
    const int64_t split = opts.split_cols == 0 ? 256 : opts.split_cols;
    if (split > 0) {
      vector<int64_t> nfirst, nlast;
      vector<vector<int32_t>> nA;
      vector<char> nalive;
      for (int64_t k = 0; k < ns; ++k) {
        if (!alive[k]) continue;
        const int64_t w = last[k] - first[k] + 1;
        if (w <= split + split / 2) {
          nfirst.push_back(first[k]);
          nlast.push_back(last[k]);
          nA.push_back(A[k]);
          nalive.push_back(1);
          continue;
        }
        for (int64_t c0 = first[k]; c0 <= last[k]; c0 += split) {
          const int64_t c1 = std::min(last[k], c0 + split - 1);
          vector<int32_t> anc;
          for (int64_t j = c1 + 1; j <= last[k]; ++j) anc.push_back((int32_t)j);
          anc.insert(anc.end(), A[k].begin(), A[k].end());
          nfirst.push_back(c0);
          nlast.push_back(c1);
          nA.push_back(std::move(anc));
          nalive.push_back(1);
        }
      }
      first.swap(nfirst);
      last.swap(nlast);
      A.swap(nA);
      alive.swap(nalive);
      ns = (int64_t)first.size();
    }
  }

  // ---- final supernodes, clique tree, J lists, relative indices -----------
  vector<int64_t> ids;
  for (int64_t k = 0; k < ns; ++k)
    if (alive[k]) ids.push_back(k);
  const int64_t nsn = (int64_t)ids.size();
  s->n = n;
  s->perm = perm;
  s->nsn = nsn;
  s->sn_ptr.assign(nsn + 1, 0);
  s->sn_par.assign(nsn, -1);
  s->rows_ptr.assign(nsn + 1, 0);
  vector<int64_t> col_owner(n);
  for (int64_t t = 0; t < nsn; ++t) {
    int64_t k = ids[t];
    s->sn_ptr[t] = first[k];
    for (int64_t j = first[k]; j <= last[k]; ++j) col_owner[j] = t;
  }
  s->sn_ptr[nsn] = n;
  for (int64_t t = 0; t < nsn; ++t) {
    if (s->sn_ptr[t + 1] <= s->sn_ptr[t]) return CHD_ERR_INVALID;
    s->rows_ptr[t + 1] = s->rows_ptr[t] + (s->sn_ptr[t + 1] - s->sn_ptr[t]) + (int64_t)A[ids[t]].size();
  }
  s->rows.assign(s->rows_ptr[nsn], 0);
  s->rel.assign(s->rows_ptr[nsn], -1);
  int64_t maxJ = 0;
  for (int64_t t = 0; t < nsn; ++t) {
    int64_t k = ids[t];
    int64_t o = s->rows_ptr[t];
    for (int64_t j = s->sn_ptr[t]; j < s->sn_ptr[t + 1]; ++j) s->rows[o++] = (int32_t)j;
    for (int32_t r : A[k]) s->rows[o++] = r;
    if (!A[k].empty()) s->sn_par[t] = col_owner[A[k][0]];
    maxJ = std::max(maxJ, s->rows_ptr[t + 1] - s->rows_ptr[t]);
  }
  s->max_front = maxJ;
  // relative positions of A_t inside J_par(t) (E_{J_p A_t}, §1.5)
  {
    vector<int32_t> pos(n, -1);
    vector<vector<int64_t>> kids(nsn);
    for (int64_t t = 0; t < nsn; ++t)
      if (s->sn_par[t] >= 0) kids[s->sn_par[t]].push_back(t);
    s->ch_ptr.assign(nsn + 1, 0);
    for (int64_t p = 0; p < nsn; ++p) s->ch_ptr[p + 1] = s->ch_ptr[p] + (int64_t)kids[p].size();
    s->ch.assign(s->ch_ptr[nsn], 0);
    for (int64_t p = 0; p < nsn; ++p) {
      for (size_t q = 0; q < kids[p].size(); ++q) s->ch[s->ch_ptr[p] + q] = (int32_t)kids[p][q];
      for (int64_t o = s->rows_ptr[p]; o < s->rows_ptr[p + 1]; ++o) pos[s->rows[o]] = (int32_t)(o - s->rows_ptr[p]);
      for (int64_t c : kids[p]) {
        int64_t nc = s->sn_ptr[c + 1] - s->sn_ptr[c];
        for (int64_t o = s->rows_ptr[c] + nc; o < s->rows_ptr[c + 1]; ++o) {
          int32_t r = pos[s->rows[o]];
          if (r < 0) return CHD_ERR_INVALID;  // A_c ⊄ J_p: not a clique tree
          s->rel[o] = r;
        }
      }
      for (int64_t o = s->rows_ptr[p]; o < s->rows_ptr[p + 1]; ++o) pos[s->rows[o]] = -1;
    }
  }

  // ---- leaf groups -----------------------------------------------------------
  // A run of at least kMinLeafGroup consecutive supernodes that are leaves
  // with one column each, below the dense-tier size, sharing their parent and
  // their ancestor set A (the border of a block-arrow pattern, for instance)
  // forms a group.  With n_k = 1 the per-front formulas of Algorithms 7.1-7.3
  // and of the Hessian recursions become, over the whole group, products of
  // the a x L block of the leaves' columns (L leaves), and the update blocks
  // the parent adds are one sum over the group, computed as such products.
  {
    constexpr int64_t kMinLeafGroup = 16;
    const int64_t big_rows = opts.big_rows > 0 ? opts.big_rows : 320;
    s->grp_first.clear();
    s->grp_count.clear();
    s->grp_of.assign(nsn, -1);
    auto leaf1 = [&](int64_t t) {
      const int64_t J = s->rows_ptr[t + 1] - s->rows_ptr[t];
      return s->ch_ptr[t + 1] == s->ch_ptr[t] && s->sn_ptr[t + 1] - s->sn_ptr[t] == 1 && s->sn_par[t] >= 0 &&
             J > 1 && J < big_rows;
    };
    auto sameA = [&](int64_t t, int64_t u) {
      const int64_t Jt = s->rows_ptr[t + 1] - s->rows_ptr[t];
      if (s->rows_ptr[u + 1] - s->rows_ptr[u] != Jt) return false;
      for (int64_t q = 1; q < Jt; ++q)
        if (s->rows[s->rows_ptr[t] + q] != s->rows[s->rows_ptr[u] + q]) return false;
      return true;
    };
    for (int64_t t = 0; t < nsn;) {
      if (!leaf1(t)) {
        ++t;
        continue;
      }
      int64_t u = t + 1;
      while (u < nsn && leaf1(u) && s->sn_par[u] == s->sn_par[t] && sameA(t, u)) ++u;
      if (u - t >= kMinLeafGroup) {
        for (int64_t k = t; k < u; ++k) s->grp_of[k] = (int32_t)s->grp_first.size();
        s->grp_first.push_back(t);
        s->grp_count.push_back(u - t);
      }
      t = u;
    }
    s->ea_ptr.assign(nsn + 1, 0);
    s->ea.clear();
    for (int64_t p = 0; p < nsn; ++p) {
      for (int64_t q = s->ch_ptr[p]; q < s->ch_ptr[p + 1]; ++q) {
        const int32_t c = s->ch[q];
        if (s->grp_of[c] >= 0 && s->grp_first[s->grp_of[c]] != c) continue;
        s->ea.push_back(c);
      }
      s->ea_ptr[p + 1] = (int64_t)s->ea.size();
    }
  }

  // ---- CSC of the filled pattern V (column j of N_k: rows J_k[c:]) -------
  s->colptr.assign(n + 1, 0);
  for (int64_t t = 0; t < nsn; ++t) {
    int64_t J = s->rows_ptr[t + 1] - s->rows_ptr[t];
    for (int64_t j = s->sn_ptr[t]; j < s->sn_ptr[t + 1]; ++j)
      s->colptr[j + 1] = J - (j - s->sn_ptr[t]);
  }
  for (int64_t j = 0; j < n; ++j) s->colptr[j + 1] += s->colptr[j];
  s->rowind.assign(s->colptr[n], 0);
  for (int64_t t = 0; t < nsn; ++t) {
    for (int64_t j = s->sn_ptr[t]; j < s->sn_ptr[t + 1]; ++j) {
      int64_t c = j - s->sn_ptr[t];
      int64_t o = s->colptr[j];
      for (int64_t q = s->rows_ptr[t] + c; q < s->rows_ptr[t + 1]; ++q) s->rowind[o++] = s->rows[q];
    }
  }

  // ---- workspace offsets and algorithmic flop counts (§8 measurement) ----
  s->f_off.assign(nsn + 1, 0);
  s->d_off.assign(nsn + 1, 0);
  s->v_off.assign(nsn + 1, 0);
  for (double& f : s->flops) f = 0;
  for (int64_t t = 0; t < nsn; ++t) {
    int64_t nn = s->sn_ptr[t + 1] - s->sn_ptr[t];
    int64_t J = s->rows_ptr[t + 1] - s->rows_ptr[t];
    int64_t a = J - nn;
    // front F (J x J) + two J x n temporaries; rounded to 4 doubles (32 B)
    int64_t fsz = J * J + 2 * J * nn;
    fsz = (fsz + 3) & ~int64_t(3);
    s->f_off[t + 1] = s->f_off[t] + fsz;
    s->d_off[t + 1] = s->d_off[t] + ((nn * nn + 3) & ~int64_t(3));
    // a leaf group keeps one V (its members share A) in its first member's slot
    const bool v_shared = s->grp_of[t] >= 0 && s->grp_first[s->grp_of[t]] != t;
    s->v_off[t + 1] = s->v_off[t] + (v_shared ? 0 : ((a * a + 3) & ~int64_t(3)));
    double dn = (double)nn, da = (double)a;
    s->flops[0] += dn * dn * dn / 3 + da * dn * dn + da * da * dn;
    s->flops[1] += 2 * da * da * dn + da * dn * dn + 2 * dn * dn * dn / 3;
    s->flops[2] += 6 * da * da * dn + 8 * da * dn * dn + 2 * dn * dn * dn;
    s->flops[3] += 6 * da * da * dn + 8 * da * dn * dn + 2 * dn * dn * dn + 4 * da * da * dn;
    s->flops[4] += da * da * da / 3 + da * da * dn + da * dn * dn + dn * dn * dn;
  }

  // ---- schedule -------------------------------------------------------------
  // Each front gets a tier: warp (|N| <= 8 and |J| <= 32, one warp per front),
  // wide warp (|N| <= 8 and |J| <= 64, one warp per front), CTA (one
  // 256-thread CTA per front) or dense (|J| >= big_rows or |N| >= big_cols,
  // multi-CTA sequence).  Maximal subtrees of warp-tier
  // fronts whose total work is at most total/(8*152) become single-warp
  // tasks processed in postorder (tree parallelism, §8); the fronts above
  // form chains (a front joins its only such child when both have the same
  // tier, dense fronts never chain), one task each.  A task's level exceeds
  // the levels of the tasks it depends on; every level is launched as one
  // warp-tier kernel, one CTA-tier kernel and one dense sequence per front.
  {
    const int64_t big_rows = opts.big_rows > 0 ? opts.big_rows : 320;
    const int64_t big_cols = opts.big_cols > 0 ? opts.big_cols : 160;
    s->is_big.assign(nsn, 0);
    vector<int> tier(nsn, 1);
    for (int64_t t = 0; t < nsn; ++t) {
      int64_t nn = s->sn_ptr[t + 1] - s->sn_ptr[t];
      int64_t J = s->rows_ptr[t + 1] - s->rows_ptr[t];
      s->is_big[t] = (J >= big_rows || nn >= big_cols) ? 1 : 0;
      if (opts.tier_table) {
        auto bucket = [](int64_t v) {
          int b = 0;
          while (v > 0 && b < CHD_TIER_BUCKETS - 1) {
            ++b;
            v >>= 1;
          }
          return b;
        };
        const int32_t e = opts.tier_table[bucket(nn) * CHD_TIER_BUCKETS + bucket(J - nn)];
        if (e == 0) s->is_big[t] = 0;
        if (e == 1) s->is_big[t] = 1;
      }
      tier[t] = s->is_big[t] ? 2 : (nn <= 8 && J <= 32) ? 0 : (nn <= 8 && J <= 64) ? 3 : 1;
      if (s->grp_of[t] >= 0) {
        tier[t] = 4;
        s->is_big[t] = 0;
      }
    }
    // The wide warp tier runs one warp per CTA (its fronts take most of the
    // shared memory), which pays off for chains, where one front waits for
    // the previous one, not for many independent fronts: a front keeps it
    // only when it is linked to another such front as only child or parent.
    {
      vector<int64_t> nkids(nsn, 0);
      for (int64_t t = 0; t < nsn; ++t)
        if (s->sn_par[t] >= 0) nkids[s->sn_par[t]]++;
      vector<char> chained(nsn, 0);
      for (int64_t t = 0; t < nsn; ++t) {
        const int64_t p = s->sn_par[t];
        if (p >= 0 && tier[t] == 3 && tier[p] == 3 && nkids[p] == 1) chained[t] = chained[p] = 1;
      }
      for (int64_t t = 0; t < nsn; ++t)
        if (tier[t] == 3 && !chained[t]) tier[t] = 1;
    }
    s->tier.assign(tier.begin(), tier.end());
    s->small_fronts.clear();
    s->cta_fronts.clear();
    s->warp_fronts.clear();
    s->big_fronts.clear();
    s->plain_fronts.clear();
    for (int64_t t = 0; t < nsn; ++t) {
      // V^{-1} per front (a group's members share their first member's)
      const bool member = s->grp_of[t] >= 0 && s->grp_first[s->grp_of[t]] != t;
      if (!s->is_big[t] && !member) s->small_fronts.push_back((int32_t)t);
      if (tier[t] == 0) s->warp_fronts.push_back((int32_t)t);
      if (tier[t] == 1 || tier[t] == 3) s->cta_fronts.push_back((int32_t)t);
      if (tier[t] == 2) s->big_fronts.push_back((int32_t)t);
      if (tier[t] == 0 || tier[t] == 1 || tier[t] == 3) s->plain_fronts.push_back((int32_t)t);
    }
    // subtree ranges (the numbering is a postorder: subtrees are contiguous);
    // a leaf group's first member stands for the whole group
    {
      vector<int64_t> size(nsn, 1);
      for (int64_t t = 0; t < nsn; ++t)
        if (s->sn_par[t] >= 0) size[s->sn_par[t]] += size[t];
      s->sub_lo.assign(nsn, 0);
      s->sub_hi.assign(nsn, 0);
      for (int64_t t = 0; t < nsn; ++t) {
        s->sub_lo[t] = (int32_t)(t - size[t] + 1);
        s->sub_hi[t] = (int32_t)t;
      }
      for (size_t g = 0; g < s->grp_first.size(); ++g)
        s->sub_hi[s->grp_first[g]] = (int32_t)(s->grp_first[g] + s->grp_count[g] - 1);
    }
    vector<double> W(nsn, 0.0);
    double total = 0;
    for (int64_t t = 0; t < nsn; ++t) {  // children precede parents
      int64_t nn = s->sn_ptr[t + 1] - s->sn_ptr[t];
      int64_t a = (s->rows_ptr[t + 1] - s->rows_ptr[t]) - nn;
      double dn = (double)nn, da = (double)a;
      W[t] += 6 * da * da * dn + 8 * da * dn * dn + 2 * dn * dn * dn + (tier[t] == 0 ? 2.0e4 : 5.0e4);
      if (s->sn_par[t] >= 0) W[s->sn_par[t]] += W[t];
      else total += W[t];
    }
    const double thr = total / (8.0 * 152.0);
    vector<char> top(nsn, 0);
    for (int64_t t = 0; t < nsn; ++t) top[t] = W[t] > thr || tier[t] != 0;
    for (int64_t t = 0; t < nsn; ++t)  // ancestors of top fronts are top fronts
      if (top[t] && s->sn_par[t] >= 0) top[s->sn_par[t]] = 1;
    vector<int64_t> task_of(nsn, -1);
    vector<vector<int32_t>> tasks;
    vector<int64_t> tlevel;
    vector<int> ttier;
    // chain runs (option chain_runs): maximal sequences t0 < ... < t1 of
    // one-column fronts with rows {j, j+1, .., j+a}, the same a (1..64), each
    // the only child of the next, t0 a leaf; at least kMinRun fronts.  Each
    // run is one task of task tier 5 (|J| <= 32) or 6 (|J| <= 64).
    constexpr int64_t kMinRun = 8;
    vector<int64_t> run_of(nsn, -1);
    if (opts.chain_runs > 0) {
      auto a_of = [&](int64_t t) { return (s->rows_ptr[t + 1] - s->rows_ptr[t]) - (s->sn_ptr[t + 1] - s->sn_ptr[t]); };
      auto nkids = [&](int64_t t) { return s->ch_ptr[t + 1] - s->ch_ptr[t]; };
      auto fits = [&](int64_t t) {
        if (s->sn_ptr[t + 1] - s->sn_ptr[t] != 1 || s->is_big[t] || s->grp_of[t] >= 0) return false;
        const int64_t a = a_of(t);
        if (a < 1 || a > 64) return false;
        for (int64_t i = 0; i <= a; ++i)
          if (s->rows[s->rows_ptr[t] + i] != s->sn_ptr[t] + i) return false;
        return true;
      };
      int64_t t = 0;
      while (t < nsn) {
        if (!fits(t) || nkids(t) != 0) {
          ++t;
          continue;
        }
        int64_t u = t;
        while (u + 1 < nsn && s->sn_par[u] == u + 1 && fits(u + 1) && a_of(u + 1) == a_of(t) && nkids(u + 1) == 1)
          ++u;
        if (u - t + 1 >= kMinRun) {
          const int64_t id = (int64_t)tasks.size();
          vector<int32_t> seq;
          for (int64_t v = t; v <= u; ++v) {
            seq.push_back((int32_t)v);
            run_of[v] = id;
            task_of[v] = id;
          }
          tasks.push_back(seq);
          tlevel.push_back(0);
          ttier.push_back(a_of(t) + 1 <= 32 ? 5 : 6);
        }
        t = u + 1;
      }
    }
    // Supernode numbering is a postorder of the clique tree (children precede
    // parents, subtrees are contiguous), so the subtree of t is [t - size(t) + 1, t].
    vector<int64_t> sub(nsn, 1);
    for (int64_t t = 0; t < nsn; ++t)
      if (s->sn_par[t] >= 0) sub[s->sn_par[t]] += sub[t];
    for (int64_t t = 0; t < nsn; ++t) {
      if (top[t]) continue;
      int64_t p = s->sn_par[t];
      if (p >= 0 && !top[p]) continue;
      vector<int32_t> seq;
      for (int64_t u = t - sub[t] + 1; u <= t; ++u) {
        if (run_of[u] >= 0) continue;  // in its own chain-run task
        seq.push_back((int32_t)u);
        task_of[u] = (int64_t)tasks.size();
      }
      if (seq.empty()) continue;
      tasks.push_back(seq);
      tlevel.push_back(0);
      ttier.push_back(0);
    }
    vector<int64_t> ntopkids(nsn, 0), onlykid(nsn, -1);
    for (int64_t t = 0; t < nsn; ++t)
      if (top[t] && s->sn_par[t] >= 0) { ntopkids[s->sn_par[t]]++; onlykid[s->sn_par[t]] = t; }
    for (int64_t t = 0; t < nsn; ++t) {
      if (!top[t] || run_of[t] >= 0) continue;
      if (tier[t] == 4) {  // leaf group: one task, run with the dense fronts
        const int64_t g0 = s->grp_first[s->grp_of[t]];
        if (g0 == t) {
          task_of[t] = (int64_t)tasks.size();
          tasks.push_back({(int32_t)t});
          tlevel.push_back(1);
          ttier.push_back(2);
        } else {
          task_of[t] = task_of[g0];
        }
        continue;
      }
      if (ntopkids[t] == 1 && tier[t] != 2 && tier[onlykid[t]] == tier[t] && run_of[onlykid[t]] < 0) {
        int64_t tk = task_of[onlykid[t]];
        tasks[tk].push_back((int32_t)t);
        task_of[t] = tk;
      } else {
        task_of[t] = (int64_t)tasks.size();
        tasks.push_back({(int32_t)t});
        tlevel.push_back(1);
        ttier.push_back(tier[t]);
      }
    }
    // A task's level must exceed the levels of all tasks it depends on.  One
    // pass in postorder suffices: when front t is reached, every child task
    // that ends below t is complete (its fronts all precede t).
    for (int64_t t = 0; t < nsn; ++t) {
      const int64_t tk = task_of[t];
      for (int64_t q = s->ch_ptr[t]; q < s->ch_ptr[t + 1]; ++q) {
        const int64_t tc = task_of[s->ch[q]];
        if (tc != tk && tlevel[tk] <= tlevel[tc]) tlevel[tk] = tlevel[tc] + 1;
      }
    }
    int64_t nlev = 0;
    for (int64_t l : tlevel) nlev = std::max(nlev, l + 1);
    vector<vector<int64_t>> bylev(nlev);
    for (size_t q = 0; q < tasks.size(); ++q) bylev[tlevel[q]].push_back((int64_t)q);
    s->task_ptr.assign(1, 0);
    s->task_fronts.clear();
    s->lvl_ptr.assign(1, 0);
    s->lvl_r32.clear();
    s->lvl_r64.clear();
    s->lvl_counts.clear();
    s->lvl_warp.clear();
    s->lvl_w64.clear();
    s->lvl_big.clear();
    for (int64_t l = 0; l < nlev; ++l) {
      int32_t cnt[7] = {0, 0, 0, 0, 0, 0, 0};
      // chain runs, warp, wide warp, CTA tasks, then dense fronts
      for (int tr : {5, 6, 0, 3, 1, 2}) {
        for (int64_t q : bylev[l]) {
          if (ttier[q] != tr) continue;
          for (int32_t f : tasks[q]) s->task_fronts.push_back(f);
          s->task_ptr.push_back((int32_t)s->task_fronts.size());
          cnt[tr]++;
        }
      }
      s->lvl_ptr.push_back((int32_t)(s->task_ptr.size() - 1));
      s->lvl_r32.push_back(cnt[5]);
      s->lvl_r64.push_back(cnt[6]);
      for (int c : {cnt[5], cnt[6], cnt[0], cnt[3], cnt[2]}) s->lvl_counts.push_back(c);
      s->lvl_warp.push_back(cnt[0]);
      s->lvl_w64.push_back(cnt[3]);
      s->lvl_big.push_back(cnt[2]);
    }
    // per-position records of the task lists
    s->tmeta.assign(s->task_fronts.size(), WMeta{});
    for (size_t t = 0; t + 1 < s->task_ptr.size(); ++t) {
      const int32_t q0 = s->task_ptr[t], q1 = s->task_ptr[t + 1];
      for (int32_t q = q0; q < q1; ++q) {
        const int64_t k = s->task_fronts[q];
        WMeta& w = s->tmeta[q];
        w.col0 = s->sn_ptr[k];
        w.base = s->colptr[w.col0];
        w.f_off = s->f_off[k];
        w.rows_off = s->rows_ptr[k];
        w.d_off = s->d_off[k];
        w.v_off = s->v_off[k];
        w.k = (int32_t)k;
        w.n = (int32_t)(s->sn_ptr[k + 1] - s->sn_ptr[k]);
        w.J = (int32_t)(s->rows_ptr[k + 1] - s->rows_ptr[k]);
        w.ch_beg = (int32_t)s->ea_ptr[k];
        w.ch_end = (int32_t)s->ea_ptr[k + 1];
        w.flags = 0;
        if (q > q0 && s->sn_par[s->task_fronts[q - 1]] == k) {
          w.flags |= WM_PREV_CHILD;
          if (w.ch_end - w.ch_beg == 1) w.flags |= WM_ONLY_CHILD_PREV;
        }
        if (q + 1 < q1 && s->sn_par[k] == s->task_fronts[q + 1]) w.flags |= WM_NEXT_PARENT;
      }
    }
  }
  factored_completion_plan(s);
  return CHD_OK;
}
