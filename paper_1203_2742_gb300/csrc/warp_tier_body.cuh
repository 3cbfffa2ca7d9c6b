// Warp tier body, compiled twice by warp_tier.cu: WT_J is the largest |J|
// of the tier (32 or 64), WT_TPF the threads that work on one front (a warp,
// or a whole CTA), WT_WPB the fronts per CTA, WT_NS the namespace.
// See warp_tier.cu for the description.

namespace chd {
namespace WT_NS {

constexpr int WJ = WT_J;             // largest |J|
constexpr int WN = 8;                // largest |N|
constexpr int WPB = WT_WPB;           // fronts (task walkers) per CTA
constexpr int TPF = WT_TPF;           // threads per front: one warp, or a CTA
constexpr int PK = WJ * (WJ + 1) / 2;  // packed lower front
constexpr int BLK = WJ * WN;         // J x n block (column-major, ld WJ)
constexpr int NN = WN * WN;          // n x n block (column-major, ld WN)
constexpr int NS = (WJ * WN + TPF - 1) / TPF;  // staged values per thread
constexpr int NR = (WJ + TPF - 1) / TPF;       // staged relative indices per thread
// two packed fronts (the current one and the previous front of the task),
// three J x n blocks, two n x n blocks, WJ reciprocal pivots, WJ relative
// indices
constexpr int PER_WARP = 2 * PK + 3 * BLK + 2 * NN + WJ + WJ / 2;

__device__ __forceinline__ int pk(int J, int r, int c) { return c * J - c * (c - 1) / 2 + (r - c); }

// barrier of the threads working on one front
__device__ __forceinline__ void fsync() {
  if (TPF == 32) __syncwarp();
  else __syncthreads();
}

// e = q*d + r (0 <= r < d) without the integer-division sequence: an FP32
// quotient estimate, off by at most one for the small e here, then fixed.
__device__ __forceinline__ void divmod(int e, int d, int& r, int& q) {
  int qq = __float2int_rz(__fdividef((float)e, (float)d));
  int rr = e - qq * d;
  if (rr < 0) {
    --qq;
    rr += d;
  } else if (rr >= d) {
    ++qq;
    rr -= d;
  }
  r = rr;
  q = qq;
}

struct Smem {
  double* F;   // packed front
  double* P;   // packed front of the previous front of the task
  double* A1;  // J x n blocks, element (r, c) at r + c*WJ
  double* A2;
  double* A3;
  double* D1;  // n x n blocks, element (r, c) at r + c*WN
  double* D2;
  double* rv;  // reciprocal pivots of the last Cholesky factorisation
  int* rel;    // relative indices of a child (bottom-up) or of this front (top-down)
};

struct Fr {
  int k, n, a, J, flags;
  int64_t col0, base, rows_off, d_off, v_off;
  int ch_beg, ch_end;
  double* G;  // dense workspace front (ld J)
};

__device__ __forceinline__ Fr fr_meta(const WMeta& w, double* ws) {
  Fr f;
  f.k = w.k;
  f.n = w.n;
  f.J = w.J;
  f.a = w.J - w.n;
  f.flags = w.flags;
  f.col0 = w.col0;
  f.base = w.base;
  f.rows_off = w.rows_off;
  f.d_off = w.d_off;
  f.v_off = w.v_off;
  f.ch_beg = w.ch_beg;
  f.ch_end = w.ch_end;
  f.G = ws ? ws + w.f_off : nullptr;
  return f;
}

// Loads of a front's inputs, all issued before the first store so that they
// take one memory round trip: up to 32*NS consecutive values from each of two
// sources (a front's N-part has at most WJ*8 - 28 values) and up to WJ
// relative indices.
struct Stage {
  double v[NS], w[NS];
  int r[NR];
};
__device__ __forceinline__ void stage_issue(Stage& g, const double* s1, int c1, const double* s2, int c2,
                                            const int32_t* rel, int nrel, int lane) {
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int e = lane + TPF * i;
    g.v[i] = (s1 && e < c1) ? s1[e] : 0.0;
    g.w[i] = (s2 && e < c2) ? s2[e] : 0.0;
  }
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int e = lane + TPF * i;
    g.r[i] = (rel && e < nrel) ? __ldg(rel + e) : 0;
  }
}
__device__ __forceinline__ void stage_commit(const Stage& g, double* d1, int c1, double* d2, int c2, int* rdst,
                                             int nrel, int lane) {
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int e = lane + TPF * i;
    if (d1 && e < c1) d1[e] = g.v[i];
    if (d2 && e < c2) d2[e] = g.w[i];
  }
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int e = lane + TPF * i;
    if (rdst && e < nrel) rdst[e] = g.r[i];
  }
}

// record of front k read from the symbolic arrays (fronts outside a task walk)
// Asynchronous 8-byte copies global -> shared (all in flight at once; wait
// with cp_async_wait_all before reading the destination).
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// lower triangle of the m x m column-major block M (ld m) into dst, packed
// (entry (r, c), r >= c, at pk(m, r, c)); asynchronous
__device__ __forceinline__ void stage_lower_async(double* dst, const double* M, int m, int lane) {
  for (int c = 0; c < m; ++c)
    for (int r = c + lane; r < m; r += TPF) cp_async8(dst + (c * m - c * (c - 1) / 2 + (r - c)), M + r + (int64_t)c * m);
}

// record of front k read from the symbolic arrays (fronts outside a task walk)
__device__ __forceinline__ Fr fr(const SymDev& S, int k, double* ws) {
  Fr f{};
  f.k = k;
  f.col0 = S.sn_ptr[k];
  f.n = (int)(S.sn_ptr[k + 1] - f.col0);
  f.J = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  f.a = f.J - f.n;
  f.base = S.colptr[f.col0];
  f.G = ws ? ws + S.f_off[k] : nullptr;
  return f;
}
__device__ __forceinline__ int nnz_front(const Fr& f) { return f.n * f.J - f.n * (f.n - 1) / 2; }

__device__ void store_front(const Fr& f, const Smem& m, double* dst, double scale, int lane) {
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += TPF) dst[f.base + e] = scale * m.F[e];
}
// extend-add of the children's update blocks (children in a fixed order).
// A child that is the previous front of the task (flag WM_PREV_CHILD) is read
// from its packed front in m.P, with its relative indices already in m.rel;
// the others from their workspace fronts.
__device__ void extend_add(const SymDev& S, const Fr& f, const Fr& prev, const Smem& m, const double* ws,
                           int lane, const uint8_t* act = nullptr) {
  const bool chain = f.flags & WM_PREV_CHILD;
  if (chain && (f.flags & WM_ONLY_CHILD_PREV)) {
    if (act && !act[prev.k]) return;  // pruned child (§5.5): its update block is zero
    const int ac = prev.a, nc = prev.n, Jc = prev.J;
    for (int e = lane; e < ac * ac; e += TPF) {
      int r, s;
    divmod(e, ac, r, s);
      if (r >= s) m.F[pk(f.J, m.rel[r], m.rel[s])] += m.P[pk(Jc, nc + r, nc + s)];
    }
    fsync();
    return;
  }
  for (int q = f.ch_beg; q < f.ch_end; ++q) {
    const int c = S.ea[q];
    if (act && !act[c]) continue;
    if (chain && c == prev.k) {
      const int ac = prev.a, nc = prev.n, Jc = prev.J;
      for (int e = lane; e < ac * ac; e += TPF) {
        int r, s;
    divmod(e, ac, r, s);
        if (r >= s) m.F[pk(f.J, m.rel[r], m.rel[s])] += m.P[pk(Jc, nc + r, nc + s)];
      }
      fsync();
      continue;
    }
    const int nc = (int)(S.sn_ptr[c + 1] - S.sn_ptr[c]);
    const int Jc = (int)(S.rows_ptr[c + 1] - S.rows_ptr[c]);
    const int ac = Jc - nc;
    const int32_t* rel = S.rel + S.rows_ptr[c] + nc;
    const double* U = ws + S.f_off[c] + nc + (int64_t)nc * Jc;
    for (int e = lane; e < ac * ac; e += TPF) {
      int r, s;
    divmod(e, ac, r, s);
      if (r >= s) m.F[pk(f.J, __ldg(rel + r), __ldg(rel + s))] += __ldcg(U + r + (int64_t)s * Jc);
    }
    fsync();
  }
}
// V block <- parent's front at the relative positions (m.rel holds this
// front's relative indices): from m.P when the parent is the previous front
// processed (flag WM_NEXT_PARENT), else from the parent's workspace front.
__device__ void gather_parent(const SymDev& S, const Fr& f, const Fr& prev, const Smem& m, const double* ws,
                              int lane) {
  if (f.a == 0) return;
  if (f.flags & WM_NEXT_PARENT) {
    const int Jp = prev.J;
    for (int e = lane; e < f.a * f.a; e += TPF) {
      int r, s;
    divmod(e, f.a, r, s);
      if (r >= s) m.F[pk(f.J, f.n + r, f.n + s)] = m.P[pk(Jp, m.rel[r], m.rel[s])];
    }
    fsync();
    return;
  }
  const int p = (int)S.sn_par[f.k];
  if (p < 0) return;
  const int Jp = (int)(S.rows_ptr[p + 1] - S.rows_ptr[p]);
  const double* Fp = ws + S.f_off[p];
  for (int e = lane; e < f.a * f.a; e += TPF) {
    int r, s;
    divmod(e, f.a, r, s);
    if (r >= s) m.F[pk(f.J, f.n + r, f.n + s)] = __ldcg(Fp + m.rel[r] + (int64_t)m.rel[s] * Jp);
  }
  fsync();
}
// the update block for the parent, unless the parent is the next front of the
// task (it then reads this front from shared memory)
__device__ void write_update(const Fr& f, const Smem& m, int lane) {
  if (f.flags & WM_NEXT_PARENT) return;
  for (int e = lane; e < f.a * f.a; e += TPF) {
    int r, s;
    divmod(e, f.a, r, s);
    if (r >= s) f.G[(f.n + r) + (int64_t)(f.n + s) * f.J] = m.F[pk(f.J, f.n + r, f.n + s)];
  }
}
// the whole front for the children, unless the only child is the next front
// processed (it then reads this front from shared memory)
__device__ void write_full(const Fr& f, const Smem& m, int lane) {
  if (f.flags & WM_ONLY_CHILD_PREV) return;
  if (f.ch_end == f.ch_beg) return;
  for (int e = lane; e < f.J * f.J; e += TPF) {
    int r, s;
    divmod(e, f.J, r, s);
    if (r >= s) f.G[r + (int64_t)s * f.J] = m.F[pk(f.J, r, s)];
  }
}

// accessors
struct PkSym {  // symmetric, packed lower, rows/cols offset by o
  const double* F;
  int J, o;
  __device__ double operator()(int r, int c) const {
    r += o;
    c += o;
    return r >= c ? F[pk(J, r, c)] : F[pk(J, c, r)];
  }
};
struct PkRect {  // rows [ro, ..) x cols [0, n) of the packed front (below the diagonal block)
  double* F;
  int J, ro;
  __device__ double& operator()(int r, int c) const { return F[pk(J, r + ro, c)]; }
};
struct PkRectT {
  const double* F;
  int J, ro;
  __device__ double operator()(int r, int c) const { return F[pk(J, c + ro, r)]; }
};
struct Bk {  // column-major block with ld
  double* p;
  int ld;
  __device__ double& operator()(int r, int c) const { return p[r + c * ld]; }
};
struct BkT {
  const double* p;
  int ld;
  __device__ double operator()(int r, int c) const { return p[c + r * ld]; }
};
struct BkSym {  // symmetric, lower stored
  const double* p;
  int ld;
  __device__ double operator()(int r, int c) const { return r >= c ? p[r + c * ld] : p[c + r * ld]; }
};
struct GSym {  // symmetric, lower stored, global memory
  const double* p;
  int64_t ld;
  __device__ double operator()(int r, int c) const {
    return r >= c ? p[r + (int64_t)c * ld] : p[c + (int64_t)r * ld];
  }
};
struct PkBlk {  // the diagonal block starting at row/column o of the packed front (lower use)
  double* F;
  int J, o;
  __device__ double& operator()(int r, int c) const { return F[pk(J, o + r, o + c)]; }
};
struct CscOut {  // output rows [ro, ..) of the N-part in a CSC array
  double* p;
  int J, ro;
  __device__ double& operator()(int r, int c) const { return p[pk(J, r + ro, c)]; }
};

// C = beta*C + alpha*A(RxK)B(KxN), the R*N outputs dealt to the lanes
template <class FA, class FB, class FC>
__device__ void wgemm(int R, int N, int K, double alpha, FA A, FB B, double beta, FC C, bool lower, int lane) {
  const int tot = R * N;
  for (int e = lane; e < tot; e += TPF) {
    int r, c;
    divmod(e, R, r, c);
    if (lower && r < c) continue;
    // four independent partial sums: the dependent FP64 chain is a quarter as long
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = 0;
    for (; k + 3 < K; k += 4) {
      a0 = fma(A(r, k), B(k, c), a0);
      a1 = fma(A(r, k + 1), B(k + 1, c), a1);
      a2 = fma(A(r, k + 2), B(k + 2, c), a2);
      a3 = fma(A(r, k + 3), B(k + 3, c), a3);
    }
    for (; k < K; ++k) a0 = fma(A(r, k), B(k, c), a0);
    const double acc = (a0 + a1) + (a2 + a3);
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, C(r, c), v);
    C(r, c) = v;
  }
  fsync();
}

// In-place Cholesky of an m x m lower matrix given by accessor (m <= 32);
// rv[j] = 1 / L_jj.  A non-positive pivot is recorded and replaced by 1.
template <class FM>
__device__ void wpotrf(int m, FM A, double* rv, int64_t* st, int64_t code, int64_t snode, int64_t col0,
                       int lane) {
  for (int j = 0; j < m; ++j) {
    double d = A(j, j);
    if (!(d > 0.0)) {
      if (lane == 0) record_error(st, code, snode, col0 < 0 ? -1 : col0 + j);
      d = 1.0;
    }
    const double r = rsqrt(d);
    fsync();
    if (lane == 0) {
      A(j, j) = d * r;
      rv[j] = r;
    }
    for (int i = j + 1 + lane; i < m; i += TPF) A(i, j) = A(i, j) * r;
    fsync();
    const int q = m - j - 1;
    for (int e = lane; e < q * q; e += TPF) {
      int i, k;
      divmod(e, q, i, k);
      i += j + 1;
      k += j + 1;
      if (i >= k) A(i, k) = A(i, k) - A(i, j) * A(k, j);
    }
    fsync();
  }
}
// B (R x m) := B L^{-T} (fwd) or B L^{-1} (!fwd), L m x m lower (accessor),
// rv[c] = 1 / L_cc
template <class FB, class FL>
__device__ void wtrsm_r(int R, int m, FB B, FL L, const double* rv, bool fwd, int lane) {
  if (fwd) {
    for (int c = 0; c < m; ++c) {
      const double inv = rv[c];
      for (int r = lane; r < R; r += TPF) B(r, c) = B(r, c) * inv;
      fsync();
      const int q = m - c - 1;
      for (int e = lane; e < R * q; e += TPF) {
        int r, t;
        divmod(e, R, r, t);
        t += c + 1;
        B(r, t) = B(r, t) - B(r, c) * L(t, c);
      }
      fsync();
    }
  } else {
    for (int c = m - 1; c >= 0; --c) {
      const double inv = rv[c];
      for (int r = lane; r < R; r += TPF) B(r, c) = B(r, c) * inv;
      fsync();
      for (int e = lane; e < R * c; e += TPF) {
        int r, t;
    divmod(e, R, r, t);
        B(r, t) = B(r, t) - B(r, c) * L(c, t);
      }
      fsync();
    }
  }
}
// out(r, c, sum_{t < K} term(t, r, c)) for the n x n outputs (lower only if
// `lower`), one warp per output: the K terms are split over the lanes and
// summed by shuffles, so a long K costs K/32 dependent steps, not K
template <class Term, class Out>
__device__ void wreduce_nn(int n, int K, bool lower, Term term, Out out, int lane) {
  const int warp = lane >> 5, wl = lane & 31;
  for (int o = warp; o < n * n; o += TPF / 32) {
    int r, c;
    divmod(o, n, r, c);
    if (lower && r < c) continue;  // the same for the whole warp
    double acc = 0.0;
    for (int t = wl; t < K; t += 32) acc += term(t, r, c);
    for (int x = 16; x > 0; x >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, x);
    if (wl == 0) out(r, c, acc);
  }
  fsync();
}

// sum over i < n of 2 log(diag(i)) by the lanes, written by lane 0
template <class FD>
__device__ void wlogdet(int n, FD diag, double* out, int lane) {
  if (lane < 32) {  // n <= 8: the first warp holds every term
    double s = lane < n ? 2.0 * log(diag(lane)) : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *out = s;
  }
}
struct BkTW {  // transposed writable view of a column-major block
  double* p;
  int ld;
  __device__ double& operator()(int r, int c) const { return p[c + r * ld]; }
};
struct GTW {  // transposed writable view of a global column-major block
  double* p;
  int64_t ld;
  __device__ double& operator()(int r, int c) const { return p[c + (int64_t)r * ld]; }
};
struct GL {  // global column-major (lower triangular use)
  double* p;
  int64_t ld;
  __device__ double& operator()(int r, int c) const { return p[r + (int64_t)c * ld]; }
};

// L_AN (a x n) -> A1, D^{-1} (n x n, lower) -> D1 from the front's Wc values
// staged (packed, CSC order) in Wp
__device__ void scatter_w(const Fr& f, const Smem& m, const double* Wp, int lane) {
  for (int e = lane; e < f.a * f.n; e += TPF) {
    int r, c;
    divmod(e, f.a, r, c);
    m.A1[r + c * WJ] = Wp[pk(f.J, f.n + r, c)];
  }
  for (int e = lane; e < f.n * f.n; e += TPF) {
    int r, c;
    divmod(e, f.n, r, c);
    if (r >= c) m.D1[r + c * WN] = Wp[pk(f.J, r, c)];
  }
  fsync();
}
// inputs of a bottom-up front: values (N-part) into F (A x A block zeroed or
// the whole front zeroed), Wc into A3 (then A1/D1), the chain child's
// relative indices into m.rel
__device__ void load_up(const SymDev& S, const Fr& f, const Fr& prev, const Smem& m, const double* vals,
                        double* vdst, const double* Wc, bool zero_all, int lane) {
  const int nz = nnz_front(f);
  const bool chain = f.flags & WM_PREV_CHILD;
  Stage g;
  stage_issue(g, vals ? vals + f.base : nullptr, nz, Wc ? Wc + f.base : nullptr, nz,
              chain ? S.rel + prev.rows_off + prev.n : nullptr, chain ? prev.a : 0, lane);
  const int tot = f.J * (f.J + 1) / 2;
  for (int e = (zero_all ? 0 : nz) + lane; e < tot; e += TPF) m.F[e] = 0.0;
  stage_commit(g, vals ? vdst : nullptr, nz, Wc ? m.A3 : nullptr, nz, chain ? m.rel : nullptr,
               chain ? prev.a : 0, lane);
  fsync();
  if (Wc) scatter_w(f, m, m.A3, lane);
}
// inputs of a top-down front: values (N-part) into F, Wc into A3 (then
// A1/D1), this front's relative indices into m.rel
__device__ void load_down(const SymDev& S, const Fr& f, const Smem& m, const double* vals, const double* Wc,
                          int lane) {
  const int nz = nnz_front(f);
  Stage g;
  stage_issue(g, vals ? vals + f.base : nullptr, nz, Wc ? Wc + f.base : nullptr, nz, S.rel + f.rows_off + f.n,
              f.a, lane);
  stage_commit(g, vals ? m.F : nullptr, nz, Wc ? m.A3 : nullptr, nz, m.rel, f.a, lane);
  fsync();
  if (Wc) scatter_w(f, m, m.A3, lane);
}

// ---------------------------------------------------------------------------
// front procedures
// ---------------------------------------------------------------------------
__device__ void factor_front(const SymDev& S, const Fr& f, const Fr& prev, const double* X, double* Lc,
                             double* Wc, double* Dd, const double* ws, double* ldet, int64_t* st, const Smem& m,
                             int lane) {
  const int k = f.k, J = f.J, n = f.n, a = f.a;
  load_up(S, f, prev, m, X, m.F, nullptr, false, lane);
  extend_add(S, f, prev, m, ws, lane);
  if (n == 1) {
    // one column (chains of bands, leaves): D = F_11, C = sqrt(D),
    // B = F_21 / C, L_AN = F_21 / D, U = F_22 - F_21 F_21^T / D
    double d = m.F[0];
    if (!(d > 0.0)) {
      if (lane == 0) record_error(st, CHD_ERR_NOT_PD, k, f.col0);
      d = 1.0;
    }
    const double r = rsqrt(d), r2 = r * r;
    for (int e = lane; e < a * a; e += TPF) {
      int i, j;
      divmod(e, a, i, j);
      if (i >= j) m.F[pk(J, 1 + i, 1 + j)] -= m.F[1 + i] * m.F[1 + j] * r2;
    }
    double* Lo = Lc + f.base;
    double* W = Wc + f.base;
    for (int i = lane; i < a; i += TPF) {
      const double x = m.F[1 + i];
      Lo[1 + i] = x * r;
      W[1 + i] = x * r2;
    }
    if (lane == 0) {
      Lo[0] = d * r;
      W[0] = r2;
      Dd[f.d_off] = d;
      ldet[k] = log(d);
    }
    fsync();
    write_update(f, m, lane);
    fsync();
    return;
  }
  double* D = Dd + f.d_off;
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r >= c) D[r + c * n] = m.F[pk(J, r, c)];
  }
  // C = chol(F11), B = F21 C^{-T}, U = F22 - B B^T
  wpotrf(n, PkRect{m.F, J, 0}, m.rv, st, CHD_ERR_NOT_PD, k, f.col0, lane);
  wtrsm_r(a, n, PkRect{m.F, J, n}, PkRect{m.F, J, 0}, m.rv, true, lane);
  for (int e = lane; e < a * a; e += TPF) {
    int r, s;
    divmod(e, a, r, s);
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(m.F[pk(J, n + r, t)], m.F[pk(J, n + s, t)], acc);
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  fsync();
  store_front(f, m, Lc, 1.0, lane);
  wlogdet(n, [&](int i) { return m.F[pk(J, i, i)]; }, ldet + k, lane);
  // Cinv (D2) = C^{-1}; D^{-1} = Cinv^T Cinv (D1, lower); L_AN = B C^{-1} (A1)
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    m.D2[r + c * WN] = r == c ? 1.0 : 0.0;
  }
  fsync();
  wtrsm_r(n, n, BkTW{m.D2, WN}, PkRect{m.F, J, 0}, m.rv, true, lane);
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r < c) continue;
    double acc = 0.0;
    for (int t = r; t < n; ++t) acc = fma(m.D2[t + r * WN], m.D2[t + c * WN], acc);
    m.D1[r + c * WN] = acc;
  }
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    m.A1[r + c * WJ] = m.F[pk(J, n + r, c)];
  }
  fsync();
  wtrsm_r(a, n, Bk{m.A1, WJ}, PkRect{m.F, J, 0}, m.rv, false, lane);
  double* W = Wc + f.base;
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r >= c) W[pk(J, r, c)] = m.D1[r + c * WN];
  }
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    W[pk(J, n + r, c)] = m.A1[r + c * WJ];
  }
  write_update(f, m, lane);
  fsync();
}

// Algorithm 3.2 (Cholesky product) for one front: F = the children's blocks
// + G G^T with G = [C; B] (the front's N-part of Lc, staged and scattered
// into D1 = C and A1 = B); the N-part of F is X, the A x A block stays.
__device__ void product_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Lc, double* Xo,
                              const double* ws, const Smem& m, int lane) {
  const int J = f.J, n = f.n;
  load_up(S, f, prev, m, nullptr, nullptr, Lc, true, lane);
  extend_add(S, f, prev, m, ws, lane);
  // G(r, t): C(r, t) for r < n (lower), B(r - n, t) below
  auto G = [&](int r, int t) { return r < n ? (r >= t ? m.D1[r + t * WN] : 0.0) : m.A1[(r - n) + t * WJ]; };
  for (int e = lane; e < J * J; e += TPF) {
    int r, c;
    divmod(e, J, r, c);
    if (r < c) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(G(r, t), G(c, t), acc);
    m.F[pk(J, r, c)] += acc;
  }
  fsync();
  store_front(f, m, Xo, 1.0, lane);
  write_update(f, m, lane);
  fsync();
}

__device__ void gradient_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Wc, double* Sc,
                               double* g, double* Vd, const double* ws, const Smem& m, int lane) {
  const int J = f.J, n = f.n, a = f.a;
  load_down(S, f, m, nullptr, Wc, lane);
  gather_parent(S, f, prev, m, ws, lane);
  // S_AN = -V L_AN
  wgemm(a, n, a, -1.0, PkSym{m.F, J, n}, Bk{m.A1, WJ}, 0.0, PkRect{m.F, J, n}, false, lane);
  // S_NN = D^{-1} - S_AN^T L_AN
  wreduce_nn(
      n, a, true, [&](int t, int r, int c) { return m.F[pk(J, n + t, r)] * m.A1[t + c * WJ]; },
      [&](int r, int c, double acc) { m.F[pk(J, r, c)] = m.D1[r + c * WN] - acc; }, lane);
  store_front(f, m, Sc, 1.0, lane);
  if (g) store_front(f, m, g, -1.0, lane);
  double* V = Vd + f.v_off;
  for (int e = lane; e < a * a; e += TPF) {
    int r, s;
    divmod(e, a, r, s);
    if (r >= s) V[r + s * a] = m.F[pk(J, n + r, n + s)];
  }
  write_full(f, m, lane);
  fsync();
}

__device__ void hess_up_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Wc, const double* Vd,
                              const double* Y, double* T, const double* ws, const Smem& m, int lane,
                              const uint8_t* act) {
  const int J = f.J, n = f.n, a = f.a;
  load_up(S, f, prev, m, Y, m.F, Wc, false, lane);
  extend_add(S, f, prev, m, ws, lane, act);
  // V_k (lower, packed) into the previous front's buffer, free from here on
  stage_lower_async(m.P, Vd + f.v_off, a, lane);
  // A2 = K_AN = Y_AN - L Y_NN
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    double acc = m.F[pk(J, n + r, c)];
    for (int t = 0; t < n; ++t)
      acc = fma(-m.A1[r + t * WJ], t >= c ? m.F[pk(J, t, c)] : m.F[pk(J, c, t)], acc);
    m.A2[r + c * WJ] = acc;
  }
  fsync();
  // U' = Y_AA - K_AN L^T - L Y_AN^T  (lower)
  for (int e = lane; e < a * a; e += TPF) {
    int r, s;
    divmod(e, a, r, s);
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) {
      acc = fma(m.A2[r + t * WJ], m.A1[s + t * WJ], acc);
      acc = fma(m.A1[r + t * WJ], m.F[pk(J, n + s, t)], acc);
    }
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  fsync();
  // D2 = K_NN D^{-1};  M_NN = D^{-1} D2 -> T (lower)
  wgemm(n, n, n, 1.0, PkSym{m.F, J, 0}, BkSym{m.D1, WN}, 0.0, Bk{m.D2, WN}, false, lane);
  wgemm(n, n, n, 1.0, BkSym{m.D1, WN}, Bk{m.D2, WN}, 0.0, CscOut{T + f.base, J, 0}, true, lane);
  // A3 = K_AN D^{-1};  M_AN = V A3 -> T
  wgemm(a, n, n, 1.0, Bk{m.A2, WJ}, BkSym{m.D1, WN}, 0.0, Bk{m.A3, WJ}, false, lane);
  cp_async_wait_all();
  fsync();
  wgemm(a, n, a, 1.0, PkSym{m.P, a, 0}, Bk{m.A3, WJ}, 0.0, CscOut{T + f.base, J, n}, false, lane);
  write_update(f, m, lane);
  fsync();
}

__device__ void hess_down_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Wc, double* T,
                                const double* ws, const Smem& m, int lane) {
  const int J = f.J, n = f.n, a = f.a;
  load_down(S, f, m, T, Wc, lane);
  gather_parent(S, f, prev, m, ws, lane);
  // A2 = V' L
  wgemm(a, n, a, 1.0, PkSym{m.F, J, n}, Bk{m.A1, WJ}, 0.0, Bk{m.A2, WJ}, false, lane);
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    m.F[pk(J, n + r, c)] -= 0.5 * m.A2[r + c * WJ];
  }
  fsync();
  // T_NN = M_NN - (Q^T L + L^T Q)
  wreduce_nn(
      n, a, true,
      [&](int t, int r, int c) {
        return fma(m.F[pk(J, n + t, r)], m.A1[t + c * WJ], m.A1[t + r * WJ] * m.F[pk(J, n + t, c)]);
      },
      [&](int r, int c, double acc) { m.F[pk(J, r, c)] -= acc; }, lane);
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    m.F[pk(J, n + r, c)] -= 0.5 * m.A2[r + c * WJ];
  }
  fsync();
  store_front(f, m, T, 1.0, lane);
  write_full(f, m, lane);
  fsync();
}

__device__ void ihess_down_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Wc,
                                 const double* Dd, const double* Rd, const double* Tin, double* Y,
                                 const double* ws, const Smem& m, int lane) {
  const int J = f.J, n = f.n, a = f.a;
  load_down(S, f, m, Tin, Wc, lane);
  gather_parent(S, f, prev, m, ws, lane);
  // V_k^{-1} and D_NN (lower, packed) into the previous front's buffer
  // (a(a+1)/2 + n(n+1)/2 <= PK since a + n <= WJ)
  double* Rp = m.P;
  double* Dp = m.P + a * (a + 1) / 2;
  stage_lower_async(Rp, Rd + f.v_off, a, lane);
  stage_lower_async(Dp, Dd + f.d_off, n, lane);
  // A2 = M_AN = T_AN + V' L  (four partial sums per output)
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    const PkSym Vp{m.F, J, n};
    double a0 = m.F[pk(J, n + r, c)], a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int t = 0;
    for (; t + 3 < a; t += 4) {
      a0 = fma(Vp(r, t), m.A1[t + c * WJ], a0);
      a1 = fma(Vp(r, t + 1), m.A1[t + 1 + c * WJ], a1);
      a2 = fma(Vp(r, t + 2), m.A1[t + 2 + c * WJ], a2);
      a3 = fma(Vp(r, t + 3), m.A1[t + 3 + c * WJ], a3);
    }
    for (; t < a; ++t) a0 = fma(Vp(r, t), m.A1[t + c * WJ], a0);
    m.A2[r + c * WJ] = (a0 + a1) + (a2 + a3);
  }
  fsync();
  // D2 = M_NN = T_NN + T_AN^T L + L^T M_AN  (full)
  wreduce_nn(
      n, a, false,
      [&](int t, int r, int c) {
        return fma(m.F[pk(J, n + t, r)], m.A1[t + c * WJ], m.A1[t + r * WJ] * m.A2[t + c * WJ]);
      },
      [&](int r, int c, double acc) { m.D2[r + c * WN] = acc + (r >= c ? m.F[pk(J, r, c)] : m.F[pk(J, c, r)]); },
      lane);
  cp_async_wait_all();
  fsync();
  const PkSym D{Dp, n, 0};
  // D1 = M_NN D ;  K_NN = D D1 -> Y (lower)
  wgemm(n, n, n, 1.0, Bk{m.D2, WN}, D, 0.0, Bk{m.D1, WN}, false, lane);
  wgemm(n, n, n, 1.0, D, Bk{m.D1, WN}, 0.0, CscOut{Y + f.base, J, 0}, true, lane);
  if (a > 0) {
    // A3 = M_AN D ; K_AN = V^{-1} A3 -> Y  (V^{-1} cached per factor)
    wgemm(a, n, n, 1.0, Bk{m.A2, WJ}, D, 0.0, Bk{m.A3, WJ}, false, lane);
    wgemm(a, n, a, 1.0, PkSym{Rp, a, 0}, Bk{m.A3, WJ}, 0.0, CscOut{Y + f.base, J, n}, false, lane);
  }
  write_full(f, m, lane);
  fsync();
}

__device__ void ihess_up_front(const SymDev& S, const Fr& f, const Fr& prev, const double* Wc, double* Y,
                               const double* ws, const Smem& m, int lane) {
  const int J = f.J, n = f.n, a = f.a;
  // K (this front's N-part of the output, written by the top-down pass) is
  // staged packed in A2
  load_up(S, f, prev, m, Y, m.A2, Wc, true, lane);
  extend_add(S, f, prev, m, ws, lane);
  const double* Kc = m.A2;
  // A3 = P = K_AN + 1/2 L K_NN
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(m.A1[r + t * WJ], t >= c ? Kc[pk(J, t, c)] : Kc[pk(J, c, t)], acc);
    m.A3[r + c * WJ] = Kc[pk(J, n + r, c)] + 0.5 * acc;
  }
  fsync();
  // U' = Z_AA - (P L^T + L P^T)
  for (int e = lane; e < a * a; e += TPF) {
    int r, s;
    divmod(e, a, r, s);
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) {
      acc = fma(m.A3[r + t * WJ], m.A1[s + t * WJ], acc);
      acc = fma(m.A1[r + t * WJ], m.A3[s + t * WJ], acc);
    }
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  fsync();
  double* Yo = Y + f.base;
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    const int o = pk(J, n + r, c);
    Yo[o] = 2.0 * m.A3[r + c * WJ] - Kc[o] - m.F[o];
  }
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r < c) continue;
    const int o = pk(J, r, c);
    Yo[o] = Kc[o] - m.F[o];
  }
  write_update(f, m, lane);
  fsync();
}

// S-front of the completion: S_NN and S_AN from the input's columns N_k,
// V_k = S_{A_k A_k} from its later columns (a submatrix of S, Algorithm 7.3),
// so the front depends on no other front.  With Gq (factored update
// matrices, Algorithm 4.3) the factor G = P R_k P of V_k = R_k R_k^T comes
// from Gq and the solves run on S_AN and L_AN with reversed rows.
__device__ void complete_front(const SymDev& S, int k, const double* Sin, double* Lc, double* Wc, double* Dd,
                               double* Vd, double* Rd, const double* Gq, double* ldet, int64_t* st, const Smem& m,
                               int lane) {
  Fr f = fr(S, k, nullptr);
  const int J = f.J, n = f.n, a = f.a;
  const int32_t* A = S.rows + S.rows_ptr[k] + n;
  for (int e = lane; e < a * a; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    if (r >= c) m.F[pk(J, n + r, n + c)] = Sin[csc_find(S, __ldg(A + r), __ldg(A + c))];
  }
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += TPF) m.F[e] = Sin[f.base + e];
  fsync();
  double* V = Vd + S.v_off[k];
  double* R = Rd + S.v_off[k];
  for (int e = lane; e < a * a; e += TPF) {
    int r, s;
    divmod(e, a, r, s);
    if (r >= s) V[r + s * a] = m.F[pk(J, n + r, n + s)];
  }
  fsync();
  PkBlk Rv{m.F, J, n};
  if (Gq) {
    const double* G = Gq + S.v_off[k];
    for (int e = lane; e < a * a; e += TPF) {
      int r, s;
      divmod(e, a, r, s);
      if (r >= s) m.F[pk(J, n + r, n + s)] = G[r + s * a];
    }
    for (int r = lane; r < a; r += TPF) m.rv[r] = 1.0 / G[r + r * a];
  } else {
    if (a > 0) wpotrf(a, Rv, m.rv, st, CHD_ERR_NOT_COMPLETABLE, k, -1, lane);
    for (int e = lane; e < a * a; e += TPF) {
      int r, s;
      divmod(e, a, r, s);
      if (r >= s) R[r + s * a] = m.F[pk(J, n + r, n + s)];
    }
  }
  // A1 = Z = R^{-1} S_AN (rows reversed with Gq)
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    m.A1[r + c * WJ] = m.F[pk(J, n + (Gq ? a - 1 - r : r), c)];
  }
  fsync();
  if (a > 0) wtrsm_r(n, a, BkTW{m.A1, WJ}, Rv, m.rv, true, lane);
  // D1 = P = S_NN - Z^T Z (lower);  A2 = L_AN = -R^{-T} Z
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r < c) continue;
    double acc = 0.0;
    for (int t = 0; t < a; ++t) acc = fma(m.A1[t + r * WJ], m.A1[t + c * WJ], acc);
    m.D1[r + c * WN] = m.F[pk(J, r, c)] - acc;
  }
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    m.A2[r + c * WJ] = -m.A1[r + c * WJ];
  }
  fsync();
  if (a > 0) wtrsm_r(n, a, BkTW{m.A2, WJ}, Rv, m.rv, false, lane);
  if (Gq) {  // L_AN back to the order of A_k
    const int h = a / 2;
    for (int e = lane; e < h * n; e += TPF) {
      int r, c;
      divmod(e, h, r, c);
      const double t = m.A2[r + c * WJ];
      m.A2[r + c * WJ] = m.A2[(a - 1 - r) + c * WJ];
      m.A2[(a - 1 - r) + c * WJ] = t;
    }
    fsync();
  }
  double* W = Wc + f.base;
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r >= c) W[pk(J, r, c)] = m.D1[r + c * WN];
  }
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    W[pk(J, n + r, c)] = m.A2[r + c * WJ];
  }
  // D2 = Q = chol(P); D1 = Q^{-1} ... D = Q^{-T} Q^{-1}
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    m.D2[r + c * WN] = r >= c ? m.D1[r + c * WN] : 0.0;
  }
  fsync();
  wpotrf(n, Bk{m.D2, WN}, m.rv, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0, lane);
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    m.D1[r + c * WN] = r == c ? 1.0 : 0.0;
  }
  fsync();
  wtrsm_r(n, n, BkTW{m.D1, WN}, Bk{m.D2, WN}, m.rv, true, lane);  // D1 = Q^{-1} (lower)
  double* Dk = Dd + S.d_off[k];
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r < c) continue;
    double acc = 0.0;
    for (int t = r; t < n; ++t) acc = fma(m.D1[t + r * WN], m.D1[t + c * WN], acc);
    m.D2[r + c * WN] = acc;  // D (lower)
    Dk[r + c * n] = acc;
  }
  fsync();
  wpotrf(n, Bk{m.D2, WN}, m.rv, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0, lane);  // C
  double* Lo = Lc + f.base;
  for (int e = lane; e < n * n; e += TPF) {
    int r, c;
    divmod(e, n, r, c);
    if (r >= c) Lo[pk(J, r, c)] = m.D2[r + c * WN];
  }
  for (int e = lane; e < a * n; e += TPF) {
    int r, c;
    divmod(e, a, r, c);
    double acc = 0.0;
    for (int t = c; t < n; ++t) acc = fma(m.A2[r + t * WJ], m.D2[t + c * WN], acc);
    Lo[pk(J, n + r, c)] = acc;
  }
  wlogdet(n, [&](int i) { return m.D2[i + i * WN]; }, ldet + k, lane);
  fsync();
}

// ---------------------------------------------------------------------------
// kernels: warp w of block b takes task task0 + b*WPB + w; blockIdx.y = RHS.
// A warp walks its task's fronts with the record of the next front already
// loaded, alternating two packed-front buffers so that the previous front
// stays in shared memory for the chain child (bottom-up) or the chain parent
// (top-down).
// ---------------------------------------------------------------------------
__shared__ double wsm[WPB * PER_WARP];

__device__ __forceinline__ Smem smem_for_warp(int w, int parity) {
  Smem m;
  double* b = wsm + w * PER_WARP;
  m.F = b + parity * PK;
  m.P = b + (1 - parity) * PK;
  m.A1 = b + 2 * PK;
  m.A2 = m.A1 + BLK;
  m.A3 = m.A2 + BLK;
  m.D1 = m.A3 + BLK;
  m.D2 = m.D1 + NN;
  m.rv = m.D2 + NN;
  m.rel = reinterpret_cast<int*>(m.rv + WJ);
  return m;
}

// bottom-up walk of task t (fronts in order), body(f, prev, m)
template <class Body>
__device__ __forceinline__ void walk_up(const SymDev& S, int t, double* ws, int w, Body&& body) {
  const int q0 = S.task_ptr[t], q1 = S.task_ptr[t + 1];
  WMeta nxt = S.tmeta[q0];
  Fr prev{};
  prev.k = -1;
  for (int q = q0; q < q1; ++q) {
    const WMeta cur = nxt;
    if (q + 1 < q1) nxt = S.tmeta[q + 1];
    const Fr f = fr_meta(cur, ws);
    body(f, prev, smem_for_warp(w, (q - q0) & 1));
    prev = f;
  }
}
// top-down walk of task t (fronts in reverse order)
template <class Body>
__device__ __forceinline__ void walk_down(const SymDev& S, int t, double* ws, int w, Body&& body) {
  const int q0 = S.task_ptr[t], q1 = S.task_ptr[t + 1];
  WMeta nxt = S.tmeta[q1 - 1];
  Fr prev{};
  prev.k = -1;
  for (int q = q1 - 1; q >= q0; --q) {
    const WMeta cur = nxt;
    if (q > q0) nxt = S.tmeta[q - 1];
    const Fr f = fr_meta(cur, ws);
    body(f, prev, smem_for_warp(w, (q - q0) & 1));
    prev = f;
  }
}

#define WARP_TASK_PROLOGUE                                     \
  const int w = threadIdx.x / TPF, lane = threadIdx.x % TPF;   \
  const int t = task0 + blockIdx.x * WPB + w;                  \
  if (t >= task_end) return;

__global__ void __launch_bounds__(WPB * TPF) kw_factor(SymDev S, int task0, int task_end, const double* X,
                                                      double* Lc, double* Wc, double* Dd, double* ws,
                                                      double* ldet, int64_t* st) {
  WARP_TASK_PROLOGUE
  walk_up(S, t, ws, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    factor_front(S, f, prev, X, Lc, Wc, Dd, ws, ldet, st, m, lane);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_product(SymDev S, int task0, int task_end, const double* Lc,
                                                         double* X, double* ws) {
  WARP_TASK_PROLOGUE
  walk_up(S, t, ws, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    product_front(S, f, prev, Lc, X, ws, m, lane);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_gradient(SymDev S, int task0, int task_end, const double* Wc,
                                                        double* Sc, double* g, double* Vd, double* ws) {
  WARP_TASK_PROLOGUE
  walk_down(S, t, ws, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    gradient_front(S, f, prev, Wc, Sc, g, Vd, ws, m, lane);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_hess_up(SymDev S, int task0, int task_end, const double* Wc,
                                                       const double* Vd, const double* Y, int64_t ldy, double* T,
                                                       int64_t ldt, double* ws, const uint8_t* act) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  double* wsy = ws + y * S.f_total;
  const uint8_t* ay = act ? act + y * S.nsn : nullptr;
  walk_up(S, t, wsy, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    if (ay && !ay[f.k]) return;  // pruned (§5.5): K, U' and M are zero here
    hess_up_front(S, f, prev, Wc, Vd, Y + y * ldy, T + y * ldt, wsy, m, lane, ay);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_hess_down(SymDev S, int task0, int task_end, const double* Wc,
                                                         double* T, int64_t ldt, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  double* wsy = ws + y * S.f_total;
  walk_down(S, t, wsy, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    hess_down_front(S, f, prev, Wc, T + y * ldt, wsy, m, lane);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_ihess_down(SymDev S, int task0, int task_end, const double* Wc,
                                                          const double* Dd, const double* Rd, const double* Tin,
                                                          int64_t ldt, double* Y, int64_t ldy, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  double* wsy = ws + y * S.f_total;
  walk_down(S, t, wsy, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    ihess_down_front(S, f, prev, Wc, Dd, Rd, Tin + y * ldt, Y + y * ldy, wsy, m, lane);
  });
}
__global__ void __launch_bounds__(WPB * TPF) kw_ihess_up(SymDev S, int task0, int task_end, const double* Wc,
                                                        double* Y, int64_t ldy, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  double* wsy = ws + y * S.f_total;
  walk_up(S, t, wsy, w, [&](const Fr& f, const Fr& prev, const Smem& m) {
    ihess_up_front(S, f, prev, Wc, Y + y * ldy, wsy, m, lane);
  });
}
#if WT_J == 32
// all warp-tier fronts at once, one warp each (the completion has no
// dependencies between fronts)
__global__ void __launch_bounds__(WPB * TPF) kw_complete(SymDev S, const double* Sin, double* Lc, double* Wc,
                                                        double* Dd, double* Vd, double* Rd, const double* Gq,
                                                        double* ldet, int64_t* st) {
  const int w = threadIdx.x / TPF, lane = threadIdx.x % TPF;
  const int64_t i = (int64_t)blockIdx.x * WPB + w;
  if (i >= S.warp_count) return;
  const Smem m = smem_for_warp(w, 0);
  complete_front(S, S.warp_fronts[i], Sin, Lc, Wc, Dd, Vd, Rd, Gq, ldet, st, m, lane);
}
#endif

}  // namespace WT_NS
}  // namespace chd

namespace chd_launch {
namespace WT_NS {
using namespace chd::WT_NS;
static inline dim3 wgrid(int nt, int m) { return dim3((nt + WPB - 1) / WPB, m); }

void warp_product(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Lc, double* X, double* ws) {
  kw_product<<<wgrid(nt, 1), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Lc, X, ws);
  chd_launch::count_launch();
}
void warp_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                 double* Dd, double* ws, double* ldet, int64_t* status) {
  kw_factor<<<wgrid(nt, 1), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, X, Lc, Wc, Dd, ws, ldet, status);
  chd_launch::count_launch();
}
void warp_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc,
                   double* g, double* Vd, double* ws) {
  kw_gradient<<<wgrid(nt, 1), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Wc, Sc, g, Vd, ws);
  chd_launch::count_launch();
}
void warp_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                  const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                  const uint8_t* act) {
  kw_hess_up<<<wgrid(nt, m), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Wc, Vd, Y, ldy, T, ldt, ws, act);
  chd_launch::count_launch();
}
void warp_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws) {
  kw_hess_down<<<wgrid(nt, m), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Wc, T, ldt, ws);
  chd_launch::count_launch();
}
void warp_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                     const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                     double* ws) {
  kw_ihess_down<<<wgrid(nt, m), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
  chd_launch::count_launch();
}
void warp_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                   int64_t ldy, double* ws) {
  kw_ihess_up<<<wgrid(nt, m), WPB * TPF, 0, st>>>(s->dev, t0, t0 + nt, Wc, Y, ldy, ws);
  chd_launch::count_launch();
}
#if WT_J == 32
void warp_complete_all(const chd_symbolic* s, cudaStream_t st, const double* Sin, double* Lc, double* Wc,
                       double* Dd, double* Vd, double* Rd, const double* Gq, double* ldet, int64_t* status) {
  kw_complete<<<wgrid((int)s->dev.warp_count, 1), WPB * TPF, 0, st>>>(s->dev, Sin, Lc, Wc, Dd, Vd, Rd, Gq, ldet,
                                                                      status);
  chd_launch::count_launch();
}
#endif
}  // namespace WT_NS
}  // namespace chd_launch
