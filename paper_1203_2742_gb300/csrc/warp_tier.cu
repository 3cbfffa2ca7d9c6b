// Warp tier: small fronts (|J| <= 32, |N| <= 8), one warp per task and
// right-hand side, the front staged in the warp's shared memory.
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
// cones": the per-front formulas are those of the supernodal Algorithms
// 7.1-7.3 and of the block forms of Algorithms 5.1 and 5.2 (the same as the
// per-task and dense tiers); here every dense product is a warp-wide loop in
// which the 32 lanes take the output entries in turn.
//
// The front is held packed: entry (r, c), r >= c, of the lower triangle of
// the J x J front at  c*J - c*(c-1)/2 + (r - c).  The first n columns of this
// layout coincide with the front's N-part in the CSC value arrays, so loads
// and stores of values are contiguous copies.  Results other tiers read go
// to the front's workspace region in its dense layout (column-major, ld J):
// the update block (bottom-up passes) or the whole lower front (top-down).
#include <cuda_runtime.h>

#include <cstdint>

#include "chd_internal.h"
#include "front_views.cuh"

namespace chd_launch {
void count_launch();
}

namespace chd {
namespace warp {

constexpr int WJ = 32;               // largest |J|
constexpr int WN = 8;                // largest |N|
constexpr int WPB = 4;               // warps per CTA
constexpr int PK = WJ * (WJ + 1) / 2;  // packed lower front
constexpr int BLK = WJ * WN;         // J x n block (column-major, ld WJ)
constexpr int NN = WN * WN;          // n x n block (column-major, ld WN)
constexpr int PER_WARP = PK + 3 * BLK + 2 * NN;

__device__ __forceinline__ int pk(int J, int r, int c) { return c * J - c * (c - 1) / 2 + (r - c); }

struct Smem {
  double* F;   // packed front
  double* A1;  // J x n blocks, element (r, c) at r + c*WJ
  double* A2;
  double* A3;
  double* D1;  // n x n blocks, element (r, c) at r + c*WN
  double* D2;
};

struct Fr {
  int k, n, a, J;
  int64_t col0, base;
  double* G;  // dense workspace front (ld J)
};

__device__ __forceinline__ Fr fr(const SymDev& S, int k, double* ws) {
  Fr f;
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

// F (packed) <- CSC N-part of `src`, A x A block <- 0
__device__ void load_front(const Fr& f, const Smem& m, const double* src, int lane) {
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += 32) m.F[e] = src[f.base + e];
  const int tot = f.J * (f.J + 1) / 2;
  for (int e = nz + lane; e < tot; e += 32) m.F[e] = 0.0;
}
__device__ void store_front(const Fr& f, const Smem& m, double* dst, double scale, int lane) {
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += 32) dst[f.base + e] = scale * m.F[e];
}
// extend-add of the children's update blocks (children in a fixed order)
__device__ void extend_add(const SymDev& S, const Fr& f, const Smem& m, const double* ws, int lane) {
  for (int64_t q = S.ch_ptr[f.k]; q < S.ch_ptr[f.k + 1]; ++q) {
    const int c = S.ch[q];
    const int nc = (int)(S.sn_ptr[c + 1] - S.sn_ptr[c]);
    const int Jc = (int)(S.rows_ptr[c + 1] - S.rows_ptr[c]);
    const int ac = Jc - nc;
    const int32_t* rel = S.rel + S.rows_ptr[c] + nc;
    const double* U = ws + S.f_off[c] + nc + (int64_t)nc * Jc;
    for (int e = lane; e < ac * ac; e += 32) {
      const int r = e % ac, s = e / ac;
      if (r >= s) m.F[pk(f.J, __ldg(rel + r), __ldg(rel + s))] += __ldcg(U + r + (int64_t)s * Jc);
    }
    __syncwarp();
  }
}
// V block <- parent's dense front at the relative positions
__device__ void gather_parent(const SymDev& S, const Fr& f, const Smem& m, const double* ws, int lane) {
  const int p = (int)S.sn_par[f.k];
  if (p < 0 || f.a == 0) return;
  const int Jp = (int)(S.rows_ptr[p + 1] - S.rows_ptr[p]);
  const double* Fp = ws + S.f_off[p];
  const int32_t* rel = S.rel + S.rows_ptr[f.k] + f.n;
  for (int e = lane; e < f.a * f.a; e += 32) {
    const int r = e % f.a, s = e / f.a;
    if (r >= s) m.F[pk(f.J, f.n + r, f.n + s)] = __ldcg(Fp + __ldg(rel + r) + (int64_t)__ldg(rel + s) * Jp);
  }
  __syncwarp();
}
__device__ void write_update(const Fr& f, const Smem& m, int lane) {
  for (int e = lane; e < f.a * f.a; e += 32) {
    const int r = e % f.a, s = e / f.a;
    if (r >= s) f.G[(f.n + r) + (int64_t)(f.n + s) * f.J] = m.F[pk(f.J, f.n + r, f.n + s)];
  }
}
__device__ void write_full(const Fr& f, const Smem& m, int lane) {
  for (int e = lane; e < f.J * f.J; e += 32) {
    const int r = e % f.J, s = e / f.J;
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
  for (int e = lane; e < tot; e += 32) {
    const int r = e % R, c = e / R;
    if (lower && r < c) continue;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc = fma(A(r, k), B(k, c), acc);
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, C(r, c), v);
    C(r, c) = v;
  }
  __syncwarp();
}

// In-place Cholesky of an m x m lower matrix given by accessor (m <= 32);
// a non-positive pivot is recorded and replaced by 1.
template <class FM>
__device__ void wpotrf(int m, FM A, int64_t* st, int64_t code, int64_t snode, int64_t col0, int lane) {
  for (int j = 0; j < m; ++j) {
    double d = A(j, j);
    if (!(d > 0.0)) {
      if (lane == 0) record_error(st, code, snode, col0 < 0 ? -1 : col0 + j);
      d = 1.0;
    }
    const double piv = sqrt(d);
    __syncwarp();
    if (lane == 0) A(j, j) = piv;
    for (int i = j + 1 + lane; i < m; i += 32) A(i, j) = A(i, j) / piv;
    __syncwarp();
    const int q = m - j - 1;
    for (int e = lane; e < q * q; e += 32) {
      const int i = j + 1 + e % q, k = j + 1 + e / q;
      if (i >= k) A(i, k) = A(i, k) - A(i, j) * A(k, j);
    }
    __syncwarp();
  }
}
// B (R x m) := B L^{-T} (fwd) or B L^{-1} (!fwd), L m x m lower (accessor)
template <class FB, class FL>
__device__ void wtrsm_r(int R, int m, FB B, FL L, bool fwd, int lane) {
  if (fwd) {
    for (int c = 0; c < m; ++c) {
      const double inv = 1.0 / L(c, c);
      for (int r = lane; r < R; r += 32) B(r, c) = B(r, c) * inv;
      __syncwarp();
      const int q = m - c - 1;
      for (int e = lane; e < R * q; e += 32) {
        const int r = e % R, t = c + 1 + e / R;
        B(r, t) = B(r, t) - B(r, c) * L(t, c);
      }
      __syncwarp();
    }
  } else {
    for (int c = m - 1; c >= 0; --c) {
      const double inv = 1.0 / L(c, c);
      for (int r = lane; r < R; r += 32) B(r, c) = B(r, c) * inv;
      __syncwarp();
      for (int e = lane; e < R * c; e += 32) {
        const int r = e % R, t = e / R;
        B(r, t) = B(r, t) - B(r, c) * L(c, t);
      }
      __syncwarp();
    }
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

// L_AN (a x n) -> A1, D^{-1} (n x n, lower) -> D1 from the Wc CSC block
__device__ void load_w(const Fr& f, const Smem& m, const double* Wc, int lane) {
  const double* W = Wc + f.base;
  for (int e = lane; e < f.a * f.n; e += 32) {
    const int r = e % f.a, c = e / f.a;
    m.A1[r + c * WJ] = W[pk(f.J, f.n + r, c)];
  }
  for (int e = lane; e < f.n * f.n; e += 32) {
    const int r = e % f.n, c = e / f.n;
    if (r >= c) m.D1[r + c * WN] = W[pk(f.J, r, c)];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// front procedures
// ---------------------------------------------------------------------------
__device__ void factor_front(const SymDev& S, int k, const double* X, double* Lc, double* Wc, double* Dd,
                             double* ws, double* ldet, int64_t* st, const Smem& m, int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  load_front(f, m, X, lane);
  __syncwarp();
  extend_add(S, f, m, ws, lane);
  double* D = Dd + S.d_off[k];
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r >= c) D[r + c * n] = m.F[pk(J, r, c)];
  }
  // C = chol(F11), B = F21 C^{-T}, U = F22 - B B^T
  wpotrf(n, PkRect{m.F, J, 0}, st, CHD_ERR_NOT_PD, k, f.col0, lane);
  wtrsm_r(a, n, PkRect{m.F, J, n}, PkRect{m.F, J, 0}, true, lane);
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(m.F[pk(J, n + r, t)], m.F[pk(J, n + s, t)], acc);
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  __syncwarp();
  store_front(f, m, Lc, 1.0, lane);
  if (lane == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += 2.0 * log(m.F[pk(J, i, i)]);
    ldet[k] = s;
  }
  // Cinv (D2) = C^{-1}; D^{-1} = Cinv^T Cinv (D1, lower); L_AN = B C^{-1} (A1)
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    m.D2[r + c * WN] = r == c ? 1.0 : 0.0;
  }
  __syncwarp();
  wtrsm_r(n, n, BkTW{m.D2, WN}, PkRect{m.F, J, 0}, true, lane);
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    double acc = 0.0;
    for (int t = r; t < n; ++t) acc = fma(m.D2[t + r * WN], m.D2[t + c * WN], acc);
    m.D1[r + c * WN] = acc;
  }
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    m.A1[r + c * WJ] = m.F[pk(J, n + r, c)];
  }
  __syncwarp();
  wtrsm_r(a, n, Bk{m.A1, WJ}, PkRect{m.F, J, 0}, false, lane);
  double* W = Wc + f.base;
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r >= c) W[pk(J, r, c)] = m.D1[r + c * WN];
  }
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    W[pk(J, n + r, c)] = m.A1[r + c * WJ];
  }
  write_update(f, m, lane);
  __syncwarp();
}

__device__ void gradient_front(const SymDev& S, int k, const double* Wc, double* Sc, double* g, double* Vd,
                               double* ws, const Smem& m, int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_parent(S, f, m, ws, lane);
  load_w(f, m, Wc, lane);
  // S_AN = -V L_AN
  wgemm(a, n, a, -1.0, PkSym{m.F, J, n}, Bk{m.A1, WJ}, 0.0, PkRect{m.F, J, n}, false, lane);
  // S_NN = D^{-1} - S_AN^T L_AN
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    double acc = 0.0;
    for (int t = 0; t < a; ++t) acc = fma(m.F[pk(J, n + t, r)], m.A1[t + c * WJ], acc);
    m.F[pk(J, r, c)] = m.D1[r + c * WN] - acc;
  }
  __syncwarp();
  store_front(f, m, Sc, 1.0, lane);
  if (g) store_front(f, m, g, -1.0, lane);
  double* V = Vd + S.v_off[k];
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r >= s) V[r + s * a] = m.F[pk(J, n + r, n + s)];
  }
  write_full(f, m, lane);
  __syncwarp();
}

__device__ void hess_up_front(const SymDev& S, int k, const double* Wc, const double* Vd, const double* Y,
                              double* T, double* ws, const Smem& m, int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  load_front(f, m, Y, lane);
  load_w(f, m, Wc, lane);
  extend_add(S, f, m, ws, lane);
  // A2 = K_AN = Y_AN - L Y_NN
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    double acc = m.F[pk(J, n + r, c)];
    for (int t = 0; t < n; ++t)
      acc = fma(-m.A1[r + t * WJ], t >= c ? m.F[pk(J, t, c)] : m.F[pk(J, c, t)], acc);
    m.A2[r + c * WJ] = acc;
  }
  __syncwarp();
  // U' = Y_AA - K_AN L^T - L Y_AN^T  (lower)
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) {
      acc = fma(m.A2[r + t * WJ], m.A1[s + t * WJ], acc);
      acc = fma(m.A1[r + t * WJ], m.F[pk(J, n + s, t)], acc);
    }
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  __syncwarp();
  // D2 = K_NN D^{-1};  M_NN = D^{-1} D2 -> T (lower)
  wgemm(n, n, n, 1.0, PkSym{m.F, J, 0}, BkSym{m.D1, WN}, 0.0, Bk{m.D2, WN}, false, lane);
  wgemm(n, n, n, 1.0, BkSym{m.D1, WN}, Bk{m.D2, WN}, 0.0, CscOut{T + f.base, J, 0}, true, lane);
  // A3 = K_AN D^{-1};  M_AN = V A3 -> T
  wgemm(a, n, n, 1.0, Bk{m.A2, WJ}, BkSym{m.D1, WN}, 0.0, Bk{m.A3, WJ}, false, lane);
  wgemm(a, n, a, 1.0, GSym{Vd + S.v_off[k], a}, Bk{m.A3, WJ}, 0.0, CscOut{T + f.base, J, n}, false, lane);
  write_update(f, m, lane);
  __syncwarp();
}

__device__ void hess_down_front(const SymDev& S, int k, const double* Wc, double* T, double* ws, const Smem& m,
                                int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_parent(S, f, m, ws, lane);
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += 32) m.F[e] = T[f.base + e];
  load_w(f, m, Wc, lane);
  // A2 = V' L
  wgemm(a, n, a, 1.0, PkSym{m.F, J, n}, Bk{m.A1, WJ}, 0.0, Bk{m.A2, WJ}, false, lane);
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    m.F[pk(J, n + r, c)] -= 0.5 * m.A2[r + c * WJ];
  }
  __syncwarp();
  // T_NN = M_NN - (Q^T L + L^T Q)
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    double acc = 0.0;
    for (int t = 0; t < a; ++t) {
      acc = fma(m.F[pk(J, n + t, r)], m.A1[t + c * WJ], acc);
      acc = fma(m.A1[t + r * WJ], m.F[pk(J, n + t, c)], acc);
    }
    m.F[pk(J, r, c)] -= acc;
  }
  __syncwarp();
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    m.F[pk(J, n + r, c)] -= 0.5 * m.A2[r + c * WJ];
  }
  __syncwarp();
  store_front(f, m, T, 1.0, lane);
  write_full(f, m, lane);
  __syncwarp();
}

__device__ void ihess_down_front(const SymDev& S, int k, const double* Wc, const double* Dd, const double* Rd,
                                 const double* Tin, double* Y, double* ws, const Smem& m, int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_parent(S, f, m, ws, lane);
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += 32) m.F[e] = Tin[f.base + e];
  load_w(f, m, Wc, lane);
  // A2 = M_AN = T_AN + V' L
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    double acc = m.F[pk(J, n + r, c)];
    for (int t = 0; t < a; ++t)
      acc = fma(n + r >= n + t ? m.F[pk(J, n + r, n + t)] : m.F[pk(J, n + t, n + r)], m.A1[t + c * WJ], acc);
    m.A2[r + c * WJ] = acc;
  }
  __syncwarp();
  // D2 = M_NN = T_NN + T_AN^T L + L^T M_AN  (full)
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    double acc = r >= c ? m.F[pk(J, r, c)] : m.F[pk(J, c, r)];
    for (int t = 0; t < a; ++t) {
      acc = fma(m.F[pk(J, n + t, r)], m.A1[t + c * WJ], acc);
      acc = fma(m.A1[t + r * WJ], m.A2[t + c * WJ], acc);
    }
    m.D2[r + c * WN] = acc;
  }
  __syncwarp();
  const double* D = Dd + S.d_off[k];
  // D1 = M_NN D ;  K_NN = D D1 -> Y (lower)
  wgemm(n, n, n, 1.0, Bk{m.D2, WN}, GSym{D, n}, 0.0, Bk{m.D1, WN}, false, lane);
  wgemm(n, n, n, 1.0, GSym{D, n}, Bk{m.D1, WN}, 0.0, CscOut{Y + f.base, J, 0}, true, lane);
  if (a > 0) {
    // A3 = M_AN D ; K_AN = V^{-1} A3 -> Y  (V^{-1} cached per factor)
    wgemm(a, n, n, 1.0, Bk{m.A2, WJ}, GSym{D, n}, 0.0, Bk{m.A3, WJ}, false, lane);
    wgemm(a, n, a, 1.0, GSym{Rd + S.v_off[k], a}, Bk{m.A3, WJ}, 0.0, CscOut{Y + f.base, J, n}, false, lane);
  }
  write_full(f, m, lane);
  __syncwarp();
}

__device__ void ihess_up_front(const SymDev& S, int k, const double* Wc, double* Y, double* ws, const Smem& m,
                               int lane) {
  Fr f = fr(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  const int tot = J * (J + 1) / 2;
  for (int e = lane; e < tot; e += 32) m.F[e] = 0.0;
  load_w(f, m, Wc, lane);
  extend_add(S, f, m, ws, lane);
  const double* Kc = Y + f.base;
  // A3 = P = K_AN + 1/2 L K_NN
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) acc = fma(m.A1[r + t * WJ], t >= c ? Kc[pk(J, t, c)] : Kc[pk(J, c, t)], acc);
    m.A3[r + c * WJ] = Kc[pk(J, n + r, c)] + 0.5 * acc;
  }
  __syncwarp();
  // U' = Z_AA - (P L^T + L P^T)
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r < s) continue;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) {
      acc = fma(m.A3[r + t * WJ], m.A1[s + t * WJ], acc);
      acc = fma(m.A1[r + t * WJ], m.A3[s + t * WJ], acc);
    }
    m.F[pk(J, n + r, n + s)] -= acc;
  }
  __syncwarp();
  double* Yo = Y + f.base;
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    const int o = pk(J, n + r, c);
    Yo[o] = 2.0 * m.A3[r + c * WJ] - Yo[o] - m.F[o];
  }
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    const int o = pk(J, r, c);
    Yo[o] = Yo[o] - m.F[o];
  }
  write_update(f, m, lane);
  __syncwarp();
}

// S-front of the completion: S_NN and S_AN from the input's columns N_k,
// V_k = S_{A_k A_k} from its later columns (a submatrix of S, Algorithm 7.3),
// so the front depends on no other front.
__device__ void complete_front(const SymDev& S, int k, const double* Sin, double* Lc, double* Wc, double* Dd,
                               double* Vd, double* Rd, double* ldet, int64_t* st, const Smem& m, int lane) {
  Fr f = fr(S, k, nullptr);
  const int J = f.J, n = f.n, a = f.a;
  const int32_t* A = S.rows + S.rows_ptr[k] + n;
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, c = e / a;
    if (r >= c) m.F[pk(J, n + r, n + c)] = Sin[csc_find(S, __ldg(A + r), __ldg(A + c))];
  }
  const int nz = nnz_front(f);
  for (int e = lane; e < nz; e += 32) m.F[e] = Sin[f.base + e];
  __syncwarp();
  double* V = Vd + S.v_off[k];
  double* R = Rd + S.v_off[k];
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r >= s) V[r + s * a] = m.F[pk(J, n + r, n + s)];
  }
  __syncwarp();
  PkBlk Rv{m.F, J, n};
  if (a > 0) wpotrf(a, Rv, st, CHD_ERR_NOT_COMPLETABLE, k, -1, lane);
  for (int e = lane; e < a * a; e += 32) {
    const int r = e % a, s = e / a;
    if (r >= s) R[r + s * a] = m.F[pk(J, n + r, n + s)];
  }
  // A1 = Z = R^{-1} S_AN
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    m.A1[r + c * WJ] = m.F[pk(J, n + r, c)];
  }
  __syncwarp();
  if (a > 0) wtrsm_r(n, a, BkTW{m.A1, WJ}, Rv, true, lane);
  // D1 = P = S_NN - Z^T Z (lower);  A2 = L_AN = -R^{-T} Z
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    double acc = 0.0;
    for (int t = 0; t < a; ++t) acc = fma(m.A1[t + r * WJ], m.A1[t + c * WJ], acc);
    m.D1[r + c * WN] = m.F[pk(J, r, c)] - acc;
  }
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    m.A2[r + c * WJ] = -m.A1[r + c * WJ];
  }
  __syncwarp();
  if (a > 0) wtrsm_r(n, a, BkTW{m.A2, WJ}, Rv, false, lane);
  double* W = Wc + f.base;
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r >= c) W[pk(J, r, c)] = m.D1[r + c * WN];
  }
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    W[pk(J, n + r, c)] = m.A2[r + c * WJ];
  }
  // D2 = Q = chol(P); D1 = Q^{-1} ... D = Q^{-T} Q^{-1}
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    m.D2[r + c * WN] = r >= c ? m.D1[r + c * WN] : 0.0;
  }
  __syncwarp();
  wpotrf(n, Bk{m.D2, WN}, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0, lane);
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    m.D1[r + c * WN] = r == c ? 1.0 : 0.0;
  }
  __syncwarp();
  wtrsm_r(n, n, BkTW{m.D1, WN}, Bk{m.D2, WN}, true, lane);  // D1 = Q^{-1} (lower)
  double* Dk = Dd + S.d_off[k];
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r < c) continue;
    double acc = 0.0;
    for (int t = r; t < n; ++t) acc = fma(m.D1[t + r * WN], m.D1[t + c * WN], acc);
    m.D2[r + c * WN] = acc;  // D (lower)
    Dk[r + c * n] = acc;
  }
  __syncwarp();
  wpotrf(n, Bk{m.D2, WN}, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0, lane);  // C
  double* Lo = Lc + f.base;
  for (int e = lane; e < n * n; e += 32) {
    const int r = e % n, c = e / n;
    if (r >= c) Lo[pk(J, r, c)] = m.D2[r + c * WN];
  }
  for (int e = lane; e < a * n; e += 32) {
    const int r = e % a, c = e / a;
    double acc = 0.0;
    for (int t = c; t < n; ++t) acc = fma(m.A2[r + t * WJ], m.D2[t + c * WN], acc);
    Lo[pk(J, n + r, c)] = acc;
  }
  if (lane == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += 2.0 * log(m.D2[i + i * WN]);
    ldet[k] = s;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// kernels: warp w of block b takes task task0 + b*WPB + w; blockIdx.y = RHS
// ---------------------------------------------------------------------------
__shared__ double wsm[WPB * PER_WARP];

__device__ __forceinline__ Smem smem_for_warp(int w) {
  Smem m;
  double* b = wsm + w * PER_WARP;
  m.F = b;
  m.A1 = b + PK;
  m.A2 = m.A1 + BLK;
  m.A3 = m.A2 + BLK;
  m.D1 = m.A3 + BLK;
  m.D2 = m.D1 + NN;
  return m;
}

#define WARP_TASK_PROLOGUE                                   \
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;   \
  const int t = task0 + blockIdx.x * WPB + w;                \
  if (t >= task_end) return;                                 \
  const Smem m = smem_for_warp(w);

__global__ void __launch_bounds__(WPB * 32) kw_factor(SymDev S, int task0, int task_end, const double* X,
                                                      double* Lc, double* Wc, double* Dd, double* ws,
                                                      double* ldet, int64_t* st) {
  WARP_TASK_PROLOGUE
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q)
    factor_front(S, S.task_fronts[q], X, Lc, Wc, Dd, ws, ldet, st, m, lane);
}
__global__ void __launch_bounds__(WPB * 32) kw_gradient(SymDev S, int task0, int task_end, const double* Wc,
                                                        double* Sc, double* g, double* Vd, double* ws) {
  WARP_TASK_PROLOGUE
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    gradient_front(S, S.task_fronts[q], Wc, Sc, g, Vd, ws, m, lane);
}
__global__ void __launch_bounds__(WPB * 32) kw_hess_up(SymDev S, int task0, int task_end, const double* Wc,
                                                       const double* Vd, const double* Y, int64_t ldy, double* T,
                                                       int64_t ldt, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q)
    hess_up_front(S, S.task_fronts[q], Wc, Vd, Y + y * ldy, T + y * ldt, ws + y * S.f_total, m, lane);
}
__global__ void __launch_bounds__(WPB * 32) kw_hess_down(SymDev S, int task0, int task_end, const double* Wc,
                                                         double* T, int64_t ldt, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    hess_down_front(S, S.task_fronts[q], Wc, T + y * ldt, ws + y * S.f_total, m, lane);
}
__global__ void __launch_bounds__(WPB * 32) kw_ihess_down(SymDev S, int task0, int task_end, const double* Wc,
                                                          const double* Dd, const double* Rd, const double* Tin,
                                                          int64_t ldt, double* Y, int64_t ldy, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    ihess_down_front(S, S.task_fronts[q], Wc, Dd, Rd, Tin + y * ldt, Y + y * ldy, ws + y * S.f_total, m, lane);
}
__global__ void __launch_bounds__(WPB * 32) kw_ihess_up(SymDev S, int task0, int task_end, const double* Wc,
                                                        double* Y, int64_t ldy, double* ws) {
  WARP_TASK_PROLOGUE
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q)
    ihess_up_front(S, S.task_fronts[q], Wc, Y + y * ldy, ws + y * S.f_total, m, lane);
}
// all warp-tier fronts at once, one warp each (the completion has no
// dependencies between fronts)
__global__ void __launch_bounds__(WPB * 32) kw_complete(SymDev S, const double* Sin, double* Lc, double* Wc,
                                                        double* Dd, double* Vd, double* Rd, double* ldet,
                                                        int64_t* st) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * WPB + w;
  if (i >= S.warp_count) return;
  const Smem m = smem_for_warp(w);
  complete_front(S, S.warp_fronts[i], Sin, Lc, Wc, Dd, Vd, Rd, ldet, st, m, lane);
}

}  // namespace warp
}  // namespace chd

namespace chd_launch {
using namespace chd::warp;
static inline dim3 wgrid(int nt, int m) { return dim3((nt + WPB - 1) / WPB, m); }

void warp_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                 double* Dd, double* ws, double* ldet, int64_t* status) {
  kw_factor<<<wgrid(nt, 1), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, X, Lc, Wc, Dd, ws, ldet, status);
  count_launch();
}
void warp_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc,
                   double* g, double* Vd, double* ws) {
  kw_gradient<<<wgrid(nt, 1), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, Wc, Sc, g, Vd, ws);
  count_launch();
}
void warp_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                  const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws) {
  kw_hess_up<<<wgrid(nt, m), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, Wc, Vd, Y, ldy, T, ldt, ws);
  count_launch();
}
void warp_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws) {
  kw_hess_down<<<wgrid(nt, m), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, Wc, T, ldt, ws);
  count_launch();
}
void warp_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                     const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                     double* ws) {
  kw_ihess_down<<<wgrid(nt, m), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
  count_launch();
}
void warp_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                   int64_t ldy, double* ws) {
  kw_ihess_up<<<wgrid(nt, m), WPB * 32, 0, st>>>(s->dev, t0, t0 + nt, Wc, Y, ldy, ws);
  count_launch();
}
void warp_complete_all(const chd_symbolic* s, cudaStream_t st, const double* Sin, double* Lc, double* Wc,
                       double* Dd, double* Vd, double* Rd, double* ldet, int64_t* status) {
  kw_complete<<<wgrid((int)s->dev.warp_count, 1), WPB * 32, 0, st>>>(s->dev, Sin, Lc, Wc, Dd, Vd, Rd, ldet, status);
  count_launch();
}
}  // namespace chd_launch
