// Completion with factored update matrices (Algorithm 4.3; its supernodal
// form at the end of §7.2): device pieces shared by the CTA path
// (kernels.cu) and the dense tier (bigfront.cu).
//
// For a front k with parent p, V_k = S_{A_k A_k} = R_k R_k^T, R_k upper
// triangular, is held reversed as the lower triangular G_k = P R_k P (P the
// reversal of the order of A_k), which is the lower Cholesky factor of
// P V_k P: row t of G_k belongs to A_k[a_k - 1 - t].  In this order the q_k
// rows of A_k that lie in A_p (positions pi >= n_p of J_p) come first, then
// the p_k = a_k - q_k rows that lie in N_p.
//
//  * rows t < q_k: the rows rho_t = J_p - 1 - pi_t of G_p, copied into the
//    q_k x w_k matrix X (column-major), are lower staircase (row t has
//    entries in columns 0 .. rho_t).  Householder reflections applied from
//    the right reduce X to lower triangular form X = [L 0] Q (the reversed
//    form of C = R Q^T, Eq. (e-mfp-compl-3-factored)); L L^T = X X^T is the
//    reversed S on those rows, so G_k[0:q, 0:q] = L.  Reflection t maps
//    row t's entries in columns t .. rho_t onto column t with a positive
//    result; a row with rho_t = t needs none (its columns were never mixed).
//  * rows t >= q_k: M = S~ L^{-T} (the reversed (R^{-1} B)^T) and
//    G~ = chol(A~ - M M^T) (the reversed R~), both with entries of S read
//    from front p's columns: the rows of A_k in N_p have the smaller
//    positions, so every entry (pi_s, pi_t), s <= t, is a column pi_t < n_p
//    entry of front p.
#pragma once

#include "chd_internal.h"
#include "front_views.cuh"

namespace chd {
namespace fc {

struct Info {
  int k, p, a, q, w, np, Jp;
  int64_t base_p;      // CSC offset of front p's first column
  const int32_t* rel;  // positions of A_k in J_p (increasing)
};

__device__ inline Info info(const SymDev& S, int k) {
  Info f;
  f.k = k;
  f.p = (int)S.sn_par[k];
  const int nk = (int)(S.sn_ptr[k + 1] - S.sn_ptr[k]);
  f.a = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]) - nk;
  f.rel = S.rel + S.rows_ptr[k] + nk;
  f.np = (int)(S.sn_ptr[f.p + 1] - S.sn_ptr[f.p]);
  f.Jp = (int)(S.rows_ptr[f.p + 1] - S.rows_ptr[f.p]);
  f.base_p = S.colptr[S.sn_ptr[f.p]];
  // first position >= n_p (rel is increasing)
  int lo = 0, hi = f.a;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(f.rel + mid) >= f.np) hi = mid;
    else lo = mid + 1;
  }
  f.q = f.a - lo;
  f.w = f.q > 0 ? f.Jp - __ldg(f.rel + lo) : 0;
  return f;
}

// number of gather elements: the q x w matrix X, then the a x (a - q) block
// of G_k's last a - q rows (lower part only is written)
__device__ inline int64_t gather_count(const Info& f) {
  return (int64_t)f.q * f.w + (int64_t)(f.a - f.q) * f.a;
}

__device__ inline void gather_one(const Info& f, int64_t e, const double* Sin, const double* Gp, int ap, double* X,
                                  double* G) {
  const int64_t nx = (int64_t)f.q * f.w;
  if (e < nx) {
    const int t = (int)(e % f.q), c = (int)(e / f.q);
    const int rho = f.Jp - 1 - __ldg(f.rel + f.a - 1 - t);
    X[e] = c <= rho ? Gp[rho + (int64_t)c * ap] : 0.0;
    return;
  }
  e -= nx;
  const int pp = f.a - f.q;
  const int t = f.q + (int)(e % pp), s = (int)(e / pp);
  if (s > t) return;
  const int pit = __ldg(f.rel + f.a - 1 - t), pis = __ldg(f.rel + f.a - 1 - s);
  G[t + (int64_t)s * f.a] = Sin[f.base_p + csc_off(f.Jp, pis, pit)];
}

// CTA-wide sum (every thread gets the total); red: 32 doubles of shared memory
__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Householder reduction of X (q x w, column-major) to lower triangular form
// from the right, then G[0:q, 0:q] = the lower triangle.  Reflection t:
// x = X[t, t..rho], alpha = ||x||, v = x - alpha e_t (v_t computed without
// cancellation when x_t > 0), X[r, t..rho] -= (2 / v^T v) (X[r, .] v) v^T
// for r > t; row t becomes alpha e_t.  A zero row means V_k is singular.
__device__ inline void reduce(const Info& f, double* X, double* G, int64_t* st) {
  __shared__ double red[32];
  const int q = f.q, nt = blockDim.x, tid = threadIdx.x;
  for (int t = 0; t < q; ++t) {
    const int rho = f.Jp - 1 - __ldg(f.rel + f.a - 1 - t);
    if (rho <= t) continue;  // nothing to annihilate (uniform over the CTA)
    double part = 0.0;
    for (int c = t + 1 + tid; c <= rho; c += nt) {
      const double x = X[t + (int64_t)c * q];
      part = fma(x, x, part);
    }
    const double sigma = block_sum(part, red);
    const double x0 = X[t + (int64_t)t * q];
    if (sigma == 0.0 && x0 >= 0.0) continue;
    const double alpha = sqrt(fma(x0, x0, sigma));
    if (!(alpha > 0.0)) {
      if (tid == 0) record_error(st, CHD_ERR_NOT_COMPLETABLE, f.k, -1);
      continue;
    }
    const double v0 = x0 > 0.0 ? -sigma / (x0 + alpha) : x0 - alpha;
    const double tau = 2.0 / fma(v0, v0, sigma);
    for (int r = t + 1 + tid; r < q; r += nt) {
      double d = X[r + (int64_t)t * q] * v0;
      for (int c = t + 1; c <= rho; ++c) d = fma(X[r + (int64_t)c * q], X[t + (int64_t)c * q], d);
      d *= tau;
      X[r + (int64_t)t * q] -= d * v0;
      for (int c = t + 1; c <= rho; ++c) X[r + (int64_t)c * q] -= d * X[t + (int64_t)c * q];
    }
    __syncthreads();
    for (int c = t + 1 + tid; c <= rho; c += nt) X[t + (int64_t)c * q] = 0.0;
    if (tid == 0) X[t + (int64_t)t * q] = alpha;
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)q * q; e += nt) {
    const int r = (int)(e % q), c = (int)(e / q);
    if (r >= c) G[r + (int64_t)c * f.a] = X[r + (int64_t)c * q];
  }
  __syncthreads();
}

}  // namespace fc
}  // namespace chd
