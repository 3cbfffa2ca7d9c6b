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
//    q_k x w_k matrix X (row-major: a row is contiguous, so the warp that
//    works on a row reads it coalesced), are lower staircase (row t has
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
    X[(int64_t)t * f.w + c] = c <= rho ? Gp[rho + (int64_t)c * ap] : 0.0;
    return;
  }
  e -= nx;
  const int pp = f.a - f.q;
  const int t = f.q + (int)(e % pp), s = (int)(e / pp);
  if (s > t) return;
  const int pit = __ldg(f.rel + f.a - 1 - t), pis = __ldg(f.rel + f.a - 1 - s);
  G[t + (int64_t)s * f.a] = Sin[f.base_p + csc_off(f.Jp, pis, pit)];
}

// One reflection of row t (columns t .. rho) of the row-major X (ld w),
// applied to the rows (t, r_end): warp 0 forms the reflector (alpha = the
// row's norm, v = x - alpha e_t with v_t computed without cancellation when
// x_t > 0, tau = 2 / v^T v) while the row stays in place; then one warp per
// row r computes d = tau (X[r, .] v) and X[r, t..rho] -= d v^T.  Returns tau
// (0: nothing to annihilate, or a zero row, recorded as a failed
// completion).  Row t itself is left unreduced (its final value alpha e_t
// is written by the caller once no warp reads the reflector).  sh: 4 doubles
// of shared memory.
__device__ inline double reflect(const Info& f, double* X, int t, int rho, int r_end, double* sh, int64_t* st) {
  const int w = f.w, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* xt = X + (int64_t)t * w;
  if (warp == 0) {
    double part = 0.0;
    for (int c = t + 1 + lane; c <= rho; c += 32) part = fma(xt[c], xt[c], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) {
      const double x0 = xt[t], sigma = part;
      double alpha = 0.0, v0 = 0.0, tau = 0.0;
      if (!(sigma == 0.0 && x0 >= 0.0)) {
        alpha = sqrt(fma(x0, x0, sigma));
        if (alpha > 0.0) {
          v0 = x0 > 0.0 ? -sigma / (x0 + alpha) : x0 - alpha;
          tau = 2.0 / fma(v0, v0, sigma);
        } else {
          record_error(st, CHD_ERR_NOT_COMPLETABLE, f.k, -1);
        }
      }
      sh[0] = alpha;
      sh[1] = v0;
      sh[2] = tau;
    }
  }
  __syncthreads();
  const double v0 = sh[1], tau = sh[2];
  if (tau != 0.0) {
    for (int r = t + 1 + warp; r < r_end; r += nw) {
      double* xr = X + (int64_t)r * w;
      double d = lane == 0 ? xr[t] * v0 : 0.0;
      for (int c = t + 1 + lane; c <= rho; c += 32) d = fma(xr[c], xt[c], d);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      d *= tau;
      if (lane == 0) xr[t] -= d * v0;
      for (int c = t + 1 + lane; c <= rho; c += 32) xr[c] = fma(-d, xt[c], xr[c]);
    }
  }
  __syncthreads();
  return tau;
}

// Householder reduction of X (q x w, row-major) to lower triangular form
// from the right, then G[0:q, 0:q] = the lower triangle.  A row with
// rho_t <= t needs no reflection (the condition is the same for the whole
// CTA).  A zero row means V_k is singular.
__device__ inline void reduce(const Info& f, double* X, double* G, int64_t* st) {
  __shared__ double sh[4];
  const int q = f.q, w = f.w, nt = blockDim.x, tid = threadIdx.x;
  for (int t = 0; t < q; ++t) {
    const int rho = f.Jp - 1 - __ldg(f.rel + f.a - 1 - t);
    if (rho <= t) continue;
    if (reflect(f, X, t, rho, q, sh, st) != 0.0) {
      double* xt = X + (int64_t)t * w;
      for (int c = t + 1 + tid; c <= rho; c += nt) xt[c] = 0.0;
      if (tid == 0) xt[t] = sh[0];
      __syncthreads();
    }
  }
  for (int64_t e = tid; e < (int64_t)q * q; e += nt) {
    const int r = (int)(e % q), c = (int)(e / q);
    if (r >= c) G[r + (int64_t)c * f.a] = X[(int64_t)r * w + c];
  }
  __syncthreads();
}

// Blocked form of `reduce` for the dense tier: rows [t0, t1) (a panel of at
// most NB rows) are reduced among themselves, with the panel's reflectors in
// V (L x NB column-major, column j = the reflector of row t0 + j, entry
// c - t0 for its columns c in [t, rho_t], zero elsewhere) and the upper
// triangular T (NB x NB) with H_{t0} ... H_{t1-1} = I - V T V^T (forward
// accumulation: T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] V[:, 0:j]^T v_j).
// The rows below the panel are then updated by three products,
// X[t1:, t0:t0+L] -= (X[t1:, t0:t0+L] V T) V^T (see fc_front).
constexpr int NB = 32;
__device__ inline void panel(const Info& f, double* X, int t0, int t1, int L, double* V, double* T, int64_t* st) {
  __shared__ double sh[4];
  __shared__ double tau[NB];
  __shared__ double gram[NB][NB + 1];
  __shared__ double Ts[NB][NB + 1];
  const int w = f.w, nt = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int64_t e = tid; e < (int64_t)L * NB; e += nt) V[e] = 0.0;
  if (tid < NB) tau[tid] = 0.0;
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int j = t - t0;
    const int rho = f.Jp - 1 - __ldg(f.rel + f.a - 1 - t);
    if (rho <= t) continue;
    const double tj = reflect(f, X, t, rho, t1, sh, st);
    if (tj == 0.0) continue;
    double* xt = X + (int64_t)t * w;
    double* v = V + (int64_t)j * L - t0;  // v[c] for c in [t, rho]
    for (int c = t + tid; c <= rho; c += nt) {
      v[c] = c == t ? sh[1] : xt[c];
      xt[c] = c == t ? sh[0] : 0.0;
    }
    if (tid == 0) tau[j] = tj;
    __syncthreads();
  }
  // Gram matrix of the reflectors (upper part), then T column by column
  for (int pr = warp; pr < NB * NB; pr += nw) {
    const int i = pr % NB, jj = pr / NB;
    if (i >= jj) continue;
    double d = 0.0;
    for (int c = lane; c < L; c += 32) d = fma(V[c + (int64_t)i * L], V[c + (int64_t)jj * L], d);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) gram[i][jj] = d;
  }
  if (tid < NB)
    for (int c = 0; c < NB; ++c) Ts[tid][c] = 0.0;
  __syncthreads();
  for (int jj = 0; jj < NB; ++jj) {
    if (tid < jj) {
      double acc = 0.0;
      for (int l = tid; l < jj; ++l) acc = fma(Ts[tid][l], gram[l][jj], acc);
      Ts[tid][jj] = -tau[jj] * acc;
    }
    if (tid == jj) Ts[jj][jj] = tau[jj];
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += nt) T[e] = Ts[e % NB][e / NB];
  __syncthreads();
}

}  // namespace fc
}  // namespace chd
