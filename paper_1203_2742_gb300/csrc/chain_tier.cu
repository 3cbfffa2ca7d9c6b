// Chain tier: runs of one-column fronts whose rows are contiguous and whose
// ancestor count a is the same along the run (the elimination chains of band
// patterns in natural order), one CTA per run and right-hand side.
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
// cones": for one-column fronts the supernodal Algorithms 7.1 and 7.2 and the
// block forms of Algorithm 5.1 reduce to the scalar recursions of Algorithms
// 3.1, 4.1 and 5.1.  Along such a run, front j has rows j .. j+a, its child
// is front j-1, and the child's update matrix (bottom-up) or the parent's
// front (top-down) covers rows j+1 .. j+a-1 of it.  So the a x a block that
// passes from front to front is a window that slides by one row per column:
// it stays in shared memory (rows addressed modulo WS), each step adds one
// row and drops one, and the only global traffic per column is the column's
// own values.  The run hands over to the rest of the tree through the
// workspace fronts exactly like the other tiers: its top front writes its
// update block (bottom-up) or reads the parent's front (top-down) there.
#include <cuda_runtime.h>

#include <cstdint>

#include "chd_internal.h"
#include "front_views.cuh"

namespace chd_launch {
void count_launch();
}

namespace chd {
namespace chain {

constexpr int CT = 256;       // threads per run
constexpr int AMAX = 64;      // largest a
constexpr int WS = AMAX + 1;  // window slots: rows j .. j + a
constexpr int TPR = 4;        // threads per row of a window product

// run of task t: its first front's record, the run length and a
struct Run {
  int L, a;
  int k0;                         // first supernode (the others follow)
  int64_t base0, col0, d0, v0, vstride, f0, fstride;
};
__device__ __forceinline__ Run run_of(const SymDev& S, int t) {
  Run r;
  const int q0 = S.task_ptr[t], q1 = S.task_ptr[t + 1];
  const WMeta w = S.tmeta[q0];
  r.L = q1 - q0;
  r.a = w.J - 1;
  r.k0 = w.k;
  r.base0 = w.base;
  r.col0 = w.col0;
  r.d0 = w.d_off;
  r.v0 = w.v_off;
  // per-front offsets of one-column fronts (the symbolic phase rounds each
  // block up to a multiple of four doubles)
  r.vstride = ((int64_t)r.a * r.a + 3) & ~int64_t(3);
  const int64_t J = r.a + 1;
  r.f0 = w.f_off;
  r.fstride = (J * J + 2 * J + 3) & ~int64_t(3);
  return r;
}
__device__ __forceinline__ int slot(int g) { return g % WS; }

// out[r] = sum_s Win(r, s) x[s] for r, s < a, Win the window rows/columns
// i0 .. i0 + a - 1 (symmetric, both triangles stored); TPR threads per row,
// the partial sums combined by shuffles.  Valid in the threads with
// tid % TPR == 0 (returned), for row tid / TPR.
__device__ __forceinline__ double window_row_dot(const double (*W)[WS + 1], int i0, int a, const double* x,
                                                 int tid) {
  const int r = tid / TPR, part = tid % TPR;
  double acc = 0.0;
  if (r < a) {
    const int sr = slot(i0 + r);
    for (int s = part; s < a; s += TPR) acc = fma(W[sr][slot(i0 + s)], x[s], acc);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  return acc;
}
// The thread's share of row tid / TPR of the symmetric a x a block B (lower
// triangle stored column-major, ld a): entries s = part, part + TPR, ...
// loaded into registers at once (independent loads, one memory latency),
// so that a step can issue them before its synchronised work and use them
// after it.  Zero beyond a.
constexpr int PF = AMAX / TPR;
struct RowPart {
  double v[PF];
};
__device__ __forceinline__ RowPart load_row_part(const double* B, int a, int tid) {
  RowPart p;
  const int r = tid / TPR, part = tid % TPR;
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int s = part + u * TPR;
    p.v[u] = (r < a && s < a) ? __ldg(B + (r >= s ? r + (int64_t)s * a : s + (int64_t)r * a)) : 0.0;
  }
  return p;
}
// sum over the row's entries of v[s] * x[s] * scale, reduced over the TPR
// threads of the row (valid where tid % TPR == 0)
__device__ __forceinline__ double row_part_dot(const RowPart& p, const double* x, int a, double scale, int tid) {
  const int part = tid % TPR;
  double acc = 0.0;
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int s = part + u * TPR;
    if (s < a) acc = fma(p.v[u], x[s] * scale, acc);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  return acc;
}
// sum over r < a of term(r), the same value in every thread (each warp
// reduces all terms)
template <class Term>
__device__ __forceinline__ double all_sum(int a, Term term, int tid) {
  const int lane = tid & 31;
  double acc = 0.0;
  for (int r = lane; r < a; r += 32) acc += term(r);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Algorithm 7.1 for one-column fronts (Algorithm 3.1): D = F_11, C = sqrt(D),
// B = F_21 / C, L_AN = F_21 / D, U = F_22 - F_21 F_21^T / D.
__global__ void __launch_bounds__(CT) kc_factor(SymDev S, int task0, const double* X, double* Lc, double* Wc,
                                               double* Dd, double* ws, double* ldet, int64_t* st) {
  __shared__ double U[WS][WS + 1];
  __shared__ double f[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int a = R.a, tid = threadIdx.x;
  for (int e = tid; e < WS * (WS + 1); e += CT) (&U[0][0])[e] = 0.0;
  double xv = tid <= a ? X[R.base0 + tid] : 0.0;
  __syncthreads();
  for (int i = 0; i < R.L; ++i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    // column i of the front: its values plus the child's update block
    if (tid <= a) f[tid] = xv + U[slot(i + tid)][slot(i)];
    if (i + 1 < R.L && tid <= a) xv = X[base + (a + 1) + tid];
    __syncthreads();
    double d = f[0];
    if (!(d > 0.0)) {
      if (tid == 0) record_error(st, CHD_ERR_NOT_PD, R.k0 + i, R.col0 + i);
      d = 1.0;
    }
    const double r = rsqrt(d), r2 = r * r;
    if (tid <= a) {
      const double x = f[tid];
      Lc[base + tid] = tid == 0 ? d * r : x * r;
      Wc[base + tid] = tid == 0 ? r2 : x * r2;
    }
    if (tid == 0) {
      Dd[R.d0 + 4 * (int64_t)i] = d;
      ldet[R.k0 + i] = log(d);
    }
    for (int e = tid; e < a * a; e += CT) {
      const int p = e / a, q = e - (e / a) * a;
      U[slot(i + 1 + p)][slot(i + 1 + q)] -= f[1 + p] * f[1 + q] * r2;
    }
    const int si = slot(i);  // row i leaves; its slot is row i + WS, zero until it enters
    for (int e = tid; e < WS; e += CT) {
      U[si][e] = 0.0;
      U[e][si] = 0.0;
    }
    __syncthreads();
  }
  // update block of the top front for the parent (lower, ld J = a + 1)
  double* G = ws + R.f0 + (int64_t)(R.L - 1) * R.fstride;
  const int J = a + 1;
  for (int e = tid; e < a * a; e += CT) {
    const int p = e / a, q = e - (e / a) * a;
    if (p >= q) G[(1 + p) + (int64_t)(1 + q) * J] = U[slot(R.L + p)][slot(R.L + q)];
  }
}

// V (rows i0 .. i0 + a - 1 of the window) <- the parent's front at the
// relative positions of the top front's A (top-down passes)
__device__ void gather_window(const SymDev& S, const Run& R, const double* ws, double (*V)[WS + 1], int tid) {
  const int k1 = R.k0 + R.L - 1;
  const int64_t p = S.sn_par[k1];
  const int a = R.a;
  const int Jp = (int)(S.rows_ptr[p + 1] - S.rows_ptr[p]);
  const double* Fp = ws + S.f_off[p];
  const int32_t* rel = S.rel + S.rows_ptr[k1] + 1;
  const int i0 = R.L;  // rows L .. L + a - 1: the A of the top front L - 1
  for (int e = tid; e < a * a; e += CT) {
    const int r = e / a, s = e - (e / a) * a;
    const int pr = __ldg(rel + r), ps = __ldg(rel + s);
    V[slot(i0 + r)][slot(i0 + s)] = __ldcg(Fp + (pr >= ps ? pr + (int64_t)ps * Jp : ps + (int64_t)pr * Jp));
  }
}

// Algorithm 7.2 for one-column fronts (Algorithm 4.1): S_AN = -V L_AN,
// S_NN = D^{-1} - S_AN^T L_AN; V of the child = [S_NN S_AN^T; S_AN V] on the
// child's rows; V_j is also stored per front (the Hessian-type calls use it).
__global__ void __launch_bounds__(CT) kc_gradient(SymDev S, int task0, const double* Wc, double* Sc, double* g,
                                                 double* Vd, double* ws) {
  __shared__ double V[WS][WS + 1];
  __shared__ double lw[WS];
  __shared__ double sa[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int a = R.a, tid = threadIdx.x;
  gather_window(S, R, ws, V, tid);
  double wv = tid <= a ? Wc[R.base0 + (int64_t)(R.L - 1) * (a + 1) + tid] : 0.0;
  __syncthreads();
  for (int i = R.L - 1; i >= 0; --i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    if (tid <= a) lw[tid] = wv;
    if (i > 0 && tid <= a) wv = Wc[base - (a + 1) + tid];
    // V_i (rows i+1 .. i+a) to the front's block (lower, ld a)
    double* Vb = Vd + R.v0 + (int64_t)i * R.vstride;
    for (int e = tid; e < a * a; e += CT) {
      const int r = e / a, s = e - (e / a) * a;
      if (r >= s) Vb[r + (int64_t)s * a] = V[slot(i + 1 + r)][slot(i + 1 + s)];
    }
    __syncthreads();
    const double sv = -window_row_dot(V, i + 1, a, lw + 1, tid);
    if (tid % TPR == 0 && tid / TPR < a) sa[tid / TPR] = sv;
    __syncthreads();
    const double snn = lw[0] - all_sum(a, [&](int r) { return sa[r] * lw[1 + r]; }, tid);
    if (tid <= a) {
      const double v = tid == 0 ? snn : sa[tid - 1];
      Sc[base + tid] = v;
      if (g) g[base + tid] = -v;
    }
    // row i enters the window: V of the child covers rows i .. i + a - 1
    const int si = slot(i);
    if (tid == 0) V[si][si] = snn;
    for (int r = tid; r < a - 1; r += CT) {
      V[si][slot(i + 1 + r)] = sa[r];
      V[slot(i + 1 + r)][si] = sa[r];
    }
    __syncthreads();
  }
}

// Algorithm 5.1 steps 1-2 for one-column fronts: with Yh the front's values
// plus the child's U', K_jj = Yh_jj, K_A = Yh_A - L_A Yh_jj,
// U' = Yh_AA - K_A L_A^T - L_A Yh_A^T, M_jj = K_jj / D^2, M_A = V K_A / D.
// act (pruned R(Y), §5.5): a front with act == 0 has Y zero in its subtree,
// so K, U' and M are zero and the column is skipped (its output was cleared).
__global__ void __launch_bounds__(CT) kc_hess_up(SymDev S, int task0, const double* Wc, const double* Vd,
                                                const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                                                const uint8_t* act) {
  __shared__ double U[WS][WS + 1];
  __shared__ double h[WS];
  __shared__ double lw[WS];
  __shared__ double kk[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int64_t y = blockIdx.y;
  Y += y * ldy;
  T += y * ldt;
  ws += y * S.f_total;
  const uint8_t* ay = act ? act + y * S.nsn + R.k0 : nullptr;
  const int a = R.a, tid = threadIdx.x;
  for (int e = tid; e < WS * (WS + 1); e += CT) (&U[0][0])[e] = 0.0;
  double yv = tid <= a ? Y[R.base0 + tid] : 0.0;
  double wv = tid <= a ? Wc[R.base0 + tid] : 0.0;
  __syncthreads();
  for (int i = 0; i < R.L; ++i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    const double ycur = yv, wcur = wv;
    if (i + 1 < R.L && tid <= a) {
      yv = Y[base + (a + 1) + tid];
      wv = Wc[base + (a + 1) + tid];
    }
    if (ay && !ay[i]) continue;  // the same decision in every thread
    // V_i's row part, loaded now and used after the window update
    const RowPart vrow = load_row_part(Vd + R.v0 + (int64_t)i * R.vstride, a, tid);
    if (tid <= a) {
      h[tid] = ycur + U[slot(i + tid)][slot(i)];
      lw[tid] = wcur;
    }
    __syncthreads();
    const double h0 = h[0], dinv = lw[0];
    if (tid < a) kk[tid] = h[1 + tid] - lw[1 + tid] * h0;
    __syncthreads();
    for (int e = tid; e < a * a; e += CT) {
      const int p = e / a, q = e - (e / a) * a;
      U[slot(i + 1 + p)][slot(i + 1 + q)] -= fma(kk[p], lw[1 + q], lw[1 + p] * h[1 + q]);
    }
    // M_A = V (K_A / D): V_i from its stored block (lower, ld a)
    {
      const double acc = row_part_dot(vrow, kk, a, 1.0, tid);
      if (tid % TPR == 0 && tid / TPR < a) T[base + 1 + tid / TPR] = acc * dinv;
    }
    if (tid == 0) T[base] = dinv * h0 * dinv;
    const int si = slot(i);
    for (int e = tid; e < WS; e += CT) {
      U[si][e] = 0.0;
      U[e][si] = 0.0;
    }
    __syncthreads();
  }
  double* G = ws + R.f0 + (int64_t)(R.L - 1) * R.fstride;
  const int J = a + 1;
  for (int e = tid; e < a * a; e += CT) {
    const int p = e / a, q = e - (e / a) * a;
    if (p >= q) G[(1 + p) + (int64_t)(1 + q) * J] = U[slot(R.L + p)][slot(R.L + q)];
  }
}

// Algorithm 5.1 step 3 for one-column fronts: with w = V' L_A,
// T_A = M_A - w, T_jj = M_jj - 2 L_A^T M_A + L_A^T w; V' of the child =
// [T_jj T_A^T; T_A V'] on the child's rows.
__global__ void __launch_bounds__(CT) kc_hess_down(SymDev S, int task0, const double* Wc, double* T, int64_t ldt,
                                                  double* ws) {
  __shared__ double V[WS][WS + 1];
  __shared__ double lw[WS];
  __shared__ double mv[WS];
  __shared__ double wl[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int64_t y = blockIdx.y;
  T += y * ldt;
  ws += y * S.f_total;
  const int a = R.a, tid = threadIdx.x;
  gather_window(S, R, ws, V, tid);
  const int64_t top = R.base0 + (int64_t)(R.L - 1) * (a + 1);
  double wv = tid <= a ? Wc[top + tid] : 0.0;
  double tv = tid <= a ? T[top + tid] : 0.0;
  __syncthreads();
  for (int i = R.L - 1; i >= 0; --i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    if (tid <= a) {
      lw[tid] = wv;
      mv[tid] = tv;
    }
    if (i > 0 && tid <= a) {
      wv = Wc[base - (a + 1) + tid];
      tv = T[base - (a + 1) + tid];
    }
    __syncthreads();
    const double wr = window_row_dot(V, i + 1, a, lw + 1, tid);
    if (tid % TPR == 0 && tid / TPR < a) wl[tid / TPR] = wr;
    __syncthreads();
    const double tnn = mv[0] + all_sum(a, [&](int r) { return lw[1 + r] * (wl[r] - 2.0 * mv[1 + r]); }, tid);
    if (tid <= a) T[base + tid] = tid == 0 ? tnn : mv[tid] - wl[tid - 1];
    const int si = slot(i);
    if (tid == 0) V[si][si] = tnn;
    for (int r = tid; r < a - 1; r += CT) {
      const double v = mv[1 + r] - wl[r];
      V[si][slot(i + 1 + r)] = v;
      V[slot(i + 1 + r)][si] = v;
    }
    __syncthreads();
  }
}

// Algorithm 5.2 steps 1-2 for one-column fronts (top-down): with the window
// V' (the input T on A_j x A_j, gathered from the parent's T-front),
// M_A = T_A + V' L_A, M_jj = T_jj + L_A^T (T_A + M_A), K_jj = D M_jj D,
// K_A = V^{-1} (M_A D) (V^{-1} per front, formed by the inverse-Hessian
// setup); the child's window is [T_jj T_A^T; T_A V'] on its rows.
__global__ void __launch_bounds__(CT) kc_ihess_down(SymDev S, int task0, const double* Wc, const double* Dd,
                                                   const double* Rd, const double* Tin, int64_t ldt, double* Y,
                                                   int64_t ldy, double* ws) {
  __shared__ double V[WS][WS + 1];
  __shared__ double lw[WS];
  __shared__ double tt[WS];
  __shared__ double ma[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int64_t y = blockIdx.y;
  Tin += y * ldt;
  Y += y * ldy;
  ws += y * S.f_total;
  const int a = R.a, tid = threadIdx.x;
  gather_window(S, R, ws, V, tid);
  const int64_t top = R.base0 + (int64_t)(R.L - 1) * (a + 1);
  double wv = tid <= a ? Wc[top + tid] : 0.0;
  double tv = tid <= a ? Tin[top + tid] : 0.0;
  __syncthreads();
  for (int i = R.L - 1; i >= 0; --i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    if (tid <= a) {
      lw[tid] = wv;
      tt[tid] = tv;
    }
    if (i > 0 && tid <= a) {
      wv = Wc[base - (a + 1) + tid];
      tv = Tin[base - (a + 1) + tid];
    }
    // V_i^{-1}'s row part, loaded now and used after the window products
    const RowPart rrow = load_row_part(Rd + R.v0 + (int64_t)i * R.vstride, a, tid);
    __syncthreads();
    const double wr = window_row_dot(V, i + 1, a, lw + 1, tid);
    if (tid % TPR == 0 && tid / TPR < a) ma[tid / TPR] = tt[1 + tid / TPR] + wr;
    __syncthreads();
    const double dd = Dd[R.d0 + 4 * (int64_t)i];
    const double mnn = tt[0] + all_sum(a, [&](int r) { return lw[1 + r] * (tt[1 + r] + ma[r]); }, tid);
    if (tid == 0) Y[base] = dd * (mnn * dd);
    {
      const double acc = row_part_dot(rrow, ma, a, dd, tid);
      if (tid % TPR == 0 && tid / TPR < a) Y[base + 1 + tid / TPR] = acc;
    }
    const int si = slot(i);
    if (tid == 0) V[si][si] = tt[0];
    for (int r = tid; r < a - 1; r += CT) {
      V[si][slot(i + 1 + r)] = tt[1 + r];
      V[slot(i + 1 + r)][si] = tt[1 + r];
    }
    __syncthreads();
  }
}

// Algorithm 5.2 step 3 for one-column fronts (bottom-up): with K from the
// top-down pass and F the child's U' on this front's rows,
// P = K_A + L_A K_jj / 2, Y_jj = K_jj - F_jj, Y_A = 2 P - K_A - F_A,
// U' = F_AA - (P L_A^T + L_A P^T).
__global__ void __launch_bounds__(CT) kc_ihess_up(SymDev S, int task0, const double* Wc, double* Y, int64_t ldy,
                                                 double* ws) {
  __shared__ double U[WS][WS + 1];
  __shared__ double lw[WS];
  __shared__ double kk[WS];
  __shared__ double ff[WS];
  __shared__ double pp[WS];
  const Run R = run_of(S, task0 + blockIdx.x);
  const int64_t y = blockIdx.y;
  Y += y * ldy;
  ws += y * S.f_total;
  const int a = R.a, tid = threadIdx.x;
  for (int e = tid; e < WS * (WS + 1); e += CT) (&U[0][0])[e] = 0.0;
  double kv = tid <= a ? Y[R.base0 + tid] : 0.0;
  double wv = tid <= a ? Wc[R.base0 + tid] : 0.0;
  __syncthreads();
  for (int i = 0; i < R.L; ++i) {
    const int64_t base = R.base0 + (int64_t)i * (a + 1);
    if (tid <= a) {
      kk[tid] = kv;
      lw[tid] = wv;
      ff[tid] = U[slot(i + tid)][slot(i)];
    }
    if (i + 1 < R.L && tid <= a) {
      kv = Y[base + (a + 1) + tid];
      wv = Wc[base + (a + 1) + tid];
    }
    __syncthreads();
    if (tid < a) pp[tid] = fma(0.5 * lw[1 + tid], kk[0], kk[1 + tid]);
    __syncthreads();
    if (tid <= a) Y[base + tid] = tid == 0 ? kk[0] - ff[0] : 2.0 * pp[tid - 1] - kk[tid] - ff[tid];
    for (int e = tid; e < a * a; e += CT) {
      const int p = e / a, q = e - (e / a) * a;
      U[slot(i + 1 + p)][slot(i + 1 + q)] -= fma(pp[p], lw[1 + q], lw[1 + p] * pp[q]);
    }
    const int si = slot(i);
    for (int e = tid; e < WS; e += CT) {
      U[si][e] = 0.0;
      U[e][si] = 0.0;
    }
    __syncthreads();
  }
  double* G = ws + R.f0 + (int64_t)(R.L - 1) * R.fstride;
  const int J = a + 1;
  for (int e = tid; e < a * a; e += CT) {
    const int p = e / a, q = e - (e / a) * a;
    if (p >= q) G[(1 + p) + (int64_t)(1 + q) * J] = U[slot(R.L + p)][slot(R.L + q)];
  }
}

}  // namespace chain
}  // namespace chd

namespace chd_launch {
using namespace chd::chain;
void chain_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                  double* Dd, double* ws, double* ldet, int64_t* status) {
  kc_factor<<<nt, CT, 0, st>>>(s->dev, t0, X, Lc, Wc, Dd, ws, ldet, status);
  count_launch();
}
void chain_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc, double* g,
                    double* Vd, double* ws) {
  kc_gradient<<<nt, CT, 0, st>>>(s->dev, t0, Wc, Sc, g, Vd, ws);
  count_launch();
}
void chain_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, const double* Vd,
                   const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws, const uint8_t* act) {
  kc_hess_up<<<dim3(nt, m), CT, 0, st>>>(s->dev, t0, Wc, Vd, Y, ldy, T, ldt, ws, act);
  count_launch();
}
void chain_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                     int64_t ldt, double* ws) {
  kc_hess_down<<<dim3(nt, m), CT, 0, st>>>(s->dev, t0, Wc, T, ldt, ws);
  count_launch();
}
void chain_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                      const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                      double* ws) {
  kc_ihess_down<<<dim3(nt, m), CT, 0, st>>>(s->dev, t0, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
  count_launch();
}
void chain_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                    int64_t ldy, double* ws) {
  kc_ihess_up<<<dim3(nt, m), CT, 0, st>>>(s->dev, t0, Wc, Y, ldy, ws);
  count_launch();
}
}  // namespace chd_launch
