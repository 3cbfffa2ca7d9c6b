// FP64 supernodal multifrontal kernels for sm_103a.
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
// cones".  One CTA processes one task (a sequence of fronts in postorder,
// bottom-up; reversed, top-down) for one right-hand side.  A front k has
// N_k (n columns, contiguous) and A_k (a rows), J = n + a.  Its workspace in
// global memory (L2-resident in practice) is the dense J x J front F
// (column-major, ld = J, lower triangle used) followed by two J x n
// temporaries T1, T2.  Value arrays (X, Y, S, T, the factor) are in the CSC
// of the filled pattern: column c of front k holds rows c..J-1 of the
// front, so element (r, c), r >= c, sits at
//     base_k + c*(J-1) - c*(c-1)/2 + r,   base_k = colptr[first column of k].
//
// Per-front storage kept by a factor object:
//   Lc  (CSC)  : [C; B], the supernodal Cholesky factor, D_NN = C C^T,
//                B = L_{AN} C  (Algorithm 7.1: D_NN = F11, L_AN = F21 D^-1)
//   Wc  (CSC)  : [D_NN^{-1}; L_AN]
//   Dd  (n x n): D_NN
//   Vd  (a x a): V_k = S_{A_k A_k}  (Algorithm 7.2)
//   Rd  (a x a): V_k^{-1} (lower triangle; inverse Hessian, §5.3) for the
//                warp and CTA tiers, R = chol(V_k) for dense-tier fronts
//   Qd  (a x a): chol(P V_k P), P the order reversal (Hessian factor, §5.4)
//   Sc  (CSC)  : S = P(X^{-1})
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "chd_internal.h"
#include "fc_body.cuh"
#include "front_views.cuh"

namespace chd {

constexpr int NT = 256;      // threads per CTA
constexpr int TB = 32;       // gemm tile (TB x TB outputs)
constexpr int TK = 16;       // gemm k-chunk
constexpr int PB = 32;       // potrf panel width
constexpr int PCH = 96;      // rows per panel chunk staged in shared memory

// Shared-memory staging pool, declared once at namespace scope so that every
// routine of a kernel uses the same 34 KB: the GEMM stages its A and B
// chunks at the start of the pool, the panel Cholesky its diagonal block and
// row panel (never live at the same time as a GEMM's chunks).
constexpr int GMAX = 128;  // largest GEMM tile side
constexpr int POOL_GEMM = 2 * TK * GMAX;
constexpr int POOL_POTRF = PB * (PB + 1) + PCH * (PB + 1);
constexpr int POOL = POOL_GEMM > POOL_POTRF ? POOL_GEMM : POOL_POTRF;
__shared__ double sh_pool[POOL];

// ---------------------------------------------------------------------------
// CTA GEMM:  C = beta*C + alpha * A(MxK) B(KxN), optionally lower triangle only.
// Output blocks of BM x BN (BM*BN = 1024, 2x2 outputs per thread) picked from
// the shape so that skinny products do not pay for padding; k-chunks of up
// to 16 staged in shared memory, the k loop runs only over real K.
// beta == 0 never reads C.
// ---------------------------------------------------------------------------
template <int BM, int BN, class MA, class MB, class MC>
__device__ void cta_gemm_t(int M, int N, int K, double alpha, MA A, MB B, double beta, MC C, bool lower) {
  double* As = sh_pool;            // TK x BM
  double* Bs = sh_pool + TK * GMAX;  // TK x BN
  const int tid = threadIdx.x;
  constexpr int HX = BN / 2, HY = BM / 2;
  const int tx = tid % HX, ty = tid / HX;
  for (int tm = 0; tm < M; tm += BM) {
    for (int tn = 0; tn < N; tn += BN) {
      if (lower && tn >= tm + BM) continue;
      double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
      for (int k0 = 0; k0 < K; k0 += TK) {
        const int kc = min(TK, K - k0);
        for (int e = tid; e < BM * kc; e += NT) {
          const int r = e % BM, kk = e / BM;
          As[kk * BM + r] = (tm + r < M) ? A.at(tm + r, k0 + kk) : 0.0;
        }
        for (int e = tid; e < BN * kc; e += NT) {
          const int kk = e % kc, c = e / kc;
          Bs[kk * BN + c] = (tn + c < N) ? B.at(k0 + kk, tn + c) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kc; ++kk) {
          const double a0 = As[kk * BM + ty], a1 = As[kk * BM + ty + HY];
          const double b0 = Bs[kk * BN + tx], b1 = Bs[kk * BN + tx + HX];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        __syncthreads();
      }
      const double acc[2][2] = {{c00, c01}, {c10, c11}};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = tm + ty + HY * i, c = tn + tx + HX * j;
          if (r < M && c < N && (!lower || r >= c)) {
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C.at(r, c), v);
            C.at(r, c) = v;
          }
        }
    }
  }
  __syncthreads();
}

template <class MA, class MB, class MC>
__device__ void cta_gemm(int M, int N, int K, double alpha, MA A, MB B, double beta, MC C, bool lower) {
  if (M <= 0 || N <= 0) return;
  if (N <= 8 && M > 32) cta_gemm_t<128, 8>(M, N, K, alpha, A, B, beta, C, lower);
  else if (N <= 16 && M > 32) cta_gemm_t<64, 16>(M, N, K, alpha, A, B, beta, C, lower);
  else if (M <= 8 && N > 32) cta_gemm_t<8, 128>(M, N, K, alpha, A, B, beta, C, lower);
  else if (M <= 16 && N > 32) cta_gemm_t<16, 64>(M, N, K, alpha, A, B, beta, C, lower);
  else cta_gemm_t<32, 32>(M, N, K, alpha, A, B, beta, C, lower);
}

// ---------------------------------------------------------------------------
// Unblocked Cholesky of a small block held in shared memory (row-major,
// stride PB+1).  Non-positive pivots are recorded and replaced by 1.
// ---------------------------------------------------------------------------
__device__ void smem_potrf(double* Ls, int jb, int64_t* st, int64_t code, int64_t snode,
                           int64_t col0) {
  const int tid = threadIdx.x;
  for (int j = 0; j < jb; ++j) {
    if (tid == 0) {
      double d = Ls[j * (PB + 1) + j];
      if (!(d > 0.0)) {
        record_error(st, code, snode, col0 + j);
        d = 1.0;
      }
      Ls[j * (PB + 1) + j] = sqrt(d);
    }
    __syncthreads();
    const double piv = Ls[j * (PB + 1) + j];
    for (int i = j + 1 + tid; i < jb; i += NT) Ls[i * (PB + 1) + j] /= piv;
    __syncthreads();
    const int m = jb - j - 1;
    for (int e = tid; e < m * m; e += NT) {
      int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) Ls[i * (PB + 1) + k] -= Ls[i * (PB + 1) + j] * Ls[k * (PB + 1) + j];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky of the first n columns of the J x J front
// F (column-major, ld): afterwards F[0:n,0:n] = C (lower), F[n:J,0:n] =
// F21 C^{-T}, F[n:J,n:J] -= (F21 C^{-T})(F21 C^{-T})^T (lower).  With n == J
// this is a plain dense Cholesky factorisation.
// ---------------------------------------------------------------------------
__device__ void cta_potrf_partial(double* F, int64_t ld, int J, int n, int64_t* st, int64_t code,
                                  int64_t snode, int64_t col0) {
  double* Ls = sh_pool;
  double* Ps = sh_pool + PB * (PB + 1);
  const int tid = threadIdx.x;
  for (int j0 = 0; j0 < n; j0 += PB) {
    const int jb = min(PB, n - j0);
    for (int e = tid; e < jb * jb; e += NT) {
      int r = e % jb, c = e / jb;
      Ls[r * (PB + 1) + c] = (r >= c) ? F[(j0 + r) + (int64_t)(j0 + c) * ld] : 0.0;
    }
    __syncthreads();
    smem_potrf(Ls, jb, st, code, snode, col0 + j0);
    for (int e = tid; e < jb * jb; e += NT) {
      int r = e % jb, c = e / jb;
      if (r >= c) F[(j0 + r) + (int64_t)(j0 + c) * ld] = Ls[r * (PB + 1) + c];
    }
    // panel rows below the diagonal block: X := P L11^{-T}
    const int rbeg = j0 + jb;
    for (int r0 = rbeg; r0 < J; r0 += PCH) {
      const int rc = min(PCH, J - r0);
      for (int e = tid; e < rc * jb; e += NT) {
        int r = e % rc, c = e / rc;
        Ps[r * (PB + 1) + c] = F[(r0 + r) + (int64_t)(j0 + c) * ld];
      }
      __syncthreads();
      for (int c = 0; c < jb; ++c) {
        const double inv = 1.0 / Ls[c * (PB + 1) + c];
        for (int r = tid; r < rc; r += NT) Ps[r * (PB + 1) + c] *= inv;
        __syncthreads();
        const int m = jb - c - 1;
        for (int e = tid; e < rc * m; e += NT) {
          int r = e % rc, t = c + 1 + e / rc;
          Ps[r * (PB + 1) + t] -= Ps[r * (PB + 1) + c] * Ls[t * (PB + 1) + c];
        }
        __syncthreads();
      }
      for (int e = tid; e < rc * jb; e += NT) {
        int r = e % rc, c = e / rc;
        F[(r0 + r) + (int64_t)(j0 + c) * ld] = Ps[r * (PB + 1) + c];
      }
      __syncthreads();
    }
    // trailing update of the lower triangle of F[rbeg:J, rbeg:J]
    const int m = J - rbeg;
    if (m > 0) {
      double* P = F + rbeg + (int64_t)j0 * ld;
      cta_gemm(m, m, jb, -1.0, Dn{P, ld}, DnT{P, ld}, 1.0, Dn{F + rbeg + (int64_t)rbeg * ld, ld}, true);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Right-side triangular solves on an R x n matrix B (any writable view with
// colshift) with a lower triangular n x n matrix L (column-major, ld):
//   trsm_rLT:  B := B L^{-T}      trsm_rL:  B := B L^{-1}
// Blocked: 32-column panels solved in shared memory (row chunks of 96,
// column sweeps against the 32 x 32 diagonal block), the rest of B updated
// by the tiled CTA GEMM.  Left-side solves are the same on the transposed
// view of B.
// ---------------------------------------------------------------------------
template <class MB>
__device__ void cta_panel_solve(int R, MB B, int p0, int pb, const double* L, int64_t ld, bool fwd) {
  double* Ls = sh_pool;
  double* Ps = sh_pool + PB * (PB + 1);
  const int tid = threadIdx.x;
  for (int e = tid; e < pb * pb; e += NT) {
    const int i = e % pb, j = e / pb;
    Ls[i * (PB + 1) + j] = i >= j ? L[(p0 + i) + (int64_t)(p0 + j) * ld] : 0.0;
  }
  for (int r0 = 0; r0 < R; r0 += PCH) {
    const int rc = min(PCH, R - r0);
    for (int e = tid; e < rc * pb; e += NT) {
      const int r = e % rc, c = e / rc;
      Ps[r * (PB + 1) + c] = B.at(r0 + r, p0 + c);
    }
    __syncthreads();
    if (fwd) {
      for (int c = 0; c < pb; ++c) {
        const double inv = 1.0 / Ls[c * (PB + 1) + c];
        for (int r = tid; r < rc; r += NT) Ps[r * (PB + 1) + c] *= inv;
        __syncthreads();
        const int m = pb - c - 1;
        for (int e = tid; e < rc * m; e += NT) {
          const int r = e % rc, t = c + 1 + e / rc;
          Ps[r * (PB + 1) + t] -= Ps[r * (PB + 1) + c] * Ls[t * (PB + 1) + c];
        }
        __syncthreads();
      }
    } else {
      for (int c = pb - 1; c >= 0; --c) {
        const double inv = 1.0 / Ls[c * (PB + 1) + c];
        for (int r = tid; r < rc; r += NT) Ps[r * (PB + 1) + c] *= inv;
        __syncthreads();
        for (int e = tid; e < rc * c; e += NT) {
          const int r = e % rc, t = e / rc;
          Ps[r * (PB + 1) + t] -= Ps[r * (PB + 1) + c] * Ls[c * (PB + 1) + t];
        }
        __syncthreads();
      }
    }
    for (int e = tid; e < rc * pb; e += NT) {
      const int r = e % rc, c = e / rc;
      B.at(r0 + r, p0 + c) = Ps[r * (PB + 1) + c];
    }
    __syncthreads();
  }
}
template <class MB>
__device__ void cta_trsm_rLT(int R, int n, MB B, const double* L, int64_t ld) {
  if (R <= 0 || n <= 0) return;
  for (int p0 = 0; p0 < n; p0 += PB) {
    const int pb = min(PB, n - p0);
    cta_panel_solve(R, B, p0, pb, L, ld, true);
    const int rest = n - p0 - pb;
    if (rest > 0)
      cta_gemm(R, rest, pb, -1.0, colshift(B, p0), DnT{L + (p0 + pb) + (int64_t)p0 * ld, ld}, 1.0,
               colshift(B, p0 + pb), false);
  }
}
template <class MB>
__device__ void cta_trsm_rL(int R, int n, MB B, const double* L, int64_t ld) {
  if (R <= 0 || n <= 0) return;
  const int np = (n + PB - 1) / PB;
  for (int q = np - 1; q >= 0; --q) {
    const int p0 = q * PB, pb = min(PB, n - p0);
    cta_panel_solve(R, B, p0, pb, L, ld, false);
    if (p0 > 0)
      cta_gemm(R, p0, pb, -1.0, colshift(B, p0), Dn{const_cast<double*>(L) + p0, ld}, 1.0, colshift(B, 0),
               false);
  }
}

// ---------------------------------------------------------------------------
// small element-wise helpers
// ---------------------------------------------------------------------------
__device__ void csc_to_front(double* F, int J, int n, const double* csc) {
  for (int e = threadIdx.x; e < J * n; e += NT) {
    int r = e % J, c = e / J;
    if (r >= c) F[r + (int64_t)c * J] = csc[csc_off(J, r, c)];
  }
}
__device__ void front_to_csc(double* csc, const double* F, int J, int n, double scale) {
  for (int e = threadIdx.x; e < J * n; e += NT) {
    int r = e % J, c = e / J;
    if (r >= c) csc[csc_off(J, r, c)] = scale * F[r + (int64_t)c * J];
  }
}
__device__ void zero_lower(double* F, int64_t ld, int m, int off) {
  for (int e = threadIdx.x; e < m * m; e += NT) {
    int r = e % m, c = e / m;
    if (r >= c) F[(off + r) + (int64_t)(off + c) * ld] = 0.0;
  }
}
__device__ void copy_lower(double* dst, int64_t ldd, const double* src, int64_t lds, int m) {
  for (int e = threadIdx.x; e < m * m; e += NT) {
    int r = e % m, c = e / m;
    if (r >= c) dst[r + (int64_t)c * ldd] = src[r + (int64_t)c * lds];
  }
}
__device__ void copy_rect(double* dst, int64_t ldd, const double* src, int64_t lds, int R, int C) {
  for (int e = threadIdx.x; e < R * C; e += NT) {
    int r = e % R, c = e / R;
    dst[r + (int64_t)c * ldd] = src[r + (int64_t)c * lds];
  }
}
__device__ void set_identity(double* dst, int64_t ld, int m) {
  for (int e = threadIdx.x; e < m * m; e += NT) {
    int r = e % m, c = e / m;
    dst[r + (int64_t)c * ld] = (r == c) ? 1.0 : 0.0;
  }
}

struct FrontInfo {
  int k, n, a, J;
  int64_t col0;     // first column of N_k
  int64_t base;     // colptr[col0]
  double* F;        // J x J front
  double* T1;       // J x n
  double* T2;       // J x n
};

__device__ FrontInfo front_info(const SymDev& S, int k, double* ws) {
  FrontInfo f;
  f.k = k;
  f.col0 = S.sn_ptr[k];
  f.n = (int)(S.sn_ptr[k + 1] - f.col0);
  f.J = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  f.a = f.J - f.n;
  f.base = S.colptr[f.col0];
  f.F = ws + S.f_off[k];
  f.T1 = f.F + (int64_t)f.J * f.J;
  f.T2 = f.T1 + (int64_t)f.J * f.n;
  return f;
}

// Extend-add of every child's update matrix (the A x A block of the child's
// front) into this front: F += E_{J A_c} U_c E_{J A_c}^T  (children in a
// fixed order, entries of one child touch distinct positions).
__device__ void extend_add_children(const SymDev& S, const FrontInfo& f, double* ws, double sign,
                                    const uint8_t* act = nullptr) {
  for (int64_t q = S.ea_ptr[f.k]; q < S.ea_ptr[f.k + 1]; ++q) {
    const int c = S.ea[q];
    if (act && !act[c]) continue;  // pruned subtree: its update block is zero
    const int nc = (int)(S.sn_ptr[c + 1] - S.sn_ptr[c]);
    const int Jc = (int)(S.rows_ptr[c + 1] - S.rows_ptr[c]);
    const int ac = Jc - nc;
    const int32_t* rel = S.rel + S.rows_ptr[c] + nc;
    const double* U = ws + S.f_off[c] + nc + (int64_t)nc * Jc;
    for (int e = threadIdx.x; e < ac * ac; e += NT) {
      int r = e % ac, s = e / ac;
      if (r >= s) {
        int pr = __ldg(rel + r), ps = __ldg(rel + s);
        f.F[pr + (int64_t)ps * f.J] += sign * __ldcg(U + r + (int64_t)s * Jc);
      }
    }
    __syncthreads();
  }
}

// Gather V_k = E_{J_p A_k}^T F_p E_{J_p A_k} from the parent's full front
// into the A x A block of this front (top-down propagation, Eq. (e-sn-gradient-2)).
__device__ void gather_from_parent(const SymDev& S, const FrontInfo& f, double* ws) {
  const int p = (int)S.sn_par[f.k];
  if (p < 0 || f.a == 0) return;
  const int Jp = (int)(S.rows_ptr[p + 1] - S.rows_ptr[p]);
  const double* Fp = ws + S.f_off[p];
  const int32_t* rel = S.rel + S.rows_ptr[f.k] + f.n;
  for (int e = threadIdx.x; e < f.a * f.a; e += NT) {
    int r = e % f.a, s = e / f.a;
    if (r >= s) {
      int pr = __ldg(rel + r), ps = __ldg(rel + s);
      f.F[(f.n + r) + (int64_t)(f.n + s) * f.J] = __ldcg(Fp + pr + (int64_t)ps * Jp);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Front procedures
// ---------------------------------------------------------------------------

// Algorithm 7.1 for one front, then the derived blocks D_NN^{-1} and L_AN.
__device__ void factor_front(const SymDev& S, int k, const double* X, double* Lc, double* Wc,
                             double* Dd, double* ws, double* ldet, int64_t* st) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  csc_to_front(f.F, J, n, X + f.base);
  zero_lower(f.F, J, a, n);
  __syncthreads();
  extend_add_children(S, f, ws, 1.0);
  // D_NN = F11 (kept for the inverse Hessian)
  copy_lower(Dd + S.d_off[k], n, f.F, J, n);
  cta_potrf_partial(f.F, J, J, n, st, CHD_ERR_NOT_PD, k, f.col0);
  front_to_csc(Lc + f.base, f.F, J, n, 1.0);
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += 2.0 * log(f.F[i + (int64_t)i * J]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) ldet[k] = s;
  }
  // Cinv = C^{-1} in T1[0:n,0:n]; D^{-1} = Cinv^T Cinv -> T2[0:n,0:n];
  // L_AN = B C^{-1} -> T2[n:J, 0:n]
  set_identity(f.T1, J, n);
  __syncthreads();
  cta_trsm_rLT(n, n, DnTW{f.T1, J}, f.F, J);  // (I^T C^{-T})^T = C^{-1}
  cta_gemm(n, n, n, 1.0, TriLT{f.T1, J}, TriL{f.T1, J}, 0.0, Dn{f.T2, J}, true);
  copy_rect(f.T2 + n, J, f.F + n, J, a, n);
  __syncthreads();
  cta_trsm_rL(a, n, Dn{f.T2 + n, J}, f.F, J);
  front_to_csc(Wc + f.base, f.T2, J, n, 1.0);
  __syncthreads();
}

// Algorithm 3.2 (Cholesky product) for one front, supernodal form: F = the
// children's blocks + G G^T with G = [C; B] = [I; L_AN] C (so G G^T =
// [I; L_AN] D_NN [I; L_AN]^T); the N-part of F is X_{J N}, and the A x A
// block (-U in Eq. (e-mf-prod)) stays in the front for the parent.
__device__ void product_front(const SymDev& S, int k, const double* Lc, double* Xo, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n;
  zero_lower(f.F, J, J, 0);
  __syncthreads();
  extend_add_children(S, f, ws, 1.0);
  cta_gemm(J, J, n, 1.0, CscL{Lc + f.base, J}, CscLT{Lc + f.base, J}, 1.0, Dn{f.F, J}, true);
  front_to_csc(Xo + f.base, f.F, J, n, 1.0);
  __syncthreads();
}

// Algorithm 7.2 for one front: S_AN = -V L_AN, S_NN = D^{-1} - S_AN^T L_AN.
__device__ void gradient_front(const SymDev& S, int k, const double* Wc, double* Sc, double* g,
                               double* Vd, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_from_parent(S, f, ws);
  const double* W = Wc + f.base;
  // S_AN = -V L_AN
  cta_gemm(a, n, a, -1.0, SymL{f.F + n + (int64_t)n * J, J}, CscRO{W, J, n}, 0.0,
           Dn{f.F + n, J}, false);
  // S_NN = D^{-1} - S_AN^T L_AN
  for (int e = threadIdx.x; e < n * n; e += NT) {
    int r = e % n, c = e / n;
    if (r >= c) f.F[r + (int64_t)c * J] = W[csc_off(J, r, c)];
  }
  __syncthreads();
  cta_gemm(n, n, a, -1.0, DnT{f.F + n, J}, CscRO{W, J, n}, 1.0, Dn{f.F, J}, true);
  front_to_csc(Sc + f.base, f.F, J, n, 1.0);
  if (g) front_to_csc(g + f.base, f.F, J, n, -1.0);
  copy_lower(Vd + S.v_off[k], a, f.F + n + (int64_t)n * J, J, a);
  __syncthreads();
}

// Algorithm 5.1 steps 1-2 (block form) for one front and one right-hand side:
// K_NN = Yh_NN, K_AN = Yh_AN - L Yh_NN, U' = Yh_AA - K_AN L^T - L Yh_AN^T,
// M_NN = D^{-1} K_NN D^{-1}, M_AN = V K_AN D^{-1}; M is written to the
// output array (CSC), U' stays in the front for the parent.
__device__ void hess_up_front(const SymDev& S, int k, const double* Wc, const double* Vd,
                              const double* Y, double* T, double* ws, const uint8_t* act) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  csc_to_front(f.F, J, n, Y + f.base);
  zero_lower(f.F, J, a, n);
  __syncthreads();
  extend_add_children(S, f, ws, 1.0, act);
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  // T1[n:J] = K_AN = Yh_AN - L Yh_NN
  copy_rect(f.T1 + n, J, f.F + n, J, a, n);
  __syncthreads();
  cta_gemm(a, n, n, -1.0, L, SymL{f.F, J}, 1.0, Dn{f.T1 + n, J}, false);
  // U' = Yh_AA - K_AN L^T - L Yh_AN^T   (lower)
  cta_gemm(a, a, n, -1.0, Dn{f.T1 + n, J}, CscT{W, J, n}, 1.0, Dn{f.F + n + (int64_t)n * J, J}, true);
  cta_gemm(a, a, n, -1.0, L, DnT{f.F + n, J}, 1.0, Dn{f.F + n + (int64_t)n * J, J}, true);
  // M_NN = D^{-1} (K_NN D^{-1})
  CscSym Dinv{W, J};
  cta_gemm(n, n, n, 1.0, SymL{f.F, J}, Dinv, 0.0, Dn{f.T2, J}, false);
  cta_gemm(n, n, n, 1.0, Dinv, Dn{f.T2, J}, 0.0, Csc{T + f.base, J, 0}, true);
  // M_AN = V (K_AN D^{-1})
  cta_gemm(a, n, n, 1.0, Dn{f.T1 + n, J}, Dinv, 0.0, Dn{f.T2 + n, J}, false);
  cta_gemm(a, n, a, 1.0, SymL{Vd + S.v_off[k], a}, Dn{f.T2 + n, J}, 0.0, Csc{T + f.base, J, n}, false);
}

// Hessian factor (§5.4, block form).  Step 2 of Algorithm 5.1 maps K to
// M = (D^{-1} K_NN D^{-1}, V K_AN D^{-1}).  With D = C C^T (C the lower
// Cholesky factor of the factor's D_NN) and V = Q Q^T (Q upper triangular,
// the factor §5.4 prescribes), W = R(Y) ends with W_NN = C^{-1} K_NN C^{-T},
// W_AN = Q^T K_AN C^{-T}: for a supernode this equals the per-column
// formulas of Algorithm 5.3, since C = L_NN D_NN^{1/2} in terms of the
// scalar factors and the R_j of the columns of N_k are trailing blocks of
// the upper factor of S_{J_k J_k}.  In terms of M: W_NN = C^T M_NN C,
// W_AN = Q^{-1} M_AN C; and R^adj starts with M_NN = C^{-T} W_NN C^{-1},
// M_AN = Q W_AN C^{-1}.  Q is held as Q' = P Q P (lower, P the order
// reversal), applied to the A-rows in reverse order.  dir = 0: M -> W,
// 1: W -> M, in place on the front's N-part of `Z` (one right-hand side).
__device__ void rtrans_front(const SymDev& S, int k, int dir, const double* Lc, const double* Qd, double* Z,
                             double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  const double* Q = Qd + S.v_off[k];
  double* C = f.T2;  // n x n, ld J, lower: C from the factor
  double* B = f.T1;  // J x n, ld J: the N-part of Z (NN block full, A-rows reversed for dir 1)
  for (int e = threadIdx.x; e < n * n; e += NT) {
    const int r = e % n, c = e / n;
    C[r + (int64_t)c * J] = r >= c ? Lc[f.base + csc_off(J, r, c)] : 0.0;
  }
  for (int e = threadIdx.x; e < J * n; e += NT) {
    const int r = e % J, c = e / J;
    const int rb = (dir == 1 && r >= n) ? n + a - 1 - (r - n) : r;
    B[rb + (int64_t)c * J] = Z[f.base + (r >= c ? csc_off(J, r, c) : csc_off(J, c, r))];
  }
  __syncthreads();
  if (dir == 0) {
    // W_NN = C^T (M_NN C);  W_AN = Q^{-1} (M_AN C) = P Q'^{-1} P (M_AN C)
    cta_gemm(n, n, n, 1.0, Dn{B, J}, TriL{C, J}, 0.0, Dn{f.F, J}, false);
    cta_gemm(n, n, n, 1.0, TriLT{C, J}, Dn{f.F, J}, 0.0, Csc{Z + f.base, J, 0}, true);
    if (a > 0) {
      cta_gemm(a, n, n, 1.0, Dn{B + n, J}, TriL{C, J}, 0.0, DnRev{f.F + n, J, a}, false);
      cta_trsm_rLT(n, a, DnTW{f.F + n, J}, Q, a);
      for (int e = threadIdx.x; e < a * n; e += NT) {
        const int r = e % a, c = e / a;
        Z[f.base + csc_off(J, n + r, c)] = f.F[(n + a - 1 - r) + (int64_t)c * J];
      }
    }
  } else {
    // M_NN = C^{-T} (W_NN C^{-1});  M_AN = Q (W_AN C^{-1}) = P Q' P (W_AN C^{-1})
    cta_trsm_rL(J, n, Dn{B, J}, C, J);
    cta_trsm_rL(n, n, DnTW{B, J}, C, J);
    for (int e = threadIdx.x; e < n * n; e += NT) {
      const int r = e % n, c = e / n;
      if (r >= c) Z[f.base + csc_off(J, r, c)] = B[r + (int64_t)c * J];
    }
    if (a > 0)
      cta_gemm(a, n, a, 1.0, TriL{Q, a}, Dn{B + n, J}, 0.0, CscRev{Z + f.base, J, n, a}, false);
  }
  __syncthreads();
}

// Algorithm 5.1 step 3 (block form): V' gathered from the parent,
// T_AN = M_AN - V' L, T_NN = M_NN - M_AN^T L - L^T T_AN.
__device__ void hess_down_front(const SymDev& S, int k, const double* Wc, double* T, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_from_parent(S, f, ws);
  csc_to_front(f.F, J, n, T + f.base);
  __syncthreads();
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  // T1[n:J] = V' L
  cta_gemm(a, n, a, 1.0, SymL{f.F + n + (int64_t)n * J, J}, L, 0.0, Dn{f.T1 + n, J}, false);
  // Q = M_AN - 1/2 V'L ; T_NN = M_NN - (Q^T L + L^T Q) ; T_AN = Q - 1/2 V'L
  for (int e = threadIdx.x; e < a * n; e += NT) {
    int r = n + e % a, c = e / a;
    f.F[r + (int64_t)c * J] -= 0.5 * f.T1[r + (int64_t)c * J];
  }
  __syncthreads();
  cta_gemm(n, n, a, -1.0, DnT{f.F + n, J}, L, 1.0, Dn{f.F, J}, true);
  cta_gemm(n, n, a, -1.0, CscT{W, J, n}, Dn{f.F + n, J}, 1.0, Dn{f.F, J}, true);
  for (int e = threadIdx.x; e < a * n; e += NT) {
    int r = n + e % a, c = e / a;
    f.F[r + (int64_t)c * J] -= 0.5 * f.T1[r + (int64_t)c * J];
  }
  __syncthreads();
  front_to_csc(T + f.base, f.F, J, n, 1.0);
  __syncthreads();
}

// Algorithm 5.2 steps 1-2 (block form), top-down:
// M_AN = T_AN + V' L, M_NN = T_NN + T_AN^T L + L^T M_AN,
// K_NN = D M_NN D, K_AN = V^{-1} M_AN D.  K is written to the output array.
__device__ void ihess_down_front(const SymDev& S, int k, const double* Wc, const double* Dd,
                                 const double* Rd, const double* Tin, double* Yout, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  gather_from_parent(S, f, ws);
  csc_to_front(f.F, J, n, Tin + f.base);
  __syncthreads();
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  // T1[n:J] = M_AN = T_AN + V' L
  copy_rect(f.T1 + n, J, f.F + n, J, a, n);
  __syncthreads();
  cta_gemm(a, n, a, 1.0, SymL{f.F + n + (int64_t)n * J, J}, L, 1.0, Dn{f.T1 + n, J}, false);
  // T1[0:n] = M_NN = T_NN + T_AN^T L + L^T M_AN   (full square)
  for (int e = threadIdx.x; e < n * n; e += NT) {
    int r = e % n, c = e / n;
    f.T1[r + (int64_t)c * J] = r >= c ? f.F[r + (int64_t)c * J] : f.F[c + (int64_t)r * J];
  }
  __syncthreads();
  cta_gemm(n, n, a, 1.0, DnT{f.F + n, J}, L, 1.0, Dn{f.T1, J}, false);
  cta_gemm(n, n, a, 1.0, CscT{W, J, n}, Dn{f.T1 + n, J}, 1.0, Dn{f.T1, J}, false);
  // K_NN = D (M_NN D)
  const double* D = Dd + S.d_off[k];
  cta_gemm(n, n, n, 1.0, Dn{f.T1, J}, SymL{D, n}, 0.0, Dn{f.T2, J}, false);
  cta_gemm(n, n, n, 1.0, SymL{D, n}, Dn{f.T2, J}, 0.0, Csc{Yout + f.base, J, 0}, true);
  // K_AN = V^{-1} (M_AN D), with V^{-1} cached per factor
  if (a > 0) {
    cta_gemm(a, n, n, 1.0, Dn{f.T1 + n, J}, SymL{D, n}, 0.0, Dn{f.T2 + n, J}, false);
    cta_gemm(a, n, a, 1.0, SymL{Rd + S.v_off[k], a}, Dn{f.T2 + n, J}, 0.0, Csc{Yout + f.base, J, n}, false);
  }
  __syncthreads();
}

// Algorithm 5.2 step 3 (block form), bottom-up:
// Z = sum of children's extend-add, Y_NN = K_NN - Z_NN,
// Y_AN = L K_NN + K_AN - Z_AN, U' = Z_AA - (L K_NN L^T + K_AN L^T + L K_AN^T).
__device__ void ihess_up_front(const SymDev& S, int k, const double* Wc, double* Y, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  zero_lower(f.F, J, J, 0);
  __syncthreads();
  extend_add_children(S, f, ws, 1.0);
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  CscSym Kn{Y + f.base, J};
  // T2[n:J] = P = K_AN + 1/2 L K_NN
  for (int e = threadIdx.x; e < a * n; e += NT) {
    int r = e % a, c = e / a;
    f.T2[n + r + (int64_t)c * J] = Y[f.base + csc_off(J, n + r, c)];
  }
  __syncthreads();
  cta_gemm(a, n, n, 0.5, L, Kn, 1.0, Dn{f.T2 + n, J}, false);
  // U' = Z_AA - (P L^T + L P^T)
  cta_gemm(a, a, n, -1.0, Dn{f.T2 + n, J}, CscT{W, J, n}, 1.0, Dn{f.F + n + (int64_t)n * J, J}, true);
  cta_gemm(a, a, n, -1.0, L, DnT{f.T2 + n, J}, 1.0, Dn{f.F + n + (int64_t)n * J, J}, true);
  // Y_AN = K_AN + L K_NN - Z_AN = 2P - K_AN - Z_AN ;  Y_NN = K_NN - Z_NN
  for (int e = threadIdx.x; e < a * n; e += NT) {
    int r = e % a, c = e / a;
    int64_t o = f.base + csc_off(J, n + r, c);
    double kan = Y[o];
    Y[o] = 2.0 * f.T2[n + r + (int64_t)c * J] - kan - f.F[n + r + (int64_t)c * J];
  }
  for (int e = threadIdx.x; e < n * n; e += NT) {
    int r = e % n, c = e / n;
    if (r >= c) {
      int64_t o = f.base + csc_off(J, r, c);
      Y[o] = Y[o] - f.F[r + (int64_t)c * J];
    }
  }
  __syncthreads();
}

// rows r and R-1-r of the R x C block B (ld) exchanged, CTA-wide
__device__ void reverse_rows(double* B, int64_t ld, int R, int C) {
  __syncthreads();
  const int h = R / 2;
  for (int e = threadIdx.x; e < h * C; e += NT) {
    const int r = e % h, c = e / h;
    double* x = B + r + (int64_t)c * ld;
    double* y = B + (R - 1 - r) + (int64_t)c * ld;
    const double t = *x;
    *x = *y;
    *y = t;
  }
  __syncthreads();
}

// Algorithm 7.3 for one front (each front needs only S and V_k = S_AA):
// R = chol(V), Z = R^{-1} S_AN, P = S_NN - Z^T Z = D_NN^{-1},
// L_AN = -R^{-T} Z, D_NN = P^{-1}, C = chol(D_NN), B = L_AN C.
// S-front of front k: S_NN and S_AN from the input's columns N_k, and
// V_k = S_{A_k A_k}, a submatrix of the input, read from its later columns
// (Eq. (e-sn-compl-2) re-extracts exactly these entries from the parent's
// S-front; reading them from S makes the fronts independent).
__device__ void complete_load_front(const SymDev& S, int k, const double* Sin, double* ws) {
  FrontInfo f = front_info(S, k, ws);
  const int32_t* A = S.rows + S.rows_ptr[k] + f.n;
  for (int e = threadIdx.x; e < f.a * f.a; e += NT) {
    const int r = e % f.a, c = e / f.a;
    if (r >= c) f.F[(f.n + r) + (int64_t)(f.n + c) * f.J] = Sin[csc_find(S, __ldg(A + r), __ldg(A + c))];
  }
  csc_to_front(f.F, f.J, f.n, Sin + f.base);
  __syncthreads();
}

// Algorithm 7.3 arithmetic for one front whose S-front is loaded.  With Gq
// (completion with factored update matrices), G = P R_k P of V_k = R_k R_k^T
// is read from Gq instead of factoring V_k: the solves then run on S_AN and
// L_AN with their rows in reversed order (Z^T Z is unchanged).
__device__ void complete_front(const SymDev& S, int k, const double* Sin, double* Lc, double* Wc,
                               double* Dd, double* Vd, double* Rd, const double* Gq, double* ws, double* ldet,
                               int64_t* st) {
  FrontInfo f = front_info(S, k, ws);
  const int J = f.J, n = f.n, a = f.a;
  double* V = Vd + S.v_off[k];
  double* R = Gq ? const_cast<double*>(Gq) + S.v_off[k] : Rd + S.v_off[k];
  copy_lower(V, a, f.F + n + (int64_t)n * J, J, a);
  if (!Gq) copy_lower(R, a, f.F + n + (int64_t)n * J, J, a);
  __syncthreads();
  if (a > 0 && !Gq) cta_potrf_partial(R, a, a, a, st, CHD_ERR_NOT_COMPLETABLE, k, -1);
  // T1[n:J] = Z = R^{-1} S_AN
  copy_rect(f.T1 + n, J, f.F + n, J, a, n);
  __syncthreads();
  if (Gq) reverse_rows(f.T1 + n, J, a, n);
  if (a > 0) cta_trsm_rLT(n, a, DnTW{f.T1 + n, J}, R, a);
  // T1[0:n] (lower) = P = S_NN - Z^T Z
  copy_lower(f.T1, J, f.F, J, n);
  __syncthreads();
  cta_gemm(n, n, a, -1.0, DnT{f.T1 + n, J}, Dn{f.T1 + n, J}, 1.0, Dn{f.T1, J}, true);
  // T2[n:J] = L_AN = -R^{-T} Z
  for (int e = threadIdx.x; e < a * n; e += NT) {
    int r = n + e % a, c = e / a;
    f.T2[r + (int64_t)c * J] = -f.T1[r + (int64_t)c * J];
  }
  __syncthreads();
  if (a > 0) cta_trsm_rL(n, a, DnTW{f.T2 + n, J}, R, a);
  if (Gq) reverse_rows(f.T2 + n, J, a, n);
  // Wc = [P; L_AN]
  for (int e = threadIdx.x; e < J * n; e += NT) {
    int r = e % J, c = e / J;
    if (r >= c) Wc[f.base + csc_off(J, r, c)] = (r < n) ? f.T1[r + (int64_t)c * J] : f.T2[r + (int64_t)c * J];
  }
  // T2[0:n] = chol(P) = Q ; D = P^{-1} = Q^{-T} Q^{-1}
  copy_lower(f.T2, J, f.T1, J, n);
  __syncthreads();
  cta_potrf_partial(f.T2, J, n, n, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0);
  double* Dk = Dd + S.d_off[k];
  set_identity(Dk, n, n);
  __syncthreads();
  cta_trsm_rLT(n, n, DnTW{Dk, n}, f.T2, J);  // Dk = Q^{-1}
  cta_gemm(n, n, n, 1.0, TriLT{Dk, n}, TriL{Dk, n}, 0.0, Dn{f.T1, J}, true);  // T1 = D (lower)
  copy_lower(Dk, n, f.T1, J, n);
  __syncthreads();
  // C = chol(D) in T1[0:n]; B = L_AN C
  cta_potrf_partial(f.T1, J, n, n, st, CHD_ERR_NOT_COMPLETABLE, k, f.col0);
  for (int e = threadIdx.x; e < n * n; e += NT) {
    int r = e % n, c = e / n;
    if (r >= c) Lc[f.base + csc_off(J, r, c)] = f.T1[r + (int64_t)c * J];
  }
  cta_gemm(a, n, n, 1.0, Dn{f.T2 + n, J}, TriL{f.T1, J}, 0.0, Csc{Lc + f.base, J, n}, false);
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += 2.0 * log(f.T1[i + (int64_t)i * J]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) ldet[k] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// kernels: blockIdx.x = task within the launch, blockIdx.y = right-hand side
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_factor(SymDev S, int task0, const double* X, double* Lc,
                                               double* Wc, double* Dd, double* ws, double* ldet,
                                               int64_t* st) {
  const int t = task0 + blockIdx.x;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q)
    factor_front(S, S.task_fronts[q], X, Lc, Wc, Dd, ws, ldet, st);
}
__global__ void __launch_bounds__(NT) k_product(SymDev S, int task0, const double* Lc, double* X, double* ws) {
  const int t = task0 + blockIdx.x;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q) product_front(S, S.task_fronts[q], Lc, X, ws);
}
__global__ void __launch_bounds__(NT) k_gradient(SymDev S, int task0, const double* Wc, double* Sc,
                                                 double* g, double* Vd, double* ws) {
  const int t = task0 + blockIdx.x;
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    gradient_front(S, S.task_fronts[q], Wc, Sc, g, Vd, ws);
}
__global__ void __launch_bounds__(NT) k_hess_up(SymDev S, int task0, const double* Wc,
                                                const double* Vd, const double* Y, int64_t ldy,
                                                double* T, int64_t ldt, double* ws) {
  const int t = task0 + blockIdx.x;
  const int64_t y = blockIdx.y;
  const uint8_t* act = S.act ? S.act + y * S.nsn : nullptr;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q) {
    const int k = S.task_fronts[q];
    if (act && !act[k]) continue;  // pruned (§5.5): K, U' and M are zero here
    hess_up_front(S, k, Wc, Vd, Y + y * ldy, T + y * ldt, ws + y * S.f_total, act);
  }
}
__global__ void __launch_bounds__(NT) k_hess_down(SymDev S, int task0, const double* Wc, double* T,
                                                  int64_t ldt, double* ws) {
  const int t = task0 + blockIdx.x;
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    hess_down_front(S, S.task_fronts[q], Wc, T + y * ldt, ws + y * S.f_total);
}
__global__ void __launch_bounds__(NT) k_ihess_down(SymDev S, int task0, const double* Wc,
                                                   const double* Dd, const double* Rd,
                                                   const double* Tin, int64_t ldt, double* Y,
                                                   int64_t ldy, double* ws) {
  const int t = task0 + blockIdx.x;
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t + 1] - 1; q >= S.task_ptr[t]; --q)
    ihess_down_front(S, S.task_fronts[q], Wc, Dd, Rd, Tin + y * ldt, Y + y * ldy, ws + y * S.f_total);
}
__global__ void __launch_bounds__(NT) k_ihess_up(SymDev S, int task0, const double* Wc, double* Y,
                                                 int64_t ldy, double* ws) {
  const int t = task0 + blockIdx.x;
  const int64_t y = blockIdx.y;
  for (int q = S.task_ptr[t]; q < S.task_ptr[t + 1]; ++q)
    ihess_up_front(S, S.task_fronts[q], Wc, Y + y * ldy, ws + y * S.f_total);
}
// M <-> W of every front of the warp and CTA tiers, one CTA per (front, RHS)
__global__ void __launch_bounds__(NT) k_rtrans(SymDev S, int dir, const double* Lc, const double* Qd, double* Z,
                                               int64_t ldz, double* ws) {
  const int64_t y = blockIdx.y;
  const int k = S.plain_fronts[blockIdx.x];
  if (S.act && !S.act[y * S.nsn + k]) return;  // pruned: M = W = 0 here
  rtrans_front(S, k, dir, Lc, Qd, Z + y * ldz, ws + y * S.f_total);
}

// Sparse arguments (§5.5): front k of right-hand side y is active when Y has
// a nonzero in the columns of the fronts whose update blocks reach k
// ([sub_lo[k], sub_hi[k]], contiguous in the postorder).  cnt[y][k] first
// flags a nonzero among front k's own values, then holds the prefix sums.
__global__ void __launch_bounds__(NT) k_front_nz(SymDev S, const double* Y, int64_t ldy, int32_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  if (k >= S.nsn) return;
  const int64_t y = blockIdx.y;
  const double* v = Y + y * ldy;
  const int64_t b = S.colptr[S.sn_ptr[k]], e = S.colptr[S.sn_ptr[k + 1]];
  bool nz = false;
  for (int64_t i = b + lane; i < e && !nz; i += 32) nz = v[i] != 0.0;
  nz = __any_sync(0xffffffffu, nz);
  if (lane == 0) cnt[y * S.nsn + k] = nz ? 1 : 0;
}
constexpr int kScanT = 1024;
__global__ void __launch_bounds__(kScanT) k_active(SymDev S, int32_t* cnt, uint8_t* act) {
  __shared__ int32_t wsum[kScanT / 32];
  const int64_t y = blockIdx.x;
  int32_t* c = cnt + y * S.nsn;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t carry = 0;
  for (int64_t k0 = 0; k0 < S.nsn; k0 += kScanT) {
    const int64_t k = k0 + threadIdx.x;
    int32_t v = k < S.nsn ? c[k] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      int32_t x = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    v += carry + (w > 0 ? wsum[w - 1] : 0);
    if (k < S.nsn) c[k] = v;
    carry += wsum[kScanT / 32 - 1];
    __syncthreads();
  }
  for (int64_t k = threadIdx.x; k < S.nsn; k += kScanT) {
    const int32_t lo = S.sub_lo[k], hi = S.sub_hi[k];
    act[y * S.nsn + k] = (c[hi] - (lo > 0 ? c[lo - 1] : 0)) > 0 ? 1 : 0;
  }
}
// all CTA-tier fronts at once, one CTA each
__global__ void __launch_bounds__(NT) k_complete(SymDev S, const double* Sin, double* Lc, double* Wc, double* Dd,
                                                 double* Vd, double* Rd, const double* Gq, double* ws, double* ldet,
                                                 int64_t* st) {
  const int k = S.cta_fronts[blockIdx.x];
  complete_load_front(S, k, Sin, ws);
  complete_front(S, k, Sin, Lc, Wc, Dd, Vd, Rd, Gq, ws, ldet, st);
}
// Completion with factored update matrices, one level of the clique tree
// (parents done): G_k = P R_k P of every front of fc_fronts[first ..], one
// CTA each (fc_body.cuh): gather, Householder reduction of the rows kept
// from G_parent, then M = S~ L^{-T} and G~ = chol(A~ - M M^T).
__global__ void __launch_bounds__(NT) k_fc(SymDev S, int first, const double* Sin, double* Gq, double* fcs,
                                           int64_t* st) {
  const int k = S.fc_fronts[first + blockIdx.x];
  const fc::Info f = fc::info(S, k);
  double* G = Gq + S.v_off[k];
  double* X = fcs + S.fc_off[k];
  const double* Gp = Gq + S.v_off[f.p];
  const int ap = f.Jp - f.np;
  const int64_t tot = fc::gather_count(f);
  for (int64_t e = threadIdx.x; e < tot; e += NT) fc::gather_one(f, e, Sin, Gp, ap, X, G);
  __syncthreads();
  if (f.q > 0) fc::reduce(f, X, G, st);
  const int pp = f.a - f.q;
  if (pp > 0) {
    double* M = G + f.q;
    double* At = G + f.q + (int64_t)f.q * f.a;
    if (f.q > 0) {
      cta_trsm_rLT(pp, f.q, Dn{M, f.a}, G, f.a);
      __syncthreads();
      cta_gemm(pp, pp, f.q, -1.0, Dn{M, f.a}, DnT{M, f.a}, 1.0, Dn{At, f.a}, true);
      __syncthreads();
    }
    cta_potrf_partial(At, f.a, pp, pp, st, CHD_ERR_NOT_COMPLETABLE, k, -1);
  }
}
// Inverses of the cached V_k (inverse Hessian step 2), one CTA per front of
// `front_list` (no dependencies between fronts; big fronts use the dense
// tier): R = chol(V), R^{-1} in the front's workspace, V^{-1} = R^{-T} R^{-1}.
// what & 1: V_k^{-1} into Rd (inverse Hessian); what & 2: chol(P V_k P) into
// Qd (Hessian factor)
__global__ void __launch_bounds__(NT) k_inv_v(SymDev S, const double* Vd, double* Rd, double* Qd, double* ws,
                                              int64_t* st, const int32_t* front_list, int what) {
  const int k = front_list[blockIdx.x];
  const int n = (int)(S.sn_ptr[k + 1] - S.sn_ptr[k]);
  const int a = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]) - n;
  if (a == 0 || a >= kInvVMulti) return;  // large V_k: multi-CTA kernels (big_inv_v)
  double* R = Rd + S.v_off[k];
  double* Ri = ws + S.f_off[k];  // a x a scratch inside the front's J x J region
  const double* V = Vd + S.v_off[k];
  // Hessian factor (§5.4): V = Q Q^T with Q upper triangular, kept as
  // Q' = chol(P V P) = P Q P, P the order reversal
  if (what & 2) {
    double* Qk = Qd + S.v_off[k];
    for (int e = threadIdx.x; e < a * a; e += NT) {
      const int r = e % a, c = e / a;
      if (r >= c) Qk[r + (int64_t)c * a] = V[(a - 1 - c) + (int64_t)(a - 1 - r) * a];
    }
    __syncthreads();
    cta_potrf_partial(Qk, a, a, a, st, CHD_ERR_NOT_PD, k, -1);
  }
  if (what & 1) {
    copy_lower(R, a, V, a, a);
    set_identity(Ri, a, a);
    __syncthreads();
    cta_potrf_partial(R, a, a, a, st, CHD_ERR_NOT_PD, k, -1);
    cta_trsm_rLT(a, a, DnTW{Ri, a}, R, a);  // Ri = R^{-1}
    cta_gemm(a, a, a, 1.0, TriLT{Ri, a}, TriL{Ri, a}, 0.0, Dn{R, a}, true);
  }
}
// Deterministic sum of the per-front log det contributions.
__global__ void k_sum(const double* v, int64_t m, double* out) {
  __shared__ double red[NT];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += NT) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
// Schur complement H_ij = A_i . T_j (T_j = H(A_j)) in the trace inner product
// (§5.5): partial sums over chunks of the value arrays, CTA (chunk, pair):
// 2 sum_e a_i[e] t_j[e] minus the diagonal entries (at colptr[c]) once.
constexpr int64_t kSchurChunk = 65536;
__global__ void __launch_bounds__(NT) k_schur_partial(int m, const double* A, int64_t lda, const double* T,
                                                      int64_t ldt, int64_t nnz, const int64_t* colptr, int64_t n,
                                                      double* partial) {
  __shared__ double red[NT];
  const int64_t chunk = blockIdx.y;
  const int pair = blockIdx.x, i = pair % m, j = pair / m;
  const double* a = A + i * lda;
  const double* t = T + j * ldt;
  const int64_t e0 = chunk * kSchurChunk;
  double s = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < min(nnz, e0 + kSchurChunk); e += NT) s = fma(2.0 * a[e], t[e], s);
  for (int64_t c = e0 + threadIdx.x; c < min(n, e0 + kSchurChunk); c += NT) {
    const int64_t d = colptr[c];
    s = fma(-a[d], t[d], s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)pair * gridDim.y + chunk] = red[0];
}
// sum of the chunk partials in chunk order, H column-major (ld m)
__global__ void k_schur_sum(int m, int64_t nchunk, const double* partial, double* H) {
  const int pair = blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= m * m) return;
  double s = 0.0;
  for (int64_t c = 0; c < nchunk; ++c) s += partial[(int64_t)pair * nchunk + c];
  H[pair] = s;
}
// Deterministic sums of v over the segments [seg[i], seg[i+1]), one CTA each.
__global__ void k_segsum(const double* v, const int64_t* seg, double* out) {
  __shared__ double red[NT];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int64_t q = seg[i] + threadIdx.x; q < seg[i + 1]; q += NT) s += v[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}
// Unique scalar L D L^T from the supernodal Cholesky factor G = [C; B]:
// L = G diag(1/G_ii), D_ii = G_ii^2.
__global__ void k_export(SymDev S, const double* Lc, double* l, double* d) {
  const int k = blockIdx.x;
  const int64_t col0 = S.sn_ptr[k];
  const int n = (int)(S.sn_ptr[k + 1] - col0);
  const int J = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  const int64_t base = S.colptr[col0];
  for (int e = threadIdx.x; e < J * n; e += NT) {
    int r = e % J, c = e / J;
    if (r >= c) {
      double gcc = Lc[base + csc_off(J, c, c)];
      l[base + csc_off(J, r, c)] = (r == c) ? 1.0 : Lc[base + csc_off(J, r, c)] / gcc;
      if (r == c && d) d[col0 + c] = gcc * gcc;
    }
  }
}

// FP64 throughput probe: 8 independent DFMA chains per thread.
__global__ void __launch_bounds__(NT) k_dfma_probe(double* out, int iters, double s) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], s, 1e-9);
  }
  double r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r += a[i];
  out[blockIdx.x * NT + threadIdx.x] = r;
}

}  // namespace chd

// ---------------------------------------------------------------------------
// host launchers (called from capi.cpp)
// ---------------------------------------------------------------------------
namespace chd_launch {
using namespace chd;

static int64_t g_launches = 0;
static int64_t g_split_k = 0;
static double g_tc_flops = 0.0;
int64_t launches() { return g_launches; }
double tc_flops() { return g_tc_flops; }
void count_tc_flops(double f) { g_tc_flops += f; }
void count_launch() { ++g_launches; }
int64_t split_k_launches() { return g_split_k; }
void count_split_k() { ++g_split_k; }
void add_launches(int64_t d) { g_launches += d; }

static inline void count() { ++g_launches; }

// dense-tier sequences (bigfront.cu); xs/xcap: split-K scratch (may be null)
void big_factor(const chd_symbolic* s, const Slot& sl, int k, const double* X,
                double* Lc, double* Wc, double* Dd, double* ws, double* ldet, int64_t* status);
void big_product(const chd_symbolic* s, const Slot& sl, int k, const double* Lc,
                 double* X, double* ws);
void big_gradient(const chd_symbolic* s, const Slot& sl, int k, const double* Wc,
                  double* Sc, double* g, double* Vd, double* ws);
void big_hess_up(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                 const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                 const uint8_t* act);
void big_hess_down(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                   double* T, int64_t ldt, double* ws);
void big_ihess_down(const chd_symbolic* s, const Slot& sl, int m, int k,
                    const double* Wc, const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y,
                    int64_t ldy, double* ws);
void big_ihess_up(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                  double* Y, int64_t ldy, double* ws);
void big_complete(const chd_symbolic* s, const Slot& sl, int k, const double* Sin,
                  double* Lc, double* Wc, double* Dd, double* Vd, double* Rd, const double* Gq, double* ws,
                  double* ldet, int64_t* status);

// chain-tier launches (chain_tier.cu): runs of one-column band fronts
void chain_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                  double* Dd, double* ws, double* ldet, int64_t* status);
void chain_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc, double* g,
                    double* Vd, double* ws);
void chain_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, const double* Vd,
                   const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws, const uint8_t* act);
void chain_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                     int64_t ldt, double* ws);
void chain_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                      const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                      double* ws);
void chain_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                    int64_t ldy, double* ws);

// warp-tier launches (warp_tier.cu): w32 for |J| <= 32, w64 for |J| <= 64
namespace w32 {
void warp_product(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Lc, double* X, double* ws);
void warp_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                 double* Dd, double* ws, double* ldet, int64_t* status);
void warp_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc,
                   double* g, double* Vd, double* ws);
void warp_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                  const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                  const uint8_t* act);
void warp_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws);
void warp_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                     const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                     double* ws);
void warp_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                   int64_t ldy, double* ws);
void warp_complete_all(const chd_symbolic* s, cudaStream_t st, const double* Sin, double* Lc, double* Wc,
                       double* Dd, double* Vd, double* Rd, const double* Gq, double* ldet, int64_t* status);
}  // namespace w32
namespace w64 {
void warp_product(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Lc, double* X, double* ws);
void warp_factor(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* X, double* Lc, double* Wc,
                 double* Dd, double* ws, double* ldet, int64_t* status);
void warp_gradient(const chd_symbolic* s, cudaStream_t st, int t0, int nt, const double* Wc, double* Sc,
                   double* g, double* Vd, double* ws);
void warp_hess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                  const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                  const uint8_t* act);
void warp_hess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws);
void warp_ihess_down(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc,
                     const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                     double* ws);
void warp_ihess_up(const chd_symbolic* s, cudaStream_t st, int t0, int nt, int m, const double* Wc, double* Y,
                   int64_t ldy, double* ws);
}  // namespace w64


// Runs body(i, stream, scratch, cap) for the `count` independent big fronts
// of one level: on the caller's stream if there is one front or no side
// streams, else round-robin over the side streams, forked after the work
// already queued on `st` and joined back into `st` at `join_now` (the caller
// may queue independent work on `st` in between).
struct BigFork {
  const Exec* ex;
  cudaStream_t st;
  int used = 0;
  template <class Body>
  void run(int count, Body&& body) {
    if (count <= 0) return;
    auto slot = [&](int j, cudaStream_t bs) {
      Slot sl;
      sl.st = bs;
      if (ex) {
        sl.xs = ex->slice[j];
        sl.xcap = ex->slice_cap[j];
        sl.tc = ex->tc[j];
        sl.tc_cap = ex->tc_cap[j];
        sl.status = ex->status;
        sl.tc_mode = ex->tc_mode;
      }
      return sl;
    };
    if (!ex || ex->nside == 0 || count == 1) {
      const Slot sl = slot(0, st);
      for (int i = 0; i < count; ++i) body(i, sl);
      return;
    }
    used = std::min(count, ex->nside);
    cudaEventRecord(ex->fork, st);
    for (int j = 0; j < used; ++j) cudaStreamWaitEvent(ex->side[j], ex->fork, 0);
    for (int i = 0; i < count; ++i) {
      const int j = i % used;
      body(i, slot(1 + j, ex->side[j]));
    }
  }
  void join_now() {
    for (int j = 0; j < used; ++j) {
      cudaEventRecord(ex->join[j], ex->side[j]);
      cudaStreamWaitEvent(st, ex->join[j], 0);
    }
    used = 0;
  }
};

// Level l holds tasks [t0, t0 + nwarp) of the warp tier (|J| <= 32), then
// [tw, tw + nw64) of the wide warp tier (|J| <= 64), then [tc, tc + ncta) of
// the CTA tier, then nbig single big fronts of the dense tier.
struct Level {
  int tr, nr32, nr64;  // chain runs: [tr, tr + nr32) |J| <= 32, then nr64 with |J| <= 64
  int t0, nwarp, tw, nw64, tc, ncta, nbig;
};
static inline Level level(const chd_symbolic* s, int l) {
  Level v;
  v.tr = s->lvl_ptr[l];
  v.nr32 = s->lvl_r32.empty() ? 0 : s->lvl_r32[l];
  v.nr64 = s->lvl_r64.empty() ? 0 : s->lvl_r64[l];
  v.t0 = v.tr + v.nr32 + v.nr64;
  const int nt = s->lvl_ptr[l + 1] - v.t0;
  v.nwarp = s->lvl_warp[l];
  v.nw64 = s->lvl_w64[l];
  v.nbig = s->lvl_big[l];
  v.tw = v.t0 + v.nwarp;
  v.tc = v.tw + v.nw64;
  v.ncta = nt - v.nwarp - v.nw64 - v.nbig;
  return v;
}
static inline int big_front(const chd_symbolic* s, const Level& v, int i) {
  return s->task_fronts[s->task_ptr[v.tc + v.ncta + i]];
}

void factor(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* X, double* Lc, double* Wc,
            double* Dd, double* ws, double* ldet, int64_t* status) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  for (int l = 0; l < nl; ++l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_factor(s, sl, big_front(s, v, i), X, Lc, Wc, Dd, ws, ldet, status);
    });
    if (v.nr32 + v.nr64) chain_factor(s, st, v.tr, v.nr32 + v.nr64, X, Lc, Wc, Dd, ws, ldet, status);
    if (v.nwarp) w32::warp_factor(s, st, v.t0, v.nwarp, X, Lc, Wc, Dd, ws, ldet, status);
    if (v.nw64) w64::warp_factor(s, st, v.tw, v.nw64, X, Lc, Wc, Dd, ws, ldet, status);
    if (v.ncta) {
      k_factor<<<v.ncta, NT, 0, st>>>(s->dev, v.tc, X, Lc, Wc, Dd, ws, ldet, status);
      count();
    }
    bf.join_now();
  }
}
// Cholesky product X = L D L^T on V (Algorithm 3.2), bottom-up like the factor.
void product(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Lc, double* X, double* ws) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  for (int l = 0; l < nl; ++l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_product(s, sl, big_front(s, v, i), Lc, X, ws);
    });
    if (v.nr32) w32::warp_product(s, st, v.tr, v.nr32, Lc, X, ws);
    if (v.nr64) w64::warp_product(s, st, v.tr + v.nr32, v.nr64, Lc, X, ws);
    if (v.nwarp) w32::warp_product(s, st, v.t0, v.nwarp, Lc, X, ws);
    if (v.nw64) w64::warp_product(s, st, v.tw, v.nw64, Lc, X, ws);
    if (v.ncta) {
      k_product<<<v.ncta, NT, 0, st>>>(s->dev, v.tc, Lc, X, ws);
      count();
    }
    bf.join_now();
  }
}
void gradient(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Wc, double* Sc, double* g,
              double* Vd, double* ws) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  for (int l = nl - 1; l >= 0; --l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_gradient(s, sl, big_front(s, v, i), Wc, Sc, g, Vd, ws);
    });
    if (v.ncta) {
      k_gradient<<<v.ncta, NT, 0, st>>>(s->dev, v.tc, Wc, Sc, g, Vd, ws);
      count();
    }
    if (v.nr32 + v.nr64) chain_gradient(s, st, v.tr, v.nr32 + v.nr64, Wc, Sc, g, Vd, ws);
    if (v.nwarp) w32::warp_gradient(s, st, v.t0, v.nwarp, Wc, Sc, g, Vd, ws);
    if (v.nw64) w64::warp_gradient(s, st, v.tw, v.nw64, Wc, Sc, g, Vd, ws);
    bf.join_now();
  }
}
void hess_up_pass(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, const double* Vd,
                  const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws, const uint8_t* act) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  SymDev D = s->dev;
  D.act = act;
  for (int l = 0; l < nl; ++l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_hess_up(s, sl, m, big_front(s, v, i), Wc, Vd, Y, ldy, T, ldt, ws, act);
    });
    if (v.nr32 + v.nr64) chain_hess_up(s, st, v.tr, v.nr32 + v.nr64, m, Wc, Vd, Y, ldy, T, ldt, ws, act);
    if (v.nwarp) w32::warp_hess_up(s, st, v.t0, v.nwarp, m, Wc, Vd, Y, ldy, T, ldt, ws, act);
    if (v.nw64) w64::warp_hess_up(s, st, v.tw, v.nw64, m, Wc, Vd, Y, ldy, T, ldt, ws, act);
    if (v.ncta) {
      k_hess_up<<<dim3(v.ncta, m), NT, 0, st>>>(D, v.tc, Wc, Vd, Y, ldy, T, ldt, ws);
      count();
    }
    bf.join_now();
  }
}
void hess_down_pass(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  for (int l = nl - 1; l >= 0; --l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_hess_down(s, sl, m, big_front(s, v, i), Wc, T, ldt, ws);
    });
    if (v.ncta) {
      k_hess_down<<<dim3(v.ncta, m), NT, 0, st>>>(s->dev, v.tc, Wc, T, ldt, ws);
      count();
    }
    if (v.nr32 + v.nr64) chain_hess_down(s, st, v.tr, v.nr32 + v.nr64, m, Wc, T, ldt, ws);
    if (v.nwarp) w32::warp_hess_down(s, st, v.t0, v.nwarp, m, Wc, T, ldt, ws);
    if (v.nw64) w64::warp_hess_down(s, st, v.tw, v.nw64, m, Wc, T, ldt, ws);
    bf.join_now();
  }
}
void hessian(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, const double* Vd,
             const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws) {
  hess_up_pass(s, st, ex, m, Wc, Vd, Y, ldy, T, ldt, ws, nullptr);
  hess_down_pass(s, st, ex, m, Wc, T, ldt, ws);
}
// M <-> W for every front (independent fronts): plain fronts in one launch,
// dense fronts and leaf groups on the side streams
void big_rtrans(const chd_symbolic* s, const Slot& sl, int m, int k, int dir,
                const double* Lc, const double* Qd, double* Z, int64_t ldz, double* ws);
// per right-hand side and front: active for the pruned Hessian factor
void prune_mask(const chd_symbolic* s, cudaStream_t st, int m, const double* Y, int64_t ldy, int32_t* cnt,
                uint8_t* act) {
  if (s->nsn == 0 || m == 0) return;
  k_front_nz<<<dim3((unsigned)((s->nsn + NT / 32 - 1) / (NT / 32)), m), NT, 0, st>>>(s->dev, Y, ldy, cnt);
  count();
  k_active<<<m, kScanT, 0, st>>>(s->dev, cnt, act);
  count();
}
void rtrans(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, int dir, const double* Lc,
            const double* Qd, double* Z, int64_t ldz, double* ws, const uint8_t* act) {
  std::vector<int32_t> dense = s->big_fronts;
  for (int64_t g0 : s->grp_first) dense.push_back((int32_t)g0);
  BigFork bf{ex, st};
  bf.run((int)dense.size(), [&](int i, const Slot& sl) {
    big_rtrans(s, sl, m, dense[i], dir, Lc, Qd, Z, ldz, ws);
  });
  if (s->dev.plain_count > 0) {
    SymDev D = s->dev;
    D.act = act;
    k_rtrans<<<dim3((unsigned)s->dev.plain_count, m), NT, 0, st>>>(D, dir, Lc, Qd, Z, ldz, ws);
    count();
  }
  bf.join_now();
}
void inv_hessian(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, const double* Dd,
                 const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy, double* ws) {
  const int nl = (int)s->lvl_ptr.size() - 1;
  for (int l = nl - 1; l >= 0; --l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_ihess_down(s, sl, m, big_front(s, v, i), Wc, Dd, Rd, T, ldt, Y, ldy, ws);
    });
    if (v.ncta) {
      k_ihess_down<<<dim3(v.ncta, m), NT, 0, st>>>(s->dev, v.tc, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
      count();
    }
    if (v.nr32 + v.nr64) chain_ihess_down(s, st, v.tr, v.nr32 + v.nr64, m, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
    if (v.nwarp) w32::warp_ihess_down(s, st, v.t0, v.nwarp, m, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
    if (v.nw64) w64::warp_ihess_down(s, st, v.tw, v.nw64, m, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
    bf.join_now();
  }
  for (int l = 0; l < nl; ++l) {
    Level v = level(s, l);
    BigFork bf{ex, st};
    bf.run(v.nbig, [&](int i, const Slot& sl) {
      big_ihess_up(s, sl, m, big_front(s, v, i), Wc, Y, ldy, ws);
    });
    if (v.nr32 + v.nr64) chain_ihess_up(s, st, v.tr, v.nr32 + v.nr64, m, Wc, Y, ldy, ws);
    if (v.nwarp) w32::warp_ihess_up(s, st, v.t0, v.nwarp, m, Wc, Y, ldy, ws);
    if (v.nw64) w64::warp_ihess_up(s, st, v.tw, v.nw64, m, Wc, Y, ldy, ws);
    if (v.ncta) {
      k_ihess_up<<<dim3(v.ncta, m), NT, 0, st>>>(s->dev, v.tc, Wc, Y, ldy, ws);
      count();
    }
    bf.join_now();
  }
}
// Completion: the arithmetic of Algorithm 7.3 for one front needs only the
// input S (its columns N_k and the submatrix V_k = S_{A_k A_k}), so every
// front is independent: the big fronts run on the side streams, all CTA-tier
// fronts in one launch and all warp-tier fronts in one launch, concurrently.
void big_complete_load(const chd_symbolic* s, cudaStream_t st, int k, const double* Sin, double* ws);
void big_fc(const chd_symbolic* s, const Slot& sl, int k, const double* Sin, double* Gq, double* fcs,
            int64_t* status);
// Algorithm 7.3 over all fronts (independent).  With Gq (chd_opts.completion
// = 1), first the factored update matrices of Algorithm 4.3: G_k = P R_k P
// for every front, level by level from the roots (one launch of k_fc per
// level, dense-tier sequences on the side streams), then the fronts use G_k.
void complete(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Sin, double* Lc, double* Wc,
              double* Dd, double* Vd, double* Rd, double* Gq, double* fcs, double* ws, double* ldet,
              int64_t* status) {
  if (Gq) {
    const int levels = (int)s->fc_lvl.size() - 1;
    for (int l = 0; l < levels; ++l) {
      const int b0 = s->fc_big_lvl[l], b1 = s->fc_big_lvl[l + 1];
      const int c0 = s->fc_lvl[l], c1 = s->fc_lvl[l + 1];
      BigFork bf{ex, st};
      bf.run(b1 - b0, [&](int i, const Slot& sl) { big_fc(s, sl, s->fc_big[b0 + i], Sin, Gq, fcs, status); });
      if (c1 > c0) {
        k_fc<<<c1 - c0, NT, 0, st>>>(s->dev, c0, Sin, Gq, fcs, status);
        count();
      }
      bf.join_now();
    }
  }
  std::vector<int32_t> bigs = s->big_fronts;  // dense fronts and leaf groups
  for (int64_t g0 : s->grp_first) bigs.push_back((int32_t)g0);
  BigFork bf{ex, st};
  bf.run((int)bigs.size(), [&](int i, const Slot& sl) {
    big_complete_load(s, sl.st, bigs[i], Sin, ws);
    big_complete(s, sl, bigs[i], Sin, Lc, Wc, Dd, Vd, Rd, Gq, ws, ldet, status);
  });
  if (s->dev.cta_count > 0) {
    k_complete<<<(int)s->dev.cta_count, NT, 0, st>>>(s->dev, Sin, Lc, Wc, Dd, Vd, Rd, Gq, ws, ldet, status);
    count();
  }
  if (s->dev.warp_count > 0) w32::warp_complete_all(s, st, Sin, Lc, Wc, Dd, Vd, Rd, Gq, ldet, status);
  bf.join_now();
}
void big_inv_v(const chd_symbolic* s, const Slot& sl, int k, const double* Vd,
               double* Rd, double* Qd, double* ws, int64_t* status, int what);
void inv_v(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Vd, double* Rd, double* Qd,
           double* ws, int64_t* status, int what) {
  // dense-tier fronts and the other fronts with a large V_k: multi-CTA
  // kernels on the side streams; the rest: one CTA per front (k_inv_v)
  std::vector<int> bigs;
  for (int64_t k = 0; k < s->nsn; ++k)
    if (s->is_big[k]) bigs.push_back((int)k);
  for (int32_t k : s->small_fronts)
    if (front_J(s, k) - front_n(s, k) >= kInvVMulti) bigs.push_back((int)k);
  BigFork bf{ex, st};
  bf.run((int)bigs.size(), [&](int i, const Slot& sl) {
    big_inv_v(s, sl, bigs[i], Vd, Rd, Qd, ws, status, what);
  });
  if (s->dev.small_count > 0) {
    k_inv_v<<<(int)s->dev.small_count, NT, 0, st>>>(s->dev, Vd, Rd, Qd, ws, status, s->dev.small_fronts, what);
    count();
  }
  bf.join_now();
}
// H (m x m) = [A_i . T_j]; `scratch` holds m*m*ceil(max(nnz, n)/chunk) doubles
int64_t schur_scratch(const chd_symbolic* s, int m) {
  const int64_t len = std::max<int64_t>(s->colptr[s->n], s->n);
  return (int64_t)m * m * ((len + kSchurChunk - 1) / kSchurChunk);
}
void schur(const chd_symbolic* s, cudaStream_t st, int m, const double* A, int64_t lda, const double* T, int64_t ldt,
           double* H, double* scratch) {
  const int64_t nnz = s->colptr[s->n];
  const int64_t nchunk = (std::max<int64_t>(nnz, s->n) + kSchurChunk - 1) / kSchurChunk;
  k_schur_partial<<<dim3((unsigned)(m * m), (unsigned)nchunk), NT, 0, st>>>(m, A, lda, T, ldt, nnz, s->dev.colptr,
                                                                           s->n, scratch);
  count();
  k_schur_sum<<<(m * m + NT - 1) / NT, NT, 0, st>>>(m, nchunk, scratch, H);
  count();
}
void sum(cudaStream_t st, const double* v, int64_t m, double* out) {
  k_sum<<<1, NT, 0, st>>>(v, m, out);
  count();
}
void segsum(cudaStream_t st, const double* v, const int64_t* seg, int nseg, double* out) {
  k_segsum<<<nseg, NT, 0, st>>>(v, seg, out);
  count();
}
void export_ldl(const chd_symbolic* s, cudaStream_t st, const double* Lc, double* l, double* d) {
  k_export<<<(int)s->nsn, NT, 0, st>>>(s->dev, Lc, l, d);
  count();
}
cudaError_t fp64_peak(cudaStream_t st, double* gflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 4, iters = 4000;
  double* buf = nullptr;
  e = cudaMalloc(&buf, (size_t)blocks * NT * sizeof(double));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma_probe<<<blocks, NT, 0, st>>>(buf, 50, 0.999);
  cudaEventRecord(e0, st);
  k_dfma_probe<<<blocks, NT, 0, st>>>(buf, iters, 0.999);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e == cudaSuccess) *gflops = 2.0 * 8 * iters * (double)blocks * NT / (ms * 1e-3) * 1e-9;
  return e;
}
}  // namespace chd_launch
