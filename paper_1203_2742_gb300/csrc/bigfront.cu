// Dense tier: fronts too large for one CTA are processed by a host-issued
// sequence of multi-CTA kernels, each batched over the right-hand sides
// (blockIdx.z).  The per-front formulas are those of kernels.cu (supernodal
// Algorithms 7.1-7.3 and the block forms of Algorithms 5.1 and 5.2); only
// the distribution of the work differs: every dense product is a tiled FP64
// GEMM over the whole GPU, Cholesky factorisations and triangular solves are
// blocked right-looking (panel kernel + trailing GEMM).
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix cones".
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "chd_internal.h"
#include "front_views.cuh"
#include "tc_gemm.cuh"
#include "fc_body.cuh"

namespace chd_launch {
void count_launch();
void count_split_k();
void count_tc_flops(double f);
}

namespace chd {
namespace big {

constexpr int BT = 256;  // threads per CTA
constexpr int GT = 64;   // GEMM output tile
constexpr int GK = 16;   // GEMM k-chunk

template <class V>
__host__ __device__ __forceinline__ V shifted(V v, int64_t off) {
  v.p += off;
  return v;
}

// Launch context of the dense tier: the stream, a scratch buffer for split-K
// partial products and the counter of the Cholesky panel kernel (both may be
// absent: then no split, and panels take two launches).
struct Ctx {
  cudaStream_t s;
  double* xs;
  int64_t cap;  // doubles
  int* ctr;
  void* tc = nullptr;          // tensor-core product scratch (digit planes)
  size_t tc_cap = 0;
  int64_t* status = nullptr;   // the factor's status
  int tc_mode = -1;            // chd_opts.tc_products (-1: FP64 units only)
  operator cudaStream_t() const { return s; }
};
// A stream's scratch slice of xcap doubles: the first xcap - kCtrDoubles hold
// split-K partials, the rest the panel counter (zeroed when allocated).
constexpr int64_t kCtrDoubles = 8;
inline Ctx make_ctx(cudaStream_t s, double* xs, int64_t xcap) {
  if (!xs || xcap <= kCtrDoubles) return Ctx{s, nullptr, 0, nullptr};
  return Ctx{s, xs, xcap - kCtrDoubles, reinterpret_cast<int*>(xs + (xcap - kCtrDoubles))};
}
inline Ctx make_ctx(const Slot& sl) {
  Ctx c = make_ctx(sl.st, sl.xs, sl.xcap);
  c.tc = sl.tc;
  c.tc_cap = sl.tc_cap;
  c.status = sl.status;
  c.tc_mode = sl.tc_mode;
  return c;
}

// ---------------------------------------------------------------------------
// batched tiled GEMM: C = beta*C + alpha*A(MxK)*B(KxN), lower triangle only
// if `lower`.  BM x BN output tiles, TM x TN outputs per thread (256
// threads), k-chunks of up to 16 in shared memory, the k loop runs over the
// real K only.  The tile shape follows the output shape (skinny products do
// not pay for padding).  With nsplit > 1 the CTA (tile, split, batch)
// computes the K range of its split and writes the raw partial tile to
// `part`; mk_gemm_reduce then sums the splits in a fixed order.
// ---------------------------------------------------------------------------
template <int BM, int BN, int TM, int TN, class MA, class MB, class MC>
__global__ void __launch_bounds__(BT) mk_gemm(int M, int N, int K, double alpha, MA A, int64_t sA, MB B,
                                              int64_t sB, double beta, MC C, int64_t sC, int lower, int tiles_n,
                                              int nsplit, double* part) {
  constexpr int HX = BN / TN, HY = BM / TM;
  static_assert(HX * HY == BT, "thread layout");
  const int tile = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  const int tm = (tile / tiles_n) * BM, tn = (tile % tiles_n) * BN;
  if (lower && tn >= tm + BM) return;
  const int64_t z = blockIdx.z;
  A.p += z * sA;
  B.p += z * sB;
  C.p += z * sC;
  __shared__ double As[GK * 128];
  __shared__ double Bs[GK * 128];
  const int tid = threadIdx.x, tx = tid % HX, ty = tid / HX;
  const int kper = ((K + nsplit - 1) / nsplit + GK - 1) / GK * GK;
  const int kbeg = split * kper, kend = min(K, kbeg + kper);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    const int kc = min(GK, kend - k0);
    for (int e = tid; e < BM * kc; e += BT) {
      const int r = e % BM, k = e / BM;
      As[k * BM + r] = (tm + r < M) ? A.at(tm + r, k0 + k) : 0.0;
    }
    for (int e = tid; e < BN * kc; e += BT) {
      const int k = e % kc, c = e / kc;
      Bs[k * BN + c] = (tn + c < N) ? B.at(k0 + k, tn + c) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kc; ++k) {
      double a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k * BM + ty + HY * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[k * BN + tx + HX * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (nsplit > 1) {
    const int tiles = gridDim.x / nsplit;
    double* P = part + (((int64_t)z * nsplit + split) * tiles + tile) * (BM * BN);
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) P[(ty + HY * i) + (tx + HX * j) * BM] = acc[i][j];
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = tm + ty + HY * i, c = tn + tx + HX * j;
      if (r < M && c < N && (!lower || r >= c)) {
        double v = alpha * acc[i][j];
        if (beta != 0.0) v = fma(beta, C.at(r, c), v);
        C.at(r, c) = v;
      }
    }
}

// Sum of the split partial tiles in split order, then C = beta*C + alpha*sum.
template <int BM, int BN, class MC>
__global__ void __launch_bounds__(BT) mk_gemm_reduce(int M, int N, double alpha, double beta, MC C, int64_t sC,
                                                     int lower, int tiles_n, int tiles, int nsplit,
                                                     const double* part) {
  const int tile = blockIdx.x;
  const int tm = (tile / tiles_n) * BM, tn = (tile % tiles_n) * BN;
  if (lower && tn >= tm + BM) return;
  const int64_t z = blockIdx.z;
  C.p += z * sC;
  for (int e = threadIdx.x; e < BM * BN; e += BT) {
    const int lr = e % BM, lc = e / BM;
    const int r = tm + lr, c = tn + lc;
    if (r >= M || c >= N || (lower && r < c)) continue;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(((int64_t)z * nsplit + s) * tiles + tile) * (BM * BN) + e];
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, C.at(r, c), v);
    C.at(r, c) = v;
  }
}

template <int BM, int BN, int TM, int TN, class MA, class MB, class MC>
void gemm_cfg(const Ctx& st, int batch, int M, int N, int K, double alpha, MA A, int64_t sA, MB B, int64_t sB,
              double beta, MC C, int64_t sC, bool lower) {
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const int tiles = tm * tn;
  // split K when the tiles alone cannot fill the GPU and K is long
  int nsplit = 1;
  const int64_t ctas = (int64_t)tiles * batch;
  if (st.xs && ctas < 2 * 152 && K >= 256) {
    nsplit = (int)std::min<int64_t>((2 * 152 + ctas - 1) / ctas, K / 128);
    const int64_t need = (int64_t)batch * tiles * (BM * BN);
    nsplit = (int)std::min<int64_t>(nsplit, need > 0 ? st.cap / need : 1);
    if (nsplit < 2) nsplit = 1;
  }
  mk_gemm<BM, BN, TM, TN><<<dim3(tiles * nsplit, 1, batch), BT, 0, st>>>(
      M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower ? 1 : 0, tn, nsplit, st.xs);
  chd_launch::count_launch();
  if (nsplit > 1) {
    mk_gemm_reduce<BM, BN><<<dim3(tiles, 1, batch), BT, 0, st>>>(M, N, alpha, beta, C, sC, lower ? 1 : 0, tn,
                                                                  tiles, nsplit, st.xs);
    chd_launch::count_launch();
    chd_launch::count_split_k();
  }
}

// Output tiles of a product: the FP64 rate of one SM is low (about 1.6
// lane-FMAs per clock), so a product is worth splitting into smaller tiles
// whenever 64 x 64 tiles would leave SMs idle; split-K (gemm_cfg) covers
// long K on top of that.
inline int64_t tile_count(int M, int N, int bm, int bn, bool lower) {
  const int64_t tm = (M + bm - 1) / bm, tn = (N + bn - 1) / bn;
  return lower && bm == bn && tm == tn ? tm * (tm + 1) / 2 : tm * tn;
}

// Share of the busiest SM's time that does useful work when `units` equal
// tiles are spread over the 152 SMs.
inline double balance(int64_t units) {
  const int64_t per = (units + 151) / 152;
  return per > 0 ? (double)units / (double)(per * 152) : 0.0;
}

// Products large enough for the tensor cores run there (tc_gemm.cuh: FP64
// accuracy from exact bf16 digit products), in as many right-hand sides at
// once as the stream slot's scratch holds; everything else, and every
// product on a slot without tensor-core scratch, runs on the FP64 units.
// Default rule (tc_mode 0): the estimated tensor-core time -- a fixed cost
// for its launches, the digit products (36 bf16 products of each output
// tile), the assembly of every output (mostly integer work, one or two FP64
// operations) and the digit planes' bytes (read twice, written once) --
// below 0.8 of the FP64-unit time of the product (2 M N K flops at about
// 0.9 TFLOP/s).  The model sees one product alone: where many fronts share
// the GPU (many small independent patterns) the FP64 units can be faster,
// and the autotuner then turns the tensor cores off (tc_products = -1).
inline bool tc_worth(const Ctx& st, int batch, int M, int N, int K, bool shared_a, bool shared_b) {
  if (!st.tc || st.tc_mode < 0 || K < 1) return false;
  if (st.tc_mode > 0) return M >= 64 && N >= 16;
  if (M < 16 || K < 16) return false;
  const double Mp = (M + 127) / 128 * 128.0, Np = (N + 31) / 32 * 32.0, Kp = (K + 31) / 32 * 32.0;
  const double fp64 = 2.0 * M * N * static_cast<double>(K) * batch / 0.9e12;
  const double digits = (Mp * (shared_a ? 1 : batch) + Np * (shared_b ? 1 : batch)) * Kp * 32.0 / 4.0e12;
  const double tc = 15e-6 + Mp * Np * Kp * batch * 72.0 / 2.0e15 + Mp * Np * batch * 6.0 / 0.9e12 + digits;
  return tc < 0.8 * fp64;
}
template <class MA, class MB, class MC>
bool tc_products(const Ctx& st, int batch, int M, int N, int K, double alpha, MA A, int64_t sA, MB B, int64_t sB,
                 double beta, MC C, int64_t sC, bool lower) {
  auto bytes = [&](int z) { return tc::scratch_bytes(sA == 0 ? 1 : z, sB == 0 ? 1 : z, M, N, K); };
  int zc = batch;
  while (zc > 1 && bytes(zc) > st.tc_cap) zc = (zc + 1) / 2;
  while (zc > 1 && bytes(zc) > st.tc_cap) --zc;
  if (bytes(zc) > st.tc_cap) zc = 0;
  if (zc < 1) return false;
  for (int z0 = 0; z0 < batch; z0 += zc) {
    const int nz = std::min(zc, batch - z0);
    if (tc::gemm(st.s, st.tc, st.tc_cap, st.status, nz, M, N, K, alpha, shifted(A, z0 * sA), sA,
                 shifted(B, z0 * sB), sB, beta, shifted(C, z0 * sC), sC, lower) != cudaSuccess)
      return false;
    for (int p = 0; p < 3 * std::max(1, (K + tc::KMAX - 1) / tc::KMAX); ++p) chd_launch::count_launch();
    chd_launch::count_tc_flops(static_cast<double>(nz) * tc::mma_flops(M, N, K, lower));
  }
  return true;
}

template <class MA, class MB, class MC>
void gemm(const Ctx& st, int batch, int M, int N, int K, double alpha, MA A, int64_t sA, MB B, int64_t sB,
          double beta, MC C, int64_t sC, bool lower) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (tc_worth(st, batch, M, N, K, sA == 0, sB == 0) && tc_products(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower)) return;
  constexpr int64_t kFill = 2 * 152;
  if (N <= 8 && M > 64) gemm_cfg<128, 8, 4, 1>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
  else if (N <= 16 && M > 64) gemm_cfg<128, 16, 4, 2>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
  else if (M <= 8 && N > 64) gemm_cfg<8, 128, 1, 4>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
  else if (M <= 16 && N > 64) gemm_cfg<16, 128, 2, 4>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
  else {
    // 64 x 64 tiles unless 32 x 32 tiles balance the SMs clearly better (the
    // FP64 pipe, not shared-memory traffic, bounds both tile shapes)
    const int64_t t64 = tile_count(M, N, 64, 64, lower) * batch;
    const int64_t t32 = tile_count(M, N, 32, 32, lower) * batch;
    if (t64 >= kFill && balance(t64) >= 0.9 * balance(t32))
      gemm_cfg<64, 64, 4, 4>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
    else if (t32 >= kFill || M <= 32 || N <= 32 || K >= 512)
      gemm_cfg<32, 32, 2, 2>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
    else
      gemm_cfg<16, 16, 1, 1>(st, batch, M, N, K, alpha, A, sA, B, sB, beta, C, sC, lower);
  }
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky (panels of PP columns) and triangular
// solves (panels of TW columns).  On GB300 an SM retires about 1.6 FP64
// lane-operations per clock, spread over its four sub-partitions: a single
// warp issuing FP64 instructions keeps one sub-partition busy and leaves
// three idle.  The panel kernels therefore run four warps per CTA and only
// PR = 8 rows per CTA (two rows per warp, sixteen lanes per row, lane q
// owning the panel columns c = q mod 16), so that a panel of R rows keeps
// R / 2 warps issuing; the substitution along the panel columns passes each
// solved entry within its 16-lane group by a shuffle.
// ---------------------------------------------------------------------------
constexpr int PP = 32;   // Cholesky panel width
constexpr int TW = 64;   // triangular-solve panel width
constexpr int PR = 8;    // panel rows per CTA
constexpr int PT = 128;  // threads per panel CTA

// Cooperative Cholesky of the pb x pb block held in shared memory (ld
// PP + 1, identity beyond pb) by the CTA's PT threads: column by column,
// pivot, scale of the column below it, rank-one update of the trailing
// lower triangle.  On return Ls holds the lower factor C and rinv the
// reciprocal pivots; a non-positive pivot is recorded and replaced by 1.
// Every CTA of a launch computes the same values in the same order.
__device__ __forceinline__ void cta_potrf32(double (*Ls)[PP + 1], double* rinv, int pb, int64_t* st, int64_t code,
                                            int64_t snode, int64_t col) {
  const int tid = threadIdx.x;
  for (int j = 0; j < pb; ++j) {
    if (tid == 0) {
      double d = Ls[j][j];
      if (!(d > 0.0)) {
        record_error(st, code, snode, col < 0 ? -1 : col + j);
        d = 1.0;
      }
      Ls[j][j] = sqrt(d);
      rinv[j] = rsqrt(d);
    }
    __syncthreads();
    const double r = rinv[j];
    for (int i = j + 1 + tid; i < pb; i += PT) Ls[i][j] *= r;
    __syncthreads();
    const int w = pb - j - 1;
    for (int e = tid; e < w * w; e += PT) {
      const int i = j + 1 + e % w, k = j + 1 + e / w;
      if (k <= i) Ls[i][k] = fma(-Ls[i][j], Ls[k][j], Ls[i][k]);
    }
    __syncthreads();
  }
}

// One panel of the Cholesky of F (ld): the pb x pb block at (j0, j0) and the
// R rows below it (rows j0+pb ..).  Every CTA factors the diagonal block
// (the same arithmetic in every CTA, so the copies agree bitwise) and
// solves its PR rows, B := B C^{-T}.  The CTA that arrives last at the
// counter -- when every CTA has read the unfactored block -- writes the
// factored block back and resets the counter.  ctr == nullptr is allowed
// for a single-CTA launch with R == 0.
__global__ void __launch_bounds__(PT) mk_potrf_panel(double* F, int64_t ld, int j0, int pb, int R, int* ctr,
                                                     int64_t* st, int64_t code, int64_t snode, int64_t col0) {
  __shared__ double Ls[PP][PP + 1];
  __shared__ double rinv[PP];
  __shared__ int last;
  const int tid = threadIdx.x;
  double* D = F + j0 + (int64_t)j0 * ld;
  for (int e = tid; e < PP * PP; e += PT) {
    const int i = e % PP, c = e / PP;
    Ls[i][c] = (i < pb && c < pb && i >= c) ? D[i + (int64_t)c * ld] : (i == c ? 1.0 : 0.0);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = (ctr == nullptr) ? 1 : (atomicAdd(ctr, 1) == (int)gridDim.x - 1);
  }
  cta_potrf32(Ls, rinv, pb, st, code, snode, col0 < 0 ? -1 : col0 + j0);
  const int lane = tid & 31, q = lane & 15;
  const int i = blockIdx.x * PR + 2 * (tid >> 5) + (lane >> 4);
  const bool ok = i < R;
  double* Bi = F + (j0 + pb + (ok ? i : 0)) + (int64_t)j0 * ld;
  double b[PP / 16];
#pragma unroll
  for (int u = 0; u < PP / 16; ++u) {
    const int c = 16 * u + q;
    b[u] = (ok && c < pb) ? Bi[(int64_t)c * ld] : 0.0;
  }
#pragma unroll
  for (int c = 0; c < PP; ++c) {
    if (c < pb) {
      double x = b[c / 16] * rinv[c];
      x = __shfl_sync(0xffffffffu, x, (lane & 16) | (c & 15));
      if (q == (c & 15)) b[c / 16] = x;
#pragma unroll
      for (int u = c / 16; u < PP / 16; ++u) {
        const int t = 16 * u + q;
        if (t > c && t < pb) b[u] = fma(-Ls[t][c], x, b[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PP / 16; ++u) {
    const int c = 16 * u + q;
    if (ok && c < pb) Bi[(int64_t)c * ld] = b[u];
  }
  if (last) {
    for (int e = tid; e < pb * pb; e += PT) {
      const int r = e % pb, c = e / pb;
      if (r >= c) D[r + (int64_t)c * ld] = Ls[r][c];
    }
    if (tid == 0 && ctr) *ctr = 0;
  }
}

// Panel triangular solve on PR rows per CTA of B (R rows), panel columns
// [p0, p0+pb), pb <= TW, against the diagonal block L[p0.., p0..] (lower):
//   fwd = 1:  B_p := B_p L_pp^{-T}      fwd = 0:  B_p := B_p L_pp^{-1}
template <class MB>
__global__ void __launch_bounds__(PT) mk_trsm_panel(int R, MB B, int64_t sB, int p0, int pb, const double* L,
                                                    int64_t ld, int fwd) {
  __shared__ double Ls[TW][TW + 1];
  __shared__ double rinv[TW];
  const int tid = threadIdx.x;
  B.p += (int64_t)blockIdx.z * sB;
  for (int e = tid; e < pb * pb; e += PT) {
    const int i = e % pb, j = e / pb;
    Ls[i][j] = i >= j ? L[(p0 + i) + (int64_t)(p0 + j) * ld] : 0.0;
  }
  __syncthreads();
  for (int c = tid; c < pb; c += PT) rinv[c] = 1.0 / Ls[c][c];
  __syncthreads();
  const int lane = tid & 31, q = lane & 15;
  const int r = blockIdx.x * PR + 2 * (tid >> 5) + (lane >> 4);
  const bool ok = r < R;
  double b[TW / 16];
#pragma unroll
  for (int u = 0; u < TW / 16; ++u) {
    const int c = 16 * u + q;
    b[u] = (ok && c < pb) ? B.at(r, p0 + c) : 0.0;
  }
  if (fwd) {
#pragma unroll
    for (int c = 0; c < TW; ++c) {
      if (c < pb) {
        double x = b[c / 16] * rinv[c];
        x = __shfl_sync(0xffffffffu, x, (lane & 16) | (c & 15));
        if (q == (c & 15)) b[c / 16] = x;
#pragma unroll
        for (int u = c / 16; u < TW / 16; ++u) {
          const int t = 16 * u + q;
          if (t > c && t < pb) b[u] = fma(-Ls[t][c], x, b[u]);
        }
      }
    }
  } else {
#pragma unroll
    for (int c = TW - 1; c >= 0; --c) {
      if (c < pb) {
        double x = b[c / 16] * rinv[c];
        x = __shfl_sync(0xffffffffu, x, (lane & 16) | (c & 15));
        if (q == (c & 15)) b[c / 16] = x;
#pragma unroll
        for (int u = 0; u <= c / 16; ++u) {
          const int t = 16 * u + q;
          if (t < c) b[u] = fma(-Ls[c][t], x, b[u]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < TW / 16; ++u) {
    const int c = 16 * u + q;
    if (ok && c < pb) B.at(r, p0 + c) = b[u];
  }
}

template <class MB>
void panel_solve(const Ctx& st, int batch, int R, MB B, int64_t sB, int p0, int pb, const double* L,
                 int64_t ld, int fwd) {
  mk_trsm_panel<MB><<<dim3((R + PR - 1) / PR, 1, batch), PT, 0, st>>>(R, B, sB, p0, pb, L, ld, fwd);
  chd_launch::count_launch();
}


// Two-level blocking: within an outer block of NBT (solves) or NBC
// (Cholesky) columns the panels update only the block's own columns; the
// columns beyond the block are updated once per block, by one product with
// the block's width as inner dimension -- long enough for the tensor cores.
constexpr int NBT = 256;  // outer block of the triangular solves (a multiple of TW)
constexpr int NBC = 128;  // outer block of the Cholesky (a multiple of PP)

// B := B L^{-T} (R x n view B, n x n lower L), blocked forward.
template <class MB>
void trsm_rLT(const Ctx& st, int batch, int R, int n, MB B, int64_t sB, const double* L, int64_t ld) {
  if (R <= 0 || n <= 0) return;
  for (int b0 = 0; b0 < n; b0 += NBT) {
    const int bw = std::min(NBT, n - b0);
    for (int p0 = b0; p0 < b0 + bw; p0 += TW) {
      const int pb = std::min(TW, b0 + bw - p0);
      panel_solve(st, batch, R, B, sB, p0, pb, L, ld, 1);
      const int rest = b0 + bw - p0 - pb;
      if (rest > 0)
        gemm(st, batch, R, rest, pb, -1.0, colshift(B, p0), sB, DnT{L + (p0 + pb) + (int64_t)p0 * ld, ld}, 0,
             1.0, colshift(B, p0 + pb), sB, false);
    }
    const int rest = n - b0 - bw;
    if (rest > 0)
      gemm(st, batch, R, rest, bw, -1.0, colshift(B, b0), sB, DnT{L + (b0 + bw) + (int64_t)b0 * ld, ld}, 0, 1.0,
           colshift(B, b0 + bw), sB, false);
  }
}
// B := B L^{-1}, blocked backward.
template <class MB>
void trsm_rL(const Ctx& st, int batch, int R, int n, MB B, int64_t sB, const double* L, int64_t ld) {
  if (R <= 0 || n <= 0) return;
  for (int b0 = (n - 1) / NBT * NBT; b0 >= 0; b0 -= NBT) {
    const int b1 = std::min(n, b0 + NBT);
    for (int p0 = (b1 - 1 - b0) / TW * TW + b0; p0 >= b0; p0 -= TW) {
      const int pb = std::min(TW, b1 - p0);
      panel_solve(st, batch, R, B, sB, p0, pb, L, ld, 0);
      if (p0 > b0)
        gemm(st, batch, R, p0 - b0, pb, -1.0, colshift(B, p0), sB,
             Dn{const_cast<double*>(L) + p0 + (int64_t)b0 * ld, ld}, 0, 1.0, colshift(B, b0), sB, false);
    }
    if (b0 > 0)
      gemm(st, batch, R, b0, b1 - b0, -1.0, colshift(B, b0), sB, Dn{const_cast<double*>(L) + b0, ld}, 0, 1.0,
           colshift(B, 0), sB, false);
  }
}

// Partial Cholesky of the first n columns of the J x J matrix F (ld): F11 =
// C C^T, F21 := F21 C^{-T}, F22 -= F21 F21^T (lower).  Not batched.  One
// launch per panel (diagonal block and the rows below) when the context has
// a panel counter, else the diagonal block and the row solve separately.
void potrf_partial(const Ctx& st, double* F, int64_t ld, int J, int n, int64_t* status, int64_t code,
                   int64_t snode, int64_t col0) {
  for (int b0 = 0; b0 < n; b0 += NBC) {
    const int bw = std::min(NBC, n - b0);
    for (int j0 = b0; j0 < b0 + bw; j0 += PP) {
      const int pb = std::min(PP, b0 + bw - j0);
      const int R = J - j0 - pb;
      if (st.ctr) {
        mk_potrf_panel<<<std::max(1, (R + PR - 1) / PR), PT, 0, st>>>(F, ld, j0, pb, R, st.ctr, status, code,
                                                                        snode, col0);
        chd_launch::count_launch();
      } else {
        mk_potrf_panel<<<1, PT, 0, st>>>(F, ld, j0, pb, 0, nullptr, status, code, snode, col0);
        chd_launch::count_launch();
        if (R > 0) panel_solve(st, 1, R, Dn{F + j0 + pb, ld}, 0, j0, pb, F, ld, 1);
      }
      // update of the block's remaining columns (all rows below them)
      const int rest = b0 + bw - j0 - pb;
      if (rest > 0) {
        double* P = F + (j0 + pb) + (int64_t)j0 * ld;
        gemm(st, 1, R, rest, pb, -1.0, Dn{P, ld}, 0, DnT{P, ld}, 0, 1.0,
             Dn{F + (j0 + pb) + (int64_t)(j0 + pb) * ld, ld}, 0, true);
      }
    }
    // trailing update beyond the block: F[b1:, b1:] -= P P^T, P = F[b1:, b0:b1]
    const int b1 = b0 + bw, R = J - b1;
    if (R > 0) {
      double* P = F + b1 + (int64_t)b0 * ld;
      gemm(st, 1, R, R, bw, -1.0, Dn{P, ld}, 0, DnT{P, ld}, 0, 1.0, Dn{F + b1 + (int64_t)b1 * ld, ld}, 0, true);
    }
  }
}

// ---------------------------------------------------------------------------
// element-wise kernels (batched over blockIdx.z)
// ---------------------------------------------------------------------------
constexpr int EW = 4096;  // elements per CTA

__global__ void __launch_bounds__(BT) mk_csc_to_front(double* F, int64_t sF, int J, int n, const double* csc,
                                                      int64_t sC) {
  F += blockIdx.z * sF;
  csc += blockIdx.z * sC;
  const int64_t tot = (int64_t)J * n;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % J), c = (int)(e / J);
    if (r >= c) F[r + (int64_t)c * J] = csc[csc_off(J, r, c)];
  }
}
// csc(r, c) = scale * F(r, c) for rows r_lo <= r < r_hi with r >= c, columns
// c < n, of a front with J rows
__global__ void __launch_bounds__(BT) mk_front_to_csc(double* csc, int64_t sC, const double* F, int64_t sF,
                                                      int64_t ldF, int J, int n, int r_lo, int r_hi,
                                                      double scale) {
  F += blockIdx.z * sF;
  csc += blockIdx.z * sC;
  const int64_t tot = (int64_t)J * n;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % J), c = (int)(e / J);
    if (r >= c && r >= r_lo && r < r_hi) csc[csc_off(J, r, c)] = scale * F[r + (int64_t)c * ldF];
  }
}
// dst = alpha * src (+ beta * dst) on an R x C block, or its lower part
__global__ void __launch_bounds__(BT) mk_copy(double* dst, int64_t sD, int64_t ldd, const double* src, int64_t sS,
                                              int64_t lds, int R, int C, double alpha, double beta, int lower,
                                              int transpose_fill) {
  dst += blockIdx.z * sD;
  if (src) src += blockIdx.z * sS;
  const int64_t tot = (int64_t)R * C;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % R), c = (int)(e / R);
    if (lower && r < c) continue;
    double v = 0.0;
    if (src) {
      // transpose_fill: read the symmetric partner from the lower triangle
      v = (transpose_fill && r < c) ? src[c + (int64_t)r * lds] : src[r + (int64_t)c * lds];
    }
    double* d = dst + r + (int64_t)c * ldd;
    *d = beta != 0.0 ? fma(beta, *d, alpha * v) : alpha * v;
  }
}
// dst (lower, ld m) = P src P for the symmetric src stored lower, P the
// order reversal
__global__ void __launch_bounds__(BT) mk_rev_lower(double* dst, const double* src, int m) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % m), c = (int)(e / m);
    if (r >= c) dst[r + (int64_t)c * m] = src[(m - 1 - c) + (int64_t)(m - 1 - r) * m];
  }
}
__global__ void __launch_bounds__(BT) mk_identity(double* dst, int64_t ld, int m) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % m), c = (int)(e / m);
    dst[r + (int64_t)c * ld] = r == c ? 1.0 : 0.0;
  }
}

// Extend-add of the children's update blocks into front k, one CTA per 64x64
// tile of the lower triangle; children are added in a fixed order, and the
// child rows landing in a tile are a contiguous range because the relative
// indices are increasing.
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__global__ void __launch_bounds__(BT) mk_extend_add(SymDev S, int k, double* ws, int64_t sws, int tiles,
                                                    const uint8_t* act) {
  const int tm = (blockIdx.x / tiles) * GT, tn = (blockIdx.x % tiles) * GT;
  if (tn > tm) return;
  ws += blockIdx.z * sws;
  if (act) act += blockIdx.z * S.nsn;
  const int Jp = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  double* F = ws + S.f_off[k];
  for (int64_t q = S.ea_ptr[k]; q < S.ea_ptr[k + 1]; ++q) {
    const int c = S.ea[q];
    if (act && !act[c]) continue;  // pruned child (§5.5): its update block is zero
    const int nc = (int)(S.sn_ptr[c + 1] - S.sn_ptr[c]);
    const int Jc = (int)(S.rows_ptr[c + 1] - S.rows_ptr[c]);
    const int ac = Jc - nc;
    const int32_t* rel = S.rel + S.rows_ptr[c] + nc;
    const int i0 = lower_bound_i32(rel, ac, tm), i1 = lower_bound_i32(rel, ac, tm + GT);
    const int j0 = lower_bound_i32(rel, ac, tn), j1 = lower_bound_i32(rel, ac, tn + GT);
    const int ni = i1 - i0, nj = j1 - j0;
    const double* U = ws + S.f_off[c] + nc + (int64_t)nc * Jc;
    for (int e = threadIdx.x; e < ni * nj; e += BT) {
      const int i = i0 + e % ni, j = j0 + e / ni;
      if (i >= j) F[__ldg(rel + i) + (int64_t)__ldg(rel + j) * Jp] += __ldcg(U + i + (int64_t)j * Jc);
    }
    __syncthreads();
  }
}
// V block of front k gathered from the parent's front (top-down passes)
__global__ void __launch_bounds__(BT) mk_gather_parent(SymDev S, int k, double* ws, int64_t sws) {
  ws += blockIdx.z * sws;
  const int p = (int)S.sn_par[k];
  const int n = (int)(S.sn_ptr[k + 1] - S.sn_ptr[k]);
  const int J = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  const int a = J - n;
  const int Jp = (int)(S.rows_ptr[p + 1] - S.rows_ptr[p]);
  const double* Fp = ws + S.f_off[p];
  double* F = ws + S.f_off[k];
  const int32_t* rel = S.rel + S.rows_ptr[k] + n;
  const int64_t tot = (int64_t)a * a;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % a), s = (int)(e / a);
    if (r >= s) F[(n + r) + (int64_t)(n + s) * J] = __ldcg(Fp + __ldg(rel + r) + (int64_t)__ldg(rel + s) * Jp);
  }
}
// V_k = S_{A_k A_k} of front k read directly from the input S (completion)
__global__ void __launch_bounds__(BT) mk_gather_saa(SymDev S, int k, const double* Sin, double* ws) {
  const int n = (int)(S.sn_ptr[k + 1] - S.sn_ptr[k]);
  const int J = (int)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
  const int a = J - n;
  double* F = ws + S.f_off[k];
  const int32_t* A = S.rows + S.rows_ptr[k] + n;
  const int64_t tot = (int64_t)a * a;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % a), c = (int)(e / a);
    if (r >= c) F[(n + r) + (int64_t)(n + c) * J] = Sin[csc_find(S, __ldg(A + r), __ldg(A + c))];
  }
}
// rows r and R-1-r of the R x C block B (ld) exchanged
__global__ void __launch_bounds__(BT) mk_rev_rows(double* B, int64_t ld, int R, int C) {
  const int h = R / 2;
  const int64_t tot = (int64_t)h * C;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % h), c = (int)(e / h);
    double* x = B + r + (int64_t)c * ld;
    double* y = B + (R - 1 - r) + (int64_t)c * ld;
    const double t = *x;
    *x = *y;
    *y = t;
  }
}
// factored update matrices (fc_body.cuh): the gather of front k
__global__ void __launch_bounds__(BT) mk_fc_gather(SymDev S, int k, const double* Sin, double* Gq, double* fcs) {
  const fc::Info f = fc::info(S, k);
  const int64_t tot = fc::gather_count(f);
  const double* Gp = Gq + S.v_off[f.p];
  double* X = fcs + S.fc_off[k];
  double* G = Gq + S.v_off[k];
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT)
    fc::gather_one(f, e, Sin, Gp, f.Jp - f.np, X, G);
}
// ... its Householder reduction in panels of fc::NB rows: one panel among
// itself (one CTA), its reflectors V and T after X in the front's scratch
__global__ void __launch_bounds__(BT) k_fc_panel(SymDev S, int k, int t0, int t1, int L, double* fcs, int64_t* st) {
  const fc::Info f = fc::info(S, k);
  double* X = fcs + S.fc_off[k];
  double* V = X + (int64_t)f.q * f.w;
  fc::panel(f, X, t0, t1, L, V, V + (int64_t)f.w * fc::NB, st);
}
// ... and the reduced X's lower triangle into G_k's first q columns
__global__ void __launch_bounds__(BT) mk_fc_copy(SymDev S, int k, double* Gq, const double* fcs) {
  const fc::Info f = fc::info(S, k);
  const double* X = fcs + S.fc_off[k];
  double* G = Gq + S.v_off[k];
  const int64_t tot = (int64_t)f.q * f.q;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % f.q), c = (int)(e / f.q);
    if (r >= c) G[r + (int64_t)c * f.a] = X[(int64_t)r * f.w + c];
  }
}
__global__ void k_logdet_diag(const double* F, int64_t ld, int n, double* out) {
  __shared__ double red[BT];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += BT) s += 2.0 * log(F[i + (int64_t)i * ld]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = BT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
// inverse-Hessian step 3 finish: Y_AN = 2P - K_AN - Z_AN, Y_NN = K_NN - Z_NN
__global__ void __launch_bounds__(BT) mk_ihess_finish(double* Y, int64_t sY, const double* F, const double* P,
                                                      int64_t sF, int J, int n) {
  Y += blockIdx.z * sY;
  F += blockIdx.z * sF;
  P += blockIdx.z * sF;
  const int64_t tot = (int64_t)J * n;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % J), c = (int)(e / J);
    if (r < c) continue;
    const int64_t o = csc_off(J, r, c);
    const double z = F[r + (int64_t)c * J];
    if (r >= n) Y[o] = 2.0 * P[r + (int64_t)c * J] - Y[o] - z;
    else Y[o] = Y[o] - z;
  }
}

inline int ew_blocks(int64_t tot) { return (int)std::max<int64_t>(1, (tot + EW - 1) / EW); }
#define CHD_EW(kernel, tot, batch, st, ...)                                  \
  do {                                                                       \
    kernel<<<dim3(ew_blocks(tot), 1, (batch)), BT, 0, (st)>>>(__VA_ARGS__); \
    chd_launch::count_launch();                                              \
  } while (0)

// ---------------------------------------------------------------------------
// per-front sequences
// ---------------------------------------------------------------------------
struct Front {
  int k, n, a, J;
  int64_t base, col0;
  int64_t foff;
};
inline Front front(const chd_symbolic* s, int k) {
  Front f;
  f.k = k;
  f.col0 = s->sn_ptr[k];
  f.n = (int)(s->sn_ptr[k + 1] - f.col0);
  f.J = (int)(s->rows_ptr[k + 1] - s->rows_ptr[k]);
  f.a = f.J - f.n;
  f.base = s->colptr[f.col0];
  f.foff = s->f_off[k];
  return f;
}

void assemble_children(const chd_symbolic* s, const Ctx& st, int batch, int k, double* ws, int64_t sws,
                       const uint8_t* act = nullptr) {
  if (s->ea_ptr[k + 1] == s->ea_ptr[k]) return;
  const int J = (int)(s->rows_ptr[k + 1] - s->rows_ptr[k]);
  const int t = (J + GT - 1) / GT;
  mk_extend_add<<<dim3(t * t, 1, batch), BT, 0, st>>>(s->dev, k, ws, sws, t, act);
  chd_launch::count_launch();
}
void gather_parent(const chd_symbolic* s, const Ctx& st, int batch, const Front& f, double* ws, int64_t sws) {
  if (s->sn_par[f.k] < 0 || f.a == 0) return;
  CHD_EW(mk_gather_parent, (int64_t)f.a * f.a, batch, st, s->dev, f.k, ws, sws);
}

void factor_front(const chd_symbolic* s, const Ctx& st, int k, const double* X, double* Lc, double* Wc,
                  double* Dd, double* ws, double* ldet, int64_t* status) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  double* T2 = T1 + (int64_t)J * n;
  CHD_EW(mk_csc_to_front, (int64_t)J * n, 1, st, F, 0, J, n, X + f.base, 0);
  if (a > 0) CHD_EW(mk_copy, (int64_t)a * a, 1, st, F + n + (int64_t)n * J, 0, J, nullptr, 0, 0, a, a, 0.0, 0.0, 1, 0);
  assemble_children(s, st, 1, k, ws, 0);
  CHD_EW(mk_copy, (int64_t)n * n, 1, st, Dd + s->d_off[k], 0, n, F, 0, J, n, n, 1.0, 0.0, 1, 0);
  potrf_partial(st, F, J, J, n, status, CHD_ERR_NOT_PD, k, f.col0);
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Lc + f.base, 0, F, 0, J, J, n, 0, J, 1.0);
  k_logdet_diag<<<1, BT, 0, st>>>(F, J, n, ldet + k);
  chd_launch::count_launch();
  // Cinv = C^{-1} (T1), D^{-1} = Cinv^T Cinv (T2 top), L_AN = B C^{-1} (T2 bottom)
  CHD_EW(mk_identity, (int64_t)n * n, 1, st, T1, J, n);
  trsm_rLT(st, 1, n, n, DnTW{T1, J}, 0, F, J);
  gemm(st, 1, n, n, n, 1.0, TriLT{T1, J}, 0, TriL{T1, J}, 0, 0.0, Dn{T2, J}, 0, true);
  if (a > 0) {
    CHD_EW(mk_copy, (int64_t)a * n, 1, st, T2 + n, 0, J, F + n, 0, J, a, n, 1.0, 0.0, 0, 0);
    trsm_rL(st, 1, a, n, Dn{T2 + n, J}, 0, F, J);
  }
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Wc + f.base, 0, T2, 0, J, J, n, 0, J, 1.0);
}

void gradient_front(const chd_symbolic* s, const Ctx& st, int k, const double* Wc, double* Sc, double* g,
                    double* Vd, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  double* F = ws + f.foff;
  gather_parent(s, st, 1, f, ws, 0);
  const double* W = Wc + f.base;
  CHD_EW(mk_csc_to_front, (int64_t)J * n, 1, st, F, 0, J, n, W, 0);  // D^{-1}; rows >= n overwritten next
  gemm(st, 1, a, n, a, -1.0, SymL{F + n + (int64_t)n * J, J}, 0, CscRO{W, J, n}, 0, 0.0, Dn{F + n, J}, 0, false);
  gemm(st, 1, n, n, a, -1.0, DnT{F + n, J}, 0, CscRO{W, J, n}, 0, 1.0, Dn{F, J}, 0, true);
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Sc + f.base, 0, F, 0, J, J, n, 0, J, 1.0);
  if (g) CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, g + f.base, 0, F, 0, J, J, n, 0, J, -1.0);
  if (a > 0) CHD_EW(mk_copy, (int64_t)a * a, 1, st, Vd + s->v_off[k], 0, a, F + n + (int64_t)n * J, 0, J, a, a, 1.0, 0.0, 1, 0);
}

void hess_up_front(const chd_symbolic* s, const Ctx& st, int m, int k, const double* Wc, const double* Vd,
                   const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws, const uint8_t* act) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  const int64_t sw = s->dev.f_total;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  double* T2 = T1 + (int64_t)J * n;
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  CHD_EW(mk_csc_to_front, (int64_t)J * n, m, st, F, sw, J, n, Y + f.base, ldy);
  if (a > 0) CHD_EW(mk_copy, (int64_t)a * a, m, st, F + n + (int64_t)n * J, sw, J, nullptr, 0, 0, a, a, 0.0, 0.0, 1, 0);
  assemble_children(s, st, m, k, ws, sw, act);
  if (a > 0) {
    CHD_EW(mk_copy, (int64_t)a * n, m, st, T1 + n, sw, J, F + n, sw, J, a, n, 1.0, 0.0, 0, 0);
    gemm(st, m, a, n, n, -1.0, L, 0, SymL{F, J}, sw, 1.0, Dn{T1 + n, J}, sw, false);
    gemm(st, m, a, a, n, -1.0, Dn{T1 + n, J}, sw, CscT{W, J, n}, 0, 1.0, Dn{F + n + (int64_t)n * J, J}, sw, true);
    gemm(st, m, a, a, n, -1.0, L, 0, DnT{F + n, J}, sw, 1.0, Dn{F + n + (int64_t)n * J, J}, sw, true);
  }
  CscSym Dinv{W, J};
  gemm(st, m, n, n, n, 1.0, SymL{F, J}, sw, Dinv, 0, 0.0, Dn{T2, J}, sw, false);
  gemm(st, m, n, n, n, 1.0, Dinv, 0, Dn{T2, J}, sw, 0.0, Csc{T + f.base, J, 0}, ldt, true);
  if (a > 0) {
    gemm(st, m, a, n, n, 1.0, Dn{T1 + n, J}, sw, Dinv, 0, 0.0, Dn{T2 + n, J}, sw, false);
    gemm(st, m, a, n, a, 1.0, SymL{Vd + s->v_off[k], a}, 0, Dn{T2 + n, J}, sw, 0.0, Csc{T + f.base, J, n}, ldt, false);
  }
}

void hess_down_front(const chd_symbolic* s, const Ctx& st, int m, int k, const double* Wc, double* T,
                     int64_t ldt, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  const int64_t sw = s->dev.f_total;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  gather_parent(s, st, m, f, ws, sw);
  CHD_EW(mk_csc_to_front, (int64_t)J * n, m, st, F, sw, J, n, T + f.base, ldt);
  if (a > 0) {
    gemm(st, m, a, n, a, 1.0, SymL{F + n + (int64_t)n * J, J}, sw, L, 0, 0.0, Dn{T1 + n, J}, sw, false);
    CHD_EW(mk_copy, (int64_t)a * n, m, st, F + n, sw, J, T1 + n, sw, J, a, n, -0.5, 1.0, 0, 0);
    gemm(st, m, n, n, a, -1.0, DnT{F + n, J}, sw, L, 0, 1.0, Dn{F, J}, sw, true);
    gemm(st, m, n, n, a, -1.0, CscT{W, J, n}, 0, Dn{F + n, J}, sw, 1.0, Dn{F, J}, sw, true);
    CHD_EW(mk_copy, (int64_t)a * n, m, st, F + n, sw, J, T1 + n, sw, J, a, n, -0.5, 1.0, 0, 0);
  }
  CHD_EW(mk_front_to_csc, (int64_t)J * n, m, st, T + f.base, ldt, F, sw, J, J, n, 0, J, 1.0);
}

void ihess_down_front(const chd_symbolic* s, const Ctx& st, int m, int k, const double* Wc, const double* Dd,
                      const double* Rd, const double* Tin, int64_t ldt, double* Yout, int64_t ldy, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  const int64_t sw = s->dev.f_total;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  double* T2 = T1 + (int64_t)J * n;
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  gather_parent(s, st, m, f, ws, sw);
  CHD_EW(mk_csc_to_front, (int64_t)J * n, m, st, F, sw, J, n, Tin + f.base, ldt);
  // T1 = [M_NN (full); M_AN]
  CHD_EW(mk_copy, (int64_t)n * n, m, st, T1, sw, J, F, sw, J, n, n, 1.0, 0.0, 0, 1);
  if (a > 0) {
    CHD_EW(mk_copy, (int64_t)a * n, m, st, T1 + n, sw, J, F + n, sw, J, a, n, 1.0, 0.0, 0, 0);
    gemm(st, m, a, n, a, 1.0, SymL{F + n + (int64_t)n * J, J}, sw, L, 0, 1.0, Dn{T1 + n, J}, sw, false);
    gemm(st, m, n, n, a, 1.0, DnT{F + n, J}, sw, L, 0, 1.0, Dn{T1, J}, sw, false);
    gemm(st, m, n, n, a, 1.0, CscT{W, J, n}, 0, Dn{T1 + n, J}, sw, 1.0, Dn{T1, J}, sw, false);
  }
  const double* D = Dd + s->d_off[k];
  gemm(st, m, n, n, n, 1.0, Dn{T1, J}, sw, SymL{D, n}, 0, 0.0, Dn{T2, J}, sw, false);
  gemm(st, m, n, n, n, 1.0, SymL{D, n}, 0, Dn{T2, J}, sw, 0.0, Csc{Yout + f.base, J, 0}, ldy, true);
  if (a > 0) {
    // K_AN = V^{-1} (M_AN D), V^{-1} formed once per factor
    gemm(st, m, a, n, n, 1.0, Dn{T1 + n, J}, sw, SymL{D, n}, 0, 0.0, Dn{T2 + n, J}, sw, false);
    gemm(st, m, a, n, a, 1.0, SymL{Rd + s->v_off[k], a}, 0, Dn{T2 + n, J}, sw, 0.0, Csc{Yout + f.base, J, n}, ldy,
         false);
  }
}

void ihess_up_front(const chd_symbolic* s, const Ctx& st, int m, int k, const double* Wc, double* Y,
                    int64_t ldy, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  const int64_t sw = s->dev.f_total;
  double* F = ws + f.foff;
  double* T2 = F + (int64_t)J * J + (int64_t)J * n;
  const double* W = Wc + f.base;
  CscRO L{W, J, n};
  CHD_EW(mk_copy, (int64_t)J * J, m, st, F, sw, J, nullptr, 0, 0, J, J, 0.0, 0.0, 1, 0);
  assemble_children(s, st, m, k, ws, sw);
  if (a > 0) {
    // T2[n:J] = P = K_AN + 1/2 L K_NN   (K in the output array)
    CHD_EW(mk_csc_to_front, (int64_t)J * n, m, st, T2, sw, J, n, Y + f.base, ldy);
    gemm(st, m, a, n, n, 0.5, L, 0, CscSym{Y + f.base, J}, ldy, 1.0, Dn{T2 + n, J}, sw, false);
    gemm(st, m, a, a, n, -1.0, Dn{T2 + n, J}, sw, CscT{W, J, n}, 0, 1.0, Dn{F + n + (int64_t)n * J, J}, sw, true);
    gemm(st, m, a, a, n, -1.0, L, 0, DnT{T2 + n, J}, sw, 1.0, Dn{F + n + (int64_t)n * J, J}, sw, true);
  }
  CHD_EW(mk_ihess_finish, (int64_t)J * n, m, st, Y + f.base, ldy, F, T2, sw, J, n);
}

// Hessian factor (§5.4) for one big front, M <-> W in place on the N-part
// of Z: dir 0: W_NN = C^T M_NN C, W_AN = Q^{-1} (M_AN C); dir 1: M_NN =
// C^{-T} W_NN C^{-1}, M_AN = Q (W_AN C^{-1}); C = chol(D_NN) from the
// factor, Q the upper factor of V held as Q' = P Q P (A-rows reversed).
template <class MD, class MS>
__global__ void __launch_bounds__(BT) mk_copy_view(MD D, int64_t sD, MS S, int64_t sS, int R, int C) {
  D.p += blockIdx.z * sD;
  S.p += blockIdx.z * sS;
  const int64_t tot = (int64_t)R * C;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % R), c = (int)(e / R);
    D.at(r, c) = S.at(r, c);
  }
}
template <class MD, class MS>
void copy_view(const Ctx& st, int batch, MD D, int64_t sD, MS S, int64_t sS, int R, int C) {
  if ((int64_t)R * C <= 0 || batch <= 0) return;
  mk_copy_view<<<dim3(ew_blocks((int64_t)R * C), 1, batch), BT, 0, st>>>(D, sD, S, sS, R, C);
  chd_launch::count_launch();
}
void rtrans_front(const chd_symbolic* s, const Ctx& st, int m, int k, int dir, const double* Lc, const double* Qd,
                  double* Z, int64_t ldz, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  const int64_t sw = s->dev.f_total;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  double* T2 = T1 + (int64_t)J * n;
  const double* Q = Qd + s->v_off[k];
  const double* Lk = Lc + f.base;
  double* Zk = Z + f.base;
  if (dir == 0) {
    // T1 = [M_NN C; P M_AN C], W_NN = C^T (M_NN C), then Q'^{-1} on the A-rows
    gemm(st, m, n, n, n, 1.0, CscSym{Zk, J}, ldz, CscL{Lk, J}, 0, 0.0, Dn{T1, J}, sw, false);
    if (a > 0)
      gemm(st, m, a, n, n, 1.0, CscRO{Zk, J, n}, ldz, CscL{Lk, J}, 0, 0.0, DnRev{T1 + n, J, a}, sw, false);
    gemm(st, m, n, n, n, 1.0, CscLT{Lk, J}, 0, Dn{T1, J}, sw, 0.0, Csc{Zk, J, 0}, ldz, true);
    if (a > 0) {
      trsm_rLT(st, m, n, a, DnTW{T1 + n, J}, sw, Q, a);
      copy_view(st, m, Csc{Zk, J, n}, ldz, DnRev{T1 + n, J, a}, sw, a, n);
    }
  } else {
    // C (dense lower, ld J) in the first right-hand side's T2; T1 = [W_NN; P W_AN]
    CHD_EW(mk_csc_to_front, (int64_t)J * n, 1, st, T2, 0, J, n, Lk, 0);
    copy_view(st, m, Dn{T1, J}, sw, CscSym{Zk, J}, ldz, n, n);
    if (a > 0) copy_view(st, m, DnRev{T1 + n, J, a}, sw, CscRO{Zk, J, n}, ldz, a, n);
    trsm_rL(st, m, J, n, Dn{T1, J}, sw, T2, J);
    trsm_rL(st, m, n, n, DnTW{T1, J}, sw, T2, J);
    CHD_EW(mk_front_to_csc, (int64_t)J * n, m, st, Zk, ldz, T1, sw, J, J, n, 0, n, 1.0);
    if (a > 0) gemm(st, m, a, n, a, 1.0, TriL{Q, a}, 0, Dn{T1 + n, J}, sw, 0.0, CscRev{Zk, J, n, a}, ldz, false);
  }
}

// Algorithm 3.2 (Cholesky product) for one big front: F = the children's
// blocks + G G^T, G = [C; B]; the N-part of F is X, the A x A block stays.
void product_front(const chd_symbolic* s, const Ctx& st, int k, const double* Lc, double* Xo, double* ws) {
  Front f = front(s, k);
  const int J = f.J, n = f.n;
  double* F = ws + f.foff;
  CHD_EW(mk_copy, (int64_t)J * J, 1, st, F, 0, J, nullptr, 0, 0, J, J, 0.0, 0.0, 1, 0);
  assemble_children(s, st, 1, k, ws, 0);
  gemm(st, 1, J, J, n, 1.0, CscL{Lc + f.base, J}, 0, CscLT{Lc + f.base, J}, 0, 1.0, Dn{F, J}, 0, true);
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Xo + f.base, 0, F, 0, J, J, n, 0, J, 1.0);
}

// S-front of a big front for the completion: S_NN and S_AN from the input's
// columns N_k, V_k = S_{A_k A_k} from the input's later columns.
void complete_load_front(const chd_symbolic* s, const Ctx& st, int k, const double* Sin, double* ws) {
  Front f = front(s, k);
  if (f.a > 0) CHD_EW(mk_gather_saa, (int64_t)f.a * f.a, 1, st, s->dev, k, Sin, ws);
  CHD_EW(mk_csc_to_front, (int64_t)f.J * f.n, 1, st, ws + f.foff, 0, f.J, f.n, Sin + f.base, 0);
}

// With Gq (factored update matrices, Algorithm 4.3): G = P R_k P of
// V_k = R_k R_k^T from Gq instead of chol(V_k); the solves run on S_AN and
// L_AN with reversed rows (Z^T Z is unchanged).
void complete_front(const chd_symbolic* s, const Ctx& st, int k, const double* Sin, double* Lc, double* Wc,
                    double* Dd, double* Vd, double* Rd, const double* Gq, double* ws, double* ldet,
                    int64_t* status) {
  Front f = front(s, k);
  const int J = f.J, n = f.n, a = f.a;
  double* F = ws + f.foff;
  double* T1 = F + (int64_t)J * J;
  double* T2 = T1 + (int64_t)J * n;
  // the S-front F was loaded by complete_load_front
  double* V = Vd + s->v_off[k];
  double* R = Gq ? const_cast<double*>(Gq) + s->v_off[k] : Rd + s->v_off[k];
  if (a > 0) {
    CHD_EW(mk_copy, (int64_t)a * a, 1, st, V, 0, a, F + n + (int64_t)n * J, 0, J, a, a, 1.0, 0.0, 1, 0);
    if (!Gq) {
      CHD_EW(mk_copy, (int64_t)a * a, 1, st, R, 0, a, F + n + (int64_t)n * J, 0, J, a, a, 1.0, 0.0, 1, 0);
      potrf_partial(st, R, a, a, a, status, CHD_ERR_NOT_COMPLETABLE, k, -1);
    }
    CHD_EW(mk_copy, (int64_t)a * n, 1, st, T1 + n, 0, J, F + n, 0, J, a, n, 1.0, 0.0, 0, 0);
    if (Gq) CHD_EW(mk_rev_rows, (int64_t)(a / 2) * n, 1, st, T1 + n, J, a, n);
    trsm_rLT(st, 1, n, a, DnTW{T1 + n, J}, 0, R, a);  // Z = R^{-1} S_AN
  }
  CHD_EW(mk_copy, (int64_t)n * n, 1, st, T1, 0, J, F, 0, J, n, n, 1.0, 0.0, 1, 0);
  if (a > 0) {
    gemm(st, 1, n, n, a, -1.0, DnT{T1 + n, J}, 0, Dn{T1 + n, J}, 0, 1.0, Dn{T1, J}, 0, true);  // P
    CHD_EW(mk_copy, (int64_t)a * n, 1, st, T2 + n, 0, J, T1 + n, 0, J, a, n, -1.0, 0.0, 0, 0);
    trsm_rL(st, 1, n, a, DnTW{T2 + n, J}, 0, R, a);  // L_AN = -R^{-T} Z
    if (Gq) CHD_EW(mk_rev_rows, (int64_t)(a / 2) * n, 1, st, T2 + n, J, a, n);
  }
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Wc + f.base, 0, T1, 0, J, J, n, 0, n, 1.0);
  if (a > 0) CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Wc + f.base, 0, T2, 0, J, J, n, n, J, 1.0);
  // Q = chol(P) in T2[0:n]; D = P^{-1} = Q^{-T} Q^{-1}
  CHD_EW(mk_copy, (int64_t)n * n, 1, st, T2, 0, J, T1, 0, J, n, n, 1.0, 0.0, 1, 0);
  potrf_partial(st, T2, J, n, n, status, CHD_ERR_NOT_COMPLETABLE, k, f.col0);
  double* Dk = Dd + s->d_off[k];
  CHD_EW(mk_identity, (int64_t)n * n, 1, st, Dk, n, n);
  trsm_rLT(st, 1, n, n, DnTW{Dk, n}, 0, T2, J);
  gemm(st, 1, n, n, n, 1.0, TriLT{Dk, n}, 0, TriL{Dk, n}, 0, 0.0, Dn{T1, J}, 0, true);
  CHD_EW(mk_copy, (int64_t)n * n, 1, st, Dk, 0, n, T1, 0, J, n, n, 1.0, 0.0, 1, 0);
  potrf_partial(st, T1, J, n, n, status, CHD_ERR_NOT_COMPLETABLE, k, f.col0);
  CHD_EW(mk_front_to_csc, (int64_t)J * n, 1, st, Lc + f.base, 0, T1, 0, J, J, n, 0, n, 1.0);
  if (a > 0) gemm(st, 1, a, n, n, 1.0, Dn{T2 + n, J}, 0, TriL{T1, J}, 0, 0.0, Csc{Lc + f.base, J, n}, 0, false);
  k_logdet_diag<<<1, BT, 0, st>>>(T1, J, n, ldet + k);
  chd_launch::count_launch();
}

// ---------------------------------------------------------------------------
// Leaf groups: L consecutive one-column leaves c_0 .. c_{L-1} of one parent
// with the same ancestor set A (a = |A|, J = a + 1).  Their value columns are
// consecutive in the CSC (J entries each), so the A-parts of X, Y, S, T, the
// factor blocks and the outputs are a x L blocks with leading dimension J.
// With n = 1 the per-front formulas reduce to scalar and a-vector operations
// per leaf (one warp per leaf) and, across the group, to products with the
// a x L blocks: the update block the parent adds is their sum, and the
// products with V, V' or V^{-1} (the same for every member) cover all leaves.
// Scratch: the members' own workspace fronts, beyond the first member's.
// ---------------------------------------------------------------------------
struct Group {
  int c0, L, a, J, Jp;
  int64_t col0, base0, f0, f1, fp, d0, v0;
  const int32_t* rel;  // device: positions of A in J_parent
  const int32_t* rows; // device: A (global rows)
};
Group group(const chd_symbolic* s, int g) {
  Group G;
  G.c0 = (int)s->grp_first[g];
  G.L = (int)s->grp_count[g];
  G.J = (int)(s->rows_ptr[G.c0 + 1] - s->rows_ptr[G.c0]);
  G.a = G.J - 1;
  const int64_t p = s->sn_par[G.c0];
  G.Jp = (int)(s->rows_ptr[p + 1] - s->rows_ptr[p]);
  G.col0 = s->sn_ptr[G.c0];
  G.base0 = s->colptr[G.col0];
  G.f0 = s->f_off[G.c0];
  G.f1 = s->f_off[G.c0 + 1];
  G.fp = s->f_off[p];
  G.d0 = s->d_off[G.c0];
  G.v0 = s->v_off[G.c0];
  G.rel = s->dev.rel + s->rows_ptr[G.c0] + 1;
  G.rows = s->dev.rows + s->rows_ptr[G.c0] + 1;
  return G;
}
constexpr int GW = BT / 32;  // leaves (warps) per CTA
inline dim3 leaf_grid(int L, int m) { return dim3((L + GW - 1) / GW, 1, m); }
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
#define LEAF_PROLOGUE                                          \
  const int lane = threadIdx.x & 31;                           \
  const int i = blockIdx.x * GW + (threadIdx.x >> 5);          \
  if (i >= L) return;                                          \
  const int64_t z = blockIdx.z;                                \
  const int64_t b = base0 + (int64_t)i * J;

// Algorithm 7.1 for one-column leaves: D = x_jj, L = x_Aj / D, and the
// Cholesky form C = sqrt(D), B = x_Aj / C
__global__ void __launch_bounds__(BT) mg_factor(const double* X, double* Lc, double* Wc, double* Dd, double* ldet,
                                                int64_t base0, int J, int L, int c0, int64_t d0, int64_t col0,
                                                int64_t* st) {
  LEAF_PROLOGUE
  (void)z;
  double d = X[b];
  if (!(d > 0.0)) {
    if (lane == 0) record_error(st, CHD_ERR_NOT_PD, c0 + i, col0 + i);
    d = 1.0;
  }
  const double r = rsqrt(d), r2 = r * r;
  for (int q = 1 + lane; q < J; q += 32) {
    const double x = X[b + q];
    Lc[b + q] = x * r;
    Wc[b + q] = x * r2;
  }
  if (lane == 0) {
    Lc[b] = d * r;
    Wc[b] = r2;
    Dd[d0 + 4 * (int64_t)i] = d;
    ldet[c0 + i] = log(d);
  }
}
// V (a x a, lower) <- parent's front at the relative positions, per RHS z
__global__ void __launch_bounds__(BT) mg_gather_v(const double* ws, int64_t sws, int64_t fp, int Jp,
                                                  const int32_t* rel, int a, double* V, int64_t sV) {
  ws += blockIdx.z * sws;
  V += blockIdx.z * sV;
  const double* Fp = ws + fp;
  const int64_t tot = (int64_t)a * a;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % a), c = (int)(e / a);
    if (r >= c) V[r + (int64_t)c * a] = __ldcg(Fp + __ldg(rel + r) + (int64_t)__ldg(rel + c) * Jp);
  }
}
// V = S_AA (a x a, lower) read from the input S (completion)
__global__ void __launch_bounds__(BT) mg_gather_saa(SymDev S, const int32_t* A, int a, const double* Sin,
                                                    double* V, double* R) {
  const int64_t tot = (int64_t)a * a;
  for (int64_t e = blockIdx.x * (int64_t)EW + threadIdx.x; e < min(tot, (blockIdx.x + 1) * (int64_t)EW); e += BT) {
    const int r = (int)(e % a), c = (int)(e / a);
    if (r >= c) {
      const double v = Sin[csc_find(S, __ldg(A + r), __ldg(A + c))];
      V[r + (int64_t)c * a] = v;
      R[r + (int64_t)c * a] = v;
    }
  }
}
// Algorithm 7.2, after S_AN = -V L: S_NN = D^{-1} - S_AN^T L; g = -S
__global__ void __launch_bounds__(BT) mg_grad_finish(double* Sc, double* g, const double* Wc, int64_t base0,
                                                     int J, int L) {
  LEAF_PROLOGUE
  (void)z;
  double t = 0.0;
  for (int q = 1 + lane; q < J; q += 32) t = fma(Sc[b + q], Wc[b + q], t);
  t = warp_sum(t);
  if (lane == 0) Sc[b] = Wc[b] - t;
  __syncwarp();
  if (g)
    for (int q = lane; q < J; q += 32) g[b + q] = -Sc[b + q];
}
// Hessian step 1 per leaf: K_AN = Y_AN - L Y_NN (into the a x L scratch K)
__global__ void __launch_bounds__(BT) mg_hess_k(const double* Y, int64_t ldy, const double* Wc, double* K,
                                                int64_t sK, int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  const double* y = Y + z * ldy + b;
  double* k = K + z * sK + (int64_t)i * (J - 1);
  const double yn = y[0];
  for (int q = 1 + lane; q < J; q += 32) k[q - 1] = fma(-Wc[b + q], yn, y[q]);
}
// Hessian step 2 per leaf: M_NN = D^{-1} K_NN D^{-1} -> T; K_AN D^{-1} in place
__global__ void __launch_bounds__(BT) mg_hess_m(const double* Y, int64_t ldy, double* T, int64_t ldt,
                                                const double* Wc, double* K, int64_t sK, int64_t base0, int J,
                                                int L) {
  LEAF_PROLOGUE
  const double dinv = Wc[b];
  double* k = K + z * sK + (int64_t)i * (J - 1);
  if (lane == 0) T[z * ldt + b] = dinv * dinv * Y[z * ldy + b];
  for (int q = 1 + lane; q < J; q += 32) k[q - 1] *= dinv;
}
// Hessian step 3 per leaf, after W = V' L: T_NN = M_NN - 2 M_AN^T L + W^T L,
// T_AN = M_AN - W
__global__ void __launch_bounds__(BT) mg_hess_down(double* T, int64_t ldt, const double* Wc, const double* W,
                                                   int64_t sW, int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  double* t = T + z * ldt + b;
  const double* w = W + z * sW + (int64_t)i * (J - 1);
  double s1 = 0.0, s2 = 0.0;
  for (int q = 1 + lane; q < J; q += 32) {
    s1 = fma(t[q], Wc[b + q], s1);
    s2 = fma(w[q - 1], Wc[b + q], s2);
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  for (int q = 1 + lane; q < J; q += 32) t[q] -= w[q - 1];
  if (lane == 0) t[0] = t[0] - 2.0 * s1 + s2;
}
// Inverse-Hessian steps 1-2 per leaf, after W = V' L: M_AN = T_AN + W,
// M_NN = T_NN + T_AN^T L + L^T M_AN, K_NN = D M_NN D -> Y, M_AN D in place of W
__global__ void __launch_bounds__(BT) mg_ihess_down(const double* Tin, int64_t ldt, double* Y, int64_t ldy,
                                                    const double* Wc, const double* Dd, int64_t d0, double* W,
                                                    int64_t sW, int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  const double* t = Tin + z * ldt + b;
  double* w = W + z * sW + (int64_t)i * (J - 1);
  double s1 = 0.0, s2 = 0.0;
  for (int q = 1 + lane; q < J; q += 32) {
    const double l = Wc[b + q], tq = t[q];
    s1 = fma(tq, l, s1);
    s2 = fma(tq + w[q - 1], l, s2);
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  const double d = Dd[d0 + 4 * (int64_t)i];
  for (int q = 1 + lane; q < J; q += 32) w[q - 1] = (t[q] + w[q - 1]) * d;
  if (lane == 0) Y[z * ldy + b] = d * d * (t[0] + s1 + s2);
}
// Inverse-Hessian step 3 per leaf (no children): P = K_AN + 1/2 L K_NN into
// the scratch, Y_AN = K_AN + L K_NN (Y_NN = K_NN stays)
__global__ void __launch_bounds__(BT) mg_ihess_up(double* Y, int64_t ldy, const double* Wc, double* P, int64_t sP,
                                                  int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  double* y = Y + z * ldy + b;
  double* pp = P + z * sP + (int64_t)i * (J - 1);
  const double kn = y[0];
  for (int q = 1 + lane; q < J; q += 32) {
    const double l = Wc[b + q], ka = y[q];
    pp[q - 1] = fma(0.5 * l, kn, ka);
    y[q] = fma(l, kn, ka);
  }
}
// Algorithm 7.3 per leaf, after Z = R^{-1} S_AN (scratch): P = S_NN - Z^T Z
// (kept in Wc's diagonal entry), scratch <- -Z
__global__ void __launch_bounds__(BT) mg_comp_mid(const double* Sin, double* Wc, double* Z, int64_t base0, int J,
                                                  int L) {
  LEAF_PROLOGUE
  (void)z;
  double* zz = Z + (int64_t)i * (J - 1);
  double t = 0.0;
  for (int q = lane; q < J - 1; q += 32) t = fma(zz[q], zz[q], t);
  t = warp_sum(t);
  for (int q = lane; q < J - 1; q += 32) zz[q] = -zz[q];
  if (lane == 0) Wc[b] = Sin[b] - t;
}
// Algorithm 7.3 per leaf, after L_AN = -R^{-T} Z (scratch): D = P^{-1},
// C = sqrt(D), factor blocks and log det
__global__ void __launch_bounds__(BT) mg_comp_finish(double* Lc, double* Wc, double* Dd, double* ldet,
                                                     const double* Z, int64_t base0, int J, int L, int c0,
                                                     int64_t d0, int64_t col0, int64_t* st) {
  LEAF_PROLOGUE
  (void)z;
  double P = Wc[b];
  if (!(P > 0.0)) {
    if (lane == 0) record_error(st, CHD_ERR_NOT_COMPLETABLE, c0 + i, col0 + i);
    P = 1.0;
  }
  const double D = 1.0 / P, C = sqrt(D);
  const double* l = Z + (int64_t)i * (J - 1);
  for (int q = 1 + lane; q < J; q += 32) {
    Wc[b + q] = l[q - 1];
    Lc[b + q] = l[q - 1] * C;
  }
  if (lane == 0) {
    Lc[b] = C;
    Dd[d0 + 4 * (int64_t)i] = D;
    ldet[c0 + i] = 2.0 * log(C);
  }
}

// Algorithm 3.2 per leaf: X_jj = C^2, X_Aj = B C (the group adds +B B^T)
__global__ void __launch_bounds__(BT) mg_product(const double* Lc, double* X, int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  (void)z;
  const double c = Lc[b];
  for (int q = 1 + lane; q < J; q += 32) X[b + q] = Lc[b + q] * c;
  if (lane == 0) X[b] = c * c;
}

// Hessian factor (§5.4): M <-> W of a leaf group (n = 1, C = sqrt(d)):
// dir 0: W_jj = d M_jj, W_Aj = Q^{-1} (C M_Aj); dir 1: M_jj = W_jj / d,
// M_Aj = Q (W_Aj / C).  Q is the group's shared upper factor of V, held as
// Q' = P Q P; the scaled A-rows go to the scratch P in reverse order.
__global__ void __launch_bounds__(BT) mg_rscale(double* Z, int64_t ldz, const double* Lc, double* Pr, int64_t sP,
                                                int dir, int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  double* zz = Z + z * ldz + b;
  const int a = J - 1;
  double* pr = Pr + z * sP + (int64_t)i * a;
  const double c = Lc[b];
  const double s = dir == 0 ? c : 1.0 / c;
  for (int q = 1 + lane; q < J; q += 32) pr[a - q] = zz[q] * s;
  if (lane == 0) zz[0] *= s * s;
}
__global__ void __launch_bounds__(BT) mg_unreverse(double* Z, int64_t ldz, const double* Pr, int64_t sP,
                                                   int64_t base0, int J, int L) {
  LEAF_PROLOGUE
  double* zz = Z + z * ldz + b;
  const int a = J - 1;
  const double* pr = Pr + z * sP + (int64_t)i * a;
  for (int q = 1 + lane; q < J; q += 32) zz[q] = pr[a - q];
}
void group_rtrans(const chd_symbolic* s, const Ctx& st, int m, int g, int dir, const double* Lc, const double* Qd,
                  double* Z, int64_t ldz, double* ws) {
  const Group G = group(s, g);
  const int64_t sw = s->dev.f_total;
  const double* Q = Qd + G.v0;
  double* P = ws + G.f1;  // a x L per RHS
  mg_rscale<<<leaf_grid(G.L, m), BT, 0, st>>>(Z, ldz, Lc, P, sw, dir, G.base0, G.J, G.L);
  chd_launch::count_launch();
  if (dir == 0) {
    trsm_rLT(st, m, G.L, G.a, DnTW{P, G.a}, sw, Q, G.a);
    mg_unreverse<<<leaf_grid(G.L, m), BT, 0, st>>>(Z, ldz, P, sw, G.base0, G.J, G.L);
    chd_launch::count_launch();
  } else {
    gemm(st, m, G.a, G.L, G.a, 1.0, TriL{Q, G.a}, 0, Dn{P, G.a}, sw, 0.0, DnRev{Z + G.base0 + 1, G.J, G.a}, ldz,
         false);
  }
}

// per-group sequences
void group_product(const chd_symbolic* s, const Ctx& st, int g, const double* Lc, double* X, double* ws) {
  const Group G = group(s, g);
  mg_product<<<leaf_grid(G.L, 1), BT, 0, st>>>(Lc, X, G.base0, G.J, G.L);
  chd_launch::count_launch();
  gemm(st, 1, G.a, G.a, G.L, 1.0, Dn{const_cast<double*>(Lc) + G.base0 + 1, G.J}, 0,
       DnT{const_cast<double*>(Lc) + G.base0 + 1, G.J}, 0, 0.0, Dn{ws + G.f0 + 1 + G.J, G.J}, 0, true);
}
void group_factor(const chd_symbolic* s, const Ctx& st, int g, const double* X, double* Lc, double* Wc, double* Dd,
                  double* ws, double* ldet, int64_t* status) {
  const Group G = group(s, g);
  mg_factor<<<leaf_grid(G.L, 1), BT, 0, st>>>(X, Lc, Wc, Dd, ldet, G.base0, G.J, G.L, G.c0, G.d0, G.col0, status);
  chd_launch::count_launch();
  // update block the parent adds: -sum_i B_i B_i^T, in the first member's front
  gemm(st, 1, G.a, G.a, G.L, -1.0, Dn{Lc + G.base0 + 1, G.J}, 0, DnT{Lc + G.base0 + 1, G.J}, 0, 0.0,
       Dn{ws + G.f0 + 1 + G.J, G.J}, 0, true);
}
void group_gradient(const chd_symbolic* s, const Ctx& st, int g, const double* Wc, double* Sc, double* gr,
                    double* Vd, double* ws) {
  const Group G = group(s, g);
  double* V = Vd + G.v0;
  CHD_EW(mg_gather_v, (int64_t)G.a * G.a, 1, st, ws, 0, G.fp, G.Jp, G.rel, G.a, V, 0);
  gemm(st, 1, G.a, G.L, G.a, -1.0, SymL{V, G.a}, 0, Dn{const_cast<double*>(Wc) + G.base0 + 1, G.J}, 0, 0.0,
       Dn{Sc + G.base0 + 1, G.J}, 0, false);
  mg_grad_finish<<<leaf_grid(G.L, 1), BT, 0, st>>>(Sc, gr, Wc, G.base0, G.J, G.L);
  chd_launch::count_launch();
}
void group_hess_up(const chd_symbolic* s, const Ctx& st, int m, int g, const double* Wc, const double* Vd,
                   const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws) {
  const Group G = group(s, g);
  const int64_t sw = s->dev.f_total;
  double* K = ws + G.f1;
  const Dn Lb{const_cast<double*>(Wc) + G.base0 + 1, G.J};
  mg_hess_k<<<leaf_grid(G.L, m), BT, 0, st>>>(Y, ldy, Wc, K, sw, G.base0, G.J, G.L);
  chd_launch::count_launch();
  // U' = -(K_AN L^T + L Y_AN^T), summed over the group
  Dn U{ws + G.f0 + 1 + G.J, G.J};
  gemm(st, m, G.a, G.a, G.L, -1.0, Dn{K, G.a}, sw, DnT{Lb.p, G.J}, 0, 0.0, U, sw, true);
  gemm(st, m, G.a, G.a, G.L, -1.0, Lb, 0, DnT{const_cast<double*>(Y) + G.base0 + 1, G.J}, ldy, 1.0, U, sw, true);
  mg_hess_m<<<leaf_grid(G.L, m), BT, 0, st>>>(Y, ldy, T, ldt, Wc, K, sw, G.base0, G.J, G.L);
  chd_launch::count_launch();
  // M_AN = V (K_AN D^{-1})
  gemm(st, m, G.a, G.L, G.a, 1.0, SymL{const_cast<double*>(Vd) + G.v0, G.a}, 0, Dn{K, G.a}, sw, 0.0,
       Dn{T + G.base0 + 1, G.J}, ldt, false);
}
void group_hess_down(const chd_symbolic* s, const Ctx& st, int m, int g, const double* Wc, double* T, int64_t ldt,
                     double* ws) {
  const Group G = group(s, g);
  const int64_t sw = s->dev.f_total;
  double* Vs = ws + G.f1;
  double* W = Vs + (int64_t)G.a * G.a;
  CHD_EW(mg_gather_v, (int64_t)G.a * G.a, m, st, ws, sw, G.fp, G.Jp, G.rel, G.a, Vs, sw);
  gemm(st, m, G.a, G.L, G.a, 1.0, SymL{Vs, G.a}, sw, Dn{const_cast<double*>(Wc) + G.base0 + 1, G.J}, 0, 0.0,
       Dn{W, G.a}, sw, false);
  mg_hess_down<<<leaf_grid(G.L, m), BT, 0, st>>>(T, ldt, Wc, W, sw, G.base0, G.J, G.L);
  chd_launch::count_launch();
}
void group_ihess_down(const chd_symbolic* s, const Ctx& st, int m, int g, const double* Wc, const double* Dd,
                      const double* Rd, const double* Tin, int64_t ldt, double* Y, int64_t ldy, double* ws) {
  const Group G = group(s, g);
  const int64_t sw = s->dev.f_total;
  double* Vs = ws + G.f1;
  double* W = Vs + (int64_t)G.a * G.a;
  CHD_EW(mg_gather_v, (int64_t)G.a * G.a, m, st, ws, sw, G.fp, G.Jp, G.rel, G.a, Vs, sw);
  gemm(st, m, G.a, G.L, G.a, 1.0, SymL{Vs, G.a}, sw, Dn{const_cast<double*>(Wc) + G.base0 + 1, G.J}, 0, 0.0,
       Dn{W, G.a}, sw, false);
  mg_ihess_down<<<leaf_grid(G.L, m), BT, 0, st>>>(Tin, ldt, Y, ldy, Wc, Dd, G.d0, W, sw, G.base0, G.J, G.L);
  chd_launch::count_launch();
  // K_AN = V^{-1} (M_AN D), V^{-1} of the group in its first member's slot
  gemm(st, m, G.a, G.L, G.a, 1.0, SymL{const_cast<double*>(Rd) + G.v0, G.a}, 0, Dn{W, G.a}, sw, 0.0,
       Dn{Y + G.base0 + 1, G.J}, ldy, false);
}
void group_ihess_up(const chd_symbolic* s, const Ctx& st, int m, int g, const double* Wc, double* Y, int64_t ldy,
                    double* ws) {
  const Group G = group(s, g);
  const int64_t sw = s->dev.f_total;
  double* P = ws + G.f1;
  mg_ihess_up<<<leaf_grid(G.L, m), BT, 0, st>>>(Y, ldy, Wc, P, sw, G.base0, G.J, G.L);
  chd_launch::count_launch();
  // U' = -(P L^T + L P^T), summed over the group
  const Dn Lb{const_cast<double*>(Wc) + G.base0 + 1, G.J};
  Dn U{ws + G.f0 + 1 + G.J, G.J};
  gemm(st, m, G.a, G.a, G.L, -1.0, Dn{P, G.a}, sw, DnT{Lb.p, G.J}, 0, 0.0, U, sw, true);
  gemm(st, m, G.a, G.a, G.L, -1.0, Lb, 0, DnT{P, G.a}, sw, 1.0, U, sw, true);
}
void group_complete(const chd_symbolic* s, const Ctx& st, int g, const double* Sin, double* Lc, double* Wc,
                    double* Dd, double* Vd, double* Rd, const double* Gq, double* ws, double* ldet,
                    int64_t* status) {
  const Group G = group(s, g);
  double* V = Vd + G.v0;
  double* R = Gq ? const_cast<double*>(Gq) + G.v0 : Rd + G.v0;
  double* Z = ws + G.f1;
  CHD_EW(mg_gather_saa, (int64_t)G.a * G.a, 1, st, s->dev, G.rows, G.a, Sin, V, Rd + G.v0);
  if (!Gq) potrf_partial(st, R, G.a, G.a, G.a, status, CHD_ERR_NOT_COMPLETABLE, G.c0, -1);
  // Z = R^{-1} S_AN for all leaves, then P per leaf, then L_AN = -R^{-T} Z
  // (with Gq: G = P R_k P and the rows of S_AN and L_AN reversed)
  CHD_EW(mk_copy, (int64_t)G.a * G.L, 1, st, Z, 0, G.a, Sin + G.base0 + 1, 0, G.J, G.a, G.L, 1.0, 0.0, 0, 0);
  if (Gq) CHD_EW(mk_rev_rows, (int64_t)(G.a / 2) * G.L, 1, st, Z, G.a, G.a, G.L);
  trsm_rLT(st, 1, G.L, G.a, DnTW{Z, G.a}, 0, R, G.a);
  mg_comp_mid<<<leaf_grid(G.L, 1), BT, 0, st>>>(Sin, Wc, Z, G.base0, G.J, G.L);
  chd_launch::count_launch();
  trsm_rL(st, 1, G.L, G.a, DnTW{Z, G.a}, 0, R, G.a);
  if (Gq) CHD_EW(mk_rev_rows, (int64_t)(G.a / 2) * G.L, 1, st, Z, G.a, G.a, G.L);
  mg_comp_finish<<<leaf_grid(G.L, 1), BT, 0, st>>>(Lc, Wc, Dd, ldet, Z, G.base0, G.J, G.L, G.c0, G.d0, G.col0,
                                                   status);
  chd_launch::count_launch();
}

// Factored update matrices (Algorithm 4.3) for front k of the dense tier,
// its parent's G done: gather; the Householder reduction of the rows kept
// from G_parent in panels of fc::NB rows (a panel with nothing to annihilate
// launches nothing), the rows below each panel updated by
// X[t1:, C] -= (X[t1:, C] V T) V^T over the panel's columns C; then
// M = S~ L^{-T}, G~ = chol(A~ - M M^T) with the blocked multi-CTA kernels
// (fc_body.cuh has the layout).
void fc_front(const chd_symbolic* s, const Ctx& st, int k, const double* Sin, double* Gq, double* fcs,
              int64_t* status) {
  const int64_t nk = s->sn_ptr[k + 1] - s->sn_ptr[k];
  const int a = (int)(s->rows_ptr[k + 1] - s->rows_ptr[k] - nk);
  const int64_t p = s->sn_par[k];
  const int np = (int)(s->sn_ptr[p + 1] - s->sn_ptr[p]);
  const int Jp = (int)(s->rows_ptr[p + 1] - s->rows_ptr[p]);
  const int32_t* rel = s->rel.data() + s->rows_ptr[k] + nk;
  int q = 0;
  for (int r = 0; r < a; ++r) q += rel[r] >= np ? 1 : 0;
  const int w = q > 0 ? Jp - rel[a - q] : 0;
  const int pp = a - q;
  double* G = Gq + s->v_off[k];
  CHD_EW(mk_fc_gather, (int64_t)q * w + (int64_t)pp * a, 1, st, s->dev, k, Sin, Gq, fcs);
  if (q > 0) {
    constexpr int NB = fc::NB;
    double* X = fcs + s->fc_off[k];
    double* V = X + (int64_t)q * w;
    double* T = V + (int64_t)w * NB;
    double* VT = T + NB * NB;
    double* Y = VT + (int64_t)w * NB;
    auto rho = [&](int t) { return Jp - 1 - rel[a - 1 - t]; };
    for (int t0 = 0; t0 < q; t0 += NB) {
      const int t1 = std::min(q, t0 + NB);
      bool any = false;
      for (int t = t0; t < t1 && !any; ++t) any = rho(t) > t;
      if (!any) continue;
      const int L = rho(t1 - 1) - t0 + 1;
      k_fc_panel<<<1, BT, 0, st>>>(s->dev, k, t0, t1, L, fcs, status);
      chd_launch::count_launch();
      if (t1 < q) {
        // X row-major (ld w): rows t1.., columns t0.. as the transpose of a
        // column-major block
        const int rows = q - t1;
        double* Xb = X + (int64_t)t1 * w + t0;
        gemm(st, 1, L, NB, NB, 1.0, Dn{V, L}, 0, Dn{T, NB}, 0, 0.0, Dn{VT, L}, 0, false);
        gemm(st, 1, rows, NB, L, 1.0, DnT{Xb, w}, 0, Dn{VT, L}, 0, 0.0, Dn{Y, rows}, 0, false);
        gemm(st, 1, rows, L, NB, -1.0, Dn{Y, rows}, 0, DnT{V, L}, 0, 1.0, DnTW{Xb, w}, 0, false);
      }
    }
    CHD_EW(mk_fc_copy, (int64_t)q * q, 1, st, s->dev, k, Gq, fcs);
  }
  if (pp > 0) {
    double* M = G + q;
    double* At = G + q + (int64_t)q * a;
    if (q > 0) {
      trsm_rLT(st, 1, pp, q, Dn{M, a}, 0, G, a);
      gemm(st, 1, pp, pp, q, -1.0, Dn{M, a}, 0, DnT{M, a}, 0, 1.0, Dn{At, a}, 0, true);
    }
    potrf_partial(st, At, a, pp, pp, status, CHD_ERR_NOT_COMPLETABLE, k, -1);
  }
}

}  // namespace big
}  // namespace chd

namespace chd_launch {
using chd::big::Ctx;
void big_factor(const chd_symbolic* s, const Slot& sl, int k, const double* X,
                double* Lc, double* Wc, double* Dd, double* ws, double* ldet, int64_t* status) {
  if (s->grp_of[k] >= 0) return chd::big::group_factor(s, chd::big::make_ctx(sl), s->grp_of[k], X, Lc, Wc, Dd, ws, ldet, status);
  chd::big::factor_front(s, chd::big::make_ctx(sl), k, X, Lc, Wc, Dd, ws, ldet, status);
}
void big_product(const chd_symbolic* s, const Slot& sl, int k, const double* Lc,
                 double* X, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_product(s, chd::big::make_ctx(sl), s->grp_of[k], Lc, X, ws);
  chd::big::product_front(s, chd::big::make_ctx(sl), k, Lc, X, ws);
}
void big_gradient(const chd_symbolic* s, const Slot& sl, int k, const double* Wc,
                  double* Sc, double* g, double* Vd, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_gradient(s, chd::big::make_ctx(sl), s->grp_of[k], Wc, Sc, g, Vd, ws);
  chd::big::gradient_front(s, chd::big::make_ctx(sl), k, Wc, Sc, g, Vd, ws);
}
void big_hess_up(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                 const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws,
                 const uint8_t* act) {
  // a leaf group has no children; with `act` (pruned Hessian factor) a dense
  // front still runs, skipping pruned children, and gives exact zeros where
  // its own subtree is pruned
  if (s->grp_of[k] >= 0) return chd::big::group_hess_up(s, chd::big::make_ctx(sl), m, s->grp_of[k], Wc, Vd, Y, ldy, T, ldt, ws);
  chd::big::hess_up_front(s, chd::big::make_ctx(sl), m, k, Wc, Vd, Y, ldy, T, ldt, ws, act);
}
void big_hess_down(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                   double* T, int64_t ldt, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_hess_down(s, chd::big::make_ctx(sl), m, s->grp_of[k], Wc, T, ldt, ws);
  chd::big::hess_down_front(s, chd::big::make_ctx(sl), m, k, Wc, T, ldt, ws);
}
void big_ihess_down(const chd_symbolic* s, const Slot& sl, int m, int k,
                    const double* Wc, const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y,
                    int64_t ldy, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_ihess_down(s, chd::big::make_ctx(sl), m, s->grp_of[k], Wc, Dd, Rd, T, ldt, Y, ldy, ws);
  chd::big::ihess_down_front(s, chd::big::make_ctx(sl), m, k, Wc, Dd, Rd, T, ldt, Y, ldy, ws);
}
void big_ihess_up(const chd_symbolic* s, const Slot& sl, int m, int k, const double* Wc,
                  double* Y, int64_t ldy, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_ihess_up(s, chd::big::make_ctx(sl), m, s->grp_of[k], Wc, Y, ldy, ws);
  chd::big::ihess_up_front(s, chd::big::make_ctx(sl), m, k, Wc, Y, ldy, ws);
}
void big_complete(const chd_symbolic* s, const Slot& sl, int k, const double* Sin,
                  double* Lc, double* Wc, double* Dd, double* Vd, double* Rd, const double* Gq, double* ws,
                  double* ldet, int64_t* status) {
  if (s->grp_of[k] >= 0) return chd::big::group_complete(s, chd::big::make_ctx(sl), s->grp_of[k], Sin, Lc, Wc, Dd, Vd, Rd, Gq, ws, ldet, status);
  chd::big::complete_front(s, chd::big::make_ctx(sl), k, Sin, Lc, Wc, Dd, Vd, Rd, Gq, ws, ldet, status);
}
void big_fc(const chd_symbolic* s, const Slot& sl, int k, const double* Sin, double* Gq, double* fcs,
            int64_t* status) {
  chd::big::fc_front(s, chd::big::make_ctx(sl), k, Sin, Gq, fcs, status);
}
void big_rtrans(const chd_symbolic* s, const Slot& sl, int m, int k, int dir,
                const double* Lc, const double* Qd, double* Z, int64_t ldz, double* ws) {
  if (s->grp_of[k] >= 0) return chd::big::group_rtrans(s, chd::big::make_ctx(sl), m, s->grp_of[k], dir, Lc, Qd, Z, ldz, ws);
  chd::big::rtrans_front(s, chd::big::make_ctx(sl), m, k, dir, Lc, Qd, Z, ldz, ws);
}
void big_complete_load(const chd_symbolic* s, cudaStream_t st, int k, const double* Sin, double* ws) {
  if (s->grp_of[k] >= 0) return;  // a leaf group reads S itself
  chd::big::complete_load_front(s, chd::big::make_ctx(st, nullptr, 0), k, Sin, ws);
}
// V_k^{-1} of the cached V_k = S_{A_k A_k} of one front (lower, into Rd),
// and the reversed upper factor of V_k (into Qd), with the multi-CTA
// kernels: for the dense tier and for other fronts with a large V_k.
void big_inv_v(const chd_symbolic* s, const Slot& sl, int k, const double* Vd,
               double* Rd, double* Qd, double* ws, int64_t* status, int what) {
  using namespace chd;
  using namespace chd::big;
  const Ctx st = chd::big::make_ctx(sl);
  const int n = (int)(s->sn_ptr[k + 1] - s->sn_ptr[k]);
  const int a = (int)(s->rows_ptr[k + 1] - s->rows_ptr[k]) - n;
  if (a == 0) return;
  (void)ws;
  if (what & 1) {
    // V^{-1} = W^T W with W = R^{-1}, R = chol(V): blocked Cholesky into the
    // V^{-1} slot, W in the front's workspace, the product (a tensor-core
    // product for large a) back into the slot.  Every inverse-Hessian call
    // then applies V^{-1} with one product per front.
    double* R = Rd + s->v_off[k];
    double* Wk = ws + s->f_off[k];  // a x a inside the front's J x J region
    CHD_EW(mk_copy, (int64_t)a * a, 1, st, R, 0, a, Vd + s->v_off[k], 0, a, a, a, 1.0, 0.0, 1, 0);
    potrf_partial(st, R, a, a, a, status, CHD_ERR_NOT_PD, k, -1);
    CHD_EW(mk_identity, (int64_t)a * a, 1, st, Wk, a, a);
    trsm_rLT(st, 1, a, a, DnTW{Wk, a}, 0, R, a);
    gemm(st, 1, a, a, a, 1.0, TriLT{Wk, a}, 0, TriL{Wk, a}, 0, 0.0, Dn{R, a}, 0, true);
  }
  if (what & 2) {
    // the upper factor Q of V = Q Q^T (Hessian factor, §5.4), held as
    // Q' = chol(P V P) = P Q P
    double* Qk = Qd + s->v_off[k];
    CHD_EW(mk_rev_lower, (int64_t)a * a, 1, st, Qk, Vd + s->v_off[k], a);
    potrf_partial(st, Qk, a, a, a, status, CHD_ERR_NOT_PD, k, -1);
  }
}
}  // namespace chd_launch
