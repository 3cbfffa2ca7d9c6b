// FP64-accurate matrix products on the bf16 tensor cores (tcgen05), by
// splitting every operand into integer digits (Ozaki, Ogita, Oishi, Rump,
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59 (2012): each operand is written as an unevaluated sum of
// low-precision pieces whose pairwise products are exact, and the product
// is assembled from the piece products).
//
// Splitting.  Row r of A (M x K) gets the exponent eA_r with max_k |a_rk| <
// 2^(eA_r - 1); then a_rk 2^-eA_r, |.| < 1/2, is written in balanced base
// 128 with ND = 8 digits,
//     a_rk = 2^eA_r * sum_{s=0..7} d_s 2^(-7(s+1)),   d_s integer, |d_s| <= 64,
// by integer operations on the binary representation (the 53-bit mantissa
// becomes a 56-bit fixed-point fraction; bits below 2^-56 of the row scale
// are rounded).  Column c of B (K x N) likewise, with eB_c and digits e_t.
// Digits are exact in bf16 (7 significant bits).
//
// Products.  A digit-pair product d_s e_t is at most 2^12 in magnitude, so
// a sum of them over K <= 1024 stays below 2^22 and is exact in the FP32
// accumulator.  The pairs are grouped by level l = s + t: level l collects
// l + 1 pairs, exactly for l <= 3 at K <= 1024 (its FP32 sum stays below
// 2^24); for l >= 4 a rounding of the accumulator changes the result by
// less than 2^-50 of K max|a| max|b|.  Levels l >= 8 (pairs beyond the
// digits' own precision) are dropped: together they are below 2^-52 of
// that scale.  The product is then
//     (AB)_rc = 2^(eA_r + eB_c - 14) * sum_{l=0..7} L_l 2^(-7 l),
// with L_l the level sums.  The error is of the order of the classical FP64
// product's bound, 2^-53 K max_k |a_rk| max_k |b_kc|, relative to the row
// and column maxima (not to sum_k |a_rk b_kc|).
//
// Tensor-core mapping (one CTA per 128 x 32 output tile, 4 warps).  The
// eight digit planes of B are stacked along N: a tile of B is 8 x 32 = 256
// rows.  For A digit s, one tcgen05.mma (M = 128, N = (8 - s) * 32, K = 16)
// multiplies it with B digits t = 0 .. 7 - s and accumulates into the TMEM
// columns of levels s .. 7 (level l occupies columns 32 l .. 32 l + 31), so
// every level lands in its own accumulator without any data movement: 8
// MMAs per 16-wide K step, 36 digit pairs.  The first MMA (s = 0, N = 256)
// overwrites all 256 columns, the rest accumulate.  Operands reach shared
// memory by TMA (cp.async.bulk.tensor, 64-byte swizzle, 32-wide K chunks,
// two stages); one thread issues the copies and the MMAs and signals
// through mbarriers; tcgen05.commit releases a stage when its MMAs have
// read it.  The epilogue reads the eight levels from TMEM (tcgen05.ld),
// sums levels 0..3 exactly in an int64 and levels 4..7 in FP32, converts
// once to FP64, scales by the digit exponents (an exponent add) and writes
// beta C + alpha AB through the output view: one or two FP64 operations per
// output instead of a dozen.  Every wait is bounded (about two seconds of the global
// timer): on a timeout the kernel raises an error flag, waits (bounded) for
// the copies it issued, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "chordal_barrier.h"

namespace chd {
namespace tc {

constexpr int ND = 8;        // digits per operand element
constexpr int DBITS = 7;     // bits per digit
constexpr int TM = 128;      // output rows per tile (MMA M)
constexpr int TN = 32;       // output columns per tile (per digit of B)
constexpr int KC = 32;       // K per pipeline stage (64-byte rows of bf16)
constexpr int STAGES = 2;
constexpr int A_STAGE = ND * TM * KC * 2;  // bytes: 64 KiB
constexpr int B_STAGE = ND * TN * KC * 2;  // bytes: 16 KiB
constexpr int SMEM_BYTES = STAGES * (A_STAGE + B_STAGE) + 1024;
constexpr int TMEM_COLS = ND * TN;         // 256: eight levels of 32 columns
constexpr int KMAX = 1024;                 // longest K per tensor-core pass

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after about
// `limit_ns` nanoseconds of the global timer.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (bf16 inputs, FP32 accumulation)
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `bar` once every tcgen05.mma issued so far by this thread is complete
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 8 consecutive 32-bit columns: thread i of the warp gets lane (base lane + i)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 64-byte
// swizzled layout written by TMA: rows of 64 bytes (32 bf16), 8-row groups
// 512 bytes apart (stride byte offset); the leading byte offset is unused
// for swizzled K-major layouts (encoded as 1); descriptor version 1; layout
// type 4 = 64-byte swizzle.  Advancing the start address by 32 bytes
// selects the second 16-wide K step of the row.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(512 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(4) << 61;
  return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// digit splitting
// ---------------------------------------------------------------------------
// exponent e with |x| < 2^(e - 1) for the largest |x| of a row or column
__device__ __forceinline__ int scale_exponent(double amax) {
  if (!(amax > 0.0)) return 0;
  const int E = static_cast<int>((__double_as_longlong(amax) >> 52) & 0x7FF);  // amax < 2^(E - 1022)
  return E - 1021;
}
// ND balanced base-128 digits of x 2^-e (|x 2^-e| < 1/2), most significant first
__device__ __forceinline__ void split_digits(double x, int e, int (&d)[ND]) {
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
  int E = static_cast<int>((bits >> 52) & 0x7FF);
  uint64_t mant = bits & ((1ull << 52) - 1);
  if (E == 0) E = 1;  // zero or subnormal
  else mant |= 1ull << 52;
  // |x| 2^(56 - e) = mant 2^sh, sh <= 2
  const int sh = (E - 1023) - 52 + ND * DBITS - e;
  uint64_t F;
  if (sh >= 0) F = mant << sh;
  else if (sh > -60) F = (mant >> (-sh)) + ((mant >> (-sh - 1)) & 1ull);
  else F = 0;
#pragma unroll
  for (int s = ND - 1; s >= 1; --s) {
    int v = static_cast<int>(F & 127ull);
    F >>= 7;
    if (v >= 64) {
      v -= 128;
      F += 1;
    }
    d[s] = v;
  }
  d[0] = static_cast<int>(F);  // 0 .. 64
  if (bits >> 63) {
#pragma unroll
    for (int s = 0; s < ND; ++s) d[s] = -d[s];
  }
}
__device__ __forceinline__ uint16_t digit_bf16(int v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(v)));
}

// Digit planes are written in two passes over the operands, both parallel
// over rows (columns of B) and 64-wide blocks of K, A and B in the same
// launches (blockIdx.x below `ablocks` works on A):
//   1. k_tc_amax: the largest |entry| of each row of A and each column of
//      B, combined across the K blocks by an integer atomicMax on the bits
//      of the non-negative doubles (order-independent, so deterministic);
//   2. k_tc_digits: each thread turns 8 consecutive K entries of one row
//      (column) into 8 digit planes of 16 bytes each.
// dig[z][s][rows][Kp] (row-major, zero padding), ex[z][rows].
constexpr int SPLIT_ROWS = 32;  // rows per CTA in k_tc_digits
constexpr int SPLIT_K = 64;     // K per CTA in both passes
template <class MA, class MB>
__global__ void __launch_bounds__(128) k_tc_amax(int M, int N, int K, int k0ff, int Mp, int Np, int ablocks, MA A,
                                                 int64_t sA, MB B, int64_t sB, unsigned long long* amA,
                                                 unsigned long long* amB) {
  const int z = blockIdx.z;
  const int kb = blockIdx.y * SPLIT_K, ke = min(K, kb + SPLIT_K);
  double mx = 0.0;
  if ((int)blockIdx.x < ablocks) {
    if (sA == 0 && z > 0) return;  // an operand shared by the batch is split once
    A.p += static_cast<int64_t>(z) * sA;
    const int r = blockIdx.x * 128 + threadIdx.x;
    if (r >= M) return;
    for (int k = kb; k < ke; ++k) mx = fmax(mx, fabs(A.at(r, k0ff + k)));
    if (mx > 0.0) atomicMax(amA + static_cast<int64_t>(z) * Mp + r, static_cast<unsigned long long>(__double_as_longlong(mx)));
  } else {
    if (sB == 0 && z > 0) return;
    B.p += static_cast<int64_t>(z) * sB;
    const int c = (blockIdx.x - ablocks) * 128 + threadIdx.x;
    if (c >= N) return;
    for (int k = kb; k < ke; ++k) mx = fmax(mx, fabs(B.at(k0ff + k, c)));
    if (mx > 0.0) atomicMax(amB + static_cast<int64_t>(z) * Np + c, static_cast<unsigned long long>(__double_as_longlong(mx)));
  }
}
template <class MA, class MB>
__global__ void __launch_bounds__(256) k_tc_digits(int M, int N, int K, int k0ff, int Mp, int Np, int Kp, int ablocks,
                                                   MA A, int64_t sA, MB B, int64_t sB, const unsigned long long* amA,
                                                   const unsigned long long* amB, uint16_t* digA, uint16_t* digB,
                                                   int* exA, int* exB) {
  const int z = blockIdx.z;
  const bool isA = (int)blockIdx.x < ablocks;
  if ((isA ? sA : sB) == 0 && z > 0) return;  // shared operand: split once
  const int r = (isA ? blockIdx.x : blockIdx.x - ablocks) * SPLIT_ROWS + (threadIdx.x & 31);
  const int k0 = blockIdx.y * SPLIT_K + 8 * (threadIdx.x >> 5);
  const int rows = isA ? Mp : Np, lim = isA ? M : N;
  if (r >= rows || k0 >= Kp) return;
  const unsigned long long bits = r < lim ? (isA ? amA : amB)[static_cast<int64_t>(z) * rows + r] : 0ull;
  const int e = scale_exponent(__longlong_as_double(static_cast<long long>(bits)));
  if (blockIdx.y == 0 && threadIdx.x < 32) (isA ? exA : exB)[static_cast<int64_t>(z) * rows + r] = e;
  if (isA) A.p += static_cast<int64_t>(z) * sA;
  else B.p += static_cast<int64_t>(z) * sB;
  uint16_t* D = (isA ? digA : digB) + static_cast<int64_t>(z) * ND * rows * Kp + static_cast<int64_t>(r) * Kp + k0;
  const int64_t plane = static_cast<int64_t>(rows) * Kp;
  uint32_t w[ND][4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    int d0[ND], d1[ND];
    const bool in0 = r < lim && k0 + j < K, in1 = r < lim && k0 + j + 1 < K;
    const double x0 = in0 ? (isA ? A.at(r, k0ff + k0 + j) : B.at(k0ff + k0 + j, r)) : 0.0;
    const double x1 = in1 ? (isA ? A.at(r, k0ff + k0 + j + 1) : B.at(k0ff + k0 + j + 1, r)) : 0.0;
    split_digits(x0, e, d0);
    split_digits(x1, e, d1);
#pragma unroll
    for (int s = 0; s < ND; ++s) w[s][j / 2] = digit_bf16(d0[s]) | (static_cast<uint32_t>(digit_bf16(d1[s])) << 16);
  }
#pragma unroll
  for (int s = 0; s < ND; ++s)
    *reinterpret_cast<uint4*>(D + s * plane) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// 2^e as a double
__device__ __forceinline__ double pow2(int e) {
  return (e > -1020 && e < 1020) ? __longlong_as_double(static_cast<int64_t>(e + 1023) << 52) : ldexp(1.0, e);
}
// v 2^e, exactly: an integer add to the exponent field when the result stays
// normal, else an FP64 multiply
__device__ __forceinline__ double times_pow2(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  if (ex == 0 || ex + e <= 0 || ex + e >= 2047) return v * pow2(e);
  return __longlong_as_double(b + (static_cast<long long>(e) << 52));
}

// ---------------------------------------------------------------------------
// the product of the digit planes: one CTA per 128 x 32 tile of C and batch z
// ---------------------------------------------------------------------------
template <class MC>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N, int Kp,
              int Mp, int Np, const int* exA, const int* exB, double alpha, double beta, MC C, int64_t sC, int lower,
              int tiles_n, int shA, int shB, int64_t* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tm = (blockIdx.x / tiles_n) * TM, tn = (blockIdx.x % tiles_n) * TN;
  if (lower && tn >= tm + TM) return;  // tile strictly above the diagonal
  const int z = blockIdx.z;
  C.p += static_cast<int64_t>(z) * sC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    fence_mbar_init();
    failed = 0;
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int nch = Kp / KC;

  if (threadIdx.x == 0) {
    int loads = 0;   // stage loads issued
    int landed = 0;  // stage loads observed complete
    auto load = [&](int c) {
      const int st = c % STAGES;
      uint8_t* a = sm + st * (A_STAGE + B_STAGE);
      mbar_expect_tx(&full[st], A_STAGE + B_STAGE);
      tma_load_3d(a, &mapA, &full[st], c * KC, tm, (shA ? 0 : z) * ND);
      tma_load_3d(a + A_STAGE, &mapB, &full[st], c * KC, tn, (shB ? 0 : z) * ND);
      ++loads;
    };
    bool ok = true;
    int c = 0;
    load(0);
    for (; c < nch; ++c) {
      const int st = c % STAGES;
      if (!mbar_wait(&full[st], (c / STAGES) & 1)) {
        ok = false;
        break;
      }
      ++landed;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sm + st * (A_STAGE + B_STAGE));
      const uint32_t b0 = a0 + A_STAGE;
#pragma unroll
      for (int q = 0; q < KC / 16; ++q) {
#pragma unroll
        for (int s = 0; s < ND; ++s) {
          const uint64_t ad = desc_sw64(a0 + s * (TM * KC * 2) + q * 32);
          const uint64_t bd = desc_sw64(b0 + q * 32);
          mma_bf16(tmem + s * TN, ad, bd, idesc_bf16(TM, (ND - s) * TN), (c | q | s) != 0 ? 1u : 0u);
        }
      }
      mma_commit(&empty[st]);
      if (c + 1 < nch) {
        // stage (c + 1) % STAGES was last read by the MMAs of chunk c + 1 - STAGES
        if (c + 1 >= STAGES && !mbar_wait(&empty[(c + 1) % STAGES], ((c + 1 - STAGES) / STAGES) & 1)) {
          ok = false;
          break;
        }
        load(c + 1);
      }
    }
    mma_commit(&done);
    if (!ok) {
      failed = 1;
      if (status)
        atomicCAS(reinterpret_cast<unsigned long long*>(status), 0ull,
                  static_cast<unsigned long long>(CHD_ERR_TIMEOUT));
      // let the copies already issued land before the CTA's shared memory is released
      for (int i = landed; i < loads; ++i) mbar_wait(&full[i % STAGES], (i / STAGES) & 1);
    }
  }
  // epilogue: every warp reads its 32 TMEM lanes (rows tm + 32 warp + lane)
  const bool ready = mbar_wait(&done, 0);
  __syncwarp();
  tc_fence_after();
  __syncthreads();
  if (ready && !failed) {
    const int r = tm + warp * 32 + lane;
    const int er = (r < Mp) ? exA[static_cast<int64_t>(shA ? 0 : z) * Mp + r] : 0;
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
#pragma unroll 1
    for (int g = 0; g < TN / 8; ++g) {
      uint32_t v[ND][8];
#pragma unroll
      for (int l = 0; l < ND; ++l) tmem_ld8(lane_addr + l * TN + g * 8, v[l]);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int cc = tn + g * 8 + j;
        // Levels 0..3 are exact integers (below 2^24 for K <= KMAX): their
        // weighted sum I is exact in an int64 (|I| < 2^44), in units of
        // 2^-21 of level 0.  Levels 4..7 fold in FP32 (their rounding is
        // below 2^-50 of K max|a| max|b|) and join I with 11 fractional
        // bits: the sum is X 2^-39, |X| < 2^62, converted once to FP64.
        int64_t I = __float2int_rn(__uint_as_float(v[0][j]));
#pragma unroll
        for (int l = 1; l < 4; ++l) I = I * 128 + __float2int_rn(__uint_as_float(v[l][j]));
        float lo = __uint_as_float(v[7][j]);
        lo = fmaf(lo, 0.0078125f, __uint_as_float(v[6][j]));
        lo = fmaf(lo, 0.0078125f, __uint_as_float(v[5][j]));
        lo = fmaf(lo, 0.0078125f, __uint_as_float(v[4][j]));
        const int64_t X = I * (int64_t(1) << 18) + __float2ll_rn(lo * 2048.0f);
        if (r < M && cc < N && (!lower || r >= cc)) {
          const int ec = exB[static_cast<int64_t>(shB ? 0 : z) * Np + cc];
          double out = times_pow2(__ll2double_rn(X), er + ec - 53);
          if (alpha != 1.0) out = alpha == -1.0 ? -out : alpha * out;
          if (beta != 0.0) out = beta == 1.0 ? out + C.at(r, cc) : fma(beta, C.at(r, cc), out);
          C.at(r, cc) = out;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// 3-D bf16 tensor map over digit planes [planes][rows][Kp] with a
// {KC, box_rows, ND} box and 64-byte swizzle (tc_gemm.cu).
bool make_plane_map(CUtensorMap* map, void* base, int64_t Kp, int64_t rows, int64_t planes, int box_rows);

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
struct Layout {
  int Mp, Np, Kp;
  size_t offB, offEA, offEB, offMA, offMB, bytes;
};
// ba, bb: number of distinct A and B operands in the batch (1 when an
// operand is shared by every product of the batch, else the batch size)
inline Layout layout(int ba, int bb, int M, int N, int K) {
  Layout L;
  L.Mp = static_cast<int>(round_up(M, TM));
  L.Np = static_cast<int>(round_up(N, TN));
  L.Kp = static_cast<int>(round_up(K < KMAX ? K : KMAX, KC));
  const size_t a = static_cast<size_t>(ba) * ND * L.Mp * L.Kp * 2;
  const size_t b = static_cast<size_t>(bb) * ND * L.Np * L.Kp * 2;
  L.offB = static_cast<size_t>(round_up(a, 256));
  L.offEA = L.offB + static_cast<size_t>(round_up(b, 256));
  L.offEB = L.offEA + static_cast<size_t>(round_up(static_cast<int64_t>(ba) * L.Mp * 4, 256));
  L.offMA = L.offEB + static_cast<size_t>(round_up(static_cast<int64_t>(bb) * L.Np * 4, 256));
  L.offMB = L.offMA + static_cast<size_t>(round_up(static_cast<int64_t>(ba) * L.Mp * 8, 256));
  L.bytes = L.offMB + static_cast<size_t>(round_up(static_cast<int64_t>(bb) * L.Np * 8, 256));
  return L;
}
// bf16 tensor-core flops one product executes: per computed 128 x 32 tile
// and 16-wide K step, eight MMAs of N = 256, 224, .., 32 (36 digit pairs)
inline double mma_flops(int M, int N, int K, bool lower) {
  const int64_t tm = round_up(M, TM) / TM, tn = round_up(N, TN) / TN;
  int64_t tiles = 0;
  for (int64_t i = 0; i < tm; ++i)
    for (int64_t j = 0; j < tn; ++j)
      if (!lower || j * TN < (i + 1) * TM) ++tiles;
  int64_t kp = 0;
  for (int k0 = 0; k0 < K || k0 == 0; k0 += KMAX) {
    kp += round_up((K - k0 < KMAX ? K - k0 : KMAX) > 0 ? (K - k0 < KMAX ? K - k0 : KMAX) : 1, KC);
    if (K <= 0) break;
  }
  return static_cast<double>(tiles) * kp * 2.0 * TM * TN * 36;
}
// scratch bytes of one product (digit planes and exponents of one K piece)
inline size_t scratch_bytes(int batch, int M, int N, int K) { return layout(batch, batch, M, N, K).bytes; }
inline size_t scratch_bytes(int ba, int bb, int M, int N, int K) { return layout(ba, bb, M, N, K).bytes; }

// C = beta C + alpha A B (lower triangle of C only if `lower`) for `batch`
// products at the given strides, with FP64-level accuracy on the tensor
// cores.  `scratch` holds at least scratch_bytes(batch, M, N, K) bytes;
// `status` (may be null) receives CHD_ERR_TIMEOUT if a bounded wait ran
// out.  Products with K > KMAX run as K pieces accumulated into C.
template <class MA, class MB, class MC>
cudaError_t gemm(cudaStream_t st, void* scratch, size_t scratch_cap, int64_t* status, int batch, int M, int N, int K,
                 double alpha, MA A, int64_t sA, MB B, int64_t sB, double beta, MC C, int64_t sC, bool lower) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  const int shA = sA == 0 ? 1 : 0, shB = sB == 0 ? 1 : 0;
  const int ba = shA ? 1 : batch, bb = shB ? 1 : batch;
  const Layout L = layout(ba, bb, M, N, K);
  if (L.bytes > scratch_cap || batch * ND > 65535) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  uint8_t* base = static_cast<uint8_t*>(scratch);
  uint16_t* dA = reinterpret_cast<uint16_t*>(base);
  uint16_t* dB = reinterpret_cast<uint16_t*>(base + L.offB);
  int* eA = reinterpret_cast<int*>(base + L.offEA);
  int* eB = reinterpret_cast<int*>(base + L.offEB);
  unsigned long long* mxA = reinterpret_cast<unsigned long long*>(base + L.offMA);
  unsigned long long* mxB = reinterpret_cast<unsigned long long*>(base + L.offMB);
  CUtensorMap mA, mB;
  if (!make_plane_map(&mA, dA, L.Kp, L.Mp, static_cast<int64_t>(ba) * ND, TM) ||
      !make_plane_map(&mB, dB, L.Kp, L.Np, static_cast<int64_t>(bb) * ND, TN))
    return cudaErrorInvalidValue;
  const int tiles_m = L.Mp / TM, tiles_n = L.Np / TN;
  for (int k0 = 0; k0 < K || k0 == 0; k0 += KMAX) {
    const int kk = K - k0 < KMAX ? K - k0 : KMAX;
    const int kblocks = static_cast<int>(round_up(kk > 0 ? kk : 1, SPLIT_K) / SPLIT_K);
    cudaMemsetAsync(mxA, 0, L.bytes - L.offMA, st);
    const int am = (M + 127) / 128, an = (N + 127) / 128;
    k_tc_amax<MA, MB><<<dim3(am + an, kblocks, batch), 128, 0, st>>>(M, N, kk, k0, L.Mp, L.Np, am, A, sA, B, sB,
                                                                     mxA, mxB);
    const int dm = L.Mp / SPLIT_ROWS, dn = L.Np / SPLIT_ROWS;
    k_tc_digits<MA, MB><<<dim3(dm + dn, L.Kp / SPLIT_K + (L.Kp % SPLIT_K ? 1 : 0), batch), 256, 0, st>>>(
        M, N, kk, k0, L.Mp, L.Np, L.Kp, dm, A, sA, B, sB, mxA, mxB, dA, dB, eA, eB);
    k_tc_gemm<MC><<<dim3(tiles_m * tiles_n, 1, batch), 128, SMEM_BYTES, st>>>(
        mA, mB, M, N, L.Kp, L.Mp, L.Np, eA, eB, alpha, k0 == 0 ? beta : 1.0, C, sC, lower ? 1 : 0, tiles_n, shA, shB,
        status);
    if (K <= 0) break;
  }
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace chd
