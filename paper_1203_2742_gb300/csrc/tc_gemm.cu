// Host side of the tensor-core products (tc_gemm.cuh): tensor-map encoding,
// the C-ABI entry that runs one emulated FP64 product on caller memory (a
// test and measurement utility), and a probe of the raw bf16 tcgen05.mma
// throughput.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "chd_internal.h"
#include "front_views.cuh"
#include "tc_gemm.cuh"

namespace chd {
namespace tc {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

bool make_plane_map(CUtensorMap* map, void* base, int64_t Kp, int64_t rows, int64_t planes, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (Kp % KC) || rows % box_rows) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(Kp), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(planes)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(Kp * 2), static_cast<cuuint64_t>(Kp * rows * 2)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(KC), static_cast<cuuint32_t>(box_rows),
                             static_cast<cuuint32_t>(ND)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Raw MMA throughput: every CTA issues `reps` tcgen05.mma of shape
// 128 x 256 x 16 (bf16 in, FP32 accumulate) on zeroed shared memory.
__global__ void __launch_bounds__(128, 1) k_probe_mma(int reps, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  constexpr int BYTES = 24576;  // A: 128 rows, B: 256 rows, 64-byte rows
  for (int i = threadIdx.x; i < BYTES / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    mbar_init(&done, 1);
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(&tmem_base, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint64_t ad = desc_sw64(smem_u32(sm));
    const uint64_t bd = desc_sw64(smem_u32(sm + 8192));
    for (int i = 0; i < reps; ++i) mma_bf16(tmem, ad, bd, idesc_bf16(128, 256), i > 0 ? 1u : 0u);
    mma_commit(&done);
  }
  if (!mbar_wait(&done, 0) && threadIdx.x == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 256);
}

}  // namespace tc
}  // namespace chd

namespace chd_launch {
size_t tc_scratch_bytes(int batch, int M, int N, int K) { return chd::tc::scratch_bytes(batch, batch, M, N, K); }
}  // namespace chd_launch

using namespace chd;

extern "C" {

chd_status chd_dgemm_tc(int64_t m, int64_t n, int64_t k, double alpha, const double* a, int64_t lda, const double* b,
                        int64_t ldb, double beta, double* c, int64_t ldc, void* stream) {
  if (m < 0 || n < 0 || k < 0 || m > (1 << 30) || n > (1 << 30) || k > (1 << 30) || (m && !c) ||
      (m && k && (!a || lda < m)) || (n && k && (!b || ldb < k)) || (m && ldc < m))
    return CHD_ERR_INVALID;
  if (m == 0 || n == 0) return CHD_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = tc::scratch_bytes(1, static_cast<int>(m), static_cast<int>(n), static_cast<int>(k));
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, bytes + 256, st) != cudaSuccess) return CHD_ERR_OOM;
  int64_t* err = reinterpret_cast<int64_t*>(static_cast<uint8_t*>(scratch) + bytes);
  chd_status rc = CHD_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int64_t), st) != cudaSuccess) rc = CHD_ERR_CUDA;
  if (rc == CHD_OK &&
      tc::gemm(st, scratch, bytes, err, 1, static_cast<int>(m), static_cast<int>(n), static_cast<int>(k), alpha,
               Dn{const_cast<double*>(a), lda}, 0, Dn{const_cast<double*>(b), ldb}, 0, beta, Dn{c, ldc}, 0,
               false) != cudaSuccess)
    rc = CHD_ERR_CUDA;
  int64_t h = 0;
  if (rc == CHD_OK && (cudaMemcpyAsync(&h, err, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
    rc = CHD_ERR_CUDA;
  cudaFreeAsync(scratch, st);
  if (rc == CHD_OK && h) rc = CHD_ERR_TIMEOUT;
  return rc;
}

chd_status chd_probe_tc_bf16_peak(void* stream, double* tflops) {
  if (!tflops) return CHD_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return CHD_ERR_CUDA;
  if (cudaFuncSetAttribute(tc::k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, 24576 + 1024) !=
      cudaSuccess)
    return CHD_ERR_CUDA;
  int* err = nullptr;
  if (cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess) return CHD_ERR_OOM;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = 20000;
  tc::k_probe_mma<<<sms, 128, 24576 + 1024, st>>>(200, err);  // warm-up
  cudaEventRecord(e0, st);
  tc::k_probe_mma<<<sms, 128, 24576 + 1024, st>>>(reps, err);
  cudaEventRecord(e1, st);
  int h = 0;
  chd_status rc = CHD_OK;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rc = CHD_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(err, st);
  if (rc != CHD_OK) return rc;
  if (h) return CHD_ERR_TIMEOUT;
  *tflops = 2.0 * 128 * 256 * 16 * static_cast<double>(reps) * sms / (ms * 1e-3) / 1e12;
  return CHD_OK;
}

}  // extern "C"
