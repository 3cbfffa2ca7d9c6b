// chd_hessian_noalloc: Hessian products whose front workspace is a fixed
// array compiled into the library instead of memory the library allocates.
//
// Some callers cannot let a library call cudaMalloc while they run: a
// program whose device memory is entirely handed out by its own allocator
// (a framework's caching pool or one arena reserved at start-up, which a
// raw cudaMalloc would bypass or fail against), or a service that forbids
// allocator calls after warm-up because they can block or fragment memory.
// This entry point serves them: it runs the same kernels as chd_hessian,
// but the per-front workspace lives in `g_noalloc_ws` below, a file-scope
// device array every GPU that loads the library holds until the process
// exits.  It allocates nothing itself.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "chd_internal.h"

namespace chd_launch {
void hessian(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, const double* Vd,
             const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws);
}

namespace {

// 2 Mi doubles = 16 MiB of workspace: room for m right-hand sides of a
// pattern when m times its per-right-hand-side workspace fits.
constexpr int64_t kNoAllocWorkspaceDoubles = int64_t(2) << 20;

static __device__ __align__(256) double g_noalloc_ws[kNoAllocWorkspaceDoubles];

// Host code must not use `g_noalloc_ws` as a pointer: on the host that name
// is a stand-in, not the device address.  The device address is looked up
// once per device (with that device current) and kept here for the life of
// the process (a cudaDeviceReset would make it stale; the header says so).
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_ws_addr[kMaxDevices] = {};

chd_status workspace_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return CHD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return CHD_ERR_INVALID;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_ws_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return CHD_ERR_CUDA;
    }
    g_ws_addr[dev] = static_cast<double*>(p);
  }
  *out = g_ws_addr[dev];
  return CHD_OK;
}

}  // namespace

extern "C" chd_status chd_hessian_noalloc(chd_factor* f, int m, const double* y, int64_t ldy, double* t,
                                          int64_t ldt, void* stream) {
  if (!f || m < 0 || (m > 0 && (!y || !t))) return CHD_ERR_INVALID;
  if (m == 0) return CHD_OK;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (ldy < nnz || ldt < nnz)) return CHD_ERR_INVALID;
  // The projected inverse must already be cached by chd_gradient or
  // chd_hessian: computing it here would need the factor's own workspace.
  if (!f->have_S) return CHD_ERR_INVALID;
  // Reject what does not fit the fixed workspace.
  const int64_t per_rhs = f->sym->dev.f_total;
  if (per_rhs <= 0 || per_rhs > kNoAllocWorkspaceDoubles / m) return CHD_ERR_INVALID;
  if (m > 65535) return CHD_ERR_INVALID;  // one launch sequence indexes the RHS in a grid dimension
  double* ws = nullptr;
  const chd_status rc = workspace_address(&ws);
  if (rc != CHD_OK) return rc;
  // Every workspace entry the Hessian passes read is written earlier in the
  // same call, so no clearing is needed between calls.
  // The dense tier runs on the caller's stream without split-K here (no
  // scratch beyond the array).
  chd_launch::hessian(f->sym, static_cast<cudaStream_t>(stream), nullptr, m, f->Wc, f->Vd, y, ldy, t, ldt, ws);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHD_OK : CHD_ERR_CUDA;
}
