// C ABI of the chordal log-det barrier library: object lifetime, device
// memory, argument checks and the launch sequence of every operation.
// Declarations and the contract of each call: include/chordal_barrier.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "chd_internal.h"

namespace chd_launch {
int64_t launches();
int64_t split_k_launches();
double tc_flops();
size_t tc_scratch_bytes(int batch, int M, int N, int K);
void add_launches(int64_t d);
void factor(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* X, double* Lc,
            double* Wc, double* Dd, double* ws, double* ldet, int64_t* status);
void gradient(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Wc, double* Sc,
              double* g, double* Vd, double* ws);
void hessian(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc,
             const double* Vd, const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws);
void inv_hessian(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc,
                 const double* Dd, const double* Rd, const double* T, int64_t ldt, double* Y, int64_t ldy,
                 double* ws);
void complete(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Sin, double* Lc,
              double* Wc, double* Dd, double* Vd, double* Rd, double* Gq, double* fcs, double* ws, double* ldet,
              int64_t* status);
void inv_v(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Vd, double* Rd, double* Qd,
           double* ws, int64_t* status, int what);
void hess_up_pass(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, const double* Vd,
                  const double* Y, int64_t ldy, double* T, int64_t ldt, double* ws, const uint8_t* act);
void prune_mask(const chd_symbolic* s, cudaStream_t st, int m, const double* Y, int64_t ldy, int32_t* cnt,
                uint8_t* act);
void hess_down_pass(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, const double* Wc, double* T,
                    int64_t ldt, double* ws);
void rtrans(const chd_symbolic* s, cudaStream_t st, const Exec* ex, int m, int dir, const double* Lc,
            const double* Qd, double* Z, int64_t ldz, double* ws, const uint8_t* act);
void product(const chd_symbolic* s, cudaStream_t st, const Exec* ex, const double* Lc, double* X, double* ws);
int64_t schur_scratch(const chd_symbolic* s, int m);
void schur(const chd_symbolic* s, cudaStream_t st, int m, const double* A, int64_t lda, const double* T, int64_t ldt,
           double* H, double* scratch);
void sum(cudaStream_t st, const double* v, int64_t m, double* out);
void segsum(cudaStream_t st, const double* v, const int64_t* seg, int nseg, double* out);
void export_ldl(const chd_symbolic* s, cudaStream_t st, const double* Lc, double* l, double* d);
cudaError_t fp64_peak(cudaStream_t st, double* gflops);
}  // namespace chd_launch


namespace {

// Largest workspace (bytes) a Hessian-type call may hold; larger batches of
// right-hand sides are processed in chunks.
constexpr size_t kWorkspaceCap = size_t(48) << 30;

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch of the dense tier per stream: 2 Mi doubles (16 MiB) for the first
// kWideSlices streams, 64 Ki doubles for the others.
constexpr int64_t kSplitScratch = int64_t(2) << 20;
constexpr int64_t kSmallScratch = int64_t(64) << 10;
inline int64_t slice_doubles(int j) { return j < kWideSlices ? kSplitScratch : kSmallScratch; }

chd_status cuda_ok(cudaError_t e) {
  if (e == cudaSuccess) return CHD_OK;
  return e == cudaErrorMemoryAllocation ? CHD_ERR_OOM : CHD_ERR_CUDA;
}

chd_status alloc_factor(chd_symbolic* s, cudaStream_t stream, chd_factor** out) {
  chd_factor* f = new (std::nothrow) chd_factor();
  if (!f) return CHD_ERR_OOM;
  f->sym = s;
  f->stream = stream;
  const size_t nnz = (size_t)s->colptr[s->n];
  size_t off = 0;
  const size_t oLc = off; off = align_up(off + nnz * 8);
  const size_t oWc = off; off = align_up(off + nnz * 8);
  const size_t oSc = off; off = align_up(off + nnz * 8);
  const size_t oDd = off; off = align_up(off + (size_t)s->d_off[s->nsn] * 8);
  const size_t oVd = off; off = align_up(off + (size_t)s->v_off[s->nsn] * 8);
  const size_t oRd = off; off = align_up(off + (size_t)s->v_off[s->nsn] * 8);
  const size_t oQd = off; off = align_up(off + (size_t)s->v_off[s->nsn] * 8);
  const size_t old = off; off = align_up(off + (size_t)s->nsn * 8);
  const size_t osc = off; off = align_up(off + 4 * 8);
  const size_t ost = off; off = align_up(off + 4 * 8);
  // split-K scratch: one slice per stream (caller's + side streams), only
  // for patterns that have dense-tier fronts
  bool any_big = false;
  for (char b : s->is_big) any_big = any_big || b;
  const int nside = any_big ? kSideStreams : 0;
  const size_t oxs = off;
  size_t xs_doubles = 0;
  if (any_big) {
    for (int j = 0; j <= nside; ++j) xs_doubles += (size_t)slice_doubles(j);
    off = align_up(off + xs_doubles * 8);
  }
  // tensor-core product scratch (digit planes): one slice for the caller's
  // stream and for each side stream, sized for the largest dense front's
  // products (up to eight right-hand sides at once on the caller's stream,
  // two on a side stream; a call with more right-hand sides runs them in
  // turn, and a product that does not fit runs on the FP64 units)
  size_t tc_slice[kSideStreams + 1] = {};
  const size_t otc = off;
  if (any_big && s->tc_mode >= 0) {
    int64_t jmax = 0;
    for (int64_t k = 0; k < s->nsn; ++k)
      if (s->is_big[k]) jmax = std::max<int64_t>(jmax, front_J(s, k));
    if (jmax >= 64) {
      const size_t need = chd_launch::tc_scratch_bytes(1, (int)jmax, (int)jmax, (int)jmax);
      for (int j = 0; j <= nside; ++j) {
        tc_slice[j] = align_up(std::min<size_t>(j == 0 ? (size_t(256) << 20) : (size_t(48) << 20),
                                                (j == 0 ? 8 : 2) * need));
        off += tc_slice[j];
      }
    }
  }
  void* block = nullptr;
  chd_status rc = cuda_ok(cudaMalloc(&block, off));
  if (rc != CHD_OK) { delete f; return rc; }
  char* b = static_cast<char*>(block);
  f->block = block;
  f->Lc = reinterpret_cast<double*>(b + oLc);
  f->Wc = reinterpret_cast<double*>(b + oWc);
  f->Sc = reinterpret_cast<double*>(b + oSc);
  f->Dd = reinterpret_cast<double*>(b + oDd);
  f->Vd = reinterpret_cast<double*>(b + oVd);
  f->Rd = reinterpret_cast<double*>(b + oRd);
  f->Qd = reinterpret_cast<double*>(b + oQd);
  f->ldet = reinterpret_cast<double*>(b + old);
  f->scalar = reinterpret_cast<double*>(b + osc);
  f->status = reinterpret_cast<int64_t*>(b + ost);
  f->ex.status = f->status;
  f->ex.tc_mode = s->tc_mode;
  {
    char* t = b + otc;
    for (int j = 0; j <= kSideStreams; ++j) {
      f->ex.tc[j] = tc_slice[j] ? t : nullptr;
      f->ex.tc_cap[j] = tc_slice[j];
      t += tc_slice[j];
    }
  }
  if (any_big) {
    double* x = reinterpret_cast<double*>(b + oxs);
    for (int j = 0; j <= nside; ++j) {
      f->ex.slice[j] = x;
      f->ex.slice_cap[j] = slice_doubles(j);
      x += slice_doubles(j);
    }
    bool ok = cudaEventCreateWithFlags(&f->ex.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; ok && j < nside; ++j) {
      ok = cudaStreamCreateWithFlags(&f->ex.side[j], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&f->ex.join[j], cudaEventDisableTiming) == cudaSuccess;
      if (ok) f->ex.nside = j + 1;
    }
    if (!ok) {
      cudaGetLastError();
      f->ex.nside = 0;  // run every big front on the caller's stream
    }
  }
  if (cudaStreamCreateWithFlags(&f->gs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->g_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->g_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    f->graphs_on = false;  // run every sequence directly
  }
  rc = cuda_ok(cudaMemsetAsync(f->status, 0, 4 * 8, stream));
  // the scratch slices end with the counters of the Cholesky panel kernel
  if (rc == CHD_OK && any_big)
    rc = cuda_ok(cudaMemsetAsync(f->ex.slice[0], 0, xs_doubles * 8, stream));
  if (rc != CHD_OK) { cudaFree(block); delete f; return rc; }
  *out = f;
  return CHD_OK;
}

// Workspaces are stream-ordered allocations on the calling stream: growing or
// releasing one never synchronises the device, so calls on other factors
// (other streams) keep running.  Each ends with a guard region of 1 MiB that
// no front uses: a stream-ordered allocation can end where the pool's mapped
// memory ends, and a read just past the last front's region must not reach
// unmapped memory.
constexpr size_t kWsGuard = size_t(1) << 20;
chd_status ensure_ws(chd_factor* f, int64_t rhs) {
  if (f->ws_rhs >= rhs) return CHD_OK;
  if (f->ws) {
    cudaFreeAsync(f->ws, f->stream);
    f->ws = nullptr;
    f->ws_rhs = 0;
  }
  void* p = nullptr;
  const size_t bytes = (size_t)f->sym->dev.f_total * 8 * (size_t)rhs + kWsGuard;
  chd_status rc = cuda_ok(cudaMallocAsync(&p, bytes, f->stream));
  if (rc != CHD_OK) return rc;
  f->ws = static_cast<double*>(p);
  f->ws_rhs = rhs;
  return CHD_OK;
}

// per (right-hand side, front) counts and flags of the pruned Hessian factor
chd_status ensure_act(chd_factor* f, int64_t rhs) {
  if (f->act_rhs >= rhs) return CHD_OK;
  if (f->act_buf) {
    cudaFreeAsync(f->act_buf, f->stream);
    f->act_buf = nullptr;
    f->act_rhs = 0;
  }
  void* p = nullptr;
  const size_t bytes = (size_t)f->sym->nsn * 5 * (size_t)rhs + kWsGuard;
  chd_status rc = cuda_ok(cudaMallocAsync(&p, bytes, f->stream));
  if (rc != CHD_OK) return rc;
  f->act_buf = p;
  f->act_rhs = rhs;
  return CHD_OK;
}

// Right-hand sides processed per launch sequence: bounded by the workspace
// cap and by the grid dimension that indexes them (blockIdx.y or .z, at
// most 65535).
constexpr int64_t kMaxRhsPerLaunch = 65535;
int64_t rhs_chunk(const chd_factor* f, int m) {
  const size_t per = std::max<size_t>((size_t)f->sym->dev.f_total * 8, 1);
  const size_t cap = f->ws_limit ? std::min(f->ws_limit, kWorkspaceCap) : kWorkspaceCap;
  int64_t c = (int64_t)(cap / per);
  return std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(c, m), kMaxRhsPerLaunch));
}

chd_status launch_status() { return cuda_ok(cudaGetLastError()); }

// ---------------------------------------------------------------------------
// CUDA graphs.  The launch sequence of a call depends only on the symbolic
// object and on the call's arguments (device pointers, m, strides), and a
// large pattern issues thousands of launches per call.  A call whose
// arguments equal those of the previous call of the same kind therefore
// captures the sequence into a graph (stream capture on the object's private
// stream gs, thread-local mode), and every later call with the same
// arguments replays it: gs waits for the caller's stream, runs the graph,
// and the caller's stream waits for gs (events; no host synchronisation).
// The first call with new arguments runs the sequence directly on the
// caller's stream, so one-off calls never pay for a capture.  The key holds
// the workspace pointer too: a reallocated workspace invalidates the graph.
// ---------------------------------------------------------------------------
chd_status replay(chd_factor* f, GraphSlot& g) {
  chd_status rc = cuda_ok(cudaEventRecord(f->g_in, f->stream));
  if (rc == CHD_OK) rc = cuda_ok(cudaStreamWaitEvent(f->gs, f->g_in, 0));
  if (rc == CHD_OK) rc = cuda_ok(cudaGraphLaunch(g.exec, f->gs));
  if (rc == CHD_OK) rc = cuda_ok(cudaEventRecord(f->g_out, f->gs));
  if (rc == CHD_OK) rc = cuda_ok(cudaStreamWaitEvent(f->stream, f->g_out, 0));
  if (rc == CHD_OK) chd_launch::add_launches(g.launches);
  return rc;
}

void drop_graph(GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.seen = false;
}

// Sequences longer than this are never captured: instantiating a graph of
// tens of thousands of nodes costs seconds, more than replays save.

template <class Body>
chd_status run_sequence(chd_factor* f, GraphKind kind, GraphKey key, Body&& body) {
  key.p[3] = f->ws;
  GraphSlot& g = f->graphs[kind];
  if (!f->graphs_on || !f->gs) {
    body(f->stream);
    return launch_status();
  }
  if (g.exec && g.key == key) return replay(f, g);
  const bool same = g.seen && g.key == key;
  if (!same) {
    drop_graph(g);
    g.key = key;
    g.seen = true;
    g.capture_failed = false;
  }
  if (!same || g.capture_failed || g.launches > f->graph_limit) {
    const int64_t l0 = chd_launch::launches();
    body(f->stream);
    g.launches = chd_launch::launches() - l0;  // length of the direct run
    return launch_status();
  }
  const int64_t l0 = chd_launch::launches();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(f->gs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    body(f->gs);
    e = cudaStreamEndCapture(f->gs, &graph);
  }
  const int64_t captured = chd_launch::launches() - l0;
  chd_launch::add_launches(-captured);  // captured, not run
  if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || !g.exec) {
    // no graph for this call: run the sequence directly (and do not try to
    // capture it again for these arguments)
    cudaGetLastError();
    g.exec = nullptr;
    g.capture_failed = true;
    body(f->stream);
    return launch_status();
  }
  g.launches = captured;
  return replay(f, g);
}

chd_status ensure_projected_inverse(chd_factor* f) {
  if (f->have_S) return CHD_OK;
  chd_status rc = ensure_ws(f, 1);
  if (rc != CHD_OK) return rc;
  GraphKey key;
  rc = run_sequence(f, G_GRADIENT, key, [&](cudaStream_t st) {
    chd_launch::gradient(f->sym, st, &f->ex, f->Wc, f->Sc, nullptr, f->Vd, f->ws);
  });
  if (rc == CHD_OK) f->have_S = true;
  return rc;
}

// V_k^{-1} (Rd) of every front, once per factor; needs the projected inverse.
chd_status ensure_inv_v(chd_factor* f) {
  if (f->have_R) return CHD_OK;
  chd_status rc = run_sequence(f, G_INV_V, GraphKey{}, [&](cudaStream_t st) {
    chd_launch::inv_v(f->sym, st, &f->ex, f->Vd, f->Rd, f->Qd, f->ws, f->status, 1);
  });
  if (rc == CHD_OK) f->have_R = true;
  return rc;
}
// the reversed upper factors of every V_k (Qd) for the Hessian factor, once
// per factor; needs the projected inverse.
chd_status ensure_q(chd_factor* f) {
  if (f->have_Q) return CHD_OK;
  chd_status rc = run_sequence(f, G_Q, GraphKey{}, [&](cudaStream_t st) {
    chd_launch::inv_v(f->sym, st, &f->ex, f->Vd, f->Rd, f->Qd, f->ws, f->status, 2);
  });
  if (rc == CHD_OK) f->have_Q = true;
  return rc;
}

chd_status read_status(chd_factor* f) {
  int64_t h[4] = {0, 0, 0, 0};
  chd_status rc = cuda_ok(cudaMemcpyAsync(h, f->status, sizeof(h), cudaMemcpyDeviceToHost, f->stream));
  if (rc != CHD_OK) return rc;
  rc = cuda_ok(cudaStreamSynchronize(f->stream));
  if (rc != CHD_OK) return rc;
  return static_cast<chd_status>(h[0]);
}

}  // namespace

extern "C" {

chd_status chd_analyze(int64_t n, const int64_t* colptr, const int32_t* rowind, const chd_opts* opts,
                       chd_symbolic** out) {
  if (!out) return CHD_ERR_INVALID;
  *out = nullptr;
  chd_opts o;
  if (opts) o = *opts;
  else chd_opts_default(&o);
  chd_symbolic* s = new (std::nothrow) chd_symbolic();
  if (!s) return CHD_ERR_OOM;
  chd_status rc;
  try {
    rc = chd_symbolic_build(n, colptr, rowind, o, s);
  } catch (const std::bad_alloc&) {
    rc = CHD_ERR_OOM;
  }
  if (rc == CHD_OK) {
    s->inst_n = {0, s->n};
    s->inst_nnz = {0, s->colptr[s->n]};
    s->inst_sn = {0, s->nsn};
    rc = chd_symbolic_upload(s);
  }
  if (rc != CHD_OK) {
    chd_symbolic_free(s);
    return rc;
  }
  *out = s;
  return CHD_OK;
}

chd_status chd_symbolic_info(const chd_symbolic* s, int64_t* n, int64_t* nnz, const int64_t** colptr,
                             const int32_t** rowind, const int64_t** perm, int64_t* nsuper) {
  if (!s) return CHD_ERR_INVALID;
  if (n) *n = s->n;
  if (nnz) *nnz = s->colptr[s->n];
  if (colptr) *colptr = s->colptr.data();
  if (rowind) *rowind = s->rowind.data();
  if (perm) *perm = s->perm.data();
  if (nsuper) *nsuper = s->nsn;
  return CHD_OK;
}

chd_status chd_analyze_batch(int64_t count, const int64_t* n, const int64_t* const* colptr,
                             const int32_t* const* rowind, const chd_opts* opts, chd_symbolic** out) {
  if (!out || count < 1 || !n || !colptr || !rowind) return CHD_ERR_INVALID;
  *out = nullptr;
  chd_symbolic* s = nullptr;
  chd_status rc = CHD_OK;
  try {
    std::vector<int64_t> off(count + 1, 0);
    for (int64_t i = 0; i < count; ++i) {
      if (n[i] < 1 || !colptr[i] || !rowind[i]) return CHD_ERR_INVALID;
      off[i + 1] = off[i] + n[i];
    }
    const int64_t N = off[count];
    std::vector<int64_t> ucp(N + 1, 0), uperm(N);
    std::vector<int32_t> uri;
    for (int64_t i = 0; i < count; ++i) {
      chd_opts oi;
      if (opts) oi = opts[i];
      else chd_opts_default(&oi);
      std::vector<int64_t> pi;
      rc = chd_order_pattern(n[i], colptr[i], rowind[i], oi, pi);
      if (rc != CHD_OK) return rc;
      for (int64_t j = 0; j < n[i]; ++j) {
        uperm[off[i] + j] = off[i] + pi[j];
        for (int64_t q = colptr[i][j]; q < colptr[i][j + 1]; ++q) uri.push_back((int32_t)(rowind[i][q] + off[i]));
        ucp[off[i] + j + 1] = (int64_t)uri.size();
      }
    }
    chd_opts o;
    if (opts) o = opts[0];
    else chd_opts_default(&o);
    o.ordering = CHD_ORDER_USER;
    o.user_perm = uperm.data();
    s = new chd_symbolic();
    rc = chd_symbolic_build(N, ucp.data(), uri.data(), o, s);
    if (rc == CHD_OK) {
      // the postorder keeps every instance's columns together and in place
      for (int64_t i = 0; i < count && rc == CHD_OK; ++i)
        for (int64_t j = off[i]; j < off[i + 1]; ++j)
          if (s->perm[j] < off[i] || s->perm[j] >= off[i + 1]) {
            rc = CHD_ERR_INVALID;
            break;
          }
    }
    if (rc == CHD_OK) {
      s->inst_n = off;
      s->inst_nnz.assign(count + 1, 0);
      s->inst_sn.assign(count + 1, 0);
      for (int64_t i = 0; i <= count; ++i) {
        s->inst_nnz[i] = s->colptr[off[i]];
        s->inst_sn[i] = std::lower_bound(s->sn_ptr.begin(), s->sn_ptr.end(), off[i]) - s->sn_ptr.begin();
        if (s->sn_ptr[s->inst_sn[i]] != off[i]) rc = CHD_ERR_INVALID;  // a supernode straddles instances
      }
    }
    if (rc == CHD_OK) rc = chd_symbolic_upload(s);
  } catch (const std::bad_alloc&) {
    rc = CHD_ERR_OOM;
  }
  if (rc != CHD_OK) {
    chd_symbolic_free(s);
    return rc;
  }
  *out = s;
  return CHD_OK;
}

chd_status chd_symbolic_batch_info(const chd_symbolic* s, int64_t* count, const int64_t** n_off,
                                   const int64_t** nnz_off) {
  if (!s) return CHD_ERR_INVALID;
  if (count) *count = (int64_t)s->inst_n.size() - 1;
  if (n_off) *n_off = s->inst_n.data();
  if (nnz_off) *nnz_off = s->inst_nnz.data();
  return CHD_OK;
}

chd_status chd_symbolic_supernodes(const chd_symbolic* s, const int64_t** snode_ptr,
                                   const int64_t** snode_par, const int64_t** rows_ptr,
                                   const int32_t** rows) {
  if (!s) return CHD_ERR_INVALID;
  if (snode_ptr) *snode_ptr = s->sn_ptr.data();
  if (snode_par) *snode_par = s->sn_par.data();
  if (rows_ptr) *rows_ptr = s->rows_ptr.data();
  if (rows) *rows = s->rows.data();
  return CHD_OK;
}

chd_status chd_symbolic_schedule(const chd_symbolic* s, int64_t* nlevels, int64_t* ntasks, const int32_t** lvl_ptr,
                                 const int32_t** lvl_counts, const int32_t** task_ptr, const int32_t** task_fronts) {
  if (!s || !nlevels || !ntasks || !lvl_ptr || !lvl_counts || !task_ptr || !task_fronts) return CHD_ERR_INVALID;
  *nlevels = (int64_t)s->lvl_ptr.size() - 1;
  *ntasks = (int64_t)s->task_ptr.size() - 1;
  *lvl_ptr = s->lvl_ptr.data();
  *lvl_counts = s->lvl_counts.data();
  *task_ptr = s->task_ptr.data();
  *task_fronts = s->task_fronts.data();
  return CHD_OK;
}

chd_status chd_symbolic_flops(const chd_symbolic* s, double out[5]) {
  if (!s || !out) return CHD_ERR_INVALID;
  for (int i = 0; i < 5; ++i) out[i] = s->flops[i];
  return CHD_OK;
}

chd_status chd_symbolic_offsets(const chd_symbolic* s, const int64_t** f_off, const int64_t** d_off,
                                const int64_t** v_off) {
  if (!s || !f_off || !d_off || !v_off) return CHD_ERR_INVALID;
  *f_off = s->f_off.data();
  *d_off = s->d_off.data();
  *v_off = s->v_off.data();
  return CHD_OK;
}

chd_status chd_completion_plan(const chd_symbolic* s, int64_t* nlevels, int64_t* fc_total, const int64_t** fc_off,
                               const int32_t** fc_lvl, const int32_t** fc_fronts, const int32_t** fc_big_lvl,
                               const int32_t** fc_big) {
  if (!s || !nlevels || !fc_total || !fc_off || !fc_lvl || !fc_fronts || !fc_big_lvl || !fc_big)
    return CHD_ERR_INVALID;
  *nlevels = (int64_t)s->fc_lvl.size() - 1;
  *fc_total = s->fc_total;
  *fc_off = s->fc_off.data();
  *fc_lvl = s->fc_lvl.data();
  *fc_fronts = s->fc_fronts.data();
  *fc_big_lvl = s->fc_big_lvl.data();
  *fc_big = s->fc_big.data();
  return CHD_OK;
}

chd_status chd_completion_flops(const chd_symbolic* s, double out[3]) {
  if (!s || !out) return CHD_ERR_INVALID;
  out[0] = s->fc_flops[0];
  out[1] = s->fc_flops[1];
  int levels = 0;
  for (size_t l = 0; l + 1 < s->fc_lvl.size(); ++l)
    levels += (s->fc_lvl[l + 1] > s->fc_lvl[l] || s->fc_big_lvl[l + 1] > s->fc_big_lvl[l]) ? 1 : 0;
  out[2] = (double)levels;
  return CHD_OK;
}

void chd_symbolic_free(chd_symbolic* s) {
  if (!s) return;
  if (s->dev_buf) cudaFree(s->dev_buf);
  delete s;
}

chd_status chd_factor_new(chd_symbolic* s, const double* x, void* stream, chd_factor** out) {
  if (!s || !x || !out) return CHD_ERR_INVALID;
  *out = nullptr;
  chd_factor* f = nullptr;
  chd_status rc = alloc_factor(s, static_cast<cudaStream_t>(stream), &f);
  if (rc != CHD_OK) return rc;
  rc = chd_refactor(f, x, stream);
  if (rc != CHD_OK) {
    chd_factor_free(f);
    return rc;
  }
  *out = f;
  return CHD_OK;
}

chd_status chd_refactor(chd_factor* f, const double* x, void* stream) {
  if (!f || !x) return CHD_ERR_INVALID;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_ws(f, 1);
  if (rc != CHD_OK) return rc;
  f->have_S = f->have_R = f->have_Q = false;
  rc = cuda_ok(cudaMemsetAsync(f->status, 0, 4 * 8, f->stream));
  if (rc != CHD_OK) return rc;
  GraphKey key;
  key.p[0] = x;
  return run_sequence(f, G_FACTOR, key, [&](cudaStream_t st) {
    chd_launch::factor(f->sym, st, &f->ex, x, f->Lc, f->Wc, f->Dd, f->ws, f->ldet, f->status);
  });
}

chd_status chd_logdet(chd_factor* f, double* out) {
  if (!f || !out) return CHD_ERR_INVALID;
  chd_launch::sum(f->stream, f->ldet, f->sym->nsn, f->scalar);
  chd_status rc = launch_status();
  if (rc != CHD_OK) return rc;
  rc = cuda_ok(cudaMemcpyAsync(out, f->scalar, 8, cudaMemcpyDeviceToHost, f->stream));
  if (rc != CHD_OK) return rc;
  return read_status(f);
}

chd_status chd_logdet_batch(chd_factor* f, double* out) {
  if (!f || !out) return CHD_ERR_INVALID;
  const int64_t count = (int64_t)f->sym->inst_n.size() - 1;
  double* dsum = nullptr;
  if (count == 1) {
    chd_launch::sum(f->stream, f->ldet, f->sym->nsn, f->scalar);
    dsum = f->scalar;
  } else {
    if (!f->inst_sum) {
      chd_status rc0 = cuda_ok(cudaMalloc(&f->inst_sum, (size_t)count * 8));
      if (rc0 != CHD_OK) return rc0;
    }
    chd_launch::segsum(f->stream, f->ldet, f->sym->dev.inst_sn, (int)count, f->inst_sum);
    dsum = f->inst_sum;
  }
  chd_status rc = launch_status();
  if (rc != CHD_OK) return rc;
  rc = cuda_ok(cudaMemcpyAsync(out, dsum, (size_t)count * 8, cudaMemcpyDeviceToHost, f->stream));
  if (rc != CHD_OK) return rc;
  return read_status(f);
}

chd_status chd_gradient(chd_factor* f, double* g, void* stream) {
  if (!f || !g) return CHD_ERR_INVALID;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_ws(f, 1);
  if (rc != CHD_OK) return rc;
  GraphKey key;
  key.p[0] = g;
  rc = run_sequence(f, G_GRADIENT, key, [&](cudaStream_t st) {
    chd_launch::gradient(f->sym, st, &f->ex, f->Wc, f->Sc, g, f->Vd, f->ws);
  });
  if (rc == CHD_OK) f->have_S = true;
  return rc;
}

chd_status chd_hessian(chd_factor* f, int m, const double* y, int64_t ldy, double* t, int64_t ldt,
                       void* stream) {
  if (!f || m < 0 || (m > 0 && (!y || !t))) return CHD_ERR_INVALID;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (ldy < nnz || ldt < nnz)) return CHD_ERR_INVALID;
  if (m == 0) return CHD_OK;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_projected_inverse(f);
  if (rc != CHD_OK) return rc;
  const int64_t chunk = rhs_chunk(f, m);
  rc = ensure_ws(f, chunk);
  if (rc != CHD_OK) return rc;
  for (int64_t i = 0; i < m; i += chunk) {
    const int mc = (int)std::min<int64_t>(chunk, m - i);
    GraphKey key;
    key.p[0] = y + i * ldy;
    key.p[1] = t + i * ldt;
    key.v[0] = mc;
    key.v[1] = ldy;
    key.v[2] = ldt;
    rc = run_sequence(f, G_HESSIAN, key, [&](cudaStream_t st) {
      chd_launch::hessian(f->sym, st, &f->ex, mc, f->Wc, f->Vd, y + i * ldy, ldy, t + i * ldt, ldt, f->ws);
    });
    if (rc != CHD_OK) return rc;
  }
  return CHD_OK;
}

// W = R(Y); with `prune`, per right-hand side only the fronts whose
// subtrees hold nonzeros of Y run (§5.5), the rest of W is zero
static chd_status hessian_factor(chd_factor* f, int m, const double* y, int64_t ldy, double* w, int64_t ldw,
                                 void* stream, bool prune) {
  if (!f || m < 0 || (m > 0 && (!y || !w))) return CHD_ERR_INVALID;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (ldy < nnz || ldw < nnz)) return CHD_ERR_INVALID;
  if (m == 0) return CHD_OK;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_projected_inverse(f);
  if (rc != CHD_OK) return rc;
  const int64_t chunk = rhs_chunk(f, m);
  rc = ensure_ws(f, chunk);
  if (rc == CHD_OK) rc = ensure_q(f);
  if (rc == CHD_OK && prune) rc = ensure_act(f, chunk);
  if (rc != CHD_OK) return rc;
  const int64_t nsn = f->sym->nsn;
  int32_t* cnt = prune ? static_cast<int32_t*>(f->act_buf) : nullptr;
  uint8_t* act = prune ? reinterpret_cast<uint8_t*>(cnt + nsn * f->act_rhs) : nullptr;
  for (int64_t i = 0; i < m; i += chunk) {
    const int mc = (int)std::min<int64_t>(chunk, m - i);
    GraphKey key;
    key.p[0] = y + i * ldy;
    key.p[1] = w + i * ldw;
    key.p[2] = act;
    key.v[0] = mc;
    key.v[1] = ldy;
    key.v[2] = ldw;
    double* wi = w + i * ldw;
    cudaError_t ce = cudaSuccess;
    rc = run_sequence(f, prune ? G_HFACTOR_SPARSE : G_HFACTOR, key, [&](cudaStream_t st) {
      if (prune) {
        ce = cudaMemset2DAsync(wi, (size_t)(mc > 1 ? ldw : nnz) * 8, 0, (size_t)nnz * 8, (size_t)mc, st);
        chd_launch::prune_mask(f->sym, st, mc, y + i * ldy, ldy, cnt, act);
      }
      chd_launch::hess_up_pass(f->sym, st, &f->ex, mc, f->Wc, f->Vd, y + i * ldy, ldy, wi, ldw, f->ws, act);
      chd_launch::rtrans(f->sym, st, &f->ex, mc, 0, f->Lc, f->Qd, wi, ldw, f->ws, act);
    });
    if (rc == CHD_OK && ce != cudaSuccess) rc = cuda_ok(ce);
    if (rc != CHD_OK) return rc;
  }
  return CHD_OK;
}

chd_status chd_hessian_factor(chd_factor* f, int m, const double* y, int64_t ldy, double* w, int64_t ldw,
                              void* stream) {
  return hessian_factor(f, m, y, ldy, w, ldw, stream, false);
}

chd_status chd_hessian_factor_sparse(chd_factor* f, int m, const double* y, int64_t ldy, double* w, int64_t ldw,
                                     void* stream) {
  return hessian_factor(f, m, y, ldy, w, ldw, stream, true);
}

chd_status chd_hessian_factor_adj(chd_factor* f, int m, const double* w, int64_t ldw, double* t, int64_t ldt,
                                  void* stream) {
  if (!f || m < 0 || (m > 0 && (!w || !t))) return CHD_ERR_INVALID;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (ldw < nnz || ldt < nnz)) return CHD_ERR_INVALID;
  if (m == 0) return CHD_OK;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_projected_inverse(f);
  if (rc != CHD_OK) return rc;
  const int64_t chunk = rhs_chunk(f, m);
  rc = ensure_ws(f, chunk);
  if (rc == CHD_OK) rc = ensure_q(f);
  if (rc != CHD_OK) return rc;
  for (int64_t i = 0; i < m; i += chunk) {
    const int mc = (int)std::min<int64_t>(chunk, m - i);
    GraphKey key;
    key.p[0] = w + i * ldw;
    key.p[1] = t + i * ldt;
    key.v[0] = mc;
    key.v[1] = ldw;
    key.v[2] = ldt;
    double* ti = t + i * ldt;
    const double* wi = w + i * ldw;
    cudaError_t ce = cudaSuccess;
    rc = run_sequence(f, G_HFACTOR_ADJ, key, [&](cudaStream_t st) {
      if (ti != wi)
        ce = cudaMemcpy2DAsync(ti, (size_t)(mc > 1 ? ldt : nnz) * 8, wi, (size_t)(mc > 1 ? ldw : nnz) * 8,
                               (size_t)nnz * 8, (size_t)mc, cudaMemcpyDeviceToDevice, st);
      chd_launch::rtrans(f->sym, st, &f->ex, mc, 1, f->Lc, f->Qd, ti, ldt, f->ws, nullptr);
      chd_launch::hess_down_pass(f->sym, st, &f->ex, mc, f->Wc, ti, ldt, f->ws);
    });
    if (rc == CHD_OK && ce != cudaSuccess) rc = cuda_ok(ce);
    if (rc != CHD_OK) return rc;
  }
  return CHD_OK;
}

chd_status chd_inv_hessian(chd_factor* f, int m, const double* t, int64_t ldt, double* y, int64_t ldy,
                           void* stream) {
  if (!f || m < 0 || (m > 0 && (!y || !t))) return CHD_ERR_INVALID;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (ldy < nnz || ldt < nnz)) return CHD_ERR_INVALID;
  if (m == 0) return CHD_OK;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_projected_inverse(f);
  if (rc != CHD_OK) return rc;
  const int64_t chunk = rhs_chunk(f, m);
  rc = ensure_ws(f, chunk);
  if (rc != CHD_OK) return rc;
  rc = ensure_inv_v(f);
  if (rc != CHD_OK) return rc;
  for (int64_t i = 0; i < m; i += chunk) {
    const int mc = (int)std::min<int64_t>(chunk, m - i);
    GraphKey key;
    key.p[0] = t + i * ldt;
    key.p[1] = y + i * ldy;
    key.v[0] = mc;
    key.v[1] = ldt;
    key.v[2] = ldy;
    rc = run_sequence(f, G_INV_HESSIAN, key, [&](cudaStream_t st) {
      chd_launch::inv_hessian(f->sym, st, &f->ex, mc, f->Wc, f->Dd, f->Rd, t + i * ldt, ldt, y + i * ldy, ldy,
                              f->ws);
    });
    if (rc != CHD_OK) return rc;
  }
  return CHD_OK;
}

chd_status chd_recomplete(chd_factor* f, const double* sv, void* stream, double* fstar) {
  if (!f || !sv) return CHD_ERR_INVALID;
  chd_symbolic* s = f->sym;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_ws(f, 1);
  if (rc == CHD_OK) rc = cuda_ok(cudaMemsetAsync(f->status, 0, 4 * 8, f->stream));
  if (rc == CHD_OK)
    rc = cuda_ok(cudaMemcpyAsync(f->Sc, sv, (size_t)s->colptr[s->n] * 8, cudaMemcpyDeviceToDevice, f->stream));
  // factored update matrices: scratch of the Householder reductions (the
  // largest level's), allocated once per factor object
  const bool factored = s->completion_mode == 1;
  if (rc == CHD_OK && factored && !f->fcs && s->fc_total > 0) {
    if (cudaMalloc(reinterpret_cast<void**>(&f->fcs), (size_t)s->fc_total * 8) != cudaSuccess) {
      cudaGetLastError();
      f->fcs = nullptr;
      rc = CHD_ERR_OOM;
    }
  }
  if (rc == CHD_OK) {
    GraphKey key;
    key.p[0] = sv;
    rc = run_sequence(f, G_COMPLETE, key, [&](cudaStream_t st) {
      chd_launch::complete(s, st, &f->ex, sv, f->Lc, f->Wc, f->Dd, f->Vd, f->Rd, factored ? f->Qd : nullptr, f->fcs,
                           f->ws, f->ldet, f->status);
    });
  }
  if (rc != CHD_OK) return rc;
  f->have_S = true;
  f->have_R = false;  // Rd holds chol(V_k) or nothing here; V_k^{-1} is formed on first use
  // the factored form leaves G_k = P R_k P = chol(P V_k P) in Qd: the Hessian
  // factor's upper factors of V_k
  f->have_Q = factored;
  if (fstar) {
    double ld = 0;
    rc = chd_logdet(f, &ld);
    if (rc == CHD_ERR_NOT_PD) rc = CHD_ERR_NOT_COMPLETABLE;
    if (rc != CHD_OK) return rc;
    *fstar = ld - (double)s->n;
  }
  return CHD_OK;
}

chd_status chd_complete(chd_symbolic* s, const double* sv, void* stream, chd_factor** xhat,
                        double* fstar) {
  if (!s || !sv || !xhat) return CHD_ERR_INVALID;
  *xhat = nullptr;
  chd_factor* f = nullptr;
  chd_status rc = alloc_factor(s, static_cast<cudaStream_t>(stream), &f);
  if (rc != CHD_OK) return rc;
  rc = chd_recomplete(f, sv, stream, fstar);
  if (rc != CHD_OK) {
    chd_factor_free(f);
    return rc;
  }
  *xhat = f;
  return CHD_OK;
}

chd_status chd_schur(chd_factor* f, int m, const double* a, int64_t lda, double* t, int64_t ldt, double* h,
                     void* stream) {
  if (!f || m < 1 || !a || !t || !h) return CHD_ERR_INVALID;
  const int64_t nnz = f->sym->colptr[f->sym->n];
  if (m > 1 && (lda < nnz || ldt < nnz)) return CHD_ERR_INVALID;
  if ((int64_t)m * m > (int64_t(1) << 24)) return CHD_ERR_INVALID;
  if ((std::max<int64_t>(nnz, f->sym->n) + 65535) / 65536 > 65535) return CHD_ERR_INVALID;
  chd_status rc = chd_hessian(f, m, a, lda, t, ldt, stream);
  if (rc != CHD_OK) return rc;
  // the partial sums live in the factor's workspace (free once the Hessian
  // products are queued before them on the same stream)
  rc = ensure_ws(f, std::max<int64_t>(1, (chd_launch::schur_scratch(f->sym, m) + f->sym->dev.f_total - 1) /
                                              std::max<int64_t>(1, f->sym->dev.f_total)));
  if (rc != CHD_OK) return rc;
  chd_launch::schur(f->sym, f->stream, m, a, lda, t, ldt, h, f->ws);
  return launch_status();
}

chd_status chd_product(chd_factor* f, double* x, void* stream) {
  if (!f || !x) return CHD_ERR_INVALID;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_status rc = ensure_ws(f, 1);
  if (rc != CHD_OK) return rc;
  GraphKey key;
  key.p[0] = x;
  return run_sequence(f, G_PRODUCT, key, [&](cudaStream_t st) {
    chd_launch::product(f->sym, st, &f->ex, f->Lc, x, f->ws);
  });
}

chd_status chd_factor_export(chd_factor* f, double* l, double* d, void* stream) {
  if (!f || !l) return CHD_ERR_INVALID;
  f->stream = static_cast<cudaStream_t>(stream);
  chd_launch::export_ldl(f->sym, f->stream, f->Lc, l, d);
  return launch_status();
}

chd_status chd_status_get(chd_factor* f) {
  if (!f) return CHD_ERR_INVALID;
  return read_status(f);
}

chd_status chd_error_detail(chd_factor* f, int64_t* supernode, int64_t* column) {
  if (!f) return CHD_ERR_INVALID;
  int64_t h[4] = {0, 0, 0, 0};
  chd_status rc = cuda_ok(cudaMemcpyAsync(h, f->status, sizeof(h), cudaMemcpyDeviceToHost, f->stream));
  if (rc == CHD_OK) rc = cuda_ok(cudaStreamSynchronize(f->stream));
  if (rc != CHD_OK) return rc;
  if (supernode) *supernode = h[0] ? h[1] : -1;
  if (column) *column = h[0] ? h[2] : -1;
  return static_cast<chd_status>(h[0]);
}

int64_t chd_kernel_launches(void) { return chd_launch::launches(); }
int64_t chd_split_k_launches(void) { return chd_launch::split_k_launches(); }
double chd_tc_flops(void) { return chd_launch::tc_flops(); }

chd_status chd_factor_set_workspace_limit(chd_factor* f, size_t bytes) {
  if (!f) return CHD_ERR_INVALID;
  f->ws_limit = bytes;
  return CHD_OK;
}

chd_status chd_factor_set_graphs(chd_factor* f, int on) {
  if (!f) return CHD_ERR_INVALID;
  if (!on) {
    if (f->gs) cudaStreamSynchronize(f->gs);
    for (auto& g : f->graphs) drop_graph(g);
  }
  f->graphs_on = on && f->gs && f->g_in && f->g_out;
  return CHD_OK;
}

chd_status chd_factor_set_graph_limit(chd_factor* f, int64_t max_launches) {
  if (!f || max_launches < 0) return CHD_ERR_INVALID;
  f->graph_limit = max_launches;
  return CHD_OK;
}

chd_status chd_factor_release_workspace(chd_factor* f) {
  if (!f) return CHD_ERR_INVALID;
  if (f->ws) {
    chd_status rc = cuda_ok(cudaFreeAsync(f->ws, f->stream));
    if (rc != CHD_OK) return rc;
    f->ws = nullptr;
    f->ws_rhs = 0;
  }
  if (f->act_buf) {
    chd_status rc = cuda_ok(cudaFreeAsync(f->act_buf, f->stream));
    if (rc != CHD_OK) return rc;
    f->act_buf = nullptr;
    f->act_rhs = 0;
  }
  return CHD_OK;
}

chd_status chd_factor_workspace_bytes(const chd_factor* f, size_t* bytes) {
  if (!f || !bytes) return CHD_ERR_INVALID;
  *bytes = (size_t)f->ws_rhs * (size_t)f->sym->dev.f_total * 8;
  return CHD_OK;
}

chd_status chd_probe_fp64_peak(void* stream, double* gflops) {
  if (!gflops) return CHD_ERR_INVALID;
  return cuda_ok(chd_launch::fp64_peak(static_cast<cudaStream_t>(stream), gflops));
}

void chd_factor_free(chd_factor* f) {
  if (!f) return;
  if (f->stream) cudaStreamSynchronize(f->stream);
  for (int j = 0; j < f->ex.nside; ++j) {
    cudaStreamSynchronize(f->ex.side[j]);
    cudaStreamDestroy(f->ex.side[j]);
    if (f->ex.join[j]) cudaEventDestroy(f->ex.join[j]);
  }
  if (f->ex.fork) cudaEventDestroy(f->ex.fork);
  for (auto& g : f->graphs) drop_graph(g);
  if (f->gs) {
    cudaStreamSynchronize(f->gs);
    cudaStreamDestroy(f->gs);
  }
  if (f->g_in) cudaEventDestroy(f->g_in);
  if (f->g_out) cudaEventDestroy(f->g_out);
  if (f->ws) cudaFree(f->ws);
  if (f->fcs) cudaFree(f->fcs);
  if (f->act_buf) cudaFree(f->act_buf);
  if (f->inst_sum) cudaFree(f->inst_sum);
  if (f->block) cudaFree(f->block);
  delete f;
}

}  // extern "C"

// Device upload of the symbolic arrays the kernels read (one allocation,
// one host-to-device copy).
chd_status chd_symbolic_upload(chd_symbolic* s) {
  struct Piece {
    const void* src;
    size_t bytes;
    size_t off;
  };
  std::vector<Piece> pcs;
  size_t off = 0;
  auto add = [&](const void* p, size_t bytes) {
    pcs.push_back({p, bytes, off});
    off = align_up(off + std::max<size_t>(bytes, 8));
    return pcs.size() - 1;
  };
  size_t iColptr = add(s->colptr.data(), s->colptr.size() * 8);
  size_t iRowind = add(s->rowind.data(), s->rowind.size() * 4);
  size_t iRows = add(s->rows.data(), s->rows.size() * 4);
  size_t iSn = add(s->sn_ptr.data(), s->sn_ptr.size() * 8);
  size_t iPar = add(s->sn_par.data(), s->sn_par.size() * 8);
  size_t iRp = add(s->rows_ptr.data(), s->rows_ptr.size() * 8);
  size_t iRel = add(s->rel.data(), s->rel.size() * 4);
  size_t iCp = add(s->ch_ptr.data(), s->ch_ptr.size() * 8);
  size_t iCh = add(s->ch.data(), s->ch.size() * 4);
  size_t iEp = add(s->ea_ptr.data(), s->ea_ptr.size() * 8);
  size_t iEa = add(s->ea.data(), s->ea.size() * 4);
  size_t iF = add(s->f_off.data(), s->f_off.size() * 8);
  size_t iD = add(s->d_off.data(), s->d_off.size() * 8);
  size_t iV = add(s->v_off.data(), s->v_off.size() * 8);
  size_t iTp = add(s->task_ptr.data(), s->task_ptr.size() * 4);
  size_t iTf = add(s->task_fronts.data(), s->task_fronts.size() * 4);
  size_t iTm = add(s->tmeta.data(), s->tmeta.size() * sizeof(WMeta));
  size_t iSf = add(s->small_fronts.data(), s->small_fronts.size() * 4);
  size_t iCf = add(s->cta_fronts.data(), s->cta_fronts.size() * 4);
  size_t iWf = add(s->warp_fronts.data(), s->warp_fronts.size() * 4);
  size_t iPf = add(s->plain_fronts.data(), s->plain_fronts.size() * 4);
  size_t iSl = add(s->sub_lo.data(), s->sub_lo.size() * 4);
  size_t iSh = add(s->sub_hi.data(), s->sub_hi.size() * 4);
  size_t iIs = add(s->inst_sn.data(), s->inst_sn.size() * 8);
  size_t iFo = add(s->fc_off.data(), s->fc_off.size() * 8);
  size_t iFf = add(s->fc_fronts.data(), s->fc_fronts.size() * 4);
  std::vector<char> host(off, 0);
  for (auto& p : pcs)
    if (p.bytes) std::memcpy(host.data() + p.off, p.src, p.bytes);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    // No usable device: the symbolic object stays host-only.  Numeric calls
    // then fail with CHD_ERR_CUDA.
    cudaGetLastError();
    s->dev_buf = nullptr;
    s->dev = SymDev{};
    s->dev.f_total = s->f_off[s->nsn];
    return CHD_OK;
  }
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return CHD_ERR_OOM;
    // no device present: host-only symbolic object
    s->dev_buf = nullptr;
    s->dev = SymDev{};
    s->dev.f_total = s->f_off[s->nsn];
    return CHD_OK;
  }
  if (cudaMemcpy(buf, host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(buf);
    return CHD_ERR_CUDA;
  }
  s->dev_buf = buf;
  s->dev_id = dev;
  char* b = static_cast<char*>(buf);
  SymDev& d = s->dev;
  d.n = s->n;
  d.nsn = s->nsn;
  d.colptr = reinterpret_cast<const int64_t*>(b + pcs[iColptr].off);
  d.rowind = reinterpret_cast<const int32_t*>(b + pcs[iRowind].off);
  d.rows = reinterpret_cast<const int32_t*>(b + pcs[iRows].off);
  d.sn_ptr = reinterpret_cast<const int64_t*>(b + pcs[iSn].off);
  d.sn_par = reinterpret_cast<const int64_t*>(b + pcs[iPar].off);
  d.rows_ptr = reinterpret_cast<const int64_t*>(b + pcs[iRp].off);
  d.rel = reinterpret_cast<const int32_t*>(b + pcs[iRel].off);
  d.ch_ptr = reinterpret_cast<const int64_t*>(b + pcs[iCp].off);
  d.ch = reinterpret_cast<const int32_t*>(b + pcs[iCh].off);
  d.ea_ptr = reinterpret_cast<const int64_t*>(b + pcs[iEp].off);
  d.ea = reinterpret_cast<const int32_t*>(b + pcs[iEa].off);
  d.f_off = reinterpret_cast<const int64_t*>(b + pcs[iF].off);
  d.d_off = reinterpret_cast<const int64_t*>(b + pcs[iD].off);
  d.v_off = reinterpret_cast<const int64_t*>(b + pcs[iV].off);
  d.task_ptr = reinterpret_cast<const int32_t*>(b + pcs[iTp].off);
  d.task_fronts = reinterpret_cast<const int32_t*>(b + pcs[iTf].off);
  d.tmeta = reinterpret_cast<const WMeta*>(b + pcs[iTm].off);
  d.small_fronts = reinterpret_cast<const int32_t*>(b + pcs[iSf].off);
  d.small_count = (int64_t)s->small_fronts.size();
  d.cta_fronts = reinterpret_cast<const int32_t*>(b + pcs[iCf].off);
  d.cta_count = (int64_t)s->cta_fronts.size();
  d.warp_fronts = reinterpret_cast<const int32_t*>(b + pcs[iWf].off);
  d.warp_count = (int64_t)s->warp_fronts.size();
  d.plain_fronts = reinterpret_cast<const int32_t*>(b + pcs[iPf].off);
  d.plain_count = (int64_t)s->plain_fronts.size();
  d.sub_lo = reinterpret_cast<const int32_t*>(b + pcs[iSl].off);
  d.sub_hi = reinterpret_cast<const int32_t*>(b + pcs[iSh].off);
  d.inst_sn = reinterpret_cast<const int64_t*>(b + pcs[iIs].off);
  d.fc_off = reinterpret_cast<const int64_t*>(b + pcs[iFo].off);
  d.fc_fronts = reinterpret_cast<const int32_t*>(b + pcs[iFf].off);
  d.ninst = (int64_t)s->inst_sn.size() - 1;
  d.f_total = s->f_off[s->nsn];
  d.d_total = s->d_off[s->nsn];
  d.v_total = s->v_off[s->nsn];
  return CHD_OK;
}
