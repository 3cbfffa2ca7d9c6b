// Internal declarations shared by the host symbolic phase, the C ABI and the
// CUDA kernels of the chordal log-det barrier library.
#pragma once

#include <cuda_runtime_api.h>

#include <cstdint>
#include <vector>

#include "../../include/chordal_barrier.h"

// Device copy of the symbolic data, passed by value to every kernel.
struct SymDev {
  int64_t n = 0;
  int64_t nsn = 0;             // number of supernodes (fronts)
  const int64_t* colptr = nullptr;   // n+1: CSC of V (analysed order)
  const int32_t* rowind = nullptr;   // nnz: row indices of the CSC (sorted per column)
  const int64_t* sn_ptr = nullptr;   // nsn+1: N_k = [sn_ptr[k], sn_ptr[k+1])
  const int64_t* sn_par = nullptr;   // nsn: clique-tree parent or -1
  const int64_t* rows_ptr = nullptr; // nsn+1: offsets of J_k in `rows`/`rel`
  const int32_t* rel = nullptr;      // position of A_k[r] inside J_par(k) (A part only)
  const int32_t* rows = nullptr;     // J_k (N_k then A_k, increasing), at rows_ptr[k]
  const int64_t* ch_ptr = nullptr;   // nsn+1: children of k in ch[ch_ptr[k]..)
  const int32_t* ch = nullptr;
  const int64_t* f_off = nullptr;    // nsn+1: per-front workspace offsets (doubles)
  const int64_t* d_off = nullptr;    // nsn+1: per-front n_k*n_k block offsets
  const int64_t* v_off = nullptr;    // nsn+1: per-front a_k*a_k block offsets
  const int32_t* task_ptr = nullptr; // ntask+1
  const int32_t* task_fronts = nullptr;
  const int32_t* small_fronts = nullptr;  // fronts not in the dense tier
  int64_t small_count = 0;
  const int32_t* cta_fronts = nullptr;    // fronts of the CTA tier
  int64_t cta_count = 0;
  const int32_t* warp_fronts = nullptr;   // fronts of the warp tier
  int64_t warp_count = 0;
  const int64_t* inst_sn = nullptr;       // instances x supernode ranges
  int64_t ninst = 1;
  int64_t f_total = 0;               // workspace doubles per right-hand side
  int64_t d_total = 0;
  int64_t v_total = 0;
};

struct chd_symbolic {
  int64_t n = 0;
  std::vector<int64_t> perm;       // perm[new] = old
  std::vector<int64_t> colptr;     // n+1
  std::vector<int32_t> rowind;     // nnz(V)
  int64_t nsn = 0;
  std::vector<int64_t> sn_ptr;     // nsn+1
  std::vector<int64_t> sn_par;     // nsn
  std::vector<int64_t> rows_ptr;   // nsn+1
  std::vector<int32_t> rows;       // J_k, N_k first then A_k
  std::vector<int32_t> rel;        // aligned with rows; -1 on the N part
  std::vector<int64_t> ch_ptr;
  std::vector<int32_t> ch;
  std::vector<int64_t> f_off, d_off, v_off;
  // schedule: tasks are front sequences processed by one CTA; launches
  // group tasks by level (bottom-up order); lvl_ptr indexes tasks.
  std::vector<int32_t> task_ptr, task_fronts, lvl_ptr;
  // per level: the last lvl_big[l] tasks of the level are single big fronts
  // run by the multi-CTA dense tier
  std::vector<int32_t> lvl_big;
  // per level: the first lvl_warp[l] tasks are warp-tier tasks
  std::vector<int32_t> lvl_warp;
  std::vector<char> is_big;  // per supernode
  std::vector<int32_t> tier;  // per supernode: 0 warp, 1 CTA, 2 dense
  std::vector<int32_t> small_fronts;
  std::vector<int32_t> cta_fronts;
  std::vector<int32_t> warp_fronts;
  std::vector<int32_t> big_fronts;
  double flops[5] = {0, 0, 0, 0, 0};
  // independent instances analysed together (chd_analyze_batch): instance i
  // owns columns [inst_n[i], inst_n[i+1]), values [inst_nnz[i], inst_nnz[i+1])
  // and supernodes [inst_sn[i], inst_sn[i+1]) of the analysed numbering
  std::vector<int64_t> inst_n, inst_nnz, inst_sn;
  int64_t max_front = 0;
  // device mirror
  SymDev dev;
  void* dev_buf = nullptr;
  int dev_id = -1;
};

// Execution resources of the dense tier: side streams on which the big
// fronts of one level run concurrently (forked from and joined back to the
// caller's stream with events), and split-K scratch, one slice of xs_cap
// doubles per stream (slice 0: the caller's stream).
constexpr int kSideStreams = 8;
struct Exec {
  int nside = 0;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {};
  double* xs = nullptr;
  int64_t xs_cap = 0;
};

// A captured launch sequence of one kind of call (see capi.cpp): the
// arguments it was captured with, and the launch count of one replay.
struct GraphKey {
  const void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t v[4] = {0, 0, 0, 0};
  bool operator==(const GraphKey& o) const {
    for (int i = 0; i < 4; ++i)
      if (p[i] != o.p[i] || v[i] != o.v[i]) return false;
    return true;
  }
};
struct GraphSlot {
  GraphKey key;
  bool seen = false;
  bool capture_failed = false;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
};
enum GraphKind { G_FACTOR = 0, G_GRADIENT, G_HESSIAN, G_INV_HESSIAN, G_INV_V, G_COMPLETE, G_KINDS };

// A factor object: device-resident factor blocks, cached projected inverse
// and the per-right-hand-side front workspace (all owned by the object).
struct chd_factor {
  chd_symbolic* sym = nullptr;
  cudaStream_t stream = nullptr;
  void* block = nullptr;  // one allocation holding everything below but ws
  double* Lc = nullptr;
  double* Wc = nullptr;
  double* Sc = nullptr;
  double* Dd = nullptr;
  double* Vd = nullptr;
  double* Rd = nullptr;      // V_k^{-1} per front (lower), once have_R
  double* ldet = nullptr;
  double* scalar = nullptr;  // [0] log det
  int64_t* status = nullptr; // [0] code, [1] supernode, [2] column
  double* ws = nullptr;      // per-right-hand-side front workspace
  Exec ex;                   // dense-tier streams and split-K scratch
  double* inst_sum = nullptr;  // per-instance log det sums (batched symbolic objects)
  int64_t ws_rhs = 0;        // capacity in right-hand sides
  size_t ws_limit = 0;       // caller's cap on the workspace (0: library default)
  bool have_S = false;
  bool have_R = false;
  // CUDA graphs of the launch sequences, replayed on the private stream gs
  bool graphs_on = true;
  cudaStream_t gs = nullptr;
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  GraphSlot graphs[G_KINDS];
};

// Host helpers implemented in symbolic.cpp
chd_status chd_symbolic_build(int64_t n, const int64_t* colptr, const int32_t* rowind,
                              const chd_opts& opts, chd_symbolic* s);
chd_status chd_symbolic_upload(chd_symbolic* s);
chd_status chd_order_pattern(int64_t n, const int64_t* colptr, const int32_t* rowind, const chd_opts& opts,
                             std::vector<int64_t>& perm);

inline int64_t front_n(const chd_symbolic* s, int64_t k) { return s->sn_ptr[k + 1] - s->sn_ptr[k]; }
inline int64_t front_J(const chd_symbolic* s, int64_t k) { return s->rows_ptr[k + 1] - s->rows_ptr[k]; }
