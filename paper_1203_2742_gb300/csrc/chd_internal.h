// Internal declarations shared by the host symbolic phase, the C ABI and the
// CUDA kernels of the chordal log-det barrier library.
#pragma once

#include <cuda_runtime_api.h>

#include <cstdint>
#include <vector>

#include "chordal_barrier.h"

// One record per position of the task lists (aligned with task_fronts):
// what a warp needs to start a front with one load.  flags:
//   WM_PREV_CHILD      the previous front of the task is a child of this one
//   WM_NEXT_PARENT     the next front of the task is this one's parent
//   WM_ONLY_CHILD_PREV this front's only child is the previous front of the task
constexpr int32_t WM_PREV_CHILD = 1, WM_NEXT_PARENT = 2, WM_ONLY_CHILD_PREV = 4;
struct alignas(16) WMeta {
  int64_t col0;      // first column of N_k
  int64_t base;      // colptr[col0]: offset of the front's values
  int64_t f_off;     // workspace offset (one right-hand side)
  int64_t rows_off;  // rows_ptr[k]
  int64_t d_off;     // offset of the n x n block
  int64_t v_off;     // offset of the a x a block
  int32_t k, n, J, flags;
  int32_t ch_beg, ch_end;  // children of k in ch[ch_beg..ch_end)
  int32_t pad[2];
};

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
  const int64_t* ea_ptr = nullptr;   // nsn+1: children whose update blocks k adds (a leaf
  const int32_t* ea = nullptr;       //   group contributes through its first member only)
  const int64_t* f_off = nullptr;    // nsn+1: per-front workspace offsets (doubles)
  const int64_t* d_off = nullptr;    // nsn+1: per-front n_k*n_k block offsets
  const int64_t* v_off = nullptr;    // nsn+1: per-front a_k*a_k block offsets
  const int32_t* task_ptr = nullptr; // ntask+1
  const int32_t* task_fronts = nullptr;
  const WMeta* tmeta = nullptr;      // aligned with task_fronts
  const int32_t* small_fronts = nullptr;  // fronts not in the dense tier
  int64_t small_count = 0;
  const int32_t* cta_fronts = nullptr;    // fronts of the CTA and wide warp tiers (completion)
  int64_t cta_count = 0;
  const int32_t* warp_fronts = nullptr;   // fronts of the warp tier
  int64_t warp_count = 0;
  const int32_t* plain_fronts = nullptr;  // fronts of the warp, wide and CTA tiers (no dense, no group)
  int64_t plain_count = 0;
  // fronts whose update blocks reach front k's: [sub_lo[k], sub_hi[k]] (its
  // subtree, plus the other members when k heads a leaf group)
  const int32_t* sub_lo = nullptr;
  const int32_t* sub_hi = nullptr;
  // pruned Hessian factor (§5.5): per right-hand side y, act[y * nsn + k] != 0
  // iff Y has a nonzero in the columns of that range; null: every front active
  const uint8_t* act = nullptr;
  const int64_t* fc_off = nullptr;        // factored completion: scratch offsets (per front)
  const int32_t* fc_fronts = nullptr;     // factored completion: CTA-handled fronts by level
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
  std::vector<int64_t> ea_ptr;  // children for the extend-add (see SymDev)
  std::vector<int32_t> ea;
  // leaf groups: supernodes [grp_first[g], grp_first[g] + grp_count[g]) are
  // one-column leaves of one parent with the same A; grp_of[k] = g or -1
  std::vector<int64_t> grp_first, grp_count;
  std::vector<int32_t> grp_of;
  std::vector<int64_t> f_off, d_off, v_off;
  // schedule: tasks are front sequences processed by one CTA; launches
  // group tasks by level (bottom-up order); lvl_ptr indexes tasks.
  std::vector<int32_t> task_ptr, task_fronts, lvl_ptr;
  std::vector<WMeta> tmeta;  // aligned with task_fronts
  // per level: the last lvl_big[l] tasks of the level are single big fronts
  // run by the multi-CTA dense tier
  std::vector<int32_t> lvl_big;
  // per level: the first lvl_r32[l] + lvl_r64[l] tasks are chain-tier runs
  // (|J| <= 32, then |J| <= 64; all zero unless chain_runs)
  std::vector<int32_t> lvl_r32, lvl_r64;
  // per level l, five counts at 5*l: chain runs (|J| <= 32), chain runs
  // (|J| <= 64), warp, wide warp and dense-tier tasks (chd_symbolic_schedule)
  std::vector<int32_t> lvl_counts;
  // per level, after the runs: lvl_warp[l] warp-tier tasks (|J| <= 32),
  // the next lvl_w64[l] wide warp-tier tasks (|J| <= 64)
  std::vector<int32_t> lvl_warp, lvl_w64;
  std::vector<char> is_big;  // per supernode
  std::vector<int32_t> tier;  // per supernode: 0 warp, 3 wide warp, 1 CTA, 2 dense, 4 leaf group
  std::vector<int32_t> small_fronts;
  std::vector<int32_t> cta_fronts;
  std::vector<int32_t> warp_fronts;
  std::vector<int32_t> big_fronts;
  std::vector<int32_t> plain_fronts;
  std::vector<int32_t> sub_lo, sub_hi;
  double flops[5] = {0, 0, 0, 0, 0};
  // independent instances analysed together (chd_analyze_batch): instance i
  // owns columns [inst_n[i], inst_n[i+1]), values [inst_nnz[i], inst_nnz[i+1])
  // and supernodes [inst_sn[i], inst_sn[i+1]) of the analysed numbering
  std::vector<int64_t> inst_n, inst_nnz, inst_sn;
  int64_t max_front = 0;
  int tc_mode = 0;  // chd_opts.tc_products
  // completion with factored update matrices (chd_opts.completion = 1):
  // fronts with a_k > 0 by depth in the clique tree, parents first; the
  // per-front sequence runs one CTA per front (fc_fronts, level l at
  // [fc_lvl[l], fc_lvl[l+1])) or the dense tier (fc_big, fc_big_lvl);
  // fc_off: scratch offset (doubles) of the front's reduction within its
  // level; fc_total: largest level's scratch; fc_flops: Cholesky of every
  // V_k (independent form) and the factored form's arithmetic
  int completion_mode = 0;
  std::vector<int64_t> fc_off;
  std::vector<int32_t> fc_fronts, fc_lvl, fc_big, fc_big_lvl;
  int64_t fc_total = 0;
  double fc_flops[2] = {0, 0};
  // device mirror
  SymDev dev;
  void* dev_buf = nullptr;
  int dev_id = -1;
};

// Execution resources of the dense tier: side streams on which independent
// big fronts run concurrently (forked from and joined back to the caller's
// stream with events), and one scratch slice per stream (slice 0: the
// caller's stream) for split-K partial products, ending with the counter of
// the Cholesky panel kernel.  The first kWideSlices slices are large; the
// rest hold the counter and small partial products only.
constexpr int kSideStreams = 32;
constexpr int kWideSlices = 9;
struct Exec {
  int nside = 0;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {};
  double* slice[kSideStreams + 1] = {};
  int64_t slice_cap[kSideStreams + 1] = {};
  // scratch of the tensor-core products (digit planes), per stream slot
  void* tc[kSideStreams + 1] = {};
  size_t tc_cap[kSideStreams + 1] = {};
  int64_t* status = nullptr;  // the factor's status (tensor-core timeouts)
  int tc_mode = 0;
};

// What one dense-tier front sequence runs with: its stream, the split-K
// scratch slice (may be null), the tensor-core scratch (may be null), the
// factor's status and the tensor-core mode of the analysis.
// Fronts outside the dense tier whose ancestor set has at least this many
// rows get V_k^{-1} from the multi-CTA kernels (blocked Cholesky, blocked
// triangular inverse, tensor-core product) instead of one CTA: on one SM
// the a^3 FP64 operations of a large V_k take milliseconds.
constexpr int kInvVMulti = 96;

struct Slot {
  cudaStream_t st = nullptr;
  double* xs = nullptr;
  int64_t xcap = 0;
  void* tc = nullptr;
  size_t tc_cap = 0;
  int64_t* status = nullptr;
  int tc_mode = 0;
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
enum GraphKind {
  G_FACTOR = 0,
  G_GRADIENT,
  G_HESSIAN,
  G_INV_HESSIAN,
  G_INV_V,
  G_COMPLETE,
  G_PRODUCT,
  G_HFACTOR,
  G_HFACTOR_ADJ,
  G_HFACTOR_SPARSE,
  G_Q,
  G_KINDS
};

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
  double* Rd = nullptr;      // per front, once have_R: V_k^{-1} (lower), or chol(V_k) for dense-tier fronts
  double* Qd = nullptr;      // per front, once have_Q: Cholesky factor of P V_k P (P the order reversal),
                             // i.e. the upper factor Q of V_k = Q Q^T held reversed (Hessian factor, §5.4)
  double* ldet = nullptr;
  double* scalar = nullptr;  // [0] log det
  int64_t* status = nullptr; // [0] code, [1] supernode, [2] column
  double* ws = nullptr;      // per-right-hand-side front workspace
  double* fcs = nullptr;     // factored completion: scratch of the reductions (own allocation)
  Exec ex;                   // dense-tier streams and split-K scratch
  double* inst_sum = nullptr;  // per-instance log det sums (batched symbolic objects)
  int64_t ws_rhs = 0;        // capacity in right-hand sides
  void* act_buf = nullptr;   // pruned Hessian factor: int32 counts, then uint8 flags, per (RHS, front)
  int64_t act_rhs = 0;       // capacity of act_buf in right-hand sides
  size_t ws_limit = 0;       // caller's cap on the workspace (0: library default)
  bool have_S = false;
  bool have_R = false;
  bool have_Q = false;
  // CUDA graphs of the launch sequences, replayed on the private stream gs
  bool graphs_on = true;
  int64_t graph_limit = 8192;  // longest launch sequence that is captured
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
