/*
 * chordal_barrier.h -- C ABI of the GB300 library for the log-det barrier on
 * chordal (filled) sparsity patterns.
 *
 * Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
 * cones".  The library evaluates, for X in S^n_V (symmetric, sparsity
 * pattern V, positive definite) and S in S^n_V with a positive definite
 * completion:
 *   f(X)        = -log det X                         (§1.1)
 *   grad f(X)   = -P(X^{-1})                         (Eq. (e-grad-def))
 *   H(Y)        = P(X^{-1} Y X^{-1})                 (§1.1, §5)
 *   H^{-1}(T)                                        (§5.3)
 *   X-hat with P(X-hat^{-1}) = S, f_*(S) = log det X-hat - n
 *                                                    (§1.2, Eq. (e-Xhat-eq))
 * with supernodal multifrontal recursions over a clique tree (§6, §7).
 *
 * Conventions shared by every call
 * --------------------------------
 * Value arrays.  A matrix in S^n_V is a double array of nnz_filled entries:
 *   the lower triangle of the FILLED pattern V (returned by chd_symbolic_info)
 *   in compressed-column order, in the ANALYSED (permuted) numbering, rows
 *   ascending within a column, the diagonal first.  Batches of m matrices
 *   are stored one after another with a stride (ld) >= nnz_filled.
 * Pointers.  Every double* value argument below is a DEVICE pointer owned
 *   by the caller, except where the comment says "host".  Symbolic and
 *   factor objects are owned by the library and freed with the *_free calls.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *   default stream).  Numeric calls enqueue their kernels on it and return
 *   without synchronising; chd_analyze, chd_logdet, chd_status and
 *   chd_error_detail synchronise.
 * Errors.  Every call returns a chd_status; none traps or aborts.  Numeric
 *   failures found on the device (a non-positive pivot, an S with no
 *   positive definite completion, a bounded wait that ran out) are recorded
 *   in the factor object and reported by chd_status / chd_logdet /
 *   chd_error_detail, which synchronise.
 * Inner product.  A.B = tr(AB) (§1.1): off-diagonal entries count twice.
 */
#ifndef CHORDAL_BARRIER_H
#define CHORDAL_BARRIER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chd_symbolic chd_symbolic;
typedef struct chd_factor chd_factor;

typedef enum {
  CHD_OK = 0,
  CHD_ERR_INVALID = 1,          /* bad argument or malformed pattern */
  CHD_ERR_NOT_PD = 2,           /* X not positive definite (non-positive pivot) */
  CHD_ERR_NOT_COMPLETABLE = 3,  /* S has no positive definite completion */
  CHD_ERR_OOM = 4,              /* device or host allocation failed */
  CHD_ERR_CUDA = 5,             /* a CUDA runtime call failed */
  CHD_ERR_TIMEOUT = 6           /* a bounded device-side wait ran out */
} chd_status;

typedef enum {
  CHD_ORDER_NATURAL = 0,  /* keep the given numbering (it must be a perfect
                             elimination order if no fill is wanted) */
  CHD_ORDER_USER = 1,     /* use opts.user_perm */
  CHD_ORDER_MINDEG = 2,   /* minimum degree (exact degrees, smallest index on ties) */
  CHD_ORDER_ND_GEOMETRIC = 3 /* geometric nested dissection of a grid of opts.nd_dims
                             (vertex x + d0 (y + d1 z), d0 * d1 * d2 = n): the box is cut
                             through the middle of its longest side (first such axis) by a
                             one-vertex-thick plane; the lower half, the upper half and then
                             the plane are ordered, recursively; boxes of at most nd_leaf
                             vertices (or with all sides < 3) lexicographically, x fastest */
} chd_ordering;

/* log2 buckets of the tier table of chd_opts (front sizes up to 4095) */
#define CHD_TIER_BUCKETS 13

typedef struct {
  int32_t ordering;        /* chd_ordering */
  const int64_t* user_perm;/* host, n entries, perm[new] = old; used when ordering == CHD_ORDER_USER */
  int32_t relax;           /* relaxed supernodes: a merge of a child supernode into its
                              parent is accepted if it adds at most `relax` explicit zeros
                              to V; 0 = fundamental partition of Algorithm 6.1 */
  int32_t tie_last;        /* Algorithm 6.1 step 1 tie-break: 1 = child with the largest
                              index, 0 = smallest */
  int32_t big_rows;        /* a front with |J_k| >= big_rows (or |N_k| >= big_cols) is
                              processed by the multi-CTA dense tier; 0 = default 320 */
  int32_t big_cols;        /* 0 = default 160 */
  int32_t split_cols;      /* supernodes wider than 1.5 x split_cols columns are split into a
                              chain of supernodes of split_cols columns (V unchanged);
                              0 = default 256, negative = never split */
  int32_t chain_runs;      /* nonzero (chd_opts_default): runs of at least 8 one-column fronts
                              with contiguous rows and the same |A_k| <= 64 (band chains) get
                              their own chain-tier kernels for the factor, the gradient and
                              the passes of the Hessian, the Hessian factor and the inverse
                              Hessian (the Cholesky product runs them in the warp tier);
                              0: off */
  int32_t tc_products;     /* dense-tier products on the tensor cores (FP64-accurate digit
                              products, see chd_dgemm_tc): 0 (default) = a product runs there
                              when a cost model of both paths (launches, digit products,
                              output assembly, digit bytes against the FP64 units) predicts a
                              gain for the product alone; 1 = every product of at least
                              64 x 16 outputs; -1 = never (FP64 units only) */
  int32_t nd_dims[3];      /* grid dimensions for CHD_ORDER_ND_GEOMETRIC (use 1 for a 2D grid) */
  int32_t nd_leaf;         /* CHD_ORDER_ND_GEOMETRIC: largest box ordered without a cut; 0 = 8 */
  const int32_t* tier_table;  /* host, CHD_TIER_BUCKETS^2 entries, or NULL: per front shape, the
                              tier of a front with n_k columns and a_k ancestor rows is
                              tier_table[b(n_k) * CHD_TIER_BUCKETS + b(a_k)] with
                              b(v) = min(CHD_TIER_BUCKETS - 1, bit length of v) (b(0) = 0,
                              b(1) = 1, b(2..3) = 2, ...): -1 = by big_rows / big_cols, 0 = a
                              per-front tier (warp, wide warp or CTA by size), 1 = the dense
                              tier.  Leaf groups and chain runs are not affected.  Only the
                              distribution of the work changes, not the results beyond
                              rounding. */
  int32_t completion;      /* chd_complete / chd_recomplete: 0 (default) = every front
                              factors its V_k = S_{A_k A_k} itself (the fronts are
                              independent); 1 = factored update matrices (Algorithm 4.3, and
                              its supernodal form at the end of §7.2): the factor V_k = R_k R_k^T
                              is propagated from the parent, parents first, by deleting rows of
                              R_parent and re-triangularising them with Householder
                              reflections; the rows of A_k inside N_parent are added by a
                              triangular solve and a Cholesky factorisation.  Same result up to
                              rounding; the factors R_k are kept (the Hessian factor of the
                              completion reuses them). */
} chd_opts;

/* Fill `opts` with the defaults: natural order, relax 0, tie_last 1, default
   dense-tier thresholds, chain runs on, tensor-core products by cost,
   independent completion fronts. */
void chd_opts_default(chd_opts* opts);

/*
 * Symbolic analysis (§2, §6; Algorithm 6.1).  Host only, no device compute
 * apart from one upload of the index maps.
 *   n       order of the matrix (n >= 1)
 *   colptr  host, n+1 entries: lower-CSC column pointers of the user's pattern
 *   rowind  host, colptr[n] entries: row indices (row >= column); the
 *           diagonal may be omitted (it is always part of V)
 *   opts    NULL for defaults
 *   out     receives a new symbolic object
 * The pattern is ordered, filled to a chordal pattern (elimination fill),
 * postordered so that every supernode is a contiguous column range, and
 * partitioned into supernodes N_k with ancestor sets A_k and clique-tree
 * parents par(k) (§6.2-§6.4); optional relaxed amalgamation enlarges V.
 * Errors: CHD_ERR_INVALID for n < 1, an index out of range, an entry above
 * the diagonal or a user permutation that is not one; CHD_ERR_OOM.
 */
chd_status chd_analyze(int64_t n, const int64_t* colptr, const int32_t* rowind,
                       const chd_opts* opts, chd_symbolic** out);

/*
 * Batched analysis of `count` independent patterns, to be processed together
 * (tree parallelism across problems, §8): the symbolic object describes the
 * block-diagonal union of the patterns.  Each instance is ordered by its own
 * options (opts[i]; NULL for defaults) and keeps a contiguous block of the
 * analysed numbering; relax / tie_last / big_rows / big_cols / split_cols
 * are taken from opts[0].  Every call on the object (factor, gradient,
 * Hessian, completion, ...) then runs all instances level by level in the
 * same launches, and value arrays are the concatenation of the instances'
 * arrays (see chd_symbolic_batch_info).
 *   count            number of instances (>= 1)
 *   n[i]             order of instance i
 *   colptr[i], rowind[i]   host, lower CSC of instance i (as in chd_analyze)
 * Errors: as chd_analyze, for any instance.
 */
chd_status chd_analyze_batch(int64_t count, const int64_t* n, const int64_t* const* colptr,
                             const int32_t* const* rowind, const chd_opts* opts, chd_symbolic** out);

/*
 * Instance ranges of a (batched) symbolic object, host pointers owned by it:
 * instance i owns columns [n_off[i], n_off[i+1]) of the analysed numbering and
 * values [nnz_off[i], nnz_off[i+1]) of every value array.  A symbolic object
 * from chd_analyze has one instance.
 */
chd_status chd_symbolic_batch_info(const chd_symbolic* sym, int64_t* count, const int64_t** n_off,
                                   const int64_t** nnz_off);

/*
 * Pointers into the symbolic object (host memory, owned by it, valid until
 * chd_symbolic_free).  Any output pointer may be NULL.
 *   nnz_filled   entries of the lower triangle of the filled pattern V
 *   colptr       n+1 entries, rowind nnz_filled entries: V in CSC (analysed order)
 *   perm         n entries: perm[new] = old (user numbering)
 *   nsuper       number of supernodes
 */
chd_status chd_symbolic_info(const chd_symbolic* sym, int64_t* n, int64_t* nnz_filled,
                             const int64_t** colptr, const int32_t** rowind,
                             const int64_t** perm, int64_t* nsuper);

/*
 * Supernode partition and clique tree (host pointers into the object).
 *   snode_ptr  nsuper+1 entries: supernode k owns columns [snode_ptr[k], snode_ptr[k+1]) (N_k)
 *   snode_par  nsuper entries: clique-tree parent supernode, -1 at a root
 *   rows_ptr   nsuper+1 entries, rows: J_k = N_k followed by A_k, sorted
 */
chd_status chd_symbolic_supernodes(const chd_symbolic* sym, const int64_t** snode_ptr,
                                   const int64_t** snode_par, const int64_t** rows_ptr,
                                   const int32_t** rows);

/*
 * Algorithmic flop counts (multiply-add = 2) of one call of each operation
 * on this pattern, summed over the fronts from (n_k, a_k): out[0] factor,
 * out[1] gradient, out[2] Hessian per right-hand side, out[3] inverse Hessian
 * per right-hand side, out[4] completion.
 */
chd_status chd_symbolic_flops(const chd_symbolic* sym, double out[5]);

/*
 * The part of the completion that the two forms of chd_opts.completion do
 * differently, in flops summed over the fronts: out[0] = the Cholesky
 * factorisations of every V_k = S_{A_k A_k} (a_k^3 / 3, independent form);
 * out[1] = the factored form's propagation: the Householder reduction of the
 * rows of R_parent kept for A_k (4 x length x rows per reflection), the
 * triangular solve, update and Cholesky factorisation of the rows of A_k in
 * N_parent.  out[2] = the number of depth levels (of the clique tree) with
 * fronts to propagate, which run one after another.  Host only.
 */
chd_status chd_completion_flops(const chd_symbolic* sym, double out[3]);

/*
 * Per-front offsets of the analysis (host arrays of nsn + 1 entries owned
 * by `sym`, valid until chd_symbolic_free): f_off into the per-right-hand-
 * side workspace (front k owns [f_off[k], f_off[k+1]) doubles: its J x J
 * front and two J x n temporaries), d_off into the D_NN blocks (n x n) and
 * v_off into the V_k blocks (a x a; a leaf group's members share their
 * first member's).  Host only; for tests and tools.  Errors:
 * CHD_ERR_INVALID for NULL arguments.
 *
 * The plan of the completion with factored update matrices (host arrays
 * owned by `sym`, valid until chd_symbolic_free; built by every analysis,
 * used when chd_opts.completion = 1).  Depth levels of the clique tree,
 * roots first: level l propagates the fronts fc_fronts[fc_lvl[l] ..
 * fc_lvl[l+1]) one CTA each and fc_big[fc_big_lvl[l] .. fc_big_lvl[l+1]) on
 * the dense tier.  fc_off[k] (nsn entries) is front k's scratch offset in
 * doubles within its level's scratch of at most fc_total doubles: q_k w_k
 * for the rows of the parent's factor it reduces, plus
 * 32 (2 w_k + q_k + 32) for a dense-tier front with q_k > 0 (its panels'
 * reflectors, T, V T and the trailing product).  Host only; for tests and
 * tools.  Errors: CHD_ERR_INVALID for NULL arguments.
 */
chd_status chd_symbolic_offsets(const chd_symbolic* sym, const int64_t** f_off, const int64_t** d_off,
                                const int64_t** v_off);
chd_status chd_completion_plan(const chd_symbolic* sym, int64_t* nlevels, int64_t* fc_total, const int64_t** fc_off,
                               const int32_t** fc_lvl, const int32_t** fc_fronts, const int32_t** fc_big_lvl,
                               const int32_t** fc_big);

/*
 * The launch schedule built by the analysis (host arrays owned by `sym`,
 * valid until chd_symbolic_free).  A task is a list of fronts one worker
 * processes in order, children before parents; the tasks of a level depend
 * only on tasks of lower levels.  Level l holds tasks lvl_ptr[l] ..
 * lvl_ptr[l+1]-1 of task_ptr (nlevels+1 entries), in this order: chain runs
 * with |J| <= 32, chain runs with |J| <= 64, warp-tier, wide warp-tier,
 * CTA-tier tasks and dense-tier fronts; lvl_counts[5*l .. 5*l+4] are the
 * counts of those kinds except the CTA tier.  Task q holds the fronts
 * task_fronts[task_ptr[q] .. task_ptr[q+1]-1].  For tests and tools.
 * Errors: CHD_ERR_INVALID for NULL arguments.
 */
chd_status chd_symbolic_schedule(const chd_symbolic* sym, int64_t* nlevels, int64_t* ntasks,
                                 const int32_t** lvl_ptr, const int32_t** lvl_counts,
                                 const int32_t** task_ptr, const int32_t** task_fronts);

void chd_symbolic_free(chd_symbolic* sym);

/*
 * Cholesky factorisation X = L D L^T (supernodal Algorithm 7.1, §7.1).
 *   x_dev   device, nnz_filled values of X on V
 *   stream  cudaStream_t as void*
 *   out     receives a new factor object (device memory owned by it)
 * The factor keeps the supernodal Cholesky factor, D_NN^{-1}, the unit
 * lower blocks L_{A_k N_k} and D_NN for later calls.  A non-positive pivot
 * is recorded on the device and reported as CHD_ERR_NOT_PD by chd_status.
 * Errors returned directly: CHD_ERR_INVALID (NULL arguments), CHD_ERR_OOM,
 * CHD_ERR_CUDA.
 */
chd_status chd_factor_new(chd_symbolic* sym, const double* x_dev, void* stream,
                          chd_factor** out);

/* Refactor an existing factor object in place with new values of X (same pattern). */
chd_status chd_refactor(chd_factor* fac, const double* x_dev, void* stream);

/* log det X = sum of log D_ii (§1.1).  Synchronises; host output. */
chd_status chd_logdet(chd_factor* fac, double* out);

/* log det of every instance of a batched factor: out (host) has one entry
   per instance.  Synchronises. */
chd_status chd_logdet_batch(chd_factor* fac, double* out);

/*
 * Gradient g = -P(X^{-1}) (Eq. (e-grad-def)) by the supernodal projected
 * inverse, Algorithm 7.2 (§7.2).  g_dev: device, nnz_filled values.  The
 * projected inverse S = P(X^{-1}) and the dense blocks V_k = S_{A_k A_k}
 * are cached in the factor for chd_hessian / chd_inv_hessian.
 */
chd_status chd_gradient(chd_factor* fac, double* g_dev, void* stream);

/*
 * Hessian products T_i = P(X^{-1} Y_i X^{-1}), i < m (§5.2, Algorithm 5.1 in
 * supernodal block form).  y_dev: m matrices at stride ldy; t_dev: m
 * outputs at stride ldt (device).  Runs chd_gradient's projected inverse
 * first if it is not cached.  y_dev and t_dev must not overlap.
 */
chd_status chd_hessian(chd_factor* fac, int m, const double* y_dev, int64_t ldy,
                       double* t_dev, int64_t ldt, void* stream);

/*
 * Hessian factor (§5.4, Algorithms 5.3 and 5.4 in supernodal block form):
 * H = R^adj o R with W = R(Y) given per column j by W_jj = K_jj / D_jj and
 * W_{I_j j} = R_j^T K_{I_j j} / sqrt(D_jj), K the linearized factors of Y
 * (Eq. (e-mf-hess-vars)) and R_j the UPPER triangular factor of
 * S_{I_j I_j} = R_j R_j^T.  R^adj is its adjoint in the trace inner
 * product, so H_ij = A_i . H(A_j) = R(A_i) . R(A_j).
 *   chd_hessian_factor:      w_i = R(y_i), i < m
 *   chd_hessian_factor_adj:  t_i = R^adj(w_i), i < m; t_dev may equal w_dev
 *                            (in place), other overlaps are not allowed
 * Device arrays of m matrices at strides ldy/ldw/ldt (>= nnz_filled when
 * m > 1), values on V in the library's CSC layout.  The first call on a
 * factor computes the projected inverse (as chd_gradient) and the upper
 * factors of every V_k = S_{A_k A_k}; a pivot <= 0 there is recorded and
 * reported as CHD_ERR_NOT_PD by chd_status.  Errors returned directly:
 * CHD_ERR_INVALID (NULL arguments, m < 0, short strides), CHD_ERR_OOM,
 * CHD_ERR_CUDA.
 */
chd_status chd_hessian_factor(chd_factor* fac, int m, const double* y_dev, int64_t ldy,
                              double* w_dev, int64_t ldw, void* stream);
chd_status chd_hessian_factor_adj(chd_factor* fac, int m, const double* w_dev, int64_t ldw,
                                  double* t_dev, int64_t ldt, void* stream);

/*
 * R(Y) for sparse arguments (§5.5): the same result as chd_hessian_factor,
 * computed per right-hand side only on the fronts whose subtrees of the
 * clique tree hold a nonzero of Y (a front whose descendants' columns of Y
 * are all zero has K = 0, U' = 0 and W = 0 there).  Meant for Y with few
 * nonzeros relative to V, such as the constraint matrices A_i of a cone
 * program.  Holds nsn * 5 bytes per right-hand side of extra device
 * scratch.  Arguments, errors and overlap rules as chd_hessian_factor.
 */
chd_status chd_hessian_factor_sparse(chd_factor* fac, int m, const double* y_dev, int64_t ldy,
                                     double* w_dev, int64_t ldw, void* stream);

/*
 * Inverse-Hessian products Y_i = H^{-1}(T_i) (§5.3, Algorithm 5.2 in
 * supernodal block form): the solution in S^n_V of P(X^{-1} Y X^{-1}) = T.
 * Uses cached Cholesky factors of V_k = S_{A_k A_k}.
 */
chd_status chd_inv_hessian(chd_factor* fac, int m, const double* t_dev, int64_t ldt,
                           double* y_dev, int64_t ldy, void* stream);

/*
 * Maximum-determinant completion (§4.2; supernodal Algorithm 7.3, §7.2):
 * the factor of X-hat in S^n_V with P(X-hat^{-1}) = S, returned as a new
 * factor object (its projected inverse is S itself, so chd_hessian and
 * chd_inv_hessian on it give the dual barrier's derivatives through
 * Eq. (e-legendre-rels)).  s_dev: device, nnz_filled values of S.
 * fstar: host, receives f_*(S) = log det X-hat - n (§1.2); this call
 * synchronises when fstar is not NULL.  A pivot <= 0 in the Cholesky factor
 * of S_{A_k A_k} or of D_NN^{-1} is reported as CHD_ERR_NOT_COMPLETABLE.
 */
chd_status chd_complete(chd_symbolic* sym, const double* s_dev, void* stream,
                        chd_factor** xhat, double* fstar);

/*
 * Completion into an existing factor object (same pattern), reusing its
 * device memory: the object is overwritten with the factor of X-hat for
 * the new S.  Same contract as chd_complete otherwise.
 */
chd_status chd_recomplete(chd_factor* xhat, const double* s_dev, void* stream, double* fstar);

/*
 * Schur complement of the barrier Hessian for m matrices A_1..A_m in S^n_V
 * (the coefficients an interior-point method needs, §5.5):
 *   H_ij = A_i . grad^2 f(X)[A_j] = A_i . P(X^{-1} A_j X^{-1}),
 * the inner product counting off-diagonal entries twice.
 *   a_dev   m value arrays at stride lda (device, caller-owned)
 *   t_dev   caller-owned device workspace of m value arrays at stride ldt;
 *           receives T_j = P(X^{-1} A_j X^{-1})
 *   h_dev   device, m x m column-major (ld m), receives H (symmetric)
 * Same preconditions and error behaviour as chd_hessian; m*m <= 2^24.
 */
chd_status chd_schur(chd_factor* fac, int m, const double* a_dev, int64_t lda, double* t_dev, int64_t ldt,
                     double* h_dev, void* stream);

/*
 * Cholesky product (Algorithm 3.2, in the supernodal form of §7): x_dev
 * (device, nnz_filled values, caller-owned) receives the values on V of the
 * matrix L D L^T the factor object holds -- X itself for an object made by
 * chd_factor_new / chd_refactor, the maximum-determinant completion X-hat
 * for one made by chd_complete, so that the dual gradient is
 * grad f_*(S) = -X-hat (§1.2).  Uses the factor's workspace of one
 * right-hand side; asynchronous on `stream`.  Returns CHD_ERR_INVALID for a
 * NULL argument.
 */
chd_status chd_product(chd_factor* fac, double* x_dev, void* stream);

/*
 * Export the unique scalar factorisation X = L D L^T (§2, §3.1): l_dev gets
 * the nnz_filled entries of L on V (unit diagonal), d_dev the n pivots D_ii.
 */
chd_status chd_factor_export(chd_factor* fac, double* l_dev, double* d_dev, void* stream);

/*
 * Synchronise and report the first device-side failure of the factor:
 * CHD_OK, CHD_ERR_NOT_PD, CHD_ERR_NOT_COMPLETABLE or CHD_ERR_TIMEOUT.
 */
chd_status chd_status_get(chd_factor* fac);

/*
 * Synchronise and return the first failing supernode and column (analysed
 * numbering) recorded by the device, or -1, -1.
 */
chd_status chd_error_detail(chd_factor* fac, int64_t* supernode, int64_t* column);

/* Number of kernels the library has launched since the process started
   (host counter, for launch accounting). */
int64_t chd_kernel_launches(void);

/* Measurement utility (not an operation of the paper): number of dense-tier
   products the library has split along their inner dimension since the
   process started (each split product adds one reduction launch that sums
   the partial products in a fixed order).  Host counter of directly issued
   launches; replays of captured CUDA graphs do not add to it.  Tests use it
   to check that a workload reaches the split path. */
int64_t chd_split_k_launches(void);

/* Measurement utility (not an operation of the paper): bf16 tensor-core
   flops issued by the library's FP64-accurate digit products (chd_dgemm_tc
   excluded) since the process started, counting every MMA the product
   kernels execute (36 digit pairs of each computed 128 x 32 output tile).
   Host counter of directly issued products; replays of captured CUDA graphs
   do not add to it. */
double chd_tc_flops(void);

/*
 * Measurement utility (not an operation of the paper): FP64 fused
 * multiply-add throughput of the current device in GFLOP/s, from a kernel
 * of independent DFMA chains on every SM timed with CUDA events on
 * `stream` (synchronises).  It is the denominator of the FP64 roofline of
 * the front kernels.  Allocates and frees one small device buffer.
 */
chd_status chd_probe_fp64_peak(void* stream, double* gflops);

/*
 * Measurement and test utility (not an operation of the paper): C = beta C +
 * alpha A B for column-major FP64 matrices on the device (A m x k, lda >= m;
 * B k x n, ldb >= k; C m x n, ldc >= m) computed on the bf16 tensor cores
 * by splitting A's rows and B's columns into eight 7-bit integer digits
 * (error-free digit products, Ozaki et al. 2012) and summing the digit
 * products by level in FP32 tensor-memory accumulators.  The error is of
 * the order of an FP64 product's, 2^-53 k max_l |a_il| max_l |b_lj|, relative
 * to row and column maxima.  The dense tier of the library uses the same
 * kernels for its large products.  Allocates and frees scratch on `stream`
 * (stream-ordered) and synchronises it.  Errors: CHD_ERR_INVALID for
 * negative sizes or short leading dimensions, CHD_ERR_OOM, CHD_ERR_CUDA,
 * CHD_ERR_TIMEOUT if a bounded wait inside the kernel ran out.
 */
chd_status chd_dgemm_tc(int64_t m, int64_t n, int64_t k, double alpha, const double* a, int64_t lda,
                        const double* b, int64_t ldb, double beta, double* c, int64_t ldc, void* stream);

/*
 * Measurement utility (not an operation of the paper): throughput of raw
 * bf16 tcgen05.mma (M = 128, N = 256, K = 16, FP32 accumulation) on every
 * SM, in TFLOP/s, timed with CUDA events on `stream` (synchronises).  The
 * denominator of the tensor-core roofline of chd_dgemm_tc.
 */
chd_status chd_probe_tc_bf16_peak(void* stream, double* tflops);

/*
 * Measurement utility (not an operation of the paper): the arithmetic units
 * the front kernels can use, on every SM of the current device, timed with
 * CUDA events on `stream` (synchronises).  out[0]: FP64 FMA throughput
 * (TFLOP/s, eight independent chains per thread); out[1]: FP64 warp-level
 * MMA (mma.sync m8n8k4 .f64, TFLOP/s); out[2]: FP32 FMA throughput
 * (TFLOP/s); out[3]: latency of a dependent FP64 FMA (ns).  Allocates and
 * frees one small device buffer (stream-ordered).
 */
chd_status chd_probe_units(void* stream, double out[4]);

void chd_factor_free(chd_factor* fac);

/*
 * Workspace control of a factor object (device memory the library holds for
 * the per-front workspace of Hessian-type calls; it grows to the largest
 * batch of right-hand sides a call processes at once).  The workspace is a
 * stream-ordered allocation (cudaMallocAsync / cudaFreeAsync) on the stream
 * of the call that grows or releases it, so neither synchronises the device;
 * successive calls on one factor object must be ordered (one stream, or
 * synchronised by the caller).
 *   chd_factor_set_workspace_limit: cap it at `bytes` (0 = library default,
 *     48 GiB); larger batches are processed in chunks, at least one
 *     right-hand side at a time.
 *   chd_factor_release_workspace: free the workspace, ordered after the
 *     work already issued on the factor's last stream (the next call
 *     allocates it again).
 *   chd_factor_workspace_bytes: bytes currently held.
 */
chd_status chd_factor_set_workspace_limit(chd_factor* fac, size_t bytes);
chd_status chd_factor_release_workspace(chd_factor* fac);
chd_status chd_factor_workspace_bytes(const chd_factor* fac, size_t* bytes);

/*
 * CUDA graphs of the launch sequences (not part of the paper; an execution
 * device of the library).  With graphs on (the default), a call of the same
 * kind with the same arguments as the previous one (device pointers, m,
 * strides) replays a graph of its kernel launches: the second such call
 * captures it, later ones replay it on the factor's private stream, which
 * waits for `stream` and which `stream` then waits for (events, no host
 * synchronisation).  Results are bitwise those of the direct launches.  A
 * graph holds the device pointers it was captured with: the caller must keep
 * those buffers allocated while it keeps calling with them (a call with other
 * pointers simply runs directly).  on = 0 destroys the graphs and runs every
 * call directly.  Returns CHD_ERR_INVALID for a NULL factor.
 */
chd_status chd_factor_set_graphs(chd_factor* fac, int on);

/*
 * The longest launch sequence (in kernel launches of the direct run) that is
 * captured into a graph; longer sequences run directly.  Capturing and
 * instantiating a graph costs host time and memory in proportion to its
 * launches (about 1.5 s for the 445 579 launches of a 40 x 40 x 40 grid's
 * completion, which then replays in 0.98 s against 2.0 s launched
 * directly), paid again whenever a call repeats the previous arguments of
 * its kind after others: raise the limit for callers that repeat their
 * calls with kept buffers.  Default 8192.
 * CHD_ERR_INVALID for a NULL factor or a negative limit.
 */
chd_status chd_factor_set_graph_limit(chd_factor* fac, int64_t max_launches);

/*
 * Hessian products that allocate nothing.  The paper has no counterpart:
 * this is a service entry point of the library.
 *
 * For callers that cannot let a library call cudaMalloc while they run:
 * programs whose device memory is all handed out by their own allocator
 * (a framework's caching pool, or one arena reserved at start-up), and
 * services that forbid allocator calls after warm-up because such calls can
 * block or fragment memory.  It computes the same T_i = P(X^{-1} Y_i X^{-1})
 * as chd_hessian with the same kernels, but the per-front workspace is a
 * fixed device array of 2 Mi doubles (16 MiB) compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   fac     a factor whose projected inverse is already cached (call
 *           chd_gradient or chd_hessian on it once before); it is read only
 *   m, y_dev, ldy, t_dev, ldt   as for chd_hessian (device pointers, caller-owned)
 *   stream  cudaStream_t as void*
 * Returns CHD_ERR_INVALID when the projected inverse is not cached, when
 * m times the pattern's per-right-hand-side workspace exceeds the 2 Mi
 * doubles (small and medium patterns fit; use chd_hessian otherwise), or
 * when m > 65535 (chd_hessian splits larger batches itself);
 * CHD_ERR_CUDA if a CUDA call fails.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 * Set-up: the first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after a cudaDeviceReset, which unloads the library's device
 * code, it is stale, so do not use this entry point on a device after
 * resetting it.
 * Sharing: all calls on a device share the one array and it keeps the
 * contents of the last call; calls whose kernels overlap on the GPU (on
 * different streams, or from several threads) race on it and give wrong
 * results.  Serialise them, e.g. on one stream.
 */
chd_status chd_hessian_noalloc(chd_factor* fac, int m, const double* y_dev, int64_t ldy, double* t_dev,
                               int64_t ldt, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CHORDAL_BARRIER_H */
