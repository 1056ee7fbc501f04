/*
 * ibmi.h -- C ABI of the GB300 IBMI block-sweep inverter.
 *
 * IBMI (Iterative Block Matrix Inversion) approximates the whole inverse
 * H ~= A^{-1} of a dense symmetric positive definite A in R^{p x p}
 * (Section 2, Algorithm 1).  The index range {0..p-1} is covered by K
 * contiguous, possibly overlapping sets I_k = [lo_k, hi_k).  One sweep visits
 * k = 1..K in order and rewrites rows and columns I_k of H with the approximate
 * block-inversion formula (eq. IBMI), taking T = H[I_k^c, I_k^c] from the most
 * recent iterate as the approximation of the inverse Schur complement:
 *
 *     H[I,I^c] = -A_I^{-1} A_{I,I^c} T,   H[I^c,I] = H[I,I^c]^T,
 *     H[I,I]   =  A_I^{-1} + A_I^{-1} A_{I,I^c} T A_{I^c,I} A_I^{-1}.
 *
 * Sweeps repeat until the stop quantity is <= tol (Algorithm 1).  The default
 * stop quantity is rho_F = ||I - A H||_F / sqrt(p); the paper's own estimate
 * (eq. error, on the last set) can be selected instead.  An optional
 * Newton-Schulz tail (eq. newton) refines H once ||I - A H||_F <= ns_theta.
 *
 * Conventions for every entry point:
 *   - Matrices are dense, row-major, FP64, with a leading dimension ld >= p
 *     (in elements).  Since A and H are symmetric, row- and column-major agree.
 *   - A is read-only, and only its lower triangle (i >= j) is read: the
 *     strict upper triangle may hold anything.  H is owned by the caller and
 *     written in full.
 *   - Device pointers must be CUDA device memory of the current device (or
 *     managed memory); a pointer into another GPU's memory is rejected;
 *     "_host" variants take host memory and copy inside the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are synchronous with respect to the host: when an entry point
 *     returns, its result is final.
 *   - Every call returns an ibmi_status; nothing aborts the process.  On a CUDA
 *     error the call returns IBMI_ERR_CUDA and ibmi_last_error() describes it.
 */
#ifndef IBMI_H_
#define IBMI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ibmi_status {
  IBMI_OK = 0,
  IBMI_ERR_INVALID_ARG = 1,   /* bad size, set layout, pointer or option          */
  IBMI_ERR_NOT_SPD = 2,       /* Cholesky of a diagonal block A_{I_k} failed      */
  IBMI_NOT_CONVERGED = 3,     /* max_sweeps (and ns_max) reached; H = last iterate */
  IBMI_ERR_NONFINITE = 4,     /* the residual became NaN or Inf                   */
  IBMI_ERR_BUDGET = 5,        /* request exceeds the server's HBM budget          */
  IBMI_ERR_OOM = 6,           /* device allocation failed                         */
  IBMI_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up               */
  IBMI_ERR_CUDA = 8,          /* CUDA runtime error, see ibmi_last_error()        */
  IBMI_NOT_READY = 9,         /* served request still in flight                   */
  IBMI_ERR_CANCELLED = 10     /* served request was cancelled                     */
} ibmi_status;

/* Arithmetic of the sweep products (a3/a4).  The Cholesky of the diagonal
 * blocks and the residual are FP64-accurate in both modes: DFMA in IBMI_FP64;
 * in IBMI_MIXED the residual, and for blocks of order >= 512 the factorisation
 * updates beyond each 256-wide block column and A_I^{-1} = Y^T Y, run as
 * error-free digit-sliced products on the tensor cores. */
typedef enum ibmi_precision {
  IBMI_FP64 = 0,    /* every product in FP64 (DFMA)                                 */
  IBMI_MIXED = 1    /* sweep products on tcgen05 tensor cores with split-BF16 operands
                       and FP32 accumulation; FP64 Newton-Schulz tail restores accuracy */
} ibmi_precision;

typedef enum ibmi_stop_rule {
  IBMI_STOP_RESID_F = 0,    /* ||I - A H||_F / sqrt(p) <= tol                       */
  IBMI_STOP_PAPER_EST = 1   /* eq. error on the last set, ||(H A)_{I_K, I_K^c}||_2 <= tol
                               (FP64 path only; the residual is evaluated once at the end) */
} ibmi_stop_rule;

typedef enum ibmi_init {
  IBMI_INIT_IDENTITY = 0,   /* H[I_1^c, I_1^c] = identity (Section 2.4)              */
  IBMI_INIT_USER = 1,       /* the caller's H holds the initial guess in H[I_1^c, I_1^c];
                               it should be SPD (Theorem of Section 3)               */
  IBMI_INIT_SCHUR = 2       /* H[I_1^c, I_1^c] = A_{I_1^c}^{-1}, the inverse of A's block on
                               the complement [hi_1, p) of the first set (one of the
                               initial guesses of Section 5.6, Table 6), formed on the
                               device: FP64 Cholesky of the block and its inverse (the
                               mixed path forms Y^T Y, Y = L^{-1}, with exact sliced
                               tensor-core products from order 1024).  The plan holds
                               about 2 (p - m_1)^2 doubles for it.  A non-SPD block
                               returns IBMI_ERR_NOT_SPD with bad_block = K.             */
} ibmi_init;

/* Plan description.  Fill with ibmi_plan_desc_init() then override fields. */
typedef struct ibmi_plan_desc {
  int64_t p;               /* matrix order, >= 2                                           */
  int32_t K;               /* number of index sets, 1 <= K <= p (K = 1 is a direct inverse) */
  int64_t h;               /* overlap half-width for the default layout (see below)        */
  const int64_t* lo;       /* optional explicit sets: K ascending starts (host, copied) ... */
  const int64_t* hi;       /* ... and ends; NULL = default layout                           */
  int32_t precision;       /* ibmi_precision (with a single set, K = 1, H = A^{-1} is the
                              FP64 block inverse for either precision)                 */
  double tol;              /* stop tolerance (default 1e-10)                                */
  int32_t max_sweeps;      /* sweep cap (default 500, the cap used in Section 5)           */
  int32_t stop_rule;       /* ibmi_stop_rule                                                */
  int32_t check_every;     /* minimum sweeps between stop tests (default 1); the library
                              spaces tests up to 8 sweeps apart while the contraction seen
                              between tests predicts the target is still further away
                              (never stops earlier than a test on every sweep would)   */
  double ns_theta;         /* enter Newton-Schulz once ||I - A H||_F <= ns_theta; 0 = off  */
  int32_t ns_max;          /* Newton-Schulz step cap (default 8)                            */
  int32_t init;            /* ibmi_init                                                     */
} ibmi_plan_desc;
/* Default layout (Section 4 cost model): core k = [floor(k p/K), floor((k+1) p/K)),
 * set k = core widened by h on each side that has a neighbour, clipped to [0,p).
 * Explicit sets must be contiguous, ascending (lo_k < lo_{k+1}, hi_k < hi_{k+1}),
 * cover {0..p-1}, and each must leave a non-empty complement when K >= 2.        */

typedef struct ibmi_result {
  int32_t status;          /* same value as the call's return                              */
  int32_t sweeps;          /* sweeps r performed                                            */
  int32_t ns_steps;        /* Newton-Schulz steps performed                                 */
  int32_t bad_block;       /* IBMI_ERR_NOT_SPD: set index k (0-based), else -1              */
  int64_t bad_pivot;       /* IBMI_ERR_NOT_SPD: global row of the failed pivot, else -1     */
  double resid_f;          /* last ||I - A H||_F / sqrt(p) evaluated (FP64)                 */
  double paper_est;        /* last eq. error estimate (NaN unless evaluated)                */
  double seconds;          /* wall time of the call on the stream                          */
  double flops;            /* algorithmic flops: plan + sweeps + residuals + Newton-Schulz;
                              a digit-sliced residual or update that keeps part of its
                              pair products counts that share of its 2 p^3 (mixed)          */
} ibmi_result;

typedef struct ibmi_plan_s* ibmi_plan_t;

/* Fills *desc with defaults: K=2, h=0, FP64, tol=1e-10, max_sweeps=500,
 * RESID_F, check_every=1, ns_theta=0, ns_max=8, IDENTITY. */
void ibmi_plan_desc_init(ibmi_plan_desc* desc);

/* Validates the description (set coverage, sizes) and allocates the plan's
 * device workspace on the current device: per set A_I^{-1} (m x m) and
 * W = A_I^{-1} A_{I,:} stored m x p with zero columns on I, plus scratch.
 * The plan owns that memory until ibmi_plan_destroy.  Returns
 * IBMI_ERR_INVALID_ARG (nothing allocated) or IBMI_ERR_OOM. */
ibmi_status ibmi_plan(const ibmi_plan_desc* desc, ibmi_plan_t* out);
ibmi_status ibmi_plan_destroy(ibmi_plan_t plan);

/* Copies the plan's sets to host arrays lo[K], hi[K] (either may be NULL). */
ibmi_status ibmi_plan_sets(ibmi_plan_t plan, int32_t* K, int64_t* lo, int64_t* hi);

/* Algorithm 1 on device buffers.  A: p x p SPD (lda >= p), read-only.
 * H: p x p output (ldh >= p); with IBMI_INIT_USER it also carries the initial
 * guess.  A and H must not overlap.  Returns IBMI_OK, IBMI_NOT_CONVERGED
 * (H = last iterate), IBMI_ERR_NOT_SPD (bad_block/bad_pivot set, H undefined),
 * IBMI_ERR_NONFINITE, IBMI_ERR_INVALID_ARG or IBMI_ERR_CUDA.  `out` may be NULL. */
ibmi_status ibmi_invert(ibmi_plan_t plan, const double* A, int64_t lda, double* H,
                        int64_t ldh, void* stream, ibmi_result* out);

/* Partial inverse (Section 6, Discussion: approximating only block-diagonal
 * parts of the inverse): the diagonal blocks H[I_1, I_1] and H[I_2, I_2] of
 * the IBMI iterate for a plan with exactly two sets (any overlap), without
 * forming the rest of H.  With two sets the step for I_1 reads
 * T = H[I_1^c, I_1^c], which lies inside H[I_2, I_2], and the step for I_2
 * reads H[I_2^c, I_2^c] inside H[I_1, I_1] (eq. IBMI), so the two blocks
 * evolve on their own with the same products as the full sweep; after the
 * last sweep D holds exactly the diagonal blocks of the full iterate.
 * D: device, m_1^2 + m_2^2 doubles: H[I_1, I_1] (m_1 x m_1, row-major), then
 * H[I_2, I_2] (m_2 x m_2); written in full.  With IBMI_INIT_USER the second
 * block of D carries the initial guess of H[I_2, I_2], of which only the
 * part on I_1^c = [hi_1, p) is read.  Stop quantity (out->resid_f): the last
 * set's rows of the residual, ||(H A - I)[I_2, :]||_F / sqrt(p), evaluated
 * like the stop test of ibmi_invert (check_every and the cadence); it is zero
 * exactly when H[I_2^c, I_2^c] is the inverse Schur complement.  The plan
 * must be IBMI_FP64 with IBMI_STOP_RESID_F (else IBMI_ERR_INVALID_ARG).
 * Work per sweep as ibmi_invert's; device memory m_1^2 + m_2^2 (the caller's
 * D) plus m_max p + m_2 p doubles of scratch the plan allocates on first use,
 * instead of the p^2 of H.  Returns like ibmi_invert. */
ibmi_status ibmi_invert_block_diag(ibmi_plan_t plan, const double* A, int64_t lda, double* D, void* stream,
                                   ibmi_result* out);

/* Same on host buffers: copies A (and H for IBMI_INIT_USER) to the device,
 * runs ibmi_invert, copies H back.  Uses device scratch owned by the plan. */
ibmi_status ibmi_invert_host(ibmi_plan_t plan, const double* A_host, int64_t lda,
                             double* H_host, int64_t ldh, void* stream, ibmi_result* out);

/* rho_F = ||I - A H||_F / sqrt(p) in FP64 (DFMA) for device A, H (p x p,
 * ld >= p); the value is written to *out (host).  Allocates a small buffer of
 * per-tile partial sums (stream-ordered) for the duration of the call. */
ibmi_status ibmi_residual(const double* A, int64_t lda, const double* H, int64_t ldh,
                          int64_t p, void* stream, double* out);

/* ------------------------------------------------------------------------
 * Partition and ordering search for one matrix.
 *
 * Section 5.4 (Tables 3-4) finds the overlap of the sets decisive for the
 * convergence of Algorithm 1 and the number of sets less so; Section 5.7 finds
 * the ordering of the rows decisive as well (a red-black ordering of a matrix
 * that contiguous sets over its natural ordering invert in a few sweeps
 * mostly fails to converge), and the discussion closing Section 5 recommends
 * orderings that keep the weight of the matrix near its diagonal.
 * ------------------------------------------------------------------------ */
typedef enum ibmi_order {
  IBMI_ORDER_IDENTITY = 0,  /* the given order                                            */
  IBMI_ORDER_XSORT = 1,     /* by the first coordinate (stable)                           */
  IBMI_ORDER_HILBERT = 2,   /* along a Hilbert curve through the bounding box of the
                               points (any dimension; 62 / dim bits per axis, at most 20)  */
  IBMI_ORDER_KD = 3,        /* leaves of a k-d tree: median split across the coordinate of
                               widest spread, recursively, left half first                 */
  IBMI_ORDER_REDBLACK = 4   /* even positions of the given order, then odd positions (the
                               red-black ordering Section 5.7 compares against)           */
} ibmi_order;

/* Ordering of n points (host, n x dim row-major doubles, 1 <= dim <= 16):
 * perm[i] (host, n entries) = the index of the point placed at position i, so
 * that the covariance matrix in the new order is A'[i][j] = A[perm[i]][perm[j]].
 * Host code only.  IBMI_ERR_INVALID_ARG for a bad order, size or a non-finite
 * coordinate. */
ibmi_status ibmi_order_points(const double* points, int64_t n, int32_t dim, int32_t order, int64_t* perm);

/* Symmetric permutation on the device: B[i][j] = A[perm[i]][perm[j]]
 * (inverse = 0) or B[perm[i]][perm[j]] = A[i][j] (inverse = 1), for the
 * symmetric A of order p whose lower triangle is read (element (r, c) from
 * (max, min)).  perm: host array of p distinct indices (copied).  A and B
 * must not be the same buffer.  Allocates p indices (stream-ordered) for the
 * call; synchronises `stream`. */
ibmi_status ibmi_permute(const double* A, int64_t lda, int64_t p, const int64_t* perm, int32_t inverse, double* B,
                         int64_t ldb, void* stream);

typedef struct ibmi_tune_candidate {
  int32_t order;           /* -1: the given order; else the index of the caller's permutation */
  int32_t K;               /* sets                                                            */
  int64_t h;               /* overlap half-width of the default layout                         */
  int32_t status;          /* ibmi_status of the inversion with this choice                    */
  int32_t sweeps;
  int32_t ns_steps;
  double seconds;          /* device time of the whole inversion (CUDA events), INFINITY if none */
  double resid_f;
} ibmi_tune_candidate;

/* Measured search over orderings and partitions of one device matrix A
 * (p x p, lda): for the given order and each of the n_perms host permutations
 * (each p distinct indices, as from ibmi_order_points), and each K in
 * {2, 3, 4, 6, 8} whose cores p / K have at least 64 rows with an overlap 2h
 * of 10, 20 and 30% of the core, the whole inversion runs once with the
 * options of `base` (precision, tol, max_sweeps, ns_theta, ...; its p, K, h
 * and sets are replaced; IBMI_INIT_USER becomes the identity) on the permuted
 * matrix, timed on the device.  *best: the fastest that converged (IBMI_OK);
 * all (optional, max_all entries) and *n_all: every candidate in the order
 * tried.  Returns IBMI_OK, or IBMI_NOT_CONVERGED when no candidate converged;
 * IBMI_ERR_CUDA / IBMI_ERR_TIMEOUT abort the search.  Allocates 2 p^2
 * doubles plus each candidate's plan while it runs.  Synchronous. */
ibmi_status ibmi_tune(const double* A, int64_t lda, int64_t p, const int64_t* const* perms, int32_t n_perms,
                      const ibmi_plan_desc* base, void* stream, ibmi_tune_candidate* best,
                      ibmi_tune_candidate* all, int32_t max_all, int32_t* n_all);

/* ------------------------------------------------------------------------
 * Many matrices: batched inversion and the continuous-batching server.
 *
 * Both run the single-matrix pipeline (Algorithm 1 with the options below) on
 * a pool of worker threads, one CUDA stream each, so the kernels of different
 * matrices overlap on the GPU.  A matrix of order p is padded to a size bucket
 * (multiples of 64 up to 1024, of 128 up to 4096, of 256 beyond) by embedding
 * it in [[A, 0], [0, I]], whose inverse is [[A^{-1}, 0], [0, I]]; one plan per
 * bucket then serves all matrices of that bucket.  With autotune set, the
 * partition (K in 2..4, overlap 2h of 10/20/30% of the core width) of each
 * bucket is chosen by timing the candidates on the first matrix of the bucket
 * (cached for the process).  Results are bitwise independent of which other
 * matrices run at the same time: every kernel is deterministic and each
 * matrix has its own buffers.
 * ------------------------------------------------------------------------ */
typedef struct ibmi_batch_opts {
  int32_t precision;   /* IBMI_MIXED (default) or IBMI_FP64                     */
  double tol;          /* default 1e-10 (rho_F)                                */
  int32_t max_sweeps;  /* default 500                                          */
  double ns_theta;     /* Newton-Schulz hand-over (mixed); default 0: by order,
                          3.0 up to p = 1024, 0.9 above                       */
  int32_t ns_max;      /* default 8                                            */
  int32_t workers;     /* concurrent streams, 1..64, default 8                 */
  int32_t autotune;    /* 1 (default): tune (K, h) per size bucket              */
  int32_t graphs;      /* 1 (default): mixed plans replay captured CUDA graphs
                          (one capture per plan and phase); 0: direct launches.
                          Both give bit-identical results.                     */
  int32_t device_batch; /* 1 (default, mixed precision): matrices of order <= 2048
                          of one size bucket and partition run as groups in
                          lockstep on the device -- every launch covers one step
                          of all matrices of the group that take it, with one
                          host synchronisation per round of the group; a matrix
                          the lockstep rules leave unfinished (a stall needing
                          the spectral-radius test, a failed tail, the sweep
                          cap) is run again on the single-matrix pipeline.
                          Each result is bitwise the same whatever the group
                          around it.  0: every matrix on the single-matrix
                          pipeline of a worker.                                */
} ibmi_batch_opts;
void ibmi_batch_opts_init(ibmi_batch_opts* opts);

/* Device bytes a plan with this description allocates (estimate). */
size_t ibmi_plan_bytes(const ibmi_plan_desc* desc);

/* Inverts n SPD matrices; A[i], H[i] are device pointers to p[i] x p[i]
 * row-major FP64 matrices with leading dimensions lda[i], ldh[i].  Per-matrix
 * results in out[i] (status, sweeps, ...).  A matrix that does not converge
 * with its bucket's tuned partition is run once more with cores of about 256
 * rows (2 to 8 sets) and 30% overlap (its counts then include both runs).  Returns IBMI_OK when all
 * converged, else the first failure status (NOT_CONVERGED ranks lowest).
 * Synchronous.  The worker pool (streams, plans, captured CUDA graphs) is
 * kept for the next call on the same device until ibmi_batch_release();
 * batched calls are serialised. */
ibmi_status ibmi_invert_batched(int32_t n, const int64_t* p, const double* const* A, const int64_t* lda,
                                double* const* H, const int64_t* ldh, const ibmi_batch_opts* opts,
                                ibmi_result* out);

/* Counters of the last ibmi_invert_batched call of this process: matrices
 * run as device groups, groups, rounds (the longest group's and the sum over
 * groups), matrices handed on to the single-matrix pipeline after their group
 * (fallbacks), and the wall seconds of the group phase and of the
 * single-matrix phase.  Observability only. */
typedef struct ibmi_batch_stats {
  int64_t device_matrices;
  int64_t groups;
  int64_t rounds_max;
  int64_t rounds_total;
  int64_t fallbacks;
  double seconds_groups;
  double seconds_single;
} ibmi_batch_stats;
ibmi_status ibmi_batch_last_stats(ibmi_batch_stats* out);

/* Frees the pooled batch workers (streams, plans, graphs) of every device. */
ibmi_status ibmi_batch_release(void);

/* Continuous-batching server.  Requests (host matrices) are queued; a request
 * is admitted when its device bytes (A, H and padded staging, 16 (p^2 + pb^2)
 * bytes) fit in a quarter of hbm_budget beside the admitted ones (the other
 * three quarters cap the workers' plan caches, least recently used plans
 * going first); admitted requests run as soon
 * as a worker is free, overlapping on the device with the others; finishing
 * frees their bytes for the next ones in arrival order.  ibmi_serve_submit
 * copies A (p x p, lda); IBMI_ERR_BUDGET if one request alone exceeds the
 * budget.  ibmi_serve_poll returns IBMI_NOT_READY until the request is done,
 * then copies H (ldh) and the result and forgets the request.
 * ibmi_serve_cancel removes a queued request (IBMI_NOT_READY once it has been
 * admitted).  ibmi_serve_stats: p50/p99 latency (submit to completion,
 * seconds) and completion throughput over all completed requests. */
typedef struct ibmi_server_impl* ibmi_server_t;
ibmi_status ibmi_serve_create(size_t hbm_budget, const ibmi_batch_opts* opts, ibmi_server_t* out);
ibmi_status ibmi_serve_submit(ibmi_server_t server, const double* A_host, int64_t p, int64_t lda, double tol,
                              uint64_t* request);
ibmi_status ibmi_serve_poll(ibmi_server_t server, uint64_t request, double* H_host, int64_t ldh,
                            ibmi_result* out);
ibmi_status ibmi_serve_cancel(ibmi_server_t server, uint64_t request);
ibmi_status ibmi_serve_stats(ibmi_server_t server, double* p50_s, double* p99_s, double* inverses_per_s,
                             int64_t* completed, uint64_t* bytes_in_use);
/* Forgets the latencies and completion counts gathered so far (for example
 * after a warm-up that created the workers' plans); requests in flight are
 * counted when they finish. */
ibmi_status ibmi_serve_stats_reset(ibmi_server_t server);
ibmi_status ibmi_serve_destroy(ibmi_server_t server);

/* Kernel profiling, for the benchmark's roofline figures.  While enabled, the
 * library records a CUDA event pair on the launching stream around every
 * launch of each kernel class below and sums their durations; it also counts
 * every kernel launch it makes.  ibmi_prof_enable(1) clears the counters.
 * ibmi_prof_get synchronises the recorded events.  Not thread-safe: profile
 * one thread at a time. */
typedef enum ibmi_kernel_class {
  IBMI_K_SWEEP_X = 0,     /* a3: X = -W T and its scatter into H                 */
  IBMI_K_SWEEP_S = 1,     /* a4: S = A_I^{-1} - X W^T                             */
  IBMI_K_RESIDUAL = 2,    /* a6: ||I - A H||_F products                           */
  IBMI_K_NS = 3,          /* a7: Newton-Schulz update products                    */
  IBMI_K_INVARIANTS = 4,  /* a2: Cholesky, triangular solves (FP64 DFMA part)     */
  IBMI_K_OTHER = 5,       /* slicing, combines, symmetrisation, copies            */
  IBMI_K_INVARIANTS_TC = 6, /* a2, mixed path, on tensor cores: W = A_I^{-1} A_{I,:},
                               Y^T Y and the factorisation updates                  */
  IBMI_K_COUNT = 7
} ibmi_kernel_class;
/* The flops recorded per class are the operations issued to the unit that
 * executes them: FP64 DFMA for the FP64 path and the block factorisations;
 * tensor-pipe BF16 MMA flops for the tcgen05 kernels (a BF16x3 product issues
 * three times the flops of the product it represents, a digit-sliced FP64
 * product one plain GEMM per digit pair). */
void ibmi_prof_enable(int on);
/* launches: launches of that class; ms: summed event time; flops: algorithmic
 * flops of those launches.  Returns IBMI_ERR_INVALID_ARG for a bad class. */
ibmi_status ibmi_prof_get(int32_t kernel_class, int64_t* launches, double* ms, double* flops);
/* Algorithmic flops of the launches of that class recorded so far: the flops
 * of the products the method asks for (2 m n^2 for X = -W T, 2 p^3 for a
 * residual, ...), whatever the sliced arithmetic issued to do them; a digit-
 * sliced residual or update that keeps part of its pair products counts that
 * share.  Equal to the flops of ibmi_prof_get for the FP64 classes. */
ibmi_status ibmi_prof_get_alg(int32_t kernel_class, double* alg_flops);
/* Total kernel launches made by this library since the last ibmi_prof_enable(1)
 * (counted whether or not profiling is on). */
int64_t ibmi_launch_count(void);

/* ibmi_residual without any device allocation.  The paper has no counterpart:
 * this entry exists for callers that cannot call cudaMalloc -- code running
 * under an external manager that owns the device memory budget (a serving
 * process with hard admission limits) or a latency-critical loop in which an
 * allocation, and the device synchronisation it can imply, is not allowed.
 * Same arguments, result and meaning as ibmi_residual (FP64 DFMA,
 * rho_F = ||I - A H||_F / sqrt(p) written to *out), same kernels; like every
 * other entry point it reads only the lower triangle of A (the product reads
 * element (i, j) of A from (max(i, j), min(i, j)), so no symmetric copy is
 * needed).
 * Scratch: a fixed array of 16,386 doubles (about 128 KB) inside the library,
 * held on every GPU that loads the library until the process exits; it limits
 * the order to p <= 8192 -- larger p returns IBMI_ERR_INVALID_ARG with a
 * message in ibmi_last_error().  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress).  Every call copies the
 * result to the host and synchronises `stream`, so it must not be called
 * while that stream is being captured into a CUDA graph.  Every call reuses
 * the same array (each call writes all the partial sums it reads, so nothing
 * has to start at zero): calls that can overlap on the GPU -- on different
 * streams or from different host threads -- race on it and must be serialised
 * by the caller. */
ibmi_status ibmi_residual_noalloc(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                                  void* stream, double* out);

/* Newton-Schulz tail of the method on its own (eq. newton): refines a
 * symmetric approximate inverse X of the SPD matrix A in place,
 *     X <- sym(X + X (I - A X)),
 * until ||I - A X||_F / sqrt(p) <= tol, at most ns_max updates, stopping early
 * when an update does not reduce the residual.  IBMI_FP64 runs every product
 * with DFMA; IBMI_MIXED evaluates the residual with the error-free sliced
 * tensor-core products (FP64-accurate) and the update X (I - A X) from the five
 * leading digit slices of each operand (exact digit-pair products on tcgen05,
 * 2^-34 relative truncation).  Converges when ||I - A X_0|| < 1 (the
 * condition stated with eq. newton).  out->ns_steps counts updates and
 * out->resid_f is the last residual evaluated.  Allocates its workspace for
 * the duration of the call. */
ibmi_status ibmi_refine(const double* A, int64_t lda, double* X, int64_t ldx, int64_t p, int32_t precision,
                        double tol, int32_t ns_max, void* stream, ibmi_result* out);

/* rho_F = ||I - A H||_F / sqrt(p) for symmetric device A, H, computed on the
 * tcgen05 tensor cores with the error-free sliced products of the Newton-Schulz
 * tail: every row of H is cut into ten signed 7-bit digits (69 bits) and every
 * row of A into eight (55 bits), relative to the row maximum; the 52 exact
 * digit-pair products of digit groups 0..9 are accumulated in integers and
 * combined once in FP64, so the value agrees with an FP64 evaluation to FP64
 * rounding.  Allocates its workspace (about 100 p^2 bytes) for the duration
 * of the call.  H must be symmetric (the kernel evaluates ||I - H A||_F); A
 * is read from its lower triangle. */
ibmi_status ibmi_residual_tc(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                             void* stream, double* out);

/* Self-test of the bounded device-side waits (no counterpart in the paper):
 * runs one small tcgen05 launch whose loads are never issued, so the MMA
 * thread's wait on its first stage expires after about 2 s; the kernel then
 * records the timeout, waits for its own issued work, frees its tensor memory
 * and exits, and the call reads the error word.  Returns IBMI_ERR_TIMEOUT when
 * all of that worked (the intended outcome), IBMI_OK if the wait did not
 * expire, or IBMI_ERR_CUDA.  The CUDA context stays usable afterwards.
 * Allocates 16 KB for the call; synchronises `stream`. */
ibmi_status ibmi_selftest_wait_timeout(void* stream);

/* Human-readable name of a status, and the text of the last CUDA error seen by
 * this thread (empty if none). */
const char* ibmi_status_string(ibmi_status s);
const char* ibmi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IBMI_H_ */
