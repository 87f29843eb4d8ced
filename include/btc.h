/*
 * btc.h - C ABI of libbtc.so: nested-dissection Cholesky factorization and
 * solve of symmetric positive-definite block-tridiagonal matrices on GB300.
 *
 * The matrix (Sec. 3 of arXiv 2601.03754, the block-tridiagonal Psi) has N
 * diagonal blocks D_i and N-1 sub-diagonal blocks B_i = Psi(i+1, i), each
 * n x n (the paper names the sub-diagonal blocks E_i). The library factors
 * P Psi P^T = L L^T where P is the multi-stage permutation P_inf of Sec. 4.3
 * (recursive odd/even, i.e. nested dissection): all eliminations of one
 * dissection level are independent and run concurrently, over
 * floor(log2 N) + 1 levels (Alg. 5, hybrid left/right-looking), and solves
 * Psi x = b by level-wise forward and backward substitution (Alg. 7).
 *
 * Conventions for every entry point:
 *  - Return value: BTC_OK (0) or a negative BTC_ERR_* code; btc_last_error()
 *    then returns a message for the calling thread.
 *  - Indices are 0-based; arrays are dense row-major.
 *  - "device pointer" = memory the GPU can address (cudaMalloc'd or a torch
 *    CUDA tensor's data_ptr()); "host pointer" = ordinary host memory.
 *  - Work is enqueued on the CUDA stream given to btc_plan (NULL = legacy
 *    default stream) and is asynchronous unless stated otherwise.
 *  - The caller owns every pointer it passes; the plan owns its factor pools,
 *    work vectors and captured CUDA graphs, all released by btc_free.
 *  - One plan must not be used from two host threads at the same time.
 */
#ifndef BTC_H
#define BTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btc_plan_s *btc_plan_t;

/* Arithmetic of a plan. Input element type: FP64 for BTC_F64 and the three
 * BTC_MIXED_* dtypes, FP32 for BTC_F32. */
enum btc_dtype {
  BTC_F64 = 0,        /* factor and solve in FP64 (the plain FP64 path)                         */
  BTC_F32 = 1,        /* factor and solve in FP32                                                */
  BTC_MIXED_F32 = 2,  /* FP64 inputs; factor and correction solves in FP32 except the root
                         (top-separator) Cholesky, which runs in FP64 (or, as an option, in
                         double-FP32: btc_plan_set_root_precision); FP64 residual and update in
                         btc_solve_refined                                                       */
  BTC_MIXED_TF32 = 3, /* as BTC_MIXED_F32, with the four n^3 products of every node (the two
                         deferred syrk, the immediate syrk and the fill gemm of Alg. 5) on the
                         tcgen05 tensor cores with TF32 operands and FP32 accumulation, for
                         padded block size 128 (97 <= n <= 128); smaller blocks run the
                         BTC_MIXED_F32 kernels. Its factor is less accurate than FP32 (TF32 has
                         a 10-bit mantissa); the FP64 refinement of btc_solve_refined recovers
                         the solution's accuracy in a few more steps                            */
  BTC_MIXED_BF16 = 4, /* as BTC_MIXED_TF32 with BF16 operands (8-bit mantissa; kind::f16 MMAs,
                         FP32 accumulation) for the four n^3 products: twice the tensor rate and
                         half the operand bytes of TF32, a factor about 8 times less accurate, so
                         refinement needs more steps, and for ill-conditioned matrices classical
                         refinement can stall where btc_solve_gmres_ir still converges          */
};

enum btc_status {
  BTC_OK = 0,
  BTC_ERR_ARG = -1,           /* invalid argument (sizes, NULL, misaligned pointer)        */
  BTC_ERR_OOM = -2,           /* device allocation failed                                  */
  BTC_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the CUDA error)   */
  BTC_ERR_NOT_SPD = -4,       /* a pivot was not positive (see btc_info)                   */
  BTC_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up                        */
  BTC_ERR_NOT_FACTORED = -6,  /* solve called before a successful btc_factor               */
  BTC_ERR_UNSUPPORTED = -7,   /* block size or dtype not compiled into this library        */
  BTC_ERR_NOT_CONVERGED = -8, /* refinement stopped above the tolerance                    */
};

/* Static description of a plan, produced by the host planner alone. */
typedef struct btc_plan_info {
  int N, n, np;            /* blocks, block size, padded block size used on the device          */
  int levels;              /* floor(log2 N) + 1 (Sec. 4.3)                                      */
  int dtype;
  int64_t offdiag_blocks;  /* all off-diagonal factor blocks, original + fill (sum over levels
                              of floor(N / 2^(l-1)) - 1)                                         */
  int64_t fill_blocks;     /* offdiag_blocks - (N - 1)                                          */
  double factor_flops;     /* (N/3 + 2 offdiag + 2 fill) n^3, Table 1 costs summed over Alg. 5 */
  double seq_factor_flops; /* (7/3 N - 2) n^3, Alg. 1 (Sec. 3.1)                                */
  double critical_path_flops; /* sum over levels of the largest per-node cost (p = infinity)   */
  double critical_path_formula; /* the closed form of Sec. 4.3 with p = infinity, N >= 2       */
  double solve_flops_per_rhs;   /* 2 n^2 per node (trsm) + 4 n^2 per off-diagonal block        */
  double factor_bytes;     /* compulsory bytes: read D, B once; write Dhat and every U block    */
  double solve_bytes;      /* compulsory bytes per solve with m=1: read the factor twice        */
  int64_t device_bytes;    /* bytes the plan allocates on the device                            */
} btc_plan_info;

/*
 * Host-only planner (no GPU needed): fill *info for an (N, n, dtype) plan.
 * Returns BTC_ERR_ARG for N < 1 or n < 1, BTC_ERR_UNSUPPORTED when n exceeds
 * the largest compiled block size for dtype.
 */
int btc_describe(int N, int n, int dtype, btc_plan_info *info);

/*
 * Host-only: the per-level schedule of Alg. 5 for an N-block plan, for
 * inspection and tests. levels_out[t] receives the dissection level (1-based)
 * of the t-th eliminated node and order_out[t] the node (0-based), for
 * t = 0..N-1, in the order the levels run (within a level: ascending node).
 * This is the elimination order P_inf of Sec. 4.3.
 */
int btc_schedule(int N, int *order_out, int *levels_out);

/*
 * Host-only: the launch order of the interlaced factorization + forward
 * substitution (btc_factor_solve) for an N-block plan, for inspection and
 * tests. root_separate != 0: the mixed-precision form, whose top-separator
 * factor and forward item run outside the interlaced launch. On input *count
 * is the capacity of the arrays (all four may be NULL to query the length);
 * on output it is the number of entries. Entry t: kind[t] 0 = factor item,
 * 1 = forward item; node[t] 1-based node; level[t] dissection level;
 * deps[6t .. 6t+5] earlier entries it waits for (-1: none; d >= 0: entry d
 * complete; d <= -2: only the factor blocks of entry -d-2, which a factor
 * entry stores and publishes before its trailing products). *tail_count (may
 * be NULL): items of the second launch (top-separator forward item when
 * root_separate, then every backward item).
 */
int btc_schedule_interlaced(int N, int root_separate, int *kind, int *node, int *level, int *deps, int *count,
                            int *tail_count);

/*
 * Create a plan for one N-block, n x n system: plans the dissection levels on
 * the host, allocates the device pools (padded n_p x n_p blocks, level-major),
 * and binds `stream` (a cudaStream_t, NULL for the legacy default stream).
 * The plan must be released with btc_free. Errors: BTC_ERR_ARG,
 * BTC_ERR_UNSUPPORTED, BTC_ERR_OOM, BTC_ERR_CUDA.
 */
int btc_plan(btc_plan_t *out, int N, int n, int dtype, void *stream);

/*
 * Launch schedule of a plan's factor and solve (default BTC_SCHED_FLOW).
 * BTC_SCHED_LEVELS: one kernel launch per dissection level (Alg. 5 and 7 run
 * level by level, the launches ordered on the stream). BTC_SCHED_FLOW: one
 * persistent launch for all levels; each node starts as soon as the (at most
 * three) nodes of the previous level that produce its inputs are done, with
 * bounded device-side waits (BTC_ERR_TIMEOUT from btc_info if one gives up).
 * Both schedules perform identical arithmetic per node, so their results are
 * bitwise equal.
 */
enum btc_schedule_mode { BTC_SCHED_LEVELS = 0, BTC_SCHED_FLOW = 1 };
int btc_plan_set_schedule(btc_plan_t p, int mode);

/*
 * Factorization variant (default BTC_VARIANT_HYBRID).
 * BTC_VARIANT_HYBRID: Alg. 5 — hybrid left/right-looking; the update of the
 *   upper neighbour is deferred to the next level, every block has one writer
 *   per level, results are deterministic.
 * BTC_VARIANT_RIGHT_LOOKING: Alg. 6 — fully right-looking; after an explicit
 *   packing pass (its first parallel loop), each node updates both neighbours'
 *   diagonal blocks at once with floating-point atomics (at most two writers
 *   per block), shortening the per-level chain by the deferred syrk; the
 *   summation order of the two updates is not fixed, so results may differ
 *   from run to run by rounding.
 */
enum btc_variant { BTC_VARIANT_HYBRID = 0, BTC_VARIANT_RIGHT_LOOKING = 1 };
int btc_plan_set_variant(btc_plan_t p, int variant);

/*
 * Elimination order of the plan (default BTC_ORDER_ND).
 * BTC_ORDER_ND: the multi-stage (nested-dissection) permutation P_inf of
 *   Sec. 4.3, floor(log2 N) + 1 dependent levels, about (19/3) N n^3 flops.
 * BTC_ORDER_PARTITION: the partition permutation Psi_p of Sec. 4.1 (Alg. 4)
 *   with `chunks` = p chunks and p - 1 pivots, chunk sizes by Proposition 1
 *   (N_1 / N_k = 19 / 7, rounded to the split with the smaller larger phase
 *   cost): every chunk is eliminated left to right as a chain (chunks in
 *   parallel), then the pivots in order. chunks = 1 is the natural order of
 *   Alg. 1 ((7/3) N n^3 flops, a chain of N nodes). Fewer flops than ND for
 *   few chunks, a longer dependent chain: for throughput modes with much
 *   instance parallelism rather than for the latency of one system.
 * The plan's pools and schedules are rebuilt (synchronizes the plan's stream;
 * the previous factor is lost). Partition plans convert the caller's D and B
 * in a packing pass, solve with the persistent schedule only, and do not use
 * the interlaced launch or the right-looking variant; the blocked 256 plans
 * keep ND. Errors: BTC_ERR_ARG (too many chunks for N), BTC_ERR_UNSUPPORTED.
 */
enum btc_order { BTC_ORDER_ND = 0, BTC_ORDER_PARTITION = 1 };
int btc_plan_set_order(btc_plan_t p, int order, int chunks);

/*
 * Host-only planner (no GPU needed) for either elimination order: fills *info
 * as btc_describe does (info may be NULL) and, when not NULL, order_out[t] =
 * the t-th eliminated node (0-based) and levels_out[t] its launch level
 * (1-based: the chain position, then one level per pivot, for
 * BTC_ORDER_PARTITION), t = 0..N-1. Errors: BTC_ERR_ARG (bad arguments, too
 * many chunks), BTC_ERR_UNSUPPORTED (block size; partition orders of blocked
 * 256 plans).
 */
int btc_describe_order(int N, int n, int dtype, int order, int chunks, btc_plan_info *info, int *order_out,
                       int *levels_out);

/*
 * Host-only, for inspection and tests: the work items of a plan of N blocks in
 * either order, with every block offset in units of blocks (pool index).
 * Each count is the capacity of its array on input (rows; arrays may be NULL
 * to query) and the number of rows on output.
 * fac_rows, 14 per factor item in launch order: level (1-based), d_self,
 *   d_next, r_up, r_down, p_a, p_b, fill, d_prev (diagonal pool indices d_*,
 *   off-diagonal pool indices r_*, p_*, fill; -1: none), node (0-based),
 *   flags (1: the fill block holds S'(up, down), else S'(down, up); 2: top
 *   separator), then the three items it waits for (-1: none; d >= 0: item d
 *   complete; d <= -2: only item -d-2's factor blocks, i.e. its U blocks are
 *   stored before its trailing products: the next diagonal block and the fill).
 *   One item eliminates node e with the Schur complement S_e = Dhat[d_self]
 *   - P^T P (P = U[p_a]): S_e = U_e^T U_e; U[r_up] <- U_e^-T S(e, up);
 *   U[r_down] <- U_e^-T S(e, down); Dhat[d_next] -= U[r_down]^T U[r_down]
 *   (- U[p_b]^T U[p_b]); U[fill] <- -U[r_up]^T U[r_down] (or its transpose).
 * solve_rows, 10 per solve item: y_self, y_a, e_a, y_b, e_b, d_self, kind,
 *   three dependencies. kind 0 (forward): y_self -= U[e_a]^T y_a + U[e_b]^T
 *   y_b, then y_self <- U_self^-T y_self when d_self >= 0; kind 1 (backward):
 *   y_self <- U_self^-1 (y_self - U[e_a] y_a - U[e_b] y_b).
 * slot_rows, 3 per off-diagonal pool block: the node whose variables are its
 *   rows, the partner node, and for an original coupling slot v (nodes v,
 *   v + 1) 1 when it starts as B_v^T, 0 when B_v (-1 for fill slots).
 */
int btc_schedule_items(int N, int order, int chunks, int64_t *fac_rows, int *n_fac, int64_t *solve_rows,
                       int *n_solve, int *slot_rows, int *n_slots);

/*
 * Precision of the top-separator Cholesky of the mixed paths (the potrf of
 * Alg. 5's last iteration; the BTC_MIXED_* dtypes; other dtypes ignore
 * it). BTC_ROOT_FP64 (default): FP64 arithmetic; the pivots of this step
 * decide the factorization's stability. BTC_ROOT_DOUBLE_FP32 (option):
 * double-FP32 arithmetic (pairs of FP32, about 48 significant bits) on the
 * FP32 pipe, somewhat faster on this GPU, whose FP64 pipe issues two lanes per
 * clock per SM. Either way the Schur complement comes from the FP32 pool and
 * the factor is rounded back to it, so the two agree up to rounding ties of
 * that last step. Takes effect at the next factorization. Batched plans and
 * servers use the FP64 default.
 */
enum btc_root_precision { BTC_ROOT_DOUBLE_FP32 = 0, BTC_ROOT_FP64 = 1 };
int btc_plan_set_root_precision(btc_plan_t p, int precision);

/*
 * Device-side trace of the persistent launches (for profiling; off by
 * default). factor_trace / solve_trace: caller-owned device buffers of
 * 4 * (number of work items) uint64 each (factor items = N; solve items =
 * forward items of all levels + N backward items), or NULL to disable. Every
 * item records the global timer (ns) when it was claimed, when its inputs were
 * ready and when it finished, and the SM it ran on. Items that do not run
 * (the top-separator root of the mixed path, launched separately) stay untouched.
 */
int btc_plan_set_trace(btc_plan_t p, void *factor_trace, void *solve_trace);

/*
 * Per-node phase stamps of the factorization (the steps of one Alg. 5 node;
 * for profiling; off by default).
 * phase: caller-owned device buffer of 8 * N uint64, or NULL to disable. Each
 * node e (0-based) eliminated by the FP32 or FP64 node kernels (Alg. 5 and
 * Alg. 6 items; not the top separator of the mixed path, not the TF32
 * tensor-core kernels) writes the global timer (ns) at phase[8e + k] for
 * k = 0 entry, 1 operands and deferred updates in place, 2 Cholesky and both
 * triangular solves done, 3 factor blocks stored, 4 next diagonal block
 * updated, 5 end (fill block stored), and its SM id at phase[8e + 6]. Each
 * stamp adds one CTA barrier; the results are unchanged.
 */
int btc_plan_set_phase_trace(btc_plan_t p, void *phase);

/*
 * Test hook for the failure detection of the persistent launches (no paper
 * counterpart; the bounded waits are this library's own). Makes factor item
 * `item` (0-based, in the order of btc_schedule: level by level) of the next
 * persistent factorizations, plain and interlaced, wait for a completion flag
 * that no item ever sets, and lowers the poll limit of every wait of the
 * plan's persistent launches to max_polls (>= 64; the default is 2^23 polls,
 * about a second). That wait runs out after max_polls polls: the CTA records
 * the timeout in the launch's status word and moves on, every later wait of
 * the launch gives up at once, the launch drains, and btc_info and the solve
 * calls report BTC_ERR_TIMEOUT (results are then undefined). No kernel traps
 * or faults; the CUDA context stays usable. item = -1 restores the planner's
 * dependencies and the default limit. On the mixed paths the top separator
 * (run by its own kernel, without waits) cannot be chosen. Synchronizes the
 * plan's stream. Errors: BTC_ERR_ARG.
 */
int btc_plan_inject_stall(btc_plan_t p, int item, int64_t max_polls);

/* Rebind the plan's work to another CUDA stream (NULL = legacy default
 * stream). Work already enqueued on the old stream is not waited for. */
int btc_plan_set_stream(btc_plan_t p, void *stream);

/* Copy the plan's static description into *info. */
int btc_plan_query(btc_plan_t p, btc_plan_info *info);

/*
 * Factor (Alg. 5). D: device pointer to N blocks [N][n][n]; only the lower
 * triangle of each D_i is read. B: device pointer to N-1 blocks [N-1][n][n],
 * B_i = Psi(i+1, i) (may be NULL when N = 1). Element type FP64 for BTC_F64
 * and BTC_MIXED_F32, FP32 for BTC_F32; both 16-byte aligned. D and B are not
 * modified. For BTC_MIXED_F32 and BTC_F64 the plan keeps the two pointers for
 * the FP64 residual of btc_solve_refined: the caller must keep D and B alive
 * and unchanged until the next btc_factor or btc_free.
 * Asynchronous: a non-positive pivot is reported by btc_info, and makes the
 * next btc_solve / btc_solve_refined return BTC_ERR_NOT_SPD.
 */
int btc_factor(btc_plan_t p, const void *D, const void *B);

/*
 * Solve Psi X = RHS in place with the current factor (Alg. 7), for nrhs
 * right-hand sides. rhs: device pointer, [N*n][nrhs] row-major, element type
 * of the factor inputs (FP64 for BTC_F64 / BTC_MIXED_F32, FP32 for BTC_F32);
 * overwritten by X. For BTC_MIXED_F32 this is ONE FP32 correction solve of an
 * FP64 vector (no refinement). Asynchronous. Errors: BTC_ERR_NOT_FACTORED,
 * BTC_ERR_ARG.
 */
int btc_solve(btc_plan_t p, void *rhs, int nrhs);

/*
 * Iterative refinement: x_0 = solve(b); repeat r = b - Psi x (FP64, using the
 * D and B of the last btc_factor), stop when ||r||_inf <= tol ||Psi||_inf
 * ||x||_inf (max over right-hand sides), else x += solve(r). b, x: device
 * pointers, FP64, [N*n][nrhs] row-major (plans of dtype BTC_F64 or
 * BTC_MIXED_F32 only). Synchronous (reads the norms once per iteration).
 * *iters (may be NULL): refinement steps taken (0 when the first solve
 * already meets tol); *relres (may be NULL): final relative residual.
 * Returns BTC_ERR_NOT_CONVERGED if maxit steps did not reach tol (x then
 * holds the last iterate) or a residual norm is NaN (a NaN in b; *relres is
 * then NaN), BTC_ERR_NOT_SPD if the factor failed.
 */
int btc_solve_refined(btc_plan_t p, const double *b, double *x, int nrhs, double tol, int maxit, int *iters,
                      double *relres);

/*
 * Autotuning of the persistent factorization (on by default). The library
 * compiles the persistent factor kernels for several register budgets (one per
 * cap of 1-4 resident CTAs per SM; 1, 2, 4, 8, 16 for 64-thread CTAs). On the first
 * persistent factorization of a plan shape (dtype, padded n, N, variant) it
 * times every compiled cap at every CTAs-per-SM count that fits, three runs
 * each on the caller's D and B, keeps the fastest median and remembers it for
 * the process; the factor itself is the same in every configuration (only the
 * schedule changes). The interlaced factor + forward launch (btc_factor_solve
 * and the refined calls) is tuned the same way on its own, on the first
 * interlaced call of a plan shape: its kernel has other register and shared
 * memory needs, and its best residency differs; the packed right-hand side is
 * saved and restored around its trial runs. enable = 0: no tuning, the default
 * configuration for both launches. enable = 2: a configuration remembered for
 * the shape earlier in the process is used, but no trial launches are run
 * (the default configuration otherwise; for latency-bound callers such as a
 * request server). btc_plan_tuning and
 * btc_plan_tuning_interlaced report the configuration in use for the plain and
 * the interlaced launch (host pointers, each may be NULL): the register-budget
 * cap, the CTAs per SM of the launch, and whether it was tuned.
 */
int btc_plan_set_autotune(btc_plan_t p, int enable);
int btc_plan_tuning(btc_plan_t p, int *resident_cap, int *ctas_per_sm, int *tuned);
int btc_plan_tuning_interlaced(btc_plan_t p, int *resident_cap, int *ctas_per_sm, int *tuned);

/*
 * Pin the persistent factorization's configuration (turns autotuning off):
 * the compiled register-budget cap and the CTAs per SM of the launch
 * (0: as many as fit); the interlaced launch takes the same cap and as many of
 * those CTAs per SM as fit for it. Errors: BTC_ERR_UNSUPPORTED when no variant has that
 * cap, BTC_ERR_ARG when the CTAs do not fit. btc_plan_flow_configs lists the
 * compiled caps and the CTAs per SM each allows (host arrays; on input *count
 * is their capacity, on output the number of variants).
 */
int btc_plan_set_flow_config(btc_plan_t p, int resident_cap, int ctas_per_sm);
int btc_plan_flow_configs(btc_plan_t p, int *caps, int *max_ctas, int *count);

/*
 * CUDA graphs for btc_factor_solve_refined (on by default). With the
 * interlaced form, one column pass and a settled persistent configuration,
 * the whole refined factor + solve is captured once as an executable graph
 * (pack, interlaced factorization + forward sweep, top-separator root, solve tail,
 * unpack, FP64 residual, stopping test, and a device-side while loop of
 * correction solves that runs until the stopping test says stop) and replayed
 * on later calls with the same pointers, sizes and configuration (re-captured
 * otherwise): one graph launch and one host synchronization per call. The
 * graph runs on a plan-owned stream ordered after the plan's stream. Results
 * are identical to the path without graphs. enable = 0: plain launches.
 */
int btc_plan_set_graphs(btc_plan_t p, int enable);

/*
 * Optional event timing of a plan's kernels, by class. While enabled, every
 * launch of the classes below is bracketed by CUDA events recorded on the
 * plan's stream (a few microseconds of host work per launch; leave disabled in
 * production). btc_plan_timing synchronizes the stream, returns per class the
 * summed device time in ms[c] and the launch count in launches[c] (host
 * arrays of BTC_TIMING_CLASSES entries) since the last call, and resets them.
 * Enabling or disabling discards what is pending. The autotuner's trial
 * launches are not recorded.
 */
enum btc_timing_class {
  BTC_TIME_FACTOR = 0,          /* persistent factorization launch (or its level launches)        */
  BTC_TIME_FACTOR_FORWARD = 1,  /* interlaced factorization + forward substitution launch         */
  BTC_TIME_ROOT = 2,            /* top-separator Cholesky of the mixed path (FP64 or double-FP32)  */
  BTC_TIME_SOLVE = 3,           /* full solve launch (forward + backward)                          */
  BTC_TIME_SOLVE_TAIL = 4,      /* solve tail after an interlaced factorization                    */
  BTC_TIME_RESIDUAL = 5,        /* FP64 residual and norms of the refinement                       */
  BTC_TIMING_CLASSES = 6
};
int btc_plan_set_timing(btc_plan_t p, int enable);
int btc_plan_timing(btc_plan_t p, double *ms, int *launches);

/*
 * Factorization with the forward substitution interlaced (the paper's fused
 * factor + forward variant, Sec. 5: the forward sweep of level l runs as soon
 * as the blocks it reads are factored), then the backward substitution:
 * RHS <- Psi^{-1} RHS. D, B as for btc_factor; rhs as for btc_solve, in
 * place. The factor stays valid for later btc_solve / btc_solve_refined
 * calls. The interlaced form applies with the hybrid variant, the persistent
 * schedule and nrhs <= the plan's columns per pass; otherwise this is
 * btc_factor followed by btc_solve (same results). Asynchronous. Errors as
 * for btc_factor and btc_solve.
 */
int btc_factor_solve(btc_plan_t p, const void *D, const void *B, void *rhs, int nrhs);

/*
 * btc_factor_solve followed by the FP64 refinement of btc_solve_refined: the
 * first solve is the interlaced one; b, x, tol, maxit, iters, relres and the
 * return codes as for btc_solve_refined (plans of dtype BTC_F64 or
 * BTC_MIXED_F32; nrhs up to the plan's columns per pass). Synchronous.
 */
int btc_factor_solve_refined(btc_plan_t p, const void *D, const void *B, const double *b, double *x, int nrhs,
                             double tol, int maxit, int *iters, double *relres);

/*
 * GMRES-based iterative refinement (GMRES-IR; Carson and Higham 2018) on the
 * current factorization (Alg. 5 as the preconditioner, applied by the solves
 * of Alg. 7; the paper names mixed precision as future work, Sec. 7), for one
 * right-hand side: x0 = M^{-1} b, then per
 * outer step r = b - Psi x in FP64 and, until ||r||_inf <= tol ||Psi||_inf
 * ||x||_inf, the correction equation Psi d = r solved by GMRES on
 * M^{-1} Psi d = M^{-1} r (M = the plan's FP32 or TF32 factor applied by the
 * solve kernels, Psi applied in FP64; at most `restart` Arnoldi steps, stopped
 * when the preconditioned residual falls by inner_tol), x += d. Its analysis
 * (Carson and Higham) covers factors too inaccurate for classical refinement
 * (condition number times the factor's relative error near or above 1); on
 * the ill-conditioned TF32 cases measured with this library both converge,
 * GMRES-IR in fewer outer steps and to a smaller residual. b, x: device
 * FP64 [N*n]; needs an FP64 or mixed plan, factored (D, B kept as for
 * btc_solve_refined). *outer: outer steps taken, *inner: Arnoldi steps in
 * all, *relres: final relative residual (each may be NULL). Synchronous.
 * Errors: BTC_ERR_ARG (restart outside 1..200, inner_tol outside (0, 1)),
 * BTC_ERR_NOT_FACTORED, BTC_ERR_NOT_SPD, BTC_ERR_NOT_CONVERGED (x holds the
 * last iterate).
 */
int btc_solve_gmres_ir(btc_plan_t p, const double *b, double *x, double tol, int max_outer, int restart,
                       double inner_tol, int *outer, int *inner, double *relres);

/*
 * End-to-end call on HOST buffers: brings D, B (element type as for
 * btc_factor) and b (FP64 for BTC_F64 / BTC_MIXED_F32, FP32 for BTC_F32)
 * into plan-owned device buffers, factors, solves (refined to tol for BTC_F64
 * and BTC_MIXED_F32; one solve for BTC_F32) and copies the solution to x.
 * b, x: [N*n][nrhs]. Synchronous. When D and B are page-locked host memory
 * (cudaHostAlloc, cudaHostRegister, a pinned tensor) and N >= 2 on the FP64
 * or FP32-factor mixed path (hybrid variant, persistent schedule, no tensor
 * cores), they are not copied up front: the level-1 eliminations read them
 * over the CPU-GPU link (of each D_i only its lower triangle) while the rest
 * of level 1 runs, and write the device copies the FP64 residuals use; the
 * factor and solution are the same as with device inputs. Otherwise (pageable
 * memory, other paths) D and B are copied first. D and B must stay unchanged
 * during the call.
 */
int btc_factor_solve_host(btc_plan_t p, const void *D, const void *B, const void *b, void *x, int nrhs, double tol,
                          int maxit, int *iters, double *relres);

/*
 * Synchronize the plan's stream and report the first failed pivot of the
 * last factorization: *block = 0-based node, *col = column within the block,
 * both -1 when the factorization succeeded. Returns BTC_OK, BTC_ERR_NOT_SPD,
 * or BTC_ERR_TIMEOUT when a bounded device-side wait of a persistent launch
 * gave up (results are then undefined).
 */
int btc_info(btc_plan_t p, int *block, int *col);

/*
 * Debug readback (synchronous). Dhat: host buffer [N][n][n] of the factor's
 * diagonal blocks L(i,i) by node. U: host buffer [offdiag_blocks][n][n] of
 * the off-diagonal factor blocks in level-major slot order, each stored as the
 * row block U(e, o) = L(o, e)^T of the node e eliminated at that level; its
 * partner o is returned in pairs[2*k] = e, pairs[2*k+1] = o (0-based nodes).
 * Element type: FP64 for BTC_F64, FP32 otherwise. Any pointer may be NULL.
 */
int btc_get_factor(btc_plan_t p, void *Dhat, void *U, int *pairs);

/*
 * ||b - Psi x||_inf, ||Psi||_inf and ||x||_inf (max over right-hand sides),
 * computed on the device in FP64 for FP64 device arrays D [N][n][n] (lower
 * triangles read), B [N-1][n][n], x and b [N*n][nrhs]; the three numbers are
 * written to out3 (host pointer) after a synchronization of `stream`. A NaN
 * anywhere in the inputs comes back as a NaN norm. Uses a small scratch
 * buffer allocated and freed inside the call.
 */
int btc_residual(int N, int n, int nrhs, const double *D, const double *B, const double *x, const double *b,
                 double *out3, void *stream);

/*
 * btc_residual without any device allocation (the paper has no counterpart;
 * this is a deployment convenience). Computes the same three numbers as
 * btc_residual, with the same FP64 arithmetic, into out3 (host pointer): each
 * call copies them to the host and synchronizes `stream` before it returns.
 * A NaN anywhere in b, x or the matrix comes back as a NaN norm.
 *
 * For callers that cannot allocate device memory: real-time control loops
 * that forbid allocation after start-up, processes whose memory is entirely
 * owned by another allocator (for example a framework's caching allocator)
 * where a stray cudaMalloc could fail or fragment, and code that is not allowed
 * to call the CUDA allocator at all. This entry point calls no cudaMalloc,
 * cudaMallocAsync, cudaFree or allocating library routine. Its scratch (one
 * partial triple per block row) lives in a fixed device array compiled into
 * libbtc.so, 3 * 65536 + 3 doubles (about 1.5 MiB), which every GPU that loads
 * the library keeps until the process exits. Hence:
 *  - N may not exceed 65536 block rows (BTC_ERR_ARG otherwise); n up to 96
 *    (BTC_ERR_UNSUPPORTED when the three staged blocks exceed shared memory);
 *  - all calls share that one array: calls that overlap on the GPU (on two
 *    streams, or from two host threads) race and may return wrong norms;
 *    serialize them;
 *  - the first call on each device does a one-time set-up: it looks up the
 *    array's device address (cudaGetSymbolAddress) with that device current.
 *    A caller that captures CUDA graphs on that device should make this first
 *    call before any stream capture begins.
 * D, B, x, b: device pointers as for btc_residual. Errors: BTC_ERR_ARG,
 * BTC_ERR_UNSUPPORTED, BTC_ERR_CUDA (message in btc_last_error()).
 */
int btc_residual_noalloc(int N, int n, int nrhs, const double *D, const double *B, const double *x, const double *b,
                         double *out3, void *stream);

/* Release every device resource of the plan (synchronizes its stream). */
int btc_free(btc_plan_t p);

/* ---------------------------------------------------------------- batches
 * Many independent systems of different (N_k, n_k) in one plan. Instances are
 * grouped by padded block size; each group runs one persistent launch for the
 * factor and one for each solve, whose work items are the (instance, node)
 * eliminations of Alg. 5 / the substitutions of Alg. 7 of all its instances,
 * in level order, each waiting only for the producer nodes of its own instance.
 * Pointer arrays are HOST arrays of `count` DEVICE pointers; one right-hand
 * side per instance; rhs/x of instance k have N_k * n_k entries.
 */
typedef struct btc_batch_s *btc_batch_t;

/* Plan a batch (host planning + device pools). N, n: host arrays of `count`
 * sizes. Errors: BTC_ERR_ARG, BTC_ERR_UNSUPPORTED, BTC_ERR_OOM, BTC_ERR_CUDA. */
int btc_batch_plan(btc_batch_t *out, int count, const int *N, const int *n, int dtype, void *stream);

/* btc_batch_plan with an elimination order per instance: chunks[k] = 0 for
 * the nested-dissection order P_inf (Sec. 4.3), c >= 1 for the partition
 * permutation with c chunks (Sec. 4.1, Alg. 4, Proposition 1 split; c = 1 is
 * the natural order of Alg. 1), as btc_plan_set_order; chunks NULL: all
 * nested dissection. A block-size group holding a partition-order instance
 * converts every instance's inputs in one batched packing pass before its
 * factor launch. Errors as btc_batch_plan; BTC_ERR_ARG when c chunks do not
 * fit in N_k. */
int btc_batch_plan_orders(btc_batch_t *out, int count, const int *N, const int *n, const int *chunks, int dtype,
                          void *stream);

/* The per-instance chunk counts a batch was planned with (0: nested
 * dissection); chunks: host array of `count` ints. */
int btc_batch_orders(btc_batch_t b, int *chunks);

/* Host-only method dispatch for a batch (the adaptive choice between
 * elimination orders that the paper leaves as future work, Sec. 4.3): writes
 * chunks[k] for btc_batch_plan_orders (0 = nested dissection). Model of a
 * block-size group's persistent launches, which claim items level by level
 * across the batch: each factor launch level lasts max(its slowest item, its
 * total item time over the group's share of two resident CTAs per SM) plus
 * the latency of one dependency hop (2 us), and so does each forward and
 * backward solve level (two solves per refined call);
 * an item's time follows a per-block-size node time measured on GB300. Per
 * group, the policy "systems with N <= t take the partition order with c
 * chunks, the rest nested dissection" with the smallest modelled makespan is
 * chosen over c in {1, 2, 3, 4, 6, ..., 64} and t over 16 quantiles of the
 * group's N (all nested dissection when nothing beats it). The groups run
 * concurrently, so only the group with the longest nested-dissection makespan
 * takes its policy; the others keep nested dissection. Uses the current
 * device's SM count when a device is present (152 otherwise). Errors:
 * BTC_ERR_ARG, BTC_ERR_UNSUPPORTED (a block size batches do not take). */
int btc_dispatch_orders(int count, const int *N, const int *n, int dtype, int *chunks);

/* Number of block-size groups, total Alg. 5 flops, device bytes of the batch. */
int btc_batch_query(btc_batch_t b, int *groups, double *factor_flops, int64_t *device_bytes);

/* Factor every instance (element types as btc_factor). Asynchronous. The D and
 * B arrays must stay alive and unchanged for btc_batch_solve_refined. */
int btc_batch_factor(btc_batch_t b, const void *const *D, const void *const *B);

/* One solve per instance: x_k = Psi_k^{-1} rhs_k (for BTC_MIXED_F32 one FP32
 * correction solve of FP64 vectors). Asynchronous. */
int btc_batch_solve(btc_batch_t b, const void *const *rhs, void *const *x);

/* Refined solve of every instance until max_k ||r_k||/(||Psi_k|| ||x_k||) <= tol
 * (FP64 residuals; plans of dtype BTC_F64 or BTC_MIXED_F32). Synchronous.
 * *iters: refinement steps; *max_relres: the largest final relative residual. */
int btc_batch_solve_refined(btc_batch_t b, const double *const *rhs, double *const *x, double tol, int maxit,
                            int *iters, double *max_relres);

/* Synchronize; report the first instance whose factorization met a pivot that
 * was not positive (*failed_instance = -1 if none). BTC_OK, BTC_ERR_NOT_SPD or
 * BTC_ERR_TIMEOUT. */
int btc_batch_info(btc_batch_t b, int *failed_instance, int *block, int *col);

/*
 * Factor every instance and solve with FP64 refinement in one call: the same
 * results as btc_batch_factor followed by btc_batch_solve_refined (arguments
 * and return codes as those two). Once the groups' launch configurations are
 * settled (tuned on the first call, or tuning off), the whole sequence runs as
 * one captured CUDA graph: every group's persistent factorization and top
 * separators, the first solve, the FP64 residuals with the matrix-norm bounds,
 * and a device-side while loop of correction solves and residuals that runs
 * until the worst instance meets tol (or maxit steps); one graph launch and
 * one host synchronization per call. The instances' pointers are read from
 * device arrays at run time, so the graph is captured once per (tol, maxit)
 * and replayed for new inputs. If capture is refused, plain launches are used.
 * Synchronous.
 */
int btc_batch_factor_solve_refined(btc_batch_t b, const void *const *D, const void *const *B, const double *const *rhs,
                                   double *const *x, double tol, int maxit, int *iters, double *max_relres);

/* Autotuning of the groups' persistent factor launches (on by default): on the
 * first factorization each group times every compiled register-budget variant
 * at 1, 2, 4, ... CTAs per SM up to what fits (the number of nodes one SM holds
 * at once), three runs each on the batch's own inputs, and keeps the fastest;
 * the factor is the same in every configuration. */
int btc_batch_set_autotune(btc_batch_t b, int enable);

/* CUDA graphs for btc_batch_factor_solve_refined (on by default). */
int btc_batch_set_graphs(btc_batch_t b, int enable);

/* Launch configuration of group `group` (groups in launch order, largest work
 * first): padded block size, register-budget cap, CTAs per SM, whether it was
 * tuned and the tuned launch's median time in ms (host pointers, may be NULL). */
int btc_batch_tuning(btc_batch_t b, int group, int *np, int *resident_cap, int *ctas_per_sm, int *tuned,
                     double *factor_ms);

/* Release the batch (synchronizes its stream). */
int btc_batch_free(btc_batch_t b);

/* Message of the last error on the calling thread ("" if none). */
const char *btc_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int btc_version(void);

/* ---------------------------------------------------------------- bordered systems
 * Arrow structures: the block-tridiagonal Psi bordered by m dense coupling
 * rows C and a dense block A,
 *     Psi_a = [[Psi, C^T], [C, A]],
 * which the permuted Cholesky view of Sec. 4.3 extends to by eliminating the
 * border after the whole nested-dissection tree (the paper names arrow
 * structures as a natural extension there, and as future work in its
 * conclusion). The border's Schur complement S = A - C Psi^{-1} C^T is formed
 * in FP64 from Z = Psi^{-1} C^T (the plan's FP64-refined solves) and factored
 * in FP64; solves combine Psi^{-1} (refined), S^{-1} and Z, with FP64 residuals
 * of the whole bordered system. Layouts: C [m][N*n] row-major (C[r][i*n + c]
 * couples border variable r with variable c of block i); A [m][m] (lower
 * triangle read); b, x [N*n + m] (the block-tridiagonal part first). Every
 * pointer is a device pointer; the caller keeps D, B, C and A alive and
 * unchanged from btc_arrow_factor until the last btc_arrow_solve.
 */
typedef struct btc_arrow_s *btc_arrow_t;

/* Plan a bordered system of N blocks of size n and border width m
 * (1 <= m <= 64). dtype: BTC_F64 or a BTC_MIXED_* dtype (the arithmetic of the
 * block-tridiagonal factor; the border is FP64). Errors: BTC_ERR_ARG,
 * BTC_ERR_UNSUPPORTED, BTC_ERR_OOM, BTC_ERR_CUDA. */
int btc_arrow_plan(btc_arrow_t *out, int N, int n, int m, int dtype, void *stream);

/* Factor: Psi (Alg. 5), Z = Psi^{-1} C^T by refined solves to tol (at most
 * maxit refinement steps each), S = A - C Z and its FP64 Cholesky factor, and
 * ||Psi_a||_inf. Synchronous. BTC_ERR_NOT_SPD when Psi or S is not positive
 * definite (for S the message names its column). */
int btc_arrow_factor(btc_arrow_t a, const double *D, const double *B, const double *C, const double *A, double tol,
                     int maxit);

/* Solve Psi_a x = b (one right-hand side) with FP64 refinement of the whole
 * bordered system until ||b - Psi_a x||_inf <= tol ||Psi_a||_inf ||x||_inf:
 * x = [z - Z x_A; x_A] with z = Psi^{-1} b_T and x_A = S^{-1} (b_A - C z).
 * *iters: correction passes taken; *relres: final relative residual (each may
 * be NULL). Synchronous. BTC_ERR_NOT_CONVERGED when maxit passes did not reach
 * tol (x holds the last iterate). */
int btc_arrow_solve(btc_arrow_t a, const double *b, double *x, double tol, int maxit, int *iters, double *relres);

/* Release the bordered plan (synchronizes its stream). */
int btc_arrow_free(btc_arrow_t a);

/* ---------------------------------------------------------------- block-banded systems
 * Psi with Nb block rows of size b and lower block bandwidth w >= 1:
 * Psi(i+k, i) = A_k[i] for k = 0..w, zero for k > w (w = 1 is the
 * block-tridiagonal case). The paper's conclusion names block-banded matrices
 * with larger bandwidth as the extension of its method. Grouping w
 * consecutive block rows into one super-row gives a block-tridiagonal matrix
 * of N = ceil(Nb / w) blocks of size n = w b,
 *     D'_I(p, q) = Psi(Iw + p, Iw + q),   B'_I(p, q) = Psi((I+1)w + p, Iw + q),
 * equal to Psi, so the multi-stage permutation of Sec. 4.3 (whose separators
 * are then w consecutive block rows) and every path of the plan apply to it
 * unchanged; a ragged last super-row is padded with identity blocks. n = w b
 * must be a block size the dtype supports (btc_describe).
 * Layouts: A [w+1][Nb][b][b] row-major FP64, A[k][i] = Psi(i+k, i) (blocks
 * with i + k >= Nb are not read; of A_0 only the lower triangles are read);
 * rhs, x [Nb*b][nrhs] row-major FP64. Every pointer is a device pointer; the
 * grouped blocks are plan-owned copies, so A may change after a factor.
 */
typedef struct btc_banded_s *btc_banded_t;

/* Plan a banded system; dtype BTC_F64 or a BTC_MIXED_* dtype (FP64 inputs).
 * Errors: BTC_ERR_ARG, BTC_ERR_UNSUPPORTED (w b above the dtype's largest
 * block), BTC_ERR_OOM, BTC_ERR_CUDA. */
int btc_banded_plan(btc_banded_t *out, int Nb, int b, int w, int dtype, void *stream);

/* The inner block-tridiagonal plan (N super-rows of size w b), for its
 * settings (order, schedule, autotuning, timing) and inspection; owned by the
 * banded plan. NULL for a NULL handle. */
btc_plan_t btc_banded_inner(btc_banded_t a);

/* Copy the grouped blocks of the last factor call, D' [N][n][n] and
 * B' [N-1][n][n], into caller memory (host or device), and report N, n (each
 * output may be NULL). Synchronous. */
int btc_banded_grouped(btc_banded_t a, double *D, double *B, int *N, int *n);

/* Group the band on the device and factor it (Alg. 5). Synchronous.
 * BTC_ERR_NOT_SPD names the failing block row (of Psi) and column. */
int btc_banded_factor(btc_banded_t a, const double *A);

/* FP64-refined solve with the last factor (btc_solve_refined on the grouped
 * system: tol, maxit, *iters, *relres as there, the relative residual of the
 * grouped system). Synchronous. */
int btc_banded_solve_refined(btc_banded_t a, const double *rhs, double *x, int nrhs, double tol, int maxit,
                             int *iters, double *relres);

/* Group, factor and solve with FP64 refinement in one call
 * (btc_factor_solve_refined on the grouped system). Synchronous. */
int btc_banded_factor_solve_refined(btc_banded_t a, const double *A, const double *rhs, double *x, int nrhs,
                                    double tol, int maxit, int *iters, double *relres);

/* Release the banded plan and its inner plan (synchronizes its stream). */
int btc_banded_free(btc_banded_t a);

/* ---------------------------------------------------------------- serving
 * A continuous-batching request server (no paper counterpart beyond the
 * real-time setting of Sec. 1). Requests enter a FIFO queue; `slots` worker
 * threads, each with its own CUDA stream, take the oldest request that is
 * admissible (a slot is free and its HBM footprint fits the budget together
 * with the work in flight and the cached factors; least-recently-used cached
 * factors are evicted to make room), so requests arriving while others run
 * are admitted as slots and memory free up and their kernels overlap. Each
 * request is factor + refined solve (one RHS) or, with factor_id >= 0, a
 * refined re-solve with the cached factor of an earlier request. Re-solves of
 * one cached factor run one at a time (they share that factor's plan and its
 * work vectors); requests queued behind such a re-solve may start before it.
 * Plans are made per block size and bucket of N (sizes growing by 2^(1/4));
 * a request is copied into its plan's staging buffers and padded to the
 * bucket size with identity diagonal blocks, zero coupling blocks and a zero
 * right-hand side, which leaves its solution and residual unchanged (the
 * stopping test's matrix norm is max(||Psi||_inf, 1)). Plans made on the
 * request path run no tuning trials (btc_plan_set_autotune mode 2);
 * btc_server_prewarm builds and tunes them ahead of the traffic.
 */
typedef struct btc_server_s *btc_server_t;

typedef struct btc_request {
  int N, n;           /* system size                                                           */
  const double *D;    /* device FP64 [N][n][n] (lower triangles), alive until completion, and
                         for a factor that may be cached, until the server stops                */
  const double *B;    /* device FP64 [N-1][n][n]                                                */
  const double *b;    /* device FP64 [N*n] right-hand side                                      */
  double *x;          /* device FP64 [N*n] solution (written)                                   */
  int64_t factor_id;  /* -1: new factor (cached under this request's ticket when caching is on);
                         >= 0: ticket of an earlier factor request whose factor is reused (the
                         request is factored anew if that factor is no longer cached)            */
  double tol;         /* relative residual target, e.g. 1e-10                                   */
  int maxit;          /* refinement step limit                                                  */
} btc_request;

typedef struct btc_server_stats_s {
  int64_t completed, failed, queued, evictions, cache_hits, cache_misses;
  double p50_us, p99_us, mean_us; /* latency = completion - submission                         */
  double solves_per_s;            /* completed / (last completion - first submission)          */
  int64_t device_bytes;           /* plans in flight, cached and idle                          */
  double p50_queue_us, p99_queue_us;     /* submission -> a slot takes the request              */
  double p50_service_us, p99_service_us; /* a slot takes the request -> completion              */
} btc_server_stats_t;

/* Start a server. dtype: BTC_F64 or a BTC_MIXED_* dtype. slots: 1..64 concurrent
 * requests. hbm_budget_bytes: device memory the server may hold in plans.
 * cache_factors: keep factors for re-solve requests. */
int btc_server_start(btc_server_t *out, int dtype, int slots, int64_t hbm_budget_bytes, int cache_factors);

/* Enqueue a request (returns at once); *ticket identifies it. Errors:
 * BTC_ERR_ARG, BTC_ERR_UNSUPPORTED, BTC_ERR_OOM (larger than the budget). */
int btc_server_submit(btc_server_t s, const btc_request *req, int64_t *ticket);

/* Result of a request: returns 1 while it is queued or running (wait = 0),
 * BTC_OK once done (wait = 1 blocks until then); *status is the request's own
 * status (BTC_OK, BTC_ERR_NOT_SPD, BTC_ERR_NOT_CONVERGED, ...). */
int btc_server_poll(btc_server_t s, int64_t ticket, int wait, int *status, int *iters, double *relres,
                    double *latency_us);

int btc_server_stats(btc_server_t s, btc_server_stats_t *st);

/* Restart the statistics of btc_server_stats (counters, latencies, the throughput window); requests in
 * flight are counted when they complete. */
int btc_server_reset_stats(btc_server_t s);

/*
 * Device bytes that a request of size (N, n) reserves in a server of this
 * dtype: the plan of its size bucket (plans serve every N up to a bucket size,
 * buckets growing by 2^(1/4)) and that plan's staging copy of the padded
 * system. Host-only. Errors: BTC_ERR_ARG, BTC_ERR_UNSUPPORTED.
 */
int btc_server_footprint(int dtype, int N, int n, int64_t *bytes);

/*
 * Build, tune and capture ahead of the traffic `copies` plans of every size
 * bucket up to N_max for block size n, so that requests never pay plan
 * construction, tuning or graph capture: each plan factors and solves a
 * placeholder system (identity blocks) three times and is kept idle for
 * requests of its bucket. A factor request takes an idle plan of its bucket,
 * else the plan of the bucket's least recently used cached factor (that
 * factor is dropped; a later re-solve of it factors anew), and builds a plan
 * only when the bucket has neither, so `copies` bounds how many factors of one
 * bucket stay cached. Stops early (BTC_OK) when the HBM budget is full.
 * Synchronous. Errors: BTC_ERR_ARG, BTC_ERR_UNSUPPORTED, BTC_ERR_OOM,
 * BTC_ERR_CUDA.
 */
int btc_server_prewarm(btc_server_t s, int n, int N_max, int copies);

/* Finish every queued request, release all plans and streams. */
int btc_server_stop(btc_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* BTC_H */
