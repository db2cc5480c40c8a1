/*
 * hq.h -- C ABI of the GB300 stationary solver for the spatial hypercube queue
 * with heterogeneous service rates (Hua, Luo, Swersey & Wen, arXiv 2603.03019).
 *
 * Model (Section 2.1): N units, J demand nodes.  Calls from node j arrive as a
 * Poisson stream of rate lambda_j (= lambda f_j) and go to the first idle unit on
 * node j's preference list zeta_j; unit i serves at exponential rate nu_i.  A call
 * that finds every unit busy is lost (HQ_LOSS), waits in a buffer of C places
 * (HQ_FINITE, Proposition 2) or waits in an unbounded queue (HQ_INFINITE, the
 * Remark after Proposition 2).  A state B is an N-bit mask, bit i = unit i busy
 * ("y-order", Section 4.2: y(B) = sum_i b_i 2^(i-1) with 1-based units).
 *
 * Method: the conditional-probability reformulation (Proposition 1, Eq. 8-10) solved
 * by the layer-by-layer iteration of Algorithm 1 (Eq. 12-14), with the upward
 * rates of Eq. (3) built once per instance into a device-resident table.
 *
 * Conventions for every call:
 *   - Return value: HQ_OK (0) or a negative hq_status.  No call throws, aborts or
 *     exits.  hq_strerror() gives a static message; hq_last_error() gives the
 *     last failing call's detail on this thread.
 *   - Memory: arguments named *_mem say where the matching pointer lives:
 *     HQ_HOST (ordinary or pinned host memory) or HQ_DEVICE (memory of the device
 *     that was current when the solver was created).  The caller owns every
 *     buffer it passes; the library copies inputs in and results out and keeps
 *     no caller pointer after a call returns.
 *   - The solver owns all device memory it allocates (hq_create) and frees it in
 *     hq_destroy.  Calls on one handle must not overlap (thread-compatible, not
 *     thread-safe); separate handles are independent.
 *   - Every call returns after its device work has finished on the solver's
 *     stream (the stream given to hq_create).
 */
#ifndef HQ_H_
#define HQ_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HQ_OK = 0,
  HQ_EINVAL = -1,          /* bad argument or instance (see hq_last_error) */
  HQ_ENOMEM = -2,          /* device allocation failed */
  HQ_EUNSTABLE = -3,       /* infinite queue with lambda >= sum nu (Remark) */
  HQ_ENOTCONVERGED = -4,   /* max_sweeps reached; results are readable */
  HQ_EDIVERGED = -5,       /* non-finite or growing iterate; results are not valid */
  HQ_ETIMEOUT = -6,        /* a bounded device-side wait gave up */
  HQ_ECUDA = -7,           /* a CUDA runtime call failed */
  HQ_ESTATE = -8           /* call out of order (e.g. results before a solve) */
} hq_status;

typedef enum { HQ_LOSS = 0, HQ_FINITE = 1, HQ_INFINITE = 2 } hq_mode;
typedef enum { HQ_HOST = 0, HQ_DEVICE = 1 } hq_mem;

/* Arithmetic of the sweeps.  Layer totals lambda(n), mu(n), the within-layer
 * solve, the birth-death step and the residual are FP64 in every mode. */
typedef enum {
  HQ_PREC_FP64 = 0,      /* IEEE double sweeps */
  HQ_PREC_DF64 = 1,      /* double-float sweeps: values as (hi, lo) float pairs,
                            48-bit significand, FP32 ALU */
  HQ_PREC_FP32 = 2,      /* FP32 sweeps only (accuracy ~1e-6 relative) */
  HQ_PREC_FP32_DF64 = 3, /* FP32 sweeps until they stall, then DF64 sweeps */
  HQ_PREC_FP32_FP64 = 4, /* FP32 sweeps until they stall, then FP64 sweeps */
  HQ_PREC_FP32_IR = 5    /* FP32 sweeps until they stall, then iterative refinement:
                            FP32 sweeps of the correction e = p - p0 against an FP64
                            base p0 (one FP64 pass over p0 per base; the base absorbs
                            e and restarts when the correction's steps stall, at most
                            3 times); the correction's FP32 rounding is relative to
                            |e|, so the result is FP64-accurate */
} hq_precision;

typedef enum {
  HQ_TOL_STEP = 0,     /* max_{n,m} |p_n^k(B_m) - p_n^{k-1}(B_m)| <= tol (Algorithm 1's epsilon) */
  HQ_TOL_RESIDUAL = 1  /* max_m |out_m - in_m| / max_m out_m of Eq. (1) <= tol, FP64 */
} hq_tol_kind;

typedef enum { HQ_WARM_NONE = 0, HQ_WARM_GIVEN = 1, HQ_WARM_MLP = 2, HQ_WARM_PRODUCT = 3 } hq_warm;

typedef enum { HQ_ORDER_ASCENDING = 0, HQ_ORDER_REDBLACK = 1 } hq_order;

typedef struct hq_opts {
  double tol;          /* stopping tolerance (see tol_kind) */
  int tol_kind;        /* hq_tol_kind */
  int max_sweeps;      /* cap on outer iterations k (all precisions together) */
  int precision;       /* hq_precision */
  int check_every;     /* sweeps between host-side convergence checks (>= 1) */
  int warm_start;      /* hq_warm */
  int warm_mem;        /* hq_mem of warm_p */
  const double* warm_p;/* HQ_WARM_GIVEN: start vector p_n(B) in y-order, length 2^N */
  double fp32_stall;   /* mixed modes: leave FP32 when the step's decay per check is
                          worse than this ratio at two checks in a row, or at one once
                          the step is below 1e-6 (0 = default: 0.75 for HQ_PREC_FP32_IR,
                          whose correction sweeps cost about an FP32 sweep, 0.9 for
                          DF64 / FP64 refinement); HQ_PREC_FP32_IR
                          also re-bases when four checks in a row decay worse than it,
                          or one does after the correction shrank by 1e4 */
  double omega;        /* over-relaxation of the outer iteration (not in the paper):
                          each finalised layer becomes p_old + omega (p_new - p_old);
                          0 or 1 = Algorithm 1 as printed; (1, 2) fixed; negative =
                          automatic (Young's optimal omega for the contraction rate
                          observed over the second check, at most 1.9, backed off
                          when the steps stop shrinking).  The fixed point
                          is the same for any omega. */
  int sweep_order;     /* HQ_ORDER_ASCENDING (0): Algorithm 1's order, layers 1..N-1 in
                          turn; HQ_ORDER_REDBLACK (1, not in the paper): all odd layers,
                          then all even layers, each from the other's latest values (the
                          same fixed point; two grid barriers per sweep instead of N-1) */
  int debug_barrier;   /* testing only, 0 = off: k > 0 makes CTA k-1 of the first sweep
                          launch skip its first grid-barrier arrival and every bounded
                          device wait of that launch give up after 2^20 polls, so the solve
                          (hq_solve or hq_batch_solve) returns HQ_ETIMEOUT without hanging;
                          the handle stays usable */
  int reserved[2];
} hq_opts;

typedef struct hq_stats {
  int sweeps_fp32;        /* sweeps done in FP32 */
  int sweeps_hi;          /* sweeps of the refinement phase (FP64, DF64 or FP32
                             correction sweeps), or all sweeps of FP64 / DF64 solves */
  int residual_checks;    /* FP64 residual evaluations */
  int converged;          /* 1 if the tolerance was met */
  double final_step;      /* last max |p^k - p^{k-1}| */
  double final_residual;  /* last evaluated residual, -1 if none */
  double ms_total;        /* wall time of hq_solve */
  double ms_table;        /* wall time of the table build in the last hq_load */
  double state_updates;   /* (2^N - 2) * total sweeps */
  int warm_used;          /* 1 if a warm start was kept, 0 if cold (or fell back) */
  int ir_bases;           /* HQ_PREC_FP32_IR: FP64 bases the refinement set up (0 otherwise) */
  double omega;           /* over-relaxation in use at the end of the solve */
  double ms_sweeps_fp32;  /* device time of the FP32 sweep launches (CUDA events on the
                             solver's stream around each launch; hq_solve only, 0 in
                             hq_batch_solve) */
  double ms_sweeps_hi;    /* the same for the refinement phase's sweep launches */
  int reserved[2];
} hq_stats;

typedef struct hq_solver hq_solver;

/* Fill opts with defaults (library configuration, no counterpart in the paper; the
 * paper leaves epsilon open): tol 1e-10 on the residual, FP32 then DF64 sweeps (valid
 * for single and batched solves; HQ_PREC_FP32_IR is faster for single solves), check
 * every 8 sweeps, max 100000 sweeps, omega 1 (Algorithm 1 unrelaxed), the uniform
 * start of Algorithm 1. */
void hq_default_opts(hq_opts* opts);

/* The model of Section 2.1 (N units with their own service rates, J demand nodes with
 * preference lists, first-idle dispatch) in the loss form, the finite-buffer form of
 * Section 2.2's finite-buffer reformulation or the infinite-queue form of its Remark.
 * Allocate a solver for N units (1..29), J nodes (>= 1) and a queue mode
 * (capacity_C >= 1 iff HQ_FINITE, ignored otherwise) on the current device.
 * stream: a cudaStream_t, or NULL for the default stream.  Allocates every device
 * buffer the solve needs: the upward-rate table in FP64, double-float and FP32 (state
 * records padded to a multiple of 4 rates: about 20 (N/2 + 1.5) 2^N bytes) and the
 * transform scratch (4 N 2^N bytes), plus about 124 bytes per state (masks, iterates and
 * r in three precisions, weights, the refinement's base and base terms, the outputs);
 * e.g. 8.2 GB at N=24, 146 GB at N=28.  At N = 29 the double-float table and iterates
 * and the batched kernel's lists are not allocated (the rest is about 215 GB):
 * HQ_PREC_DF64 and HQ_PREC_FP32_DF64 return HQ_EINVAL there, and hq_batch_create takes
 * N <= 28.  Builds
 * the N-dependent layout (layer-ranked state masks and rank tables).  Writes the
 * handle to *out. */
int hq_create(int N, int J, int mode, int capacity_C, void* stream, hq_solver** out);

/* Load an instance (Section 2.1) and build its upward-rate table (Eq. 3).
 *   lambda_j: J doubles, lambda_j >= 0, sum > 0 (the per-node rates lambda f_j)
 *   nu:       N doubles > 0 (service rates nu_i)
 *   pref:     J*N int32, row-major; row j = zeta_j as 0-based unit ids, each row
 *             a permutation of 0..N-1
 * All three live in memory `mem`.  Validates (HQ_EINVAL / HQ_EUNSTABLE), copies
 * the inputs to the device and builds the table by a subset-sum transform over
 * the preference prefixes.  Discards any previous solution. */
int hq_load(hq_solver* h, const double* lambda_j, const double* nu, const int32_t* pref,
            int mem);

/* Algorithm 1 to the tolerance in opts (NULL = defaults).  Returns HQ_OK,
 * HQ_ENOTCONVERGED (results readable), HQ_EDIVERGED or an error.  stats may be
 * NULL.  After it returns, the result getters below are valid. */
int hq_solve(hq_solver* h, const hq_opts* opts, hq_stats* stats);

/* P{B} = p(w(B)) p_{w(B)}(B) (Proposition 1) for all 2^N states, y-order. */
int hq_get_stationary(hq_solver* h, double* P, int mem);

/* p(n), the birth-death distribution of the number of calls in the system
 * (Eq. 10 / Proposition 2): N+1 values (loss, infinite) or N+C+1 (finite).  For
 * HQ_INFINITE, queue[0] receives sum_{c>=1} P~{c} if queue != NULL. */
int hq_get_layer_marginals(hq_solver* h, double* pn, double* queue_tail, int mem);

/* Conditional probabilities p_n(B) of Proposition 1 (the iterate of Algorithm 1; each
 * layer sums to 1, Lemma 1), y-order, 2^N values, host or device memory per mem. */
int hq_get_conditional(hq_solver* h, double* p, int mem);

/* rho_i: fraction of time unit i is busy (queued states count as busy), N values:
 * the unit utilisation of Section 5.5 (its Table of utilisation errors), the sum of
 * P{B} over the states with unit i busy plus the queue's mass.  The throughput
 * identity sum_i nu_i rho_i = carried load holds. */
int hq_get_utilisation(hq_solver* h, double* rho, int mem);

/* Response pattern: the Introduction names it among the measures the stationary
 * distribution yields but does not define it; this is the standard hypercube
 * definition (first-idle dispatch of Section 2.1 applied to P{B}).
 * R[j*N + i]: probability that a call from node j is served by unit i (J x N).
 * Calls that wait are served by the unit that frees first: unit i w.p.
 * nu_i / sum nu.  Rows sum to 1 - P(call lost). */
int hq_get_response_pattern(hq_solver* h, double* R, int mem);

/* Unit workload by node (named in the Introduction, not defined in the paper; the
 * standard hypercube split of rho_i over the nodes):
 * W[i*J + j] = lambda_j R_ji / nu_i: fraction of time unit i serves node j (N x J). */
int hq_get_workload(hq_solver* h, double* W, int mem);

/* Scalars derived from P (not in the paper except the residual, which measures Eq. (1)
 * of Section 2.1 on the returned P): out[0] throughput sum_i nu_i rho_i, out[1] P(call lost),
 * out[2] P(call waits), out[3] relative balance residual of the returned P,
 * out[4] mean number of busy units. 5 doubles, host memory. */
int hq_get_summary(hq_solver* h, double* out5);

/* Pull-form upward-rate table in layer-ranked order, for checking: for layer
 * n (1..N), state rank k (colex order inside the layer) and busy slot s (s-th
 * busy unit in increasing id order), entry toff(n) + s*C(N,n) + k holds
 * lambda_{l m} for l = B minus that unit (Eq. 3).  count = N 2^(N-1) doubles.
 * Also writes the layer-ranked state masks (2^N uint32) if masks != NULL. */
int hq_get_table(hq_solver* h, double* T, uint32_t* masks, int mem);

/* Sizes of the solver (library bookkeeping, not in the paper): out[0]=N, [1]=J,
 * [2]=mode, [3]=C, [4]=2^N, [5]=table entries (N 2^(N-1), the pull entries of Eq. 3),
 * [6]=device bytes allocated.  8 int64 slots, host memory. */
int hq_get_info(const hq_solver* h, int64_t* out8);

/* Timing of the hot path: run `sweeps` outer iterations (Algorithm 1) of the current
 * iterate in precision `precision` (HQ_PREC_FP64 / HQ_PREC_DF64 / HQ_PREC_FP32, or
 * HQ_PREC_FP32_IR for correction sweeps; the iterate is converted if needed, a
 * conversion to HQ_PREC_FP32_IR sets up a base) as one launch of the persistent sweep kernel,
 * with CUDA events on the solver's stream around it.  ms_out (host, 1 float)
 * receives the mean milliseconds per sweep.  The iterate advances by `sweeps`
 * iterations; call hq_solve again for results.  Needs a previous hq_solve. */
int hq_profile_sweep(hq_solver* h, int precision, int sweeps, float* ms_out);

/* Phase timing of the last launch of the sweep kernel (for profiling; not in the
 * paper): the kernel runs one phase per layer of Algorithm 1 per sweep plus a closing
 * phase, separated by grid barriers.  us_out (host, max_out doubles) receives the wall time of each phase in
 * microseconds, measured on the GPU's global timer; returns the number of phases
 * written (at most 64 are recorded), or a negative hq_status. */
int hq_profile_phases(hq_solver* h, double* us_out, int max_out);

/* Algorithmic HBM bytes of one outer iteration (Algorithm 1) in `precision`: per
 * state of layers 1..N-1, its n table entries, r_m, one read and one write of p
 * (neighbour layers are L2-resident and not counted): (n + 3) values per state;
 * HQ_PREC_FP32_IR: an FP32 correction sweep, which also reads three FP32 base terms
 * per state (12 bytes).  Not in the paper: a measurement aid.  Host double. */
double hq_sweep_bytes(const hq_solver* h, int precision);

/* Upward-rate table without any device allocation.  The paper has no
 * counterpart: this exists for callers that may not allocate device memory
 * themselves -- code whose every buffer must come from an external pool or a fixed
 * device-memory budget, or latency-sensitive loops where a cudaMalloc (which can
 * synchronise the whole device) is not acceptable.
 *   N: 1..16 units, J: 1..4096 nodes (larger sizes return HQ_EINVAL: the working
 *      memory is one fixed 4.25 MiB static device array in the library);
 *   lambda_j (J doubles), pref (J*N int32, rows permutations of 0..N-1): device memory;
 *   T: device memory for N*2^(N-1) doubles, written in the same pull-form layer-ranked
 *      layout as hq_get_table;
 *   stream: a cudaStream_t or NULL.
 * Calls no cudaMalloc/cudaFree.  The first call on each device looks up the static
 * array's device address (with that device current).  All calls share the array: calls that overlap on the GPU
 * race and must be ordered (same stream, or synchronise in between).  Returns after
 * the work has finished on `stream`; on HQ_EINVAL from a bad row the contents of T
 * are unspecified. */
int hq_dispatch_table_static(int N, int J, const double* lambda_j, const int32_t* pref,
                             double* T, void* stream);

/* ---- batched solves ----------------------------------------------------------------
 * Algorithm 1 (Sec. 3.2, Eq. 12-14) on many independent instances of uneven N at once.
 * The paper solves one instance at a time; the batch runs layer n of every instance in
 * the same phase of one persistent launch (a device-side grid barrier between phases),
 * so that small instances, whose per-layer work cannot fill the GPU, share it.
 *
 * hq_batch_create: solvers[0..count-1] are loaded solvers (hq_load succeeded, N >= 2)
 *   on the current device; they are borrowed (not owned) and must outlive the batch; a
 *   solver may be loaded with another instance (hq_load) between batched calls.
 *   stream: a cudaStream_t, or NULL for a stream of the batch's own.  Builds the
 *   combined work lists (host memory for the build, device memory for the lists).
 *   Errors: HQ_EINVAL (NULL, count < 1, N < 2, another device), HQ_ESTATE (a solver not
 *   loaded), HQ_ENOMEM.
 * hq_batch_tune: the autotuner.  Times each kernel variant (threads per CTA x CTAs per
 *   SM: 0 = 512 x 2, 1 = 1024 x 1, 2 = 512 x 1, 3 = 256 x up to 4) for `sweeps` sweeps of
 *   `precision` (HQ_PREC_FP64, _DF64 or _FP32) from a cold start and keeps the fastest
 *   for later solves; variant_out (may be NULL) receives it, ms_out (may be NULL, 4
 *   floats) the ms per sweep of each variant.
 *   Untuned precisions use variant 0.  Overwrites the solvers' iterates.
 * hq_batch_solve: solves every instance cold to opts->tol on Algorithm 1's step
 *   (opts->tol_kind must be HQ_TOL_STEP; warm starts and HQ_PREC_FP32_IR are not
 *   supported: HQ_EINVAL); precision,
 *   check_every, max_sweeps, fp32_stall and omega (per instance) as for hq_solve (a
 *   mixed precision leaves
 *   FP32 for every instance at once, when all have stalled).  Each check replays one
 *   captured CUDA graph: [reset step buffers, one cooperative launch of check_every
 *   sweeps, copy the steps to the host].  Then each solver is finalised as hq_solve does
 *   (its getters work, its FP64 residual is in stats[c].final_residual).  stats: NULL or
 *   count entries; ms_total: NULL or the wall time.  Returns HQ_ENOTCONVERGED if some
 *   instance missed the tolerance, HQ_EDIVERGED, HQ_ETIMEOUT (a bounded device wait gave
 *   up) or HQ_ECUDA.  Calls on one batch, or on its solvers, must not overlap.
 * hq_batch_set_variant: use kernel variant `variant` (0..3, as numbered for
 *   hq_batch_tune) for `precision` (HQ_PREC_FP64, _DF64 or _FP32) in later solves,
 *   instead of the tuned or default one.  Errors: HQ_EINVAL.
 * hq_batch_info: out8 = {count, largest N, states swept per sweep (sum of 2^N - 2), work
 *   items, graph state (1 replayed graph, -1 capture refused and direct launches, 0 not
 *   tried yet), variant in use for FP64, DF64, FP32}. */
typedef struct hq_batch hq_batch;
int hq_batch_create(hq_solver* const* solvers, int count, void* stream, hq_batch** out);
int hq_batch_tune(hq_batch* b, int precision, int sweeps, int* variant_out, float* ms_out);
int hq_batch_solve(hq_batch* b, const hq_opts* opts, hq_stats* stats, double* ms_total);
int hq_batch_set_variant(hq_batch* b, int precision, int variant);
int hq_batch_info(const hq_batch* b, int64_t* out8);
void hq_batch_destroy(hq_batch* b);

/* ---- learned warm start ---------------------------------------------------------------
 * Not in the paper (which starts Algorithm 1 from p_n = 1/C(N,n), Sec. 3.2).  A small
 * network predicts, for every layer n = 1..N-1 and unit i, the conditional occupancy
 * q_i(n) = P(unit i busy | n units busy) from 9 inputs (hq_mlp_features): the unit's
 * nu_i / mean nu, the demand shares of the nodes ranking it first, second and third,
 * lambda s1_i / nu_i, lambda / sum nu, log(nu_i / mean nu), N / 16, and n / N.  hq_solve
 * with warm_start = HQ_WARM_MLP then starts from the layer-wise product form
 * p_n(B) = prod_{i in B} x_i(n) / e_n(x(n)), x_i(n) = q_i(n) / (1 - q_i(n)), and keeps it
 * only if its FP64 relative balance residual of Eq. (1) is below the uniform start's
 * (two residual evaluations, no sweep; stats.warm_used says which was kept).
 * warm_start = HQ_WARM_PRODUCT is the analytic control, with no network: the same
 * product form and fallback with q_i(n) = rho0_i for every layer, rho0_i the unit's
 * first-choice utilisation lambda1_i / nu_i clipped to [0.02, 0.98], lambda1_i the
 * demand of the nodes that rank unit i first (so x_i = rho0_i / (1 - rho0_i)).
 *
 * Network, weights shared across units and layers: 9 -> hidden (ReLU) -> hidden (ReLU)
 * -> 1, the output estimating logit(q_i(n)); activations stored in BF16, the hidden x
 * hidden product on BF16 tensor cores with FP32 accumulation, master weights FP32.
 * Parameter order of the flat FP32 vector: W1 [9 x hidden] row-major, b1 [hidden],
 * W2 [hidden x hidden] row-major (input index first), b2 [hidden], W3 [hidden], b3 [1].
 *
 * hq_mlp_create: hidden a multiple of 16 in 16..4096; He-uniform weights from a
 *   splitmix64 stream seeded by `seed`, zero biases; stream as for hq_create.
 * hq_mlp_set_weights / _get_weights: n must equal hq_mlp_num_params; mem: HQ_HOST or
 *   HQ_DEVICE; setting resets the optimiser state.
 * hq_mlp_forward: X (B x 9 FP32, device), y (B FP32, device).
 * hq_mlp_gradients: loss = mean (y - target)^2 over the B rows and its gradient with
 *   respect to the flat parameters into grad (device, num_params FP32; may be NULL);
 *   loss (host float, may be NULL).  X and target: device memory.
 * hq_mlp_train_step: the same gradient, then one Adam step (beta 0.9 / 0.999, eps 1e-8)
 *   with learning rate lr > 0.
 * hq_mlp_features: the network inputs of a loaded solver (N >= 2), one row per (layer
 *   n = 1..N-1, unit i), row (n-1) N + i, N (N-1) x 9 FP32, host or device per mem.
 * hq_mlp_predict: for a loaded solver, q ((N+1) x N doubles, row n = q_(.)(n), rows 0 and
 *   N exact), the layer law P(n) of the loss system with lambda(n) = lambda and
 *   mu(n) = sum_i nu_i q_i(n) (Eq. 10; N+1 doubles, may be NULL) and
 *   rho_i = sum_n P(n) q_i(n) (N doubles, may be NULL), all in the memory given by mem.
 * hq_attach_mlp: borrow a model for HQ_WARM_MLP solves of this solver (NULL detaches).
 * Errors: HQ_EINVAL for NULL or inconsistent arguments, HQ_ESTATE if not loaded,
 * HQ_ENOMEM, HQ_ECUDA. */
typedef struct hq_mlp hq_mlp;
int hq_mlp_create(int hidden, uint64_t seed, void* stream, hq_mlp** out);
int64_t hq_mlp_num_params(const hq_mlp* m);
int hq_mlp_set_weights(hq_mlp* m, const float* w, int64_t n, int mem);
int hq_mlp_get_weights(hq_mlp* m, float* w, int64_t n, int mem);
int hq_mlp_forward(hq_mlp* m, const float* X, int B, float* y);
int hq_mlp_gradients(hq_mlp* m, const float* X, const float* target, int B, float* grad, float* loss);
int hq_mlp_train_step(hq_mlp* m, const float* X, const float* target, int B, float lr, float* loss);
int hq_mlp_features(hq_solver* h, float* X, int mem);
int hq_mlp_predict(hq_solver* h, hq_mlp* m, double* q, double* pn, double* rho, int mem);
int hq_attach_mlp(hq_solver* h, hq_mlp* m);
void hq_mlp_destroy(hq_mlp* m);

/* ---- discrete-event simulation of the loss system (Section 5.5) -----------------------
 * The paper checks its exponential-service solution against simulations of the loss
 * system with other service-time distributions of the same means (Section 5.5, its
 * Table of MRT and utilisation errors): for a system without a queue the stationary
 * solution is insensitive to the service distribution.  hq_des_simulate runs `reps`
 * independent replications of that system on the GPU, one thread each: Poisson
 * arrivals of rate sum_j lambda_j, node j with probability lambda_j / lambda, the first
 * idle unit of pref row j serves (Section 2.1), else the call is lost; unit i's service
 * times have mean 1/nu_i and shape service_kind: 0 exponential, 1 log-normal with the
 * exponential's variance, 2 gamma of shape 5 (scale 1/(5 nu_i)), 3 gamma of shape 1/2
 * (scale 2/nu_i), 4 uniform on [0, 2/nu_i].  Each replication starts empty; arrivals
 * 0..warmup-1 are not counted; the window runs from arrival `warmup` to the last of
 * `arrivals`.  Random numbers: a counter-based splitmix64 stream per replication (key
 * from `seed` and the replication index), 8 draws per arrival.
 *   N 1..32, J >= 1; lambda_j (J), nu (N), pref (J*N int32 rows, permutations of
 *   0..N-1), travel (J*N doubles, travel[j*N + i] = response time of unit i to node j):
 *   inputs.  Outputs: busy (reps*N: busy time of unit i in the window, exact overlap),
 *   served (reps*N int64: calls served in the window), lost (reps int64), window (reps:
 *   window length), resp (reps: summed travel time of the calls served in the window).
 *   mem: HQ_HOST or HQ_DEVICE for every array; stream as for hq_create.  Utilisation is
 *   busy / window, the mean response time resp / sum(served).  Blocks until done.
 *   The variates are formed in FP32, so the rates have a range: nu_i and the total rate
 *   sum_j lambda_j must lie in [2^-60, 2^60] (every service and inter-arrival time is
 *   then a finite FP32 number).
 *   Errors: HQ_EINVAL (sizes, kind, NULL, a bad pref row, negative or non-finite rates,
 *   rates out of that range), HQ_ECUDA. */
int hq_des_simulate(int N, int J, const double* lambda_j, const double* nu, const int32_t* pref,
                    const double* travel, int service_kind, int64_t reps, int64_t arrivals,
                    int64_t warmup, uint64_t seed, double* busy, int64_t* served, int64_t* lost,
                    double* window, double* resp, int mem, void* stream);

/* Release a solver and every device buffer it holds (the model of hq_create; not in
 * the paper).  NULL is ignored.  A model attached by hq_attach_mlp is not freed. */
void hq_destroy(hq_solver* h);
/* Library housekeeping, not in the paper: a static text for an hq_status code, and the
 * calling thread's message for its last failed call ("" if none). */
const char* hq_strerror(int code);
const char* hq_last_error(void);

/* Device kernel launches made by the calling thread since the last reset (for
 * accounting of the work the library does; not in the paper). */
int64_t hq_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* HQ_H_ */
