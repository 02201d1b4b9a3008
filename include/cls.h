/*
 * cls.h -- C ABI of the B300 (sm_103a) parallel Continuous Local Search
 * hot path: batched evaluation of a weighted sum of symmetric pseudo-Boolean
 * constraints' Walsh-Fourier expansions and their gradient, projected
 * gradient steps, rounding to +-1 and exact satisfaction counts.
 *
 * Paper: "A Study of Parallel Continuous Local Search" (arXiv 2606.06656).
 *   Sec. 2.1, Eq. 1  Walsh-Fourier expansion FE of a Boolean function on the
 *                    cube Q^n = [-1,1]^n, True -> -1, False -> +1.
 *   Sec. 2.1, Eq. 3  symmetric constraints: FE depends on the spectrum sp_t
 *                    (t = number of true literals).
 *   Sec. 2.2         constraint types AMO, EO, EK, NAE, XOR, CARD, OR.
 *   Sec. 2.3, Eq. 5  objective: min sum_c FE_c(X) over Q^n; satisfied iff
 *                    sum_c FE_c(sign X) = -m; projected gradient descent,
 *                    evaluated through a DFT.
 *   Sec. 3.3         many restarts iterate together in lockstep.
 *
 * Conventions shared by every call
 *   - Return value: CLS_OK (0) or a negative CLS_ERR_* code; no call throws
 *     or aborts.  cls_strerror() names a code; cls_last_error() returns the
 *     calling thread's last detailed message (e.g. the CUDA error string).
 *   - Assignments are FP32 arrays laid out variable-major, restart-minor:
 *     x[v * R + r] is variable v of restart r (R restarts, 0 <= r < R).
 *     Each variable row is therefore contiguous over restarts; this is the
 *     layout every kernel reads coalesced.
 *   - A literal with sign s on variable v has value y = s * x_v; it is true
 *     at a corner when y == -1.
 *   - "Device" pointers are CUDA global-memory pointers on the device the
 *     problem was created on (e.g. torch tensor data_ptr()).  They are owned
 *     by the caller; the library never frees them.  "Host" pointers are
 *     ordinary CPU memory, read only during the call.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Every device
 *     call only enqueues work on that stream and returns without
 *     synchronising; it performs no allocation and no host<->device copy
 *     except where stated (cls_problem_create, cls_solve_host), so it may be
 *     captured into a CUDA graph.
 *   - Scratch memory is supplied by the caller: ws must point to at least
 *     cls_workspace_size() bytes of device memory, 256-byte aligned.
 */
#ifndef CLS_B300_H
#define CLS_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define CLS_OK               0
#define CLS_ERR_INVALID     -1  /* bad argument or malformed constraint set  */
#define CLS_ERR_CUDA        -2  /* a CUDA runtime call or launch failed      */
#define CLS_ERR_NOMEM       -3  /* device or host allocation failed          */
#define CLS_ERR_UNSUPPORTED -4  /* no usable sm_103 device                   */
#define CLS_ERR_WORKSPACE   -5  /* workspace missing, too small or unaligned */

/* ---- constraint types (Sec. 2.2; Table 2 PB forms; t = # true literals) */
#define CLS_OR        0  /* t >= 1                        (disjunction)      */
#define CLS_XOR       1  /* t odd                                           */
#define CLS_CARD_GE   2  /* t >= k   (cardinality, at-least-k)               */
#define CLS_CARD_LE   3  /* t <= k   (at-most-k)                             */
#define CLS_NAE       4  /* 0 < t < L (not-all-equal)                        */
#define CLS_EO        5  /* t == 1   (exactly-one)                           */
#define CLS_EK        6  /* t == k   (exactly-k)                             */
#define CLS_AMO       7  /* t <= 1   (at-most-one)                           */
#define CLS_SPECTRUM  8  /* explicit spectrum sp_t, t = 0..L (Eq. 3)         */

#define CLS_MAX_LEN 1024 /* longest constraint accepted (literals)           */

typedef struct cls_problem cls_problem; /* opaque, owned by the library      */

/* Validate a constraint set without touching a GPU (Sec. 2.2 / 2.3).
 *   n_vars   number of variables n >= 0
 *   n_cons   number of constraints m >= 0
 *   offsets  host int32[m+1]: constraint c owns literals offsets[c] ..
 *            offsets[c+1]-1; offsets[0] == 0, non-decreasing,
 *            1 <= length <= CLS_MAX_LEN
 *   lit_var  host int32[nnz]: variable of each literal, 0 <= v < n, no
 *            variable twice in one constraint
 *   lit_sign host int8[nnz]: +1 (positive literal) or -1 (negated)
 *   type     host int32[m]: CLS_OR .. CLS_SPECTRUM
 *   k        host int32[m]: threshold, 0 <= k <= L, for CARD_GE, CARD_LE
 *            and EK; ignored for the other types (may be NULL if none of
 *            those types occurs)
 *   weight   host float[m], finite (NULL = all 1; the paper's sum is
 *            unweighted)
 *   spectra  host int8: for each CLS_SPECTRUM constraint in order, L+1
 *            entries in {-1,+1} (sp_t = -1 where the constraint holds); NULL
 *            if no such constraint
 *   fixed    host uint8[n] or NULL: 1 pins the variable (partial assignment,
 *            Sec. 3.2); pinned variables never move in a step
 *   fixed_val host float[n] or NULL: the pinned value (-1 or +1) of each
 *            pinned variable; required when fixed is given
 * Returns CLS_OK or CLS_ERR_INVALID.  Errors are reported for the first
 * offending item through cls_last_error(). */
int cls_problem_check(int32_t n_vars, int32_t n_cons, const int32_t* offsets,
                      const int32_t* lit_var, const int8_t* lit_sign,
                      const int32_t* type, const int32_t* k, const float* weight,
                      const int8_t* spectra, const uint8_t* fixed,
                      const float* fixed_val);

/* Build the device-resident problem on the current CUDA device: validate
 * (as cls_problem_check), compute every constraint's spectrum and its
 * Fourier tables in FP64 (Eq. 3, evaluated at the L+1 roots of unity,
 * Sec. 2.3), the variable-major transpose of the literal list, the kernel
 * work lists, and copy them to the device (synchronously).  The host arrays
 * are copied; the caller keeps ownership.  On success *out receives a handle
 * to free with cls_problem_destroy.  Errors: CLS_ERR_INVALID,
 * CLS_ERR_UNSUPPORTED (no sm_103 device), CLS_ERR_NOMEM, CLS_ERR_CUDA; *out
 * is left NULL on error. */
int cls_problem_create(int32_t n_vars, int32_t n_cons, const int32_t* offsets,
                       const int32_t* lit_var, const int8_t* lit_sign,
                       const int32_t* type, const int32_t* k, const float* weight,
                       const int8_t* spectra, const uint8_t* fixed,
                       const float* fixed_val, cls_problem** out);

/* As cls_problem_create, with flags:
 *   CLS_SIMPLIFY_FIXED  fold pinned variables into the spectra (Sec. 3.2's
 *     partial assignment): a pinned literal's factor is exactly 1 (false) or
 *     w^j (true), so a constraint with f pinned-true literals and L' free ones
 *     has the expansion of the spectrum sp'_t = sp_{t+f}, t = 0..L', over its
 *     free literals -- the same FE for every assignment of the free
 *     variables.  Pinned literals are then skipped by the FE+gradient
 *     kernels (pinned variables get a zero gradient; they never move), while
 *     scoring still counts every literal.  Ignored when fixed is NULL. */
#define CLS_SIMPLIFY_FIXED 1u
int cls_problem_create_ex(int32_t n_vars, int32_t n_cons, const int32_t* offsets,
                          const int32_t* lit_var, const int8_t* lit_sign,
                          const int32_t* type, const int32_t* k, const float* weight,
                          const int8_t* spectra, const uint8_t* fixed,
                          const float* fixed_val, uint32_t flags, cls_problem** out);

/* Free a problem (NULL is accepted).  Synchronises the device first. */
int cls_problem_destroy(cls_problem* p);

/* Problem facts for callers: sizes and the per-path constraint counts.
 *   info[0] n, info[1] m, info[2] nnz, info[3] # constraints whose spectrum
 *   is a closed-form product of real roots (OR, XOR, NAE and their
 *   complements, Appendix A) with L <= 16 (one thread per (constraint,
 *   restart)), info[4] # such constraints with L > 16, info[5] # on the
 *   DFT path (every other spectrum), info[6] number of DFT roots summed
 *   over DFT constraints, info[7] sum over DFT constraints of L * roots,
 *   info[8] literals entering FE (nnz minus folded pinned literals),
 *   info[9] constraints whose expansion is constant.  info must hold 10
 *   int64. */
int cls_problem_info(const cls_problem* p, int64_t* info);

/* Bytes of device workspace the compute calls need for R restarts. */
int cls_workspace_size(const cls_problem* p, int32_t R, size_t* bytes);

/* x[v*R + r] ~ U[-1, 1) for r = 0..R-1 from Philox4x64-10 (Salmon et al.,
 * SC'11) with key (seed, 0) and counter (r + r_offset, v / 4, 0, 0), output
 * word v % 4, x = (word >> 40) * 2^-23 - 1; pinned variables get their
 * fixed value.  r_offset lets a shard of restarts reproduce the same points
 * as one run over all restarts.  x: device float[n*R]. */
int cls_init_uniform(const cls_problem* p, int32_t R, uint64_t seed,
                     int64_t r_offset, float* x, void* stream);

/* Per-restart convergence tracking and refills (Sec. 3.3: in a lockstep
 * batch, restarts that have converged idle and waste the batch's compute;
 * the section studies the distribution of steps to convergence).  The state
 * is a caller-owned device int32[4*R]: trk[r] = best satisfied count so far,
 * trk[R+r] = the step it was reached, trk[2R+r] = steps since the last
 * improvement, trk[3R+r] = first step at which every constraint was
 * satisfied (-1 = none yet).
 *   cls_track_reset      best = -1, its step = -1, since = 0, solved = -1.
 *   cls_track_step       with this step's nsat (cls_step / cls_round_score):
 *                        nsat > best: best = nsat, its step = step, since = 0;
 *                        otherwise since += 1; nsat == m and solved < 0:
 *                        solved = step.  step >= 0.
 *   cls_refill           every restart with solved < 0 and since >= patience
 *                        (>= 1) gets fresh points: the cls_init_uniform draw
 *                        with the Philox counter's third word = generation
 *                        (>= 1; the first draw is generation 0), pinned
 *                        variables untouched; its best, best step and since
 *                        restart (-1, -1, 0); *count (device int32) is
 *                        increased by the number refilled.
 *   cls_unsat_histogram  hist[k] = number of restarts with exactly k
 *                        unsatisfied constraints, k = 0..m (device
 *                        int32[m+1], overwritten).
 * All asynchronous on stream; integer results are exact.  CLS_ERR_INVALID
 * on NULL pointers (R > 0) or out-of-range patience / generation / step. */
int cls_track_reset(const cls_problem* p, int32_t R, int32_t* trk, void* stream);
int cls_track_step(const cls_problem* p, int32_t R, const int32_t* nsat, int32_t step,
                   int32_t* trk, void* stream);
int cls_refill(const cls_problem* p, int32_t R, float* x, int32_t* trk, int32_t patience,
               uint64_t seed, int64_t r_offset, int32_t generation, int32_t* count,
               void* stream);
int cls_unsat_histogram(const cls_problem* p, int32_t R, const int32_t* nsat, int32_t* hist,
                        void* stream);

/* Convergence of projected gradient descent per restart (Sec. 3.3 studies
 * the number of steps restarts take to converge; Sec. 3.1 notes that a
 * small step can meet a convergence criterion on a plateau):
 *   cls_movement         maxdelta[r] = max over variables v of
 *                        |x[v*R + r] - x_prev[v*R + r]| (device float[R],
 *                        overwritten; FP32 subtraction, exact maximum, so
 *                        bit-reproducible); x_prev is the caller's copy of
 *                        x from before the step.
 *   cls_track_converged  conv[r] (device int32[R], -1 = not yet, set by the
 *                        caller) becomes `step` the first time
 *                        maxdelta[r] <= tol.
 * Asynchronous on stream.  CLS_ERR_INVALID on NULL pointers (R > 0),
 * step < 0 or tol < 0 / NaN. */
int cls_movement(const cls_problem* p, int32_t R, const float* x_prev, const float* x,
                 float* maxdelta, void* stream);
int cls_track_converged(const cls_problem* p, int32_t R, const float* maxdelta, float tol,
                        int32_t step, int32_t* conv, void* stream);

/* Adaptive constraint weighting (Sec. 3.1 proposes weights informed by the
 * constraints' gradient magnitudes, after observing that a doubled edge
 * gradient overwhelms the balancing constraints; the paper gives no rule,
 * so the rule below is this library's).  Weights are per constraint, shared
 * by all restarts; they enter the objective, the gradient and wsat as the
 * weights given at creation do.
 *   cls_constraint_stats  per constraint c over the R restarts:
 *       gnorm[c] = sum_r || dFE_c/dy (x_r) ||_2 over the literals entering
 *                  FE (all literals; the free ones with CLS_SIMPLIFY_FIXED),
 *                  from the literal partials that the last cls_eval or
 *                  cls_step with this workspace and R left in it, divided
 *                  by |w_c| (0 where w_c = 0 or FE_c is constant);
 *       unsat[c] = number of restarts whose rounded point (bits, the
 *                  bitset format of cls_round_score) violates c.
 *     gnorm device double[m], unsat device int32[m], overwritten.  Each
 *     restart's norm is computed in FP32 from the FP32 partials; the 32
 *     norms of a restart tile are added in FP32, the tiles in FP64, both in
 *     a fixed order (deterministic).  unsat is exact.  The partials are
 *     only read; the workspace's objective scratch holds per-tile sums.
 *   cls_reweight  from those statistics, with u_c = unsat[c]/R,
 *     g_c = gnorm[c]/R and gbar the mean of g_c over the constraints with
 *     FE work:
 *       rho_c = kappa            if g_c * kappa <= gbar   (weak or no pull)
 *             = gbar / g_c       otherwise
 *       w_c  <- min(w_max, w_c (1 + eta u_c rho_c))      (FP64, stored FP32)
 *     so constraints violated in many restarts gain weight, the more the
 *     weaker their gradient.  The new weights go to w_out (device
 *     float[m]) and into the problem.  Needs 0 <= eta, 0 < kappa,
 *     0 < w_max, all finite.
 *   cls_set_weights  w (device float[m], finite; not checked) become
 *     the weights.
 * Both weight calls are asynchronous on stream and change the problem:
 * calls on one problem must be ordered (one stream).  A graph created while
 * every weight was 1 recorded the unweighted score kernel: once weights
 * change, cls_graph_launch refuses it (CLS_ERR_INVALID) and it must be
 * created again.  cls_tuning_set / cls_autotune first synchronise the
 * device and read the current weights back into the host plan.  Errors:
 * CLS_ERR_INVALID on NULL pointers, R < 1 or out-of-range parameters;
 * CLS_ERR_WORKSPACE as cls_eval. */
int cls_constraint_stats(const cls_problem* p, int32_t R, const uint32_t* bits, void* ws,
                         size_t ws_bytes, double* gnorm, int32_t* unsat, void* stream);
int cls_reweight(cls_problem* p, int32_t R, const double* gnorm, const int32_t* unsat, double eta,
                 double kappa, double w_max, float* w_out, void* stream);
int cls_set_weights(cls_problem* p, const float* w, void* stream);

/* Objective and gradient at x (Sec. 2.3, Eq. 5 with weights):
 *   obj[r]        = sum_c w_c FE_c(s_c o x_r)            (device float[R] or NULL)
 *   grad[v*R+r]   = dF/dx_v at restart r                 (device float[n*R] or NULL)
 *   fe_con[c*R+r] = FE_c at restart r, unweighted        (device float[m*R] or NULL)
 * FE_c and its literal partials come from the DFT of the constraint's
 * spectrum (Sec. 2.3; Eq. 3 basis), computed in FP32; partials are summed
 * per variable in a fixed order (deterministic).  x: device float[n*R]. */
int cls_eval(const cls_problem* p, int32_t R, const float* x, float* obj,
             float* grad, float* fe_con, void* ws, size_t ws_bytes, void* stream);

/* Vector-Jacobian product of the per-restart objective for reverse-mode
 * differentiation (the adjoint of cls_eval's obj output):
 * out[v*R + r] = scale[r] * g[v*R + r], where g is cls_eval's gradient and
 * scale[r] = dLoss/dobj[r].  g, out: device float[n*R] (may alias);
 * scale: device float[R]. */
int cls_restart_scale(const cls_problem* p, int32_t R, const float* g, const float* scale,
                      float* out, void* stream);

/* Projected gradient step (Sec. 2.3, PGD on Q^n) with a given gradient:
 * x <- min(max(fl(x - fl(lr * grad)), -1), 1) for free variables (pinned
 * ones are left as they are), then, if bits is not NULL, writes the rounded
 * assignment (see cls_round_score).  x: device float[n*R] updated in place;
 * grad: device float[n*R]; bits: device uint32[n*ceil(R/32)] or NULL. */
int cls_pgd_update(const cls_problem* p, int32_t R, float* x, const float* grad,
                   float lr, uint32_t* bits, void* stream);

/* Round and score (Sec. 2.3): variable v of restart r is True iff
 * x[v*R+r] < 0 (so +0, -0 and NaN are False).  bits[v*RW + r/32] bit r%32
 * holds that truth value (RW = ceil(R/32); device uint32[n*RW], may be NULL
 * to use workspace).  Constraint c is satisfied iff its predicate holds on
 * t = number of its true literals; nsat[r] = # satisfied constraints
 * (device int32[R]), wsat[r] = sum of their weights in FP64 (device
 * double[R] or NULL).  Exact integer work. */
int cls_round_score(const cls_problem* p, int32_t R, const float* x,
                    uint32_t* bits, int32_t* nsat, double* wsat, void* ws,
                    size_t ws_bytes, void* stream);

/* n_steps full CLS steps on x in place (Sec. 2.3): evaluate the gradient,
 * take the projected step with rate lr, round and score.  After the call
 * bits/nsat/wsat (each may be NULL) describe the final rounded point.
 * x: device float[n*R].  n_steps >= 0. */
int cls_step(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
             uint32_t* bits, int32_t* nsat, double* wsat, void* ws,
             size_t ws_bytes, void* stream);

/* The n-step loop as ONE persistent launch (all restarts and all
 * constraints in one launch; Sec. 3.3's lockstep batch).  Same
 * arguments and results as cls_step (x, bits and counts bit for bit).
 * Supported when every constraint that needs FE work is a closed-form
 * product of at most 16 literals (e.g. random k-SAT); otherwise
 * CLS_ERR_UNSUPPORTED (use cls_step or a graph).  Two forms:
 *   - when one tile of 32 restarts -- x (128 B per variable), every literal
 *     partial row (128 B per FE literal), the literal records (8 B each),
 *     the items (32 B per constraint) and the bitset -- fits in 220 KB of
 *     shared memory (random 3-SAT with n = 100, m = 426 needs 197 KB),
 *     one CTA per tile runs all n steps with the tile on chip and
 *     __syncthreads between the phases; the restarts are independent, so
 *     no CTA waits on another;
 *   - otherwise a cooperative kernel whose warps take, in turn, the
 *     FE+gradient items, the accumulate/step/round items and the scoring
 *     items of every step, separated by grid barriers
 *     (CLS_ERR_UNSUPPORTED without cooperative launch).  The barriers
 *     never spin unboundedly: a barrier that waits too long (~2^22 polls)
 *     sets an error flag in the workspace and every block returns.
 * cls_persistent_status reads that flag (synchronous; 0 = ok, 1 = a
 * barrier timed out; the one-CTA-per-tile form always leaves 0). */
int cls_step_persistent(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
                        uint32_t* bits, int32_t* nsat, double* wsat, void* ws, size_t ws_bytes,
                        void* stream);
int cls_persistent_status(const cls_problem* p, int32_t R, const void* ws, size_t ws_bytes,
                          int32_t* status);

/* Self-check of the persistent loop's grid barrier (no counterpart in the
 * paper): a cooperative launch of one block per SM passes `rounds` barriers
 * that release after (blocks + extra) arrivals.  With extra = 0 all rounds
 * pass (*status = 0, *passed = rounds); with extra > 0 no barrier can
 * release, every block gives up after spin_limit polls (0 < spin_limit <=
 * 2^24; ~100 ns each) and returns, *status = 1 and *passed = 0: the bounded
 * wait ends the kernel instead of hanging it.  scratch: >= 16 device bytes,
 * overwritten.  Synchronous on the legacy default stream. */
int cls_grid_barrier_check(int32_t rounds, int32_t extra, uint32_t spin_limit, void* scratch,
                           size_t scratch_bytes, int32_t* status, int32_t* passed);

/* End-to-end solve from HOST buffers: copies x0 (host float[n*R], pinned
 * memory recommended) to the device workspace, runs n_steps as cls_step,
 * and copies the final nsat (host int32[R]) and x (host float[n*R], may be
 * NULL) back, all on stream; synchronises the stream before returning.
 * Whole chunks of 10 steps run through a step-loop graph (as
 * cls_graph_create) that the problem records on first use and keeps while
 * ws, R, lr, the tuning and the weight mode stay the same; the remaining
 * steps run as cls_step.  Results are those of cls_step.  Recording needs
 * profiling off; with profiling on every step runs as cls_step.
 * ws must hold cls_workspace_size() + 4*n*R + 4*R + 8*R bytes (see
 * cls_solve_host_workspace_size). */
int cls_solve_host_workspace_size(const cls_problem* p, int32_t R, size_t* bytes);
int cls_solve_host(const cls_problem* p, int32_t R, const float* x0_host,
                   float lr, int32_t n_steps, int32_t* nsat_host,
                   float* x_host, void* ws, size_t ws_bytes, void* stream);

/* The step loop as one CUDA graph (Sec. 3.3: all restarts iterate in
 * lockstep).  cls_graph_create
 * records n_steps steps exactly as cls_step would run them (same kernels,
 * same arguments, same results) on private streams and instantiates the
 * graph.  Inside a step the FE+gradient launches of the different length
 * classes run concurrently (they write disjoint partial rows); step k's
 * score runs concurrently with step k+1's FE launches, and step k+1's
 * accumulate waits for it.  The pointers (x, bits, nsat, wsat, ws) are
 * baked into the graph and must stay valid; each cls_graph_launch then
 * performs the n_steps steps on `stream`.  Profiling must be off while
 * creating.  cls_graph_kernel_count returns the number of kernel launches
 * one graph launch performs.  Errors as cls_step; CLS_ERR_CUDA if capture
 * or instantiation fails. */
typedef struct cls_graph cls_graph;
/* cls_batch_graph_create: the same for `count` independent problems (e.g.
 * several instances, each with its own restarts, as in Sec. 3.2's
 * partial-assignment study), captured as concurrent branches of ONE graph;
 * per-problem arrays of restarts, iterates, outputs (bits/nsats/wsats may
 * be NULL or hold NULL entries) and workspaces. */
int cls_batch_graph_create(int32_t count, const cls_problem* const* ps, const int32_t* Rs,
                           float* const* xs, float lr, int32_t n_steps, uint32_t* const* bits,
                           int32_t* const* nsats, double* const* wsats, void* const* wss,
                           const size_t* ws_bytes, cls_graph** out);
int cls_graph_create(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
                     uint32_t* bits, int32_t* nsat, double* wsat, void* ws, size_t ws_bytes,
                     cls_graph** out);
int cls_graph_launch(cls_graph* g, void* stream);
int cls_graph_kernel_count(const cls_graph* g, int64_t* n);
int cls_graph_destroy(cls_graph* g);

/* Autotuning of the FE+gradient launch shapes: the split of constraints
 * over lanes and blocks and the tile sizes.
 * Constraints on the lane-group paths are bucketed by length; every bucket
 * is served by one lane-group configuration (lanes per (constraint,
 * restart) G, literal slots per lane Q, DFT or real roots, literal values in
 * registers or re-read from shared memory).  cls_autotune times every
 * admissible configuration on each non-empty bucket of this problem (reps
 * launches each, x = device float[n*R] as the input, ws as for cls_eval),
 * keeps the fastest and synchronises the stream.  Results do not depend on
 * the tuning beyond FP32 rounding order of the DFT products.
 * cls_tuning_get/cls_tuning_set read or replace the bucket -> configuration
 * map (n must equal the number of buckets, 25); cls_config_info(id, out[4])
 * describes configuration id (G, Q, kind, shared-memory y?) and, for
 * id = 1000 + b, bucket b (DFT?, maximum length).  Configuration ids run
 * 0..98 (kind 0 = real roots, 1 = DFT roots, 2 = DFT roots in packed pairs,
 * 3 = DFT roots in factored form, cos(phi) - i y sin(phi) scaled per lane)
 * plus 100, the checkpointed kernel for real-root buckets.  An invalid map
 * is rejected with CLS_ERR_INVALID. */
int cls_autotune(cls_problem* p, int32_t R, const float* x, int32_t reps, void* ws,
                 size_t ws_bytes, void* stream);
int cls_tuning_get(const cls_problem* p, int32_t* cfg, int32_t n);
int cls_tuning_set(cls_problem* p, const int32_t* cfg, int32_t n);
int cls_config_info(int32_t id, int32_t* out);

/* Algorithmic FP32 work of the DFT buckets under the current tuning (no
 * counterpart in the paper; for roofline accounting): out[0] = flops per
 * restart of one FE+gradient evaluation (a fused multiply-add counts 2):
 * per (literal, root) 20 for the direct factor alpha + beta w^j (kinds 1
 * and 2), 14 or 16 for the factored forms (kind 3; 14 in the two
 * forms with 3-operation complex products); out[1] = the number of
 * (literal, root) pairs per restart.  Host-only; CLS_ERR_INVALID on NULL. */
int cls_dft_work(const cls_problem* p, int64_t* out);

/* Flops of the DFT roots evaluated by the factored path since the last
 * reset (no counterpart in the paper; for roofline accounting): the direct
 * and packed-pair DFT kernels add 20 flops per (literal, root) of every
 * restart (all J roots); the dense
 * factored kernel skips, per restart, the roots whose terms are provably
 * below 2^-24 in total (a bound on the factors' moduli from the sums of
 * (1 - y_i^2)^m, m = 1..4), so its work depends on the point; it adds 14 or
 * 16 flops per (literal, evaluated root) of every restart to a per-problem
 * device counter.  The power-sum pass (constraints of 64 literals or more,
 * see cls_series_range) adds L (4 + 8K) + j (8K + 40) per restart for the j
 * roots it evaluates with K terms and the partials by Clenshaw's recurrence,
 * L (4 + 6K) + K^2 + j (8K + 40) with the partials by Horner's rule, and
 * L (4 + 4K) + j (8K + 40) when it hands the remaining roots to the dense
 * kernel (which counts the other 4K per literal).  Synchronises
 * the device; *flops = the count; reset != 0 zeroes it afterwards.
 * CLS_ERR_INVALID on NULL. */
int cls_dft_flops_counter(cls_problem* p, int64_t* flops, int32_t reset);

/* Range of the power-sum pass (an evaluation route of the Fourier form of
 * Sec. 2.3 that the paper does not use): with the logarithm of every factor
 * alpha + beta w^j of a constraint of L literals written as a Chebyshev
 * series in the literal's value on [-1, 1], the number of low
 * roots j = 1..js whose truncation after K terms is at most 2^-24, both for
 * log G_j over the L literals and for each literal's partial, capped at 96.
 * Host-only.  Returns js >= 0, or -1 (CLS_ERR_INVALID) for L < 1 or K < 1. */
int cls_series_range(int32_t L, int32_t K);

/* cls_step without any allocation, for callers that cannot allocate device
 * memory while they run (a real-time loop that must not touch the allocator
 * after start-up, a process confined to a fixed device-memory budget owned
 * by another runtime, a host language with no route to cudaMalloc).  The
 * paper has no counterpart; this is an interface convenience.
 * Same arguments and results as cls_step, minus the workspace: the scratch
 * lives in a file-scope device array of 32 MiB that every GPU loading this
 * library holds until the process exits.  Problems whose
 * cls_workspace_size(p, R) exceeds 32 MiB are rejected with
 * CLS_ERR_WORKSPACE (use cls_step with a caller workspace instead).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The current device must be the problem's
 * device (CLS_ERR_INVALID otherwise).  The looked-up address is kept for the
 * life of the process: after a cudaDeviceReset it is stale, so do not call
 * this entry point again in that process.  All calls on a device share the one array and
 * it keeps the previous call's contents (the step writes every scratch byte
 * it reads), so calls that may overlap on the GPU -- on different streams,
 * or from different threads -- race and must be serialised by the caller.
 * Profiling must be off (it creates CUDA events); CLS_ERR_INVALID
 * otherwise.  It calls no cudaMalloc/cudaFree. */
int cls_step_noalloc(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
                     uint32_t* bits, int32_t* nsat, double* wsat, void* stream);

/* Learned initial points: a small message-passing network over the
 * constraint-variable incidence graph proposes initial points (the paper
 * has no learned component).  Model, per node, hidden width 64:
 *   embed   h_v = relu(W_vin f_v + b_vin),  h_c = relu(W_cin f_c + b_cin),
 *           f_v = [1, deg/16, pos/deg, neg/deg],
 *           f_c = [onehot(type, 9), L/64, k/L, w]
 *   layers  a_c = L^-1/2 sum_{e in c} s_e h_v[v_e];   h_c = relu(W_cl [h_c, a_c] + b_cl)
 *   (x2)    a_v = deg^-1/2 sum_{e on v} s_e h_c[c_e]; h_v = relu(W_vl [h_v, a_v] + b_vl)
 *   head    z_v = w_out . h_v + b_out
 *   points  x0[v*R + r] = tanh(z_v + tau u[v,r]) with u the draws of
 *           cls_init_uniform (same seed / counter convention); pinned
 *           variables keep their fixed value.
 * The four 128-wide dense layers run on tensor cores with bf16 operands
 * and fp32 accumulation (forward and both backward products); everything
 * else is fp32.  Parameters are one flat fp32 vector (cls_mpnn_sizes gives
 * its length and the activation workspace size); the layout is
 * W_vin(64x4) b_vin W_cin(64x12) b_cin, then per layer W_c(64x128) b_c
 * W_v(64x128) b_v, then w_out(64) b_out(1).  All reductions are blocked and
 * summed in a fixed order: results are deterministic.
 *   cls_mpnn_create     build the graph view of a problem (allocates, sync)
 *   cls_mpnn_param_init weights U(-a, a), a = fan_in^-1/2 (Philox), ReLU
 *                       biases 0.01, head bias 0
 *   cls_mpnn_forward    z[n]; keeps activations in act for the backward
 *   cls_mpnn_points     x0 from z (device float[n*R])
 *   cls_mpnn_head_grad  dz_v = sum_r gx0[v,r](1 - x0^2) +
 *                       lam/n_free * d/dz softplus(-2 t_v z_v) (target may
 *                       be NULL: no target term); pinned variables get 0
 *   cls_mpnn_backward   dparams = d(sum_v dz_v z_v)/dparams, using the act
 *                       of the immediately preceding forward with the same
 *                       params
 *   cls_adam_step       one bias-corrected Adam update (Kingma & Ba), step
 *                       t >= 1, all arrays device float[n] */
typedef struct cls_mpnn cls_mpnn;
int cls_mpnn_create(const cls_problem* p, cls_mpnn** out);
int cls_mpnn_destroy(cls_mpnn* g);
int cls_mpnn_sizes(const cls_mpnn* g, int64_t* n_params, size_t* act_bytes);
int cls_mpnn_param_init(const cls_mpnn* g, uint64_t seed, float* params, void* stream);
int cls_mpnn_forward(const cls_mpnn* g, const float* params, float* z, void* act,
                     size_t act_bytes, void* stream);
int cls_mpnn_points(const cls_mpnn* g, const float* z, int32_t R, uint64_t seed,
                    int64_t r_offset, float tau, float* x0, void* stream);
int cls_mpnn_head_grad(const cls_mpnn* g, const float* z, const float* x0, const float* gx0,
                       int32_t R, const int8_t* target, float lam, float* dz, void* stream);
int cls_mpnn_backward(const cls_mpnn* g, const float* params, const float* dz, float* dparams,
                      void* act, size_t act_bytes, void* stream);
int cls_adam_step(int64_t n, float* params, const float* grads, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int32_t t, void* stream);

/* Per-kernel timing (tracing): when enabled, each kernel launch of the
 * compute calls is bracketed by CUDA events on its stream; cls_profile_read
 * synchronises and returns, for kernel class kc (0 = thread-path FE+grad,
 * 1 = lane-group real FE+grad, 2 = lane-group DFT FE+grad, 3 = gradient
 * accumulate + step + round, 4 = score, 5 = reductions, 6 = init), the
 * number of launches and their summed duration in ms since the last reset.
 * Profiling must be off while a stream is being captured. */
int cls_profile_enable(cls_problem* p, int on);
int cls_profile_read(cls_problem* p, int kc, int64_t* launches, double* total_ms);
int cls_profile_reset(cls_problem* p);

const char* cls_strerror(int code);
const char* cls_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLS_B300_H */
