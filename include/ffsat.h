/*
 * ffsat.h — C ABI of the GB300 FastFourierSAT hot path (libffsat.so).
 *
 * The library evaluates the relaxed objective of a hybrid Boolean formula,
 * F(x) = sum_c w_c FE_c(x) (Def. "Objective", Eq. objective), and its gradient
 * at B restart points x in [-1,1]^n at once, runs fixed-step projected
 * gradient descent with restarts (Alg. 1 with App. A.3 "Projected Gradient
 * Descent"), and checks assignments exactly (Thm. "SAT Certificate").
 *
 * Conventions.
 *  - -1 encodes True and +1 False (Preliminaries, "Walsh Expansions").
 *  - Literals are DIMACS-style signed 1-based integers: +v is x_v, -v is -x_v.
 *  - Constraint types: FFSAT_OR (clause), FFSAT_XOR (satisfied iff the number of
 *    True literals has parity `param`; param=1 is the usual exclusive-or),
 *    FFSAT_ATLEAST (satisfied iff at least `param` literals are True).
 *  - FE_c is the Walsh expansion of c (Thm. "Walsh Transform"): -1 at satisfying
 *    corners, +1 at violating corners, multilinear in between.
 *  - Points are row-major [B, n] arrays in device memory, float32 or float64.
 *  - Every entry point returns FFSAT_OK (0) or a negative error code;
 *    ffsat_last_error() returns a thread-local message for the last failure.
 *  - Work is enqueued asynchronously on the given CUDA stream (a cudaStream_t
 *    passed as void*; NULL = legacy default stream).  Argument errors are
 *    returned synchronously; device-side errors (NaN inputs) are latched in a
 *    device status word and reported by ffsat_sync_status().
 *  - The caller owns every x / f / g / sat / solved buffer; the library never
 *    frees them.  The library owns the instance and its device tables.
 *  - An instance lives on the device it was loaded on (ffsat_options.device);
 *    every entry point makes that device current for its own work and restores
 *    the calling thread's current device before it returns.
 *  - An instance is read-only during ffsat_eval_grad / ffsat_check, which may run
 *    concurrently on different streams.  ffsat_step uses per-instance scratch for
 *    large n and ffsat_set_weights rewrites device tables: do not overlap those
 *    with other calls on the same instance.
 */
#ifndef FFSAT_H
#define FFSAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffsat_instance ffsat_instance;

enum { FFSAT_OR = 0, FFSAT_XOR = 1, FFSAT_ATLEAST = 2 };
enum { FFSAT_F32 = 0, FFSAT_F64 = 1 };
/* Node parametrisation of the DFT evaluation (see ffsat_options.form). */
enum { FFSAT_FORM_STABLE = 0, FFSAT_FORM_PAPER = 1 };

#define FFSAT_OK 0
#define FFSAT_ERR_ARG (-1)       /* NULL pointer, negative size, bad dtype/option */
#define FFSAT_ERR_VAR_RANGE (-2) /* literal 0 or |literal| > n_vars */
#define FFSAT_ERR_DUPVAR (-3)    /* a variable occurs twice in one constraint */
#define FFSAT_ERR_EMPTY (-4)     /* constraint with no literals */
#define FFSAT_ERR_PARAM (-5)     /* unknown type, parity not 0/1, K < 0, bad CSR */
#define FFSAT_ERR_WEIGHT (-6)    /* negative or non-finite weight */
#define FFSAT_ERR_TOOLONG (-7)   /* constraint longer than the kernels support */
#define FFSAT_ERR_CUDA (-8)      /* a CUDA runtime call failed (message has the detail) */
#define FFSAT_ERR_NAN (-9)       /* a NaN was found in x (latched on the device) */
#define FFSAT_ERR_DEVICE (-10)   /* another device-side error was latched */

/* Longest constraint accepted (literals). */
#define FFSAT_MAX_LEN 512

typedef struct ffsat_options {
    /* FFSAT_FORM_STABLE (default): node factors q_i + p_i w^j with
     * q_i = (1+y_i)/2, p_i = (1-y_i)/2 — the paper's polynomial prod_i(1 + y_i z)
     * evaluated at z_j = (1-w^j)/(1+w^j) and scaled by ((1+w^j)/2)^L per node, so
     * that every factor and every partial product has modulus <= 1 in FP32.
     * FFSAT_FORM_PAPER: the paper's literal factors 1 + y_i w^j with weights
     * b_j from the Walsh coefficients (Eq. forward / Eq. inverse); only for
     * constraints of <= 60 literals (it cancels catastrophically above that). */
    int32_t form;
    /* 1: evaluate OR and XOR constraints through the node (DFT) kernel as well
     * instead of their closed forms (cross-check / study mode). */
    int32_t node_all;
    /* Literals per lane in the node kernel: 0 = automatic (autotuned when
     * `autotune` is set), else 8 or 16. */
    int32_t node_r;
    /* 1: autotune the FP32 tile choices at load: time one evaluation on two
     * points per SM for each candidate of a coordinate search (node literals per
     * lane and segment shape, clause groups per task, points per CTA) and keep
     * the fastest; the choice is cached by instance shape, so later instances of
     * the same shape load without timing.  Costs up to about ten evaluations per
     * newly seen shape. */
    int32_t autotune;
    /* CUDA device ordinal, -1 = the current device. */
    int32_t device;
    /* CTAs per point of FP64 fixed-step calls (ffsat_step, ffsat_step_noalloc)
     * whose x and gradient fit in shared memory: 0 = automatic (a thread-block
     * cluster of 8, 4 or 2 CTAs when B clusters of that size fit on the GPU at
     * once and every CTA gets at least one warp task; GB300's FP64 rate is far
     * below its FP32 rate, so a few points otherwise leave most SMs' FP64 pipes
     * idle), 1 = one CTA per point, 2, 4 or 8 = that cluster size whenever a
     * cluster of it fits on the GPU.  The CTAs of a cluster split the point's
     * warp tasks and combine their partial gradients through distributed
     * shared memory (the sum of the partials, in rank order, replaces one
     * floating-point accumulation order by another). */
    int32_t cluster;
} ffsat_options;

typedef struct ffsat_step_args {
    int32_t T;         /* projected-GD iterations per call (>= 0) */
    int32_t restart;   /* 1: points whose sign vector is not a model restart uniformly */
    double lr;         /* step size eta of x <- clip(x - eta * grad F(x), -1, 1) */
    uint64_t seed;     /* restart seed */
    uint64_t epoch;    /* outer-round counter (part of the restart draw's key) */
    uint64_t b_offset; /* global index of point 0, so that sharded runs draw alike */
    /* Device int32 [n_cons] or NULL.  When set, the exact check that ends the
     * call adds to unsat_counts[c] the number of the B points (after their T
     * iterations, before any restart) whose sign vector violates c: the
     * unsatisfaction counts U_c of the ERWA weighting (Sec. 5).  The caller
     * zeroes the array; ffsat_batch_step ignores the field. */
    int32_t *unsat_counts;
} ffsat_step_args;

typedef struct ffsat_info {
    int32_t n, m;
    int64_t nnz;
    int32_t n_clause3;     /* clauses of <= 3 literals (thread-per-clause path) */
    int32_t n_product;     /* OR/XOR constraints on the product (closed-form) path */
    int32_t n_node;        /* constraints on the node (DFT) path */
    int32_t n_const;       /* constraints whose value is constant (K <= 0 or K > L) */
    int32_t n_tables;      /* distinct node tables */
    int32_t n_tasks;       /* warp tasks per point and iteration */
    int32_t node_r;        /* literals per lane chosen for the node kernel */
    int32_t smem_mode_f32; /* 0: x and g in shared memory, 1: x only, 2: neither,
                              3: x, g and the constraint data in shared memory */
    int32_t smem_mode_f64;
    int32_t threads_f32;   /* threads per CTA of the fused kernel */
    int64_t node_lane_work; /* sum over node constraints of nodes x (lanes x R) per point */
    int64_t device_bytes;  /* device memory held by the instance */
    int32_t autotuned;     /* 1 if the FP32 tile choices were set by the autotuner (ffsat_options.autotune) */
    float autotune_us[2];  /* FP32 evaluation time on the autotuner's probe batch (two points per SM),
                              microseconds: [0] the default choices, [1] the chosen ones */
    int32_t n_xor2;        /* XOR constraints of <= 2 literals (thread-per-constraint records, like clauses) */
    int32_t pad;
    int64_t smem_bytes_f32; /* dynamic shared memory per CTA of the fused kernel */
    int64_t smem_bytes_f64;
    /* FP32 tile choices (defaults unless autotuned) */
    int32_t tune_shape;       /* node segment shape: 0 cost model, 1 fewest lanes, 2 fewest literal slots */
    int32_t tune_clause_k;    /* clause groups of 32 per clause task: 0 automatic, else 1, 2 or 4 */
    int32_t tune_pts_per_cta; /* points per CTA of the fused kernel */
    int32_t tune_candidates;  /* candidate images timed at load (0 when the choice came from the cache) */
    int32_t tune_cached;      /* 1 if an earlier instance of the same shape supplied the choice */
    int32_t fix_words_f32;    /* 32-bit words of the FP32 shared-memory-resident fixed-point gradient:
                                 1 where the weights and degrees allow (each contribution rounded to
                                 2^-20 of the smallest max(w_c, 1) or finer), else 2; follows
                                 ffsat_set_weights */
} ffsat_info;

/* Fill `opt` with the defaults (stable form, closed forms for OR/XOR,
 * automatic node_r, autotune off, current device). */
void ffsat_default_options(ffsat_options *opt);

/* Build an instance from a CSR constraint list (all arrays in HOST memory):
 *   row_ptr[n_cons+1] int64, row_ptr[0] = 0, non-decreasing;
 *   lits[row_ptr[n_cons]] signed 1-based literals;
 *   type[n_cons] FFSAT_OR / FFSAT_XOR / FFSAT_ATLEAST;
 *   param[n_cons] parity (XOR, 0 or 1), K (ATLEAST, K >= 0; K > L is allowed and
 *     makes the constraint constantly violated), ignored for OR;
 *   weights[n_cons] finite, >= 0, or NULL for all ones.
 * Validates everything before touching the device (errors above), then
 * precomputes in FP64 on the host the DFT node tables of every distinct
 * (type, length, parameter) — the conjugated coefficients of Eq. inverse,
 * "computed in preprocessing" — buckets constraints by length and uploads all
 * tables once.  `opt` may be NULL.  On success *out owns device memory until
 * ffsat_free(). */
int ffsat_load_instance(int32_t n_vars, int32_t n_cons, const int64_t *row_ptr, const int32_t *lits,
                        const uint8_t *type, const int32_t *param, const double *weights,
                        const ffsat_options *opt, ffsat_instance **out);

/* Replace all constraint weights (HOST array of n_cons finite, non-negative values).
 * Synchronous with respect to the host; callers must not run other work on the
 * instance concurrently. */
int ffsat_set_weights(ffsat_instance *inst, const double *weights);

/* f[b] = F(x_b) (FP64, accumulated in FP64 across threads) and, if g != NULL,
 * g[b,:] = grad F(x_b) for the B points of x (Def. "Objective"; gradient by the
 * chain rule of Prop. "Chain rule", realised with prefix/suffix products).
 *   x: device [B, n] of dtype (FFSAT_F32 or FFSAT_F64), read only;
 *   f: device [B] double, or NULL;  g: device [B, n] of dtype, or NULL.
 * B = 0 is a no-op. */
int ffsat_eval_grad(ffsat_instance *inst, int32_t B, const void *x, int32_t dtype, double *f, void *g,
                    void *stream);

/* The plain FP64 comparator: the same mathematics in double precision with a
 * naive mapping (one thread per (constraint, point), global atomics, no
 * bucketing or shared-memory staging).  x, f, g: device double arrays
 * ([B,n], [B], [B,n]); f and g are overwritten. */
int ffsat_eval_grad_plain64(ffsat_instance *inst, int32_t B, const double *x, double *f, double *g,
                            void *stream);

/* One outer round of Alg. 1 for B points in place: args->T iterations of
 * x <- clip(x - lr grad F(x), -1, 1) (App. A.3 with a fixed step), then the exact
 * check of sgn(x) (sgn(x) = -1 iff x < 0), then, if args->restart, a uniform
 * redraw of every point that is not a model.  All iterations run inside one
 * kernel launch per call (FP64 calls on few points: one thread-block cluster
 * per point, see ffsat_options.cluster).
 *   x: device [B, n] of dtype, updated in place;
 *   solved: device [B] uint8 (1 iff sgn(x) satisfies every constraint), or NULL;
 *   n_unsat: device [B] int32 (violated constraints at sgn(x) before any restart), or NULL. */
int ffsat_step(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, const ffsat_step_args *args,
               uint8_t *solved, int32_t *n_unsat, void *stream);

/* Size of the scratch that ffsat_step_noalloc uses instead of allocating. */
#define FFSAT_STATIC_SCRATCH_BYTES (32u << 20)

/* ffsat_step without any device allocation; the paper has no counterpart.
 * Some callers cannot call cudaMalloc: a host that hands all device memory to
 * its own pool allocator, or a latency-critical loop that cannot accept the
 * implicit device synchronisation of an allocation.  ffsat_step allocates a
 * gradient scratch buffer of B * n values (and keeps it with the instance) when
 * a point's x and gradient do not fit in shared memory (ffsat_info.smem_mode
 * 1 or 2); this entry point uses instead a buffer of FFSAT_STATIC_SCRATCH_BYTES
 * that is reserved statically in the library's device image, so every GPU that
 * loads the library holds it until the process exits.
 *  - Same arguments, results and errors as ffsat_step.
 *  - Returns FFSAT_ERR_ARG when the instance needs scratch and
 *    B * n * sizeof(dtype) exceeds FFSAT_STATIC_SCRATCH_BYTES.
 *  - The first call on a device looks up the buffer's device address (with that
 *    device current) and caches it; make that first call before any stream
 *    capture.
 *  - Every call shares the one buffer and the kernel clears the part it uses
 *    before accumulating.  Calls whose kernels overlap on the GPU (other streams,
 *    other instances, other threads) race on it: order them. */
int ffsat_step_noalloc(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, const ffsat_step_args *args,
                       uint8_t *solved, int32_t *n_unsat, void *stream);

/* Exact checker (Alg. 1, line 5, evaluated on integers rather than through F):
 * sat[b] = 1 iff sgn(x_b) satisfies every constraint, regardless of weights;
 * n_unsat[b] = number of violated constraints.  Either output may be NULL. */
int ffsat_check(ffsat_instance *inst, int32_t B, const void *x, int32_t dtype, uint8_t *sat, int32_t *n_unsat,
                void *stream);

/* ---- projected gradient with line search (App. A.3, Alg. PGFP) ------------------------ */

typedef struct ffsat_pgfp_args {
    int32_t T;         /* at most T iterations per call (>= 0) */
    int32_t restart;   /* 1: points whose sign vector is not a model restart uniformly */
    double eta0;       /* initial step size of every point (> 0) */
    double beta;       /* backtracking factor in (0, 1); 0.5 is usual */
    int32_t maxls;     /* trial steps per iteration (>= 1); the last trial is taken when none passes */
    int32_t pad;
    double eta_min;    /* a point stops once its step size falls below this (the paper: 1e-12) */
    double slack;      /* absolute slack (>= 0) of the sufficient-decrease test, for the rounding of F */
    uint64_t seed;     /* restart seed, epoch and global index of point 0, as in ffsat_step_args */
    uint64_t epoch;
    uint64_t b_offset;
    int32_t *unsat_counts; /* device int32 [n_cons] or NULL, as in ffsat_step_args */
    int32_t *iters;    /* device int32 [B] or NULL: iterations each point took */
    double *eta_out;   /* device double [B] or NULL: each point's final step size */
} ffsat_pgfp_args;

/* One CLS round with the paper's projected-gradient fixed-point update and a
 * FISTA line search (App. A.3: "Default method ... is FISTA"; Beck and
 * Teboulle's backtracking variant), per point, starting from x_0 = x[b]:
 *   y_1 = x_0, t_1 = 1, eta = eta0;  for k = 1..T:
 *     g = grad F(y_k);  eta <- eta * beta^i for the first i = 0, 1, .. (at most
 *     maxls trials) with F(p) <= F(y_k) + <g, p - y_k> + |p - y_k|^2 / (2 eta) + slack,
 *     p = clip(y_k - eta g, -1, 1);
 *     x_k = p;  t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
 *     y_{k+1} = clip(x_k + (t_k - 1) / t_{k+1} (x_k - x_{k-1}), -1, 1);
 *     stop once eta < eta_min;
 * then the exact check and the uniform restart as in ffsat_step, all in one
 * launch.  The step size and the momentum start afresh in every call.
 *   x: device [B, n] of dtype, updated in place;  solved, n_unsat: as in ffsat_step.
 * Uses a per-instance [B, n] device scratch (allocated on first use or growth).
 * Errors: FFSAT_ERR_ARG for bad parameters, or when the instance's x does not
 * fit in shared memory (its shared-memory mode for dtype is 2). */
int ffsat_step_pgfp(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, const ffsat_pgfp_args *args,
                    uint8_t *solved, int32_t *n_unsat, void *stream);

/* ---- restart heuristics (Sec. 5: weighting and rephasing) ---------------------------- */

/* Rephasing phases (Sec. 5, "Rephasing Heuristics"). */
#define FFSAT_PHASE_ORIGINAL 0 /* keep the point the previous round ended at */
#define FFSAT_PHASE_FLIPPED 1  /* negate every coordinate */
#define FFSAT_PHASE_RANDOM 2   /* a fresh uniform draw from [-1, 1)^n */

/* U[c] = number of the B points whose sign vector violates constraint c: the
 * unsatisfaction counts of the ERWA weighting (Sec. 5, "Weighting Heuristics").
 *   x: device [B, n] of dtype, read only;  U: device int32 [n_cons], overwritten.
 * ffsat_step produces the same counts inside its final check when
 * ffsat_step_args.unsat_counts is set. */
int ffsat_unsat_counts(ffsat_instance *inst, int32_t B, const void *x, int32_t dtype, int32_t *U, void *stream);

/* ERWA update of every constraint weight (Prop. "Adaptive weight"):
 *   w_c <- (1 - alpha) w_c + alpha r_c,  r_c = U_c / max_c' U_c'  (r = 0 when max U = 0),
 * computed in FP64 on the device (each operation rounded, no contraction) and
 * written to every device copy of the weights; F, its gradient and ffsat_step
 * use the new weights from the next call on the stream.  Negative U_c count as 0.
 *   U: device int32 [n_cons];  alpha in [0, 1] (the paper uses 0.4).
 * No host synchronisation and no allocation.  The host-side weights given at
 * load or by ffsat_set_weights are not updated (read them with
 * ffsat_get_weights); ffsat_set_weights overwrites the device weights again. */
int ffsat_erwa_update(ffsat_instance *inst, const int32_t *U, double alpha, void *stream);

/* Rephase the restart points (Sec. 5, "Rephasing Heuristics"): every point b
 * with solved == NULL or solved[b] == 0 gets phase
 *   FFSAT_PHASE_ORIGINAL: x_b unchanged;  FFSAT_PHASE_FLIPPED: x_b <- -x_b;
 *   FFSAT_PHASE_RANDOM: x_b <- uniform draw on the 2^-23 grid of [-1, 1), the
 *   generator and key (seed, epoch, b_offset + b) of ffsat_step's restarts.
 *   x: device [B, n] of dtype, updated in place;  solved: device uint8 [B] or NULL.
 * Errors: FFSAT_ERR_ARG for a bad phase, dtype or NULL x with B > 0. */
int ffsat_rephase(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, int32_t phase, const uint8_t *solved,
                  uint64_t seed, uint64_t epoch, uint64_t b_offset, void *stream);

/* ffsat_rephase with the epoch read on the device from *epoch_dev (a uint64 in
 * device memory) when the kernel runs, so that a CUDA graph that captures the
 * call draws fresh random phases on every replay when something in the graph
 * advances the counter.  Errors: as ffsat_rephase, and FFSAT_ERR_ARG for a NULL
 * epoch_dev. */
int ffsat_rephase_at(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, int32_t phase, const uint8_t *solved,
                     uint64_t seed, const uint64_t *epoch_dev, uint64_t b_offset, void *stream);

/* Copy the current device weights (after ERWA updates) into a HOST array of
 * n_cons doubles.  Synchronises the device. */
int ffsat_get_weights(ffsat_instance *inst, double *weights);

/* ---- several instances of uneven size in one launch ---------------------------------- */

typedef struct ffsat_batch ffsat_batch;

/* Per-instance buffers of a batch call (all device pointers of the call's dtype). */
typedef struct ffsat_batch_io {
    int32_t B;         /* points of this instance (>= 0) */
    int32_t pad;
    void *x;           /* [B, n]: read by eval; updated in place by step */
    double *f;         /* eval: [B] or NULL */
    void *g;           /* eval: [B, n] or NULL */
    uint8_t *solved;   /* step: [B] or NULL */
    int32_t *n_unsat;  /* step: [B] or NULL */
    uint64_t b_offset; /* step: global index of point 0 of this instance (restart key) */
} ffsat_batch_io;

/* Group `count` loaded instances (same device) for single-launch evaluation: one
 * persistent kernel whose CTAs pull (instance, point) items, longest first, from a
 * device counter; every point runs exactly as in ffsat_eval_grad / ffsat_step of
 * its instance (same shared-memory mode and constraint layout).  The instances
 * must outlive the batch.  Configuration 4 of the benchmark ("uneven instances
 * in one launch") is this call.  When every instance was loaded with
 * ffsat_options.autotune and the batch has FP32 node-path work, the CTA width of
 * its FP32 kernel (384 or 512 threads) is chosen here by timing one evaluation
 * of two points per instance at each width (synchronous); otherwise 512. */
int ffsat_batch_create(ffsat_instance *const *insts, int32_t count, ffsat_batch **out);

/* Threads per CTA of the batch's kernel for dtype, and the FP32 probe times of
 * the two widths in microseconds (us384, us512: 0 when not timed; may be NULL). */
int ffsat_batch_threads(const ffsat_batch *bt, int32_t dtype, int32_t *threads, float *us384, float *us512);

/* ffsat_eval_grad for every instance of the batch in one launch (plus one
 * memset of the work counter).  io: host array of `count` entries. */
int ffsat_batch_eval_grad(ffsat_batch *bt, const ffsat_batch_io *io, int32_t dtype, void *stream);

/* ffsat_step for every instance of the batch in one launch; args->b_offset is
 * ignored in favour of io[k].b_offset.  Uses batch-owned gradient scratch for
 * instances whose x and gradient do not fit in shared memory. */
int ffsat_batch_step(ffsat_batch *bt, const ffsat_batch_io *io, int32_t dtype, const ffsat_step_args *args,
                     void *stream);

/* Release the batch (not its instances). */
void ffsat_batch_free(ffsat_batch *bt);

/* ---- learned restart proposal (no counterpart in the paper) -------------------------- */

typedef struct ffsat_mpnn ffsat_mpnn;

/* A message-passing network over the variable-constraint graph proposing restart
 * points (hidden width H = 64, `layers` = L rounds):
 *   h_v = relu(Wv0 f_v + bv0), h_c = relu(Wc0 f_c + bc0)
 *   per round: m_c = mean_{v in c} s_cv (A h_v);  h_c = relu(Uc [h_c; m_c] + buc)
 *              m_v = mean_{c ni v} s_cv (B h_c);  h_v = relu(Uv [h_v; m_v] + buv)
 *   z_v = wo . h_v + bo, proposal x0_v = tanh(z_v);  s_cv = -1 for a negated literal.
 * Variable features f_v (8): 1, positive and negative clause occurrences over the
 * mean degree (nnz / n), (pos - neg) / (pos + neg + 1) over clause occurrences,
 * XOR occurrences over the mean degree, (pos - neg) / (pos + neg + 1) over
 * cardinality occurrences, total occurrences over the mean degree, 0.
 * Constraint features f_c (8): 1, is OR, is XOR, is ATLEAST, length / 10, XOR
 * parity as +1 (odd) / -1 (even) else 0, K / length for ATLEAST else 0, 0.
 * Parameter vector (FP32, weights row-major [out x in]): Wv0 [64x8], bv0 [64],
 * Wc0 [64x8], bc0 [64], then per round A [64x64], Uc [64x128], buc [64],
 * B [64x64], Uv [64x128], buv [64], then wo [64], bo [1].
 * Kernels use the weights as BF16 (FP32 master copy for Adam) with FP32
 * activations and accumulation.  Initialisation: Glorot-uniform weights from
 * splitmix64(seed), zero biases.  The network lives on the current device. */
int ffsat_mpnn_create(int32_t layers, uint64_t seed, ffsat_mpnn **out);
int32_t ffsat_mpnn_num_params(const ffsat_mpnn *net);
/* Copy the FP32 master parameters to / from a HOST array of num_params floats. */
int ffsat_mpnn_get_params(const ffsat_mpnn *net, float *host);
int ffsat_mpnn_set_params(ffsat_mpnn *net, const float *host);
/* x0 (device [n] float) = the proposal for the instance. */
int ffsat_mpnn_forward(ffsat_mpnn *net, ffsat_instance *inst, float *x0, void *stream);
/* Loss mean_v softplus(-t_v z_v) for sign targets t (device [n], values -1/+1)
 * into *loss (device float), proposal into x0 (device [n] or NULL), and the
 * parameter gradient (kept for ffsat_mpnn_adam_step; copied to grad_host, a HOST
 * array of num_params floats, when not NULL — that copy synchronises). */
int ffsat_mpnn_loss_grad(ffsat_mpnn *net, ffsat_instance *inst, const float *target, float *loss, float *x0,
                         float *grad_host, void *stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradient. */
int ffsat_mpnn_adam_step(ffsat_mpnn *net, float lr, void *stream);
/* Restart from a proposal: every point b with solved[b] == 0 (all points when
 * solved is NULL) gets x_v = clip(proposal_v + noise * u, -1, 1), where u is the
 * same counter-based uniform draw on [-1, 1) as the uniform restart of ffsat_step
 * for (seed, epoch, b_offset + b, v). */
int ffsat_restart_from_proposal(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, const float *proposal,
                                float noise, const uint8_t *solved, uint64_t seed, uint64_t epoch, uint64_t b_offset,
                                void *stream);
void ffsat_mpnn_free(ffsat_mpnn *net);

/* Synchronise `stream`, read and clear the instance's device status word:
 * FFSAT_OK, FFSAT_ERR_NAN or FFSAT_ERR_DEVICE. */
int ffsat_sync_status(ffsat_instance *inst, void *stream);

/* Describe the instance's layout (host struct). */
int ffsat_instance_info(const ffsat_instance *inst, ffsat_info *info);

/* Number of kernel launches the last eval/step/check call on this thread enqueued. */
int32_t ffsat_last_launch_count(void);

/* CTAs per point of the last ffsat_step / ffsat_step_noalloc call on this
 * thread (1 unless it ran one thread-block cluster per point; 0 before any). */
int32_t ffsat_last_cluster_size(void);

/* Points per CTA of the last ffsat_step / ffsat_step_noalloc call on this
 * thread: 2 where an FP32 fixed step on the shared-memory-resident image with
 * one fixed-point word would otherwise need more than one wave of one CTA per SM
 * and two points' x and gradient words fit beside the image (each warp task then
 * serves both points with one load of its records; results are those of one
 * point per CTA, bit for bit where every contribution is fixed point, to FP32
 * rounding where XOR products add with FP32 atomics), else 1; 0 before any. */
int32_t ffsat_last_points_per_cta(void);

/* Measured fused multiply-add throughput of the current device, for the
 * arithmetic rooflines of a benchmark (the paper has no counterpart).
 * dtype FFSAT_F32 or FFSAT_F64.  Runs independent FMA chains on every SM
 * (4 CTAs of 256 threads per SM, 8 chains per thread) in one launch sized to
 * take about target_ms milliseconds (0 < target_ms <= 10000) after a warm-up
 * launch, timed with CUDA events on `stream`, and writes the rate in TFLOP/s
 * (2 flops per FMA) to *tflops and the timed launch's duration to *ms (may be
 * NULL).  Synchronous: it waits for its launches.  Allocates and frees a small
 * output buffer; reads and changes no clock setting.  Returns FFSAT_ERR_ARG for
 * a bad dtype / target or NULL tflops, FFSAT_ERR_CUDA if a launch fails. */
int ffsat_alu_peak(int32_t dtype, double target_ms, double *tflops, double *ms, void *stream);

/* Message for the last error on this thread ("" if none). */
const char *ffsat_last_error(void);

/* Release the instance and its device memory (NULL is ignored).  The caller must
 * make sure no enqueued work still uses it. */
void ffsat_free(ffsat_instance *inst);

#ifdef __cplusplus
}
#endif
#endif /* FFSAT_H */
