/*
 * ppca.h -- C ABI of the GB300 primed-PCA (pPCA) library.
 *
 * Primed PCA (Algorithm 1, "Primed PCA (pPCA_l)") takes a centred data set of
 * n points in d dimensions and two integers k > 0, l >= 0, runs a PRIMING
 * method that returns m = k + l approximate principal directions (step 1),
 * projects the data onto their span (steps 2-3) and runs an exact PCA in that
 * m-dimensional subspace (step 4), returning the first k principal components
 * (step 5).  This library implements the data-parallel hot path on one GPU:
 *
 *   ppca_create    borrow X (n x d, device) and validate it           (Input)
 *   ppca_prime     PRIMING(X, k + l): block power, Oja, EigenGame     (step 1)
 *   ppca_finalize  span -> project -> full-PCA -> top k               (steps 2-5)
 *
 * plus the individual steps (one X-pass, orthonormalisation, the small
 * eigensolve, quantisation) so that each can be checked and timed alone.
 *
 * Conventions shared by every call:
 *   - Pointers marked "device" are CUDA device pointers on the handle's device;
 *     "host" pointers are ordinary host memory.  The caller owns every buffer
 *     it passes (X, scales, V0, outputs); the library never frees them and does
 *     not retain them beyond the handle's lifetime.  A handle owns only its own
 *     workspace, allocated on first use and freed by ppca_destroy.
 *   - X is row-major with leading dimension ld (elements), ld >= d; its base
 *     address and the row pitch ld * sizeof(element) must be multiples of 16
 *     bytes (the kernels stage X with the Tensor Memory Accelerator).
 *   - Basis and eigenvector matrices (V0, V, Z, Q, E) are d x m column-major
 *     FP32: column j (one direction) is d contiguous floats, columns d apart.
 *   - X is assumed already centred (Section 1); the library does not centre.
 *   - All device work is enqueued on the handle's stream (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream) and is asynchronous.  Errors
 *     found on the host (arguments, allocation, launch) are returned at once.
 *     Errors found on the device (a Cholesky breakdown, a Jacobi sweep cap, a
 *     bounded wait that ran out) are written to a device status word and
 *     returned by the next ppca_sync() on that handle.
 *   - No call throws; every call returns a ppca_status.  ppca_last_error()
 *     gives a message for the last non-OK status of the calling thread.
 *   - Eigenvalues are reported as eig(X^T X) / n, in descending order;
 *     eigenvectors are unit vectors signed so that each one's largest-magnitude
 *     entry (lowest index among ties) is positive.
 */
#ifndef PPCA_H
#define PPCA_H

#include <stdint.h>

#if defined(__GNUC__)
#define PPCA_API __attribute__((visibility("default")))
#else
#define PPCA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ppca_status {
    PPCA_OK = 0,
    PPCA_ERR_INVALID = 1,     /* an argument is out of range or inconsistent          */
    PPCA_ERR_OOM = 2,         /* workspace allocation failed or exceeds the set limit  */
    PPCA_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed           */
    PPCA_ERR_STATE = 4,       /* call out of order (e.g. finalize before prime)        */
    PPCA_ERR_NUMERICAL = 5,   /* device reported a breakdown (see ppca_sync)           */
    PPCA_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out (see ppca_sync)    */
    PPCA_ERR_UNSUPPORTED = 7  /* valid request the library does not implement          */
} ppca_status;

/* Storage type of X. */
typedef enum ppca_dtype {
    PPCA_F32 = 0,             /* IEEE binary32                                          */
    PPCA_BF16 = 1,            /* bfloat16                                               */
    PPCA_FP8_E4M3 = 2         /* OCP FP8 E4M3 codes with one FP32 scale per row:       */
                              /*   x[r][j] = e4m3(code[r][j]) * scale[r]                */
} ppca_dtype;

/* PRIMING methods (Section 2; Section 5 for the optimiser). */
typedef enum ppca_method {
    PPCA_POWER = 0,           /* simultaneous (block) power iteration, Section 2.1     */
    PPCA_OJA = 1,             /* generalised Oja / Sanger rule, Section 2.2            */
    PPCA_EIGENGAME = 2,       /* EigenGame utilities (Section 2.3, Eqs. 1-3), SGD with */
                              /* Nesterov momentum (Section 5), parallel players        */
    PPCA_POWER_SEQ = 3        /* the power method of Section 2.1 one direction at a    */
                              /* time: x <- X^T X x / |X^T X x|, each step kept in the  */
                              /* complement of the directions found, until             */
                              /* |x_t - x_{t+1}| < eps or T steps                       */
} ppca_method;

/* Arithmetic of the X-streaming products (tensor cores, FP32 accumulation). */
typedef enum ppca_precision {
    PPCA_PREC_AUTO = 0,       /* prime: FAST; finalize: ACCURATE                        */
    PPCA_PREC_FAST = 1,       /* one product in the storage type (BF16 / FP8 / TF32)    */
    PPCA_PREC_ACCURATE = 2    /* split precision: the FP32 operand is split into BF16   */
                              /* (or TF32) pieces, about FP32 accuracy (BF16x3, 3xTF32) */
} ppca_precision;

typedef struct ppca_handle ppca_handle;

/* Parameters of ppca_prime.  Zero-initialise, then call
 * ppca_prime_params_default() to get the defaults of a method. */
typedef struct ppca_prime_params {
    const float *V0;          /* device, d x m column-major starting basis; NULL: the  */
                              /* library draws a Gaussian d x m basis from `seed`.      */
                              /* Either way the first basis is orth(V0).                */
    uint64_t seed;            /* seed of the library's own initial basis               */
    int64_t batch;            /* Oja / EigenGame minibatch rows (> 0)                   */
    double lr;                /* Oja: step t uses lr / (t + lr_offset);                 */
    double lr_offset;         /* EigenGame: constant lr (lr_offset ignored)             */
    double momentum;          /* EigenGame Nesterov momentum                            */
    int64_t t0;               /* step counter of the first step (for resume)            */
    int32_t precision;        /* ppca_precision of the priming passes                   */
    int32_t reserved;         /* must be 0                                              */
    double eps;               /* POWER_SEQ: termination threshold on |x_t - x_{t+1}|    */
} ppca_prime_params;

/* Library version, (major << 16) | minor.  Infrastructure: no counterpart in the paper. */
PPCA_API int32_t ppca_version(void);

/* Message for the last non-OK status returned to the calling thread (infrastructure:
 * no counterpart in the paper). */
PPCA_API const char *ppca_last_error(void);

/* Defaults: POWER -- nothing; OJA -- batch 256, lr 1, lr_offset 100 (so step t
 * uses 1/(t+100)); EIGENGAME -- batch 1024, lr 0.05, momentum 0.9; POWER_SEQ --
 * eps 1e-6.  Sets every
 * other field to zero / NULL.  Returns PPCA_ERR_INVALID for a NULL p or an
 * unknown method.  The momentum 0.9 is Section 5's; the paper tunes the rates
 * per data set (Section 5), so the other values are the library's. */
PPCA_API ppca_status ppca_prime_params_default(ppca_prime_params *p, ppca_method method);

/*
 * Create a handle over the data set X (Algorithm 1, Input).
 *   X           device, n x d row-major, leading dimension ld (>= d) elements,
 *               type dtype; borrowed, must stay valid until ppca_destroy.
 *   row_scales  device, n FP32 per-row scales; required for PPCA_FP8_E4M3,
 *               must be NULL otherwise.
 *   stream      cudaStream_t (as void*) every call of this handle enqueues on.
 * Requires n >= 2, d >= 1, ld >= d, 16-byte aligned X and row pitch.
 * No device work is enqueued.  On error *out is set to NULL.
 */
PPCA_API ppca_status ppca_create(ppca_handle **out, const void *X, int64_t n, int64_t d, int64_t ld,
                        ppca_dtype dtype, const float *row_scales, void *stream);

/*
 * Optional second copy of the same data in a wider type (e.g. BF16 when X is
 * FP8) that ppca_finalize reads instead of X.  Same shape n x d; borrowed.
 * Pass NULL to remove it.  Algorithm 1 reads one X throughout; this lets the
 * priming (step 1) run on a narrower type than the pPCA step (steps 2-5).
 */
PPCA_API ppca_status ppca_set_refine(ppca_handle *h, const void *X_refine, int64_t ld, ppca_dtype dtype);

/* Cap the handle's workspace (bytes, 0 = no cap); exceeding it gives PPCA_ERR_OOM.
 * Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_set_workspace_limit(ppca_handle *h, int64_t bytes);

/*
 * PRIMING (Algorithm 1, step 1): compute m = k + l approximate directions.
 *   POWER      T iterations of V <- orth(X^T X V) (Section 2.1, simultaneous
 *              iteration), orth = thin QR with positive diagonal by CholeskyQR2.
 *   OJA        T minibatch steps of the Sanger rule (Section 2.2), averaged over
 *              the batch: W += lr_t / |b| (X_b^T Y - W triu(Y^T Y)), Y = X_b W.
 *   EIGENGAME  T minibatch steps; every player ascends its utility (Eq. 3)
 *              with M_b = X_b^T X_b / |b|, gradient projected on the sphere's
 *              tangent space, Nesterov momentum, then renormalised.
 *   POWER_SEQ  the power method as Section 2.1 describes it: direction j
 *              starts from column j of orth(V0) and takes steps
 *              x <- P (X^T X x) / |P (X^T X x)|, P the projection on the
 *              complement of the directions already found (classical
 *              Gram-Schmidt, twice), until |x_t - x_{t+1}| < p->eps or T steps
 *              (T is a cap per direction).  The stopping test reads one number
 *              back per step, so this call blocks the host until it is done.
 *              ppca_prime_continue is not available for it.
 * Minibatch t covers rows [j b, min((j+1) b, n)), j = t mod ceil(n / b).
 * Requires 1 <= m <= min(d, n - 1, 128) and T >= 0.  p may be NULL (defaults).
 * Resets the handle's priming state (basis, step counter, momentum).
 */
PPCA_API ppca_status ppca_prime(ppca_handle *h, ppca_method method, int32_t m, int64_t T,
                       const ppca_prime_params *p);

/*
 * Continue the current priming run for T more steps / iterations (same method
 * and parameters), so that pPCA can be evaluated along the priming trajectory
 * (Section 5 evaluates it at checkpoints of one priming run).
 */
PPCA_API ppca_status ppca_prime_continue(ppca_handle *h, int64_t T);

/*
 * pPCA step (Algorithm 1, steps 2-5): Q = orth(V); one pass over X gives the
 * m x m matrix G = (X Q)^T (X Q); G = U diag(w) U^T by Jacobi; E = Q U[:, :k].
 *   k       1 <= k <= m (m of the last ppca_prime)
 *   E       device, d x k column-major FP32 output (unit eigenvectors, signed)
 *   lambda  device, k FP64 output: w[:k] / n, descending
 * Does not change the priming state: it can be called at any point of a run.
 * Returns PPCA_ERR_STATE if ppca_prime was never called.
 */
PPCA_API ppca_status ppca_finalize(ppca_handle *h, int32_t k, float *E, double *lambda,
                          ppca_precision precision);

/*
 * Host-buffer entry points (Algorithm 1's input, and its steps 2-5), for data
 * that lives in host memory.  Both are
 * stream-ordered on the handle's stream and asynchronous when the host buffers
 * are page-locked (cudaHostAlloc / cudaHostRegister); with pageable memory the
 * copies complete before the call returns.  Results are valid after ppca_sync.
 *
 * ppca_upload: copy all n rows of X from host memory into the device buffer the
 * handle was created with (which it overwrites), e.g. to stream a new data set
 * of the same shape through one handle.  X_host has the handle's dtype and
 * leading dimension ld_host >= d (elements).  row_scales_host: n FP32 row
 * scales for FP8 data (required then, NULL otherwise).  The FP32/BF16 copy set
 * by ppca_set_refine is not touched.
 *
 * ppca_finalize_host: ppca_finalize into the handle's workspace, then E (d x k
 * column-major FP32) and lambda (k FP64) are copied to the host buffers.
 */
PPCA_API ppca_status ppca_upload(ppca_handle *h, const void *X_host, int64_t ld_host,
                                 const float *row_scales_host);
PPCA_API ppca_status ppca_finalize_host(ppca_handle *h, int32_t k, float *E_host, double *lambda_host,
                                        ppca_precision precision);

/*
 * pPCA step on a seeded sample of the rows.  For its large runs the paper
 * projects only 10 % of the data in the full-PCA step, which cuts that step's
 * cost about tenfold (Section 5, large-scale datasets).  Rows are taken in
 * blocks of 128 consecutive rows (the last block may be shorter): block t is
 * kept when the t-th output of the SplitMix64 stream seeded with `seed`
 * (Steele, Lea and Flood, 2014: z = seed + t' * 0x9E3779B97F4A7C15 for
 * t' = t + 1, then the published mixing steps), as a 53-bit fraction, is below
 * `fraction`; if no block is kept, the block with the smallest output is.
 * Steps 2-5 then run as in ppca_finalize with G = (X_S Q)^T (X_S Q) over the
 * sampled rows S and lambda = eig(G) / |S|.
 *   fraction  in (0, 1]; 1 keeps every block (the result equals ppca_finalize's)
 *   rows_used host, may be NULL: |S|
 * BF16 or FP32 data (or the ppca_set_refine copy) on tensor cores only:
 * PPCA_ERR_UNSUPPORTED otherwise.
 */
PPCA_API ppca_status ppca_finalize_sampled(ppca_handle *h, int32_t k, float *E, double *lambda,
                                           ppca_precision precision, double fraction, uint64_t seed,
                                           int64_t *rows_used);

/*
 * Variance captured by each of k directions, the evaluation of the paper's
 * large-scale runs (Section 5.3): var[j] = e_j^T (X^T X) e_j for the columns
 * e_j of E (device, d x k column-major FP32, taken as given), one pass over X
 * (the ppca_set_refine copy when set).  var: device, k FP64.  ACCURATE/AUTO:
 * split-precision products (about 2^-24); FAST: the fast products.  After
 * ppca_prime, k may not exceed its m (PPCA_ERR_INVALID).
 */
PPCA_API ppca_status ppca_variance_captured(ppca_handle *h, const float *E, int32_t k, double *var,
                                            ppca_precision precision);

/* Device copy of the current primed basis V (d x m column-major FP32): the
 * output of Algorithm 1, step 1.  Only span(V) passes to the pPCA step; after
 * block power steps V's columns are orthonormal to about 1e-4 (the second
 * CholeskyQR pass of a step runs only when the first leaves more). */
PPCA_API ppca_status ppca_get_basis(const ppca_handle *h, float *V_out);

/* Wait for the handle's stream; return the first device-side error, if any,
 * and clear it.  Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_sync(ppca_handle *h);

/*
 * Schedule of the fast X-pass over BF16 data (the knobs an autotuner sets).
 * The product X^T X V needs every element of X once; the fused form reads each
 * 128-row tile of X from HBM once: a producer pipeline computes Y = X V for the
 * tile (or for one half of its columns, kparts = 2, the two halves summed in
 * FP32) while consumer pipelines, each owning a 256-column slice of Z for the
 * whole pass, re-read the tile from L2 for Z += X^T Y.  The unfused form runs
 * the two products as separate kernels (X read twice).  An implementation
 * choice of the product of Sections 2.1-2.3; no counterpart in the paper.
 */
typedef struct ppca_schedule {
    int32_t fused;            /* 1: fused single-read pass; 0: two kernels; -1: library default */
    int32_t producers;        /* CTAs running Y = X V in the fused pass (0: one per SM)           */
    int32_t window;           /* tiles a producer may run ahead of the slowest consumer (0: the  */
                              /* tiles being produced plus four per consumer row group)           */
    int32_t flush;            /* projected Gram (split-precision Y = X Q) and the fused pass's    */
                              /* Z = X^T Y: K-stages (64 wide) an FP32 tensor-core accumulator    */
                              /* takes before it is folded into a double-float sum (0: library    */
                              /* default -- 4 for BF16 data and 1 for FP32 data in the projected  */
                              /* Gram, 4096 (2048 row tiles) in the fused pass; larger = fewer    */
                              /* folds, less accurate).  The two-kernel X-passes fold at fixed    */
                              /* intervals.                                                       */
    int32_t engine;           /* X-pass engine: 0 library choice, 1 tensor cores (BF16 / FP32     */
                              /* data), 2 CUDA cores (any data type)                              */
    int32_t kparts;           /* fused pass: K parts per 128-row tile of Y = X V (1 or 2, 2 only  */
                              /* when d spans two 64-column stages; 0: library default, 1)        */
    int32_t l2_keep;          /* fused pass: percent (1-100) of each row tile's columns loaded    */
                              /* with the L2 evict_last hint for the consumers' re-read, the rest */
                              /* evict_first (0: library default, what fits in 70 % of L2)        */
    int32_t fp8_mma;          /* FP8 data, FAST passes: 0 library default (= 1), 1 the FP8 tensor  */
                              /* cores (kind::f8f6f4: V and Y as two E4M3 pieces), 2 E4M3 widened */
                              /* to BF16 in shared memory (kind::f16)                             */
} ppca_schedule;

/* Set the X-pass schedule of a handle (takes effect at its next pass).
 * Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_set_schedule(ppca_handle *h, const ppca_schedule *s);

/*
 * Row sharding over processes, one GPU each.  The priming passes and the
 * projected Gram matrix of the pPCA step are sums over the rows of X
 * (X^T X V = sum_r x_r x_r^T V in Section 2.1's power step and the
 * minibatch sums of Sections 2.2-2.3; G = sum_r (Q^T x_r)(x_r^T Q) in
 * Algorithm 1, step 3), so with the rows split over ranks each rank streams
 * its own rows and one sum across ranks per pass gives every rank the whole
 * data set's result: Z (d x m FP32) after each priming pass, the minibatch
 * size of Oja and EigenGame (their minibatch t is the union of every rank's
 * local minibatch t), and G (m x m FP64) of the pPCA step and of
 * ppca_variance_captured.  Everything after a sum is identical on every rank.
 *   fn       sums `count` elements (elem_bytes 4: FP32, 8: FP64) of the
 *            device buffer `buf` over all ranks, in place: after the work
 *            already enqueued on `stream` and before the work the library
 *            enqueues after fn returns (an NCCL all-reduce enqueued on that
 *            stream, or: synchronise, copy to the host, sum, copy back).  A
 *            status other than PPCA_OK is returned by the library call.
 *            NULL: one process again (the other arguments are ignored).
 *   ctx      passed to fn unchanged.
 *   n_total  rows of X over all ranks (eigenvalues are eig(X^T X) / n_total).
 *   staging  optional device buffer of staging_bytes the library copies each
 *            sum's operand into before fn (and back from after), so fn always
 *            sees the same buffer (at most d * m * 4 bytes are summed); NULL
 *            and 0: fn sees the library's own buffers.
 * Every rank must make the same calls with the same arguments (same m, T,
 * V0, seeds, precisions).  ppca_xpass and ppca_projected_gram stay local
 * (the rows of this rank).  Infrastructure (the data-parallel layout of the
 * method's sums): no counterpart in the paper, which runs on one GPU.
 */
typedef ppca_status (*ppca_allreduce_fn)(void *buf, int64_t count, int32_t elem_bytes, void *stream, void *ctx);
PPCA_API ppca_status ppca_set_allreduce(ppca_handle *h, ppca_allreduce_fn fn, void *ctx, int64_t n_total,
                                        void *staging, int64_t staging_bytes);

/*
 * Limit of every bounded wait inside the library's tensor-core kernels on the
 * current device, in nanoseconds (0 restores the default, 2 s; at most 60 s).
 * A wait that runs out sets the handle's device status word to a timeout, the
 * kernel drains its copies and MMAs in flight, frees its tensor memory and
 * returns; the next synchronising call returns PPCA_ERR_TIMEOUT and clears the
 * word, and the handle stays usable.  The limit is a device-wide setting that
 * holds for later launches until changed; set it while no pass is running.
 * Infrastructure (fault detection): no counterpart in the paper.
 */
PPCA_API ppca_status ppca_set_wait_limit(uint64_t ns);

/*
 * Autotuner: time one fast X-pass over rows [0, rows) of the handle's data
 * (rows = 0: all n) with m directions for every candidate schedule -- engine
 * (tensor cores / CUDA cores) and, for BF16 data, the fused single-read pass
 * or two kernels -- taking the fastest of `reps` timed runs after a warm-up
 * each, then set the winner on the handle and copy it to *best (may be NULL).
 * Uses the handle's scratch buffers (not the primed basis); blocks the host
 * until the handle's stream is idle.  Infrastructure: no counterpart in the paper.
 */
PPCA_API ppca_status ppca_autotune(ppca_handle *h, int32_t m, int64_t rows, int32_t reps, ppca_schedule *best);

/* Device-time accounting of the X-passes (the hot step), for measurement. */
typedef struct ppca_timing {
    double pass_ms[3];        /* summed device time of the X-passes since the reset,     */
                              /* indexed by the pass's ppca_precision (FAST, ACCURATE)    */
    int64_t passes[3];        /* X-passes timed, by precision                              */
    int64_t pass_rows[3];     /* rows of X those passes streamed, by precision             */
    int64_t launches;         /* kernels the library launched (all handles) since the reset */
} ppca_timing;

/*
 * Graph-replayed minibatch steps (enable != 0, the default).  Oja (Section 2.2)
 * and EigenGame (Section 2.3) take one minibatch per step; the steps of full
 * minibatches differ only in the batch's first row and, for Oja, in the step
 * size lr / (t + lr_offset).  With this on, ppca_prime / ppca_prime_continue
 * read both from device memory and run blocks of 16 such steps from a CUDA graph
 * captured once (per handle, shape and parameters) on a private stream joined
 * to the handle's stream by events; steps that hold an epoch's partial batch,
 * FP8 data, minibatches that are not whole 128-row tiles, row sharding, pass
 * timing, the CUDA-core engine and calls made while the handle's stream is
 * being captured run step by step.  The results are the same
 * bits either way (the same kernels and arithmetic).  enable == 0: always step
 * by step.  Infrastructure: no counterpart in the paper.
 */
PPCA_API ppca_status ppca_set_step_graphs(ppca_handle *h, int32_t enable);

/* enable != 0: record a CUDA event pair around every X-pass of this handle,
 * on its stream, and reset the counters; enable == 0: stop recording.
 * Measurement infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_set_timing(ppca_handle *h, int32_t enable);

/* Synchronise the handle's stream and report the counters since the reset
 * (measurement infrastructure: no counterpart in the paper). */
PPCA_API ppca_status ppca_get_timing(ppca_handle *h, ppca_timing *out);

/*
 * Checkpoint of the priming state (basis, momentum, step counter, method and
 * parameters) to host memory.  With buf == NULL, *bytes receives the size
 * needed.  ppca_set_state restores it into a handle over the same (n, d).
 * Synchronises the handle's stream.  Section 5 evaluates pPCA at checkpoints of
 * one priming run; this lets such a run stop and resume.
 */
PPCA_API ppca_status ppca_get_state(ppca_handle *h, void *buf, int64_t *bytes);
PPCA_API ppca_status ppca_set_state(ppca_handle *h, const void *buf, int64_t bytes);

/* Free the handle and its workspace (after the stream's work completes).
 * Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_destroy(ppca_handle *h);

/* ---------------------------------------------------------------------------
 * Batches: many independent primed-PCA problems of uneven size (each one
 * Algorithm 1 with block power priming), run as a single CUDA-graph launch.
 * ------------------------------------------------------------------------- */

typedef struct ppca_instance_desc {
    const void *X;            /* device, n x d row-major, leading dimension ld (as in ppca_create) */
    int64_t n, d, ld;
    int32_t dtype;            /* ppca_dtype                                                      */
    int32_t k;                /* components returned, 1 <= k <= m                                */
    int32_t m;                /* k + l, 1 <= m <= min(d, n - 1, 128)                             */
    int32_t T;                /* power iterations of the priming, >= 0                           */
    const float *row_scales;  /* FP8 only, else NULL                                             */
    const float *V0;          /* device d x m starting basis, or NULL: drawn from `seed`         */
    uint64_t seed;
    float *E;                 /* device output, d x k column-major                               */
    double *lambda;           /* device output, k eigenvalues / n, descending                    */
    float *V_out;             /* device output d x m, the primed basis (optional, NULL = none)   */
} ppca_instance_desc;

typedef struct ppca_batch ppca_batch;

/*
 * Validate `count` instance descriptors (copied; the buffers they point to are
 * borrowed and must stay valid) and set up `slots` concurrent slots (0 = 8),
 * each with a workspace sized for the largest instance it runs.  No device
 * work is enqueued.  Each instance is one Algorithm 1; the paper runs them one
 * at a time, so the batching itself has no counterpart in the paper.
 */
PPCA_API ppca_status ppca_batch_create(ppca_batch **out, const ppca_instance_desc *descs, int32_t count,
                                       int32_t slots, void *stream);

/*
 * Run every instance: block power priming (Algorithm 1, step 1; T iterations,
 * FAST precision) then the pPCA step (steps 2-5, ACCURATE), writing each
 * instance's E and lambda.  The
 * first call captures the whole batch -- instances spread round-robin over
 * the slots' streams -- into a CUDA graph; every call launches that graph on
 * the batch's stream (asynchronous).
 */
PPCA_API ppca_status ppca_batch_run(ppca_batch *b);

/*
 * Tune the batch before its first run: instances are grouped by (data type,
 * d, m, n rounded up to a power of two); for each group the autotuner
 * (ppca_autotune, cooperative fused pass excluded because slots run
 * concurrently) times the candidates on the group's first instance, and every
 * instance of the group then runs with the winner.  Returns the number of
 * groups in *groups (may be NULL).  PPCA_ERR_STATE after the first run.
 * Infrastructure: no counterpart in the paper.
 */
PPCA_API ppca_status ppca_batch_autotune(ppca_batch *b, int32_t reps, int32_t *groups);

/*
 * Data type the batch's FP32 instances are primed in: PPCA_F32 (the default:
 * the priming passes read X as given) or PPCA_BF16 (each run first rounds
 * every FP32 instance's X to BF16, round to nearest even, into a buffer of its
 * slot -- this call allocates them, for the largest FP32 instance of each slot
 * -- primes on that rounding with the BF16 fast passes, and runs the pPCA step
 * on the FP32 X at split precision).  The paper does not vary the precision;
 * this is the library's use of Algorithm 1's structure: only span(V) carries
 * from the priming to the pPCA step, which reads the data as stored.  Call
 * before ppca_batch_autotune and the first ppca_batch_run (PPCA_ERR_STATE
 * after them).
 */
PPCA_API ppca_status ppca_batch_set_priming(ppca_batch *b, int32_t dtype);

/*
 * Lockstep priming (enable != 0, the default): when every instance primes on
 * BF16 data (BF16 X, or FP32 X with ppca_batch_set_priming(PPCA_BF16) and
 * d % 8 == 0) and all share one T, the first ppca_batch_run captures step 1 of
 * Algorithm 1 for all instances at once -- the BF16 rounding, V = orth(V0) and
 * T times (Z = X^T X V on the BF16 tensor cores, V = orth(Z) by CholeskyQR2)
 * -- one kernel launch per kernel kind and iteration for the whole batch, the
 * work of the instances dealt out over the launch's blocks; the pPCA step
 * (steps 2-5) of each instance then runs on the slots as before.  It keeps
 * per-instance buffers for the whole batch (the BF16 copies of all FP32
 * instances at once instead of one per slot); when they cannot be allocated,
 * or the batch is not eligible, the batch primes on its slots.  enable == 0
 * always primes on the slots.  The paper runs one problem at a time: the
 * batching has no counterpart in it.  PPCA_ERR_STATE after the first run.
 */
PPCA_API ppca_status ppca_batch_set_lockstep(ppca_batch *b, int32_t enable);

/* *active = 1 if the captured graph primes in lockstep, else 0 (also before the
 * first run).  Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_batch_lockstep(const ppca_batch *b, int32_t *active);

/* Kernel launches one ppca_batch_run performs (the kernels captured in its graph;
 * 0 before the first run).  Measurement infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_batch_kernel_count(const ppca_batch *b, int64_t *count);

/* Wait for the batch's stream; report the first device-side error of any slot.
 * Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_batch_sync(ppca_batch *b);

/* Free the batch, its graph, streams and workspaces (after its work completes;
 * NULL is a no-op).  Infrastructure: no counterpart in the paper. */
PPCA_API ppca_status ppca_batch_destroy(ppca_batch *b);

/* ---------------------------------------------------------------------------
 * Individual steps of the hot path.
 * ------------------------------------------------------------------------- */

/*
 * Projected Gram matrix of the pPCA step (Algorithm 1, steps 3-4; Section 3):
 *   G = (X[r0:r1] Q)^T (X[r0:r1] Q)
 * over the data the pPCA step reads (the ppca_set_refine copy if one was set,
 * else X).
 *   Q  device, d x m column-major FP32 input (1 <= m <= 128), normally orthonormal
 *   G  device, m x m FP64 output, row-major, exactly symmetric
 * ACCURATE/AUTO: split-precision products, error about 1e-6 of |X Q|^2 entrywise
 * scale; FAST: BF16-level products.  Requires 0 <= r0 < r1 <= n.
 */
PPCA_API ppca_status ppca_projected_gram(ppca_handle *h, const float *Q, int32_t m, int64_t r0, int64_t r1,
                                double *G, ppca_precision precision);

/*
 * One fused X-pass (the product X^T X V of Sections 2.1-2.3, restricted to rows
 * [r0, r1)):  Y = X[r0:r1] V,  Z = X[r0:r1]^T Y.
 *   V  device, d x m column-major FP32 input (1 <= m <= 128)
 *   Z  device, d x m column-major FP32 output
 * Requires 0 <= r0 < r1 <= n.
 */
PPCA_API ppca_status ppca_xpass(ppca_handle *h, const float *V, int32_t m, int64_t r0, int64_t r1,
                       float *Z, ppca_precision precision);

/*
 * Orthonormalise the columns of V (d x m column-major, device) into Q (may
 * alias V) -- Algorithm 1, step 2 (an orthonormal basis of span(V)), and the
 * orth of Section 2.1's iteration: thin QR with positive diagonal by CholeskyQR2 -- G = V^T V, G = R^T R,
 * V <- V R^-1, twice.  G is accumulated in double-float FP32 (for d >= 16384 from
 * three BF16 pieces on the tensor cores); the first factorisation runs in FP32
 * on the diagonally scaled G and is redone in double-float when its
 * conditioning bound fails; the second, of a matrix within rounding of the
 * identity, in FP32 (a series when close enough).  A numerically rank-deficient
 * V (pivot below 1e-15 trace(G)) is reported as PPCA_ERR_NUMERICAL by ppca_sync.
 */
PPCA_API ppca_status ppca_orthonormalize(ppca_handle *h, const float *V, float *Q, int32_t m);

/*
 * Symmetric eigensolve of an m x m FP64 matrix (the full PCA of Algorithm 1, step 4):
 * G (device, m x m, symmetric) -> w (device, m, descending) and U (device,
 * m x m column-major, column j = unit eigenvector of w[j], sign convention as
 * above).  1 <= m <= 128.  G is not modified.  Parallel-order two-sided Jacobi
 * sweeps in FP32 on one CTA, a rotation skipped when its off-diagonal entry is
 * below the relative threshold (which keeps small eigenvalues accurate); the
 * eigenvalues are the FP64 Rayleigh quotients of the FP32 eigenvectors.  A
 * sweep cap reached is reported by ppca_sync.
 */
PPCA_API ppca_status ppca_eigh(ppca_handle *h, const double *G, int32_t m, double *w, double *U);

/*
 * The same symmetric eigensolve as ppca_eigh, for callers that cannot
 * allocate device memory at the point where they need it: a host program
 * whose device memory is handed out by its own allocator (a fixed budget
 * carved up front), or code on a latency-critical path where a cudaMalloc,
 * which may synchronise the device, is not acceptable.  This call has
 * no counterpart in the paper; it exists for those callers only.
 *
 * It takes no handle and allocates nothing: its scratch is a fixed array of
 * 256 KiB in the library's device memory, which every device that loads the
 * library holds until the process exits.
 *   G       device, m x m FP64 symmetric input (not modified)
 *   m       1 <= m <= 128 (the size the fixed scratch holds); anything else
 *           returns PPCA_ERR_INVALID with a message, and nothing is enqueued
 *   w, U    device outputs as in ppca_eigh (descending, column-major, signed)
 *   status  device int or NULL: set to a nonzero code if the Jacobi sweeps hit
 *           their cap (left unchanged otherwise); the caller clears it
 *   stream  cudaStream_t (as void*) the solve is enqueued on
 * The first call on a device looks up the device address of the scratch array
 * (with that device current) and caches it for the process; make that first
 * call before any stream capture.  A cudaDeviceReset after that first call is
 * not supported (the cached address would be stale).  Every call on a device
 * shares the one array and leaves its contents behind, so calls that overlap
 * on the same GPU race: order them (one stream, or events).  It runs the same
 * kernels as ppca_eigh, so its outputs equal ppca_eigh's bit for bit.
 */
PPCA_API ppca_status ppca_eigh_noalloc(const double *G, int32_t m, double *w, double *U, int *status,
                                       void *stream);

/*
 * Data-format step (the storage types of the priming passes; the paper does not
 * vary the data's precision, so this has no counterpart in the paper): quantise
 * FP32 rows (device, n x d, leading dimension ld_in) to BF16 (round to nearest even) or to FP8 E4M3 with one scale per row,
 *   scale[r] = max_j |x[r][j]| / 448 (1 for an all-zero row),
 *   code[r][j] = E4M3_RNE(x[r][j] / scale[r])  (both divisions in FP32).
 * Outputs are device arrays with leading dimension ld_out.  stream as above.
 */
PPCA_API ppca_status ppca_quantize_bf16(const float *X, int64_t n, int64_t d, int64_t ld_in,
                               uint16_t *out, int64_t ld_out, void *stream);
PPCA_API ppca_status ppca_quantize_fp8(const float *X, int64_t n, int64_t d, int64_t ld_in,
                              uint8_t *out, int64_t ld_out, float *scales, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PPCA_H */
