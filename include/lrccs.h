/*
 * lrccs.h -- C ABI of liblrccs, a GB300 (sm_103a) implementation of the
 * altGDmin hot path for low-rank column-wise compressive sensing (LRcCS) in
 * dynamic MRI (Babu, Lingala, Vaswani, arXiv 2212.09664).
 *
 * Problem (Sec. II-A, measurement model): recover the n x q matrix X = U B
 * (rank r) from y_k = A_k x_k, k = 1..q, with the multi-coil operator
 *     A_k = [H_k F D_1; ...; H_k F D_C],
 * F the unitary 2D DFT (forward kernel exp(-2 pi i k x / N), DC at index 0),
 * D_j = diag(d_j) the coil sensitivities and H_k the sampling of frame k.
 * The solver is auto-altGDmin (Alg. 2): truncated spectral initialisation,
 * then per iteration a least-squares B-step, one gradient step on U with
 * eta = 0.14 / ||grad f(U_0, B_0)||_2, and QR re-orthonormalisation.
 *
 * Conventions used by every entry point
 *   complex     : interleaved float32 pairs (re, im), "complex64", 8 bytes
 *   pixel index : i = y * nx + x, k-space index i = ky * nx + kx
 *   U           : n x r, row-major  (element (i, l) at U[i * r + l])
 *   B           : r x q, column-major, b_k contiguous (element (l, k) at B[k * r + l])
 *   X           : n x q, column-major, frame k contiguous (element (i, k) at X[k * n + i])
 *   y           : ragged, frame k / coil j / sample s at y[C * fp[k] + j * m_k + s],
 *                 m_k = fp[k+1] - fp[k] samples per coil, samples of a frame in
 *                 ascending k-space index
 *   pointers    : every d_* pointer is device memory owned by the caller; the
 *                 library only reads inputs during the call's stream work and
 *                 writes outputs in place.  The context owns all other memory.
 *   streams     : all work is ordered on the stream given to lrccs_create.
 *   errors      : every call returns an lrccs_status; nothing throws or aborts
 *                 across the ABI.  lrccs_last_error() describes the last failure.
 *                 Device-side failures (a non-SPD normal matrix, a wait that timed
 *                 out) are recorded in a device status word and returned by the
 *                 next call that synchronises (lrccs_init, lrccs_synchronize,
 *                 lrccs_iterate when info is requested).
 *
 * Scope of this build: images with ny, nx multiples of 32 in [32, 256];
 * rank r <= 16; q <= 128 frames; C <= 64 coils.  Masks are arbitrary sample
 * sets on the Cartesian grid.  Masks whose rows are either fully sampled or
 * empty (1D Cartesian lines, Sec. V) take a faster path with no x-direction
 * transforms; any other mask (pseudo-radial spokes gridded onto the grid,
 * scattered samples) takes the general path with full 2D transforms.
 */
#ifndef LRCCS_H
#define LRCCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrccs_ctx lrccs_ctx;

typedef enum lrccs_status {
    LRCCS_OK = 0,
    LRCCS_E_INVALID = 1,          /* bad argument, descriptor or layout */
    LRCCS_E_NOMEM = 2,            /* device allocation failed */
    LRCCS_E_CUDA = 3,             /* a CUDA runtime call failed */
    LRCCS_E_RANK_DEFICIENT = 4,   /* some frame's (A_k U)^H (A_k U) is not SPD, or m_k C < r */
    LRCCS_E_TIMEOUT = 5,          /* a bounded device wait gave up */
    LRCCS_E_ADMISSION = 6,        /* not enough free device memory to admit the work */
    LRCCS_E_STATE = 7,            /* call out of order (e.g. iterate before init) */
    LRCCS_E_UNSUPPORTED = 8       /* valid input outside this build's scope (see above) */
} lrccs_status;

/* Arithmetic of the iteration's forward transform (the DFT along ky of the
 * coil images of U on the sampled rows).  The precision forms run it as a
 * dense GEMM with the DFT matrix of the sampled rows on the tcgen05 tensor
 * cores, accumulating in FP32 (Sec. II-A's A_k U, F as a matrix):
 *   BF16X3: operands split into bf16 hi + lo, three products (hi hi, hi lo, lo hi);
 *   FP16S : one FP16 product, the U-side operand scaled per 128-column tile by
 *           a power of two (from the tile's largest entry), unscaled after.
 * Everything else (the adjoint, the Grams, the solves, the QR, the init) is
 * the same in every form.  Other values: LRCCS_E_UNSUPPORTED. */
typedef enum lrccs_precision {
    LRCCS_PREC_FP32_FFT = 0,      /* FP32 fast Fourier transforms, FP32 accumulation */
    LRCCS_PREC_BF16X3_GEMM = 1,   /* DFT as a tcgen05 GEMM, 3-term BF16 split products */
    LRCCS_PREC_FP16S_GEMM = 2     /* DFT as a tcgen05 GEMM, FP16 with per-tile scaling */
} lrccs_precision;

typedef struct lrccs_dims {
    int32_t ny, nx;     /* image size */
    int32_t q;          /* number of frames */
    int32_t ncoil;      /* number of coils C */
    int32_t rank;       /* r > 0 fixes the rank; 0 selects it by the energy rule of Alg. 2 */
    int32_t rank_max;   /* buffer capacity for the rank (>= rank, <= 16); 0 -> 16 */
    int32_t precision;  /* lrccs_precision */
} lrccs_dims;

typedef struct lrccs_params {
    double trunc_factor;   /* 36   : gamma = 36 * mean |y|^2 over measured entries (Alg. 2, init) */
    double energy_pct;     /* 85   : b in the rank rule (Alg. 2) */
    double eta_c;          /* 0.14 : eta = eta_c / ||grad f(U_0, B_0)||_2 (Alg. 2) */
    double eps_exit;       /* 0.01 : exit when SD(U_{t-1}, U_t)/sqrt(r) < eps_exit (Alg. 2) */
    int32_t t_max;         /* 70   : iteration cap used by callers that solve to completion */
    int32_t exit_enabled;  /* 1: lrccs_iterate stops at the exit test (one host sync per iteration) */
    double admit_reserve_bytes;  /* 256 MiB: device memory that must stay free after lrccs_create's
                                    buffers, or the context is not admitted (LRCCS_E_ADMISSION) */
    /* tuning variants from the paper's discussion of its limitations (the
       defaults give Alg. 2 as printed) */
    int32_t exit_patience; /* 1    : with exit_enabled, stop once this many consecutive iterations
                                     pass the exit test (a more robust exit) */
    int32_t reserved;
    double eta_scale0;     /* 1    : variable step size eta_t = eta * eta_scale0 * eta_decay^k, */
    double eta_decay;      /* 1    :   k = iterations since eta was set (larger steps first) */
} lrccs_params;

/* Launch plan of the transform kernels (tile and grouping choices that do not
 * change the result's definition, only its speed and summation grouping): a
 * zero field keeps the built-in default.
 *   fwd_tx      : image columns per block of the forward column transform
 *                 (even, divides nx, fwd_tx * r <= 256, and fits shared memory)
 *   coil_groups : coil groups (thread-block cluster size, 1..8) of the column
 *                 adjoint and the line-mask row passes
 *   row_groups  : coil groups (1..8) of the general-mask row transforms
 *   bstep_form  : line masks only.  0 (default): when every sampled k-space
 *                 row of the iteration fits one block's shared memory and all
 *                 rows' blocks can be resident at once, the row Grams, the
 *                 per-frame solves (Alg. 2's B-step) and the row weighting of
 *                 the gradient run as one cooperative launch (k_bstep);
 *                 1: always the three separate kernels (k_row_gram, k_solve,
 *                 k_row_w).  Both forms compute the same quantities; their
 *                 FP32 summation order differs. */
typedef struct lrccs_plan {
    int32_t fwd_tx, coil_groups, row_groups, bstep_form;
} lrccs_plan;

typedef struct lrccs_iter_info {
    int32_t t;          /* iterations completed since lrccs_init */
    int32_t exited;     /* 1 if the exit test fired */
    double eta;         /* step size in use */
    double sd;          /* SD(U_{t-1}, U_t) of the last iteration */
    double gnorm;       /* ||grad||_2 of the first iteration (defines eta) */
} lrccs_iter_info;

/* Fill p with the paper's constants (36, 85, 0.14, 0.01, 70, exit off), a
 * 256 MiB admission reserve, exit_patience 1 and a constant step size. */
void lrccs_default_params(lrccs_params *p);

/* Create a context for one problem size on the current CUDA device.  The rank
 * may exceed q (a context that tracks mini-batches of fewer than r frames);
 * lrccs_init then refuses the fixed rank.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  Allocates every
 * device buffer the solve needs, after an admission check: the total
 * (lrccs_context_bytes) plus params->admit_reserve_bytes must not exceed the
 * device's free memory (cudaMemGetInfo), else nothing is allocated and the call
 * returns LRCCS_E_ADMISSION; a serving loop retries once other contexts are
 * destroyed.  Errors: LRCCS_E_INVALID (dims outside scope), LRCCS_E_UNSUPPORTED
 * (a precision that is not built), LRCCS_E_ADMISSION, LRCCS_E_NOMEM, LRCCS_E_CUDA. */
lrccs_status lrccs_create(const lrccs_dims *dims, const lrccs_params *params,
                          void *cuda_stream, lrccs_ctx **out);

/* Device bytes lrccs_create would allocate for dims (each buffer rounded up to
 * 256 bytes).  Not included: the general-mask and MEC work space, allocated by
 * the first call that needs them (see lrccs_init, lrccs_mec1).  Allocates
 * nothing.  Errors: LRCCS_E_INVALID, LRCCS_E_UNSUPPORTED. */
lrccs_status lrccs_context_bytes(const lrccs_dims *dims, size_t *bytes);

/* Spectral initialisation (Alg. 2, initialisation) from the measurements.
 *   d_y        : complex64, ragged (see conventions), C * fp[q] entries
 *   d_frame_ptr: int64, q + 1 offsets fp (samples per coil); must equal the
 *                running sum of the per-frame sample counts of d_mask
 *   d_mask     : uint8, q x (ny * nx) bitmap, 1 = sampled, DC at index 0
 *   d_smaps    : complex64, C x n coil sensitivities d_j
 *   out_rank   : receives r (fixed, or chosen by the energy rule); may be NULL
 * Compacts the masks, computes gamma, Z = [A_k^H y_k] and the truncated and
 * scaled X0, its top-r left singular vectors U_0, and resets t and eta.  The
 * call blocks until the device work is done.  Inputs are not retained.
 * The first general (2D) mask a context sees allocates that path's buffers
 * (about 2 q n int32 plus C n rank_max complex64).
 * Errors: LRCCS_E_INVALID (frame_ptr inconsistent with the mask, or a fixed
 * rank above q: the top-r singular vectors of the n x q X0 need r <= q),
 * LRCCS_E_RANK_DEFICIENT (sigma_r(X0) = 0), LRCCS_E_NOMEM, LRCCS_E_CUDA. */
lrccs_status lrccs_init(lrccs_ctx *ctx, const void *d_y, const int64_t *d_frame_ptr,
                        const uint8_t *d_mask, const void *d_smaps, int32_t *out_rank);

/* Run n_iter altGDmin iterations (Alg. 2, GDmin loop): B-step, gradient,
 * GD step, QR re-orthonormalisation (Cholesky QR of U - eta grad).
 * Asynchronous unless info is non-NULL or exit_enabled is set (then it
 * synchronises and reports the device status; a grid barrier that gave up
 * reports LRCCS_E_TIMEOUT).  Without exit_enabled and for n_iter > 1 the
 * n_iter iterations run as one CUDA graph captured on the context's stream
 * the first time a given n_iter (and set of timed kernels) is used and
 * replayed afterwards; the context's stream must then be a created stream
 * (on the legacy default stream, or while the caller is itself capturing
 * that stream, the kernels are launched one by one instead).  After the
 * call, X = U_{t-1} B_t is available through lrccs_get_factors /
 * lrccs_get_images.  Errors: LRCCS_E_STATE (no init), LRCCS_E_RANK_DEFICIENT,
 * LRCCS_E_CUDA. */
lrccs_status lrccs_iterate(lrccs_ctx *ctx, int32_t n_iter, lrccs_iter_info *info);

/* Copy the output pair of the last iteration: d_U <- U_{t-1} (n x r), d_B <- B_t
 * (r x q), so that X = U B (Alg. 2 output pairing).  Either pointer may be NULL.
 * Before any iteration, d_U receives U_0 and d_B is left untouched. */
lrccs_status lrccs_get_factors(lrccs_ctx *ctx, void *d_U, void *d_B);

/* Current subspace estimate U_t (n x r, row-major), the input of the next
 * iteration; also a subspace set by lrccs_set_subspace or lrccs_set_state. */
lrccs_status lrccs_get_subspace(lrccs_ctx *ctx, void *d_U);

/* Materialise X = U_{t-1} B_t into d_X (n x q column-major complex64). */
lrccs_status lrccs_get_images(lrccs_ctx *ctx, void *d_X);

/* Diagnostics: copy an internal array to caller device memory.
 *   LRCCS_BUF_Z     Z = [A_k^H y_k]            n x q, row-major (i * q + k)
 *   LRCCS_BUF_X0    truncated, scaled X0       n x q, row-major
 *   LRCCS_BUF_GRAD  last gradient              n x r, row-major
 *   LRCCS_BUF_SIGMA singular values of X0      q float64, descending
 *   LRCCS_BUF_IDX   compacted sample indices   fp[q] int32 (ascending per frame)
 *   LRCCS_BUF_SCAL  scalars                    8 float64: gamma, eta, sd, gnorm, mbar, -, -, -
 * bytes must be at least the array size. */
typedef enum lrccs_buffer {
    LRCCS_BUF_Z = 0, LRCCS_BUF_X0 = 1, LRCCS_BUF_GRAD = 2, LRCCS_BUF_SIGMA = 3,
    LRCCS_BUF_IDX = 4, LRCCS_BUF_SCAL = 5
} lrccs_buffer;
lrccs_status lrccs_get_buffer(lrccs_ctx *ctx, lrccs_buffer which, void *d_dst, size_t bytes);

/* ---- Mean step (Alg. 1, steps 1 and 2a) -------------------------------------
 * zbar = argmin_z sum_k ||y_k - A_k z||^2 by CGLS (conjugate gradients on the
 * normal equations A^H A z = A^H y of the stacked A = [A_1; ...; A_q], from
 * z = 0), stopped once ||A^H r_t|| <= tol ||A^H y|| or after max_iter
 * iterations (the paper: tol 1e-3, 10 iterations), and the residual
 * measurements y~_k = y_k - A_k zbar, which Alg. 1 passes to Alg. 2
 * (lrccs_init with d_y = d_ytil).
 *   d_y, d_frame_ptr, d_mask, d_smaps : as for lrccs_init
 *   tol       : >= 0;  max_iter : 0 .. 10000
 *   d_zbar    : device complex64, n entries (caller-owned), receives zbar
 *   d_ytil    : NULL, or device complex64 laid out like d_y (C * fp[q]
 *               entries, caller-owned, not aliasing d_y), receives y~
 *   out_iters : NULL, or receives the number of CG iterations run
 * The CG vectors use the context's subspace buffers, so afterwards the context
 * holds no solve (lrccs_init starts one).  The call synchronises.
 * Errors: LRCCS_E_INVALID, LRCCS_E_UNSUPPORTED (a mask that is not a union of
 * full lines), LRCCS_E_CUDA. */
lrccs_status lrccs_mean_step(lrccs_ctx *ctx, const void *d_y, const int64_t *d_frame_ptr,
                             const uint8_t *d_mask, const void *d_smaps, double tol, int32_t max_iter,
                             void *d_zbar, void *d_ytil, int32_t *out_iters);

/* ---- Model-error correction (Alg. 3) ------------------------------------------
 * Alg. 1 follows Alg. 2 by estimating, frame by frame, what the rank-r model
 * misses: with ytt_k = y~_k - A_k x_k the residual measurements of the last
 * iterate x_k = U_{t-1} b_k (y~ = the data the context was initialised with,
 * usually the mean-subtracted output of lrccs_mean_step),
 *   MEC-1 (unstructured): e_k from `iters` CGLS iterations on
 *          min_e ||ytt_k - A_k e||^2 from e = 0 (the paper: 3 iterations; its
 *          tolerance 1e-36 never stops them early);
 *   MEC-2 (sparse in the temporal Fourier domain): ISTA from E_0 = 0: step tau
 *          forms M_tau = F_t(E_tau + A^H(ytt - A E_tau)) (F_t the unitary DFT
 *          along the q frames), sets omega = omega_frac max|M_0| at tau = 0, and
 *          E_{tau+1} = F_t^{-1} SThr_omega(M_tau) (complex soft threshold
 *          m (|m| - omega)/|m| above omega, else 0); it stops after max_iter
 *          updates or once ||M_tau - M_{tau-1}||_F < rel_change ||M_{tau-1}||_F
 *          (the paper: 10, 0.0025, 0.001).
 * Both need a context after at least one lrccs_iterate (or lrccs_online_frames).
 *   d_zbar : NULL, or device complex64 n entries: the mean added into d_X
 *   d_E    : NULL, or device complex64 q x n (row k = e_k), receives E
 *   d_X    : NULL, or device complex64 q x n, receives x_k = zbar + U_{t-1} b_k + e_k
 *   out_iters (MEC-2): NULL, or the number of ISTA updates made
 * The frames are processed rank_max at a time through the per-frame normal
 * operators A_k^H A_k (the iteration's transforms with each frame's own
 * sampling between them).  The first call allocates 5 q n complex64 of work
 * space in the context.  Both calls synchronise (MEC-2 reads its stopping test
 * after every step).  Errors: LRCCS_E_STATE (no iterate yet), LRCCS_E_INVALID,
 * LRCCS_E_NOMEM, LRCCS_E_CUDA. */
lrccs_status lrccs_mec1(lrccs_ctx *ctx, int32_t iters, const void *d_zbar, void *d_E, void *d_X);
lrccs_status lrccs_mec2(lrccs_ctx *ctx, int32_t max_iter, double rel_change, double omega_frac,
                        const void *d_zbar, void *d_E, void *d_X, int32_t *out_iters);

/* ---- Online subspace tracking (Alg. 5) ----------------------------------------
 * After the first mini-batch (solved by Alg. 1: mean step, Alg. 2, MEC), Alg. 5
 * keeps that mini-batch's mean zbar and subspace U fixed and reconstructs every
 * later frame on its own: y~_k = y_k - A_k zbar, b_k = (A_k U)^+ y~_k, e_k from
 * mec_iters CGLS iterations on y~_k - A_k U b_k (MEC-1), x_k = zbar + U b_k + e_k.
 * One call reconstructs the context's q frames (q = the number of frames per
 * call) from the subspace set by lrccs_set_subspace / lrccs_set_state (one
 * Cholesky QR pass of it first, which changes an orthonormal U by rounding
 * only).
 *   d_y, d_frame_ptr, d_mask, d_smaps : the frames, as for lrccs_init
 *   d_zbar   : device complex64, n entries (the first mini-batch's mean)
 *   mec_iters: CGLS iterations of MEC-1 (3 in the paper), 0 .. 1000
 *   d_X      : NULL, or device complex64 q x n (row k = x_k)
 *   d_B      : NULL, or device complex64 r x q (b_k contiguous)
 * The call synchronises.  Errors: LRCCS_E_STATE (no subspace), LRCCS_E_INVALID,
 * LRCCS_E_RANK_DEFICIENT, LRCCS_E_NOMEM, LRCCS_E_CUDA. */
lrccs_status lrccs_online_frames(lrccs_ctx *ctx, const void *d_y, const int64_t *d_frame_ptr,
                                 const uint8_t *d_mask, const void *d_smaps, const void *d_zbar,
                                 int32_t mec_iters, void *d_X, void *d_B);

/* ---- Mini-batch subspace tracking (Alg. 4) ----------------------------------
 * Alg. 4 reconstructs a long acquisition one mini-batch of consecutive frames
 * at a time.  The first mini-batch (alpha_1 frames) is an ordinary solve:
 * lrccs_init then lrccs_iterate (T_max,1 = 70 in the paper) on a context
 * created with q = alpha_1.  Every later mini-batch j replaces the
 * initialisation of Alg. 2 (gamma, truncation, X0 and its SVD) by
 * U_0 <- U^(j-1), the final subspace of mini-batch j - 1, and runs at most
 * T_max,j GDmin iterations (5 in the paper) on its own frames.  One context
 * created with q = alpha tracks all later mini-batches of an acquisition:
 * U stays in its device memory from one call to the next.
 *
 * Step size.  The paper sets eta = eta_c / ||grad||_2 at t = 1 from the
 * initial estimates and relies on the gradient norm only decreasing after
 * that (Sec. III-C).  Tracking calls therefore keep the step size in force,
 * the one set at the first mini-batch's first iteration, unless reset_eta
 * asks for it to be set again from the warm start's own first gradient
 * (which, near convergence, is small: the first step then has spectral norm
 * eta_c in a poorly determined direction). */

/* Set the context's subspace and, optionally, its step size:
 *   d_U  : device complex64, n x rank, row-major (element (i, l) at i * rank + l),
 *          orthonormal columns; caller-owned, copied on the context's stream
 *          (not retained).  The next iteration re-orthonormalises it by one
 *          Cholesky QR pass (which changes an orthonormal U only by rounding)
 *          and forms its first right-hand sides U^H Z from the data then loaded.
 *   rank : 1 <= rank <= the context's rank_max; becomes the context's r
 *   eta  : > 0: the GD step size from the next iteration on;
 *          <= 0: set at the next iteration, eta = eta_c / ||grad||_2
 * Hands the first mini-batch's U^(1) (lrccs_get_subspace) and eta (from
 * lrccs_iterate's info) to the context that tracks the later mini-batches.
 * The call synchronises the context's stream.
 * Errors: LRCCS_E_INVALID (null pointer, rank out of range), LRCCS_E_CUDA. */
lrccs_status lrccs_set_subspace(lrccs_ctx *ctx, const void *d_U, int32_t rank, double eta);

/* Track one later mini-batch (Alg. 4, j > 1): U_0 <- the context's subspace,
 * then t_max GDmin iterations of Alg. 2 on this mini-batch's q frames.
 *   d_y, d_frame_ptr, d_mask : the mini-batch's samples, offsets and masks,
 *          laid out as for lrccs_init (q = the context's q); caller-owned
 *   d_smaps  : device complex64, C x n coil maps (copied)
 *   t_max    : iterations, >= 1 (with exit_enabled the loop also stops once
 *              SD(U_{t-1}, U_t) / sqrt(r) < eps_exit)
 *   reset_eta: 0 keeps the step size in force; 1 sets it again at this
 *              mini-batch's first iteration
 *   d_X      : NULL, or device memory for this mini-batch's images
 *              X = U_{t-1} B_t, q x n complex64 (row k = x_k), written
 *              asynchronously
 *   info     : NULL, or receives t, eta, sd, gnorm (the call then waits for
 *              the iterations)
 * The masks are compacted first (one wait for that step); the rest is queued
 * on the context's stream and the call returns: lrccs_synchronize waits for it
 * and reports its device status.  Afterwards the context holds this
 * mini-batch's data and final subspace, so lrccs_iterate, lrccs_get_factors
 * and lrccs_get_images work on it as after lrccs_init.  The iterations are
 * the ones lrccs_iterate launches; a captured iteration graph is replayed only
 * when it matches this mini-batch's sampled rows (none is captured here).
 * Errors: LRCCS_E_STATE (no subspace: call lrccs_init, lrccs_set_subspace or
 * lrccs_set_state first), LRCCS_E_INVALID, LRCCS_E_UNSUPPORTED (a mask that is
 * not a union of full lines), LRCCS_E_RANK_DEFICIENT, LRCCS_E_TIMEOUT,
 * LRCCS_E_CUDA. */
lrccs_status lrccs_track_minibatch(lrccs_ctx *ctx, const void *d_y, const int64_t *d_frame_ptr,
                                   const uint8_t *d_mask, const void *d_smaps, int32_t t_max,
                                   int32_t reset_eta, void *d_X, lrccs_iter_info *info);

/* Asynchronous form of lrccs_track_minibatch for serving loops (Alg. 4 as a
 * request loop).  The call only enqueues the request on the context's host
 * worker thread (started by the first such call) and returns at once with a
 * ticket; the worker runs lrccs_track_minibatch (including its wait for the
 * mask compaction) and queues the GPU work on the context's stream, so one
 * submitting thread can keep many contexts busy.  Requests of one context run
 * in submission order.  The inputs (d_y, d_frame_ptr, d_mask, d_smaps) must
 * stay valid and unchanged, and d_X untouched, until the ticket completes;
 * while any ticket of the context is pending only lrccs_ticket_query,
 * lrccs_ticket_wait and lrccs_track_minibatch_async may be called on it.
 * Errors: LRCCS_E_INVALID (null pointer, t_max < 1), LRCCS_E_CUDA. */
typedef struct lrccs_ticket { uint64_t id; } lrccs_ticket;
lrccs_status lrccs_track_minibatch_async(lrccs_ctx *ctx, const void *d_y, const int64_t *d_frame_ptr,
                                         const uint8_t *d_mask, const void *d_smaps, int32_t t_max,
                                         int32_t reset_eta, void *d_X, lrccs_ticket *ticket);
/* *done = 1 once the request has run and its GPU work has finished (0 while
 * pending).  Does not block.  Returns the request's status once it has run
 * (a host-side failure of lrccs_track_minibatch), LRCCS_OK while pending.
 * Errors: LRCCS_E_INVALID, LRCCS_E_STATE (unknown or expired ticket: results of
 * the last 256 requests are kept). */
lrccs_status lrccs_ticket_query(lrccs_ctx *ctx, const lrccs_ticket *ticket, int32_t *done);
/* Block until the request has run and its GPU work has finished; returns its
 * status, including device-side failures (non-SPD systems, timeouts) recorded
 * by its kernels. */
lrccs_status lrccs_ticket_wait(lrccs_ctx *ctx, const lrccs_ticket *ticket);

/* Checkpoint and resume of the solver state that later iterations depend on:
 * ny, nx, the rank r, the iteration count t, the step size eta (and whether it
 * is set) and the subspace U_t, as one host byte buffer (a 64-byte header
 * followed by U, n x r complex64).  The data (Z, masks) is not part of it.
 *   lrccs_get_state: host_buf NULL stores the size in *bytes; otherwise *bytes
 *     is the buffer's capacity on entry and the size written on return.
 *     Synchronises the context's stream.
 *   lrccs_set_state: takes a buffer written by lrccs_get_state of a context
 *     with the same ny and nx and r <= this context's rank_max, and
 *     synchronises.  To resume a solve, lrccs_init the same data, then
 *     lrccs_set_state, then lrccs_iterate; to resume tracking, lrccs_set_state
 *     then lrccs_track_minibatch.
 * Errors: LRCCS_E_STATE (get: no subspace yet), LRCCS_E_INVALID (null
 * pointer, short buffer, foreign or mismatched header), LRCCS_E_CUDA. */
lrccs_status lrccs_get_state(lrccs_ctx *ctx, void *host_buf, size_t *bytes);
lrccs_status lrccs_set_state(lrccs_ctx *ctx, const void *host_buf, size_t bytes);

/* Kernel profiling (measurement support; the paper reports per-step timing
 * markers, Sec. V).  Launch counts of every kernel are kept always.  CUDA-event
 * timing is recorded, on the context's stream, around every later launch of the
 * kernels whose name contains `pattern` ("*" = all; NULL or "" = none).
 * lrccs_profile_read synchronises the stream, folds the pending events into the
 * totals and fills up to `max` entries of `out` (one per kernel, in a fixed
 * order); *count receives the number of kernels.  Names are static strings.
 * Inside a replayed iteration graph (lrccs_iterate) the event records are graph
 * nodes placed on captured iterations 8, 24, 40, ... counted from 0 (the
 * `timed` count says how many), and
 * every replay since the last read reports the timings of the latest replay. */
typedef struct lrccs_kernel_stat {
    const char *name;     /* kernel name */
    int64_t launches;     /* launches since the last reset */
    int64_t timed;        /* launches that were timed */
    double ms;            /* summed CUDA-event time of the timed launches */
} lrccs_kernel_stat;
lrccs_status lrccs_profile(lrccs_ctx *ctx, const char *pattern);
lrccs_status lrccs_profile_read(lrccs_ctx *ctx, lrccs_kernel_stat *out, int32_t max, int32_t *count);
lrccs_status lrccs_profile_reset(lrccs_ctx *ctx);

/* Allocation-free truncation threshold.  The paper has no counterpart: this
 * entry point exists for callers of this library that cannot call cudaMalloc,
 * for example a reconstruction service that reserves all of its device
 * memory when it starts and forbids allocation on the acquisition path, or a
 * process whose device memory is owned by another allocator (a framework's
 * caching pool) so that a direct cudaMalloc could fail or fragment it.
 *
 * Computes, on cuda_stream, the threshold of the spectral initialisation
 *     *d_gamma = trunc_factor * sum_i |y_i|^2 / count
 * over `count` complex64 entries at d_y (device memory), with |y_i|^2 formed
 * in FP64 exactly as lrccs_init does; the result is the value lrccs_init uses
 * up to the order of the FP64 summation.  d_gamma is a device float64.
 *
 * It allocates nothing and calls no allocating routine.  Its scratch is a
 * fixed array in device memory at file scope (one FP64 partial sum per 65,536
 * entries, 4,096 at most, plus a counter: 32 KiB + 256 B) that every device
 * which loads the library holds until the process exits.  Every call looks up
 * that array's device address in the current context (cudaGetSymbolAddress,
 * which allocates nothing), so the entry point also works after a context is
 * recreated (cudaDeviceReset); make the first call on each device before any
 * stream capture (the first lookup loads the module).  Every call shares the
 * array and clears its counter before
 * use; calls whose work overlaps on the GPU (different streams, or another
 * host thread) race on it and must be serialised by the caller.
 * Errors: LRCCS_E_INVALID for null pointers or count outside
 * [1, LRCCS_NOALLOC_MAX_ENTRIES]; LRCCS_E_CUDA; text in lrccs_last_error(NULL). */
#define LRCCS_NOALLOC_MAX_ENTRIES ((int64_t)268435456)
lrccs_status lrccs_trunc_threshold_noalloc(const void *d_y, int64_t count, double trunc_factor, double *d_gamma,
                                           void *cuda_stream);

/* Set or read the context's launch plan (the next iterations use it; a
 * captured iteration graph is rebuilt).  A field that does not fit the
 * context's shape is ignored (the default is used).  Errors: LRCCS_E_INVALID. */
lrccs_status lrccs_set_plan(lrccs_ctx *ctx, const lrccs_plan *plan);
lrccs_status lrccs_get_plan(lrccs_ctx *ctx, lrccs_plan *plan);

/* Autotuner of the launch plan (measurement-driven, per problem shape): after
 * lrccs_init, times n_iter iterations (directly launched, CUDA events on the
 * context's stream, best of 2) for every candidate plan -- fwd_tx in {2, 4,
 * 8, 16, 32}, coil_groups in {1, 2, 3, 4, 6, 8} and, for general masks,
 * row_groups in {1, 2, 4, 8}, each within the shape's limits, one field at a
 * time from the defaults -- applies the fastest, and restores the solver
 * state (U, U_{t-1}, B, step size and its schedule, right-hand sides), so the solve continues
 * exactly as if it had not been tuned.  cache_path (NULL: no cache) names a
 * text file of tuned plans, one line per shape (ny nx q C r mask-kind
 * precision fwd_tx coil_groups row_groups): a shape found there is applied
 * without timing; a newly tuned one is appended.  out (may be NULL) receives
 * the plan.  Synchronises.  Errors: LRCCS_E_STATE (no init), LRCCS_E_CUDA. */
lrccs_status lrccs_autotune(lrccs_ctx *ctx, int32_t n_iter, const char *cache_path, lrccs_plan *out);

/* ---- Batched form: many independent slices, one graph launch ----------------
 * A batch holds contexts of independent problems (slices of uneven sizes,
 * each loaded by its own lrccs_init) and runs n_iter iterations of every one
 * of them as a single CUDA graph launched on cuda_stream: each context's
 * captured n_iter-iteration graph becomes a child node, one after another
 * (the GD/QR kernel of each slice is a cooperative launch that needs the whole
 * GPU, so the slices are not overlapped).  Every context must use a created
 * stream (its graph is captured there) and be idle when the batch is
 * launched; the batch graph is rebuilt when n_iter changes.  Afterwards each
 * context holds its slice's iterate as after lrccs_iterate.
 * Errors: LRCCS_E_INVALID, LRCCS_E_STATE (a context without data), LRCCS_E_CUDA. */
typedef struct lrccs_batch lrccs_batch;
lrccs_status lrccs_batch_create(lrccs_ctx *const *ctxs, int32_t count, void *cuda_stream, lrccs_batch **out);
lrccs_status lrccs_batch_iterate(lrccs_batch *batch, int32_t n_iter);
void lrccs_batch_destroy(lrccs_batch *batch);

/* Diagnostics: the iteration's forward transform of the current subspace,
 * T_j = F_y (d_j o U) on the k-space rows some frame samples (FP32 FFT, or the
 * tensor-core DFT GEMM of the context's precision form), copied to d_T as
 * complex64 [j][ky][x][l] (C x ny x nx x r; rows no frame samples are not
 * written).  bytes must be at least C n r 8.  Synchronises.  Errors:
 * LRCCS_E_INVALID, LRCCS_E_STATE (no lrccs_init yet), LRCCS_E_CUDA. */
lrccs_status lrccs_forward_transform(lrccs_ctx *ctx, void *d_T, size_t bytes);

/* Phase timing of the GD/QR kernel (measurement support, like the paper's
 * per-step timing markers, Sec. V).  enable != 0 allocates a stamp buffer and
 * makes every later GD/QR kernel of an iteration (launched directly or
 * replayed in the iteration graph, which is re-captured) record clock64() at
 * 9 points in each block: start, inputs staged, gradient and Gram partials
 * done, partials written, grid barrier 1 passed, totals reduced, barrier 2
 * passed, the r x r factors done, U_{t+1} written; and the global timer at
 * the block's entry and exit.  out (NULL, or 18 doubles) receives, for each of
 * the 8 intervals, the mean and the maximum over the blocks in SM cycles of
 * the last such launch, then the time from the first block's entry to the
 * last block's exit and the spread of the entries, in ns.  enable == 0 with out == NULL frees the buffer.
 * Errors: LRCCS_E_INVALID, LRCCS_E_STATE (out requested while off), LRCCS_E_NOMEM. */
lrccs_status lrccs_gdqr_phases(lrccs_ctx *ctx, int32_t enable, double *out);

/* Measurement support (the paper has no counterpart): phase times of the last
 * fused line-mask B-step launch (k_bstep), recorded while lrccs_gdqr_phases
 * timing is on.  out[22]: (mean, max over blocks) in ns of row load + Gram,
 * first grid barrier, the first frame's Gram sum, the rest of the per-frame
 * solves, second barrier, W_ky, row weighting, staging of the first Z chunk,
 * the rest of Z B^H, block exit; then the
 * first entry to last exit and the spread of the entries (ns).  Synchronises
 * the context's stream.
 * Errors: LRCCS_E_INVALID, LRCCS_E_STATE (timing off, or no fused launch). */
lrccs_status lrccs_bstep_phases(lrccs_ctx *ctx, double *out);

/* Test support for the bounded device waits (the paper has no counterpart).
 * With enable != 0 the next directly launched GD/QR kernel of this context (an
 * lrccs_iterate of one iteration, or one with exit_enabled or info) waits at
 * each grid barrier for one arrival more than its grid can make and gives up
 * after 2^16 polls instead of 2^24, so every barrier times out.  The kernel
 * still runs to its end (its results are then meaningless), the device status
 * word records the timeout and the next synchronising call returns
 * LRCCS_E_TIMEOUT.  The setting applies to that one launch and is never
 * captured into an iteration graph.  A later lrccs_init (or tracking call)
 * resets the status and the subspace, after which the context works as before.
 * Errors: LRCCS_E_INVALID (null ctx). */
lrccs_status lrccs_test_wait_timeout(lrccs_ctx *ctx, int32_t enable);

/* Wait for the context's stream and return any device-side failure. */
lrccs_status lrccs_synchronize(lrccs_ctx *ctx);

/* Free everything the context owns.  NULL is allowed. */
void lrccs_destroy(lrccs_ctx *ctx);

/* Text of the last failure on ctx (or of the last lrccs_create failure when
 * ctx is NULL).  Valid until the next call on the same context. */
const char *lrccs_last_error(const lrccs_ctx *ctx);

const char *lrccs_status_string(lrccs_status s);

#ifdef __cplusplus
}
#endif

#endif /* LRCCS_H */
