/*
 * emfuse.h -- C ABI of libemfuse.so: GB300 (sm_103a) gradient-domain colour correction of
 * registered EM image stacks, after Kazhdan et al., "Gradient-Domain Fusion for Color
 * Correction in Large EM Image Stacks" (arXiv 1506.02079).
 *
 * The method has two phases (Sec. 3):
 *   phase 1  I1 = I0 * G_{sigma_xy, sigma_z}: anisotropic Gaussian smoothing across the slice
 *            axis ("Anisotropic Smoothing"), Gaussian cut off beyond three standard
 *            deviations ("Implementation");
 *   phase 2  for every xy-slice j, the screened-Poisson system of Eq. (1),
 *            (alpha - Lap) I2_j = alpha I1_j - Lap I0_j,
 *            i.e. value constraints from the smoothed slice s = I1_j and gradient constraints
 *            from the original slice o = I0_j ("Screened-Poisson Blending"), solved by
 *            multigrid ("Implementation").
 *
 * Conventions shared by every entry point
 *   - Layout: a stack is [z][y][x], x fastest.  A slice is [y][x].  Sizes are in elements.
 *   - Discretisation: Lap is the 5-point graph Laplacian with Neumann (no-flux) boundaries
 *     and unit pixel spacing; Gaussian taps are exp(-d^2 / 2 sigma^2) for integer
 *     |d| <= floor(3 sigma), renormalised over the taps that fall inside the stack.
 *   - Ownership: the caller owns every buffer passed in.  The library owns its device
 *     workspace: per-call temporaries come stream-ordered from its own memory pool and go back
 *     to the pool by the end of the call; solver plans (multigrid pyramids, FP64 iterates,
 *     tensor maps, captured graphs) are kept between calls for reuse, see
 *     emfuse_release_cache().
 *   - Pointers are device pointers unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Errors: every call returns an emfuse_status; it never aborts.  On error a message is
 *     available from emfuse_last_error() (per host thread).  Invalid arguments are
 *     detected before any work is queued.
 *   - Solves (screened_poisson, fuse_color, correct_stack, backward): the whole outer loop
 *     of the solve (residual, convergence check, V-cycle, ...) runs on the device, as one
 *     CUDA graph whose loop is a conditional WHILE node (a per-slice check kernel decides
 *     after every residual pass).  By default the call then waits for the stream and returns
 *     the outcome (EMFUSE_OK / EMFUSE_ENOCONV ...) with outputs and stats complete; with
 *     opts.async_solve = 1 it returns at once and stats are valid after a stream
 *     synchronisation (see emfuse_solve_opts).
 */
#ifndef EMFUSE_H
#define EMFUSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { EMFUSE_U8 = 0, EMFUSE_F32 = 1 } emfuse_dtype;

typedef enum {
    EMFUSE_OK = 0,
    EMFUSE_EINVAL = 1,    /* bad argument (null pointer, size < 1, alpha <= 0, sigma < 0 ...) */
    EMFUSE_ECUDA = 2,     /* a CUDA call failed; see emfuse_last_error()                     */
    EMFUSE_ENOMEM = 3,    /* device workspace could not be allocated                         */
    EMFUSE_ENOCONV = 4,   /* tol not reached in max_vcycles; outputs hold the last iterate   */
    EMFUSE_ETIMEOUT = 5   /* a bounded device-side wait expired                             */
} emfuse_status;

typedef enum {
    EMFUSE_PREC_FP32 = 0,   /* everything in FP32 (iterate, residual, V-cycles)               */
    EMFUSE_PREC_MIXED = 1,  /* FP32 V-cycles inside FP64 defect correction (default)          */
    EMFUSE_PREC_FP64 = 2    /* everything in FP64                                             */
} emfuse_precision;

/* Solver options.  Fill with emfuse_default_opts() and override fields. */
typedef struct {
    double tol;          /* stop when every slice has ||b - A f||_2 / ||b||_2 <= tol,
                            b = alpha s + L o, A = alpha I + L (residual measure of the
                            solver table in Sec. 4).  Default 1e-6.  The error it bounds is
                            ||f - f*|| <= cond(A) tol ||f*||, cond(A) = 1 + 8 / alpha
                            (8001 at alpha = 0.001): on smooth EM-like slices tol 1e-6
                            keeps max |f - f*| well inside 1e-4 of the 8-bit range, on rough
                            (noise-like) slices at small alpha it may not, and a smaller
                            tol (1e-8 .. 1e-10, mixed or FP64 precision) is needed.     */
    int max_vcycles;     /* maximum outer iterations (one V-cycle each).  Default 40.      */
    int nu_pre;          /* red-black Gauss-Seidel sweeps before restriction.  Default 2.  */
    int nu_post;         /* sweeps after prolongation.  Default 2.                         */
    int precision;       /* emfuse_precision.  Default EMFUSE_PREC_MIXED.  EMFUSE_PREC_FP32
                            keeps the iterate in FP32: it meets 1e-4 of the 8-bit range at
                            alpha >= 0.01, but at alpha = 0.001 its rounding reaches the
                            smooth error modes amplified by ~1/alpha (about 4e-4 of the
                            range), and it cannot reach tol below ~1e-6.                   */
    int fused;           /* 1: fused wavefront kernels on large levels (nu_pre in 1..3,
                            nu_post in 1..4: the strips overlap by 8 cells; other counts run
                            the reference schedule); 0: one kernel per half-sweep
                            (reference schedule).  Default 1.                              */
    int first_vcycles;   /* V-cycles in the first outer iteration (the second continues from
                            the first's correction in FP32 before the first FP64 residual).
                            0 = default (2).                                               */
    int tile_rows;       /* rows of one work item (a 128-column strip) of the fused kernels
                            on the finest level: 0 = chosen from the batch size, else a
                            power of two in [8, 256].                                      */
    int autotune;        /* 1: before solving, time complete solves of this batch for
                            tile_rows in {32, 64, 128, 256} (with nu = (2, 2)), then for
                            (nu_pre, nu_post) in {(1,1), (1,2), (2,1), (2,3), (3,2), (3,3),
                            (3,4), (4,4)} with each of the two fastest tile_rows (fused
                            schedule; nu_pre = 4 runs its DOWN leg in the reference
                            schedule), keep the fastest for this batch geometry, alpha,
                            precision and tol, and solve with it (20 candidates, see
                            emfuse_autotune_result).  Default 0.                           */
    int no_graphs;       /* 1: launch every V-cycle kernel directly instead of replaying
                            the V-cycle as a captured CUDA graph.  Default 0.              */
    float robust_kappa;  /* emfuse_correct_stack only: > 0 smooths with robust averaging
                            across slices at this threshold (see emfuse_smooth_z_robust;
                            the paper uses 2); 0 = plain averaging.  Default 0.            */
    int host_pipeline;   /* emfuse_correct_stack with host buffers: 0 = choose (the whole
                            input and its smoothed copy on the device when they fit, else
                            slabs with halo planes), 1 = slabs, 2 = whole input (EMFUSE_ENOMEM
                            if it does not fit).  Default 0.                               */
    int verify_residual; /* 1: after the solve, recompute every slice's relative residual
                            with a separate plain FP64 kernel (b = alpha s + L o formed
                            directly, every operation and sum in FP64) on the solver's final
                            iterate and report it in stats.rel_residual_check: a check of
                            the reported rel_residual, whose kernel rounds A d to FP32 and
                            sums squares in FP32 per warp.  One extra pass.  Default 0.   */
    int async_solve;     /* 1: the solve is only queued on `stream` and the call returns at
                            once (emfuse_screened_poisson, emfuse_fuse_color,
                            emfuse_correct_stack on device buffers; ignored by the host-
                            buffer path and emfuse_backward, which complete): stats are
                            written by a stream callback and valid once the stream has
                            reached this point (after a stream or event synchronisation);
                            the return value reports argument and launch errors only, the
                            outcome is stats[j].converged (0 for a slice that missed tol or
                            had a non-finite residual).  Needs the graph path (fused = 1,
                            no_graphs = 0); otherwise, and while the library records
                            per-launch events, the call completes before it returns, as
                            with 0.  Default 0.                                           */
    int host_chunk;      /* emfuse_correct_stack with host buffers: slices per chunk of the
                            copy / compute pipeline; 0 = chosen (four chunks when the whole
                            input fits on the device, else as many slices as memory allows,
                            at most 64).  Default 0.                                      */
} emfuse_solve_opts;

/* Per-slice result of a solve. */
typedef struct {
    int vcycles;          /* V-cycles applied to this slice                                */
    int converged;        /* 1 if rel_residual <= tol                                      */
    double rel_residual;  /* final ||b - A f||_2 / ||b||_2, computed on the GPU              */
    double b_norm;        /* ||b||_2                                                        */
    double rel_residual_check;  /* opts.verify_residual = 1: the same measure recomputed in
                                   plain FP64 on the final iterate; else -1                  */
} emfuse_slice_stats;

/* Fill `opts` with the defaults listed above. */
void emfuse_default_opts(emfuse_solve_opts* opts);

/*
 * Phase 1: I1 = I0 * G_{sigma_xy, sigma_z}  (Sec. 3 "Anisotropic Smoothing"; truncation at
 * three standard deviations, Sec. 3 "Implementation").
 *
 *   in      device, nz planes of ny rows, row pitch `pitch` elements (>= nx), dtype `dt`
 *           (uint8 or float32).
 *   out     device float32, (z1 - z0) planes with the same row pitch; plane i holds output
 *           slice z0 + i.
 *   z0, z1  output plane range, 0 <= z0 < z1 <= nz.  Every input plane is used as context,
 *           so a z-slab with floor(3 sigma_z) halo planes on each side gives exactly the
 *           slices of the whole stack (Sec. 3 "Distributed Processing").
 *   sigma_xy, sigma_z >= 0 (0 = no smoothing along that axis).
 *
 * Weights are renormalised over in-stack taps at stack ends and slice edges.
 * Asynchronous on `stream`.
 */
int emfuse_smooth_z(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                    int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                    void* stream);

/*
 * Phase 1 with robust averaging across slices (Sec. 3, the outlier example of the figure on
 * missing data: only colour values within two standard deviations are averaged).  As
 * emfuse_smooth_z, except along z: for every voxel the in-stack taps |d| <= floor(3 sigma_z)
 * with weights w_d and xy-smoothed values v_d give the weighted mean mu and variance var;
 * samples with (v_d - mu)^2 > kappa^2 var are left out and the rest averaged with their
 * weights renormalised.  kappa >= 1 (the paper: 2).  Needs floor(3 sigma_xy) <= 8 and
 * floor(3 sigma_z) <= 9 (else EMFUSE_EINVAL).  Asynchronous on `stream`.
 */
int emfuse_smooth_z_robust(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                           int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                           float kappa, void* stream);

/*
 * Allocation-free smoothing.  The paper has no counterpart: this is a deployment variant of
 * emfuse_smooth_z for callers that cannot allocate device memory while they run (a host whose
 * device memory all belongs to its own pool or a fixed budget, or a latency-critical loop in
 * which cudaMalloc / cudaFree would synchronise the device).
 *
 * Same arguments, layout and result as emfuse_smooth_z (within float rounding: it always runs
 * the plain-load fused kernel).  Its only scratch, the per-axis normaliser tables, lives in a
 * static device array of 3 * 32768 floats (384 KiB) that every GPU loading this library holds
 * until the process exits; a small kernel fills the tables on `stream` from the Gaussian taps,
 * so the call reads no host buffer.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 *   Limits: nx + ny + nz <= 98304, floor(3 sigma_xy) <= 8, floor(3 sigma_z) <= 9; beyond
 *           them it returns EMFUSE_EINVAL with a message naming the limit.
 *   Set-up: the first call on each device looks up the array's device address (with that
 *           device current).  Make that first call before capturing any stream into a graph.
 *   Sharing: all calls share the one array, and each call rewrites the whole table it reads,
 *           stream-ordered on `stream`.  Calls that can overlap on the GPU (different streams
 *           without ordering between them, or different host threads) race on it.
 * Asynchronous on `stream`.
 */
int emfuse_smooth_z_noalloc(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                            int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                            void* stream);

/*
 * Phase 2: per-slice screened-Poisson solve, Eq. (1): (alpha I + L) f_j = alpha s_j + L o_j
 * (Sec. 3 "Screened-Poisson Blending"), by multigrid V-cycles (Sec. 3 "Implementation").
 *
 *   s, o, f   device float32, a ragged batch of `nslices` dense slices packed in one buffer:
 *             slice j has ny[j] rows of nx[j] elements starting at element offsets[j].
 *             f may not alias s or o.
 *   nx, ny, offsets   HOST arrays of length nslices.
 *   alpha     screening weight, > 0.
 *   opts      NULL = defaults.
 *   stats     NULL or a HOST array of nslices entries, filled on return.
 *
 * Initial iterate f = o.  Returns EMFUSE_ENOCONV (with f = last iterate) when some slice
 * misses opts->tol after opts->max_vcycles V-cycles.
 */
int emfuse_screened_poisson(const float* s, const float* o, float* f, int64_t nslices,
                            const int64_t* nx, const int64_t* ny, const int64_t* offsets,
                            double alpha, const emfuse_solve_opts* opts,
                            emfuse_slice_stats* stats, void* stream);

/*
 * Table of the last autotuning run on this host thread (opts.autotune = 1): one entry per
 * candidate schedule, the chosen one first.  Not in the paper: its multigrid has no tunable
 * schedule.  Writes min(count, max_entries) entries to the HOST array `out` (may be NULL)
 * and returns count (0 if this thread has not autotuned).
 */
typedef struct {
    int nu_pre, nu_post, tile_rows;
    int vcycles;          /* V-cycles the batch needed with this schedule (max over slices) */
    double ms;            /* time of the complete solve (CUDA events); -1 if it missed tol  */
} emfuse_tune_entry;
int emfuse_autotune_result(emfuse_tune_entry* out, int max_entries);

/*
 * Direct solve of Eq. (1) by fast Fourier transforms: the frequency-space form of Sec. 3
 * ("Frequency-Space Interpretation"; the FFT solver that Sec. 3 "Alternate Solutions" weighs
 * against multigrid), as an exact second solver to compare the multigrid against.  For every
 * slice, f = o + d with d = alpha A^{-1} (s - o) computed on the mirror extension of the slice
 * to 2ny x 2nx (whose periodic Laplacian is the Neumann one of the slice) by one batched
 * real-to-complex FFT, a per-frequency scaling by alpha / (alpha + lambda), and one inverse FFT
 * (cuFFT).
 *   s, o, f     device float32, nslices dense slices of ny x nx (uniform batch).
 *   precision   EMFUSE_PREC_FP32 or EMFUSE_PREC_FP64 (transforms and scaling in that type).
 * Temporaries: the extended slices and their spectra (about 4 and 4 times the slices, in the
 * chosen type), from the library's pool; cuFFT plans are cached per size, batch and precision
 * until emfuse_release_cache().  Asynchronous on `stream`.
 */
int emfuse_screened_poisson_dct(const float* s, const float* o, float* f, int64_t nslices, int64_t nx,
                                int64_t ny, double alpha, int precision, void* stream);

/*
 * Phase 1 as the 3-D gradient-domain problem of the earlier method (Sec. 3 "Alternate
 * Solutions": the target gradient field is the input's gradient with its z-components set to
 * zero), with the screening of Eq. (1):
 *     out = argmin_f  alpha |f - in|^2 + |grad_xy f - grad_xy in|^2 + |d_z f|^2
 * on the 6-neighbour graph of the stack with Neumann boundaries, i.e.
 * (alpha I + L_xy + L_z) out = alpha in + L_xy in.  Solved exactly: out = in + d.  The
 * orthonormal DCT-II along z (a dense nz x nz matrix applied to every pixel column, cuBLAS
 * GEMM) diagonalises L_z, which splits the problem into nz slice problems
 * (alpha + lambda_z[k]) d_k + L_xy d_k = -lambda_z[k] I_k; those are solved at once by the
 * batched mirror-extension FFT of emfuse_screened_poisson_dct, and the inverse z transform
 * (GEMM) gives d.
 *   in          device, nz x ny x nx dense [z][y][x], uint8 (dt = EMFUSE_U8) or float32.
 *   out         device float32, same shape; must not alias in.
 *   alpha       > 0 (finite).
 *   precision   EMFUSE_PREC_FP32 or EMFUSE_PREC_FP64 (transforms and scaling in that type).
 * Temporaries: two copies of the stack, its mirror extension and half spectrum (about 10
 * times the stack's cells in the chosen type) plus cuFFT's work area, from the library's pool;
 * EMFUSE_ENOMEM when they do not fit.  The cuFFT plan (per shape and precision) and the
 * cuBLAS handle are cached until emfuse_release_cache().  Asynchronous on `stream`.
 */
int emfuse_smooth_gradient_domain(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                  double alpha, int precision, void* stream);

/*
 * The same problem as emfuse_smooth_gradient_domain, solved by multigrid on the stack, as the
 * paper's earlier method did (Sec. 3 "Alternate Solutions"), instead of by transforms:
 * correction form out = in + d with (alpha I + L) d = -L_z in; V-cycles in FP32 on the 3-D
 * grid (cell-centred coarsening to 1 x 1 x 1, finite-volume operators on the true cells,
 * restriction by child sum / 8, trilinear prolongation, red-black Gauss-Seidel with
 * opts->nu_pre / nu_post sweeps; opts->first_vcycles FP32 cycles before the first FP64 pass);
 * after every V-cycle an FP64 pass forms d += e and r = -L_z in - A d (A d in FP64, rounded
 * once to FP32 before the subtraction from the FP32-formed -L_z in; everything in FP64 when
 * opts->tol < 1e-7) and writes out = in + d, until ||r|| / ||alpha in + L_xy in|| <= opts->tol
 * or opts->max_vcycles V-cycles.  The host reads the residual norm after every pass (the call
 * returns when out is final).  Other opts fields are ignored.
 *   in      device, nz x ny x nx dense [z][y][x], uint8 (dt = EMFUSE_U8) or float32.
 *   out     device float32, same shape; must not alias in.
 *   alpha   > 0 (finite).
 *   opts    NULL = defaults.
 *   stats   NULL or ONE host entry for the whole stack (vcycles, converged, rel_residual,
 *           b_norm; rel_residual_check = -1).
 * Temporaries (from the library's pool): the level pyramid (u and b, about 9 B per cell) and
 * the FP64 correction (8 B per cell).  Errors: EMFUSE_EINVAL (arguments; a NaN or Inf in `in`),
 * EMFUSE_ENOMEM, EMFUSE_ENOCONV (tol not reached; out holds the last iterate).
 */
int emfuse_smooth_gradient_domain_mg(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                     double alpha, const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                                     void* stream);

/*
 * Fusion of low-frequency colour images with high-frequency monochrome ones (Sec. 3, the
 * colour example): for every image i and colour channel c, Eq. (1) with the colour channel as
 * the value constraint and the grey image as the gradient constraint,
 *     (alpha I + L) f_{i,c} = alpha s_{i,c} + L o_i,
 * solved as one batch of 3 * nimages slices.
 *   s_rgb, f_rgb  device float32, planar: image i channel c is the ny x nx plane 3 i + c.
 *   o_grey        device float32, one ny x nx plane per image.
 *   stats         NULL or a HOST array of 3 * nimages entries (plane order).
 * Allocates a temporary copy of o_grey per channel (3 * nimages planes) on `stream`.
 */
int emfuse_fuse_color(const float* s_rgb, const float* o_grey, float* f_rgb, int64_t nimages, int64_t nx,
                      int64_t ny, double alpha, const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                      void* stream);

/*
 * Both phases on a stack: s = smooth(I0), then f_j = solve(s_j, o_j = I0_j) for every j.
 *
 *   in        I0, nz x ny x nx dense, dtype `dt`.
 *   out       I2, float32, same shape.
 *   in_is_host  0: `in` and `out` are device pointers.
 *               1: `in` and `out` are HOST pointers (page-locked memory is strongly
 *                  recommended); copies overlap compute on side streams, and the call returns
 *                  when `out` is written.  When the input and its smoothed copy fit on the
 *                  device, the input arrives in pieces, and each chunk of slices (four chunks
 *                  unless opts->host_chunk says otherwise) is smoothed and solved as soon as
 *                  its planes are there, its solve queued without the host waiting, and its
 *                  result copied back while the next chunks compute; otherwise the stack
 *                  streams through in z-slabs with floor(3 sigma_z) halo planes, so stacks
 *                  larger than device memory are supported (opts->host_pipeline chooses
 *                  explicitly).  The result equals the device path's bit for bit.
 *   stats     NULL or a HOST array of nz entries.
 */
int emfuse_correct_stack(const void* in, int dt, int in_is_host, float* out, int64_t nx,
                         int64_t ny, int64_t nz, float sigma_xy, float sigma_z, double alpha,
                         const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                         void* stream);

/*
 * Adjoint of emfuse_correct_stack / emfuse_screened_poisson on a dense stack of nz slices
 * of ny x nx.  With A = alpha I + L symmetric and lam_j = A^{-1} grad_f_j (solved by the same
 * multigrid), for a loss l with dl/df = grad_f:
 *     dl/ds      = alpha lam
 *     dl/do      = L lam
 *     dl/dalpha  = sum_j <lam_j, s_j - f_j>
 *     dl/dI0     = L lam + K^T (alpha lam)        (s = K I0, o = I0; K the phase-1 smoothing)
 *     dl/dsigma_z = <alpha lam, (dK/dsigma_z) I0>  (support radius held at floor(3 sigma_z))
 *
 *   grad_f, f, s   device float32 (f and s as produced by the forward call).
 *   o              device I0, dtype `dt`.
 *   grad_s, grad_o, grad_in0   device float32 outputs, each may be NULL (not computed).
 *   grad_alpha, grad_sigma_z   HOST double outputs, each may be NULL.
 *   grad_in0 / grad_sigma_z need sigma_xy, sigma_z (the forward smoothing).
 */
int emfuse_backward(const float* grad_f, const float* f, const float* s, const void* o, int dt,
                    int64_t nx, int64_t ny, int64_t nz, float sigma_xy, float sigma_z,
                    double alpha, float* grad_s, float* grad_o, float* grad_in0,
                    double* grad_alpha, double* grad_sigma_z, const emfuse_solve_opts* opts,
                    void* stream);

/*
 * Instrumentation (no counterpart in the paper).
 *
 * emfuse_kernel_launches(): number of kernels this library has launched in this process.
 * emfuse_profile_begin(): start recording a CUDA event pair around every kernel launch of
 *   the library, on the stream the kernel is launched on, together with the algorithmic
 *   bytes of the launch: every input element the kernel's function needs read once and
 *   every output element written once (counted at each launch site).  Adds two event
 *   records per launch.
 * emfuse_profile_end(): stop recording, wait for the recorded events, and fill up to
 *   `max_entries` per-kernel totals (sorted by total time, descending).  Returns the number
 *   of kernel names recorded (which may exceed max_entries), or -1 on a CUDA error.
 */
typedef struct {
    char name[48];           /* kernel family, e.g. "relax_l0" */
    int64_t launches;
    double total_ms;         /* sum of event-measured launch durations */
    double bytes;            /* sum of algorithmic bytes over the launches */
    double fp64_flops;       /* sum of algorithmic FP64 flops (add = 1, fma = 2), if any */
} emfuse_kernel_profile;

uint64_t emfuse_kernel_launches(void);
void emfuse_profile_begin(void);
int emfuse_profile_end(emfuse_kernel_profile* out, int max_entries);

/*
 * Solver plans (descriptor tables, TMA tensor maps, multigrid pyramids and the FP64 iterate)
 * are kept between calls, one per (device, stream, precision), and reused while the slice
 * geometry and schedule options stay the same.  Per-call temporaries come from a memory pool
 * of the library's own (one per device) that keeps freed pages mapped for the next call.
 * emfuse_release_cache() frees the plans and returns the pool's unused pages (plans are rebuilt
 * by the next solve).  It synchronises the device and must not be called while
 * another host thread is inside a solve.
 */
void emfuse_release_cache(void);

/*
 * Self-test of the integer-pipe binary32 <-> binary64 conversions used by the FP64 residual
 * kernels (no counterpart in the paper: an implementation check).  Runs on the current device,
 * synchronously: every binary32 bit pattern is widened and compared with the hardware
 * conversion, and 7 x 2^32 binary64 values (rounding-critical low bits around every binary32
 * value, plus pseudo-random bit patterns) are rounded and compared.  Writes the mismatch
 * counts (0 and 0 expected; NaNs match any NaN) to the two HOST pointers.  Allocates and frees
 * 16 bytes of device memory.  Takes well under a second on one GPU.
 */
int emfuse_selftest_fpconv(int64_t* f2d_mismatches, int64_t* d2f_mismatches);

/*
 * Self-test of the bounded device waits (no counterpart in the paper: failure handling).  The
 * library's kernels never wait without a bound: a wait on a shared-memory barrier that does not
 * complete within its poll limit sets a per-device error word and the kernel returns, and the
 * host call reports EMFUSE_ETIMEOUT with the context still usable.  This call launches one warp
 * that waits, with at most `limit` polls (1 .. 2^20), on a barrier that nothing completes, on
 * `stream`, synchronously; it returns EMFUSE_ETIMEOUT (the expected outcome) and clears the
 * error word, or EMFUSE_EINVAL for a limit out of range.
 */
int emfuse_selftest_wait_timeout(int limit, void* stream);

/*
 * Architecture check (no counterpart in the paper): writes the binary version of the library's
 * device code as loaded on the current device (major * 10 + minor, 103 for sm_103a) to the
 * HOST int `binary_version`.  EMFUSE_ECUDA if the code cannot run on this device.
 */
int emfuse_kernel_binary_version(int* binary_version);

/*
 * FP64 roofline probe (no counterpart in the paper: measurement).  Times, with CUDA events on
 * `stream`, a kernel of independent FP64 fused multiply-add chains filling every SM (8 chains
 * per thread, 8 CTAs of 256 threads per SM), best of three launches after a warm-up, and
 * writes the achieved FP64 rate in TFLOP/s (an FMA counts 2 flops) to the HOST double
 * `tflops`.  Synchronous; allocates nothing; takes a few milliseconds.
 */
int emfuse_probe_fp64_fma_rate(double* tflops, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* emfuse_last_error(void);

/* Library version string. */
const char* emfuse_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EMFUSE_H */
