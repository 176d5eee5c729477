/*
 * fewsum.h -- C ABI of libfewsum.so: GB300-native interpolated EMRI mode summation.
 *
 * The library computes the Schwarzschild-eccentric waveform of arXiv:2104.04582 Sec. 4,
 *
 *     h(t) = h_+ - i h_x = (mu/d_L) sum_{l,m,n} A_lmn(t) -2Y_lm(theta, phi) exp(-i Phi_mn(t)),
 *     Phi_mn(t) = m Phi_phi(t) + n Phi_r(t),
 *
 * by the "interpolated summation" of Sec. 3.C: the orbital phases Phi_phi, Phi_r and every
 * selected mode's complex amplitude A_lmn are given on a sparse trajectory grid t_0 < ... <
 * t_{K-1}; each real array is fitted with a not-a-knot cubic spline on that shared grid, and
 * the mode sum is evaluated at every dense sample t_i = t0 + i*dt.  Only modes with m >= 0 are
 * passed in; the m < 0 modes follow from Eq. (amp_symmetry) with k = 0,
 * A_{l,-m,-n} = (-1)^l conj(A_lmn), and are added for m > 0 only (an m = 0 mode of the list is
 * used as given; (l,0,n) and (l,0,-n) are distinct entries of the paper's 3843-mode grid).
 *
 * Everything between the inputs and h runs in this library's CUDA kernels on one GPU:
 * the batched spline build, the spin-weighted harmonics, the per-request fold of harmonics
 * into the spline coefficients, and the per-sample evaluation and mode sum.
 *
 * Conventions shared by every call
 * --------------------------------
 * Errors: every call returns a few_status; nothing throws or aborts across the ABI.  Inputs are
 *   validated on the host before any work is queued; on a validation error nothing is queued
 *   and no output is touched.  Problems that can only be seen on the device (a NaN in
 *   device-resident inputs, a bounded wait that expired) latch into the context and are
 *   returned by few_sync_status().  A CUDA runtime error is returned as FEW_ERR_CUDA.
 * Ownership: the caller owns every pointer it passes (host or device) and may free or reuse
 *   host input memory as soon as the call returns.  Device inputs and outputs must stay valid
 *   until the work queued on the given stream has completed.  The library owns the context,
 *   trajectory and batch handles and all memory they hold.
 * Streams: calls that take a `stream` (a cudaStream_t passed as void*; NULL = the legacy
 *   default stream) queue their device work on it and return without waiting, unless
 *   documented otherwise.  Work on one handle from several streams must be ordered by the
 *   caller.
 * Threads: a context may be used from several host threads; every call on a context takes
 *   the context's lock while it plans and queues work, and releases it before a wait for its
 *   own host copies or host output (few_traj_set_data from host memory, few_waveform into host
 *   memory), so calls from threads with their own handles and streams overlap.
 * Layouts: complex outputs are interleaved (re, im) pairs, complex128 (2 x f64) or
 *   complex64 (2 x f32).  Per-knot mode arrays are row-major [K][N] (modes contiguous).
 * Limits: 4 <= K <= FEW_MAX_KNOTS knots; 1 <= N modes; 2 <= l <= 32, 0 <= m <= l,
 *   |n| <= 1024, no duplicate (l,m,n); n_samples <= 2^31 - 1.  The per-segment harmonic table
 *   (see few_mode_slots) streams through shared memory in tiles, so its size is not limited.
 */
#ifndef FEWSUM_H
#define FEWSUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEW_ABI_VERSION 4

typedef enum few_status {
    FEW_OK = 0,
    FEW_ERR_INVALID_ARG = 1, /* null pointer, bad enum, non-finite scalar, NaN in device data */
    FEW_ERR_KNOTS = 2,       /* K < 4, knots not strictly increasing or not finite */
    FEW_ERR_MODES = 3,       /* N < 1, l < 2, m < 0, m > l, |n| > 1024, duplicate (l,m,n) */
    FEW_ERR_RANGE = 4,       /* samples outside [t_0, t_{K-1}], dt <= 0, n_samples too big */
    FEW_ERR_NOMEM = 5,       /* device or host allocation failed */
    FEW_ERR_BUDGET = 6,      /* the call would exceed the context's HBM budget */
    FEW_ERR_CUDA = 7,        /* a CUDA runtime call failed */
    FEW_ERR_TIMEOUT = 8,     /* a bounded device-side wait expired (latched) */
    FEW_ERR_LIMIT = 9,       /* a size exceeds an on-chip limit of the kernels */
    FEW_ERR_STATE = 10       /* handle used in the wrong state (e.g. no data set) */
} few_status;

typedef enum few_precision {
    FEW_FP64 = 0,  /* plain path: every step in FP64 */
    FEW_MIXED = 1  /* FP64 phase splines + mod-2pi reduction; FP32 amplitudes, exponentials, sum */
} few_precision;

typedef enum few_mem {
    FEW_MEM_HOST = 0,   /* pointer is host memory (pageable or pinned) */
    FEW_MEM_DEVICE = 1  /* pointer is device memory of the context's GPU */
} few_mem;

typedef enum few_frame {
    FEW_FRAME_SOURCE = 0,  /* (theta, phi) are the source-frame viewing angles */
    FEW_FRAME_SSB = 1      /* (theta, phi) = sky position (theta_S, phi_S) and (theta_K, phi_K)
                              the spin direction; the output is in the detector frame (Sec. 2.A) */
} few_frame;

typedef struct few_ctx few_ctx;
typedef struct few_traj few_traj;
typedef struct few_batch few_batch;
typedef struct few_basis few_basis;

/* Human-readable name of a status code (static string, never NULL). */
const char *few_strerror(few_status s);

/* Library ABI version (FEW_ABI_VERSION of the build). */
int few_abi_version(void);

/*
 * Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the device memory the
 * library may hold at once for this context (trajectories, per-call scratch, staging); 0 means
 * no cap beyond the device's free memory.  Allocations go through a stream-ordered pool owned
 * by the context.  Blocking.
 */
few_status few_ctx_create(few_ctx **out, int device, size_t hbm_budget_bytes);

/* Wait for the device, free everything the context owns (including live trajectories and
 * batches), and destroy it.  NULL is accepted. */
few_status few_ctx_destroy(few_ctx *ctx);

/* Bytes of device memory the context currently holds (allocated by the library). */
few_status few_ctx_memory(few_ctx *ctx, size_t *bytes_in_use, size_t *budget_bytes);

/*
 * Create a trajectory: the knot grid and the mode list (Sec. 3.C: all splines share one knot
 * grid; Sec. 4: the (l,m,n) mode set with m >= 0).
 *   t_knots [K]: strictly increasing finite times (s), host memory, copied.
 *   l, m, n [N]: mode indices, host memory, copied.
 * Plans the shared tridiagonal factorization on the device (one launch on an internal stream)
 * and waits for it.  Spline data are set with few_traj_set_data before first use.
 * Errors: FEW_ERR_KNOTS, FEW_ERR_MODES, FEW_ERR_LIMIT (K > FEW_MAX_KNOTS), FEW_ERR_BUDGET,
 * FEW_ERR_NOMEM, FEW_ERR_CUDA.
 */
few_status few_traj_create(few_ctx *ctx, const double *t_knots, int K, const int *l, const int *m,
                           const int *n, int N, few_traj **out);

/*
 * Set the values on the trajectory grid and build every spline (Sec. 3.C: batched not-a-knot
 * cubic splines for both phases and for the real and imaginary part of every amplitude; one
 * tridiagonal solve per spline, all sharing the knot matrix).
 *   phi_phi, phi_r [K]: orbital phases (rad) at the knots.
 *   amp_re, amp_im [K][N]: Re and Im of A_lmn at the knots, row-major, modes contiguous.
 *   where: FEW_MEM_HOST (copied to the device first; the copy is ordered on `stream` and the
 *          host arrays may be reused when the call returns) or FEW_MEM_DEVICE (read in place by
 *          the build kernel; must stay valid until the work on `stream` completes).
 * Asynchronous on `stream`.  Non-finite values are detected on the device and latched as
 * FEW_ERR_INVALID_ARG (see few_sync_status).
 */
few_status few_traj_set_data(few_ctx *ctx, few_traj *traj, const double *phi_phi,
                             const double *phi_r, const double *amp_re, const double *amp_im,
                             few_mem where, void *stream);

/* Release a trajectory and its device memory (after the device is idle on its work). */
few_status few_traj_release(few_ctx *ctx, few_traj *traj);

/* Knot count, mode count and harmonic slots per segment of a trajectory. */
few_status few_traj_info(const few_traj *traj, int *K, int *N, int *n_slots);

/*
 * One waveform request.  Output sample i (0 <= i < n_samples) is h(t0 + i*dt), Sec. 4 sum.
 *   theta, phi: source-frame viewing angles (rad) of -2Y_lm when frame == FEW_FRAME_SOURCE.
 *   frame == FEW_FRAME_SSB (Sec. 2.A): theta, phi are the sky position (theta_S, phi_S) and
 *     theta_K, phi_K the spin direction, both in the solar-system-barycentre frame.  The library
 *     derives the source-frame angles (cos theta_src = -R.S, phi_src = -pi/2, from the paper's
 *     source-frame basis) and the polarization angle psi (tan psi = (cos tS sin tK cos(pS - pK)
 *     - sin tS cos tK) / (sin tK sin(pS - pK))), applies the pi/2 basis rotation (a phase shift
 *     of pi) and the rotation by 2 psi: h_ssb = -e^{-2 i psi} h_src.  R parallel to S is
 *     rejected (FEW_ERR_INVALID_ARG).
 *   scale: the real prefactor mu/d_L (1 for the dimensionless sum).
 *   dphi_phi0, dphi_r0: constant offsets (rad) added to Phi_phi and Phi_r -- a change of the
 *     initial phases Phi_phi,0 and Phi_r,0 without rebuilding the splines.
 *   t0, dt: first sample time and cadence (s); every sample must lie in [t_0, t_{K-1}].
 *   prec: FEW_FP64 or FEW_MIXED.
 *   out: n_samples complex values, complex64 if out_c64 else complex128; device memory if
 *     out_where == FEW_MEM_DEVICE, else host memory: page-locked host memory (cudaHostAlloc,
 *     cudaHostRegister) is written directly by the summation kernel, pageable memory is staged
 *     on the device and copied back on `stream`; either way few_waveform returns once the
 *     result is in host memory.
 */
typedef struct few_request {
    const few_traj *traj;
    double theta, phi;
    double scale;
    double dphi_phi0, dphi_r0;
    double t0, dt;
    int64_t n_samples;
    int prec;       /* few_precision */
    int out_c64;    /* 1: complex64 output, 0: complex128 output */
    int out_where;  /* few_mem of `out` */
    int frame;      /* few_frame */
    void *out;
    double theta_K, phi_K;  /* spin direction, used when frame == FEW_FRAME_SSB */
} few_request;

/*
 * Compute one waveform (Sec. 3.C interpolated summation of the Sec. 4 sum).  Validates and
 * plans on the host, then queues the harmonic, fold and summation kernels on `stream`.
 * n_samples == 0 is a no-op.  Errors: FEW_ERR_INVALID_ARG, FEW_ERR_STATE, FEW_ERR_RANGE,
 * FEW_ERR_LIMIT, FEW_ERR_BUDGET, FEW_ERR_NOMEM, FEW_ERR_CUDA.
 */
few_status few_waveform(few_ctx *ctx, const few_request *req, void *stream);

/*
 * Allocation-free variant of few_waveform.  The paper has no counterpart: this entry point is
 * for callers that must not allocate memory once they are running -- e.g. a sampler or a
 * real-time pipeline that reserves all device memory at start-up, or code under a policy that
 * forbids cudaMalloc (and the synchronisation it can imply) on the call path.  It computes
 * what few_waveform computes for the same request (either frame), but keeps its scratch (plan,
 * harmonic table, folded coefficients and, for FEW_MIXED, the phase anchors) in one fixed device
 * array of FEW_NOALLOC_SCRATCH_BYTES that is part of the library image (reserved on every GPU
 * that loads the library, until the process exits) and calls no allocator of any kind.
 *   req->out_where must be FEW_MEM_DEVICE; the trajectory and the output buffer are the
 *   caller's, as for few_waveform.
 * Limits: the request's scratch must fit in FEW_NOALLOC_SCRATCH_BYTES and K <= 4096; otherwise
 *   it returns FEW_ERR_LIMIT without queuing work.  The scratch is about 64 x slots x (K - 1)
 *   bytes for FEW_FP64; for FEW_MIXED 32 x slots x (K - 1) bytes plus 3 bytes per output sample
 *   (the phase anchors), plus a few KB.  The one-year 3843-mode waveform (K = 100,
 *   3,155,760 samples) fits in both precisions; the four-year one at dt = 2 s does not.
 * The first call made on a device looks up the array's device address (once per device);
 *   make that first call before any stream capture.  All calls share the array: every call
 *   rewrites what it uses, but calls whose work overlaps on the GPU race on it -- order them
 *   (one stream, or events).  Asynchronous on `stream`; the caller's current device is
 *   restored on return.
 */
#define FEW_NOALLOC_SCRATCH_BYTES (16u << 20)
#define FEW_MAX_BASIS 256  /* reduced-basis size limit of few_basis_create */
#define FEW_MAX_KNOTS 4096 /* knots per trajectory (the spline build stages 48 bytes per knot) */
few_status few_waveform_noalloc(few_ctx *ctx, const few_request *req, void *stream);

/*
 * The per-sample phase step on its own (Sec. 2 phase integrals, interpolated as in Sec. 3.C):
 * for sample i, t_i = t0 + i*dt, writes the orbital phases Phi_phi(t_i) + dphi_phi0 and
 * Phi_r(t_i) + dphi_r0 reduced modulo 2 pi and expressed in turns, each in [-1/2, 1/2]:
 * out_dev[2i] = f_phi, out_dev[2i+1] = f_r (device memory, n_samples x 2 doubles).  The same
 * FP64 evaluation and reduction feed both summation paths.  Asynchronous on `stream`.
 * Errors: as few_waveform (FEW_ERR_STATE, FEW_ERR_RANGE, FEW_ERR_INVALID_ARG, ...).
 */
few_status few_phase_samples(few_ctx *ctx, const few_traj *traj, double t0, double dt,
                             int64_t n_samples, double dphi_phi0, double dphi_r0, double *out_dev,
                             void *stream);

/*
 * Mode Selector (Sec. 3.D), on the device.  At each knot k the power of mode i is
 * |A_i(t_k)|^2, doubled for m_i > 0 (the mode also stands for its m < 0 partner); powers are
 * sorted in descending order (ties: lower mode index first) and summed cumulatively, and the knot
 * keeps the shortest leading run whose cumulative power reaches (1 - eps) of its total (a knot
 * with zero total keeps nothing).  mask_dev[i] = 1 for the union of kept modes over all knots,
 * else 0.
 *   amp_re_dev, amp_im_dev [K][N]: device arrays, row-major (modes contiguous).
 *   m [N]: host array of the modes' m (>= 0).  eps >= 0.  N <= 4096.
 *   mask_dev: N bytes of device memory (overwritten).
 * Asynchronous on `stream`.  The result is exact with respect to this definition evaluated in
 * FP64: each power is fl(fl(re^2) + fl(im^2)) (no fused multiply-add) and each cumulative sum is
 * the left-to-right FP64 sum over the sorted powers, the total being the last of them, so the
 * mask does not depend on the GPU's scheduling.
 */
few_status few_mode_select(few_ctx *ctx, const double *amp_re_dev, const double *amp_im_dev, int K,
                           int N, const int *m, double eps, unsigned char *mask_dev, void *stream);

/*
 * Direct (non-interpolated) summation (Sec. 3.C, the basic summation module): the phases and the
 * amplitudes are given at every output sample, so no spline is built:
 *   out[i] = scale * sum_j [ A_ij Y+_j e^{-i Phi_j,i} + (m_j > 0) conj(A_ij) Y-_j e^{+i Phi_j,i} ],
 *   Phi_j,i = m_j phi_phi[i] + n_j phi_r[i] (rad), Y+ = -2Y_lm(theta, phi), Y- = (-1)^l -2Y_{l,-m}.
 *   phi_phi_dev, phi_r_dev [n_samples], amp_re_dev, amp_im_dev [n_samples][N] (modes contiguous):
 *     device memory.  l, m, n [N]: host arrays (validated as for few_traj_create).
 *   prec: FEW_MIXED (FP64 phase reduction, FP32 exponentials and sums; bound by HBM bandwidth)
 *     or FEW_FP64.  out_dev: n_samples complex64 (out_c64) or complex128, device memory.
 * Asynchronous on `stream`.
 */
few_status few_direct_sum(few_ctx *ctx, const double *phi_phi_dev, const double *phi_r_dev,
                          const double *amp_re_dev, const double *amp_im_dev, int64_t n_samples,
                          const int *l, const int *m, const int *n, int N, double theta, double phi,
                          double scale, int prec, void *out_dev, int out_c64, void *stream);

/*
 * Reduced basis of the mode amplitudes (Sec. 3.E, RomanNet): Nb complex vectors B_j over the N
 * modes of a mode list, so that a knot's amplitudes are A_i = sum_j alpha_j B_j,i.
 *   b_re, b_im [Nb][N]: row-major (modes contiguous), host (where = FEW_MEM_HOST; copied before
 *     the call returns) or device memory (FEW_MEM_DEVICE; read on `stream`, must stay valid
 *     until that work completes).  1 <= Nb <= FEW_MAX_BASIS, N >= 1.
 * The library keeps an FP64 copy of B, the Gram matrix B B^H (for the renormalisation) and the
 * scaled, split, packed fp16 operand of the tensor-core product, about 16 x Nb x N + 12 x Nb x N
 * bytes.
 * Asynchronous on `stream`; the handle is usable on any stream ordered after it.
 * Errors: FEW_ERR_INVALID_ARG, FEW_ERR_LIMIT (Nb too large), FEW_ERR_BUDGET, FEW_ERR_NOMEM,
 * FEW_ERR_CUDA.
 */
few_status few_basis_create(few_ctx *ctx, const double *b_re, const double *b_im, int Nb, int N,
                            few_mem where, void *stream, few_basis **out);

/* Release a basis (after the device is idle on the work that uses it). */
few_status few_basis_release(few_ctx *ctx, few_basis *basis);

/*
 * Mode amplitudes from reduced-basis coefficients (Sec. 3.E): for each of M knots,
 *   A_k,i = s_k sum_j alpha_k,j B_j,i,  s_k = nu_k / ||alpha_k B|| if norms_dev, else 1,
 * the renormalisation of the network output to the trajectory's norm (a zero vector stays zero).
 *   alpha_re_dev, alpha_im_dev [M][Nb], norms_dev [M] (or NULL): device memory.  Target norms
 *     must be finite and >= 0; others latch FEW_ERR_INVALID_ARG (see few_sync_status).
 *   amp_re_dev, amp_im_dev [M][N]: device memory, overwritten; the layout few_traj_set_data
 *     reads (FEW_MEM_DEVICE), so a trajectory's amplitudes can be produced in place.
 *   prec: FEW_FP64 (complex GEMM on the FP64 pipe) or FEW_MIXED (one real GEMM on the tensor
 *     cores: fp16 operands split two ways after exact power-of-two scaling of each knot's row and
 *     each mode's column, three partial products, FP32 accumulation; error near FP32 rounding of
 *     the row's and column's largest terms).
 * Asynchronous on `stream`; scratch (M x 16 bytes, plus about M x Nb x 12 bytes for FEW_MIXED)
 * comes from the context's pool.  M = 0 is a no-op.
 */
few_status few_rb_amplitudes(few_ctx *ctx, const few_basis *basis, const double *alpha_re_dev,
                             const double *alpha_im_dev, int M, const double *norms_dev, int prec,
                             double *amp_re_dev, double *amp_im_dev, void *stream);

/* Flags of few_batch_plan. */
#define FEW_BATCH_REBUILD_SPLINES 1u  /* each run also rebuilds every distinct trajectory's
                                         splines from its device-resident knot data */
#define FEW_BATCH_NO_GRAPH 2u         /* run by direct launches instead of a CUDA graph */

/*
 * Plan a batch of requests (all with the same `prec`; any mix of trajectories, durations,
 * cadences and mode counts) executed as one persistent summation launch whose CTAs take
 * slices of the concatenated (waveform, sample) work of equal pass cost.  The plan holds its own
 * scratch; the kernels are captured once into a CUDA graph (unless FEW_BATCH_NO_GRAPH), and
 * each few_batch_run replays it.  Every request must use out_where == FEW_MEM_DEVICE.  The
 * trajectories and output buffers must stay valid while the batch exists.  Blocking (uploads
 * the plan and, for the graph, captures it).
 */
few_status few_batch_plan(few_ctx *ctx, const few_request *reqs, int n, unsigned flags,
                          few_batch **out);

/* Run a planned batch on `stream` (graph launch or direct launches). Asynchronous. */
few_status few_batch_run(few_ctx *ctx, few_batch *batch, void *stream);

/* Release a batch plan.  The caller must make sure every run of the batch has completed (an
 * event or stream synchronisation); this call does not wait for the device. */
few_status few_batch_release(few_ctx *ctx, few_batch *batch);

/*
 * Wait for all work on the context's device, then return and clear the device-side error
 * latch (FEW_ERR_INVALID_ARG for non-finite device inputs, FEW_ERR_TIMEOUT for an expired
 * bounded wait), or FEW_ERR_CUDA if the device reported an error.  FEW_OK otherwise.
 */
few_status few_sync_status(few_ctx *ctx);

/*
 * Self-test of the device error latch (the paper has no counterpart; it exists so that the
 * timeout path can be exercised without a fault): queues on `stream` one kernel whose single
 * bounded wait is on a barrier that nothing arrives on and no copy targets.  The wait gives up
 * after limit_us microseconds (1 <= limit_us <= 2,000,000) and latches FEW_ERR_TIMEOUT, which
 * the next few_sync_status returns (and clears).  Errors: FEW_ERR_INVALID_ARG, FEW_ERR_CUDA.
 */
few_status few_selftest_wait_expiry(few_ctx *ctx, unsigned limit_us, void *stream);

/*
 * Tile configuration of the summation kernel for one precision:
 *   samples_per_thread (R, the sample tile: a pass covers threads x R consecutive samples):
 *     FEW_FP64: 1 or 2; FEW_MIXED: 2, 4 or 8;
 *   threads_per_block: 128 or 256;
 *   stage_slots (the mode tile: harmonic slots per shared-memory stage through which each
 *     segment's table streams): a multiple of 16 in [16, 4096].
 * Defaults: FEW_FP64 (1, 256, 256), FEW_MIXED (8, 256, 1024).  Three stages of stage_slots x 64
 * bytes (FEW_FP64) or x 32 bytes (FEW_MIXED) must fit in one CTA's shared memory, else the
 * waveform calls return FEW_ERR_LIMIT.  Affects speed only: every configuration gives
 * bit-identical results.
 */
few_status few_set_tiles(few_ctx *ctx, int prec, int samples_per_thread, int threads_per_block,
                         int stage_slots);
few_status few_get_tiles(few_ctx *ctx, int prec, int *samples_per_thread, int *threads_per_block,
                         int *stage_slots);

/*
 * Per-kernel device timing.  With timing enabled, the library records a CUDA event pair on the
 * launch stream around each kernel it queues.  few_last_timing waits for the most recent pairs
 * and returns their durations in ms: ms[0] spline build (last few_traj_set_data), ms[1]
 * harmonics, ms[2] fold, ms[3] summation (last few_waveform or few_batch_run without a graph).
 * Entries never recorded are returned as -1.
 */
few_status few_ctx_set_timing(few_ctx *ctx, int enable);
few_status few_last_timing(few_ctx *ctx, float *ms);

/* ---------------------------------------------------------------- host-only planning
 * These run on the host only (no GPU needed) and expose the planning step of few_waveform.
 */

/*
 * Sample range of every segment (Sec. 3.C: all arrays share one knot grid): segment k
 * (0 <= k < K-1) owns samples [seg_start[k], seg_start[k+1]) with seg_start[k] =
 * clamp(ceil((t_k - t0)/dt), 0, n_samples) for k >= 1, seg_start[0] = 0 and
 * seg_start[K-1] = n_samples (a sample on a knot belongs to the segment that starts there;
 * one on the last knot belongs to the last segment).  seg_start has K entries.
 * Validates as few_waveform does (FEW_ERR_KNOTS, FEW_ERR_RANGE).
 */
few_status few_plan_segments(const double *t_knots, int K, double t0, double dt, int64_t n_samples,
                             int64_t *seg_start);

/*
 * Harmonic slot plan of a mode list: the distinct signed (m, n) frequencies that the m >= 0
 * modes and their m < 0 partners (Eq. amp_symmetry) occupy, laid out as rows of constant m,
 * every m from the largest down to the most negative present, each row spanning its lowest to
 * highest n (zero-filled in between; a row without modes has no slot).  Returns the slot count
 * per segment and the number of rows.  Validates the modes (FEW_ERR_MODES).
 */
few_status few_mode_slots(const int *l, const int *m, const int *n, int N, int *n_slots, int *n_rows);

/*
 * The summation's division of work among its CTAs, as few_waveform and few_batch_plan compute
 * it: the concatenated (waveform, sample) space of n_waves waveforms is cut into `grid`
 * contiguous slices at pass boundaries (a pass = `pass` consecutive samples of one segment,
 * threads x samples per thread), each slice holding an equal share, to within one pass, of the
 * total cost (each pass costs (slots + 16) per sample of a full pass, whether or not its segment
 * ends first).
 *   seg_start: the n_waves waveforms' segment sample ranges (few_plan_segments) concatenated,
 *              K[w] entries for waveform w, the last one its sample count.
 *   K [n_waves], n_slots [n_waves]: knots and harmonic slots (few_mode_slots) per waveform.
 *   out_wave, out_sample [grid + 1]: CTA g starts at sample out_sample[g] of waveform
 *              out_wave[g] (a start at or past the end of a waveform means the next one's
 *              beginning); entry grid = (n_waves, 0), the end.
 * Host only; errors: FEW_ERR_INVALID_ARG (null pointer, n_waves < 1, grid < 1, pass < 1,
 * K < 2, n_slots < 1, decreasing segment starts).
 */
few_status few_plan_cta_slices(int n_waves, const int64_t *seg_start, const int *K,
                               const int *n_slots, int grid, int pass, int *out_wave,
                               int *out_sample);

#ifdef __cplusplus
}
#endif
#endif /* FEWSUM_H */
