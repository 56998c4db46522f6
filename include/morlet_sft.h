/*
 * morlet_sft.h - C ABI of a GB300 (sm_103a) library for the Morlet wavelet transform and Gaussian
 * smoothing by the sliding Fourier transform (SFT) and the attenuated SFT (ASFT), after
 * Y. Yamashita and T. Wakahara, "Morlet wavelet transform using attenuated sliding Fourier
 * transform and kernel integral for graphic processing unit" (arXiv:2110.11866).
 *
 * Notation. The paper's half window K is called L here (the window is k in [-L, L], 2L+1 samples,
 * beta = pi / L) and its number of Fourier terms P_D is called K.
 *
 * Conventions shared by every entry point
 *   - Plain pointers and sizes only. Device pointers are CUDA device (or managed) addresses owned by
 *     the caller; the library never frees them. Host pointers are read during the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream. Calls that
 *     launch work are asynchronous on that stream unless stated otherwise.
 *   - Every function returns a morlet_status (0 = success). Errors are reported, never abort.
 *     A timeout inside a kernel (the bounded cross-tile wait) is latched in a host-visible error
 *     word and returned as MORLET_ERR_TIMEOUT by the next call on the plan and by
 *     morlet_last_device_error.
 *   - Real input x: the signals of a batch are concatenated, signal i starting at element
 *     sum_{i'<i} lengths[i'], FP32 (precision FP32_*) or FP64 (precision FP64).
 *   - Scalogram output W: interleaved complex (complex64 for FP32 precisions, complex128 for FP64),
 *     laid out [signal][scale][n]: element S * off_i + s * N_i + n, off_i the signal's start in x.
 *   - Samples outside [0, N) count as zero (the "zero" extension of Sec. II, eq. xG).
 */
#ifndef MORLET_SFT_H
#define MORLET_SFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct morlet_plan_s* morlet_plan_t;

typedef enum {
  MORLET_OK = 0,
  MORLET_ERR_ARG = -1,          /* invalid argument (size, pointer, option) */
  MORLET_ERR_UNSUPPORTED = -2,  /* valid but not built (e.g. K > 12, ASFT adjoint) */
  MORLET_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  MORLET_ERR_TIMEOUT = -4,      /* a kernel gave up waiting on a predecessor tile */
  MORLET_ERR_NOMEM = -5         /* device or host allocation failed */
} morlet_status;

/* method */
enum { MORLET_DIRECT = 0, MORLET_GAUSS = 1, MORLET_MULTIPLY = 2 };
/* transform */
enum { MORLET_SFT = 0, MORLET_ASFT = 1 };
/* precision: arithmetic of the per-sample scan and of the cross-tile carries */
enum {
  MORLET_FP32_PLAIN = 0,  /* FP32 samples, FP32 scan, FP32 carries; the SFT runs one look-back chain
                             per row */
  MORLET_FP32_COMP = 1,   /* FP32 samples and scan; two-float (FP32 hi + lo) carries and prefix sums;
                             windows restarted per segment or started from exact prefix-sum states */
  MORLET_FP64 = 2         /* FP64 everywhere */
};
/* scan form */
enum {
  MORLET_FORM_AUTO = 0,       /* rotating frame (the faster form on this GPU) */
  MORLET_FORM_KERNEL = 1,     /* kernel integral: modulate, prefix-scan, difference, demodulate */
  MORLET_FORM_ROTATING = 2    /* the same window sums kept in the frame of each harmonic */
};
/* flags */
enum {
  MORLET_FLAG_NO_GRAPH = 1,   /* launch kernels directly instead of replaying a CUDA graph */
  MORLET_FLAG_AUTOTUNE = 2,   /* compensated FP32 SFT plans (Morlet and Gaussian), FP32 ASFT and
                                 multiplication-method plans: at plan time, time the forward (a
                                 sub-plan with a zero input and a scratch output: the whole batch if
                                 that scratch takes at most a quarter of the free device memory, else
                                 every k-th signal up to 2^28 outputs) under a few schedules -- row
                                 thresholds (morlet_plan_set_row_thresholds; for the ASFT and the
                                 multiplication method the Horner start-state limit, timed together
                                 with the ASFT's chains), segment and item lengths, item order, ASFT
                                 chains (morlet_plan_set_schedule) -- and keep the fastest (each
                                 knob keeps its value unless another is at least 1 % faster) */
  MORLET_FLAG_NO_HALO = 4,    /* force one look-back chain per row (no per-tile window recompute) */
  MORLET_FLAG_EDGE = 8,       /* forward: extend each signal with its edge values instead of zeros
                                 (Sec. II: "zero or the values on the edges"); the plan holds a padded
                                 copy of the batch (the longest window reach on each side), refreshed
                                 by every forward; morlet_backward returns MORLET_ERR_UNSUPPORTED */
  MORLET_FLAG_NO_ADJOINT = 16 /* build no adjoint: the plan does not hold the adjoint's workspace (two
                                 real planes per scale of the batch); morlet_backward returns
                                 MORLET_ERR_UNSUPPORTED */
};

typedef struct {
  int64_t n_signals;        /* >= 1 */
  const int64_t* lengths;   /* host array [n_signals], each >= 1; copied into the plan */
  int32_t n_scales;         /* >= 1 */
  const double* sigmas;     /* host array [n_scales], each >= 0.5; copied into the plan */
  double xi;                /* Morlet centre parameter; omega0 = xi / sigma (Sec. III) */
  int32_t K;                /* Fourier terms, 1..12; 0 = smallest K whose relative fit RMSE <= fit_tol */
  double fit_tol;           /* used only when K == 0 */
  int32_t method;           /* MORLET_DIRECT (Morlet, direct method of Sec. III-A) | MORLET_GAUSS |
                               MORLET_MULTIPLY (Morlet, multiplication method of Sec. III-B) */
  int32_t transform;        /* MORLET_SFT | MORLET_ASFT */
  int32_t precision;        /* MORLET_FP32_PLAIN | MORLET_FP32_COMP | MORLET_FP64 */
  int32_t norm;             /* 0: e^{-k^2/2sigma^2} e^{i omega0 k}; 1: C_xi pi^{-1/4} sigma^{-1/2} (...)(e^{i xi k/sigma} - kappa_xi) */
  int32_t n0;               /* ASFT output shift; 0 = max(1, round(sigma / 8)) per scale */
  double window_mult;       /* L = ceil(window_mult * sigma); 0 = 4.0 */
  int32_t deriv;            /* MORLET_GAUSS only: 0 = G, 1 = G_D, 2 = G_DD (Sec. II) */
  int32_t form;             /* MORLET_FORM_* */
  int32_t flags;            /* MORLET_FLAG_* */
  int64_t spin_limit;       /* bounded wait in polls of a predecessor flag; 0 = default (about 1 s) */
} morlet_plan_desc;

/*
 * morlet_plan - validate `desc`, fit the coefficients and build everything a transform needs.
 * Defines: per scale, L = ceil(window_mult * sigma), beta = pi / L, harmonics p = P_S .. P_S + K - 1
 * with P_S the least-residual start (direct method, Sec. III-A), coefficients m_p (cos) and l_p
 * (sin) minimising eq. mmse over k in [-L, L], fitted on the GPU in FP64. For MORLET_GAUSS:
 * harmonics 0..K-1 fitted to G, G_D or G_DD (eq. aproGauss). MORLET_GAUSS with MORLET_ASFT (eqs.
 * GsASFT, gddAsft): with alpha = n0 / sigma^2 and the shift identity eq. siftGauss, the fitted
 * target is G, G_D - alpha G or G_DD - 2 alpha G_D + alpha^2 G (cos terms for the even part, sin
 * terms for the odd part); the damped window sums then give G_X[n] at output n.
 * The ASFT runs in FP32 (either FP32 precision); MORLET_FP64 with MORLET_ASFT is unsupported.
 * Its window sum depends only on the last 2L + 1 samples, so in either precision a row with
 * 2L <= 8192 is cut into independent window segments, each started from a zero state 2L samples
 * before its first output; longer windows run one look-back chain per row (as do all rows under
 * MORLET_FLAG_NO_HALO).
 * MORLET_MULTIPLY (Sec. III-B): the envelope e^{-k^2/(2 sigma^2)} is fitted by K cos terms a_p
 * (p = 0 .. K-1) and the Morlet becomes sum_{p=-(K-1)}^{K-1} a'_p e^{i (omega0 + beta p) k}
 * (a'_0 = a_0, a'_{+-p} = a_p / 2): 2K - 1 non-harmonic window sums combined with complex weights.
 * Built for the SFT, norm = 0, FP32 (either FP32 precision runs the FP32 scan), 2K - 1 <= 12 and
 * L <= 4096; other cases return MORLET_ERR_UNSUPPORTED.
 * Allocates the plan's device workspace (tile table, cross-tile status, tables) and a host-mapped
 * error word; no allocation happens in forward/backward. Synchronises `stream`.
 * Errors: MORLET_ERR_ARG (bad sizes/options), MORLET_ERR_NOMEM, MORLET_ERR_CUDA.
 * On error *out is set to NULL.
 */
int morlet_plan(morlet_plan_t* out, const morlet_plan_desc* desc, void* stream);

/*
 * morlet_forward - the transform of Sec. III-A (SFT: eqs. kernel-kernelInter and the direct-method
 * combine; ASFT: eq. iir1A with the shift of eq. GsASFT), for all signals x all scales.
 * x: device, real, layout above (FP32, or FP64 for MORLET_FP64).
 * W: device, complex scalogram [signal][scale][n] for MORLET_DIRECT; for MORLET_GAUSS a real array
 *    [signal][scale][n] of the smoothed signal (or derivative).
 * Asynchronous. Returns MORLET_ERR_TIMEOUT if a previous launch on this plan timed out.
 */
int morlet_forward(morlet_plan_t plan, const void* x, void* W, void* stream);

/*
 * morlet_backward - adjoint of morlet_forward for a real-valued loss (SFT, MORLET_DIRECT only).
 * gW: device complex [signal][scale][n], gW = dLoss/dRe W + i dLoss/dIm W.
 * gx: device real, same layout as x: gx[t] = sum_scales sum_n Re(conj(gW[n]) dW[n]/dx[t]).
 * The fitted kernel has an even real and an odd imaginary part (Sec. III-A), so the adjoint of
 * scale s is gx_s = Re W_s(Re gW_s) - Im W_s(Im gW_s), W_s the forward transform of a real signal.
 * The call splits gW into its 2S real planes (planes of n_in = sum of lengths samples, held by the
 * plan), runs their real-output transforms in one launch on the forward's kernels (rotating form,
 * same precision; start states for long windows), and sums the 2S result planes in a fixed order
 * (deterministic). Asynchronous; captured once per (gW, gx) pair into a CUDA graph and replayed
 * (unless MORLET_FLAG_NO_GRAPH). A plan's forward and backward share its look-back status arrays:
 * do not run them concurrently on different streams.
 * Errors: MORLET_ERR_UNSUPPORTED for ASFT, MORLET_GAUSS, MORLET_MULTIPLY, MORLET_FLAG_EDGE or
 * MORLET_FLAG_NO_ADJOINT plans.
 */
int morlet_backward(morlet_plan_t plan, const void* gW, void* gx, void* stream);

/*
 * gauss_smooth - Gaussian smoothing (deriv 0) or its first / second derivative (deriv 1, 2) of one
 * real signal by SFT (eq. GsSFT and the two after it), harmonics p = 0..P (P + 1 terms),
 * L = ceil(4 sigma). x, y: device arrays of N elements (FP32, or FP64 if precision == MORLET_FP64).
 * Builds (first call) and caches a plan per (N, sigma, P, deriv, precision, device); later calls
 * with the same key allocate nothing. Synchronous on first use of a key, asynchronous afterwards.
 */
int gauss_smooth(const void* x, int64_t N, double sigma, int32_t P, int32_t deriv, int32_t precision,
                 void* y, void* stream);

/*
 * gauss_filter_2d - separable Gaussian filtering of an image: out = (G_{deriv_y} along y) (G_{deriv_x}
 * along x) * img. The rows and the columns of an image are independent 1-D signals (Sec. IV,
 * opening paragraph), so this is one batched 1-D transform of eq. GsSFT (or a derivative form) over
 * the ny rows, a transpose, one over the nx columns, and a transpose back.
 * img, out: device arrays [ny][nx], row-major, FP32 (FP64 if precision == MORLET_FP64); they may not
 * overlap. deriv_x, deriv_y in 0..2 (G, G_D, G_DD along that axis); harmonics p = 0..P; L =
 * ceil(4 sigma); zero extension outside the image.
 * Builds (first call) and caches, per (device, ny, nx, sigma, P, deriv_y, deriv_x, precision), the
 * two 1-D plans (with MORLET_FLAG_AUTOTUNE: the first call also times their schedules) and a
 * workspace of 2 ny nx elements; later calls with the same key allocate nothing and are
 * asynchronous on `stream`.
 * Errors: MORLET_ERR_ARG (sizes, derivatives, precision; ny or nx above 2^21), MORLET_ERR_NOMEM,
 * MORLET_ERR_CUDA, and those of morlet_plan / morlet_forward.
 */
int gauss_filter_2d(const void* img, int64_t ny, int64_t nx, double sigma, int32_t P, int32_t deriv_y,
                    int32_t deriv_x, int32_t precision, void* out, void* stream);

/* Release a plan and everything it owns. Synchronises the device. NULL is ignored. */
void morlet_plan_destroy(morlet_plan_t plan);

/* Static description of a status code. */
const char* morlet_strerror(int status);

/*
 * morlet_last_device_error - the plan's host-mapped error word after synchronising `stream`:
 * 0, or MORLET_ERR_TIMEOUT if any cross-tile wait gave up. Clears the word.
 */
int morlet_last_device_error(morlet_plan_t plan, void* stream);

/*
 * morlet_plan_info - copy the fitted parameters of scale `s` to host memory.
 * L, p0, K: host int64/int32 outputs; m, l: host double[12] (coefficients of cos / sin terms,
 * entries >= K are zero); n0: ASFT shift (0 for SFT). Any output pointer may be NULL.
 */
int morlet_plan_info(morlet_plan_t plan, int32_t s, int64_t* L, int32_t* p0, int32_t* K, double* m,
                     double* l, int32_t* n0);

/*
 * morlet_plan_stats - launch shape and work of the forward, for measurement:
 * out[0] = threads per CTA, out[1] = samples per thread, out[2] = CTAs of the look-back kernel,
 * out[3] = work items of the scan kernels, out[4] = 512-position tiles processed (incl. prologues),
 * out[5] = rows in look-back mode, out[6] = rows in window-segment mode, out[7] = kernel launches
 * per forward, out[8] = rows whose work items start from prefix sums, out[9] = prefix-sum work items,
 * out[10] = rows in lane-chunk mode, out[11] = lane-chunk work items, out[12] / out[13] = the row
 * thresholds in use (rows with L <= out[12] take the lane-chunk scan, rows with L > out[13] take
 * start-state items), out[14] = 1 when those start states are window sums of tile sums, 0 when they
 * come from prefix sums.
 */
int morlet_plan_stats(morlet_plan_t plan, int64_t out[15]);

/*
 * morlet_plan_set_spin_limit - change the bounded-wait limit (polls) of later launches; used to make
 * the timeout path fire quickly in tests.
 */
int morlet_plan_set_spin_limit(morlet_plan_t plan, int64_t polls);

/*
 * morlet_plan_set_row_thresholds - choose which rows of a compensated-FP32 rotating-form SFT
 * forward take the lane-chunk scan (L <= lane_chunk_max_L; 0: none) and which take start-state
 * work items (L > start_state_min_L), the two choices MORLET_FLAG_AUTOTUNE makes by timing. For an
 * FP32 rotating-form ASFT or multiplication-method plan start_state_min_L instead sets which rows
 * start from Horner tile-sum
 * states (L > start_state_min_L, at most 4096, the default; the other rows are window segments) and
 * lane_chunk_max_L is ignored; other plans keep their single schedule and ignore both. Only choices
 * that keep every row within the compensated-FP32 gate (1e-5 of max|W|) are accepted:
 * 0 <= lane_chunk_max_L <= 256 and 1 <= start_state_min_L <= 2048 (window segments of longer
 * windows drift past the gate on resonant inputs; start-state items hold at any window length).
 * The transform is the same for every accepted choice; only the schedule
 * changes. Rebuilds the forward's work tables synchronously (device memory is freed and
 * allocated, so no forward of this plan may be in flight). Errors: MORLET_ERR_ARG for a value out
 * of those ranges; MORLET_ERR_NOMEM or MORLET_ERR_CUDA if the rebuild fails (the plan keeps its
 * previous thresholds); MORLET_ERR_TIMEOUT if an earlier launch timed out and its error word was
 * not read yet.
 */
int morlet_plan_set_row_thresholds(morlet_plan_t plan, int64_t lane_chunk_max_L, int64_t start_state_min_L);

/*
 * morlet_plan_set_schedule - the forward's scheduling knobs (none changes the transform; all keep
 * every row within the precision gates):
 *   seg_mult (8, 12 or 16): window segments run about seg_mult * L positions after their 2L-position
 *     restart (a longer segment spends a smaller share on the restart);
 *   ss_tiles_max (4..64): start-state work items hold at most this many 512-position tiles;
 *   order (0, 1 or 2): inside each block of signals the rows go scale by scale in index order (0)
 *     or in decreasing window length (1); 2 takes order 0 and then sorts the work items of each
 *     launch longest first, so that a launch ends on short items;
 *   asft_chains (0 or 1): ASFT plans put every row on one look-back chain (1) instead of cutting
 *     rows with 2L <= 8192 into window segments (0).
 * MORLET_FLAG_AUTOTUNE picks them (and the row thresholds) by timing. Rebuilds the forward's work
 * tables synchronously (device memory is freed and allocated; no forward of this plan may be in
 * flight). Errors: MORLET_ERR_ARG for a value out of range (the plan keeps its schedule);
 * MORLET_ERR_TIMEOUT if an earlier launch timed out and its error word was not read yet.
 */
int morlet_plan_set_schedule(morlet_plan_t plan, int32_t seg_mult, int32_t ss_tiles_max, int32_t order,
                             int32_t asft_chains);

/*
 * morlet_plan_schedule - the forward's schedule, for measurement: out[0] / out[1] = the row
 * thresholds (as morlet_plan_stats out[12] / out[13]), out[2] = seg_mult, out[3] = ss_tiles_max,
 * out[4] = order, out[5] = asft_chains (see morlet_plan_set_schedule), out[6] = 1 if
 * MORLET_FLAG_AUTOTUNE timed the schedules, -1 if it was skipped because its sub-plan or scratch
 * buffers could not be allocated (the defaults are kept), 0 without the flag; out[7] = outputs of
 * the rows the autotuner timed (the whole batch, or the subset of every k-th signal).
 */
int morlet_plan_schedule(morlet_plan_t plan, int64_t out[8]);

/*
 * morlet_debug_skip_tickets - testing hook: in the next forward, the first kernel that waits on
 * predecessors (the prefix-sum kernel when the plan's start states come from prefix sums, else the
 * look-back scan kernel) starts its work-item counter at `skip` instead of 0, so its first `skip`
 * work items are never processed and items that wait on them hit the bounded wait. The outputs of
 * that forward are undefined. Must be followed by morlet_last_device_error.
 */
int morlet_debug_skip_tickets(morlet_plan_t plan, int64_t skip);

/*
 * morlet_measure_fp64_rate - measurement helper, not part of the transform (the paper has no
 * counterpart): the device's FP64 fused multiply-add rate, in flops/s (2 per FMA), written to the
 * host double *flops. It times one launch of a kernel in which every thread runs 8 independent FMA
 * chains (one grid of resident CTAs on every SM, after a shorter warm-up launch) with CUDA events
 * on `stream`. It is the denominator of the FP64 path's roofline: on this GPU the FP64 transform is
 * bound by the FP64 pipe, not by memory. Allocates and frees a small device buffer; synchronous.
 * Errors: MORLET_ERR_ARG (flops NULL), MORLET_ERR_NOMEM, MORLET_ERR_CUDA.
 */
int morlet_measure_fp64_rate(double* flops, void* stream);

/*
 * morlet_forward_noalloc - forward transform that allocates no memory (no cudaMalloc, no cudaFree,
 * no allocating library call), for callers that cannot allocate device memory themselves, such as
 * code running inside a framework or allocator that owns all device memory.
 * The paper has no counterpart; this is a deployment convenience of this library.
 * One real FP32 signal x[0..N-1] (device), one scale sigma, omega0 = xi / sigma, K terms (1..12),
 * SFT, compensated FP32, unnormalised Morlet (norm 0), L = ceil(4 sigma); W: device complex64[N],
 * the caller's. It runs the row on window segments (L <= 4096) or look-back chains (longer windows)
 * only, so its schedule differs from the plan path's: its results agree with the oracle and with
 * morlet_plan + morlet_forward (same parameters) within the compensated-FP32 gate, 1e-5 of max|W|,
 * not bit for bit.
 * All working memory (fit, tables, work-item table, look-back status) lives in one fixed device
 * array of about 8.1 MB inside the library; every GPU that loads the library holds it until the
 * process exits. The work-item table is cut on the host into a file-scope host array and copied in.
 * Limits: at most 16384 work items and 16384 look-back slots per call; larger rows return
 * MORLET_ERR_ARG. Window segments of L <= 4096 cover max(2, ceil(16 L / 512)) * 512 - 2L - 7
 * outputs each (N up to about 1.56e7 at sigma = 8, 5.9e7 at sigma = 64, 2.3e8 at sigma = 256);
 * longer windows use one slot per 4096 positions of segments of max(16384, 4L) outputs, each with a
 * 2L restart (N up to about 3.8e7 to 4.7e7).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture. Each call synchronises `stream`
 * once at entry to read the error word the previous call on the device left (MORLET_ERR_TIMEOUT if
 * its bounded cross-tile wait gave up), then enqueues its kernels asynchronously: a timeout in the
 * last call of a sequence is reported only by a further call. All calls on a device share the
 * array: calls whose kernels overlap on the GPU (different streams, no ordering) race and corrupt
 * each other's results; order them on one stream.
 */
int morlet_forward_noalloc(const void* x, int64_t N, double sigma, double xi, int32_t K, void* W, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MORLET_SFT_H */
