/*
 * zotfs.h -- C ABI of the GB300 (sm_103a) Zak-OTFS receiver library.
 *
 * The library implements the data-parallel hot path of a Zak-OTFS receiver: the
 * discrete Zak transform into the delay-Doppler (DD) grid, the point-pilot read-off
 * that yields a path list, the structured-sparse (SS) channel operator H_dd and its
 * adjoint, the compute-aware conjugate-gradient LMMSE equaliser (SS-CGA) and max-log
 * QAM demapping.  Passages cited below are sections, equations and algorithms of
 * arXiv:2604.02266 ("Real-Time and Scalable Zak-OTFS Receiver Processing on GPUs").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved {re, im}.  ZOTFS_C64 is two float32 (the layout
 *    of torch.complex64); ZOTFS_C32_F16 / ZOTFS_C32_BF16 are two 16-bit floats.
 *  - A DD grid X[k, l] (delay bin k < M, Doppler bin l < N) is stored vectorised as
 *    q = l*M + k (Sec. IV-B, "We index the q-th row ... q = l M + k").
 *  - A time-domain (TD) frame y[i], i = k + n*M < M*N, is stored in sample order.
 *  - M and N are powers of two with 16 <= M <= 256, 8 <= N <= 64 and M*N <= 16384; plans
 *    also take SISO grids up to 16384 x 32 (see zotfs_plan_create).
 *  - MIMO (n_rx x n_tx, not in the paper): unknowns are stacked per tx antenna,
 *    observations per rx antenna, one path list per (rx, tx) pair, and tx antenna t
 *    sends its own pilot frame (time-orthogonal pilots).  Layouts, per frame f:
 *        pilot TD frames  [f][t][r][MN]     data TD frames [f][r][MN]
 *        path lists       [f][r][t]         x_hat          [f][t][MN]
 *        LLRs             [f][t][MN][bps]   hard bits      [f][t][MN*bps/8] bytes
 *    where bps = log2(qam); bits are packed LSB-first (bit b -> byte b/8, position b%8)
 *    and within a symbol the I-axis Gray label (MSB first) precedes the Q-axis label.
 *  - Every pointer named "dev" is device memory owned by the caller; "host" pointers are
 *    read during the call only.  The library owns only what a plan or a batch holds.
 *  - Calls taking a stream are stream-ordered and never synchronise the host, except
 *    the create/destroy calls.  Argument errors are returned synchronously; per-frame
 *    conditions (a truncated path list, a bad path, a non-finite residual, a timed-out
 *    wait) are written to a caller-supplied device status array as zotfs_status values.
 *  - A plan is used from one host thread at a time.  Its calls may be issued on different
 *    streams (up to 16 in flight at once) and then run concurrently, except those that use
 *    the plan's own scratch (the
 *    large-frame, clustered large-frame and paper-scale kernels, and the plain form): the
 *    plan orders these after one another across streams (an event per plan; inside a CUDA
 *    graph capture the caller's stream order alone applies).
 *  - No call throws across the ABI.  zotfs_last_error() returns a thread-local message
 *    describing the most recent failure in the calling thread.
 */
#ifndef ZOTFS_H
#define ZOTFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum zotfs_status {
  ZOTFS_OK = 0,
  ZOTFS_EINVAL = 1,        /* bad argument (synchronous) or a bad path entry (per frame) */
  ZOTFS_ENOMEM = 2,        /* device or host allocation failed */
  ZOTFS_ECUDA = 3,         /* a CUDA runtime call failed */
  ZOTFS_EUNSUPPORTED = 4,  /* shape or option outside what the library handles */
  ZOTFS_ETIMEOUT = 5,      /* a bounded device wait gave up (per frame) */
  ZOTFS_ETRUNCATED = 6,    /* more than p_max taps passed the threshold (per frame, result valid) */
  ZOTFS_ENONFINITE = 7     /* a CG residual became NaN/Inf (per frame) */
} zotfs_status;

/* The CUDA stream type: identical to cudaStream_t, without including CUDA headers. */
typedef struct CUstream_st* zotfs_stream;

/* Pulse shape of the link.  Recorded in the plan; the receiver arithmetic of Eq. zak
 * does not depend on it (only the channel the frames went through does). */
typedef enum zotfs_pulse { ZOTFS_PULSE_SINC = 0, ZOTFS_PULSE_RECT = 1 } zotfs_pulse;

typedef enum zotfs_dtype {
  ZOTFS_C64 = 0,       /* complex float32 */
  ZOTFS_C32_F16 = 1,   /* complex float16 storage, float32 arithmetic */
  ZOTFS_C32_BF16 = 2,  /* complex bfloat16 storage, float32 arithmetic */
  ZOTFS_C128 = 3       /* complex float64 (plans with compute == ZOTFS_COMPUTE_FP64) */
} zotfs_dtype;

/* Arithmetic precision of a plan's kernels.  FP32: complex float32 vectors with the CG's
 * inner products combined and alpha/beta formed in FP64.  FP64: everything in float64; the
 * complex vectors the caller passes in or receives (DD inputs, operator inputs/outputs,
 * x_hat) are then ZOTFS_C128, LLRs stay float32. */
typedef enum zotfs_compute { ZOTFS_COMPUTE_FP32 = 0, ZOTFS_COMPUTE_FP64 = 1 } zotfs_compute;

typedef enum zotfs_pilot_mode {
  /* The paper's arrangement (Sec. V, Fig. 1): a point-pilot frame precedes each data
   * frame; the read-off spans the whole grid (Eq. heff's index ranges). */
  ZOTFS_PILOT_SEPARATE = 0,
  /* Pilot and data share one frame: the pilot sits at (K0, L0) inside a guard band of
   * delay offsets [-guard, guard] (all Doppler bins) carrying no data; the read-off
   * covers delay offsets [0, guard] and the pilot's response H (a_pilot e_(K0,L0)) is
   * subtracted before equalisation.  Not in the paper. */
  ZOTFS_PILOT_EMBEDDED = 1
} zotfs_pilot_mode;

/* Per-plan options.  zotfs_plan_create fills the defaults given here. */
typedef struct zotfs_options {
  int32_t pilot_mode;  /* zotfs_pilot_mode, default ZOTFS_PILOT_SEPARATE */
  int32_t K0, L0;      /* pilot position; default (M/2, N/2) (Sec. III-B "Channel Estimation") */
  float   a_pilot;     /* pilot amplitude divided out of the read-off; default sqrt(MN)
                          (a pilot frame with the energy of a data frame), 0.5 sqrt(MN) when
                          embedded */
  int32_t guard;       /* embedded mode: guard half-width in delay bins; default 2 */
  int32_t p_max;       /* path-list capacity per antenna pair, 1..256; default 64 */
  int32_t in_dtype;    /* zotfs_dtype of TD input frames; default ZOTFS_C64 */
  int32_t tap_dtype;   /* zotfs_dtype of path taps in zotfs_paths; default ZOTFS_C64 */
  int32_t compute;     /* zotfs_compute; default ZOTFS_COMPUTE_FP32 */
  float   cg_eps;      /* residual-norm stopping test of the CG (the original CGA's test that
                          Sec. IV-C describes, relative form): a frame stops iterating once
                          ||c||^2 <= cg_eps^2 ||b||^2, evaluated in FP64 inside the frame's
                          kernel (no host round trip); the iteration count stays the cap.
                          Default 0: no test, the fixed iteration count of Algorithm 1.  Must
                          be finite and >= 0.  zotfs_equalize_static ignores it. */
} zotfs_options;

typedef struct zotfs_plan_s* zotfs_plan;

/* Device-resident path lists (the structured-sparse channel of Sec. IV-B, reduced to
 * the P dominant taps {h_p, k_p - K0, l_p - L0}).  n_lists = n_frames * n_rx * n_tx,
 * ordered [frame][rx][tx].  Entries of list i occupy [i*p_max, i*p_max + count[i]) and
 * are sorted by ascending pilot-grid index q = l_p*M + k_p. */
typedef struct zotfs_paths {
  int32_t* count;   /* dev [n_lists]: number of paths P <= p_max */
  int32_t* status;  /* dev [n_lists]: ZOTFS_OK or ZOTFS_ETRUNCATED; may be NULL on input */
  int16_t* dk;      /* dev [n_lists*p_max]: delay offset k_p - K0, in [-M/2, M/2) */
  int16_t* dl;      /* dev [n_lists*p_max]: Doppler offset l_p - L0, in [-N/2, N/2) */
  void*    h;       /* dev [n_lists*p_max] complex taps h_p, element type tap_dtype */
  int32_t  p_max;   /* capacity per list (must equal the plan's p_max) */
  int32_t  tap_dtype;
} zotfs_paths;

/* ---------------------------------------------------------------- plans ------------ */

/* Create a plan for frames of M delay x N Doppler bins, n_rx x n_tx antennas and square
 * Gray QAM of order qam (4, 16 or 64).  M and N are powers of two, 16 <= M <= 16384,
 * 8 <= N <= 64, n_rx, n_tx in [1, 4].  Frames with M <= 256 and M N <= 16384 run one per CTA
 * (or per thread-block cluster); larger frames, up to the paper's (16384, 32) operating point
 * (M N <= 524288, M >= 32), must be SISO, run one at a time on the whole GPU (a cooperative
 * launch), take separate pilot frames and FP32 compute, and have no plain form
 * (ZOTFS_EUNSUPPORTED).  Builds the root-of-unity tables (FP64 on the host, stored FP32)
 * and the plan's scratch.  The only allocating calls are the create calls (and the
 * autotuner); when an allocation fails they free what they had allocated and return
 * ZOTFS_ENOMEM.  *out is set to NULL on failure. */
zotfs_status zotfs_plan_create(int M, int N, int n_rx, int n_tx, zotfs_pulse pulse, int qam,
                               zotfs_plan* out);
zotfs_status zotfs_plan_set_options(zotfs_plan plan, const zotfs_options* opts);
zotfs_status zotfs_plan_get_options(zotfs_plan plan, zotfs_options* opts);
zotfs_status zotfs_plan_destroy(zotfs_plan plan);

/* Kernel launch shape for the fused per-frame kernels: threads per frame (a multiple of
 * M dividing M*N, 32..1024) and the FFT radix (2 or 4) of the in-shared-memory Zak
 * transform.  0 keeps the library's choice.  Used by the autotuner. */
typedef struct zotfs_tuning {
  int32_t threads_per_frame;
  int32_t fft_radix;
  int32_t ctas_per_sm;  /* resident CTAs per SM the persistent grid is sized for; 0 = max */
  int32_t cluster;      /* CTAs of a thread-block cluster per frame, for plans with separate
                           pilot frames (an embedded-pilot plan runs one CTA per frame):
                           SISO frames whose extension replica fits one CTA's shared memory
                           run on the cluster receiver (replicas in shared memory, the CG
                           vectors exchanged through distributed shared memory); equalisation
                           of frames too large for the one-CTA shared-memory kernel otherwise
                           runs on the clustered large-frame kernel (vectors in one global
                           scratch slot per cluster).  2 or 4: that many CTAs wherever one of
                           them applies.  0: only frames too large for the one-CTA kernel --
                           the cluster receiver (2 CTAs) when the call has at most one frame
                           per two SMs, else the clustered large-frame kernel, 4 CTAs when the
                           call has at most one frame per four SMs and 2 otherwise (MIMO
                           frames only: loaded SISO calls keep one CTA per frame).  1: never */
  int32_t frames_per_cta;  /* frames of the one-CTA shared-memory kernel packed into one CTA, each
                              on its own threads_per_frame threads and slice of shared memory with
                              its own barriers (0 or 1: one; at most 8, reduced to what the
                              kernel's thread limit and the SM's shared memory allow) */
} zotfs_tuning;
zotfs_status zotfs_plan_set_tuning(zotfs_plan plan, const zotfs_tuning* tuning);
zotfs_status zotfs_plan_get_tuning(zotfs_plan plan, zotfs_tuning* tuning);

/* ---------------------------------------------------------- hot-path stages -------- */

/* Discrete Zak transform, Eq. zak: Y[k,l] = N^-1/2 sum_{n<N} y[k+nM] e^{-j2pi nl/N}.
 * y_td: dev [n_grids][MN] of the plan's in_dtype.  y_dd: dev [n_grids][MN] ZOTFS_C64.
 * Radix-2/4 FFT along the Doppler axis in shared memory. */
zotfs_status zotfs_dzt(zotfs_plan plan, const void* y_td, float* y_dd, int n_grids,
                       zotfs_stream stream);

/* Channel estimation: Zak transform of each received pilot frame, read-off of
 * the effective channel (Eq. heff, in its Hadamard form Eq. heff_hadamard, divided by
 * a_pilot), thresholding |h_eff| > theta (Eq. heff_thres) and stable compaction into a
 * path list.  When more than p_max taps pass, the p_max largest magnitudes are kept
 * (ties to the lower q) and the list's status is ZOTFS_ETRUNCATED.
 * y_pilot_td: dev, separate mode [n_frames][n_tx][n_rx][MN]; embedded mode the data
 *             frames [n_frames][1][1][MN].  theta: dev float [n_frames].
 * paths:      host struct of dev pointers, written for n_frames*n_rx*n_tx lists. */
zotfs_status zotfs_estimate(zotfs_plan plan, const void* y_pilot_td, const float* theta,
                            int n_frames, const zotfs_paths* paths, zotfs_stream stream);

/* Structured-sparse operator apply (Eq. sparse_mvm / Eq. sparse_herm_mvm with the
 * index maps Eq. map_chMatDD_col / Eq. herm_mapping and the twisted phase of Sec. IV-B):
 *   adjoint == 0: u = H v,   v dev [n_frames][n_tx][MN] C64, u dev [n_frames][n_rx][MN] C64
 *   adjoint != 0: u = H^H v, v dev [n_frames][n_rx][MN] C64, u dev [n_frames][n_tx][MN] C64
 * Each path's quasi-periodic wrap count and phase are computed on the fly from the path
 * list; no dense or per-entry matrix is formed.  status: dev int32 [n_frames] or NULL. */
zotfs_status zotfs_ss_apply(zotfs_plan plan, const zotfs_paths* paths, const float* v, float* u,
                            int adjoint, int n_frames, int32_t* status, zotfs_stream stream);

/* LMMSE equalisation by the compute-aware CGA (Algorithm 1): b = H^H y, then
 * `iters` fixed iterations of {a = H^H H p + lambda p; alpha = c_n / Re(p^H a); x += alpha p;
 * c -= alpha a; p = c + (c_n'/c_n) p}, lambda = noise_var[f].  Vectors stay in shared
 * memory; alpha and beta are formed in FP64.  Readings: alpha = 0 when Re(p^H a) = 0 and
 * beta = 0 when c_n = 0.
 * y:         dev data frames, TD [n_frames][n_rx][MN] in the plan's in_dtype when
 *            y_is_dd == 0, else DD [n_frames][n_rx][MN] C64 (embedded mode: TD only).
 * noise_var: dev float [n_frames].  x_hat: dev [n_frames][n_tx][MN] C64.
 * status:    dev int32 [n_frames] or NULL. */
zotfs_status zotfs_equalize(zotfs_plan plan, const void* y, int y_is_dd, const zotfs_paths* paths,
                            const float* noise_var, int iters, float* x_hat, int n_frames,
                            int32_t* status, zotfs_stream stream);

/* SS-MRC equalisation (Sec. III-B "Equalization", the maximal-ratio-combining paragraph; SS-MRC
 * of the evaluation): the decision-feedback MRC equaliser on the structured-sparse path list.
 * Per iteration the delay bins k = 0 .. M-1 are visited in order; the symbol vector of bin k
 * (all N Doppler bins) collects its components from every delay branch (the paths of one
 * delay offset) of the residual y - H x_hat, with the current estimates of the other vectors
 * cancelled, combines them with the conjugate branch gains normalised by their total power,
 * and is decided to the nearest points of the plan's QAM (Eq. demod), which are fed back into
 * the residual.  The combining runs on the delay-time grid (the DD grid's Doppler axis taken
 * back to time), where every branch is a diagonal gain and a cyclic time shift.  No noise
 * term enters (maximal ratio); `iters` sweeps, iters = 0 returns x_hat = 0.
 * x_hat receives the soft estimate of the last sweep (before the decision), which
 * zotfs_demap turns into LLRs and hard bits.  One warp per frame, FP32.
 *   Plans: SISO, FP32, separate pilot frames, M <= 256, M*N <= 16384, p_max <= 256, else
 *   ZOTFS_EUNSUPPORTED.
 *   y:      dev data frames, TD [n_frames][MN] in the plan's in_dtype when y_is_dd == 0, else
 *           DD [n_frames][MN] C64.
 *   paths:  host struct of dev pointers, one list per frame (as for zotfs_equalize).
 *   x_hat:  dev [n_frames][MN] C64 (may be NULL).  status: dev int32 [n_frames] or NULL:
 *           ZOTFS_OK, ZOTFS_EINVAL (bad count or offset; such entries are dropped) or
 *           ZOTFS_ENONFINITE. */
zotfs_status zotfs_equalize_mrc(zotfs_plan plan, const void* y, int y_is_dd, const zotfs_paths* paths, int iters,
                                float* x_hat, int32_t* status, int n_frames, zotfs_stream stream);

/* Demapping (Eq. demod extended to soft output): per bit j the max-log LLR
 * (min_{s: b_j=1} |x-s|^2 - min_{s: b_j=0} |x-s|^2) / noise_var[f] over the plan's Gray
 * square QAM with unit mean energy, and the hard bit (LLR < 0).  llr (dev float
 * [n_frames][n_tx][MN][bps]) and bits (dev uint8 [n_frames][n_tx][MN*bps/8]) may each be
 * NULL.  x_hat: dev [n_frames][n_tx][MN] C64. */
zotfs_status zotfs_demap(zotfs_plan plan, const float* x_hat, const float* noise_var, float* llr,
                         uint8_t* bits, int n_frames, zotfs_stream stream);

/* Self-check of the device-side failure detection: runs one of the library's bounded waits
 * against a condition nothing satisfies -- which = 0: the mbarrier wait of the frame
 * kernels' bulk copies with no copy issued; 1: the grid barrier of the paper-scale receiver
 * with one of two CTAs leaving without arriving -- and writes the outcome to *status (dev
 * int32): ZOTFS_ETIMEOUT once the wait gave up after max_polls polls (1 .. 2^24).  Nothing
 * traps or hangs; the context stays usable. */
zotfs_status zotfs_check_bounded_wait(int which, uint32_t max_polls, int32_t* status, zotfs_stream stream);

/* Self-check of the CG's scalar division: q[i] = (float) of alpha-style ratio a[i] / b[i] as the
 * FP32 kernels form it (FP64, by one Newton-Raphson step on the FP32 reciprocal of b, or a full
 * division when float(b) is not a normal number; 0 when b = 0), for n pairs.  a, b: dev double
 * [n]; q: dev float [n].  For testing the kernels' arithmetic against IEEE division. */
zotfs_status zotfs_check_cg_ratio(const double* a, const double* b, float* q, int n, zotfs_stream stream);

/* Host-side fault injection for tests of the allocation-failure paths: with after = n >= 0,
 * the library's next n device or pinned-host allocations (any call, any thread) succeed and
 * the one after fails as if the device were out of memory; that call then returns
 * ZOTFS_ENOMEM having freed what it had allocated, and the injection switches itself off.
 * after = -1 switches it off.  No device work is done; ZOTFS_EINVAL for after < -1. */
zotfs_status zotfs_debug_fail_alloc(int after);

/* Data frames equalised and demapped with path lists estimated earlier (pilot reuse: one
 * pilot frame's lists serve the data frames of its packet, which Sec. III-B sizes by the
 * channel coherence time).  Data frame f uses list set path_ids[f] of the
 * n_sets sets in `paths` (dev int32 [n_frames]; NULL: set f, and n_sets >= n_frames); a
 * frame whose id is outside [0, n_sets) gets status ZOTFS_EINVAL.  Fused like zotfs_rx: data
 * Zak transform -> CGA (`iters`, lambda = noise_var[f]) -> demapping, one frame per CTA
 * (or cluster, or the whole GPU for paper-scale grids).
 * y_data_td: dev TD [n_frames][n_rx][MN] in the plan's in_dtype.  x_hat, llr may be NULL;
 * bits: dev uint8 [n_frames][n_tx][MN*bps/8]; status: dev int32 [n_frames] (required). */
zotfs_status zotfs_rx_lists(zotfs_plan plan, const void* y_data_td, const zotfs_paths* paths,
                            const int32_t* path_ids, int n_sets, const float* noise_var, int iters,
                            float* x_hat, float* llr, uint8_t* bits, int32_t* status, int n_frames,
                            zotfs_stream stream);

/* The whole receiver fused: per frame in one persistent kernel whose CTAs pull
 * frames from a device work counter: pilot Zak transforms and read-off -> path lists in
 * shared memory -> data Zak transform -> CGA -> demapping.  HBM traffic is the TD
 * frames in and the results out.  Outputs paths, x_hat and llr may be NULL (bits too,
 * but then nothing is returned but status).  status: dev int32 [n_frames] (required). */
zotfs_status zotfs_rx(zotfs_plan plan, const void* y_pilot_td, const void* y_data_td,
                      const float* noise_var, const float* theta, int iters,
                      const zotfs_paths* paths, float* x_hat, float* llr, uint8_t* bits,
                      int32_t* status, int n_frames, zotfs_stream stream);

/* The plain form: the same receiver run one frame at a time with one kernel launch per
 * stage and per CG step (Zak transform, read-off, compaction, b = H^H y, and per iteration
 * H p, H^H t + lambda p, two inner products, the x/c update and the p update), vectors in
 * the plan's global scratch, FP32.  It is the comparison baseline for zotfs_rx, with the
 * same arguments and results. */
zotfs_status zotfs_rx_plain(zotfs_plan plan, const void* y_pilot_td, const void* y_data_td,
                            const float* noise_var, const float* theta, int iters,
                            const zotfs_paths* paths, float* x_hat, float* llr, uint8_t* bits,
                            int32_t* status, int n_frames, zotfs_stream stream);

/* Equalisation that allocates nothing, for callers that must not allocate device memory
 * while they run: a real-time receive loop working to a slot deadline (cudaMalloc and
 * cudaFree synchronise the device and can stall it for milliseconds), or a process whose
 * device memory is fully budgeted up front (an allocation made behind the budget's back can
 * fail, or push another part of the process out of memory).  It needs no plan.  The paper
 * has no counterpart: this is the plain-form CGA of zotfs_rx_plain (b = H^H y and `iters`
 * iterations of Algorithm 1, one kernel per step, FP32 with FP64 alpha/beta) with its
 * working vectors and root-of-unity table in one fixed 768 KiB array inside the library
 * image.  Every GPU that loads the library holds that array until the process exits.
 *   Limits: M*N <= 4096, n_rx, n_tx <= 4, path taps ZOTFS_C64 with p_max <= 64; larger
 *   problems return ZOTFS_EUNSUPPORTED and nothing runs.
 *   paths:     host struct of dev pointers, lists [frame][rx][tx] as for zotfs_equalize.
 *   y_dd:      dev DD grids [n_frames][n_rx][MN] C64;  noise_var: dev float [n_frames].
 *   x_hat:     dev [n_frames][n_tx][MN] C64;  status: dev int32 [n_frames] or NULL: per frame
 *              ZOTFS_OK, ZOTFS_EINVAL (a count outside [0, p_max] or an offset outside the
 *              centred range; such entries are dropped) or ZOTFS_ENONFINITE.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the one array -- vectors, path
 * records, flags and the root-of-unity table, which each call rewrites -- and it keeps what
 * the last call left there (each call re-initialises everything it reads), so calls whose
 * work can overlap on the GPU -- on different streams, or from different threads -- race
 * with each other: keep them on one stream. */
zotfs_status zotfs_equalize_static(int M, int N, int n_rx, int n_tx, const zotfs_paths* paths, const float* y_dd,
                                   const float* noise_var, int iters, float* x_hat, int32_t* status, int n_frames,
                                   zotfs_stream stream);

/* ------------------------------------------------------ uneven persistent batch ---- */

/* One frame of an uneven batch: its own shape, antennas, QAM order, noise and threshold,
 * and its own device buffers (layouts as above with n_frames = 1). */
typedef struct zotfs_frame_desc {
  int32_t M, N, n_rx, n_tx, qam, iters;
  int32_t pilot_mode, guard, p_max, in_dtype;
  int32_t K0, L0;           /* -1: M/2, N/2 */
  float   noise_var, theta, a_pilot;  /* a_pilot <= 0: the plan default for the mode */
  float   cg_eps;           /* CG stopping test as zotfs_options.cg_eps; 0: fixed iterations */
  const void* y_pilot;      /* dev TD pilots (separate mode) */
  const void* y_data;       /* dev TD data frames */
  float*   x_hat;           /* dev or NULL */
  float*   llr;             /* dev or NULL */
  uint8_t* bits;            /* dev or NULL */
  int32_t* path_count;      /* dev [n_rx*n_tx] or NULL: the estimated path lists ... */
  int16_t* path_dk;         /* ... dev [n_rx*n_tx*p_max] */
  int16_t* path_dl;
  float*   path_h;          /* dev [n_rx*n_tx*p_max] C64 */
} zotfs_frame_desc;

typedef struct zotfs_batch_s* zotfs_batch;

/* Launch shape for one bucket of an uneven batch (frames of equal M, N, n_rx, n_tx). */
typedef struct zotfs_tuning_entry {
  int32_t M, N, n_rx, n_tx;
  zotfs_tuning tuning;
} zotfs_tuning_entry;

typedef struct zotfs_batch_opts {
  int32_t threads_per_frame;  /* 0: per-bucket choice (tuning table entry, else the library's) */
  int32_t ctas_per_sm;        /* 0: as many as fit */
  int32_t fft_radix;          /* 0: per-bucket choice, else 2 or 4 */
  int32_t n_tuning;           /* entries in `tuning` (host array, read during create only) */
  const zotfs_tuning_entry* tuning;
  int32_t max_sms;            /* SMs the batch's grids are sized for; 0: all of the device's */
  int32_t cluster;            /* frames too large for one CTA's shared memory (separate pilot
                                 frames): 0 per-bucket choice (tuning entry, else 2-CTA
                                 clusters for MIMO buckets, one CTA per SISO frame), 1 one CTA
                                 per frame, 2 or 4 CTAs of a cluster per frame; other values
                                 are ZOTFS_EINVAL */
} zotfs_batch_opts;

/* Build a batch from host descriptors: validates every frame, groups frames into buckets
 * of equal (M, N, n_rx, n_tx, qam, pilot mode, p_max, in_dtype), uploads the descriptors
 * and the per-shape root-of-unity tables, and sizes each bucket's persistent grid in
 * proportion to its share of the batch's work so all buckets run side by side.
 * Descriptors hold device pointers that must stay valid while the batch is used.
 * Allocates. */
zotfs_status zotfs_batch_create(const zotfs_frame_desc* descs, int n_frames,
                                const zotfs_batch_opts* opts, zotfs_batch* out);
/* Run the batch: one persistent frame kernel per bucket, forked from `stream` onto the
 * batch's own streams and joined back (events), stream-ordered, no allocation and no host
 * synchronisation, so it can be captured in a CUDA graph.  status: dev int32 [n_frames]
 * in descriptor order.  One batch must not run on two streams at once. */
zotfs_status zotfs_rx_batch(zotfs_batch batch, int32_t* status, zotfs_stream stream);
zotfs_status zotfs_batch_destroy(zotfs_batch batch);

/* ------------------------------------------------- CUDA graphs and autotuning ---- */

/* An instantiated CUDA graph of one batch run (the persistent kernel of every bucket, with
 * its counter reset and the fork/join between the batch's streams).  Replaying it costs one
 * graph launch instead of a memset, a kernel launch and two events per bucket.  Not in the
 * paper. */
typedef struct zotfs_graph_s* zotfs_graph;

/* Capture zotfs_rx_batch(batch, status, .) on a private stream (thread-local capture mode)
 * and instantiate it.  The batch, its descriptors' buffers and `status` must outlive the
 * graph; the batch must not run elsewhere while the graph runs.  Allocates. */
zotfs_status zotfs_batch_capture(zotfs_batch batch, int32_t* status, zotfs_graph* out);
/* Replay the graph on `stream` (stream-ordered, no host synchronisation). */
zotfs_status zotfs_graph_launch(zotfs_graph graph, zotfs_stream stream);
zotfs_status zotfs_graph_destroy(zotfs_graph graph);

typedef struct zotfs_autotune_opts {
  int32_t warmup;      /* untimed runs per candidate; 0: 2 */
  int32_t reps;        /* timed runs per candidate; 0: 5 */
  int32_t max_frames;  /* frames of each shape group used for timing; 0: all */
} zotfs_autotune_opts;

typedef struct zotfs_tuning_result {
  zotfs_tuning_entry best;  /* the fastest launch shape of one (M, N, n_rx, n_tx) group */
  float ms_best;            /* mean time of one run of the group's frames with it */
  float ms_default;         /* the same with the library's default launch shape */
  float sm_ms_per_frame;    /* ms_best x SMs / frames timed: the group's measured cost */
  int32_t n_candidates;     /* launch shapes timed */
  int32_t n_frames;         /* frames in the group's timing set (repeats included) */
} zotfs_tuning_result;

/* The autotuner.  Groups `descs` by (M, N, n_rx, n_tx); for each group enumerates every
 * launch shape that fits -- threads per frame (M <= T, T | MN, one of the compiled rows-per-
 * thread variants), FFT radix 2 or 4, and CTAs per SM from 1 to the occupancy limit (the
 * number of frames each SM works on at once) -- and times `reps` runs of each with CUDA
 * events on `stream` after `warmup` runs.  Each group is timed in the throughput regime of a
 * large batch: its frames (the first max_frames of them) are repeated to 8 frames per SM,
 * reading the caller's received frames and writing hard bits to the tuner's own scratch, so
 * the descriptors' outputs are not touched.  Returns the fastest shape per group, with its
 * cost in SM-milliseconds per frame, in out[0 .. *n_out) (at most max_out groups;
 * ZOTFS_EINVAL if there are more); the entries go into zotfs_batch_opts.tuning.
 * Synchronises `stream`; allocates. */
zotfs_status zotfs_autotune(const zotfs_frame_desc* descs, int n_frames, const zotfs_autotune_opts* opts,
                            zotfs_tuning_result* out, int max_out, int* n_out, zotfs_stream stream);

/* ------------------------------------------------------------------- serving ---- */

/* A request loop on one GPU with continuous batching.  Frames of mixed shapes, antenna
 * counts and QAM orders are submitted as they arrive (their received pilot and data frames
 * already in device memory).  A scheduler thread owned by the server admits pending frames
 * into "waves" whenever a wave slot is free and the device output arena has room for their
 * results, and launches each wave's frames (grouped by shape) on the wave's own streams, so
 * frames admitted while earlier waves run overlap with them on the device.  A frame's
 * outputs -- hard bits, optionally LLRs, and its path lists -- stay resident in the arena
 * until the caller releases it.  Not in the paper (which processes one packet at a time). */
typedef struct zotfs_server_s* zotfs_server;

typedef struct zotfs_server_opts {
  int32_t p_max;            /* path-list capacity of every frame (1..256) */
  int32_t max_wave_frames;  /* frames admitted per wave, 1..4096 */
  int32_t waves_in_flight;  /* concurrent waves, 1..16; each holds its own scratch (large-frame
                               slots for every SM); more waves let the heavy buckets of
                               consecutive waves run side by side (16 measured best on mixed
                               loads) */
  int32_t keep_llr;         /* also keep float32 LLRs per frame */
  int64_t arena_bytes;      /* device bytes for admitted frames' outputs */
  int32_t max_M, max_N, max_ant;  /* largest frame accepted (sizes the large-frame scratch) */
  int32_t light_work;       /* > 0: frames with M*N*n_rx*n_tx <= light_work queue and run in
                               their own waves (the first half of the wave slots), so frames
                               that take long never hold a wave slot that short ones wait for;
                               0: one queue */
} zotfs_server_opts;

typedef struct zotfs_request {
  int32_t M, N, n_rx, n_tx, qam, iters;
  float noise_var, theta, a_pilot;  /* a_pilot <= 0: sqrt(MN) */
  float cg_eps;                     /* CG stopping test as zotfs_options.cg_eps; 0: off */
  const void* y_pilot;              /* dev C64 pilots [t][r][MN], resident until completion */
  const void* y_data;               /* dev C64 data [r][MN] */
  uint64_t tag;                     /* caller's id, unique among frames not yet released */
} zotfs_request;

typedef struct zotfs_completion {
  uint64_t tag;
  int32_t status;                   /* zotfs_status of the frame */
  int32_t n_lists;                  /* n_rx * n_tx */
  int64_t arrival_ns, admit_ns, done_ns;  /* steady-clock times: submit, wave launch, observed done */
  const uint8_t* bits;              /* dev [n_tx][MN*bps/8], valid until zotfs_server_release */
  const float* llr;                 /* dev [n_tx][MN][bps] or NULL */
  const int32_t* path_count;        /* dev [n_lists] */
  const int16_t* path_dk;           /* dev [n_lists][p_max] */
  const int16_t* path_dl;
  const float* path_h;              /* dev [n_lists][p_max] C64 */
} zotfs_completion;

typedef struct zotfs_server_stats {
  int64_t submitted, admitted, completed, released, pending, waves;
  int64_t arena_bytes, arena_in_use, arena_high_water;
  int64_t rejected_too_large;       /* requests whose outputs can never fit the arena */
} zotfs_server_stats;

/* Create a server on the current device.  Allocates the arena, the per-wave streams, events,
 * descriptor buffers and large-frame scratch, and the root-of-unity tables of every shape
 * up to (max_M, max_N).  Starts the scheduler thread. */
zotfs_status zotfs_server_create(const zotfs_server_opts* opts, zotfs_server* out);
/* Queue n requests (thread-safe, never blocks on the GPU; copies the request structs). */
zotfs_status zotfs_server_submit(zotfs_server server, const zotfs_request* reqs, int n);
/* Load generator: submit reqs[i] at time arrival_s[i] (seconds, non-decreasing) after the
 * call starts, spinning on the steady clock; returns once all are submitted. */
zotfs_status zotfs_server_replay(zotfs_server server, const zotfs_request* reqs, const double* arrival_s, int n);
/* Copy up to max completed frames (oldest first) into out; returns how many. */
int zotfs_server_poll(zotfs_server server, zotfs_completion* out, int max);
/* Copy a completed, unreleased frame's outputs to host memory (synchronous; any destination
 * may be NULL): bits [n_tx][MN*bps/8], llr [n_tx][MN][bps] (if kept), and the path lists
 * count [n_lists], dk/dl [n_lists][p_max], h [n_lists][p_max] C64. */
zotfs_status zotfs_server_read(zotfs_server server, uint64_t tag, uint8_t* bits, float* llr, int32_t* path_count,
                               int16_t* path_dk, int16_t* path_dl, float* path_h);
/* Return a completed frame's outputs to the arena. */
zotfs_status zotfs_server_release(zotfs_server server, uint64_t tag);
zotfs_status zotfs_server_get_stats(zotfs_server server, zotfs_server_stats* stats);
/* Stop admitting, wait for in-flight waves, stop the scheduler, free everything. */
zotfs_status zotfs_server_destroy(zotfs_server server);

/* ----------------------------------------------------------------- misc ------------ */

/* Thread-local message for the most recent failure in this thread ("" if none). */
const char* zotfs_last_error(void);
/* Number of fused-kernel launches (CTAs grids) the most recent call in this thread made. */
int zotfs_last_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ZOTFS_H */
