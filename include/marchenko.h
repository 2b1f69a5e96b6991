/*
 * marchenko.h - C ABI of the GB300 iterative Marchenko synthesis library.
 *
 * The library runs the hot loop of iterative Marchenko redatuming on one GPU:
 * per Neumann iteration the synthesis of Eq. (1),
 *     N_i(x_R, x_F, -t) = theta_t * integral_x integral_t' R(x_R, x, t - t') N_{i-1}(x, x_F, t') dt' dx,
 * done in the frequency domain (Theory section: the time convolution is a
 * per-frequency product, the space integral a sum over surface positions),
 * followed by the time reversal and sign flip, the theta mute and the
 * accumulation of f1+, f1-, f2 and p- (Algorithm 1, both loops fused into
 * one pass per iteration).  Every step runs in this library's CUDA kernels.
 *
 * Conventions (shared by every entry point):
 *  - sources and receivers coincide: nsrc == nrec == n positions x_i = i*dx;
 *  - circular time grid of nt samples (nt a power of two, 32..8192); sample j
 *    has signed time j*dt for j < nt/2 and (j - nt)*dt otherwise;
 *    X(-t)[j] = X[(nt - j) mod nt];
 *  - forward DFT unnormalised (kernel e^{-2 pi i jm/nt}), inverse 1/nt;
 *  - kept band m = 0 .. n_w-1 with n_w = min(nt/2, floor(fmax_hz * nt * dt)) + 1
 *    (FP64, evaluated left to right); fmax_hz <= 0 keeps the full band; bins
 *    outside the band are zero before every inverse transform, and the
 *    imaginary parts of the DC and Nyquist bins do not enter a real trace;
 *  - synthesis scale c = dx * dt (Riemann sums of both integrals):
 *        S_m(k, f) = c * sum_r R_m(k, r) * N_m(r, f),  s = IDFT(S);
 *  - N_i = -theta * s(-t) (Algorithm 1: time-reverse, multiply by -1, mute);
 *    theta_k(j) = 1 iff |t_j| < t_d(f, x_k) - eps (FP64 comparison
 *    j*dt < t_d - eps, exactly as written), symmetric in +-t;
 *  - accumulation per iteration index i (0-based, Algorithm 1):
 *        pmin += s;  f2p += N_i;  i even: f1min -= N_i(-t);  i odd: f1plus += N_i;
 *    initial values N_{-1} = f1plus = f2p = G_d(-t), f1min = pmin = 0;
 *  - G(t) = f2p(-t) + pmin(t).
 *
 * Layouts (row-major, last index fastest):
 *  - R band spectra passed to mk_load_R: complex64 (float re, float im)
 *    [w_count][nsrc][nrec], R[m][k][r] = R(x_R = x_k, x = x_r, f_m); the
 *    contraction sums over the last (receiver) axis, which by reciprocity
 *    R(x_k, x_r) = R(x_r, x_k) is the space integral of Eq. (1);
 *  - G_d: float [nfocal][nrec][nt], the first arrival G_d(x_r, x_F, t);
 *  - t_d: double [nfocal][nrec], first-arrival times in seconds;
 *  - every field: float [nfocal][nsrc][nt].
 *
 * Memory and ownership:
 *  - the plan allocates no device memory: the caller passes one device
 *    workspace of at least mk_workspace_size() bytes (256-byte aligned) to
 *    mk_plan and keeps it alive until mk_destroy;
 *  - input and output buffers belong to the caller and need to stay valid
 *    only during the call (the library copies from and to them);
 *  - all GPU work is issued on the stream given to mk_plan.  Calls that read
 *    host memory or write host outputs return after that work is complete;
 *    calls on device buffers only are asynchronous on the stream; mk_load_R
 *    also takes page-locked host memory asynchronously (MK_SRC_HOST_ASYNC:
 *    the caller keeps the buffer unchanged until the stream has passed the
 *    copy, e.g. until the next call that returns host results);
 *  - a plan is not thread-safe: one host thread at a time per plan.
 *
 * Errors: every entry point returns mk_status and never aborts.  The message
 * of the last failure is returned by mk_last_error(plan) (plan may be NULL
 * for failures that happen before a plan exists); the string stays valid
 * until the next call on the same plan (or on any NULL-plan call).
 */
#ifndef MARCHENKO_H
#define MARCHENKO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mk_plan_s* mk_plan_t;

typedef enum {
  MK_OK = 0,
  MK_ERR_ARG = 1,          /* invalid argument (null pointer, size, index)   */
  MK_ERR_STATE = 2,        /* call out of order (e.g. iterate before G_d)    */
  MK_ERR_OOM = 3,          /* workspace too small                            */
  MK_ERR_CUDA = 4,         /* a CUDA runtime call failed                     */
  MK_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out             */
  MK_ERR_UNSUPPORTED = 6   /* valid request the library does not support      */
} mk_status;

/* Storage precision of R in the workspace. */
typedef enum {
  MK_R_C64 = 0,        /* complex FP32                                        */
  MK_R_CBF16 = 1,      /* complex BF16 (tensor-core contraction)              */
  MK_R_CF16 = 2,       /* complex FP16 (tensor-core contraction)              */
  MK_R_SPLIT_BF16 = 3, /* BF16 hi + BF16 lo parts (3-product tensor-core form) */
  MK_R_SPLIT3_BF16 = 4, /* BF16 hi + mid + lo parts (6-product form, FP32-like) */
  MK_R_SPLIT_F16 = 5    /* FP16 hi + lo parts of R and of the field, each scaled by a
                           power of two (R per frequency, the field per frequency
                           and focal point) into FP16's normal range: about 22
                           significant bits per operand with 3 products (hh, hl,
                           lh); loaded with mk_load_R only                    */
} mk_rprec;

/* Field selection bits for mk_fetch_fields (output order = bit order). */
#define MK_F_N    (1u << 0) /* the last N_i (N_{-1} before any iteration)  */
#define MK_F_F1P  (1u << 1) /* f1plus                                      */
#define MK_F_F1M  (1u << 2) /* f1min                                       */
#define MK_F_F2P  (1u << 3) /* f2p                                         */
#define MK_F_PMIN (1u << 4) /* pmin                                        */
#define MK_F_G    (1u << 5) /* G = f2p(-t) + pmin(t)                       */
#define MK_F_GMINUS (1u << 6) /* G^- = synthesis(f1plus) - f1min          */
#define MK_F_GPLUS  (1u << 7) /* G^+ = f1plus(-t) - synthesis(f1min(-t))  */
#define MK_F_ALL  (0xFFu)

/* mk_desc.flags */
#define MK_FLAG_TIMING (1u << 0) /* record CUDA events around every kernel   */
/* where a source buffer lives (the src_on_device argument) */
#define MK_SRC_HOST 0       /* host memory; read before the call returns     */
#define MK_SRC_DEVICE 1     /* device memory                                 */
#define MK_SRC_HOST_ASYNC 2 /* page-locked host memory, read in stream order */

#define MK_FLAG_AUTOTUNE (1u << 3) /* time the candidate tile shapes of the
                                    survey's kernels at its first
                                    mk_set_Gd_window and keep the fastest
                                    (see mk_get_tuning)                     */
#define MK_FLAG_STREAM_R (1u << 2) /* keep R in pinned host memory and stream it
                                    every contraction (complex FP32 only; see
                                    mk_attach_R_host); a plan holding such a
                                    survey launches its iterations on streams
                                    (MK_FLAG_GRAPH is not applied)          */
#define MK_FLAG_GRAPH  (1u << 1) /* replay iterations as one captured CUDA graph
                                    (all surveys' kernels on parallel branches);
                                    used when every survey sets it and none
                                    sets MK_FLAG_TIMING                     */

/* One survey.  nsrc == nrec is required (coincident sources/receivers).
 *
 * Shot-row sharding (the paper's multi-GPU split, Implementation section:
 * each GPU takes its own batch of shots): row_count > 0 makes the plan hold
 * only the output positions k = row_begin .. row_begin + row_count - 1 of the
 * survey -- their rows of every R_m, their traces of every field, their mute
 * windows -- while the field spectrum that the contraction sums over keeps
 * all nrec positions.  Each iteration then computes the new field spectrum
 * of the plan's own positions only; the caller completes it from the other
 * shards between iterations (mk_export_field_spectrum /
 * mk_import_field_spectrum, e.g. around an all-gather).  row_begin must be a
 * multiple of 32.  row_count = 0 holds every position (row_begin ignored). */
typedef struct {
  int32_t nsrc;     /* number of output positions k                          */
  int32_t nrec;     /* number of summed positions r                          */
  int32_t nt;       /* time samples, power of two in [32, 8192]               */
  int32_t nfocal;   /* focal points F >= 1                                    */
  double dt;        /* sample interval, s (> 0)                               */
  double dx;        /* position spacing, m (> 0)                              */
  double fmax_hz;   /* band limit (<= 0: full band)                           */
  int32_t rprec;    /* mk_rprec                                               */
  uint32_t flags;   /* MK_FLAG_*                                              */
  int32_t row_begin; /* first output position held (shot-row sharding)      */
  int32_t row_count; /* output positions held; 0: all of them               */
} mk_desc;

/* Counters of one plan (mk_get_stats). */
typedef struct {
  uint64_t launches;           /* kernels this plan launched                  */
  uint64_t contract_launches;  /* contraction launches (Eq. 1 space integral) */
  uint64_t epilogue_launches;  /* IFFT/mute/accumulate/FFT launches           */
  uint64_t other_launches;     /* init, G and conversion launches             */
  double contract_ms;          /* summed event time (MK_FLAG_TIMING only)     */
  double epilogue_ms;          /* summed event time (MK_FLAG_TIMING only)     */
  uint64_t contract_timed;     /* launches included in contract_ms            */
  uint64_t epilogue_timed;     /* launches included in epilogue_ms            */
} mk_stats_t;

/*
 * mk_workspace_size - device bytes a plan for these surveys needs.
 *   d, ndesc: ndesc >= 1 survey descriptions (validated as in mk_plan).
 *   bytes:    out, the size to allocate.
 * Errors: MK_ERR_ARG (null pointer, invalid description), MK_ERR_UNSUPPORTED.
 */
mk_status mk_workspace_size(const mk_desc* d, int32_t ndesc, size_t* bytes);

/*
 * mk_plan - create a plan for ndesc independent surveys (Algorithm 1, one
 * Neumann series per survey and focal point).
 *   cuda_stream: cudaStream_t the plan issues all its work on (NULL: legacy
 *                default stream).  The current device at this call is the
 *                plan's device; later calls must be made with it current.
 *   workspace:   device pointer, 256-byte aligned, >= mk_workspace_size bytes;
 *                zeroed and carved by the plan, owned by the caller.
 *   out:         receives the plan handle.
 * Errors: MK_ERR_ARG, MK_ERR_OOM (workspace_bytes too small),
 *         MK_ERR_UNSUPPORTED, MK_ERR_CUDA.
 */
mk_status mk_plan(const mk_desc* d, int32_t ndesc, void* cuda_stream, void* workspace,
                  size_t workspace_bytes, mk_plan_t* out);

/*
 * mk_load_R - load band spectra R_m for bins w_begin .. w_begin+w_count-1 of
 * one survey (Implementation section: the reflection data is read, Fourier
 * transformed and kept resident; here it is resident in HBM in the plan's
 * storage precision, rows padded for aligned loads).
 *   Rw: complex64 [w_count][nsrc][nrec] on the host (src_on_device =
 *       MK_SRC_HOST), on the device (MK_SRC_DEVICE), or in page-locked host
 *       memory read asynchronously in stream order (MK_SRC_HOST_ASYNC; the
 *       call returns once the copy is queued, MK_ERR_ARG if the memory is
 *       not page-locked).
 * Loading may be done in chunks of bins, in any order; mk_set_Gd_window
 * requires every bin 0 .. n_w-1 to have been loaded.  Loading R after
 * mk_set_Gd_window keeps the state of the series: the next mk_iterate
 * continues from it with the new R, and pmin (hence G) is formed at fetch
 * with the R loaded at that time (pmin = synthesis of f2p - N_last).
 * Errors: MK_ERR_ARG (bad survey index or bin range), MK_ERR_CUDA.
 */
mk_status mk_load_R(mk_plan_t plan, int32_t survey, const void* Rw, int32_t w_begin,
                    int32_t w_count, int32_t src_on_device);

/*
 * mk_load_R_time - load R from its time traces (Implementation section: the
 * reflection data is Fourier transformed once, before the iterations).  Each
 * trace R(k, r, t), t = 0 .. nt-1, is transformed with the forward DFT
 * R_m(k, r) = sum_j R(k, r, j) e^{-2 pi i j m / nt} (unnormalised) for the
 * band m < n_w and stored in the plan's storage precision, exactly as a
 * mk_load_R of those spectra (FP32 transform, FP64 twiddles).
 *   Rt: float [nsrc][nrec][nt] (source row k, receiver r, sample), on the
 *       host (src_on_device = 0; page-locked memory is read in place,
 *       pageable memory is staged nfocal source rows at a time) or on the
 *       device (1).
 * Loads every bin; replaces any earlier mk_load_R of this survey.
 * Errors: MK_ERR_ARG (bad survey, null), MK_ERR_STATE (streamed survey),
 *         MK_ERR_CUDA.
 */
mk_status mk_load_R_time(mk_plan_t plan, int32_t survey, const float* Rt, int32_t src_on_device);

/*
 * mk_attach_R_host - out-of-core R for a survey planned with MK_FLAG_STREAM_R
 * (the paper streams batches of shots to the GPUs when R exceeds their
 * memory, Algorithm 2; here frequency chunks are streamed every contraction
 * from page-locked host memory, double-buffered so that the copy of one
 * chunk overlaps the contraction of the previous one).
 *   Rpad:  page-locked host memory, complex64 [n_w][nsrc][r_pad] with
 *          r_pad = nrec rounded up to a multiple of 32 and the padding zero;
 *          the caller keeps it alive and unchanged until mk_destroy.
 *   bytes: n_w * nsrc * r_pad * 8.
 * Replaces mk_load_R for such surveys (mk_load_R returns MK_ERR_STATE).
 * Errors: MK_ERR_ARG (size, not pinned), MK_ERR_STATE, MK_ERR_CUDA.
 */
mk_status mk_attach_R_host(mk_plan_t plan, int32_t survey, const void* Rpad, size_t bytes);

/*
 * mk_set_Gd_window - start the Neumann series of one survey (Theory:
 * initialisation N_{-1} = f1+_0 = G_d(-t)): sets N_{-1} = f1plus = f2p =
 * G_d(-t), f1min = pmin = 0, the mute windows from t_d and eps, and the band
 * spectrum of N_{-1}; resets the iteration index to 0.
 *   Gd: float [nfocal][nrec][nt]; td: double [nfocal][nrec] (seconds); both
 *       on the host (src_on_device = 0) or both on the device (1).
 *   eps_s: window shift in seconds (theta keeps |t| < t_d - eps_s).
 * Errors: MK_ERR_ARG, MK_ERR_STATE (R not fully loaded), MK_ERR_CUDA.
 */
mk_status mk_set_Gd_window(mk_plan_t plan, int32_t survey, const float* Gd, const double* td,
                           double eps_s, int32_t src_on_device);

/*
 * mk_iterate - run niter Neumann iterations of every survey, continuing the
 * series from where it stopped (Algorithm 1, loop over iter; one synthesis,
 * reversal, mute and accumulation per iteration).
 *   energy: NULL, or host double [niter][sum of nfocal over surveys]:
 *           E_i(f) = sum over (k, t) of N_i^2 (k over the plan's own positions
 *           for a shot-row shard), FP32 squares summed per trace error-free
 *           and in FP64 across traces, in a fixed order (deterministic).  With energy != NULL the call returns
 *           after the work is done; with NULL it is asynchronous.
 * Errors: MK_ERR_ARG (niter < 0), MK_ERR_STATE (a survey without G_d),
 *         MK_ERR_CUDA.
 */
mk_status mk_iterate(mk_plan_t plan, int32_t niter, double* energy);

/*
 * mk_fetch_fields - copy selected fields of one survey out, in bit order of
 * mask, each float [nfocal][nsrc][nt].  The iterations accumulate f1plus and
 * f1min only; N_last, f2p, pmin and G are formed on the GPU when fetched
 * (f2p = f1plus - f1min(-t); pmin = synthesis of f2p - N_last, one extra
 * contraction; G = f2p(-t) + pmin), which is exact algebra of Algorithm 1.
 * A resident complex FP32 survey with one focal point instead accumulates
 * pmin during the iterations as it stands in Algorithm 1, as the sum of the
 * synthesis results' band spectra, and forms it at fetch with one inverse
 * transform (no extra contraction).
 * MK_F_GMINUS is the up-going Green's function of Algorithm 1 (one extra
 * synthesis of f1plus after the loop, minus f1min); MK_F_GPLUS the
 * down-going one, f1plus(-t) minus the synthesis of f1min(-t) (Theory: each
 * component needs one extra synthesis; the G^+ formula is a reading, and
 * G - G^+ - G^- equals minus the synthesis of the last N_i).
 *   out: host (dst_on_device = 0) or device (1) buffer of out_bytes >=
 *        popcount(mask) * nfocal * nsrc * nt * 4.
 * Errors: MK_ERR_ARG, MK_ERR_STATE (G_d not set), MK_ERR_CUDA.
 */
mk_status mk_fetch_fields(mk_plan_t plan, int32_t survey, uint32_t mask, float* out,
                          size_t out_bytes, int32_t dst_on_device);

/*
 * mk_image - double-focusing image of each focal point of one survey: the
 * zero-time sample of the time convolution of G^- with f1plus, integrated
 * over the surface positions (Theory section; Algorithm 1, "imaging"):
 *     image(f) = dx dt sum_k sum_j G^-(f, x_k, t_j) f1plus(f, x_k, -t_j),
 * accumulated in FP64 in a fixed order.  Forms G^- if needed (one synthesis).
 *   image: double [nfocal], host (dst_on_device = 0) or device (1).
 * Errors: MK_ERR_ARG, MK_ERR_STATE (G_d not set), MK_ERR_CUDA.
 */
mk_status mk_image(mk_plan_t plan, int32_t survey, double* image, int32_t dst_on_device);

/*
 * mk_set_fields - resume a series from saved fields (checkpoint / restart;
 * the paper's GPU code keeps iRN on disk between iterations, Algorithm 1).
 * Sets the state of one survey from caller data -- the last N, f1plus and
 * f1min -- and the iteration index (its parity decides f1min vs f1plus,
 * Algorithm 1), and recomputes the band spectrum of N, so that the next
 * mk_iterate continues from exactly these fields.  f2p and pmin follow from
 * the state (f2p = f1plus - f1min(-t), pmin = synthesis of f2p - N); if the
 * mask includes them their data is skipped.  Windows stay those of the last
 * mk_set_Gd_window.
 *   mask: must contain MK_F_N | MK_F_F1P | MK_F_F1M; may add MK_F_F2P, MK_F_PMIN;
 *   in:   float [popcount(mask)][nfocal][nsrc][nt] in bit order, host or device.
 *   iteration: the number of iterations these fields represent (>= 0).
 * Errors: MK_ERR_ARG, MK_ERR_STATE (G_d not set), MK_ERR_CUDA.
 */
mk_status mk_set_fields(mk_plan_t plan, int32_t survey, uint32_t mask, const float* in, size_t in_bytes,
                        int32_t iteration, int32_t src_on_device);

/*
 * mk_get_stats - launch counters and (with MK_FLAG_TIMING on every survey's
 * description) summed CUDA-event times of the contraction and epilogue
 * kernels, measured on the plan's stream.  Synchronises the stream.
 *   reset != 0 zeroes the counters after reading them.
 * Errors: MK_ERR_ARG, MK_ERR_CUDA.
 */
mk_status mk_get_stats(mk_plan_t plan, mk_stats_t* out, int32_t reset);

/*
 * mk_run_noalloc - the same computation as mk_set_Gd_window followed by
 * mk_iterate(niter) for one survey, for callers that cannot allocate device
 * memory.  The paper has no counterpart; it exists because some callers
 * cannot call cudaMalloc at the point of use (a host framework that owns all
 * GPU memory through its own pool and passes only fixed input and output
 * buffers, or a process with a memory budget fixed in advance) and so cannot
 * provide the plan workspace of mk_plan.
 *
 * It allocates nothing: it calls no cudaMalloc, cudaFree or allocating
 * library routine.  Its intermediate data (mute windows, band spectra, per-
 * trace energies, FFT twiddles) lives in one file-scope device array of
 * MK_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  Surveys that need more scratch than that
 * (about 2 * n_w * r_pad * nfocal * 8 bytes) are rejected with MK_ERR_ARG
 * before any GPU work.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and sets kernel attributes; make that first call
 * before any stream capture.  Every call uses the same array and the array
 * keeps the last call's contents (each call clears what it needs zeroed), so
 * calls whose GPU work overlaps -- on different streams, or from different
 * threads -- race with each other: order them on one stream.
 *
 *   d:      one survey (rprec must be MK_R_C64).
 *   R:      device, complex64 [n_w][nsrc][r_pad], r_pad = nrec rounded up to
 *           a multiple of 32, padding entries zero.  (A plan for a single
 *           focal point pads its own R rows only to an even count; this entry
 *           point always takes rows padded to 32.)
 *   Gd, td: device, as for mk_set_Gd_window.
 *   niter:  iterations (>= 0).
 *   fields: device float [5][nfocal][nsrc][nt]: N, f1plus, f1min, f2p, pmin
 *           after niter iterations (written, not read).
 *   energy: device double [niter][nfocal], or NULL.
 *   cuda_stream: stream for all the work; the call returns without waiting.
 * Errors (message via mk_last_error(NULL)): MK_ERR_ARG, MK_ERR_UNSUPPORTED,
 *         MK_ERR_CUDA.  A bounded device wait that runs out (MK_ERR_TIMEOUT in
 *         the plan entry points) cannot be returned by a call that does not
 *         wait: the last kernel of the call then fills fields (and energy)
 *         with NaN instead.
 */
#define MK_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
mk_status mk_run_noalloc(const mk_desc* d, const void* R, const float* Gd, const double* td, double eps_s,
                         int32_t niter, float* fields, double* energy, void* cuda_stream);

/*
 * Shot-row sharding: the exchange of the field spectrum between shards.
 *
 * The paper splits the synthesis over GPUs by shots (Implementation
 * section): every GPU holds its batch of rows of R and contracts the whole
 * field with them.  A plan made with mk_desc.row_count > 0 holds the output
 * positions k in [row_begin, row_begin + row_count) of a survey; each
 * iteration (mk_iterate) computes the next field spectrum at those positions
 * only.  Before every contraction -- after mk_set_Gd_window and after each
 * mk_iterate(plan, 1, ...) -- the caller gives every shard the spectrum rows
 * of all the others: mk_export_field_spectrum on each shard, an all-gather of
 * the packed buffers (e.g. NCCL), mk_import_field_spectrum of each received
 * block.  Energies returned by mk_iterate are the sums over the shard's own
 * positions (the caller adds them up); fetched fields are the shard's own
 * positions, [nfocal][row_count][nt].  A shard keeps pmin as a band spectrum
 * during the iterations; G^-, G^+, mk_image, mk_set_fields and
 * mk_load_R_time need the whole survey and return MK_ERR_UNSUPPORTED.
 *
 * Packed layout (bytes = parts * n_w * nfocal * rows * 8, parts = 1 for
 * complex FP32 R and the scaled FP16 split, 2 for the other 16-bit and split
 * forms, 3 for the 3-way split):
 *   complex FP32 and scaled FP16 split: complex64 [n_w][nfocal][rows];
 *   16-bit forms: per part, 16-bit [n_w][2 nfocal][2 rows] (the rows of the
 *   tensor-core operand), parts one after the other.
 * Both calls run on the plan's stream, synchronously for host buffers.
 */

/*
 * mk_export_field_spectrum - the plan's own rows of the field spectrum
 * (positions row_begin .. row_begin + row_count - 1, or every position of an
 * unsharded plan) into dst (host: dst_on_device = 0, device: 1).
 * Errors: MK_ERR_ARG (null, bytes too small), MK_ERR_STATE (G_d not set),
 *         MK_ERR_CUDA.
 */
mk_status mk_export_field_spectrum(mk_plan_t plan, int32_t survey, void* dst, size_t bytes,
                                   int32_t dst_on_device);

/*
 * mk_import_field_spectrum - rows row_begin .. row_begin + row_count - 1 of
 * the field spectrum from src (packed as above, as another shard exported
 * them), before the next contraction.
 * Errors: MK_ERR_ARG (null, rows outside [0, nrec), bytes too small),
 *         MK_ERR_STATE (G_d not set), MK_ERR_CUDA.
 */
mk_status mk_import_field_spectrum(mk_plan_t plan, int32_t survey, const void* src, int32_t row_begin,
                                   int32_t row_count, size_t bytes, int32_t src_on_device);

/*
 * mk_set_timing - for a plan made with MK_FLAG_TIMING: record the CUDA
 * events around the contraction and epilogue launches of every stride-th
 * iteration only (1 = every iteration, the default), counted from this call,
 * and create reserve_pairs event pairs now, so that timed launches create
 * none.  mk_get_stats then averages over the timed launches.
 * Errors: MK_ERR_ARG (stride < 1, reserve < 0), MK_ERR_STATE (no
 * MK_FLAG_TIMING), MK_ERR_CUDA.
 */
mk_status mk_set_timing(mk_plan_t plan, int32_t stride, int32_t reserve_pairs);

/*
 * Tuning of one survey's kernels (MK_FLAG_AUTOTUNE).  Candidates: the N tile
 * of the tensor-core contraction (16, 32, 64 or 128 columns of the real
 * field embedding, up to the first power of two covering 2 nfocal) and the
 * pairs of traces per epilogue block (1, 2 or 4, within shared memory).  Each
 * candidate runs once untimed and three times timed with CUDA events on the
 * plan's stream, on the survey's own buffers, before the fields are
 * initialised; the fastest is kept.  Choices are cached per process, keyed by
 * (nsrc, nt, n_w, nfocal, rprec) and the device's SM count, so later plans of
 * the same shape skip the timing.  Results do not depend on the choice.
 */
typedef struct {
  int32_t tuned;        /* 0: heuristic choice, 1: timed now, 2: taken from the cache */
  int32_t umma_bn;      /* N tile of the tensor-core contraction (0: not on that path) */
  int32_t epi_pairs;    /* pairs per epilogue block (0: chosen at each launch) */
  int32_t candidates;   /* candidates timed */
  float contract_ms;    /* best contraction time seen while tuning (0 if none) */
  float epilogue_ms;    /* best epilogue time seen while tuning (0 if none) */
} mk_tuning_t;

/*
 * mk_get_tuning - the kernel choices of one survey (after mk_set_Gd_window
 * when tuned).  Errors: MK_ERR_ARG (bad survey, null).
 */
mk_status mk_get_tuning(mk_plan_t plan, int32_t survey, mk_tuning_t* out);

/* mk_destroy - release the plan's host state (not the caller's workspace).
 * Synchronises the plan's stream.  NULL is accepted. */
mk_status mk_destroy(mk_plan_t plan);

/* mk_last_error - message of the last failed call on plan (NULL: of the last
 * failed call made without a plan); "" when none. */
const char* mk_last_error(mk_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* MARCHENKO_H */
