/*
 * fftbf — FFT beamforming of a regular antenna lattice on one GB300 (sm_103a).
 *
 * Method: Masui et al., "Algorithms for FFT Beamforming Radio Interferometers"
 * (arXiv 1710.08591). The paper is written for a 1-D array; the library applies it on
 * both axes of an nx (E-W) x ny (N-S) lattice, the separable 2-D extension.
 *
 * Units and layouts used by every entry point:
 *   - A voltage sample is one byte: bits 7..4 = real, bits 3..0 = imaginary, each a
 *     two's-complement 4-bit integer in [-8, 7]. (The paper fixes no bit layout.)
 *   - volts   uint8 [T][nfreq][npol][nx][ny], row-major. Each polarisation is a
 *     separate set of antennas (Section 2, dual-polarisation feeds).
 *   - beams   float [T / n_int][nfreq][pad_x][pad_y]: the unnormalised integrated
 *     FFT-beam intensities
 *        P[j,f,A,B] = sum_{t in window j} sum_p |sum_{ix,iy} w[ix,iy] x[t,f,p,ix,iy]
 *                      exp(-2 pi i (A ix / pad_x + B iy / pad_y))|^2
 *     (Eq. fftbeamform with the factorizable beam of Eq. bf; the paper's 1/n_samp,
 *     1/sqrt(n_ant) and flux-unit factors are left to the caller). Beam A is at
 *     sin(theta_A) = A lambda / (pad_x d) in natural DFT order (Eq. theta_A): indices
 *     A >= pad/2 are the negative-angle aliases; there is no fftshift.
 *   - Padding: pad >= 2n - 1 keeps all the information of the redundancy-stacked
 *     visibilities (Eq. b2n-1; pad = 2n recommended). pad < n is legal: the feeds are
 *     co-added cyclically, element A being the sum of feeds with a = A mod pad
 *     (Section 3.2).
 *   - Windows are non-overlapping runs of n_int samples starting at t = 0 of each call.
 *
 * Ownership: the caller owns every buffer passed in; the plan owns its tables and
 * scratch. Device pointers are plain CUDA device addresses on the plan's device.
 *
 * Asynchrony: entry points taking a stream enqueue work on it and return; their return
 * value reports argument and launch errors. fftbf_plan_sync waits for the plan's work.
 *
 * Errors: every int-returning entry point returns FFTBF_OK (0) or a negative code; the
 * message of the last error on the calling thread is fftbf_last_error().
 */
#ifndef FFTBF_H
#define FFTBF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftbf_plan fftbf_plan;

enum fftbf_status {
  FFTBF_OK = 0,
  FFTBF_EINVAL = -1,      /* bad argument: null pointer, size, shape or pointing */
  FFTBF_ENOMEM = -2,      /* a device or pinned-host allocation failed */
  FFTBF_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
  FFTBF_ETIMEOUT = -4,    /* a bounded device-side wait ran out */
  FFTBF_EUNSUPPORTED = -5 /* valid request this build does not implement */
};

enum fftbf_precision {
  FFTBF_PREC_FP32 = 0,    /* FP32 CUDA-core spatial FFT (default) */
  FFTBF_PREC_TC_FP16 = 1, /* tensor-core GEMM stages, FP16 operands, FP32 accumulate */
  FFTBF_PREC_TC_BF16 = 2, /* tensor-core GEMM stages, BF16 operands, FP32 accumulate */
  FFTBF_PREC_TC_FP16X3 = 3 /* tensor-core GEMM stages on split FP16 operands (hi + lo,
                              three products per stage), FP32 accumulate: FP32 accuracy */
};

/*
 * Create a plan on the current CUDA device.
 *   nx, ny      lattice size, E-W x N-S (>= 1).
 *   pad_x/pad_y number of FFT beams per axis, M in the paper (>= 1; Eq. fftbeamform).
 *   npol        polarisations, summed after detection (>= 1).
 *   nfreq       frequency channels, processed independently (>= 1).
 *   n_int       samples integrated per output window (>= 1; n_samp of Eq. Vab).
 *   weights     host pointer to nx*ny complex FP32 apodisation weights, interleaved
 *               (re, im), [ix][iy] row-major; multiplied into the voltages before the
 *               spatial DFT (naive windowed beam of Section 4.1; per-feed gains of
 *               Section 4.2 fit here too). NULL means 1 + 0i everywhere. Copied.
 * Builds the FP32 twiddle and E-W DFT tables from FP64 on the device. Returns NULL on
 * error (see fftbf_last_error).
 */
fftbf_plan* fftbf_plan_create(int nx, int ny, int pad_x, int pad_y, int npol, int nfreq,
                              int n_int, const float* weights);

/*
 * Select the arithmetic of fftbf_execute (enum fftbf_precision). The tensor-core forms
 * compute the same quantity (Eq. fftbeamform, Eq. bf) with the zero-padded N-S transform
 * as two GEMM stages on 16-bit operands with FP32 accumulation; they need pad_x = 4,
 * pad_y = 512 and at most 256 N-S feeds (FFTBF_EUNSUPPORTED otherwise). With FP16
 * operands the plan scales the E-W output so every intermediate stays finite and
 * removes the scale from the result. FFTBF_PREC_TC_FP16X3 splits every operand into an
 * FP16 value and its FP16 residual (hi + lo) and forms each stage as hi*hi + hi*lo +
 * lo*hi in FP32, so the result has FP32 accuracy (the dropped lo*lo term is ~2^-22 of
 * each product). On the 4x256 lattice with 16-byte aligned voltages the FP16 and BF16
 * forms run a kernel that folds the E-W DFT into the first stage and keeps the second
 * stage's operand in tensor memory; the environment variable FFTBF_TC_KERNEL=ws selects
 * the pair-wise kernel (E-W DFT on the CUDA cores) instead and FFTBF_TC_KERNEL=serial the
 * kernel every other shape uses; all three compute the same beams within the form's
 * error. Call before fftbf_execute; not thread-safe with it.
 */
int fftbf_plan_set_precision(fftbf_plan* plan, int precision);

/*
 * Integrated FFT-beam intensities for T samples (Eq. fftbeamform, Eq. bf):
 * unpack -> apodise -> zero-padded (or cyclically folded) 2-D spatial DFT -> |.|^2 ->
 * sum over polarisation -> sum over each window of n_int samples.
 *   volts_dev  device uint8 [T][nfreq][npol][nx][ny]; any alignment.
 *   T          samples; a multiple of n_int (else FFTBF_EINVAL); 0 is a no-op.
 *   beams_dev  device float [T/n_int][nfreq][pad_x][pad_y]; overwritten.
 *   stream     cudaStream_t to run on (NULL = legacy default stream).
 * No complex beam is written to memory: detection and integration are fused into the
 * transform.
 */
int fftbf_execute(fftbf_plan* plan, const uint8_t* volts_dev, int64_t T, float* beams_dev,
                  void* stream);

/*
 * Tied-array beams at arbitrary pointings, regridded from FFT-beam intensities
 * (Eq. bp_max_arbitrary, applied per axis):
 *   tied[j,f,s] = sum_{A,B} w^A(u[f,s]) w^B(v[f,s]) beams[j,f,A,B],
 *   w^A(y) = (1/M) sin[(2n-1) pi (y - A/M)] / sin[pi (y - A/M)]   (M >= 2n - 1).
 * On an axis with pad < 2n - 1 the FFT beams do not carry all of the stacked
 * visibilities and the formula does not hold; there the pointing must sit on the
 * FFT-beam grid (y * pad an integer within 1e-9, else FFTBF_EINVAL) and the tied beam
 * uses that FFT beam itself (Eq. theta_A).
 *   beams_dev  device float [n_windows][nfreq][pad_x][pad_y] from fftbf_execute.
 *   n_windows  >= 0;  n_tied >= 1.
 *   u, v       host double [nfreq][n_tied]: (d_x / lambda_f) sin(theta_x) and
 *              (d_y / lambda_f) sin(theta_y) per frequency, so chromatic steering is the
 *              caller's choice. Copied.
 *   tied_dev   device float [n_windows][nfreq][n_tied]; overwritten.
 * The weight tables are generated in FP64 on the device, rounded to FP32 and kept in
 * the plan; a later call with identical u, v and n_tied reuses them. When the E-W axis is
 * on the FFT-beam grid (pad_x < 2 nx - 1, pad_x <= 4) and pad_y is a multiple of 64, the
 * sum runs on the tensor cores with each operand split into two FP16 parts (three
 * products per term, FP32 accumulation: FP32 accuracy); the split weight tables are also
 * kept in the plan. Environment FFTBF_TIED_TC=0 selects the CUDA-core FP32 GEMM, which
 * is also used when the split tables cannot be allocated.
 * Errors: FFTBF_EINVAL (arguments, off-grid pointing), FFTBF_ENOMEM (tables),
 * FFTBF_ETIMEOUT (reported by fftbf_plan_sync if a tensor-core wait ran out).
 */
int fftbf_tied_beams(fftbf_plan* plan, const float* beams_dev, int64_t n_windows,
                     int n_tied, const double* u, const double* v, float* tied_dev,
                     void* stream);

/*
 * Shape the tied beams of later fftbf_tied_beams calls in intensity space (Section 4.1):
 * with a real window h on an axis, the tied beam becomes the optimal windowed beam whose
 * redundant-baseline weights are g_delta = sum_alpha h^(alpha+delta) h^alpha /
 * (n - |delta|) (Eq. w_opt, unnormalised: a flat window is the plain pointed beam), so
 * the regridding coefficients are w^A(y) = (1/M) sum_delta g_delta
 * exp(-2 pi i delta (y - A/M)) (Eq. wA_from_wdelta). A window needs pad >= 2n - 1 on its
 * axis (FFTBF_EINVAL otherwise).
 *   hx, hy     host double windows of nx and ny values, or NULL for no window on that
 *              axis (Dirichlet kernel of Eq. bp_max_arbitrary). Copied.
 *   trunc_x/y  keep only the `trunc` FFT beams nearest the pointing (beams
 *              floor(y M - (trunc-1)/2 + 1/2) .. + trunc-1, cyclic) and drop the rest: the
 *              compact kernel a windowed beam allows (Section 4.1); 0 keeps every beam.
 *              When both axes have few taps (truncated, or a grid axis with pad < 2n-1)
 *              the tied beams use a gather kernel of trunc_x x trunc_y taps instead of the
 *              GEMM over all FFT beams.
 * Takes effect at the next fftbf_tied_beams call (tables are rebuilt).
 */
int fftbf_tied_set_window(fftbf_plan* plan, const double* hx, const double* hy, int trunc_x,
                          int trunc_y);

/*
 * Redundancy-stacked visibilities recovered from integrated FFT-beam intensities
 * (Eq. inv_b2n-1). Per axis with pad >= 2n - 1 the beams are inverted onto the 2n - 1
 * lags delta = -(n-1) .. n-1 (stored at index delta + n - 1):
 *   V~_delta = (1/M) sum_A exp(+2 pi i delta A / M) P_A
 * (the paper's n_ant / M factor is left to the caller, as in fftbf_execute); on an axis
 * with pad < 2n - 1 the FFT beams do not determine every lag and the beam index is kept.
 * V~_-delta = conj(V~_delta) and V~_0 is the total power.
 *   beams_dev  device float [n_windows][nfreq][pad_x][pad_y] from fftbf_execute.
 *   vis_dev    device complex FP32 (re, im interleaved) [n_windows][nfreq][Dx][Dy], with
 *              Dx, Dy from fftbf_stacked_shape; overwritten.
 */
int fftbf_stacked_shape(const fftbf_plan* plan, int* dx, int* dy);
int fftbf_stacked_visibilities(fftbf_plan* plan, const float* beams_dev, int64_t n_windows,
                               float* vis_dev, void* stream);

/*
 * Localisation of a point source from FFT-beam intensities (Section 4.3), one estimate
 * per (window, channel): start at the strongest FFT beam, then on each axis with
 * pad >= 2n - 1 (and n > 1) take n_iter Newton steps
 *   y <- y + T'(y) n^2 / (4 pi^2 MOI T(y)),   MOI = sum_delta delta^2 (n - |delta|)
 * with T, T' the pointed beam and its derivative regridded from the n_taps FFT beams
 * nearest the estimate and the curvature taken at the maximum (Eq. baseline_MOI); an axis
 * with pad < 2n - 1 keeps the beam position A / pad. The paper expects ~10 beams to hold a
 * source's information; its uncertainty is sqrt(6) / (2 pi n SNR) in y.
 *   beams_dev  device float [n_windows][nfreq][pad_x][pad_y] from fftbf_execute.
 *   n_iter >= 0; n_taps in 1 .. 64 (clipped to the pad of each axis), else FFTBF_EINVAL.
 *   out_dev    device float [n_windows][nfreq][3]: y_x, y_y in [0, 1) (lattice units,
 *              (d/lambda) sin(theta)) and the pointed beam T at the estimate.
 * Weights are evaluated in FP32 from exactly reduced phases; T is summed in FP64.
 */
int fftbf_localise(fftbf_plan* plan, const float* beams_dev, int64_t n_windows, int n_iter,
                   int n_taps, float* out_dev, void* stream);

/*
 * The same pass as fftbf_execute followed by fftbf_tied_beams, on HOST buffers: the
 * voltages are copied to the device in window-sized chunks on a copy stream owned by
 * the plan, overlapped with the transform of the previous chunk on `stream`; the
 * intensities (and tied beams, if n_tied > 0) are copied back to the host.
 *   volts_host  host uint8 [T][nfreq][npol][nx][ny]; pinned memory gives overlap.
 *   beams_host  host float [T/n_int][nfreq][pad_x][pad_y]; written.
 *   n_tied      0 (no tied beams) or the number of pointings; then u, v as in
 *               fftbf_tied_beams and tied_host = host float [T/n_int][nfreq][n_tied].
 * The first call allocates the plan's staging buffers (two chunks of voltages and the
 * device intensities/tied beams of one call); later calls reuse them, growing them if
 * a call is larger. Stream-ordered: the host outputs are complete once `stream` (or
 * fftbf_plan_sync) has been synchronised; the inputs must stay valid until then.
 */
int fftbf_execute_host(fftbf_plan* plan, const uint8_t* volts_host, int64_t T,
                       float* beams_host, int n_tied, const double* u, const double* v,
                       float* tied_host, void* stream);

/*
 * Batches: several plans (arrays of different lattice sizes, channel counts and weights)
 * transformed by ONE persistent launch of the FP32 form. Work items are (array, window,
 * channel) taken from a device work queue, costliest arrays first; each array runs the
 * transform of its own shape, with a snapshots-per-step tile picked for it by timing the
 * candidates on the device at creation. Supported shapes (pad_x x pad_y, pad_y >= ny):
 * 4x512, 8x128, 16x32, 2x1024, 1x2048, 3x256 (the N-S axis padded to twice the next
 * power of two of 256, 64, 16, 512, 1024, 128 feeds); others give FFTBF_EUNSUPPORTED.
 * The plans must outlive the batch, be on one device and not change precision.
 */
typedef struct fftbf_batch fftbf_batch;
/* n plans (1..64); allocates the work table and runs the autotuner. NULL on error. */
fftbf_batch* fftbf_batch_create(fftbf_plan* const* plans, int n);
/*
 * One pass of every plan over T samples (T a multiple of every plan's n_int):
 * volts_dev[i] / beams_dev[i] are host arrays of n device pointers laid out as in
 * fftbf_execute for plan i. Each array's beams are bit-identical to a batch of that
 * array alone in the same process (the autotuner's choice is kept per lattice shape). On a non-default stream the launch is captured in a CUDA graph and
 * replayed while stream, T and the pointers stay the same.
 */
int fftbf_batch_execute(fftbf_batch* batch, const uint8_t* const* volts_dev, int64_t T,
                        float* const* beams_dev, void* stream);
/* Snapshots per step the autotuner chose for plan i of the batch (>= 1), or < 0. */
int fftbf_batch_tuned_steps(const fftbf_batch* batch, int i);
/* CTAs of each batched launch: the launch's persistent grid (SMs x resident CTAs per SM);
 * work items beyond it are taken from the device queue in turn. */
int fftbf_batch_grid(const fftbf_batch* batch);
/* Free the batch (waits for its last launch). NULL is a no-op. */
void fftbf_batch_destroy(fftbf_batch* batch);

/*
 * Continuous-batching server for voltage frames from many independent streams. A frame is
 * one window (n_int samples) of one lattice plan: host uint8 [n_int][nfreq][npol][nx][ny];
 * its result is that window's beams, host float [nfreq][pad_x][pad_y]. A scheduler thread
 * admits frames into device slots carved from ONE allocation of hbm_budget_bytes (a frame
 * waits while no slot is free), copies them to the device, and whenever frames are staged
 * and a launch slot is free, transforms every staged frame in one persistent batched
 * launch (up to 64 frames; two launches may be in flight), so frames that arrive while
 * others are on the GPU join the next launch and their work overlaps. A frame's beams are
 * bit-identical alone and in any mix. Lattice shapes: those of fftbf_batch_create.
 * Host buffers must stay valid until the frame completes; pinned memory lets copies and
 * transforms overlap.
 */
typedef struct fftbf_server fftbf_server;
typedef struct {
  int64_t submitted, completed;  /* frames */
  int64_t launches;              /* batched launches issued */
  int64_t peak_inflight;         /* most frames holding device slots at once */
  int64_t slots;                 /* device slots the budget allows */
  int64_t max_frames_per_launch; /* largest number of frames in one launch */
  int64_t max_items_per_launch;  /* largest number of (frame, channel) items in one launch */
  int64_t grid;                  /* CTAs of every launch (items beyond it are taken in turn) */
  double frames_per_launch;      /* mean frames per launch */
  double p50_ms, p99_ms, max_ms, mean_ms;  /* completion - submission, host clock; the
                                              percentiles come from a uniform sample of at
                                              most 65536 frames (exact up to that count) */
} fftbf_server_stats_t;
/* n lattice plans (1..64, FP32 precision); starts the scheduler thread. NULL on error. */
fftbf_server* fftbf_server_create(fftbf_plan* const* lattices, int n, int64_t hbm_budget_bytes);
/* Queue one frame of lattice `lattice`; returns its ticket (>= 0) or a negative error.
 * The frame's latency clock starts on entry, before the call waits for the server lock. */
int64_t fftbf_server_submit(fftbf_server* server, int lattice, const uint8_t* frame_host,
                            float* beams_host);
/* hold != 0: admit and stage frames but start no launch until called again with 0 (then
 * every staged frame, up to 64 per launch, goes out at once). Lets a caller gather a burst
 * into one launch; fftbf_server_destroy releases a hold. FFTBF_OK or FFTBF_EINVAL. */
int fftbf_server_hold(fftbf_server* server, int hold);
/* Wait until frame `ticket` (or, with ticket < 0, every submitted frame) has completed:
 * FFTBF_OK, FFTBF_ETIMEOUT after timeout_s seconds, FFTBF_EINVAL for a ticket never
 * issued, or the server's CUDA error. */
int fftbf_server_wait(fftbf_server* server, int64_t ticket, double timeout_s);
/* Counters and latency percentiles so far; returns the server's error state. */
int fftbf_server_stats(fftbf_server* server, fftbf_server_stats_t* out);
/* Finish queued frames, stop the scheduler, free the device slots. NULL is a no-op. */
void fftbf_server_destroy(fftbf_server* server);

/* Wait for all work the plan has enqueued; returns the first device-side error seen
 * (e.g. FFTBF_ETIMEOUT) and clears it. */
int fftbf_plan_sync(fftbf_plan* plan);

/* Free the plan after waiting for its work. NULL is a no-op. */
void fftbf_destroy(fftbf_plan* plan);

/* Message of the last error on the calling thread ("" if none). Owned by the library. */
const char* fftbf_last_error(void);
/* Status code of that error (FFTBF_OK if none): the code behind a NULL from a constructor. */
int fftbf_last_error_code(void);

/*
 * Test hook for the bit layout: decode n bytes at in_dev into out_dev (device float,
 * 2n values: re, im interleaved) with the decoder the kernels use.
 */
int fftbf_debug_unpack(const uint8_t* in_dev, int64_t n, float* out_dev, void* stream);

/*
 * Test hook for the tensor-core building blocks: D[128][n] = A[128][32] B[n][32]^T with
 * 16-bit operands (FP16, or BF16 if bf16 != 0), staged in the kernels' shared-memory
 * layouts: `padded` = 0 canonical K-major A, 1 K-major A with the padded strides of the
 * stage-2 operand, 2 MN-major A (element (m, k) at byte (m%8)*2 + (k%8)*16 + (m/8)*128 +
 * (k/8)*2048, the operand layout of the warp-specialised FP16 kernel), 3 A in tensor
 * memory (row m in lane m, two elements per 32-bit column, written by tcgen05.st) with
 * K-major B, 4 canonical K-major A with MN-major B (element (n, k) at byte (n%8)*2 +
 * (k%8)*16 + (n/8)*128 + (k/8)*16n); 3 and 4 are the operand forms of the grouped
 * kernel and take n <= 128. One pair of tcgen05.mma instructions, FP32 accumulation in
 * tensor memory. n = 32, 64, 128 or 256.
 * Device pointers, row-major. Synchronises `stream`; FFTBF_ETIMEOUT if the tensor core
 * did not complete within one second.
 */
int fftbf_debug_tc_gemm(const uint16_t* a_dev, const uint16_t* b_dev, int n, int bf16,
                        int padded, float* d_dev, void* stream);

/*
 * FP32 throughput probe (measurement, not part of the method): `blocks` CTAs of 256
 * threads each run 8 independent multiply-add chains for `iters` steps, as scalar FFMA
 * (packed = 0) or as the packed two-lane FFMA2 (packed = 1, fma.rn.f32x2). out_dev:
 * device float [blocks * 256], overwritten. *flops_out receives the flops the launch
 * performs (2 per FMA); the caller times the launch on `stream` (asynchronous).
 */
int fftbf_probe_fp32(int packed, int64_t iters, int blocks, float* out_dev, double* flops_out,
                     void* stream);

/*
 * Test hook for failure detection without a GPU fault: a kernel waits, with the same
 * bounded wait the tensor-core kernels use, on an mbarrier that nothing arrives on. The
 * wait gives up after limit_us microseconds of device time (1..2000000) and the call
 * returns FFTBF_ETIMEOUT; the CUDA context stays usable. Synchronises `stream`.
 */
int fftbf_debug_wait_timeout(int limit_us, void* stream);

/*
 * fftbf_execute without a plan and without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, such
 * as an application that hands all device memory to its own pool before it starts
 * streaming, or a real-time loop that must not make allocator calls (cudaMalloc and
 * cudaFree can synchronise the device and stall every stream).
 *
 * It computes exactly what fftbf_execute computes, with the same kernels; the small
 * tables a plan would allocate (E-W DFT matrix, N-S twiddles, and unit weights when
 * weights_dev is NULL) are written instead into one fixed array of device memory that
 * the library reserves statically: FFTBF_NOALLOC_SCRATCH_BYTES on every GPU that loads
 * the library, held until the process exits.
 *   nx ... n_int  as for fftbf_plan_create; the tables must fit the array:
 *                 8 * (pad_x*nx + pad_y + (weights_dev ? 0 : nx*ny)) bytes
 *                 <= FFTBF_NOALLOC_SCRATCH_BYTES, else FFTBF_EINVAL with a message.
 *   weights_dev   device pointer (8-byte aligned) to nx*ny complex FP32 weights (re, im
 *                 interleaved, [ix][iy]), or NULL for 1 + 0i; read, not copied.
 *   volts_dev, T, beams_dev, stream  as for fftbf_execute.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture begins.
 * The address is kept for the life of the process: after cudaDeviceReset on a device,
 * the next call on that device would use the old context's address, so a caller that
 * resets a device must not call this entry point on it again.
 * Every call rewrites the tables before its transform reads them, so nothing carries
 * over from the previous call. All calls share the one array: calls whose work
 * overlaps on the GPU (on different streams, or from several host threads) race on it
 * and must be serialised by the caller.
 */
#define FFTBF_NOALLOC_SCRATCH_BYTES (64 * 1024)
int fftbf_execute_noalloc(int nx, int ny, int pad_x, int pad_y, int npol, int nfreq,
                          int n_int, const float* weights_dev, const uint8_t* volts_dev,
                          int64_t T, float* beams_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FFTBF_H */
