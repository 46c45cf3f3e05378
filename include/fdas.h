/*
 * fdas.h -- C ABI of libfdas: the FDAS overlap-and-save correlation on GB300 (sm_103a).
 *
 * The library computes the f-fdot power plane of the Fourier Domain Acceleration Search
 * (Adamek, Dimoudi, Giles & Armour 2017, arXiv 1711.10855):
 *
 *   P[z_idx][r] = | sum_{q=-h}^{h} A_{r+q} * conj(Hn_q(z)) |^2          (Section 1, Eq. 2)
 *
 * for every bin r in [0, n_bins) and every z = -zmax + z_idx*zstep, z_idx in [0, Z),
 * Z = 2*zmax/zstep + 1, with A_k = 0 outside [0, n_bins), h = tmpl_len/2, and Hn the
 * predicted Fourier response of a constant-frequency-derivative signal (Section 1, after
 * Ransom, Eikenberry & Middleditch 2002), normalised to unit L2 norm over its
 * tmpl_len + 1 taps q = -h..h:
 *
 *   H_q(z) = int_0^1 exp(i*pi*(z*u^2 - (z + 2q)*u)) du,   Hn = H / ||H||_2.
 *
 * The garbled lower limit of Eq. 2 is read as r0 - m/2; "m taps" is read as the even span
 * m = tmpl_len, i.e. m + 1 coefficients q = -m/2..m/2.
 *
 * The correlation runs by overlap-and-save (Section 2): segment s holds the L = seg_len
 * bins A[s*V - h .. s*V - h + L), V = L - tmpl_len; each segment is transformed once, multiplied
 * by the FFT of every template and transformed back, and the V outputs free of circular
 * wrap-around are kept.  Transforms follow the DFT sign of Eq. 3 (forward e^{-i2pi nm/N}).
 *
 * Conventions for every call:
 *   - Return value 0 (FDAS_OK) on success, a negative FDAS_ERR_* code otherwise; no C++
 *     exception crosses the ABI.  fdas_plan_create returns NULL on failure and records the
 *     code, readable with fdas_last_error() (thread-local).
 *   - Device pointers are plain CUDA device addresses of the current device, owned by the
 *     caller unless stated.  Streams are CUDA streams (NULL = legacy default stream).
 *   - There is no CPU fallback: without a GB300-class device (compute capability 10.3) the
 *     plan cannot be created (FDAS_ERR_UNSUPPORTED / FDAS_ERR_NO_DEVICE).
 */
#ifndef FDAS_H
#define FDAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdas_plan fdas_plan;          /* opaque plan: sizes, template bank, workspace */
typedef struct CUstream_st* fdas_stream_t;   /* identical to cudaStream_t */

enum fdas_status {
  FDAS_OK = 0,
  FDAS_ERR_INVALID = -1,      /* an argument is out of its documented range */
  FDAS_ERR_ALIGN = -2,        /* a pointer does not have the documented alignment */
  FDAS_ERR_NOT_BUILT = -3,    /* fdas_convolve_power before fdas_templates_build */
  FDAS_ERR_ALLOC = -4,        /* device allocation failed */
  FDAS_ERR_CUDA = -5,         /* a CUDA runtime call or kernel launch failed */
  FDAS_ERR_NO_DEVICE = -6,    /* no CUDA device is visible */
  FDAS_ERR_UNSUPPORTED = -7,  /* the current device is not compute capability 10.3 */
  FDAS_ERR_TIMEOUT = -8       /* a bounded device-side wait gave up (see fdas_check) */
};

/* Limits checked by fdas_plan_create. */
#define FDAS_MIN_SEG_LEN 256
#define FDAS_MAX_SEG_LEN 8192

/*
 * Create a plan for an n_bins-bin spectrum, the z grid -zmax..zmax step zstep, segment
 * length seg_len and template span tmpl_len (Section 1, Eq. 2; Section 2 overlap-and-save).
 *
 *   n_bins    >= 4 and a multiple of 4, <= 2^30.
 *   zmax      >= 0, zstep >= 1, zmax % zstep == 0; Z = 2*zmax/zstep + 1 <= 65535.
 *   seg_len   L, a power of two in [FDAS_MIN_SEG_LEN, FDAS_MAX_SEG_LEN].
 *   tmpl_len  m, a multiple of 4 with 4 <= m <= L/2 (so V = L - m >= L/2, V % 4 == 0).
 *
 * Host call.  Validates the arguments before touching the device, then allocates the plan's
 * device memory on the current device: the template bank (Z*L complex64), the FP64 taps
 * (Z*(m+1) complex128), a twiddle table (L complex64) and a status word.  Returns NULL on
 * failure with fdas_last_error() set to FDAS_ERR_INVALID, FDAS_ERR_NO_DEVICE,
 * FDAS_ERR_UNSUPPORTED, FDAS_ERR_ALLOC or FDAS_ERR_CUDA.  The plan is used only on the device
 * that was current at creation.
 */
fdas_plan* fdas_plan_create(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len);

/* Code of the last failed fdas_plan_create on this thread (FDAS_OK if none). */
int fdas_last_error(void);

/* Static, NUL-terminated description of a status code. */
const char* fdas_error_string(int code);

/*
 * Build the template bank on the GPU (stream-ordered, asynchronous): for every z_idx the taps
 * H_q(z), q = -h..h, are computed in FP64 (composite Gauss-Legendre quadrature of the response
 * integral), normalised to unit L2 norm (the "predicted, normalized Fourier response" of
 * Section 1), conjugated, placed circularly so that the valid outputs of a segment are its
 * first V bins, transformed by an FP64 DFT of length L (1/L folded in) and stored as complex64.
 * Must complete before fdas_convolve_power (same stream, or synchronise).  Returns FDAS_OK,
 * FDAS_ERR_INVALID (NULL plan) or FDAS_ERR_CUDA.
 */
int fdas_templates_build(fdas_plan* plan, fdas_stream_t stream);

/*
 * The hot path (Eq. 2 by overlap-and-save, Section 2): one fused kernel launch on `stream`.
 *
 *   d_spectrum  n_bins complex64 values (interleaved re, im floats), device memory, 16-byte
 *               aligned, read-only, caller-owned.
 *   d_plane     Z x n_bins float32, row-major (row z_idx = (z + zmax)/zstep, pitch n_bins),
 *               16-byte aligned, caller-owned; every element is overwritten.  Device memory,
 *               or pinned host memory (cudaHostAlloc / cudaHostRegister, addressable by the
 *               device): the kernel then stores the plane straight into host memory over the
 *               host link, overlapping the transfer with the computation.
 *
 * Asynchronous: no host synchronisation and no allocation.  Returns FDAS_ERR_NOT_BUILT before
 * fdas_templates_build, FDAS_ERR_INVALID for NULL pointers, FDAS_ERR_ALIGN for misaligned
 * pointers, FDAS_ERR_CUDA if the launch fails.  Calls on one plan from different streams must
 * not overlap (they share the plan's status word).  A device-side bounded wait that gives up
 * is reported by the next fdas_check().
 */
int fdas_convolve_power(fdas_plan* plan, const float* d_spectrum, float* d_plane,
                        fdas_stream_t stream);

/*
 * The correlation with the segment transforms on the tensor cores (a reduced-precision variant;
 * the paper has no counterpart): for segment length 2048 only, each forward (Eq. 3 sign) and
 * inverse segment FFT is a 64-point DFT, a twist and a 32-point DFT done as DFT-matrix
 * contractions (tcgen05 MMAs) with BF16 (precision FDAS_TC_BF16) or FP16 (FDAS_TC_FP16) operands
 * split into hi + lo parts and FP32 accumulation; the DFT matrices are built in FP64 on the GPU.
 * Same inputs, outputs and error codes as fdas_convolve_power (FDAS_ERR_INVALID also for
 * seg_len != 2048 or another precision).  The first call on a plan (and the first after
 * fdas_templates_build) allocates and fills a workspace of Z*L*8 + nseg*L*8 + 320 KB bytes; later
 * calls allocate nothing.  Two kernel launches on `stream` (forward transforms into the
 * workspace, then the correlation).  Per-row error (max over the row of |P_tc - P|, over the
 * row's peak) on the 2^22-bin, 201-template survey plane: up to 1.1-1.3e-5 with BF16 operands and
 * about 4e-6 with FP16 (bound stated by the tests: 2e-4).
 */
#define FDAS_TC_BF16 0
#define FDAS_TC_FP16 1
int fdas_convolve_power_tc(fdas_plan* plan, const float* d_spectrum, float* d_plane, int precision,
                           fdas_stream_t stream);

/*
 * The forward segment transforms of fdas_convolve_power_tc alone, for tests: d_out (nseg x L
 * complex64, natural order, 16-byte aligned) receives X_s[k] = sum_j A[s V - h + j]
 * exp(-2 pi i j k / L) (A = 0 outside [0, n)), as fdas_segment_spectra but on the tensor cores.
 * Same errors and first-call allocation as fdas_convolve_power_tc; one launch on `stream`.
 */
int fdas_segment_spectra_tc(fdas_plan* plan, const float* d_spectrum, float* d_out, int precision,
                            fdas_stream_t stream);

/*
 * Synchronise `stream` and report the plan's device status word: FDAS_OK, FDAS_ERR_TIMEOUT
 * if a kernel of this plan abandoned a bounded wait (its outputs are then unspecified), or
 * FDAS_ERR_INVALID if a work list given to fdas_convolve_power_units failed its device-side
 * check (that call then wrote nothing); the word is cleared.  FDAS_ERR_CUDA if the
 * synchronisation itself fails.
 */
int fdas_check(fdas_plan* plan, fdas_stream_t stream);

/*
 * Failure-detection self test (no counterpart in the paper): launches one thread that waits, for
 * at most limit_ns nanoseconds (1 us .. 2 s), on a device barrier that nothing ever completes,
 * through the same bounded wait the fused kernel uses, and records the timeout in the plan's
 * status word.  The next fdas_check() on the stream returns FDAS_ERR_TIMEOUT and clears it; the
 * context stays usable.  Asynchronous on `stream`; FDAS_ERR_INVALID for a NULL plan or a limit
 * out of range.
 */
int fdas_selftest_wait_timeout(fdas_plan* plan, int64_t limit_ns, fdas_stream_t stream);

/* Free the plan's device memory.  Waits first for the last work the plan enqueued (not for the whole
 * device: work of other plans and other streams keeps running).  NULL is a no-op. */
int fdas_destroy(fdas_plan* plan);

/* Plan sizes: Z templates, V valid outputs per segment, nseg = ceil(n_bins / V) segments.
 * Any output pointer may be NULL. */
int fdas_plan_dims(const fdas_plan* plan, int* Z, int* V, int64_t* nseg);

/*
 * Introspection for tests (synchronising copies, not for the hot path).
 * fdas_template_taps: the normalised FP64 taps Hn_q(z) of row z_idx, q = -h..h, as 2*(m+1)
 *   doubles (re, im) into host memory.
 * fdas_template_spectrum: the stored complex64 template spectrum of row z_idx in natural
 *   order k = 0..L-1 (2*L floats into host memory): T[k] = (1/L) sum_q conj(Hn_q) e^{+i2pi k(q+h)/L}.
 * Both return FDAS_ERR_NOT_BUILT before fdas_templates_build and FDAS_ERR_INVALID for a bad
 * z_idx or NULL pointer.
 */
int fdas_template_taps(fdas_plan* plan, int z_idx, double* host_out);
int fdas_template_spectrum(fdas_plan* plan, int z_idx, float* host_out);

/*
 * Steps a2 + a3 alone, for tests of the in-kernel FFT: the forward FFT (Eq. 3 sign) of every
 * overlap-and-save segment, X_s[k] = sum_i A[s*V - h + i] e^{-i2pi ik/L} (zeros outside
 * [0, n_bins)), written in natural order to d_out (nseg x L complex64, interleaved floats,
 * device memory, 16-byte aligned, caller-owned).  Asynchronous on `stream`.
 */
int fdas_segment_spectra(fdas_plan* plan, const float* d_spectrum, float* d_out,
                         fdas_stream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Batches: many spectra of uneven lengths (e.g. the de-dispersion trials of one observation,
 * Section 1) correlated by ONE persistent kernel launch.  Every spectrum i has its own n_bins[i]
 * and zmax[i]; zstep, seg_len and tmpl_len are shared.  The batch holds one template bank for the
 * largest zmax (rows for smaller zmax are its middle rows).  The flattened (spectrum, segment
 * group, template) work is split into equal contiguous ranges over the SMs.  Segment lengths 512
 * and 2048 have this descriptor-driven kernel; the others (256, 1024, 4096, 8192) run one
 * single-spectrum launch per spectrum, in order on the stream.
 * ------------------------------------------------------------------------------------------- */
typedef struct fdas_batch fdas_batch;

/* Host call: validate every (n_bins[i], zmax[i], zstep, seg_len, tmpl_len) as fdas_plan_create
 * does, allocate the bank, the descriptor table (device) and its pinned staging.  NULL on
 * failure, code in fdas_batch_last_error().  count in [1, 2^20]; arrays are host memory. */
fdas_batch* fdas_batch_create(int count, const int64_t* n_bins, const int* zmax, int zstep, int seg_len,
                              int tmpl_len);
int fdas_batch_last_error(void);

/* Template bank (as fdas_templates_build) for zmax = max_i zmax[i]; stream-ordered. */
int fdas_batch_templates_build(fdas_batch* batch, fdas_stream_t stream);

/* Correlate every spectrum: d_spectra[i] (n_bins[i] complex64) -> d_planes[i] (Z_i x n_bins[i]
 * float32, Z_i = 2*zmax[i]/zstep + 1, row z_idx = (z + zmax[i])/zstep); both host arrays of
 * 16-byte-aligned device pointers.  Synchronises `stream` once (the descriptor staging is
 * reused), copies the descriptor table, then issues ONE kernel launch -- directly, or with
 * use_graph != 0 as a CUDA graph holding that launch (captured and instantiated on first use,
 * replayed afterwards).  Without the descriptor-driven kernel the graph holds the per-spectrum
 * launches and is captured again whenever the pointers differ from the captured ones.
 * FDAS_ERR_NOT_BUILT / INVALID / ALIGN / CUDA as fdas_convolve_power. */
int fdas_batch_convolve_power(fdas_batch* batch, const float* const* d_spectra, float* const* d_planes,
                              int use_graph, fdas_stream_t stream);

/* As fdas_check for the batch's status word. */
int fdas_batch_check(fdas_batch* batch, fdas_stream_t stream);
/* Waits for the batch's last enqueued work (not the whole device), then frees it. */
int fdas_batch_destroy(fdas_batch* batch);
/* seg_len, template-bank rows, total work units, segments resident per CTA (0: one launch per
 * spectrum); NULL outputs skipped. */
int fdas_batch_info(const fdas_batch* batch, int* seg_len, int* z_bank, int64_t* units, int* segments_per_cta);

/*
 * Autotuner (no counterpart in the paper): for each candidate segment length, build a batch,
 * time three launches on the caller's buffers with CUDA events (after one warm-up) and keep the
 * fastest; candidates that cannot serve the batch (tmpl_len > L/2) are skipped and
 * reported as -1 in ms_out (n_candidates floats, may be NULL).  The planes are overwritten.
 * Returns FDAS_OK with *best_seg_len set, FDAS_ERR_INVALID if no candidate applies.
 */
int fdas_batch_autotune(int count, const int64_t* n_bins, const int* zmax, int zstep, int tmpl_len,
                        const int* seg_len_candidates, int n_candidates, const float* const* d_spectra,
                        float* const* d_planes, fdas_stream_t stream, int* best_seg_len, float* ms_out);

/* ---------------------------------------------------------------------------------------------
 * Work lists.  The descriptor-driven kernel (seg_len 512 and 2048) groups
 * fdas_plan_group_segments(plan) = G consecutive segments; a work unit is g*Z + z (segment
 * group g, template z_idx).  fdas_convolve_power_units computes only the listed units (ascending,
 * device int32 array, 4-byte aligned) and writes only their cells: the rows z of the bins
 * [g*G*V, (g+1)*G*V) of each listed (g, z); every other cell of d_plane is left untouched.
 * Each cell equals the one fdas_convolve_power writes.  The list is checked on the device
 * (strictly increasing, every entry in [0, ceil(nseg/G)*Z)); a list that fails is not run
 * and the next fdas_check() returns FDAS_ERR_INVALID.  Asynchronous, no allocation.
 * FDAS_ERR_INVALID for a seg_len without that kernel.
 * ------------------------------------------------------------------------------------------- */
int fdas_plan_group_segments(const fdas_plan* plan);
int fdas_convolve_power_units(fdas_plan* plan, const float* d_spectrum, float* d_plane, const int32_t* d_units,
                              int64_t n_units, fdas_stream_t stream);
/* As fdas_convolve_power_units with a segment mask per list entry (device uint16 array parallel
 * to d_units, 2-byte aligned, or NULL for all segments): bit j set = segment g*G + j of the
 * entry's group is computed for its template; only the cells of those segments (bins
 * [(g*G+j)*V, (g*G+j+1)*V)) are written.  A warp whose segments are all unset skips its
 * transforms, so sparse masks cost less. */
int fdas_convolve_power_units_masked(fdas_plan* plan, const float* d_spectrum, float* d_plane,
                                     const int32_t* d_units, const uint16_t* d_masks, int64_t n_units,
                                     fdas_stream_t stream);
/* As fdas_convolve_power_units_masked (d_masks may be NULL), with the list length read on the
 * device from *d_count (int64, 8-byte aligned: e.g. the length fdas_zband_work_units_masked
 * leaves in its workspace) instead of passed by the host, so that a proposal, its work list and
 * the correlation run without a host synchronisation.  max_units >= 1 is the capacity of d_units
 * (and d_masks); a *d_count outside [0, max_units] fails the device-side check like a bad list
 * (nothing runs, the next fdas_check() returns FDAS_ERR_INVALID).  The paper has no
 * counterpart. */
int fdas_convolve_power_units_device_count(fdas_plan* plan, const float* d_spectrum, float* d_plane,
                                           const int32_t* d_units, const uint16_t* d_masks, const int64_t* d_count,
                                           int64_t max_units, fdas_stream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Pair lists (seg_len 2048 only; the paper has no counterpart).  A pair is s*Z + z: segment s
 * (outputs [s*V, (s+1)*V), fed by the input bins [s*V - m/2, s*V - m/2 + seg_len)) and template
 * z_idx.  fdas_convolve_power_pairs computes only the listed pairs (ascending, device int32
 * array, 4-byte aligned) and writes only their cells: row z of the bins [s*V, min((s+1)*V, n))
 * of each listed (s, z); every other cell of d_plane is left untouched.  Each cell equals the one
 * fdas_convolve_power writes (the same transforms, Section 2 and Eq. 2-3).  The list is cut into
 * equal contiguous ranges, one per warp of the grid, so a sparse list costs about its share of the
 * full plane's transforms however its pairs are spread over segments and templates (each warp
 * also runs the forward transform of every segment its range enters).  The list is checked on
 * the device (strictly increasing, every entry in [0, nseg*Z)); a list that fails is not run and
 * the next fdas_check() returns FDAS_ERR_INVALID.  Asynchronous, no allocation.  FDAS_ERR_INVALID
 * for NULL pointers, n_pairs < 1 or a plan whose seg_len is not 2048; FDAS_ERR_ALIGN for
 * misaligned pointers; FDAS_ERR_NOT_BUILT before fdas_templates_build.
 * ------------------------------------------------------------------------------------------- */
int fdas_convolve_power_pairs(fdas_plan* plan, const float* d_spectrum, float* d_plane, const int32_t* d_pairs,
                              int64_t n_pairs, fdas_stream_t stream);
/* As fdas_convolve_power_pairs with the list length read on the device from *d_count (int64,
 * 8-byte aligned: e.g. the length fdas_zband_work_pairs leaves in its workspace); max_pairs >= 1
 * is the capacity of d_pairs, and a *d_count outside [0, max_pairs] fails the device-side check
 * like a bad list. */
int fdas_convolve_power_pairs_device_count(fdas_plan* plan, const float* d_spectrum, float* d_plane,
                                           const int32_t* d_pairs, const int64_t* d_count, int64_t max_pairs,
                                           fdas_stream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Learned z-band proposal (no counterpart in the paper): a 1-D convolutional network over the
 * z = 0 power spectrum (the plane's z = 0 row, Eq. 2 with the unit-impulse template) that
 * predicts, for each block of bins, which of Z templates are worth correlating there.
 *
 *   x_r    = min(|A_r|^2 * ln 2 / med, 64)   med: lower median (rank (n-1)/2) of |A|^2 over the
 *            whole spectrum, so white-noise bins have mean 1 whatever the signals (x = 0 if med = 0)
 *   window w of width W (hop H = W/2): x over bins [w*H - W/4, w*H + 3W/4), 0 outside [0, n)
 *   three k = 9 convolutions with dilations 1, 4, 16 (tap k of a layer with dilation d reads
 *   position t + (k - 4) d), 32 channels, zero padding at the window edge, ReLU: a layer-3
 *   position sees +-84 bins;
 *   the maximum of each channel over the central half [W/4, 3W/4) (= block [w*H, (w+1)*H));
 *   a linear layer to Z logits; training loss: mean BCE-with-logits against 0/1 targets.
 *
 * Parameters are one FP32 vector: W1 [32][1][9], b1 [32], W2 [32][32][9], b2 [32],
 * W3 [32][32][9], b3 [32], Wl [Z][32], bl [Z]; an FP16 copy is kept for inference.
 * Training (FP32 forward, backward and Adam) and windowed inference run on the CUDA cores;
 * fdas_zband_propose runs the layers once over a whole spectrum on the tensor cores.  The median
 * is found exactly on the device (radix selection on the FP32 bit patterns of |A_r|^2).
 * ------------------------------------------------------------------------------------------- */
typedef struct fdas_zband fdas_zband;

/* window W: a multiple of 128 in [384, 65536] (the receptive field, +-84, must fit in a quarter
 * window); n_out = Z in [1, 65535]; max_batch windows per call in [1, 65535].  Requires a compute capability 10.3 device (current device).  NULL on
 * invalid arguments, another device, or allocation failure.  Parameters start at zero: set
 * them before use.  Device memory ~ 5 * max_batch * 32 * W floats. */
fdas_zband* fdas_zband_create(int window, int n_out, int max_batch);
int fdas_zband_param_count(const fdas_zband* net);
/* Host copies of the FP32 parameters (param_count floats).  Setting refreshes the FP16 copy and
 * resets Adam (moments zero, step 0).  Both wait for the net's own last enqueued work (train
 * steps, predictions, proposals, on whatever stream) and return when the copy is complete; they
 * do not synchronise the device. */
int fdas_zband_set_params(fdas_zband* net, const float* host_params);
int fdas_zband_get_params(fdas_zband* net, float* host_params);
/* Adam state for checkpoints: first and second moments (param_count floats each) and the step
 * count.  Set after fdas_zband_set_params to resume training.  Wait as fdas_zband_get_params. */
int fdas_zband_get_adam(fdas_zband* net, float* host_m, float* host_v, int* host_step);
int fdas_zband_set_adam(fdas_zband* net, const float* host_m, const float* host_v, int step);
/* One Adam step (lr > 0; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on `batch` windows of
 * x (device, batch x W floats, as fdas_zband_spectrum_windows makes them) with 0/1 targets
 * (device, batch x Z).  The mean BCE loss is written to *host_loss when non-NULL (then
 * synchronising `stream`).  Asynchronous otherwise. */
int fdas_zband_train_step(fdas_zband* net, const float* d_windows, const float* d_targets, int batch, float lr,
                          float* host_loss, fdas_stream_t stream);
/* Gradients of the last train step (host, param_count floats; waits as fdas_zband_get_params). */
int fdas_zband_gradients(fdas_zband* net, float* host_grads);
/* Logits (device, batch x Z) for windows of x on the CUDA cores (FP32 activations);
 * half_weights != 0 uses the FP16 copy of the parameters. */
int fdas_zband_predict(fdas_zband* net, const float* d_windows, int batch, int half_weights, float* d_logits,
                       fdas_stream_t stream);
/* Logits of every block of a whole spectrum, fused on the tensor cores: d_spectrum n_bins
 * complex64 (device, 8-byte aligned), d_logits ceil(n_bins / H) x Z floats (device).  Row w is
 * the network's output for window w (the same value fdas_zband_predict gives for that window,
 * up to FP16 rounding of the activations).  Requires H = W/2 to be a multiple of 128 and at
 * most 512 (W = 512, 768 or 1024).  Asynchronous; uses the net's scratch, so calls on one net
 * must not overlap.  Its eight launches (exact median, inference) run as a CUDA graph: the first
 * call with a given (d_spectrum, n_bins, d_logits) captures and instantiates it (driver
 * allocations), later calls with the same arguments replay it with no allocation; new weights
 * need no new capture.  A bounded device wait that gives up is reported by fdas_zband_check. */
int fdas_zband_propose(fdas_zband* net, const float* d_spectrum, int64_t n_bins, float* d_logits,
                       fdas_stream_t stream);
/* Synchronise `stream`; FDAS_ERR_TIMEOUT if fdas_zband_propose abandoned a bounded wait (its
 * logits are then unspecified), else FDAS_OK; clears the net's status word. */
int fdas_zband_check(fdas_zband* net, fdas_stream_t stream);
/* Windows of x for a whole spectrum (n_bins <= 2^30 complex64, 8-byte aligned): window w covers
 * bins [w*hop - window/4, w*hop + 3*window/4), zeros outside [0, n_bins).  window a multiple of
 * 4.  d_windows: n_windows x window floats.  Uses stream-ordered scratch allocations. */
int fdas_zband_spectrum_windows(const float* d_spectrum, int64_t n_bins, int window, int hop, float* d_windows,
                                int64_t n_windows, fdas_stream_t stream);
/* Work list from block logits (device, n_windows x Z): unit g*Z + z is kept when
 * logit >= log(threshold / (1 - threshold)) (i.e. sigmoid(logit) >= threshold, 0 < threshold
 * < 1) for template z in a block w whose bins [w*hop, (w+1)*hop) meet [g*group_bins - h,
 * (g+1)*group_bins + h) (group_bins = G*V: the outputs of segment group g and the input bins
 * its templates reach).  Writes the ascending list to d_units (room for n_groups*Z int32) and
 * its length to *host_count (synchronises `stream`).  d_scratch: device workspace of at least
 * fdas_zband_work_units_scratch_bytes(n_groups, Z) bytes, 16-byte aligned, caller-owned, or
 * NULL for stream-ordered allocations inside the call (which the memory pool may return to the
 * system at the synchronisation, making every call map them again).  With a caller workspace,
 * host_count may be NULL: the call is then fully asynchronous and the length stays on the device,
 * as the int64 at ((const int64_t*)d_scratch)[n_groups], for
 * fdas_convolve_power_units_device_count. */
int64_t fdas_zband_work_units_scratch_bytes(int64_t n_groups, int Z);
int fdas_zband_work_units(const float* d_logits, int64_t n_windows, int Z, float threshold, int hop,
                          int64_t group_bins, int h, int64_t n_groups, int32_t* d_units, void* d_scratch,
                          int64_t* host_count, fdas_stream_t stream);
/* As fdas_zband_work_units, per segment: group g holds G (1..16) segments of seg_bins = V bins;
 * segment j is proposed for template z when a block meets [(g*G+j)*V - h, (g*G+j+1)*V + h) with
 * sigmoid(logit) >= threshold, and unit g*Z + z is listed when any of its G segments is.
 * d_masks (device uint16, room for n_groups*Z, 2-byte aligned; may be NULL) receives each listed
 * unit's segment bits, for fdas_convolve_power_units_masked.  fdas_zband_work_units is the case
 * G = 1, seg_bins = group_bins. */
int fdas_zband_work_units_masked(const float* d_logits, int64_t n_windows, int Z, float threshold, int hop,
                                 int64_t seg_bins, int G, int h, int64_t n_groups, int32_t* d_units,
                                 uint16_t* d_masks, void* d_scratch, int64_t* host_count, fdas_stream_t stream);
/* Pair list from block logits (device, n_windows x Z), for fdas_convolve_power_pairs.  Segment s
 * (seg_bins = V) has the outputs [s*V, (s+1)*V) and draws on the inputs [s*V - h, (s+1)*V + h).
 * A template q is proposed for it by a block w (bins [w*hop, (w+1)*hop)) that meets its outputs
 * with sigmoid(logit[w][q]) >= threshold, or by a block that meets only the inputs beyond them
 * with sigmoid(logit[w][q]) >= reach_threshold (only a strong signal there has a response that
 * reaches the segment's outputs); pair s*Z + z is listed when a template within z_halo
 * (0 <= z_halo <= Z) of z is proposed.  0 < threshold < 1, threshold <= reach_threshold <= 1
 * (reach_threshold = threshold: every block the inputs meet counts alike).  z_halo widens each
 * proposal for signals the network places only roughly in z.  Writes the ascending list to
 * d_pairs (room for n_seg*Z int32; n_seg*Z <= 2^31 - 1, Z <= 8192) and its length to *host_count
 * (synchronises `stream`), or with host_count NULL leaves it on the device as the int64 at
 * ((const int64_t*)d_scratch)[n_seg].  d_scratch: 16-byte aligned caller workspace of
 * fdas_zband_work_units_scratch_bytes(n_seg, Z) bytes (required); d_logits and d_pairs 4-byte
 * aligned (FDAS_ERR_ALIGN otherwise).  Asynchronous when host_count is NULL; three launches, no
 * allocation. */
int fdas_zband_work_pairs(const float* d_logits, int64_t n_windows, int Z, float threshold, float reach_threshold,
                          int z_halo, int hop, int64_t seg_bins, int h, int64_t n_seg, int32_t* d_pairs,
                          void* d_scratch, int64_t* host_count, fdas_stream_t stream);
/* Waits for the net's last enqueued work (not the whole device), then frees it. */
int fdas_zband_destroy(fdas_zband* net);

/*
 * Allocation-free variant of fdas_convolve_power, for callers that cannot allocate device
 * memory: code on a latency-critical path where cudaMalloc may synchronise the device and take
 * unbounded time, components whose device memory is entirely reserved up front by a pooling
 * allocator (so cudaMalloc fails or fragments the pool), and host applications or plugin hosts
 * that forbid run-time allocation.  The paper has no counterpart; this call only removes the
 * plan's allocations.
 *
 * It computes exactly what fdas_plan_create + fdas_templates_build + fdas_convolve_power compute
 * for the same arguments (same validation, same kernels), but keeps the template bank, the FP64
 * taps, the twiddle table and the status word in one file-scope device array of
 * FDAS_STATIC_SCRATCH_BYTES bytes instead of plan memory.  That array exists on every GPU that
 * loads the library and is held until the process exits.  The call makes no cudaMalloc, cudaFree
 * or other allocating call.
 *
 *   n_bins, zmax, zstep, seg_len, tmpl_len   as for fdas_plan_create; in addition
 *       Z*L*8 + Z*(m+1)*16 + L*8 (each rounded up to 256) + 256 bytes must fit in
 *       FDAS_STATIC_SCRATCH_BYTES (the 2^22-bin, 201-template, L=2048, m=512 survey geometry
 *       needs 4.96 MB), else FDAS_ERR_INVALID before any device work.
 *   d_spectrum, d_plane, stream               as for fdas_convolve_power (caller-owned, 16-byte
 *       aligned device memory; the plane is fully overwritten).
 *
 * Asynchronous on `stream`.  The first call on a device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.  The template bank is
 * rebuilt (FP64, tens of ms for the survey geometry) whenever (zmax, zstep, seg_len, tmpl_len)
 * differs from the previous call on the same device, and reused otherwise.  A call that finds the
 * bank already built still depends on the stream of the call that built it: order the first call
 * before calls on other streams.  All calls share the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other host threads without ordering)
 * race.  A bounded device wait that gives up leaves the plane unspecified and sets the array's
 * status word, which accumulates over calls until fdas_static_check reads and clears it.  Returns
 * FDAS_OK, FDAS_ERR_INVALID, FDAS_ERR_ALIGN, FDAS_ERR_NO_DEVICE, FDAS_ERR_UNSUPPORTED or
 * FDAS_ERR_CUDA.
 */
#define FDAS_STATIC_SCRATCH_BYTES (8u << 20)
int fdas_convolve_power_static(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len,
                               const float* d_spectrum, float* d_plane, fdas_stream_t stream);

/*
 * Status of the allocation-free calls on the current device (the paper has no counterpart; this is
 * the static array's analogue of fdas_check).  Synchronises `stream`, reads the status word kept in
 * the static array, clears it and returns FDAS_ERR_TIMEOUT if a bounded device wait of any
 * fdas_convolve_power_static call since the last check gave up (those planes are unspecified),
 * FDAS_OK otherwise, FDAS_ERR_CUDA on a runtime error.  Allocates nothing.
 */
int fdas_static_check(fdas_stream_t stream);

/*
 * Failure-detection self test of the static array's status word (no counterpart in the paper): as
 * fdas_selftest_wait_timeout, one thread waits at most limit_ns (1 us .. 2 s) on a barrier nothing
 * completes and records the timeout in the static array's status word; the next
 * fdas_static_check returns FDAS_ERR_TIMEOUT.  Asynchronous on `stream`; FDAS_ERR_INVALID for a
 * limit out of range.  Allocates nothing.
 */
int fdas_static_selftest_wait_timeout(int64_t limit_ns, fdas_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
