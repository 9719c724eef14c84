/*
 * corr.h -- C ABI of the GB300 FX correlator library (libcorr.so).
 *
 * What it computes.  The paper (Bruni et al., "Space-VLBI with RadioAstron:
 * new correlator capabilities at MPIfR", Abstract) describes DiFX as an FX
 * correlator: every station's sampled voltage is Fourier transformed first,
 * then each station pair is cross-multiplied and accumulated.  Its Sec. 2
 * describes the dra version's delay model (Calc extended to a spacecraft
 * with arbitrary position and velocity, general-relativistic terms, and the
 * spacecraft -> tracking-station transmission leg) and the RadioAstron ->
 * Mark5B data conversion.  Both enter this library only as inputs: per-station
 * delay-polynomial segments (corr_set_delay_poly) and packed 2-bit sample
 * streams (corr_push_samples).  Per FFT block and station the library
 *   1. evaluates the delay polynomial in FP64 at the block centre and picks
 *      the integer-sample window [b*N + n_b, +N), n_b = floor(tau*fs + 1/2);
 *   2. unpacks the 2-bit samples of that window (4-entry level table);
 *   3. takes the N-point real FFT and keeps channels k = 0..nchan-1 (N = 2*nchan);
 *   4. multiplies by exp(+2 pi i (frac(nu0 tau) + k*fs/N * eps)), eps = tau - n_b/fs
 *      (fractional-delay slope and fringe rotation, after the FFT);
 *   5. accumulates V_ab[k] += X_a[k] conj(X_b[k]) for every a <= b;
 * and at the end of each integration returns V_ab / (W_ab * N), W_ab being
 * the number of blocks valid at both stations.
 *
 * Input format.  One byte stream per station; G = subbands*pols streams are
 * interleaved per sample time, stream j = subband*pols + pol; the 2-bit code
 * of stream j at sample-time t (counted from the station's first pushed
 * sample) sits at bit 2*(t*G + j) of the byte stream, bytes least-significant
 * bit first.  Default levels: code 0 -> -3.336, 1 -> -1, 2 -> +1, 3 -> +3.336.
 *
 * Output layout.  Visibilities are complex64 stored as interleaved float
 * pairs (re, im) in [baseline][subband][pol][channel] order; baselines run
 * (0,0),(0,1),...,(0,S-1),(1,1),...,(S-1,S-1), nbl = S(S+1)/2.  Weights are
 * one double per baseline.
 *
 * Times are seconds relative to the scan epoch, in FP64.  Block b covers
 * geocentric samples [b*N, b*N + N); integration i holds the blocks with
 * i <= b*N / (fs*tint) < i+1 (fs*tint must be a whole number of samples).
 *
 * Errors.  Every entry point returns CORR_OK (0) or a negative code; no
 * exception crosses the ABI.  Arguments are checked before any device work.
 * corr_last_error() gives a text for the last failure on a handle (or, with a
 * NULL handle, for the last failed corr_create on this thread).
 *
 * Threads and devices.  A handle is not thread-safe.  It lives on the CUDA
 * device that was current at corr_create and makes that device current at
 * every call.  Device work runs on the handle's stream (its own, or the one
 * given to corr_set_stream).
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct corr_s corr_t;

enum {
  CORR_OK = 0,
  CORR_EINVAL = -1,   /* bad argument (nothing was changed)                      */
  CORR_ENOMEM = -2,   /* device or host allocation failed                         */
  CORR_EAGAIN = -3,   /* a station has not pushed the samples this integration needs */
  CORR_ETIMEOUT = -4, /* a device wait did not finish in time                     */
  CORR_ECUDA = -5,    /* a CUDA call failed (text in corr_last_error)             */
  CORR_ESTATE = -6,   /* call not allowed in the handle's current state           */
  CORR_EEND = -7,     /* after corr_flush: no station has data for the next integration */
  CORR_ETOOBIG = -8   /* corr_correlate_static: the shape needs more than its fixed scratch */
};

/* Arithmetic of the X step: FP32 on CUDA cores, or FP16 or FP8 (E4M3)
 * spectra multiplied on the tensor cores with FP32 accumulation (at most 64
 * stations).  The paper's FX correlator (Abstract: Fourier transform, then
 * cross-multiply) fixes no arithmetic precision; the reduced-precision modes
 * trade a stated error against the FP64 definition for tensor-core speed. */
enum { CORR_PREC_FP32 = 0, CORR_PREC_FP16_TC = 1, CORR_PREC_FP8_TC = 2 };

/* Create a correlator for one scan: the FX correlation the paper's Abstract
 * describes (each station's samples Fourier transformed, then every station
 * pair cross-multiplied and accumulated), for `stations` stations recording
 * `subbands` subbands in `pols` polarisations, with nchan channels per
 * subband (2*nchan-point transforms) and integrations of tint_s seconds.
 * stations 1..256, subbands*pols 1..32, pols 1 or 2, nchan a power of two in
 * 4..8192, tint_s > 0.  *h receives the handle (NULL on failure).  Allocates
 * host state only; device memory is allocated at the first corr_correlate*
 * call. */
int corr_create(corr_t **h, int stations, int subbands, int pols, int nchan, double tint_s);

/* Sample rate per stream (Hz, default 32e6) and the code -> level table
 * (NULL keeps the current one).  Only before the first correlate call. */
int corr_set_format(corr_t *h, double fs_hz, const float lut[4]);

/* Sky (LO) frequency of a subband in Hz, used for the fringe rotation
 * exp(+2 pi i frac(nu0 tau)).  Default 0 (no fringe rotation). */
int corr_set_sky_freq(corr_t *h, int subband, double nu0_hz);

/* Arithmetic of the X step: CORR_PREC_FP32 (default), CORR_PREC_FP16_TC or
 * CORR_PREC_FP8_TC.  In FP16_TC mode the F step stores X * 2^-floor(log2(N)/2)
 * in FP16 (exact power of two, undone at the end) and the X step runs as a
 * real product of interleaved [Re; Im] station rows on the tensor cores,
 * accumulating in FP32.  FP8_TC does the same with E4M3 values (3 mantissa
 * bits, largest 448) of X * 2^(2 - floor(log2(N)/2)): for 2-bit noise the RMS
 * of a component sits near 8, values beyond 448 saturate.  Rejects more than
 * 64 stations for the tensor-core modes (CORR_EINVAL).  Only before the first
 * correlate call (CORR_ESTATE). */
int corr_set_precision(corr_t *h, int mode);

/* Which unit multiplies the FP16 / FP8 spectra of the reduced-precision
 * modes (no effect in CORR_PREC_FP32).  CORR_X_AUTO (the default): the CUDA
 * cores for up to 12 (station, polarisation) rows of the X step (stations,
 * or 2 x stations with both hands) and whole 128-channel tiles, where a
 * 128-row tensor-core tile would hold at most 6 channels' worth of useful
 * products and building its operand tiles costs more than the X step it
 * speeds up; the tensor cores above.  CORR_X_CUDA_CORES: the CUDA cores
 * where that form applies (else the tensor cores).  CORR_X_TENSOR_CORES:
 * always the tensor cores.  On the CUDA cores every product of FP16 (E4M3)
 * values is exact in FP32 and the sums are FP32, as on the tensor cores,
 * so the result lies within the same stated bound of the FP64 definition;
 * the order of the FP32 additions differs.  Only before the first correlate
 * call (CORR_ESTATE); an unknown unit is CORR_EINVAL. */
enum { CORR_X_AUTO = 0, CORR_X_CUDA_CORES = 1, CORR_X_TENSOR_CORES = 2 };
int corr_set_x_unit(corr_t *h, int unit);

/* Where the fringe rotation is applied.  CORR_ROT_POST_F (the default): after
 * the transform, one phase frac(nu0 tau(t_c)) per block and channel slope, as
 * in step 4 above.  CORR_ROT_PRE_F: before the transform, every sample x[n] of
 * a block is multiplied by exp(+2 pi i (frac(nu0 tau(t_c)) + nu0 tau'(t_c)
 * (n - N/2) / fs)) -- the fringe phase linear about the block centre, tau'
 * the delay polynomial's derivative, phase and rate from the FP64 delay model
 * and FP32 increments within the block -- then a complex N-point transform
 * keeps channels 0..nchan-1 and applies exp(+2 pi i k fs/N eps).  At a
 * spacecraft's delay rate the fringe phase turns several times within one
 * block (the paper, Sec. 2: the delay model follows RadioAstron's large and
 * fast-changing velocity; at 4.8 GHz and 3e-5 s/s, 9 turns in a 64 us block);
 * post-F rotation then loses the fringe to that drift (|sinc(turns per
 * block)|) while pre-F keeps it.  The lowest channels receive the image of
 * the negative frequencies shifted by twice the fringe rate.  Pre-F takes
 * nchan <= 4096 (CORR_EINVAL otherwise) and about twice the F-step work.
 * Only before the first correlate call (CORR_ESTATE). */
enum { CORR_ROT_POST_F = 0, CORR_ROT_PRE_F = 1 };
int corr_set_fringe_rotation(corr_t *h, int mode);

/* Mark5B-style framed input (the paper, Sec. 2: RadioAstron recordings are
 * converted to Mark5B).  With payload_bytes > 0 (a multiple of 16; Mark5B
 * uses 10000) every station's pushed or attached bytes are frames of a
 * 16-byte header and payload_bytes of payload; the payloads in frame order
 * are the packed stream described at the top of this file.  A frame whose
 * first header word (32-bit little-endian) is not the sync word 0xABADDEED
 * is taken as lost: every block that reads a sample from it is not valid at
 * that station.  Only whole frames count as data.  The library deframes new
 * frames on the device before each correlate call (a copy of the payloads,
 * held in device memory of its own).  0 (the default): plain packed bytes.
 * Only before any samples are pushed or attached (CORR_ESTATE). */
int corr_set_frame_format(corr_t *h, int payload_bytes);

/* Which polarisation products the X step forms.  CORR_POL_PARALLEL (the
 * default): each polarisation with itself, V_ab^pp, output
 * [baseline][subband][pol][channel].  CORR_POL_CROSS (pols = 2 only): all
 * four hand products V_ab^pq[k] = sum over blocks of X_a^p[k] conj(X_b^q[k]),
 * p, q in {0, 1} (for circular feeds RR, RL, LR, LL), output
 * [baseline][subband][pq = 2p + q][channel] -- twice the output of the
 * parallel hands, so the out buffers of corr_correlate* hold
 * nbl * subbands * 4 * nchan complex values.  The polarisation key science
 * programmes that the paper's AO-1 correlation serves (Sec. 1) need them.
 * The X step runs over 2S (station, pol) pairs per subband, about twice the
 * parallel hands' work; the tensor-core modes then take at most 32 stations.
 * Only before the first correlate call (CORR_ESTATE). */
enum { CORR_POL_PARALLEL = 0, CORR_POL_CROSS = 1 };
int corr_set_pol_products(corr_t *h, int mode);

/* FFT blocks per F/X chunk (0, the default: as many as fit 1 GiB of FP32
 * spectra, capped at one integration).  Smaller chunks keep the spectra in
 * L2 between the F and X kernels.  Only before the first correlate call. */
int corr_set_chunk_blocks(corr_t *h, int blocks);

/* Schedule of the F and X steps.  1 (the default): two spectra (or
 * tensor-core tile) buffers, and the X step of each chunk runs on a second,
 * higher-priority stream while the F step of the next chunk runs, whenever
 * one buffer takes at most 4 GiB; 0: one buffer, F and X in turn.  Either
 * way the next integration's delay blocks are evaluated on a side stream
 * during the current one.  The results are the same; 1 is faster and holds
 * the spectra twice (corr_device_bytes tells).  Only before the first
 * correlate call. */
int corr_set_pipeline(corr_t *h, int overlap);

/* Run device work on this cudaStream_t (NULL: the handle's own stream). */
int corr_set_stream(corr_t *h, void *cuda_stream);

/* Append a delay-polynomial segment for a station:
 * tau(t) = sum_{i=0..5} coeffs[i] (t - t0_s)^i seconds, valid from t0_s until
 * the next segment.  t0_s must increase per station (CORR_EINVAL otherwise);
 * at most 64 segments per station.  A block whose centre precedes the first
 * segment is not valid.  The delay polynomials come from the delay model
 * (paper, Sec. 2); a positive tau means the station receives later. */
int corr_set_delay_poly(corr_t *h, int station, double t0_s, const double coeffs[6]);

/* Station sample index of the first sample that will be pushed (default 0):
 * a recording that starts before or after the scan epoch.  Only before the
 * station's first push or attach. */
int corr_set_stream_start(corr_t *h, int station, int64_t first_sample);

/* Reserve device room for nbytes of a station's packed samples (optional). */
int corr_reserve(corr_t *h, int station, size_t nbytes);

/* Append packed bytes (host memory) to a station's stream: the station's
 * recorded samples as the paper's data path delivers them (Sec. 2: the
 * RadioAstron recordings converted to Mark5B), in the packing described at
 * the top of this file (or in frames, see corr_set_frame_format).  nbytes
 * must be a multiple of 4.  The bytes are copied to the device before the
 * call returns, so the caller may reuse the buffer; pinned host memory copies
 * fastest. */
int corr_push_samples(corr_t *h, int station, const void *bytes, size_t nbytes);

/* Append packed bytes without waiting for the copy: the copy runs on the
 * handle's copy streams and overlaps correlation; a later corr_correlate*
 * call makes its device work wait for the pushed pieces it reads.  bytes
 * should be pinned host memory (pageable memory works but copies without
 * overlap) and must stay unchanged until corr_wait_pushes returns (or the
 * handle is reset or destroyed).  nbytes must be a multiple of 4.  Growing
 * the station's device buffer (push beyond corr_reserve) waits for earlier
 * copies first. */
int corr_push_samples_async(corr_t *h, int station, const void *bytes, size_t nbytes);

/* Wait until every asynchronous push of the handle has landed in device
 * memory (the host buffers may then be reused). */
int corr_wait_pushes(corr_t *h);

/* Use nbytes of packed samples that already live in device memory of the
 * handle's device (16-byte aligned, nbytes a multiple of 4) as the station's
 * whole stream.  The caller keeps ownership and must keep the memory alive
 * and unchanged until corr_destroy or corr_reset.  No push is allowed for
 * that station afterwards. */
int corr_attach_samples_device(corr_t *h, int station, const void *dev_bytes, size_t nbytes);

/* Use nbytes of packed samples in pinned (page-locked, mapped) host memory as
 * the station's whole stream without copying it: the F step's loads read the
 * samples over the host link (on GB300, NVLink-C2C) as it needs them, each
 * byte once.  16-byte aligned, nbytes a multiple of 4; the caller keeps the
 * memory alive and unchanged until corr_destroy or corr_reset.  No push is
 * allowed for that station afterwards. */
int corr_attach_samples_host(corr_t *h, int station, const void *host_bytes, size_t nbytes);

/* Declare the end of data: integrations that reach past a station's data are
 * then produced with those blocks marked invalid instead of CORR_EAGAIN. */
int corr_flush(corr_t *h);

/* Correlate the next integration and copy it to host memory: steps 1-5 at
 * the top of this file for every block of the integration -- the FX order of
 * the paper's Abstract, with each station's delay taken from its delay-model
 * polynomial (Sec. 2) -- and V_ab / (W_ab * N) at its end.
 * out: nbl*subbands*pols*nchan complex64 (2 floats each; with both hands of
 * two polarisations nbl*subbands*4*nchan); weights: nbl doubles or NULL.  Returns CORR_EAGAIN (nothing consumed) when some station has not
 * pushed the samples the integration needs and corr_flush was not called,
 * CORR_EEND after corr_flush when no station has data left.  Blocks until the
 * device work is done. */
int corr_correlate(corr_t *h, float *out, double *weights);

/* As corr_correlate, but writes the visibilities to device memory dev_out
 * (same layout) and, if dev_weights is not NULL, the weights to device
 * memory; returns once the work is enqueued on the handle's stream. */
int corr_correlate_device(corr_t *h, float *dev_out, double *dev_weights);

/* Index of the integration the next correlate call produces. */
int corr_next_integration(const corr_t *h, int64_t *index);

/* Start again from integration 0, keeping data and delay model. */
int corr_rewind(corr_t *h);

/* Drop all pushed or attached samples and flush state, and rewind; the delay
 * model, format and stream starts are kept.  Also clears a device timeout
 * (CORR_ETIMEOUT) that a correlate call reported, so the handle can be used
 * again. */
int corr_reset(corr_t *h);

/* Text of the last error on h (NULL h: last corr_create failure). */
const char *corr_last_error(const corr_t *h);

/* Free the handle and its device memory (NULL is allowed). */
void corr_destroy(corr_t *h);

/* ---- several scans at once ------------------------------------------------
 *
 * Correlate the next integration of each of n handles in one launch: their
 * device work is recorded as parallel branches of one CUDA graph (up to 16
 * concurrent branches) and the graph is launched on cuda_stream (NULL: an
 * internal stream).  dev_out[j] / dev_weights[j] (device memory, weights may
 * be NULL) receive handle j's visibilities in the corr_correlate_device
 * layout.  Every handle must live on the current device, have corr_flush
 * called (its samples all pushed or attached) and profiling off; blocks
 * without data simply get zero weight.  Returns once the graph is launched;
 * synchronise cuda_stream before reading the outputs.  Each handle's
 * integration counter advances by one.  Not thread-safe per device. */
int corr_batch_run(corr_t *const *handles, int n, float *const *dev_out, double *const *dev_weights,
                   void *cuda_stream);

/* Device memory the handle holds once prepared: work buffers sized by the
 * shape, precision and chunk setting, plus sample buffers it owns (attached
 * samples are not counted).  Available before the first correlate, for
 * admission control by a scheduler.  CORR_EINVAL if fs*tint is not a whole
 * number of samples >= 2*nchan. */
int corr_device_bytes(corr_t *h, size_t *bytes);

/* ---- inspection of intermediate results (for tests; slow) ---------------- */

/* Delay-block results for blocks [b0, b0+nb) of all stations, each array
 * [stations][nb]: window start (station sample index), eps (s), tau (s),
 * validity (0/1) against the data present now.  Any pointer may be NULL. */
int corr_debug_delays(corr_t *h, int64_t b0, int64_t nb, int64_t *start, double *eps, double *tau,
                      uint8_t *valid);

/* 2-bit codes of one station's stream for sample-time groups [t0, t0+count)
 * counted from its first sample, as read on the device (0xFF outside). */
int corr_debug_codes(corr_t *h, int station, int stream, int64_t t0, int64_t count, uint8_t *codes);

/* The rotated spectrum of one station, stream and block (nchan complex64),
 * as the F step produces it; *valid receives the block's validity. */
int corr_debug_spectrum(corr_t *h, int station, int stream, int64_t block, float *out, int *valid);

/* Spins (polls of an mbarrier) before a device wait of the X kernels gives
 * up, for every launch after the call, process-wide; negative restores the
 * default (2^26, far beyond any wait a working kernel needs); 0 makes every
 * such wait give up at once.  A test hook for the timeout path: a kernel
 * whose wait gives up stops its work, waits (with the default bound) for the
 * bulk copies and tensor-core operations it has in flight, frees its tensor
 * memory and sets an error flag, which a handle reports as CORR_ETIMEOUT
 * (corr_correlate / the next call) and corr_correlate_static as NaN
 * visibilities.  The visibilities of such a call are not meaningful. */
int corr_debug_set_wait_limit(long long spins);

/* Time every stage launch with CUDA events on the handle's stream (off by
 * default).  Stages: 0 delay blocks, 1 F (unpack+FFT+rotate), 2 X
 * (cross-multiply-accumulate), 3 weights+finalise. */
int corr_set_profiling(corr_t *h, int enable);

/* Wait for the recorded events, return per stage the summed device time
 * (ms) and the number of launches since the last read, and reset them. */
int corr_read_profile(corr_t *h, double ms[4], int64_t launches[4]);

/* Blocks per F/X chunk and the number of X partial accumulators the handle
 * uses (valid after the first correlate call). */
int corr_launch_shape(const corr_t *h, int *chunk_blocks, int *kz);

/* ---- delay-rate fringe search ---------------------------------------------
 *
 * The wide-window fringe search the paper lists among the dra-DiFX features
 * for RadioAstron (Sec. 2): a map of one baseline's visibilities over
 * residual delay and fringe rate, and its peak.  For V[t][k] (t: one of nsub
 * sub-integrations, k: one of nchan channels; complex64 rows of nchan, device
 * memory, e.g. one baseline/stream of successive corr_correlate_device
 * outputs) the map is the zero-padded two-dimensional inverse DFT,
 * unnormalised:
 *     M[r][l] = sum_t sum_k V[t][k] exp(+2 pi i (k l / pad_delay + t r / pad_rate)),
 * written to dev_map (complex64 [pad_rate][pad_delay], device memory, owned
 * by the caller).  Lag l is a delay of l * 2 nchan / pad_delay samples
 * (l >= pad_delay / 2: l - pad_delay); rate bin r is a fringe rate of
 * r / (pad_rate * T_sub) Hz (r >= pad_rate / 2: r - pad_rate).  The peak is
 * the largest |M|, the smaller flat index r * pad_delay + l on ties; its rate
 * bin, lag, amplitude and complex value (2 floats) go to the host pointers
 * (each may be NULL).  pad_rate >= nsub and pad_delay >= nchan are powers of
 * two <= 16384 with pad_rate * pad_delay <= 2^26 (else CORR_EINVAL).  Work
 * space (pad_delay * nsub complex values) is taken with cudaMallocAsync on
 * cuda_stream (NULL: the legacy default stream) and released there
 * (CORR_ENOMEM if that fails); the call returns when the search is done
 * (CORR_ECUDA on a CUDA error). */
int corr_fringe_search(const float *dev_vis, int nsub, int nchan, int pad_rate, int pad_delay, float *dev_map,
                       int *peak_rate, int *peak_lag, float *peak_amp, float *peak_value, void *cuda_stream);

/* ---- correlation without device allocation -------------------------------
 *
 * The paper has no counterpart of this entry point; it exists for callers of
 * this library that cannot let it call cudaMalloc: a host program that owns a
 * fixed device-memory budget and forbids libraries to allocate after start-up,
 * or a real-time pipeline that must keep cudaMalloc/cudaFree (which can
 * synchronise the whole device) off its hot path.
 *
 * corr_correlate_static computes integration `integration` of a scan whose
 * packed samples already live in device memory, exactly as the handle path
 * does after corr_flush (blocks outside a station's data are not valid), and
 * writes visibilities to dev_out ([nbl][subbands][pols][nchan] complex64,
 * device memory) and, unless NULL, the weights to dev_weights (nbl doubles,
 * device memory).  The caller owns inputs and outputs.  The library allocates
 * nothing: its intermediates live in one static device array of 64 MiB that
 * every GPU loading the library holds until the process exits.  A shape whose
 * intermediates do not fit even with one FFT block per chunk (roughly:
 * stations x (8*subbands + 13) bytes per block of the integration plus
 * 8*nbl*subbands*pols*nchan bytes) is rejected with CORR_ETOOBIG.
 *
 * The first call on a device resolves the array's device address and loads
 * the FFT constants for that device (no allocation).  (After a
 * cudaDeviceReset the next call does this set-up again for the device's new
 * context.)  The calls are not meant for stream capture into a CUDA graph:
 * their copies of the caller's host descriptor arrays would be replayed from
 * the capturing call's host pointers.  Each call copies the
 * caller's descriptor arrays below from host memory with cudaMemcpyAsync on
 * cuda_stream, writes the station views and FFT twiddles it derives itself
 * with small kernels (their values travel as kernel parameters), and only
 * enqueues the work on cuda_stream (NULL: the legacy default stream) before
 * it returns.  All calls share the one array, which keeps the last call's
 * contents (the partial sums and a timeout flag are cleared at the start of
 * every call): calls whose device work overlaps -- on two streams, or from
 * two threads -- race and give wrong results.  Errors are reported by return
 * code only; a device wait of the X step that runs out of time (see
 * CORR_ETIMEOUT) cannot be reported that way, since the call has returned by
 * then, so it makes every visibility of the call NaN instead.
 *
 * Descriptor arrays are host memory: nu0_hz[subbands], nseg[stations] (1..64),
 * seg_t0[stations][64], seg_coeffs[stations][64][6] (delay segments as for
 * corr_set_delay_poly, unused rows ignored), and per station a device pointer
 * (16-byte aligned), its byte count (a multiple of 4) and its first station
 * sample index. */
typedef struct {
  int stations, subbands, pols, nchan;
  double fs_hz, tint_s;
  float lut[4];
  const double *nu0_hz;
  const int *nseg;
  const double *seg_t0;
  const double *seg_coeffs;
  const void *const *dev_bytes;
  const size_t *nbytes;
  const int64_t *first_sample;
} corr_scan_desc;

int corr_correlate_static(const corr_scan_desc *desc, int64_t integration, float *dev_out,
                          double *dev_weights, void *cuda_stream);

/* ---- continuous-batching server -------------------------------------------
 *
 * A correlation service for many scans of uneven shape (the workloads a
 * correlator centre such as the paper's, Sec. 1, runs one after another).
 * corr_server_start starts one worker thread on the device current at the
 * call.  Jobs submitted from any thread wait in a first-come-first-served
 * queue; the worker admits them while the device memory they need (the
 * handle's work buffers, corr_device_bytes, plus their output buffers) fits
 * hbm_cap_bytes - reserve_bytes, so jobs that arrive while others are on the
 * GPU join as memory frees up.  Every step advances every admitted job by
 * one integration in one CUDA graph (corr_batch_run) and calls each job's
 * callback, on the worker thread, with that integration's visibilities
 * (host memory, [nbl][subbands][pols][nchan] complex64, the corr_correlate
 * layout) and weights (nbl doubles), valid only during the call.  A job's
 * result does not depend on the other jobs in the mix (each keeps its own
 * work buffers and accumulation order).
 *
 * A job is a corr_scan_desc (shapes, format, delay model; the stations'
 * samples in device memory of the server's device, which the caller keeps
 * alive and unchanged until the job's last callback), the X-step precision
 * (CORR_PREC_*), the fringe-rotation form (CORR_ROT_*) and the number of
 * integrations to correlate from integration 0.  The descriptor arrays are
 * copied at submission.  A job that cannot fit even alone, or whose handle
 * cannot be made, gets one callback with vis = weights = NULL and status
 * CORR_ENOMEM or the handle's error code; so does every job still queued or
 * running at corr_server_stop (status CORR_ESTATE).
 *
 * corr_server_stats: median and 99th-percentile latency (nearest rank,
 * seconds from submission to the end of the last callback) over finished
 * jobs, station-samples per second from the first submission to the last
 * finish, and the number of finished jobs (any pointer may be NULL).
 * corr_server_wait blocks until every submitted job has finished
 * (timeout_s < 0: no limit; CORR_ETIMEOUT when the limit passes first).
 * corr_server_stop finishes the step in progress, fails what is left and
 * joins the worker. */
typedef struct corr_server_s corr_server_t;
typedef struct {
  corr_scan_desc scan;
  int precision;
  int rotation;
  int64_t integrations;
} corr_job;
typedef void (*corr_result_fn)(void *user, int64_t job_id, int64_t integration, const float *vis,
                               const double *weights, int status);
int corr_server_start(corr_server_t **srv, size_t hbm_cap_bytes, size_t reserve_bytes);
int corr_server_submit(corr_server_t *srv, const corr_job *job, corr_result_fn fn, void *user, int64_t *job_id);
int corr_server_stats(corr_server_t *srv, double *p50_s, double *p99_s, double *samples_per_s, int64_t *jobs_done);
int corr_server_wait(corr_server_t *srv, double timeout_s);
void corr_server_stop(corr_server_t *srv);

#ifdef __cplusplus
}
#endif
#endif /* CORR_H */
