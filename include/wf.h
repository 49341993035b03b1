/*
 * wf.h — C ABI of the GB300 (sm_103a) B-mode reconstruction library.
 *
 * The library implements the imaging pipeline of the paper's Fig. 2 as
 * hand-written CUDA kernels:
 *
 *   RF channel data --wf_das_stai / wf_das_pwi--> beamformed image
 *                   --wf_envelope--> |analytic signal| along depth
 *                   --wf_logclip--> 20 log10(env / ref) clipped to [lo, hi] dB
 *
 * Sec. II-B of the paper lists the operators (DAS beamformer for synthetic
 * transmit aperture imaging, STAI, and plane-wave imaging, PWI; envelope
 * detection through a Hilbert transform computed with the FFT; dynamic
 * adjustment) and Sec. II-A the metadata they consume (speed of sound,
 * aperture, sampling frequency).  Sec. III fixes the RF layout
 * [acquisitions, channels, samples].  The paper prints no formulas; the
 * definitions each call implements are stated at the call.
 *
 * Conventions shared by every call
 *  - Geometry: linear array on z = 0, element e at x_e = (e - (E-1)/2) pitch.
 *    Pixel (iz, ix) at x = x_min + ix (x_max - x_min)/(nx - 1),
 *    z = z_min + iz (z_max - z_min)/(nz - 1) (an axis of 1 pixel sits at its
 *    minimum).  Physical quantities are SI (m, s, Hz, m/s) in double; the
 *    library converts them to sample units once, on the host, and the
 *    kernels work in FP32.
 *  - Layouts: RF [batch][n_tx or n_angles][n_rx][n_samples], samples fastest.
 *    Images [batch][nz][nx], x fastest.  All device arrays are dense.
 *  - Ownership: the caller allocates and owns every device buffer, including
 *    the DAS workspace.  The library never allocates, never frees and never
 *    synchronises the stream (wf_workspace_check excepted); host arrays
 *    passed in (transmit lists, angles, start times) are read before the call
 *    returns and may be reused at once.
 *  - Errors: arguments are validated on the host before any launch; a failed
 *    check returns a status and launches nothing.  Launch failures return
 *    WF_ERR_CUDA.  Faults inside kernels surface at the caller's next
 *    synchronisation.  No C++ exception crosses this boundary.
 *  - All work is enqueued on `stream` (0 = the legacy default stream).
 */
#ifndef WF_H_
#define WF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* wf_stream; /* same object as cudaStream_t */

typedef enum {
    WF_OK = 0,
    WF_ERR_INVALID_ARG = 1, /* bad pointer, size, geometry or enum value */
    WF_ERR_UNSUPPORTED = 2, /* valid but outside what the kernels handle (see limits) */
    WF_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
    WF_ERR_WORKSPACE = 4,   /* workspace NULL or smaller than wf_das_workspace_bytes() */
    WF_ERR_INTERNAL = 5     /* a kernel recorded an internal inconsistency */
} wf_status;

typedef enum { WF_F32 = 0, WF_F16 = 1, WF_I16 = 2 } wf_dtype;

/* Apodization window over the dynamic receive aperture (see wf_das_stai). */
typedef enum { WF_APOD_HANN = 0, WF_APOD_RECT = 1, WF_APOD_NONE = 2 } wf_apod;

/* Probe and medium: Sec. II-A's metadata (aperture, sampling frequency,
 * speed of sound) plus the receive f-number and window. */
typedef struct {
    int32_t n_elements;        /* E >= 1, <= WF_MAX_ELEMENTS */
    double pitch;              /* element spacing, m, > 0 */
    double fs;                 /* sampling frequency, Hz, > 0 */
    double c;                  /* speed of sound, m/s, > 0 */
    double f_number;           /* F > 0 (ignored for WF_APOD_NONE) */
    int32_t apod;              /* wf_apod */
    const float* elem_weight;  /* device [E] per-element weights g_e, or NULL (all 1) */
} wf_probe;

/* Pixel grid: pixel centres, bounds inclusive, x_max >= x_min, z_max >= z_min >= 0. */
typedef struct {
    int32_t nz, nx;            /* >= 1 each */
    double x_min, x_max, z_min, z_max; /* m */
} wf_grid;

#define WF_MAX_ELEMENTS 1024
#define WF_MAX_TX 256          /* transmits (STAI) or angles (PWI) per frame */
#define WF_MAX_SAMPLES (1 << 20)
#define WF_MAX_TAPS 255        /* FIR taps (odd count) */

/*
 * Bytes of device workspace wf_das_stai / wf_das_pwi need for this probe,
 * grid, batch and transmit (or angle) count.  The workspace holds the
 * per-split partial images that the split reduction sums in a fixed order
 * (the result is deterministic), plus a small status block.  Returns 0 if
 * the arguments are invalid.
 */
size_t wf_das_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                              int32_t n_tx_or_angles);

/*
 * STAI delay-and-sum (Sec. II-B: the DAS beamformer for synthetic transmit
 * aperture imaging; the beamforming block of Fig. 2).  For every pixel p:
 *
 *   b(p) = sum_t w(p, e_t) sum_r w(p, r) lerp(rf[t][r], s(p, t, r))
 *   s(p, t, r) = (|p - x_{e_t}| + |p - x_r|) fs / c - t_start fs      (samples)
 *
 * with e_t = tx_elem[t] the element that fired transmit t (single-element,
 * unfocused transmits), lerp the linear interpolation of a trace at
 * fractional sample s (i = floor(s), f = s - i, value (1-f) x[i] + f x[i+1]
 * when 0 <= i and i + 1 <= n_samples - 1, otherwise 0), and w the
 * apodization: a = z / (2F), u = (x_e - x) / a, Hann 0.5 (1 + cos(pi u)) or
 * rect 1 for |u| < 1, else 0 (no aperture for z <= 0), none = 1; times g_e.
 * Terms with zero weight are not part of the sum.  Accumulation is FP32.
 *
 *  probe, grid  host structs (read during the call)
 *  batch        frames >= 1; frame b reads rf + b * n_tx * n_rx * n_samples
 *  n_tx         transmits per frame, 1..WF_MAX_TX
 *  tx_elem      host [n_tx] element index of each transmit, or NULL = 0..n_tx-1
 *  n_rx         receive channels, must equal probe->n_elements
 *  n_samples    samples per trace, 1..WF_MAX_SAMPLES
 *  t_start      time of sample 0 after the transmit, s
 *  dtype        storage type of rf; WF_I16 values are multiplied by rf_scale
 *  rf           device [batch][n_tx][n_rx][n_samples], 16-byte aligned
 *  rf_scale     dequantisation scale for WF_I16 (ignored otherwise)
 *  out          device float [batch][nz][nx]
 *  ws, ws_bytes device workspace of at least wf_das_workspace_bytes() bytes
 *  stream       CUDA stream the kernels are enqueued on
 */
wf_status wf_das_stai(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                      int32_t n_tx, const int32_t* tx_elem, int32_t n_rx, int32_t n_samples,
                      double t_start, wf_dtype dtype, const void* rf, float rf_scale,
                      float* out, void* ws, size_t ws_bytes, wf_stream stream);

/*
 * PWI delay-and-sum with coherent compounding over steering angles (Sec. II-B
 * names plane-wave imaging).  For every pixel p = (x, z):
 *
 *   b(p) = sum_k sum_r w(p, r) lerp(rf[k][r], s(p, k, r))
 *   s(p, k, r) = (x sin th_k + z cos th_k + |p - x_r|) fs / c - t0_k fs
 *
 * The plane wave of angle th_k passes (0, 0) at time 0; t0_k is the time of
 * sample 0.  Receive apodization w as for STAI; no transmit weighting.
 *
 *  n_angles     angles per frame, 1..WF_MAX_TX
 *  angles_rad   host [n_angles] steering angles, radians
 *  t_start      host [n_angles] time of sample 0 per angle (s), or NULL = 0
 *  other arguments as wf_das_stai; rf is [batch][n_angles][n_rx][n_samples]
 */
wf_status wf_das_pwi(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                     int32_t n_angles, const double* angles_rad, const double* t_start,
                     int32_t n_rx, int32_t n_samples, wf_dtype dtype, const void* rf,
                     float rf_scale, float* out, void* ws, size_t ws_bytes, wf_stream stream);

/*
 * Delays in samples, s(p, t, r) above, exactly as the tiled DAS kernel forms
 * them (same device code): the integer start of the staging window plus the
 * FP32 window-relative delay, returned as the two parts (no FP64 on the GPU:
 * the caller adds them in double).  This is the check that the FP32 geometry
 * path stays within its delay-error budget.  Triples the DAS kernels never
 * evaluate (receive element outside the pixel tile's aperture range, STAI
 * transmit element outside it) have out_rel = NaN.
 *
 *  mode         0 = STAI (uses tx_elem, t_start[0]), 1 = PWI (angles_rad, t_start[k])
 *  n_tx         transmits or angles; tx_elem/angles_rad/t_start as above (host)
 *  n_pix, pix   device int32 [n_pix] linear pixel indices iz * nx + ix
 *  out_lo       device int32 [n_pix][n_tx][n_elements] window start (samples)
 *  out_rel      device float [n_pix][n_tx][n_elements] delay relative to out_lo
 */
wf_status wf_das_delays(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                        int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                        const double* t_start, int32_t n_pix, const int32_t* pix, int32_t* out_lo,
                        float* out_rel, wf_stream stream);

/*
 * RF transfer plan.  A box [t0, t1) x [r0, r1) x [s0, s1) of the
 * [n_tx][n_rx][n_samples] RF array of one frame.
 */
typedef struct {
    int32_t t0, t1, r0, r1, s0, s1;
} wf_rf_box;

/*
 * Boxes that together hold every sample wf_das_stai (mode 0) / wf_das_pwi
 * (mode 1) can read for these arguments: the staging windows of the tiled
 * kernels (Sec. II-B's per-element delays bounded over each pixel tile, every
 * tile configuration and pairing a call may select, with slack for the FP32
 * bounds) -- or whole traces where a grid sends the call to the per-pixel
 * path.  Samples outside the boxes never reach any result, so copying only the
 * boxes of a frame into the device RF buffer gives bit-identical images.  Host
 * computation only (no CUDA call); plan once per geometry.
 *
 *  mode, n_tx, tx_elem, angles_rad, t_start   as wf_das_delays (host arrays)
 *  n_rx, n_samples, dtype                     as wf_das_stai
 *  group        transmits per box (>= 1): one box per group of consecutive
 *               transmits, over the group's receive and sample hull
 *  boxes        host array of max_boxes entries, or NULL with max_boxes = 0
 *               to query the count
 *  n_boxes      receives the number of boxes; WF_ERR_INVALID_ARG (count still
 *               set) when it exceeds a non-zero max_boxes
 */
wf_status wf_das_rf_boxes(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                          int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                          const double* t_start, int32_t n_rx, int32_t n_samples,
                          wf_dtype dtype, int32_t group, wf_rf_box* boxes, int32_t max_boxes,
                          int32_t* n_boxes);

/*
 * Copy the boxes of one [n_tx][n_rx][n_samples] RF frame from src to dst
 * (same layout; one 3D copy per box, direction inferred from the pointers:
 * pinned host to device for the end-to-end path).  Asynchronous on stream.
 *
 *  elem_bytes   2 (int16 / float16) or 4 (float32)
 *  boxes        host array of n_boxes boxes inside the array's bounds
 */
wf_status wf_copy_rf_boxes(const void* src, void* dst, int32_t n_tx, int32_t n_rx,
                           int32_t n_samples, int32_t elem_bytes, const wf_rf_box* boxes,
                           int32_t n_boxes, wf_stream stream);

/*
 * Reverse-mode delay-and-sum (a differentiable beamformer: DAS inside a
 * learned pipeline, the use Sec. I and Sec. IV of the paper point to).  For a
 * cotangent y = grad_out of the beamformed image b of wf_das_stai (mode 0) or
 * wf_das_pwi (mode 1), the derivatives of L = sum_p y(p) b(p) with respect to
 *
 *   the RF:       dL/drf[t][r][i] = sum over terms of y W (1 - f) at i = floor(s)
 *                 and y W f at i + 1 (the transpose of the interpolation),
 *   the weights:  dL/dg_e (probe->elem_weight, both transmit and receive ends
 *                 for STAI), summed over the batch,
 *   sound speed:  dL/dc in 1/(m/s), through ds/dc = -(s + t_start fs) / c; the
 *                 apodization windows depend on geometry only,
 *
 * W the term's weight (w_t w_r for STAI, w_r for PWI), same terms, delays and
 * interpolation as the forward call.  Float32 RF only.  Accumulation uses
 * float atomics, so the last bits of a result depend on scheduling.
 *
 *  mode, n_tx, tx_elem, angles_rad, t_start   as wf_das_delays (host arrays)
 *  batch, n_rx, n_samples                     as wf_das_stai
 *  rf           device float [batch][n_tx][n_rx][n_samples], 16-byte aligned
 *  grad_out     device float [batch][nz][nx]
 *  grad_rf      device float, rf's shape, or NULL (not computed); overwritten
 *  grad_weight  device float [n_elements] or NULL; overwritten
 *  grad_c       device float [1] or NULL; overwritten
 *  stream       CUDA stream; no workspace is needed
 */
wf_status wf_das_backward(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                          int32_t batch, int32_t n_tx, const int32_t* tx_elem,
                          const double* angles_rad, const double* t_start, int32_t n_rx,
                          int32_t n_samples, const float* rf, const float* grad_out,
                          float* grad_rf, float* grad_weight, float* grad_c, wf_stream stream);

/*
 * Envelope detection (Fig. 2: analytic signal, then absolute value; Sec.
 * II-B: Hilbert transform through the FFT).  For every column x of every
 * frame, with N = nz:
 *
 *   Z = IDFT_N(H . DFT_N(b[:, x])),  H[0] = H[N/2] = 1, H[1..N/2-1] = 2, else 0
 *   env[:, x] = |Z|
 *
 * (the discrete analytic signal).  nz must be a power of two in [2, 4096].
 * If frame_max is not NULL it receives, per frame, the largest non-NaN
 * envelope value (0 for an all-zero frame).  Columns are transformed in
 * pairs (x = 2m, 2m+1) through one complex FFT, so a NaN or Inf anywhere in a
 * column also reaches the envelope of its pair partner.
 *
 *  bf           device float [batch][nz][nx] (16-byte aligned)
 *  env          device float [batch][nz][nx]; may not alias bf
 *  frame_max    device float [batch] or NULL
 */
wf_status wf_envelope(const float* bf, int32_t batch, int32_t nz, int32_t nx, float* env,
                      float* frame_max, wf_stream stream);

/*
 * Envelope detection and dynamic adjustment in one pass (the last two blocks
 * of Fig. 2) when the caller supplies the per-frame reference: out_db is
 * wf_logclip(wf_envelope(bf), ref) bit for bit, without the envelope's round
 * trip through memory.  Without a reference the frame maximum is a whole-frame
 * dependency: use wf_envelope (with frame_max) and then wf_logclip.
 *
 *  bf           device float [batch][nz][nx]; nz a power of two in [2, 4096]
 *  ref          device float [batch] (required); a reference that is not
 *               positive maps its frame to db_min, as in wf_logclip
 *  env          device float [batch][nz][nx] or NULL (not written); may not
 *               alias bf or out_db
 *  out_db       device float [batch][nz][nx]; may not alias bf
 *  frame_max    device float [batch] or NULL: the frames' largest non-NaN
 *               envelope values, as wf_envelope's
 * db_min <= db_max.  WF_ERR_INVALID_ARG for a NULL ref / out_db or the
 * argument errors of wf_envelope.
 */
wf_status wf_envelope_logclip(const float* bf, int32_t batch, int32_t nz, int32_t nx,
                              const float* ref, float db_min, float db_max, float* env,
                              float* out_db, float* frame_max, wf_stream stream);

/*
 * Dynamic adjustment (the last block of Fig. 2; Sec. III clips the
 * dynamic range):
 *
 *   out = clamp(20 log10(max(env, 1e-30 ref) / ref), db_min, db_max)
 *
 * with ref = ref[b] per frame, or, when ref is NULL, the frame's largest
 * non-NaN envelope value.  A frame whose ref is not positive maps to
 * db_min; NaN envelope values stay NaN.  db_min <= db_max.
 *
 *  env          device float [batch][nz][nx]
 *  ref          device float [batch] or NULL
 *  out_db       device float [batch][nz][nx]; may alias env
 */
wf_status wf_logclip(const float* env, int32_t batch, int32_t nz, int32_t nx, const float* ref,
                     float db_min, float db_max, float* out_db, wf_stream stream);

/*
 * Reverse mode of wf_envelope (the differentiable B-mode path).  For a
 * cotangent grad_env of env = |Z|, Z = A b with A = IDFT . diag(H) . DFT,
 * the cotangent of b is Re(A^H (grad_env Z / |Z|)) (0 where |Z| = 0); A is
 * Hermitian and Re(A r) = r for real r, so this equals
 * Re(g) - Hilbert(Im g) with g = grad_env Z / |Z|, computed per column pair
 * with two paired Hilbert transforms (Z is rebuilt from bf, not stored).
 *
 *  bf           device float [batch][nz][nx], the envelope's input
 *  grad_env     device float [batch][nz][nx]
 *  grad_bf      device float [batch][nz][nx]; may alias grad_env
 */
wf_status wf_envelope_backward(const float* bf, int32_t batch, int32_t nz, int32_t nx,
                               const float* grad_env, float* grad_bf, wf_stream stream);

/*
 * Reverse mode of wf_logclip.  Where the output is strictly inside (db_min,
 * db_max) and env > 1e-30 ref, d out/d env = 20 / (ln 10 env) and
 * d out/d ref = -20 / (ln 10 ref); clipped, floored and NaN pixels pass 0.
 * When ref is NULL (the forward used the frame maximum) or ref_is_frame_max is
 * non-zero (the caller's ref is that maximum, e.g. wf_envelope's frame_max),
 * the reference's cotangent is added to the first pixel (lowest index) whose
 * envelope equals ref; otherwise ref is a constant.
 *
 *  env, ref, db_min, db_max   as the forward call
 *  grad_db      device float [batch][nz][nx]
 *  grad_env     device float [batch][nz][nx]; may alias grad_db, not env
 */
wf_status wf_logclip_backward(const float* env, int32_t batch, int32_t nz, int32_t nx,
                              const float* ref, int32_t ref_is_frame_max, float db_min,
                              float db_max, const float* grad_db, float* grad_env,
                              wf_stream stream);

/*
 * Pre-processing (Sec. II-B lists a FIR filter among the signal processing operators).
 *
 * wf_fir: every trace (n_samples contiguous values) is filtered by the
 * odd-length FIR h (centre tap at lag 0, zero-phase for symmetric taps):
 *   out[n] = sum_{k<L} h[k] x[n + (L-1)/2 - k],  x = 0 outside [0, n_samples)
 * in FP32; int16 values are multiplied by rf_scale first.
 *
 *  rf           device [n_traces][n_samples] of dtype (4-byte aligned)
 *  taps         host float [n_taps], n_taps odd, 1..WF_MAX_TAPS
 *  out          device float [n_traces][n_samples]; may not alias rf
 */
wf_status wf_fir(const void* rf, wf_dtype dtype, float rf_scale, int64_t n_traces,
                 int32_t n_samples, const float* taps, int32_t n_taps, float* out,
                 wf_stream stream);

/*
 * wf_iq_demod: complex baseband of every trace: mix down by f0 with the
 * absolute sample phase, low-pass with the FIR h (alignment as wf_fir) and
 * keep every decim-th sample:
 *   iq[m] = sum_{k<L} h[k] x[i] exp(-2 pi i f0 i / fs),  i = m decim + (L-1)/2 - k
 * n_out = ceil(n_samples / decim) complex values per trace, stored as
 * (re, im) float pairs.  decim 1..16; f0 finite, fs > 0 (Hz).
 */
wf_status wf_iq_demod(const void* rf, wf_dtype dtype, float rf_scale, int64_t n_traces,
                      int32_t n_samples, double f0, double fs, const float* taps,
                      int32_t n_taps, int32_t decim, float* out_iq, wf_stream stream);

/*
 * Host utility: windowed-sinc band-pass taps (Hamming window) for wf_fir,
 * pass band [f_lo, f_hi] Hz at sampling rate fs (f_lo = 0: low-pass).
 * taps_out: host float [n_taps], n_taps odd, 1..WF_MAX_TAPS.
 */
wf_status wf_fir_bandpass(double f_lo, double f_hi, double fs, int32_t n_taps, float* taps_out);

/*
 * Delay-and-sum of complex baseband (IQ) traces: beamforming after
 * wf_iq_demod, the pre-processing variant of Sec. II-B's operators (FIR
 * filtering before the beamformer).  iq holds the demodulator's output with
 * decimation D: baseband sample m of a trace is the complex value at RF sample
 * index m D.  For every pixel p:
 *
 *   B(p) = sum_t w_t sum_r w_r lerp(iq[t][r], s / D) exp(2 pi i f0 s / fs)
 *
 * with s(p, t, r) the delay in RF samples of wf_das_stai (STAI, w_t as there)
 * or wf_das_pwi (PWI, w_t = 1), the same apodization, and lerp the linear
 * interpolation of I and Q with both recorded neighbours required (0 <=
 * floor(s / D) and floor(s / D) + 1 <= m_samples - 1, else the term is 0).
 * The phase undoes the demodulator's mixing at the interpolated sample, so for
 * taps of unit DC gain |B| is about half the envelope of the RF-domain image
 * (wf_iq_envelope takes |B|).  Accumulation in FP32; the per-stage phase
 * reduction in double-float, so no FP64 runs on the GPU.
 *
 *  n_rx         must equal probe->n_elements
 *  m_samples    baseband samples per trace, 2..WF_MAX_SAMPLES
 *  decim        D, 1..64 (wf_iq_demod's decimation)
 *  f0           mixing frequency of wf_iq_demod, Hz (finite)
 *  t_start      STAI: time of RF sample 0 (s); PWI: host [n_angles] or NULL = 0
 *  iq           device float [batch][n_tx][n_rx][m_samples][2] (re, im), 8-byte aligned
 *  out          device float [batch][nz][nx][2], the complex image B
 *  ws, ws_bytes device workspace of at least wf_das_iq_workspace_bytes() bytes
 * Grids so coarse that a pixel tile's staging window exceeds the tiled
 * kernel's limit return WF_ERR_UNSUPPORTED (there is no per-pixel path).
 */
size_t wf_das_iq_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                 int32_t batch, int32_t n_tx, int32_t m_samples, int32_t decim);
wf_status wf_das_stai_iq(const wf_probe* probe, const wf_grid* grid, int32_t batch, int32_t n_tx,
                         const int32_t* tx_elem, int32_t n_rx, int32_t m_samples, int32_t decim,
                         double f0, double t_start, const float* iq, float* out, void* ws,
                         size_t ws_bytes, wf_stream stream);
wf_status wf_das_pwi_iq(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                        int32_t n_angles, const double* angles_rad, const double* t_start,
                        int32_t n_rx, int32_t m_samples, int32_t decim, double f0, const float* iq,
                        float* out, void* ws, size_t ws_bytes, wf_stream stream);

/*
 * Envelope of an IQ-beamformed image: env = |B| for every pixel of the complex
 * image img [batch][nz][nx][2] (8-byte aligned), and, if frame_max is not
 * NULL, each frame's largest non-NaN value (device float [batch]), ready for
 * wf_logclip.  env is device float [batch][nz][nx].
 */
wf_status wf_iq_envelope(const float* img, int32_t batch, int32_t nz, int32_t nx, float* env,
                         float* frame_max, wf_stream stream);

/*
 * STAI delay-and-sum exactly as wf_das_stai, without a caller workspace.
 * (No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory, such as a real-time acquisition loop whose
 * device memory is fixed when it starts, or a plain C host program that links
 * only this library and has no device allocator of its own.)
 *
 * The split partials go to a fixed scratch array of WF_FIXED_SCRATCH_BYTES
 * that the library keeps in device memory; every GPU that loads the library
 * holds it until the process exits.  The call allocates and frees nothing.
 *  - Calls whose workspace need (wf_das_workspace_bytes) exceeds
 *    WF_FIXED_SCRATCH_BYTES return WF_ERR_WORKSPACE and launch nothing.
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents: calls that overlap on the GPU (different streams, or host
 *    threads without ordering between them) race and may return wrong images.
 *    Order such calls on one stream.
 *  - Kernel status flags (a bounded copy wait that ran out, an over-long
 *    staging window) land in the array's status block, which the caller cannot
 *    address: read them with wf_fixed_scratch_check.
 * Arguments, layouts and the rest of the error behaviour are those of
 * wf_das_stai, with one ordering difference: the checks that need no pointer
 * (sizes, counts, values) come first and return WF_ERR_INVALID_ARG as there,
 * then the size refusal (WF_ERR_WORKSPACE), then the pointer checks.
 */
#define WF_FIXED_SCRATCH_BYTES (32u << 20)
wf_status wf_das_stai_fixed_scratch(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                    int32_t n_tx, const int32_t* tx_elem, int32_t n_rx,
                                    int32_t n_samples, double t_start, wf_dtype dtype,
                                    const void* rf, float rf_scale, float* out, wf_stream stream);

/* Size in bytes of the fixed scratch array behind wf_das_stai_fixed_scratch. */
size_t wf_fixed_scratch_bytes(void);

/*
 * The wf_workspace_check of the fixed scratch array (no counterpart in the
 * paper): synchronises `stream`, reports WF_ERR_INTERNAL if a kernel of
 * wf_das_stai_fixed_scratch recorded an internal inconsistency in the array's
 * status block since that call began, WF_OK otherwise, and then clears the
 * status block (a blocking memset on the current device).  Blocks the host.
 */
wf_status wf_fixed_scratch_check(wf_stream stream);

/*
 * Plans and tuning.  wf_das_stai / wf_das_pwi plan a call (tile configuration,
 * staging, workspace layout, the CTA schedule over the pixel tiles) from its
 * probe, grid, scan, batch and RF shape and type, and keep the plan with the
 * packed kernel arguments in a small host-side cache (64 most recently used
 * keys), so a repeated call with the same geometry only sets its pointers and
 * launches.  Element weights are device data, read at run time, and not part
 * of a plan.  The optional tuning switches (environment variables
 * WF_DAS_NO_SYM, WF_DAS_NO_TMA, WF_DAS_NO_TMAP, WF_DAS_TILE, WF_DAS_GROUPS,
 * WF_DAS_BUDGET, WF_DAS_RING, WF_CHECK_BOUNDS) are read on the first DAS call;
 * wf_das_reload_tuning re-reads them and drops every cached plan.  Host only;
 * safe to call from any thread between calls.
 */
wf_status wf_das_reload_tuning(void);

/* What a DAS call with these arguments runs (diagnostics; host only). */
typedef struct {
    int32_t tiled;            /* 1: tiled gather kernels; 0: the per-pixel path */
    int32_t tile_cols;        /* pixel tile of a CTA (columns x rows) */
    int32_t tile_rows;
    int32_t window;           /* staged samples per trace (shared-memory stride) */
    int32_t ring;             /* bulk-copy ring depth (0: register-staged or per-pixel) */
    int32_t reciprocal;       /* STAI: reciprocal (t, r) / (r, t) pairing in use */
    int32_t ctas_per_frame;   /* tiled: CTAs the schedule launches for the whole batch */
    int32_t smem_bytes;       /* tiled forward: dynamic shared memory per CTA */
    int64_t workspace_bytes;  /* forward: workspace this call needs */
} wf_das_plan_info;

/*
 * Plan of wf_das_stai (mode 0) / wf_das_pwi (mode 1) -- reverse = 0 -- or of
 * wf_das_backward -- reverse = 1 -- for these arguments (as those calls;
 * t_start NULL means 0), written to *info.  The forward plan is the cached one
 * the call itself uses.
 */
wf_status wf_das_plan(const wf_probe* probe, const wf_grid* grid, int32_t mode, int32_t reverse,
                      int32_t batch, int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                      const double* t_start, int32_t n_samples, wf_dtype dtype,
                      wf_das_plan_info* info);

/*
 * Synchronises `stream` and reports whether a DAS kernel that used `ws`
 * recorded an internal inconsistency (WF_ERR_INTERNAL) since the workspace
 * was last handed to wf_das_stai / wf_das_pwi.  Debug aid; the only call that
 * blocks the host.
 */
wf_status wf_workspace_check(const void* ws, size_t ws_bytes, wf_stream stream);

/*
 * A CUDA stream of the caller's own (non-blocking with respect to the legacy
 * default stream) on the calling thread's current device, and its release.
 * The serving runtime gives every slot one, so that no other work -- a
 * stream pool handing the same stream to another request, or another
 * thread -- lands on a stream while a graph is being captured on it.
 * wf_stream_destroy returns once the stream's pending work is done; the
 * stream must not be used afterwards, by the caller or by anything that
 * remembers it (a pinned-memory allocator that records events on the streams
 * a buffer was copied on, for instance), so long-lived runtimes keep their
 * streams for reuse instead.  WF_ERR_INVALID_ARG for a NULL out / stream,
 * WF_ERR_CUDA if the runtime refuses.
 */
wf_status wf_stream_create(wf_stream* out);
wf_status wf_stream_destroy(wf_stream stream);

/* Static, human-readable name of a status code. */
const char* wf_status_string(wf_status status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int32_t wf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WF_H_ */
