/*
 * FP64 reference ("oracle") of the B-mode reconstruction path: delay-and-sum
 * beamforming (STAI and PWI), analytic signal, magnitude, log compression
 * with dynamic-range clipping.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark have an independent, obviously correct
 * answer to compare the CUDA path against.  It shares no code, header,
 * table or constant with the CUDA sources.
 *
 * Everything is plain single-threaded C in double precision, written as the
 * direct definition of each step, in the order the paper's pipeline
 * (Fig. 2) applies them: Beamforming -> Analytic Signal -> Absolute Value ->
 * Dynamic Adjustment.  The paper names the steps (Sec. II-B: DAS beamformer
 * with STAI and PWI; envelope detection; dynamic adjustment; Hilbert
 * transform built on the FFT) but prints none of their formulas, so the
 * formulas below are the standard textbook definitions; each reading the
 * paper leaves open is stated at the function that makes it.
 *
 * Geometry: a linear array on the line z = 0 with element e at
 * x_e = (e - (E-1)/2) * pitch; pixel (iz, ix) sits at
 * x = x_min + ix (x_max - x_min)/(nx - 1), z = z_min + iz (z_max - z_min)/(nz - 1)
 * (a grid of 1 along an axis sits at the lower bound).  Images are
 * [nz][nx], x fastest.  RF is [n_tx][n_rx][n_samples], samples fastest, the
 * paper's [acquisitions, channels, samples] layout (Sec. III).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define OR_HANN 0
#define OR_RECT 1
#define OR_NONE 2

typedef struct {
    int32_t n_elements;
    double pitch;          /* m */
    double fs;             /* Hz */
    double c;              /* m/s */
    double f_number;
    int32_t apod;          /* OR_HANN / OR_RECT / OR_NONE */
    const double* elem_weight; /* [n_elements] or NULL (all ones) */
} or_probe;

typedef struct {
    int32_t nz, nx;
    double x_min, x_max, z_min, z_max; /* m, pixel centres, inclusive */
} or_grid;

/* Position of element e on the array (x, at z = 0). */
double or_element_x(const or_probe* p, int32_t e)
{
    return ((double)e - 0.5 * (double)(p->n_elements - 1)) * p->pitch;
}

/* Lateral / axial position of a pixel index. */
double or_pixel_x(const or_grid* g, int32_t ix)
{
    if (g->nx <= 1) return g->x_min;
    return g->x_min + (double)ix * (g->x_max - g->x_min) / (double)(g->nx - 1);
}

double or_pixel_z(const or_grid* g, int32_t iz)
{
    if (g->nz <= 1) return g->z_min;
    return g->z_min + (double)iz * (g->z_max - g->z_min) / (double)(g->nz - 1);
}

/*
 * Apodization weight of element e for the pixel (x, z) (Sec. II-B DAS).
 * Reading: dynamic receive aperture of half-width a = z / (2F), normalised
 * offset u = (x_e - x) / a; Hann: 0.5 (1 + cos(pi u)) for |u| < 1, else 0;
 * rect: 1 for |u| < 1, else 0; none: 1 everywhere.  A pixel with z <= 0 has
 * no aperture (weight 0) unless the apodization is "none".  The optional
 * per-element weight g_e multiplies the window.
 */
double or_apod(const or_probe* p, double x, double z, int32_t e)
{
    double g = p->elem_weight ? p->elem_weight[e] : 1.0;
    if (p->apod == OR_NONE) return g;
    double a = z / (2.0 * p->f_number);
    if (!(a > 0.0)) return 0.0;
    double u = (or_element_x(p, e) - x) / a;
    if (!(fabs(u) < 1.0)) return 0.0;
    if (p->apod == OR_RECT) return g;
    return g * 0.5 * (1.0 + cos(M_PI * u));
}

/* One-way distance from element e to the pixel (x, z), m. */
static double or_dist(const or_probe* p, double x, double z, int32_t e)
{
    double dx = x - or_element_x(p, e);
    return sqrt(dx * dx + z * z);
}

/*
 * STAI delay in samples (Sec. II-B, synthetic transmit aperture): element
 * et fires at t = 0, element er records; sample 0 is taken at t_start.
 * s = (|p - e_t| + |p - e_r|) fs / c - t_start fs.
 */
double or_delay_stai(const or_probe* p, double x, double z, int32_t et, int32_t er,
                     double t_start)
{
    return (or_dist(p, x, z, et) + or_dist(p, x, z, er)) * p->fs / p->c - t_start * p->fs;
}

/*
 * PWI delay in samples (Sec. II-B, plane-wave imaging): the plane wave of
 * angle theta passes the origin at t = 0 and reaches (x, z) after
 * (x sin theta + z cos theta) / c; the echo returns to element er.
 * s = (x sin theta + z cos theta + |p - e_r|) fs / c - t_start fs.
 */
double or_delay_pwi(const or_probe* p, double x, double z, double theta, int32_t er,
                    double t_start)
{
    return (x * sin(theta) + z * cos(theta) + or_dist(p, x, z, er)) * p->fs / p->c
           - t_start * p->fs;
}

/*
 * Linear interpolation of one RF trace at fractional sample s.
 * Reading: i = floor(s), f = s - i; the value is (1-f) tr[i] + f tr[i+1]
 * when 0 <= i and i + 1 <= ns - 1, and 0 otherwise (no echo recorded).
 */
double or_lerp(const double* tr, int32_t ns, double s)
{
    double fi = floor(s);
    if (!(fi >= 0.0) || !(fi + 1.0 <= (double)(ns - 1))) return 0.0;
    int64_t i = (int64_t)fi;
    double f = s - fi;
    return (1.0 - f) * tr[i] + f * tr[i + 1];
}

/*
 * STAI delay-and-sum (Sec. II-B; the beamforming block of Fig. 2):
 *   b(p) = sum_t w(p, e_t) sum_r w(p, r) lerp(rf[t][r], s_stai(p, e_t, r)).
 * Terms whose apodization weight is zero are outside the aperture and are not
 * part of the sum.  Writes rows [row_begin, row_end) of out[nz][nx].
 */
int or_das_stai(const or_probe* p, const or_grid* g, int32_t n_tx, const int32_t* tx_elem,
                int32_t n_rx, int32_t ns, double t_start, const double* rf,
                int32_t row_begin, int32_t row_end, double* out)
{
    if (n_rx != p->n_elements) return 1;
    for (int32_t iz = row_begin; iz < row_end; ++iz) {
        double z = or_pixel_z(g, iz);
        for (int32_t ix = 0; ix < g->nx; ++ix) {
            double x = or_pixel_x(g, ix);
            double acc = 0.0;
            for (int32_t t = 0; t < n_tx; ++t) {
                int32_t et = tx_elem ? tx_elem[t] : t;
                double wt = or_apod(p, x, z, et);
                if (wt == 0.0) continue;
                double inner = 0.0;
                for (int32_t r = 0; r < n_rx; ++r) {
                    double wr = or_apod(p, x, z, r);
                    if (wr == 0.0) continue;
                    double s = or_delay_stai(p, x, z, et, r, t_start);
                    const double* tr = rf + ((size_t)t * n_rx + r) * (size_t)ns;
                    inner += wr * or_lerp(tr, ns, s);
                }
                acc += wt * inner;
            }
            out[(size_t)iz * g->nx + ix] = acc;
        }
    }
    return 0;
}

/*
 * PWI delay-and-sum with coherent compounding over angles (Sec. II-B):
 *   b(p) = sum_k sum_r w(p, r) lerp(rf[k][r], s_pwi(p, theta_k, r)).
 * Receive apodization only; every angle has transmit weight 1.
 */
int or_das_pwi(const or_probe* p, const or_grid* g, int32_t n_ang, const double* angles,
               const double* t_starts, int32_t n_rx, int32_t ns, const double* rf,
               int32_t row_begin, int32_t row_end, double* out)
{
    if (n_rx != p->n_elements) return 1;
    for (int32_t iz = row_begin; iz < row_end; ++iz) {
        double z = or_pixel_z(g, iz);
        for (int32_t ix = 0; ix < g->nx; ++ix) {
            double x = or_pixel_x(g, ix);
            double acc = 0.0;
            for (int32_t k = 0; k < n_ang; ++k) {
                double t0 = t_starts ? t_starts[k] : 0.0;
                for (int32_t r = 0; r < n_rx; ++r) {
                    double wr = or_apod(p, x, z, r);
                    if (wr == 0.0) continue;
                    double s = or_delay_pwi(p, x, z, angles[k], r, t0);
                    const double* tr = rf + ((size_t)k * n_rx + r) * (size_t)ns;
                    acc += wr * or_lerp(tr, ns, s);
                }
            }
            out[(size_t)iz * g->nx + ix] = acc;
        }
    }
    return 0;
}

/*
 * Aperture window of element e for the pixel (x, z) without the element
 * weight: or_apod / g_e, defined also where g_e = 0 (the derivative of the
 * beamformed value with respect to g_e needs it there).
 */
double or_window(const or_probe* p, double x, double z, int32_t e)
{
    if (p->apod == OR_NONE) return 1.0;
    double half_width = 0.5 * z / p->f_number;
    if (!(half_width > 0.0)) return 0.0;
    double u = (or_element_x(p, e) - x) / half_width;
    if (!(fabs(u) < 1.0)) return 0.0;
    if (p->apod == OR_RECT) return 1.0;
    return 0.5 + 0.5 * cos(M_PI * u);
}

/*
 * Reverse-mode derivatives of delay-and-sum, for a cotangent y[nz][nx] of the
 * beamformed image b (the differentiable beamformer that lets DAS sit inside a
 * learned pipeline, Sec. I and Sec. IV).  Plain definition, term by term: for
 * every (pixel p, transmit t, receive r) with both windows non-zero, the
 * weight W = w_t w_r (STAI; w = g_e window) or W = w_r (PWI), the delay s, its
 * floor i and fraction f, and when 0 <= i and i + 1 <= ns - 1:
 *   grad_rf[t][r][i] += y(p) W (1 - f),  grad_rf[t][r][i+1] += y(p) W f
 *       (the transpose of the linear interpolation);
 *   grad_g[e] += y(p) dW/dg_e lerp  (STAI: e_t and r; PWI: r);
 *   grad_c    += y(p) W (tr[i+1] - tr[i]) ds/dc,  ds/dc = -(s + t_start fs) / c
 *       (s + t_start fs is the path length in samples, proportional to 1/c;
 *        the slope is that of the segment s lies on; the windows do not
 *        depend on c).
 * mode 0 = STAI (tx_elem, t_start[0]), 1 = PWI (angles, t_start[k]).
 * Pixel rows [row_begin, row_end) only; every output accumulates (+=), so
 * callers zero them once and may split rows.  Any output may be NULL.
 */
int or_das_backward(const or_probe* p, const or_grid* g, int32_t mode, int32_t n_tx,
                    const int32_t* tx_elem, const double* angles, const double* t_start,
                    int32_t n_rx, int32_t ns, const double* rf, const double* y,
                    int32_t row_begin, int32_t row_end, double* grad_rf, double* grad_g,
                    double* grad_c)
{
    if (n_rx != p->n_elements) return 1;
    for (int32_t iz = row_begin; iz < row_end; ++iz) {
        double z = or_pixel_z(g, iz);
        for (int32_t ix = 0; ix < g->nx; ++ix) {
            double x = or_pixel_x(g, ix);
            double yp = y[(size_t)iz * g->nx + ix];
            for (int32_t t = 0; t < n_tx; ++t) {
                int32_t et = mode == 0 ? (tx_elem ? tx_elem[t] : t) : -1;
                double t0 = t_start ? t_start[mode == 0 ? 0 : t] : 0.0;
                double at = mode == 0 ? or_window(p, x, z, et) : 1.0;
                double gt = mode == 0 && p->elem_weight ? p->elem_weight[et] : 1.0;
                if (at == 0.0) continue;
                for (int32_t r = 0; r < n_rx; ++r) {
                    double ar = or_window(p, x, z, r);
                    if (ar == 0.0) continue;
                    double gr = p->elem_weight ? p->elem_weight[r] : 1.0;
                    double s = mode == 0 ? or_delay_stai(p, x, z, et, r, t0)
                                         : or_delay_pwi(p, x, z, angles[t], r, t0);
                    double fi = floor(s);
                    if (!(fi >= 0.0) || !(fi + 1.0 <= (double)(ns - 1))) continue;
                    int64_t i = (int64_t)fi;
                    double f = s - fi;
                    size_t base = ((size_t)t * n_rx + r) * (size_t)ns;
                    const double* tr = rf + base;
                    double v = or_lerp(tr, ns, s);
                    double W = gt * at * gr * ar;
                    if (grad_rf) {
                        grad_rf[base + i] += yp * W * (1.0 - f);
                        grad_rf[base + i + 1] += yp * W * f;
                    }
                    if (grad_g) {
                        if (mode == 0) grad_g[et] += yp * at * gr * ar * v;
                        grad_g[r] += yp * gt * at * ar * v;
                    }
                    if (grad_c) {
                        double dsdc = -(s + t0 * p->fs) / p->c;
                        *grad_c += yp * W * (tr[i + 1] - tr[i]) * dsdc;
                    }
                }
            }
        }
    }
    return 0;
}

/*
 * Direct O(N^2) discrete Fourier transform (textbook definition):
 *   forward  X[k] = sum_n x[n] exp(-2 pi i k n / N)
 *   inverse  x[n] = (1/N) sum_k X[k] exp(+2 pi i k n / N)
 * The phase index k n is reduced mod N in integers before the angle is
 * formed, so every twiddle is cos/sin of 2 pi m / N with m < N.
 */
void or_dft(const double* xr, const double* xi, int32_t n, int32_t inverse,
            double* yr, double* yi)
{
    double sgn = inverse ? 1.0 : -1.0;
    for (int32_t k = 0; k < n; ++k) {
        double ar = 0.0, ai = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            int64_t m = ((int64_t)k * j) % n;
            double ang = 2.0 * M_PI * (double)m / (double)n;
            double c = cos(ang), s = sgn * sin(ang);
            double vr = xr[j], vi = xi ? xi[j] : 0.0;
            ar += vr * c - vi * s;
            ai += vr * s + vi * c;
        }
        if (inverse) { ar /= n; ai /= n; }
        yr[k] = ar;
        yi[k] = ai;
    }
}

/*
 * Discrete analytic signal of a real sequence (the analytic-signal block of Fig. 2;
 * Sec. II-B: Hilbert transform built on the FFT).  Reading: the standard
 * one-sided-spectrum construction (Marple 1999): X = DFT(x); H[0] = 1,
 * H[k] = 2 for 0 < k < N/2, H[N/2] = 1 for even N (for odd N, H[k] = 2 for
 * 0 < k <= (N-1)/2), H[k] = 0 otherwise; z = IDFT(H X).
 */
void or_analytic(const double* x, int32_t n, double* zr, double* zi)
{
    double* xr = (double*)malloc(sizeof(double) * (size_t)n * 2);
    double* xi = xr + n;
    or_dft(x, NULL, n, 0, xr, xi);
    for (int32_t k = 0; k < n; ++k) {
        double h;
        if (k == 0) h = 1.0;
        else if (2 * k < n) h = 2.0;
        else if (2 * k == n) h = 1.0;
        else h = 0.0;
        xr[k] *= h;
        xi[k] *= h;
    }
    or_dft(xr, xi, n, 1, zr, zi);
    free(xr);
}

/*
 * Envelope = |analytic signal| along depth, per image column (Fig. 2
 * analytic-signal then absolute-value blocks).  bf and env are [nz][nx];
 * columns [col_begin, col_end) are written.
 */
void or_envelope(const double* bf, int32_t nz, int32_t nx, int32_t col_begin,
                 int32_t col_end, double* env)
{
    double* col = (double*)malloc(sizeof(double) * (size_t)nz * 3);
    double* zr = col + nz;
    double* zi = zr + nz;
    for (int32_t ix = col_begin; ix < col_end; ++ix) {
        for (int32_t iz = 0; iz < nz; ++iz) col[iz] = bf[(size_t)iz * nx + ix];
        or_analytic(col, nz, zr, zi);
        for (int32_t iz = 0; iz < nz; ++iz)
            env[(size_t)iz * nx + ix] = sqrt(zr[iz] * zr[iz] + zi[iz] * zi[iz]);
    }
    free(col);
}

/*
 * Frame maximum of an envelope image, NaN values ignored (the default
 * normalisation reference of the dynamic adjustment).  Returns 0 for an
 * empty or all-NaN frame.
 */
double or_frame_max(const double* env, int64_t n)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (env[i] == env[i] && env[i] > m) m = env[i];
    return m;
}

/*
 * Dynamic adjustment (the last block of Fig. 2; Sec. III clips the
 * dynamic range).  Reading: out = clamp(20 log10(max(env, 1e-30 ref) / ref),
 * lo, hi).  A frame whose reference is not positive maps every pixel to lo;
 * a NaN envelope value stays NaN.
 */
void or_logclip(const double* env, int64_t n, double ref, double lo, double hi, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = env[i];
        if (v != v) { out[i] = v; continue; }
        if (!(ref > 0.0)) { out[i] = lo; continue; }
        double e = v > 1e-30 * ref ? v : 1e-30 * ref;
        double db = 20.0 * log10(e / ref);
        out[i] = db < lo ? lo : (db > hi ? hi : db);
    }
}

/*
 * Reverse mode of the envelope (Fig. 2: analytic signal then absolute
 * Value").  Per column, z = A b with A = F^-1 diag(H) F (F the DFT matrix, H
 * the one-sided-spectrum mask above) and env = |z|.  For a cotangent g of env
 * the cotangent of z is g z / |z| (0 where |z| = 0), and since b is real the
 * cotangent of b is Re(A^H g_z) with A^H = F^H diag(H) F^-H, F^-H = F / N and
 * F^H = N F^-1: evaluated here literally as N IDFT(H (DFT(g_z) / N)).
 * Columns [col_begin, col_end) of g_bf[nz][nx] are written.
 */
void or_envelope_backward(const double* bf, int32_t nz, int32_t nx, const double* g_env,
                          int32_t col_begin, int32_t col_end, double* g_bf)
{
    double* buf = (double*)malloc(sizeof(double) * (size_t)nz * 7);
    double* col = buf;
    double* zr = col + nz;
    double* zi = zr + nz;
    double* gr = zi + nz;
    double* gi = gr + nz;
    double* yr = gi + nz;
    double* yi = yr + nz;
    for (int32_t ix = col_begin; ix < col_end; ++ix) {
        for (int32_t iz = 0; iz < nz; ++iz) col[iz] = bf[(size_t)iz * nx + ix];
        or_analytic(col, nz, zr, zi);
        for (int32_t iz = 0; iz < nz; ++iz) {
            double m = sqrt(zr[iz] * zr[iz] + zi[iz] * zi[iz]);
            double g = g_env[(size_t)iz * nx + ix];
            gr[iz] = m > 0.0 ? g * zr[iz] / m : 0.0;
            gi[iz] = m > 0.0 ? g * zi[iz] / m : 0.0;
        }
        or_dft(gr, gi, nz, 0, yr, yi);                  /* F g_z */
        for (int32_t k = 0; k < nz; ++k) {
            double h;
            if (k == 0) h = 1.0;
            else if (2 * k < nz) h = 2.0;
            else if (2 * k == nz) h = 1.0;
            else h = 0.0;
            yr[k] *= h / (double)nz;                    /* diag(H) F^-H g_z */
            yi[k] *= h / (double)nz;
        }
        or_dft(yr, yi, nz, 1, gr, gi);                  /* F^-1 (.) ; F^H = N F^-1 */
        for (int32_t iz = 0; iz < nz; ++iz) g_bf[(size_t)iz * nx + ix] = (double)nz * gr[iz];
    }
    free(buf);
}

/*
 * Reverse mode of the dynamic adjustment out = clamp(20 log10(max(env,
 * 1e-30 ref) / ref), lo, hi).  Where the value is strictly inside (lo, hi)
 * and env > 1e-30 ref, d out / d env = 20 / (ln 10 env) and d out / d ref =
 * -20 / (ln 10 ref); elsewhere (clipped, floored, NaN, ref <= 0) both are 0.
 * When ref_is_max, ref is the frame maximum of env and its cotangent is added
 * to the first pixel that attains it.  Writes g_env[n].
 */
void or_logclip_backward(const double* env, int64_t n, double ref, int32_t ref_is_max, double lo,
                         double hi, const double* g_db, double* g_env)
{
    double s_ref = 0.0;
    int64_t arg = -1;
    for (int64_t i = 0; i < n; ++i) {
        double v = env[i];
        g_env[i] = 0.0;
        if (arg < 0 && v == ref) arg = i;
        if (v != v || !(ref > 0.0) || !(v > 1e-30 * ref)) continue;
        double db = 20.0 * log10(v / ref);
        if (!(db > lo && db < hi)) continue;
        g_env[i] = g_db[i] * 20.0 / (log(10.0) * v);
        s_ref += g_db[i] * (-20.0 / (log(10.0) * ref));
    }
    if (ref_is_max && arg >= 0) g_env[arg] += s_ref;
}

/*
 * FIR filtering of one RF trace (pre-processing, Sec. II-B's signal processing
 * Operators": FIR filter).  Reading: a causal filter of odd length L with its
 * centre tap at lag 0, y[n] = sum_{k=0}^{L-1} h[k] x[n + (L-1)/2 - k], x = 0
 * outside [0, ns); for symmetric (linear-phase) taps this is zero-phase.
 */
void or_fir(const double* x, int32_t ns, const double* h, int32_t n_taps, double* y)
{
    int32_t c = (n_taps - 1) / 2;
    for (int32_t n = 0; n < ns; ++n) {
        double acc = 0.0;
        for (int32_t k = 0; k < n_taps; ++k) {
            int64_t i = (int64_t)n + c - k;
            if (i >= 0 && i < ns) acc += h[k] * x[i];
        }
        y[n] = acc;
    }
}

/*
 * IQ demodulation of one RF trace: mix down by the centre frequency f0,
 * low-pass with the FIR h (same alignment as or_fir), keep every D-th sample:
 *   iq[m] = sum_k h[k] x[i] exp(-2 pi i f0 i / fs),  i = m D + (L-1)/2 - k.
 * The mixing phase uses the absolute sample index, so sample m of the output is
 * the baseband value at time m D / fs.  Writes n_out = ceil(ns / D) complex
 * samples as (re, im) pairs.
 */
void or_iq_demod(const double* x, int32_t ns, double f0, double fs, const double* h,
                 int32_t n_taps, int32_t decim, double* iq)
{
    int32_t c = (n_taps - 1) / 2;
    int32_t n_out = (ns + decim - 1) / decim;
    for (int32_t m = 0; m < n_out; ++m) {
        double re = 0.0, im = 0.0;
        for (int32_t k = 0; k < n_taps; ++k) {
            int64_t i = (int64_t)m * decim + c - k;
            if (i < 0 || i >= ns) continue;
            double ph = 2.0 * M_PI * f0 * (double)i / fs;
            re += h[k] * x[i] * cos(ph);
            im -= h[k] * x[i] * sin(ph);
        }
        iq[2 * m] = re;
        iq[2 * m + 1] = im;
    }
}

/*
 * Delay-and-sum of complex baseband (IQ) traces, STAI (mode 0) or PWI (mode 1):
 * beamforming after IQ demodulation (pre-processing variant of Sec. II-B).
 * iq[t][r][m] = (re, im) holds the output of or_iq_demod with decimation D,
 * baseband sample m taken at RF sample index m D.  For every pixel and every
 * (t, r) with non-zero weights: the delay s in RF samples (or_delay_stai /
 * or_delay_pwi), its baseband position u = s / D, linear interpolation of I
 * and Q at u with both recorded neighbours required (0 <= floor(u) and
 * floor(u) + 1 <= M - 1, else the term is 0), and the remodulation phase
 * exp(+2 pi i f0 s / fs) that undoes the mixing at that sample:
 *   B(p) = sum_t w_t sum_r w_r lerp(iq[t][r], s / D) exp(2 pi i f0 s / fs)
 * (w_t = 1 for PWI; weights as or_das_stai / or_das_pwi).  Writes rows
 * [row_begin, row_end) of out[nz][nx][2].
 */
int or_das_iq(const or_probe* p, const or_grid* g, int32_t mode, int32_t n_tx,
              const int32_t* tx_elem, const double* angles, const double* t_start, int32_t n_rx,
              int32_t m_samples, int32_t decim, double f0, const double* iq, int32_t row_begin,
              int32_t row_end, double* out)
{
    if (n_rx != p->n_elements || decim < 1) return 1;
    for (int32_t iz = row_begin; iz < row_end; ++iz) {
        double z = or_pixel_z(g, iz);
        for (int32_t ix = 0; ix < g->nx; ++ix) {
            double x = or_pixel_x(g, ix);
            double acc_re = 0.0, acc_im = 0.0;
            for (int32_t t = 0; t < n_tx; ++t) {
                int32_t et = mode == 0 ? (tx_elem ? tx_elem[t] : t) : -1;
                double t0 = t_start ? t_start[mode == 0 ? 0 : t] : 0.0;
                double wt = mode == 0 ? or_apod(p, x, z, et) : 1.0;
                if (wt == 0.0) continue;
                double in_re = 0.0, in_im = 0.0;
                for (int32_t r = 0; r < n_rx; ++r) {
                    double wr = or_apod(p, x, z, r);
                    if (wr == 0.0) continue;
                    double s = mode == 0 ? or_delay_stai(p, x, z, et, r, t0)
                                         : or_delay_pwi(p, x, z, angles[t], r, t0);
                    double u = s / (double)decim;
                    double fu = floor(u);
                    if (!(fu >= 0.0) || !(fu + 1.0 <= (double)(m_samples - 1))) continue;
                    int64_t i = (int64_t)fu;
                    double f = u - fu;
                    const double* tr = iq + ((size_t)t * n_rx + r) * (size_t)m_samples * 2;
                    double vr = (1.0 - f) * tr[2 * i] + f * tr[2 * i + 2];
                    double vi = (1.0 - f) * tr[2 * i + 1] + f * tr[2 * i + 3];
                    double ph = 2.0 * M_PI * f0 * s / p->fs;
                    double c = cos(ph), sn = sin(ph);
                    in_re += wr * (vr * c - vi * sn);
                    in_im += wr * (vr * sn + vi * c);
                }
                acc_re += wt * in_re;
                acc_im += wt * in_im;
            }
            out[2 * ((size_t)iz * g->nx + ix)] = acc_re;
            out[2 * ((size_t)iz * g->nx + ix) + 1] = acc_im;
        }
    }
    return 0;
}
