/*
 * oracle.c -- plain, slow, obviously-correct FP64 reference of the readout
 * signal-processing stage (polyphase filter bank and direct multi-tone
 * demodulation) of Minutolo et al., "A flexible GPU-accelerated
 * radio-frequency readout for superconducting detectors" (arXiv:1812.02200).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Single-threaded, FP64 throughout, no blocking, fusion or reordering beyond
 * what each definition states.  Every entry point returns 0 on success and a
 * negative number on invalid arguments.
 *
 * Sign and layout conventions (the paper fixes none of them; the readings are
 * listed in the design notes):
 *   - complex samples are interleaved (re, im) pairs;
 *   - the forward DFT uses exp(-2*pi*i*c*p/N), natural bin order, no 1/N;
 *   - frame k of a stream uses the W samples that end at sample (k+1)*hop - 1,
 *     samples before the stream start are zero;
 *   - an NCO word w is a uint64 phase increment in units of 2*pi/2^64 per
 *     sample, the mixer is exp(-i*phase).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_WIN_RECT = 0, ORC_WIN_HANN = 1, ORC_WIN_HAMMING = 2,
       ORC_WIN_BLACKMAN = 3, ORC_WIN_KAISER = 4 };

/* ------------------------------------------------------------------------ */
/* Windows and prototype filters                                             */
/* ------------------------------------------------------------------------ */

/* Modified Bessel function of the first kind, order 0, by its power series
 * I0(x) = sum_k ((x/2)^k / k!)^2, summed until the term no longer changes
 * the sum.  Needed by the Kaiser window (the configured PFB window). */
double orc_bessel_i0(double x)
{
    double sum = 1.0, term = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

/* Symmetric window of length m (denominator m-1), evaluated in FP64.
 * Sec. III.A: the paper's PFB prototype is a Hamming-windowed sinc; the
 * direct demodulator of Sec. III.B uses a square window (moving average).
 * Hann, Blackman and Kaiser are the other windows the workloads name. */
int orc_window(int kind, double beta, int64_t m, double* w)
{
    if (m <= 0 || !w) return -1;
    if (m == 1) { w[0] = 1.0; return 0; }
    const double den = (double)(m - 1);
    for (int64_t j = 0; j < m; ++j) {
        const double a = 2.0 * M_PI * (double)j / den;
        switch (kind) {
        case ORC_WIN_RECT:     w[j] = 1.0; break;
        case ORC_WIN_HANN:     w[j] = 0.5 - 0.5 * cos(a); break;
        case ORC_WIN_HAMMING:  w[j] = 0.54 - 0.46 * cos(a); break;
        case ORC_WIN_BLACKMAN: w[j] = 0.42 - 0.5 * cos(a) + 0.08 * cos(2.0 * a); break;
        case ORC_WIN_KAISER: {
            const double r = 2.0 * (double)j / den - 1.0;
            double s = 1.0 - r * r;
            if (s < 0.0) s = 0.0;
            w[j] = orc_bessel_i0(beta * sqrt(s)) / orc_bessel_i0(beta);
            break;
        }
        default: return -1;
        }
    }
    return 0;
}

static double orc_sinc(double u)
{
    if (u == 0.0) return 1.0;
    return sin(M_PI * u) / (M_PI * u);
}

/* Windowed-sinc low-pass of length m:
 *   h[j] = w[j] * sinc(2*fc*(j - (m-1)/2)),   normalised so sum_j h[j] = 1.
 * fc is the cut-off in cycles per sample; fc <= 0 drops the sinc factor
 * (a pure window; with the square window this is the paper's moving average
 * of Sec. III.B).  Sec. III.A: the PFB prototype is such a product with its
 * cut-off placed so adjacent bins cross over near -6 dB, i.e. fc = 1/(2N). */
int orc_lowpass(int kind, double beta, double fc, int64_t m, double* h)
{
    if (orc_window(kind, beta, m, h) != 0) return -1;
    const double c = 0.5 * (double)(m - 1);
    if (fc > 0.0)
        for (int64_t j = 0; j < m; ++j) h[j] *= orc_sinc(2.0 * fc * ((double)j - c));
    double s = 0.0;
    for (int64_t j = 0; j < m; ++j) s += h[j];
    if (s == 0.0) return -1;
    for (int64_t j = 0; j < m; ++j) h[j] /= s;
    return 0;
}

/* The PFB prototype of Sec. III.A for N channels and T taps per channel
 * (length M = N*T, cut-off 1/(2N) unless fc > 0 is given), in FP64 and also
 * rounded to FP32 (the workloads fix FP32 coefficients); h32 may be NULL. */
int orc_pfb_prototype(int32_t n_chan, int32_t taps, int kind, double beta, double fc,
                      double* h64, float* h32)
{
    if (n_chan <= 0 || taps <= 0) return -1;
    const int64_t m = (int64_t)n_chan * taps;
    if (fc <= 0.0) fc = 0.5 / (double)n_chan;
    if (orc_lowpass(kind, beta, fc, m, h64) != 0) return -1;
    if (h32) for (int64_t j = 0; j < m; ++j) h32[j] = (float)h64[j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Integer NCO words and tone bins                                           */
/* ------------------------------------------------------------------------ */

/* Frequency f (Hz) at sample rate fs (Hz) -> uint64 phase increment per sample
 * in units of 2*pi/2^64.  f/fs is wrapped into [-1/2, 1/2) first, then scaled
 * by 2^64 and rounded to the nearest integer (two's complement). */
uint64_t orc_freq_to_word(double f, double fs)
{
    double r = f / fs;
    r -= floor(r + 0.5);
    const double v = ldexp(r, 64);          /* exact scaling, |v| <= 2^63 */
    return (uint64_t)(int64_t)llround(v);
}

/* The PFB bin that holds an NCO word: round(word * N / 2^64) mod N with ties
 * rounded up, in exact integer arithmetic for any N >= 2:
 *   bin = floor((word * N + 2^63) / 2^64) mod N,
 * the 128-bit product formed with unsigned __int128. */
int32_t orc_word_to_bin(uint64_t word, int32_t n_chan)
{
    if (n_chan < 2) return -1;
    const unsigned __int128 q = (unsigned __int128)word * (uint64_t)n_chan + ((unsigned __int128)1 << 63);
    return (int32_t)((uint64_t)(q >> 64) % (uint64_t)n_chan);
}

/* Phase of NCO word w at absolute sample m: w*m mod 2^64. */
uint64_t orc_nco_phase(uint64_t word, uint64_t m) { return word * m; }

/* exp(-i * 2*pi * phase / 2^64), with the angle taken in [-pi, pi). */
static void orc_mixer(uint64_t phase, double* re, double* im)
{
    const double a = (double)(int64_t)phase * ldexp(M_PI, -63);
    *re = cos(a);
    *im = -sin(a);
}

/* ------------------------------------------------------------------------ */
/* DFT: brute force and FFT                                                   */
/* ------------------------------------------------------------------------ */

/* y[c] = sum_p x[p] exp(-2*pi*i*c*p/N), O(N^2).  The index c*p is reduced
 * mod N in integer arithmetic before the angle is formed. */
int orc_dft(int32_t n, const double* x, double* y)
{
    if (n <= 0 || !x || !y || x == y) return -1;
    for (int32_t c = 0; c < n; ++c) {
        double sr = 0.0, si = 0.0;
        for (int32_t p = 0; p < n; ++p) {
            const int64_t e = ((int64_t)c * p) % n;
            const double a = -2.0 * M_PI * (double)e / (double)n;
            const double wr = cos(a), wi = sin(a);
            sr += x[2 * p] * wr - x[2 * p + 1] * wi;
            si += x[2 * p] * wi + x[2 * p + 1] * wr;
        }
        y[2 * c] = sr;
        y[2 * c + 1] = si;
    }
    return 0;
}

/* In-place iterative radix-2 decimation-in-time FFT, same sign and order as
 * orc_dft, for N a power of two.  Twiddles are evaluated directly from
 * cos/sin of the exact angle for every butterfly. */
static void orc_fft_radix2(int32_t n, double* x)
{
    for (int32_t i = 1, j = 0; i < n; ++i) {          /* bit reversal */
        int32_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = x[2 * i]; x[2 * i] = x[2 * j]; x[2 * j] = t;
            t = x[2 * i + 1]; x[2 * i + 1] = x[2 * j + 1]; x[2 * j + 1] = t;
        }
    }
    for (int32_t len = 2; len <= n; len <<= 1) {
        const int32_t half = len >> 1;
        for (int32_t s = 0; s < n; s += len) {
            for (int32_t q = 0; q < half; ++q) {
                const double a = -2.0 * M_PI * (double)q / (double)len;
                const double wr = cos(a), wi = sin(a);
                double* u = x + 2 * (s + q);
                double* v = x + 2 * (s + q + half);
                const double tr = v[0] * wr - v[1] * wi;
                const double ti = v[0] * wi + v[1] * wr;
                v[0] = u[0] - tr; v[1] = u[1] - ti;
                u[0] += tr;       u[1] += ti;
            }
        }
    }
}

/* Mixed-radix decimation in time for any N (Cooley-Tukey on the smallest
 * prime factor p of N, N = p*m):
 *   X_q[k]   = sum_{j<m} x[j*p + q] W_m^{jk}            (p transforms of size m)
 *   y[k+m*s] = sum_{q<p} W_N^{q*(k+m*s)} X_q[k]         (k < m, s < p)
 * with W_N = exp(-2*pi*i/N); a prime N is the direct sum.  The twiddles are
 * read from a table of cos/sin of -2*pi*e/N, e < N, with e reduced mod N in
 * integer arithmetic.  x is read with the given stride (complex elements). */
static int orc_fft_rec(int64_t n, const double* x, int64_t stride, double* y)
{
    if (n == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return 0;
    }
    int64_t p = 2;
    while (p * p <= n && n % p != 0) ++p;
    if (n % p != 0) p = n;                           /* n is prime */
    const int64_t m = n / p;
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* sub = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!w || !sub) {
        free(w);
        free(sub);
        return -2;
    }
    for (int64_t e = 0; e < n; ++e) {
        const double a = -2.0 * M_PI * (double)e / (double)n;
        w[2 * e] = cos(a);
        w[2 * e + 1] = sin(a);
    }
    int rc = 0;
    for (int64_t q = 0; q < p && rc == 0; ++q)
        rc = orc_fft_rec(m, x + 2 * q * stride, stride * p, sub + 2 * q * m);
    for (int64_t s = 0; s < p && rc == 0; ++s) {
        for (int64_t k = 0; k < m; ++k) {
            const int64_t c = k + m * s;
            double ar = 0.0, ai = 0.0;
            for (int64_t q = 0; q < p; ++q) {
                const int64_t e = (q * c) % n;
                const double* xq = sub + 2 * (q * m + k);
                ar += xq[0] * w[2 * e] - xq[1] * w[2 * e + 1];
                ai += xq[0] * w[2 * e + 1] + xq[1] * w[2 * e];
            }
            y[2 * c] = ar;
            y[2 * c + 1] = ai;
        }
    }
    free(w);
    free(sub);
    return rc;
}

/* In-place FFT of any length N >= 1, same sign and order as orc_dft: the
 * radix-2 form for powers of two, the mixed-radix recursion otherwise. */
int orc_fft(int32_t n, double* x)
{
    if (n <= 0 || !x) return -1;
    if ((n & (n - 1)) == 0) {
        orc_fft_radix2(n, x);
        return 0;
    }
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!y) return -2;
    const int rc = orc_fft_rec(n, x, 1, y);
    if (rc == 0) memcpy(x, y, sizeof(double) * 2 * (size_t)n);
    free(y);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Polyphase filter bank (Sec. III.A)                                        */
/* ------------------------------------------------------------------------ */

/* Critically sampled PFB over a complex FP64 stream x[0..n_samples) with
 * zero history before sample 0.  For frames k in [k_begin, k_end):
 *   window   w_k[j] = x[(k+1)N - M + j],  j < M = N*T  (x[m<0] = 0)
 *   FIR      v_k[p] = sum_{t<T} h[t*N + p] * w_k[t*N + p]   (the N x T
 *            "matrix" of the section summed along its T direction)
 *   FFT      y_k[c] = sum_p v_k[p] exp(-2*pi*i*c*p/N)   (batched FFT step)
 *   select   tone_out[s][k] = y_k[bins[s]]              (user channels)
 * Outputs (each may be NULL):
 *   v_out    [k_end-k_begin][N] complex   (the filtered, decimated frames)
 *   full     [k_end-k_begin][N] complex   (the whole spectrum)
 *   tones    [n_bins][k_end-k_begin] complex
 * h holds M taps (the caller passes the FP32-rounded values promoted to FP64
 * when it checks an FP32-coefficient implementation). */
int orc_pfb_f64(const double* x, int64_t n_samples, int32_t n_chan, int32_t taps,
                const double* h, int64_t k_begin, int64_t k_end,
                double* v_out, double* full,
                const int32_t* bins, int32_t n_bins, double* tones)
{
    if (n_chan <= 0 || taps <= 0 || !h) return -1;
    if (k_begin < 0 || k_end < k_begin) return -1;
    if ((k_end) * (int64_t)n_chan > n_samples) return -1;
    if (n_bins > 0 && (!bins || !tones)) return -1;
    for (int32_t s = 0; s < n_bins; ++s)
        if (bins[s] < 0 || bins[s] >= n_chan) return -1;
    const int64_t n = n_chan, m = n * taps, nk = k_end - k_begin;
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!y) return -2;
    for (int64_t k = k_begin; k < k_end; ++k) {
        const int64_t start = (k + 1) * n - m;
        for (int64_t p = 0; p < n; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int64_t t = 0; t < taps; ++t) {
                const int64_t j = t * n + p;
                const int64_t idx = start + j;
                if (idx < 0) continue;                /* zero history */
                ar += h[j] * x[2 * idx];
                ai += h[j] * x[2 * idx + 1];
            }
            y[2 * p] = ar;
            y[2 * p + 1] = ai;
        }
        if (v_out) memcpy(v_out + 2 * (k - k_begin) * n, y, sizeof(double) * 2 * (size_t)n);
        if (orc_fft((int32_t)n, y) != 0) {
            free(y);
            return -2;
        }
        if (full) memcpy(full + 2 * (k - k_begin) * n, y, sizeof(double) * 2 * (size_t)n);
        for (int32_t s = 0; s < n_bins; ++s) {
            tones[2 * ((int64_t)s * nk + (k - k_begin))] = y[2 * bins[s]];
            tones[2 * ((int64_t)s * nk + (k - k_begin)) + 1] = y[2 * bins[s] + 1];
        }
    }
    free(y);
    return 0;
}

/* The same on the complex int16 stream the software radio delivers
 * (interleaved I, Q; Sec. II.A).  Each sample is promoted to FP64 exactly. */
int orc_pfb_i16(const int16_t* iq, int64_t n_samples, int32_t n_chan, int32_t taps,
                const double* h, int64_t k_begin, int64_t k_end,
                double* full, const int32_t* bins, int32_t n_bins, double* tones)
{
    if (!iq || n_samples < 0) return -1;
    /* only the samples the requested frames touch are promoted */
    const int64_t m = (int64_t)n_chan * taps;
    int64_t lo = (k_begin + 1) * (int64_t)n_chan - m;
    if (lo < 0) lo = 0;
    const int64_t hi = k_end * (int64_t)n_chan;
    if (hi > n_samples || k_end < k_begin) return -1;
    const int64_t cnt = hi > lo ? hi - lo : 0;
    double* x = (double*)malloc(sizeof(double) * 2 * (size_t)(cnt + 1));
    if (!x) return -2;
    for (int64_t i = 0; i < 2 * cnt; ++i) x[i] = (double)iq[2 * lo + i];
    /* shift the frame origin so that orc_pfb_f64 sees sample lo at index 0:
     * frame k of the stream is frame k - lo/N of the slice (lo is a multiple
     * of N whenever it is positive). */
    int rc;
    if (lo == 0) {
        rc = orc_pfb_f64(x, cnt, n_chan, taps, h, k_begin, k_end, NULL, full, bins, n_bins, tones);
    } else {
        const int64_t kofs = lo / n_chan;
        rc = orc_pfb_f64(x, cnt, n_chan, taps, h, k_begin - kofs, k_end - kofs,
                         NULL, full, bins, n_bins, tones);
    }
    free(x);
    return rc;
}

/* PFB with a hop of H samples between frames (H = N: the critically sampled
 * PFB above; H < N: oversampled), on the complex int16 stream, each sample
 * promoted to FP64 exactly.  iq[i] is the sample at ABSOLUTE stream index
 * m0 + i (m0 = 0: the stream start); samples before m0 are zero.  Frame k
 * (an absolute frame index) uses the M = N*T samples that end at sample
 * (k+1)*H - 1, i.e. start at s_k = (k+1)*H - M, and its channels keep the
 * phase of the absolute time origin:
 *   v_k[p] = sum_{t<T} h[t*N + p] * x[s_k + t*N + p]
 *   y_k[c] = sum_p v_k[p] exp(-2*pi*i*c*(s_k + p)/N)
 * so channel c is the stream mixed down by exp(-2*pi*i*c*m/N) and filtered,
 * exactly as the direct demodulator gives it for the bin-centred word (for
 * H = N, s_k is a multiple of N and the factor is 1).  The exponent depends
 * on (s_k + p) mod N only, so y_k is the FFT of v_k circularly shifted by
 * s_k mod N: u[(p + s) mod N] = v_k[p]. */
int orc_pfb_hop_i16(const int16_t* iq, int64_t n_samples, int64_t m0, int32_t n_chan, int32_t taps,
                    int32_t hop, const double* h, int64_t k_begin, int64_t k_end,
                    double* full, const int32_t* bins, int32_t n_bins, double* tones)
{
    if (!iq || n_chan <= 0 || taps <= 0 || hop <= 0 || !h || k_begin < 0 || k_end < k_begin) return -1;
    if (m0 < 0 || k_end * (int64_t)hop - m0 > n_samples) return -1;
    if (n_bins > 0 && (!bins || !tones)) return -1;
    for (int32_t s = 0; s < n_bins; ++s)
        if (bins[s] < 0 || bins[s] >= n_chan) return -1;
    const int64_t n = n_chan, m = n * taps, nk = k_end - k_begin;
    double* v = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* u = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (!v || !u) {
        free(v);
        free(u);
        return -2;
    }
    int rc = 0;
    for (int64_t k = k_begin; k < k_end && rc == 0; ++k) {
        const int64_t start = (k + 1) * (int64_t)hop - m;
        for (int64_t p = 0; p < n; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int64_t t = 0; t < taps; ++t) {
                const int64_t idx = start + t * n + p;
                if (idx < m0) continue;               /* zero before the first sample */
                ar += h[t * n + p] * (double)iq[2 * (idx - m0)];
                ai += h[t * n + p] * (double)iq[2 * (idx - m0) + 1];
            }
            v[2 * p] = ar;
            v[2 * p + 1] = ai;
        }
        const int64_t sh = ((start % n) + n) % n;
        for (int64_t p = 0; p < n; ++p) {
            const int64_t q = (p + sh) % n;
            u[2 * q] = v[2 * p];
            u[2 * q + 1] = v[2 * p + 1];
        }
        rc = orc_fft((int32_t)n, u);
        if (rc != 0) break;
        if (full) memcpy(full + 2 * (k - k_begin) * n, u, sizeof(double) * 2 * (size_t)n);
        for (int32_t s = 0; s < n_bins; ++s) {
            tones[2 * ((int64_t)s * nk + (k - k_begin))] = u[2 * bins[s]];
            tones[2 * ((int64_t)s * nk + (k - k_begin)) + 1] = u[2 * bins[s] + 1];
        }
    }
    free(v);
    free(u);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Direct multi-tone demodulation (Sec. III.B)                               */
/* ------------------------------------------------------------------------ */

/* For each selected tone s (NCO word words[s]) and frame k in
 * [k_begin, k_end), with b_k = (k+1)*D - L:
 *   out[s][k] = sum_{n<L} h[n] * x[b_k + n] * exp(-i*2*pi*((w*(b_k+n)) mod 2^64)/2^64)
 * i.e. each sample is mixed against the tone (the per-tone NCO), low-pass
 * filtered by h and decimated by D.  Samples before the stream start are
 * zero.  The NCO phase is the exact uint64 product w*m. */
int orc_demod_f64(const double* x, int64_t n_samples, int32_t L, int32_t D,
                  const double* h, const uint64_t* words, int32_t n_sel,
                  int64_t k_begin, int64_t k_end, double* out)
{
    if (L <= 0 || D <= 0 || !h || !x || (n_sel > 0 && (!words || !out))) return -1;
    if (k_begin < 0 || k_end < k_begin || k_end * (int64_t)D > n_samples) return -1;
    const int64_t nk = k_end - k_begin;
    for (int32_t s = 0; s < n_sel; ++s) {
        for (int64_t k = k_begin; k < k_end; ++k) {
            const int64_t b = (k + 1) * (int64_t)D - L;
            double ar = 0.0, ai = 0.0;
            for (int64_t n = 0; n < L; ++n) {
                const int64_t m = b + n;
                if (m < 0) continue;
                double cr, ci;
                orc_mixer(orc_nco_phase(words[s], (uint64_t)m), &cr, &ci);
                const double xr = x[2 * m], xi = x[2 * m + 1];
                ar += h[n] * (xr * cr - xi * ci);
                ai += h[n] * (xr * ci + xi * cr);
            }
            out[2 * ((int64_t)s * nk + (k - k_begin))] = ar;
            out[2 * ((int64_t)s * nk + (k - k_begin)) + 1] = ai;
        }
    }
    return 0;
}

/* The same on a complex int16 stream (exact promotion of the samples) that
 * starts at ABSOLUTE sample index m0 >= 0: iq[i] is sample m0 + i, samples
 * before m0 are zero, frame indices k are absolute (b_k = (k+1)*D - L) and
 * the NCO phase is w * (absolute index) mod 2^64.  m0 = 0 is the stream
 * start with zero history. */
int orc_demod_i16(const int16_t* iq, int64_t n_samples, int64_t m0, int32_t L, int32_t D,
                  const double* h, const uint64_t* words, int32_t n_sel,
                  int64_t k_begin, int64_t k_end, double* out)
{
    if (!iq || L <= 0 || D <= 0 || m0 < 0 || k_begin < 0 || k_end < k_begin) return -1;
    if (k_end * (int64_t)D - m0 > n_samples) return -1;
    if (n_sel > 0 && (!words || !out)) return -1;
    const int64_t nk = k_end - k_begin;
    for (int32_t s = 0; s < n_sel; ++s) {
        for (int64_t k = k_begin; k < k_end; ++k) {
            const int64_t b = (k + 1) * (int64_t)D - L;
            double ar = 0.0, ai = 0.0;
            for (int64_t n = 0; n < L; ++n) {
                const int64_t m = b + n;
                if (m < m0) continue;
                double cr, ci;
                orc_mixer(orc_nco_phase(words[s], (uint64_t)m), &cr, &ci);
                const double xr = (double)iq[2 * (m - m0)], xi = (double)iq[2 * (m - m0) + 1];
                ar += h[n] * (xr * cr - xi * ci);
                ai += h[n] * (xr * ci + xi * cr);
            }
            out[2 * ((int64_t)s * nk + (k - k_begin))] = ar;
            out[2 * ((int64_t)s * nk + (k - k_begin)) + 1] = ai;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Chirped readout (Sec. III.C, Eq. 1)                                       */
/* ------------------------------------------------------------------------ */

/* Eq. 1 in sample units: phi(m) = 2*pi*(f0*t + k*t^2) with t = m/fs becomes
 * the uint64 phase  p(m) = s*m + r*m^2  (mod 2^64)  in units of 2*pi/2^64,
 * with s = f0/fs * 2^64 (a start word) and r = k/fs^2 * 2^64 (a rate word).
 * m may be negative (two's complement, reduced mod 2^64). */
uint64_t orc_chirp_phase(uint64_t start_word, uint64_t rate_word, int64_t m)
{
    const uint64_t um = (uint64_t)m;
    return start_word * um + rate_word * (um * um);
}

/* The rate word of a chirp rate k (Hz/s) at sample rate fs: k/fs^2 * 2^64,
 * rounded to nearest (two's complement for negative rates). */
uint64_t orc_chirp_rate_word(double k_hz_per_s, double fs)
{
    return (uint64_t)(int64_t)llround(ldexp(k_hz_per_s / (fs * fs), 64));
}

/* Transmit buffer of a chirp of amplitude A (Sec. III.C: generated in real
 * time instead of stored): samples m0 .. m0+n-1 as complex int16
 * (round half to even of A*cos(theta), A*sin(theta), theta = 2*pi*p(m)/2^64,
 * clamped to the int16 range). */
int orc_chirp_synth(uint64_t start_word, uint64_t rate_word, double amp, int64_t m0, int64_t n,
                    int16_t* iq)
{
    if (n < 0 || !iq) return -1;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t p = orc_chirp_phase(start_word, rate_word, m0 + i);
        const double a = (double)(int64_t)p * ldexp(M_PI, -63);
        double re = nearbyint(amp * cos(a)), im = nearbyint(amp * sin(a));
        if (re > 32767.0) re = 32767.0;
        if (re < -32768.0) re = -32768.0;
        if (im > 32767.0) im = 32767.0;
        if (im < -32768.0) im = -32768.0;
        iq[2 * i] = (int16_t)re;
        iq[2 * i + 1] = (int16_t)im;
    }
    return 0;
}

/* Demodulation against chirps (Sec. III.C, demodulated by the method of
 * Sec. III.B): as orc_demod_i16 (same absolute origin m0) with the linear NCO
 * phase replaced by the chirp phase p(m): for each chirp s and frame k,
 * b_k = (k+1)*D - L,
 *   out[s][k] = sum_{n<L} h[n] * x[b_k+n] * exp(-i*2*pi*p_s(b_k+n)/2^64). */
int orc_chirp_demod_i16(const int16_t* iq, int64_t n_samples, int64_t m0, int32_t L, int32_t D,
                        const double* h, const uint64_t* start_words, const uint64_t* rate_words,
                        int32_t n_sel, int64_t k_begin, int64_t k_end, double* out)
{
    if (!iq || L <= 0 || D <= 0 || m0 < 0 || k_begin < 0 || k_end < k_begin) return -1;
    if (k_end * (int64_t)D - m0 > n_samples) return -1;
    if (n_sel > 0 && (!start_words || !rate_words || !out)) return -1;
    const int64_t nk = k_end - k_begin;
    for (int32_t s = 0; s < n_sel; ++s) {
        for (int64_t k = k_begin; k < k_end; ++k) {
            const int64_t b = (k + 1) * (int64_t)D - L;
            double ar = 0.0, ai = 0.0;
            for (int64_t n = 0; n < L; ++n) {
                const int64_t m = b + n;
                if (m < m0) continue;
                double cr, ci;
                orc_mixer(orc_chirp_phase(start_words[s], rate_words[s], m), &cr, &ci);
                const double xr = (double)iq[2 * (m - m0)], xi = (double)iq[2 * (m - m0) + 1];
                ar += h[n] * (xr * cr - xi * ci);
                ai += h[n] * (xr * ci + xi * cr);
            }
            out[2 * ((int64_t)s * nk + (k - k_begin))] = ar;
            out[2 * ((int64_t)s * nk + (k - k_begin)) + 1] = ai;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transmit buffer (Sec. III: the GPU also generates the transmission       */
/* buffer; the tones are the same NCO words the receiver demodulates)       */
/* ------------------------------------------------------------------------ */

/* Multi-tone transmit samples m0 .. m0+n-1:
 *   s(m) = sum_t A_t exp(+i*2*pi*((w_t*m + p_t) mod 2^64)/2^64)
 * (a tone at word w is brought to DC by the receiver's mixer exp(-i*w*m)),
 * in FP64 with the angle formed from the exact integer phase as in
 * orc_mixer; value[2m], value[2m+1] receive Re, Im (may be NULL), iq the
 * round-half-even of each, clamped to int16 (may be NULL).  p may be NULL
 * (zero phase offsets). */
int orc_tones_synth(const uint64_t* words, const uint64_t* phase_words, const double* amps, int32_t n_tones,
                    int64_t m0, int64_t n, double* value, int16_t* iq)
{
    if (n < 0 || n_tones < 0 || (n_tones > 0 && (!words || !amps))) return -1;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t m = (uint64_t)(m0 + i);
        double re = 0.0, im = 0.0;
        for (int32_t t = 0; t < n_tones; ++t) {
            const uint64_t ph = words[t] * m + (phase_words ? phase_words[t] : 0);
            const double a = (double)(int64_t)ph * ldexp(M_PI, -63);
            re += amps[t] * cos(a);
            im += amps[t] * sin(a);
        }
        if (value) {
            value[2 * i] = re;
            value[2 * i + 1] = im;
        }
        if (iq) {
            double r = nearbyint(re), q = nearbyint(im);
            if (r > 32767.0) r = 32767.0;
            if (r < -32768.0) r = -32768.0;
            if (q > 32767.0) q = 32767.0;
            if (q < -32768.0) q = -32768.0;
            iq[2 * i] = (int16_t)r;
            iq[2 * i + 1] = (int16_t)q;
        }
    }
    return 0;
}
