/*
 * vspec_oracle.c — plain FP64 CPU oracle for the streaming channelizer of
 * "A GPU-Based Wide-Band Radio Spectrometer" (arXiv 1411.0436).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * reference against which the CUDA path is checked. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it. It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (§4 of the paper, "The GPU Spectrometer"):
 *   input     dual- or single-polarisation 8-bit complex voltages (§4);
 *   pre-filter an N-tap polyphase filter bank, i.e. a weighted overlap-add
 *             of P consecutive frames of N samples (§4, the PFB paragraph),
 *             or nothing in direct-FFT mode (§5);
 *   FFT       an N-point DFT per polarisation (§4, "perform parallel FFTs");
 *   detect    X^2, Y^2, Re(XY*), Im(XY*) (§4);
 *   accumulate the detected spectra over the integration (§4).
 *
 * The paper leaves several things unstated; this file fixes them as follows:
 *   - sample layout   int8 [time][pol][re, im]; single-pol is [time][re, im];
 *   - coefficients    h[i] = w[i] * sinc((i - (L-1)/2) / N), L = P*N,
 *                     sinc(u) = sin(pi u)/(pi u), symmetric windows with an
 *                     (L-1) denominator, no normalisation; direct mode uses
 *                     the bare window of length N;
 *   - tap order       h[t*N + n] multiplies frame s+t (frame s is the oldest);
 *   - hop             critically sampled: one spectrum per N new samples;
 *   - DFT             X[k] = sum_n y[n] exp(-2 pi i n k / N), unnormalised,
 *                     natural order (k = 0 is DC, no shift);
 *   - cross product   X * conj(Y);
 *   - accumulation    a plain sum over spectra (not a mean).
 *
 * Every step is written out as its definition in double precision; the FFT is
 * the textbook recursive radix-2 decimation-in-time split, and nothing is
 * blocked, fused or reordered beyond that.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VSO_PFB 0
#define VSO_DIRECT 1
#define VSO_WIN_RECT 0
#define VSO_WIN_HANN 1
#define VSO_WIN_HAMMING 2

static const double VSO_PI = 3.14159265358979323846264338327950288;

/* Window value at index i of a symmetric window of length L. */
static double window_value(int window, long i, long L)
{
    if (window == VSO_WIN_RECT || L < 2) return 1.0;
    double phase = 2.0 * VSO_PI * (double)i / (double)(L - 1);
    if (window == VSO_WIN_HANN) return 0.5 - 0.5 * cos(phase);
    return 0.54 - 0.46 * cos(phase); /* Hamming */
}

/* Normalised sinc, sin(pi u) / (pi u), equal to 1 at u = 0. */
static double sinc(double u)
{
    if (u == 0.0) return 1.0;
    return sin(VSO_PI * u) / (VSO_PI * u);
}

/* Number of frames each spectrum draws on: P in PFB mode, 1 in direct mode. */
static int taps_used(int ntaps, int mode)
{
    return mode == VSO_DIRECT ? 1 : ntaps;
}

/*
 * Filter coefficients (§4: the pre-filter's coefficients are loaded at
 * initialisation; their values are not given in the paper, see the file
 * header for the reading used). Writes L = P_eff * nchan values to h and
 * returns L, or -1 on bad arguments.
 */
long vso_coeffs(int nchan, int ntaps, int mode, int window, double *h)
{
    if (nchan < 1 || (mode != VSO_PFB && mode != VSO_DIRECT)) return -1;
    if (mode == VSO_PFB && ntaps < 1) return -1;
    if (window < VSO_WIN_RECT || window > VSO_WIN_HAMMING) return -1;
    int P = taps_used(ntaps, mode);
    long L = (long)P * nchan;
    for (long i = 0; i < L; i++) {
        double w = window_value(window, i, L);
        if (mode == VSO_PFB) {
            double u = ((double)i - 0.5 * (double)(L - 1)) / (double)nchan;
            h[i] = w * sinc(u);
        } else {
            h[i] = w;
        }
    }
    return L;
}

/*
 * Recursive radix-2 decimation-in-time DFT of n (a power of two) complex
 * values read from x with the given element stride; the result goes to out
 * in natural order. Complex values are interleaved (re, im) doubles.
 *   out[k]       = E[k] + W_n^k O[k]
 *   out[k + n/2] = E[k] - W_n^k O[k],   W_n = exp(-2 pi i / n),
 * where E and O are the DFTs of the even- and odd-indexed inputs.
 */
static void fft_rec(const double *x, long n, long stride, double *out)
{
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    long h = n / 2;
    fft_rec(x, h, 2 * stride, out);                  /* even inputs -> out[0, h)  */
    fft_rec(x + 2 * stride, h, 2 * stride, out + 2 * h); /* odd inputs -> out[h, n) */
    for (long k = 0; k < h; k++) {
        double ang = -2.0 * VSO_PI * (double)k / (double)n;
        double wr = cos(ang), wi = sin(ang);
        double er = out[2 * k], ei = out[2 * k + 1];
        double orr = out[2 * (k + h)], oi = out[2 * (k + h) + 1];
        double tr = wr * orr - wi * oi;
        double ti = wr * oi + wi * orr;
        out[2 * k] = er + tr;
        out[2 * k + 1] = ei + ti;
        out[2 * (k + h)] = er - tr;
        out[2 * (k + h) + 1] = ei - ti;
    }
}

/* Forward unnormalised DFT of n complex values (n a power of two). */
int vso_fft(const double *in, double *out, long n)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    fft_rec(in, n, 1, out);
    return 0;
}

/* Complex sample m of polarisation p, from either the int8 or the f64 input. */
static void fetch(const int8_t *in8, const double *in64, int npol, long m, int p,
                  double *re, double *im)
{
    long idx = (m * npol + p) * 2;
    if (in8) {
        *re = (double)in8[idx];
        *im = (double)in8[idx + 1];
    } else {
        *re = in64[idx];
        *im = in64[idx + 1];
    }
}

/*
 * Pre-filter for one spectrum s of polarisation p (§4, PFB paragraph):
 *   y[n] = sum_{t=0}^{P_eff-1} h[t*N + n] * x[(s + t)*N + n],  0 <= n < N.
 * In direct mode P_eff = 1 and h is the window of length N.
 */
static void fir_one(const int8_t *in8, const double *in64, int nchan, int P, int npol,
                    const double *h, long s, int p, double *y)
{
    for (long n = 0; n < nchan; n++) {
        double ar = 0.0, ai = 0.0;
        for (int t = 0; t < P; t++) {
            double xr, xi;
            fetch(in8, in64, npol, (s + t) * (long)nchan + n, p, &xr, &xi);
            ar += h[(long)t * nchan + n] * xr;
            ai += h[(long)t * nchan + n] * xi;
        }
        y[2 * n] = ar;
        y[2 * n + 1] = ai;
    }
}

/* Exported pre-filter of one spectrum, for the tests of the tap order. */
int vso_fir(const double *in64, int nchan, int ntaps, int npol, int mode, int window,
            long s, int p, double *y)
{
    int P = taps_used(ntaps, mode);
    double *h = (double *)malloc(sizeof(double) * (size_t)P * nchan);
    if (!h) return -1;
    if (vso_coeffs(nchan, ntaps, mode, window, h) < 0) { free(h); return -1; }
    fir_one(NULL, in64, nchan, P, npol, h, s, p, y);
    free(h);
    return 0;
}

/*
 * The whole path: pre-filter, DFT, detect and accumulate nspectra spectra.
 * Input holds (nspectra + P_eff - 1) * nchan time samples per polarisation.
 * Output (overwritten): npol == 2 -> out[4k + {0,1,2,3}] = XX, YY, Re(XY*),
 * Im(XY*); npol == 1 -> out[k] = XX. Spectra are split into contiguous blocks
 * over threads and the per-thread sums are added in thread order.
 */
static int channelize(const int8_t *in8, const double *in64, int nchan, int ntaps,
                      int npol, int mode, int window, long nspectra, double *out,
                      int nthreads)
{
    if (nchan < 1 || (nchan & (nchan - 1)) != 0) return -1;
    if (npol != 1 && npol != 2) return -1;
    if (nspectra < 0) return -1;
    int P = taps_used(ntaps, mode);
    int nout = npol == 2 ? 4 : 1;
    double *h = (double *)malloc(sizeof(double) * (size_t)P * nchan);
    if (!h) return -1;
    if (vso_coeffs(nchan, ntaps, mode, window, h) < 0) { free(h); return -1; }

    int T = 1;
#ifdef _OPENMP
    T = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
    if (T < 1) T = 1;
    double *part = (double *)calloc((size_t)T * nout * nchan, sizeof(double));
    if (!part) { free(h); return -1; }
    int failed = 0;

#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        long s0 = nspectra * tid / T, s1 = nspectra * (tid + 1) / T;
        double *acc = part + (size_t)tid * nout * nchan;
        double *y = (double *)malloc(sizeof(double) * 2 * (size_t)nchan);
        double *X = (double *)malloc(sizeof(double) * 2 * (size_t)nchan * npol);
        if (!y || !X) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        } else {
            for (long s = s0; s < s1; s++) {
                for (int p = 0; p < npol; p++) {
                    fir_one(in8, in64, nchan, P, npol, h, s, p, y);
                    fft_rec(y, nchan, 1, X + 2 * (size_t)nchan * p);
                }
                const double *Xp = X, *Yp = X + 2 * (size_t)nchan;
                for (long k = 0; k < nchan; k++) {
                    double xr = Xp[2 * k], xi = Xp[2 * k + 1];
                    if (npol == 1) {
                        acc[k] += xr * xr + xi * xi;
                    } else {
                        double yr = Yp[2 * k], yi = Yp[2 * k + 1];
                        acc[4 * k + 0] += xr * xr + xi * xi;     /* |X|^2       */
                        acc[4 * k + 1] += yr * yr + yi * yi;     /* |Y|^2       */
                        acc[4 * k + 2] += xr * yr + xi * yi;     /* Re(X Y*)    */
                        acc[4 * k + 3] += xi * yr - xr * yi;     /* Im(X Y*)    */
                    }
                }
            }
        }
        free(y);
        free(X);
    }

    if (!failed) {
        for (long i = 0; i < (long)nout * nchan; i++) {
            double a = 0.0;
            for (int t = 0; t < T; t++) a += part[(size_t)t * nout * nchan + i];
            out[i] = a;
        }
    }
    free(part);
    free(h);
    return failed ? -1 : 0;
}

int vso_channelize(const int8_t *in, int nchan, int ntaps, int npol, int mode, int window,
                   long nspectra, double *out, int nthreads)
{
    return channelize(in, NULL, nchan, ntaps, npol, mode, window, nspectra, out, nthreads);
}

/* Same path on real-valued (double) samples, for pins that need exact tones. */
int vso_channelize_f64(const double *in, int nchan, int ntaps, int npol, int mode,
                       int window, long nspectra, double *out, int nthreads)
{
    return channelize(NULL, in, nchan, ntaps, npol, mode, window, nspectra, out, nthreads);
}

/* Number of OpenMP threads a call with nthreads = 0 would use. */
int vso_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
