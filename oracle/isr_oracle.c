/*
 * isr_oracle.c -- plain FP64 CPU oracle for plasma-line power-spectrum integration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA library and includes nothing from it.
 *
 * What it computes (Hilliard, Vierinen & Erickson, "GPGPU Acceleration of Incoherent
 * Scatter Radar Plasma Line Analysis", Sec. 2.2, Eqs. 7-8, and the three GPU kernels of
 * Sec. 3.2):
 *
 *   for every range gate r with window start s_r = range_start + r * range_step,
 *   for every inter-pulse period (IPP) p:
 *       x[k] = conj(eps_p[k]) * m_p[s_r + k]          k <  code_len   (decode, Eq. 7)
 *       x[k] = 0                                      code_len <= k < nfft (zero pad)
 *       X[f] = sum_k x[k] exp(-2 pi i f k / nfft)     forward DFT, natural bin order
 *       P[r][f] += |X[f]|^2                           power integration (Eq. 8)
 *
 * P is the SUM over IPPs (the paper's accumulation kernel adds into the spectrum; the
 * mean of Eq. 8 is that sum divided by the number of IPPs).
 *
 * The transform is a textbook iterative radix-2 decimation-in-time FFT: bit-reversal
 * permutation followed by log2(nfft) butterfly stages, twiddles exp(-2 pi i j / len)
 * evaluated with cos()/sin() in double.  Accumulation is in double.
 *
 * Input conventions:
 *   echo  : int16 interleaved (I, Q) samples, row p starts at echo + 2 * p * echo_stride.
 *   tx    : one code row of code_len chips, row p at tx + p * tx_stride chips
 *           (tx_stride = 0: one code shared by all IPPs).  Chip formats:
 *             ORC_TX_CI16 : int16 (I, Q) pairs, eps = I + iQ
 *             ORC_TX_C32  : float (re, im) pairs, eps = re + i im
 *             ORC_TX_PM1  : int8 per chip, eps = -1 where the byte is negative, else +1
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_TX_CI16 = 0, ORC_TX_C32 = 1, ORC_TX_PM1 = 2 };

static const double ORC_PI = 3.14159265358979323846;

/* Precomputed forward twiddles: w[j] = exp(-2 pi i j / n), j < n/2. */
static void make_twiddles(int n, double* wr, double* wi)
{
    for (int j = 0; j < n / 2; ++j) {
        double a = -2.0 * ORC_PI * (double)j / (double)n;
        wr[j] = cos(a);
        wi[j] = sin(a);
    }
}

/* In-place forward FFT of length n (a power of two), radix-2 DIT. */
static void fft_inplace(double* re, double* im, int n, const double* wr, const double* wi)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    /* butterflies: stage with sub-transform length len combines two halves */
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        int tstep = n / len; /* exp(-2 pi i k / len) = w[k * n / len] */
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < half; ++k) {
                double cr = wr[k * tstep], ci = wi[k * tstep];
                int a = i + k, b = i + k + half;
                double vr = re[b] * cr - im[b] * ci;
                double vi = re[b] * ci + im[b] * cr;
                re[b] = re[a] - vr;
                im[b] = im[a] - vi;
                re[a] = re[a] + vr;
                im[a] = im[a] + vi;
            }
        }
    }
}

/* Exported: forward FFT of one vector (used by the pin tests). */
int oracle_fft(double* re, double* im, int n)
{
    if (n < 1 || (n & (n - 1))) return 1;
    if (n == 1) return 0;
    double* wr = (double*)malloc(sizeof(double) * (size_t)(n / 2));
    double* wi = (double*)malloc(sizeof(double) * (size_t)(n / 2));
    if (!wr || !wi) { free(wr); free(wi); return 2; }
    make_twiddles(n, wr, wi);
    fft_inplace(re, im, n, wr, wi);
    free(wr);
    free(wi);
    return 0;
}

/* conj(eps) of chip k of one code row */
static void tx_chip(const void* tx_row, int tx_type, int k, double* er, double* ei)
{
    if (tx_type == ORC_TX_CI16) {
        const int16_t* t = (const int16_t*)tx_row;
        *er = (double)t[2 * k];
        *ei = (double)t[2 * k + 1];
    } else if (tx_type == ORC_TX_C32) {
        const float* t = (const float*)tx_row;
        *er = (double)t[2 * k];
        *ei = (double)t[2 * k + 1];
    } else {
        const int8_t* t = (const int8_t*)tx_row;
        *er = t[k] < 0 ? -1.0 : 1.0;
        *ei = 0.0;
    }
}

static size_t tx_chip_bytes(int tx_type)
{
    return tx_type == ORC_TX_CI16 ? 4 : tx_type == ORC_TX_C32 ? 8 : 1;
}

/*
 * Exported: integrate power spectra.
 *   sel, n_sel : which range gates to compute (indices r into the gate list);
 *                sel = NULL computes gates 0 .. n_ranges-1 and n_sel must equal n_ranges.
 *   P          : [n_sel][nfft] doubles, ADDED to (the caller zeroes it for a fresh sum).
 *   n_threads  : OpenMP threads over the selected gates (<= 0: library default).
 * Returns 0 on success, nonzero on a bad argument or allocation failure.
 */
int oracle_integrate(const int16_t* echo, int64_t echo_stride,
                     const void* tx, int tx_type, int64_t tx_stride,
                     int n_ipp, int nfft, int code_len,
                     int n_ranges, int64_t range_start, int64_t range_step,
                     const int32_t* sel, int n_sel, double* P, int n_threads)
{
    if (nfft < 1 || (nfft & (nfft - 1)) || code_len < 1 || code_len > nfft) return 1;
    if (n_ipp < 0 || n_ranges < 0 || range_start < 0 || range_step < 0) return 1;
    if (!sel && n_sel != n_ranges) return 1;
    for (int i = 0; i < n_sel; ++i) {
        int64_t r = sel ? sel[i] : i;
        if (r < 0 || r >= n_ranges) return 1;
        if (range_start + r * range_step + code_len > echo_stride) return 3;
    }
    if (n_ipp == 0 || n_sel == 0) return 0;

    double* wr = (double*)malloc(sizeof(double) * (size_t)(nfft / 2 + 1));
    double* wi = (double*)malloc(sizeof(double) * (size_t)(nfft / 2 + 1));
    if (!wr || !wi) { free(wr); free(wi); return 2; }
    make_twiddles(nfft, wr, wi);
    size_t cb = tx_chip_bytes(tx_type);
    int fail = 0;

#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int i = 0; i < n_sel; ++i) {
        int64_t r = sel ? sel[i] : i;
        int64_t s_r = range_start + r * range_step;
        double* re = (double*)malloc(sizeof(double) * (size_t)nfft);
        double* im = (double*)malloc(sizeof(double) * (size_t)nfft);
        if (!re || !im) {
            free(re); free(im);
#ifdef _OPENMP
#pragma omp atomic write
#endif
            fail = 1;
            continue;
        }
        double* Pr = P + (size_t)i * (size_t)nfft;
        for (int p = 0; p < n_ipp; ++p) {
            const int16_t* m = echo + 2 * ((int64_t)p * echo_stride + s_r);
            const char* txrow = (const char*)tx + (size_t)((int64_t)p * tx_stride) * cb;
            for (int k = 0; k < nfft; ++k) {
                if (k < code_len) {
                    double er, ei;
                    tx_chip(txrow, tx_type, k, &er, &ei);
                    double mr = (double)m[2 * k], mi = (double)m[2 * k + 1];
                    /* conj(eps) * m = (er - i ei)(mr + i mi) */
                    re[k] = er * mr + ei * mi;
                    im[k] = er * mi - ei * mr;
                } else {
                    re[k] = 0.0;
                    im[k] = 0.0;
                }
            }
            fft_inplace(re, im, nfft, wr, wi);
            for (int f = 0; f < nfft; ++f) Pr[f] += re[f] * re[f] + im[f] * im[f];
        }
        free(re);
        free(im);
    }
    free(wr);
    free(wi);
    return fail ? 2 : 0;
}
