/*
 * synth_core.h -- seeded synthetic radar echoes (inputs only; no decoding, no transform,
 * no power arithmetic).
 *
 * One header compiled twice: by gcc for the host generator (synth_host.c) and by nvcc for
 * the device generator (synth_gpu.cu).  Both builds switch off floating-point
 * contraction (-ffp-contract=off / -fmad=false) and use only IEEE-exact operations
 * (+, -, *, /, sqrt, rint), so they produce bit-identical int16 samples.  The
 * transcendental functions below are this file's own Taylor / atanh series, not a
 * library's.
 *
 * Model (the paper's measurement equation, Sec. 2.2, Eqs. 2-3):
 *
 *   m_p[t] = sum_{r : s_r <= t < s_r + L} eps_p[t - s_r] * a_{r,p} * exp(2 pi i phi_{r,p}(t))
 *            + xi_p[t]
 *
 *   - eps_p : binary-phase code, +-1 chips drawn from Philox bits;
 *   - a_{r,p}: per (gate, IPP) complex amplitude (random phase for a tone, circular
 *              complex Gaussian for a Langmuir line), drawn independently per IPP as
 *              Eq. 3 states for the scatter;
 *   - phi    : frequency f_r (+ a Cauchy jitter for a line: a Lorentzian spectral line of
 *              the given half width) times t, kept as a 32-bit phase accumulator;
 *   - xi     : circular complex Gaussian noise, sigma per component (Box-Muller);
 *   - the sum is rounded to nearest-even and saturated to int16 per component.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), keyed by the 64-bit seed, one counter per (index, row,
 * purpose).
 */
#ifndef ISR_SYNTH_CORE_H
#define ISR_SYNTH_CORE_H

#include <stdint.h>

#ifdef __CUDACC__
#define SYN_HD __host__ __device__ __forceinline__
#else
#define SYN_HD static inline
#include <math.h>
#endif

enum { SYN_NOISE_ONLY = 0, SYN_TONE = 1, SYN_LINE = 2 };
enum { SYN_PURPOSE_NOISE = 1, SYN_PURPOSE_CODE = 2, SYN_PURPOSE_LINE = 3, SYN_PURPOSE_FREQ = 4 };

#define SYN_TABLE_BITS 16
#define SYN_TABLE_SIZE (1 << SYN_TABLE_BITS)

typedef struct {
    uint64_t seed;
    int64_t echo_stride;  /* complex samples per IPP row */
    int32_t n_ipp;
    int32_t code_len;     /* L: chips per code, also the span each gate's echo covers */
    int32_t n_ranges;
    int32_t range_start;
    int32_t range_step;
    int32_t kind;         /* SYN_NOISE_ONLY / SYN_TONE / SYN_LINE */
    int32_t per_ipp_code; /* 0: one code row shared by all IPPs, 1: one row per IPP */
    int32_t pad_;
    double sigma;         /* noise standard deviation per component, counts */
    double amp;           /* tone: |a|; line: rms |a| (E|a|^2 = amp^2) */
    double hwhm;          /* line half width at half maximum, cycles per sample */
    double max_jitter;    /* clamp of the line's frequency jitter, cycles per sample */
} syn_cfg;

typedef struct {
    float ar, ai;   /* complex amplitude */
    uint32_t inc;   /* phase increment per sample, turns * 2^32 (two's complement) */
    uint32_t pad_;
} syn_rp;

/* ---------------------------------------------------------------- Philox4x32-10 */
SYN_HD void syn_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

SYN_HD void syn_philox(const uint32_t ctr_in[4], uint64_t seed, uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        syn_mulhilo(0xD2511F53u, c0, &hi0, &lo0);
        syn_mulhilo(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

SYN_HD void syn_draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, purpose, 0u};
    syn_philox(ctr, seed, out);
}

/* uniform in (0, 1), exact in double */
SYN_HD double syn_u01(uint32_t w)
{
    return (double)w * 2.3283064365386963e-10 + 1.1641532182693481e-10; /* 2^-32, 2^-33 */
}

/* ---------------------------------------------------------------- own elementary functions */
SYN_HD double syn_bits_to_double(uint64_t b)
{
    union { uint64_t u; double d; } v;
    v.u = b;
    return v.d;
}

SYN_HD uint64_t syn_double_to_bits(double d)
{
    union { uint64_t u; double d; } v;
    v.d = d;
    return v.u;
}

/* round to nearest, ties to even (IEEE rint in both builds) */
SYN_HD double syn_rint(double x)
{
    return rint(x);
}

/* natural log of a positive normal double: x = m 2^e, m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(s) with s = (m - 1)/(m + 1), |s| < 0.172, 14 series terms. */
SYN_HD double syn_log(double x)
{
    uint64_t b = syn_double_to_bits(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = syn_bits_to_double((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull);
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double term = s;
    double sum = s;
    for (int k = 1; k <= 14; ++k) {
        term = term * s2;
        sum = sum + term / (double)(2 * k + 1);
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

/* sin and cos of 2 pi u (u in turns): reduce to the nearest quarter turn, then Taylor
 * series on |x| <= pi/4 (terms through x^19 / x^20). */
SYN_HD void syn_sincos_turns(double u, double* s_out, double* c_out)
{
    double q = syn_rint(4.0 * u);
    double v = u - 0.25 * q;
    double x = 6.28318530717958647692 * v;
    double x2 = x * x;
    /* sin x = x (1 - x^2/(2*3) (1 - x^2/(4*5) (1 - ...))) */
    double ps = 1.0;
    for (int k = 9; k >= 1; --k) ps = 1.0 - x2 / (double)((2 * k) * (2 * k + 1)) * ps;
    double sn = x * ps;
    /* cos x = 1 - x^2/(1*2) (1 - x^2/(3*4) (1 - ...)) */
    double pc = 1.0;
    for (int k = 10; k >= 1; --k) pc = 1.0 - x2 / (double)((2 * k - 1) * (2 * k)) * pc;
    double cs = pc;
    int qi = (int)((int64_t)q & 3);
    double so, co;
    if (qi == 0) { so = sn; co = cs; }
    else if (qi == 1) { so = cs; co = -sn; }
    else if (qi == 2) { so = -sn; co = -cs; }
    else { so = -cs; co = sn; }
    *s_out = so;
    *c_out = co;
}

/* two independent standard normals (Box-Muller) */
SYN_HD void syn_gauss2(uint32_t w0, uint32_t w1, double* g0, double* g1)
{
    double r = sqrt(-2.0 * syn_log(syn_u01(w0)));
    double s, c;
    syn_sincos_turns(syn_u01(w1), &s, &c);
    *g0 = r * c;
    *g1 = r * s;
}

/* ---------------------------------------------------------------- model pieces */

/* code chip k of code row q: +1 or -1 */
SYN_HD int syn_code_chip(uint64_t seed, int k, int q)
{
    uint32_t w[4];
    syn_draw(seed, (uint32_t)k, (uint32_t)q, SYN_PURPOSE_CODE, w);
    return (w[0] & 1u) ? -1 : 1;
}

/* tone frequency of gate r, uniform in [-0.4, 0.4) cycles per sample */
SYN_HD double syn_tone_freq(uint64_t seed, int r)
{
    uint32_t w[4];
    syn_draw(seed, (uint32_t)r, 0u, SYN_PURPOSE_FREQ, w);
    return 0.8 * syn_u01(w[0]) - 0.4;
}

/* amplitude and phase increment of gate r in IPP p; f_base in cycles per sample, amp the
 * gate's amplitude (tone: |a|; line: rms |a|) */
SYN_HD syn_rp syn_range_params(const syn_cfg* c, double f_base, double amp, int r, int p)
{
    uint32_t w[4];
    syn_draw(c->seed, (uint32_t)r, (uint32_t)p, SYN_PURPOSE_LINE, w);
    double ar, ai, f = f_base;
    if (c->kind == SYN_LINE) {
        double g0, g1;
        syn_gauss2(w[0], w[1], &g0, &g1);
        double sc = amp * 0.70710678118654752440;
        ar = sc * g0;
        ai = sc * g1;
        /* Cauchy jitter hwhm * tan(pi (u - 1/2)): Lorentzian line of half width hwhm */
        double s, co;
        syn_sincos_turns(0.5 * (syn_u01(w[2]) - 0.5), &s, &co);
        double jit = c->hwhm * (s / co);
        if (jit > c->max_jitter) jit = c->max_jitter;
        if (jit < -c->max_jitter) jit = -c->max_jitter;
        f = f_base + jit;
    } else {
        double s, co;
        syn_sincos_turns(syn_u01(w[0]), &s, &co);
        ar = amp * co;
        ai = amp * s;
    }
    syn_rp o;
    o.ar = (float)ar;
    o.ai = (float)ai;
    double fi = syn_rint(f * 4294967296.0);
    o.inc = (uint32_t)(int64_t)fi;
    o.pad_ = 0u;
    return o;
}

/* one entry of the phase table: exp(2 pi i j / 2^16) in float */
SYN_HD void syn_table_entry(int j, float* re, float* im)
{
    double s, c;
    syn_sincos_turns((double)j / (double)SYN_TABLE_SIZE, &s, &c);
    *re = (float)c;
    *im = (float)s;
}

SYN_HD int16_t syn_sat16(double v)
{
    double r = syn_rint(v);
    if (r > 32767.0) r = 32767.0;
    if (r < -32768.0) r = -32768.0;
    return (int16_t)(int32_t)r;
}

/*
 * Sample t of IPP row p.  rp: the row's per-gate parameters [n_ranges];
 * code_row: the +-1 chips of the code used in this row; table: [2 * SYN_TABLE_SIZE].
 */
SYN_HD void syn_sample(const syn_cfg* c, const syn_rp* rp, const int8_t* code_row,
                       const float* table, int64_t t, int p, int16_t* I, int16_t* Q)
{
    float sr = 0.0f, si = 0.0f;
    if (c->kind != SYN_NOISE_ONLY && c->n_ranges > 0) {
        /* gates whose window [s_r, s_r + L) holds t */
        int64_t hi = t - c->range_start;
        if (hi >= 0) {
            int64_t rhi = hi / c->range_step;
            int64_t lo = t - c->range_start - c->code_len + 1;
            int64_t rlo = lo <= 0 ? 0 : (lo + c->range_step - 1) / c->range_step;
            if (rhi > c->n_ranges - 1) rhi = c->n_ranges - 1;
            for (int64_t r = rlo; r <= rhi; ++r) {
                int64_t k = t - (c->range_start + r * c->range_step);
                float e = (float)code_row[k];
                uint32_t ph = rp[r].inc * (uint32_t)t;
                uint32_t j = ph >> (32 - SYN_TABLE_BITS);
                float tc = table[2 * j], ts = table[2 * j + 1];
                float vr = rp[r].ar * tc - rp[r].ai * ts;
                float vi = rp[r].ar * ts + rp[r].ai * tc;
                sr = sr + e * vr;
                si = si + e * vi;
            }
        }
    }
    uint32_t w[4];
    syn_draw(c->seed, (uint32_t)t, (uint32_t)p, SYN_PURPOSE_NOISE, w);
    double g0, g1;
    syn_gauss2(w[0], w[1], &g0, &g1);
    *I = syn_sat16(c->sigma * g0 + (double)sr);
    *Q = syn_sat16(c->sigma * g1 + (double)si);
}

#endif /* ISR_SYNTH_CORE_H */
