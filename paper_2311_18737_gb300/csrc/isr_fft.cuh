// isr_fft.cuh -- register-resident radix-R DFT building blocks for the fused kernel.
//
// The transform of the paper's Sec. 3.2.2 (a length-nfft forward DFT per decoded window)
// is computed as a Stockham sequence of radix-R passes; each pass applies R-point DFTs
// held entirely in registers.  Every index below is a compile-time constant after
// template expansion, so the arrays live in registers and bit reversal is free.
#pragma once

#include <cstdint>
#include <utility>

namespace isr {

// ---------------------------------------------------------------- compile-time helpers
template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F&& f)
{
    (f(std::integral_constant<int, Is>{}), ...);
}

// f(integral_constant<int, 0>) ... f(integral_constant<int, N-1>)
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f)
{
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

__host__ __device__ constexpr int bitrev(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// Taylor series on |x| <= pi/4, evaluated by the compiler in double.
__host__ __device__ constexpr double ct_sin_small(double x)
{
    double x2 = x * x, p = 1.0;
    for (int k = 10; k >= 1; --k) p = 1.0 - x2 / double((2 * k) * (2 * k + 1)) * p;
    return x * p;
}
__host__ __device__ constexpr double ct_cos_small(double x)
{
    double x2 = x * x, p = 1.0;
    for (int k = 10; k >= 1; --k) p = 1.0 - x2 / double((2 * k - 1) * (2 * k)) * p;
    return p;
}

constexpr double kPi = 3.14159265358979323846;

// cos and sin of 2 pi k / n for integer k and n a power of two (n >= 8), reduced by exact
// octant symmetry before the series.
__host__ __device__ constexpr double ct_cos2pi(int k, int n)
{
    int m = ((k % n) + n) % n;
    int q = (4 * m) / n;           // quadrant
    int rem = m - q * (n / 4);     // 0 <= rem < n/4
    bool flip = 8 * rem > n;       // past the octant: use the complementary angle
    double th = 2.0 * kPi * double(flip ? (n / 4 - rem) : rem) / double(n);
    double c = flip ? ct_sin_small(th) : ct_cos_small(th);
    double s = flip ? ct_cos_small(th) : ct_sin_small(th);
    // rotate (c, s) by q quarter turns
    return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double ct_sin2pi(int k, int n)
{
    int m = ((k % n) + n) % n;
    int q = (4 * m) / n;
    int rem = m - q * (n / 4);
    bool flip = 8 * rem > n;
    double th = 2.0 * kPi * double(flip ? (n / 4 - rem) : rem) / double(n);
    double c = flip ? ct_sin_small(th) : ct_cos_small(th);
    double s = flip ? ct_cos_small(th) : ct_sin_small(th);
    return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// z * exp(-2 pi i I / LEN) with the trivial factors special-cased.
template <int I, int LEN>
__device__ __forceinline__ float2 mul_w(float2 z)
{
    constexpr int i = ((I % LEN) + LEN) % LEN;
    if constexpr (i == 0) {
        return z;
    } else if constexpr (4 * i == LEN) {          // -i
        return make_float2(z.y, -z.x);
    } else if constexpr (2 * i == LEN) {          // -1
        return make_float2(-z.x, -z.y);
    } else if constexpr (4 * i == 3 * LEN) {      // +i
        return make_float2(-z.y, z.x);
    } else if constexpr (8 * i == LEN) {          // (1 - i)/sqrt2
        constexpr float r = 0.70710678118654752440f;
        return make_float2((z.x + z.y) * r, (z.y - z.x) * r);
    } else if constexpr (8 * i == 3 * LEN) {      // (-1 - i)/sqrt2
        constexpr float r = 0.70710678118654752440f;
        return make_float2((z.y - z.x) * r, -(z.x + z.y) * r);
    } else {
        constexpr float c = float(ct_cos2pi(i, LEN));
        constexpr float s = float(ct_sin2pi(i, LEN));
        // (x + iy)(c - is) = (xc + ys) + i(yc - xs)
        return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
    }
}

// One decimation-in-frequency radix-2 stage of sub-length LEN over v[OFF .. OFF+R).
template <int R, int LEN>
__device__ __forceinline__ void dif_stage(float2* v)
{
    constexpr int H = LEN / 2;
    static_for<R / LEN>([&](auto Sb) {
        constexpr int s = decltype(Sb)::value * LEN;
        static_for<H>([&](auto Iv) {
            constexpr int i = decltype(Iv)::value;
            float2 a = v[s + i], b = v[s + i + H];
            v[s + i] = cadd(a, b);
            v[s + i + H] = mul_w<i, LEN>(csub(a, b));
        });
    });
    if constexpr (LEN > 2) dif_stage<R, LEN / 2>(v);
}

// Two DIF radix-2 stages of sub-length LEN and LEN/2 fused (radix 2^2), then the rest.  With
// a[i] = x[i] + x[i+L/2] and d[i] = x[i] - x[i+L/2] (L = LEN, i < L/4) the four quarters are
//   a[i] + a[i+L/4],                (a[i] - a[i+L/4]) W_L^{2i},
//   (d[i] - i d[i+L/4]) W_L^{i},    (d[i] + i d[i+L/4]) W_L^{3i},
// the same values in the same places as two radix-2 stages (the output stays in bit-reversed
// order), with the first stage's twiddles merged into the second: 3 (L/4 - 1) twiddle products
// per block instead of L - 3.
template <int R, int LEN>
__device__ __forceinline__ void dif22_stage(float2* v)
{
    if constexpr (LEN == 2) {
        dif_stage<R, 2>(v);
    } else {
        constexpr int Q = LEN / 4;
        static_for<R / LEN>([&](auto Sb) {
            constexpr int s = decltype(Sb)::value * LEN;
            static_for<Q>([&](auto Iv) {
                constexpr int i = decltype(Iv)::value;
                const float2 x0 = v[s + i], x1 = v[s + i + Q], x2 = v[s + i + 2 * Q], x3 = v[s + i + 3 * Q];
                const float2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
                const float2 d0 = csub(x0, x2), d1 = csub(x1, x3);
                v[s + i] = cadd(a0, a1);
                v[s + i + Q] = mul_w<2 * i, LEN>(csub(a0, a1));
                // d0 - i d1 = (d0.x + d1.y, d0.y - d1.x); d0 + i d1 = (d0.x - d1.y, d0.y + d1.x)
                v[s + i + 2 * Q] = mul_w<i, LEN>(make_float2(d0.x + d1.y, d0.y - d1.x));
                v[s + i + 3 * Q] = mul_w<3 * i, LEN>(make_float2(d0.x - d1.y, d0.y + d1.x));
            });
        });
        if constexpr (LEN > 4) dif22_stage<R, LEN / 4>(v);
    }
}

// In-place R-point forward DFT of v[0..R): afterwards V[q] = v[bitrev(q)].  R22 selects the
// radix-2^2 network (fewer twiddle products, four values live per butterfly group).
template <int R, bool R22 = false>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R > 1) {
        if constexpr (R22) dif22_stage<R, R>(v);
        else dif_stage<R, R>(v);
    }
}

template <int R>
struct BitRev {
    static constexpr int bits = ilog2(R);
    __host__ __device__ static constexpr int at(int q) { return bitrev(q, bits); }
};

// ---------------------------------------------------------------- scaled radix-2^2 DFT
// The same network as dif22_stage, with every non-trivial twiddle product in tangent form:
// z (c - i s) = c (z.x + t z.y, z.y - t z.x) with t = s / c when |c| >= |s|, else
// s (t' z.x + z.y, t' z.y - z.x) with t' = c / s -- two FMAs instead of four instructions --
// and the real factor (c or s) left out of the stored value.  Each value then carries a
// compile-time factor that turns it into the true value; butterflies of values with unequal
// factors add with one FMA by the factor ratio (a plain add where the ratio is +-1).  The
// output X[q] of sdft<R> equals kappa_q * v[bitrev(q)] with kappa_q = ScaleNet<R>::out(q).
namespace sdft_detail {
// factor that tw_mul<I, LEN> leaves out of its result
__host__ __device__ constexpr double tw_factor(int I, int LEN)
{
    const int i = ((I % LEN) + LEN) % LEN;
    if (i == 0 || 4 * i == LEN) return 1.0;      // identity, -i (component swap)
    if (2 * i == LEN || 4 * i == 3 * LEN) return -1.0;   // -1, +i (sign left in the factor)
    const double c = ct_cos2pi(i, LEN), s = ct_sin2pi(i, LEN);
    const double ac = c < 0 ? -c : c, as = s < 0 ? -s : s;
    return ac >= as ? c : s;
}
}  // namespace sdft_detail

template <int R>
struct ScaleNet {
    static constexpr int LEVELS = ilog2(R) / 2 + (ilog2(R) & 1);
    double sc[LEVELS + 1][R];   // factor of v[i] after each level (level 0: the inputs)
    __host__ __device__ constexpr ScaleNet() : sc{}
    {
        for (int i = 0; i < R; ++i) sc[0][i] = 1.0;
        int l = 0;
        for (int LEN = R; LEN >= 2; LEN /= 4, ++l) {
            for (int i = 0; i < R; ++i) sc[l + 1][i] = sc[l][i];
            if (LEN == 2) {
                for (int s = 0; s < R; s += 2) sc[l + 1][s + 1] = sc[l][s];
            } else {
                const int Q = LEN / 4;
                for (int s = 0; s < R; s += LEN)
                    for (int i = 0; i < Q; ++i) {
                        const double s0 = sc[l][s + i];
                        sc[l + 1][s + i] = s0;
                        sc[l + 1][s + i + Q] = s0 * sdft_detail::tw_factor(2 * i, LEN);
                        sc[l + 1][s + i + 2 * Q] = s0 * sdft_detail::tw_factor(i, LEN);
                        sc[l + 1][s + i + 3 * Q] = s0 * sdft_detail::tw_factor(3 * i, LEN);
                    }
            }
        }
    }
    // factor of output X[q] (stored at v[bitrev(q)])
    __host__ __device__ constexpr double out(int q) const { return sc[LEVELS][bitrev(q, ilog2(R))]; }
};

// z (c - i s) for W = exp(-2 pi i I / LEN), up to the factor tw_factor(I, LEN)
template <int I, int LEN>
__device__ __forceinline__ float2 tw_mul(float2 z)
{
    constexpr int i = ((I % LEN) + LEN) % LEN;
    if constexpr (i == 0 || 2 * i == LEN) {
        return z;
    } else if constexpr (4 * i == LEN || 4 * i == 3 * LEN) {
        return make_float2(z.y, -z.x);
    } else {
        constexpr double c = ct_cos2pi(i, LEN), s = ct_sin2pi(i, LEN);
        constexpr bool cform = (c < 0 ? -c : c) >= (s < 0 ? -s : s);
        constexpr float t = cform ? float(s / c) : float(c / s);
        if constexpr (cform) return make_float2(fmaf(t, z.y, z.x), fmaf(-t, z.x, z.y));
        else return make_float2(fmaf(t, z.x, z.y), fmaf(t, z.y, -z.x));
    }
}

template <int R, int LEN, int L>
__device__ __forceinline__ void sdif22_stage(float2* v)
{
    constexpr ScaleNet<R> net{};
    if constexpr (LEN == 2) {
        static_for<R / 2>([&](auto Sb) {
            constexpr int s = 2 * decltype(Sb)::value;
            constexpr float r = float(net.sc[L][s + 1] / net.sc[L][s]);
            const float2 a = v[s], b = v[s + 1];
            v[s] = make_float2(fmaf(r, b.x, a.x), fmaf(r, b.y, a.y));
            v[s + 1] = make_float2(fmaf(-r, b.x, a.x), fmaf(-r, b.y, a.y));
        });
    } else {
        constexpr int Q = LEN / 4;
        static_for<R / LEN>([&](auto Sb) {
            constexpr int s = decltype(Sb)::value * LEN;
            static_for<Q>([&](auto Iv) {
                constexpr int i = decltype(Iv)::value;
                constexpr double s0 = net.sc[L][s + i], s1 = net.sc[L][s + i + Q];
                constexpr float r20 = float(net.sc[L][s + i + 2 * Q] / s0);
                constexpr float r31 = float(net.sc[L][s + i + 3 * Q] / s1);
                constexpr float r10 = float(s1 / s0);
                const float2 x0 = v[s + i], x1 = v[s + i + Q], x2 = v[s + i + 2 * Q], x3 = v[s + i + 3 * Q];
                const float2 a0 = make_float2(fmaf(r20, x2.x, x0.x), fmaf(r20, x2.y, x0.y));
                const float2 d0 = make_float2(fmaf(-r20, x2.x, x0.x), fmaf(-r20, x2.y, x0.y));
                const float2 a1 = make_float2(fmaf(r31, x3.x, x1.x), fmaf(r31, x3.y, x1.y));
                const float2 d1 = make_float2(fmaf(-r31, x3.x, x1.x), fmaf(-r31, x3.y, x1.y));
                v[s + i] = make_float2(fmaf(r10, a1.x, a0.x), fmaf(r10, a1.y, a0.y));
                v[s + i + Q] = tw_mul<2 * i, LEN>(make_float2(fmaf(-r10, a1.x, a0.x), fmaf(-r10, a1.y, a0.y)));
                // d0 - i d1 and d0 + i d1, d1 weighted by r10
                v[s + i + 2 * Q] = tw_mul<i, LEN>(make_float2(fmaf(r10, d1.y, d0.x), fmaf(-r10, d1.x, d0.y)));
                v[s + i + 3 * Q] = tw_mul<3 * i, LEN>(make_float2(fmaf(-r10, d1.y, d0.x), fmaf(r10, d1.x, d0.y)));
            });
        });
        if constexpr (LEN > 4) sdif22_stage<R, LEN / 4, L + 1>(v);
    }
}

// Scaled R-point forward DFT of v[0..R): X[q] = ScaleNet<R>{}.out(q) * v[bitrev(q)].
template <int R>
__device__ __forceinline__ void sdft(float2* v)
{
    if constexpr (R > 1) sdif22_stage<R, R, 0>(v);
}

}  // namespace isr
