// df64.cuh -- double-float arithmetic: a real number as an unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi)/2), about 48 significant bits.
//
// GB300 executes FP64 at about 1/58 of its FP32 rate, while the paper asks
// for 13-15 digit arithmetic (Sec. III.A).  Complex128 tiles are therefore
// computed on the FP32 pipes with the error-free transformations below
// (Knuth's two-sum, Dekker/Kahan two-product via FMA), and converted from and
// to IEEE double at the tile boundary with integer operations only (the
// double<->float conversion instructions run on the FP64 pipe).
//
// The functions compile for the host as well so the conversions and the
// arithmetic can be checked bit by bit on the CPU.
#pragma once

#include <cstdint>
#include <cstring>
#include <cmath>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace qsim {

struct df {
    float h, l;
};

DF_HD uint64_t df_bits64(double d) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    std::memcpy(&b, &d, 8);
    return b;
#endif
}
DF_HD double df_from_bits64(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    std::memcpy(&d, &b, 8);
    return d;
#endif
}
DF_HD uint32_t df_fbits(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
#endif
}
DF_HD float df_ffrom(uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, 4);
    return f;
#endif
}
DF_HD int df_clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
DF_HD int df_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}
DF_HD float df_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

// IEEE double -> double-float by bit manipulation: hi = the top 24
// significand bits (truncated), lo = the next 24 bits of the remainder.
// |d| < 2^-126 (and zero) maps to (0, 0): the absolute error is below 1.2e-38.
// Requires |d| < 2^127 (amplitudes are bounded by 1).
DF_HD df df_from_double(double d) {
    const uint64_t b = df_bits64(d);
    const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
    const uint32_t sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const int eh = e - 896;  // float biased exponent of hi
    df r;
    if (eh <= 0) {
        r.h = 0.0f;
        r.l = 0.0f;
        return r;
    }
    const uint32_t mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    r.h = df_ffrom(sign | ((uint32_t)eh << 23) | mh);
    const uint32_t rem = lo32 & 0x1fffffffu;  // 29 bits, worth rem * 2^(e - 1075)
    const int p = 31 - df_clz32(rem);         // leading one (-1 if rem == 0)
    const int el = p + e - 948;               // float biased exponent of lo
    const uint32_t ml = (p >= 23 ? (rem >> (p - 23)) : (rem << (23 - p))) & 0x7fffffu;
    r.l = (rem != 0u && el > 0) ? df_ffrom(sign | ((uint32_t)el << 23) | ml) : 0.0f;
    return r;
}

// double-float -> IEEE double: the exact sum hi + lo, truncated to 53 bits,
// with integer operations only.  Requires |lo| <= ulp(hi) (normalised pair).
DF_HD double df_to_double(df x) {
    const uint32_t hb = df_fbits(x.h), lb = df_fbits(x.l);
    const int eh = (int)((hb >> 23) & 0xffu);
    if (eh == 0) return 0.0;  // hi = 0 (or float subnormal): the pair is below 1.2e-38
    const int el = (int)((lb >> 23) & 0xffu);
    const uint64_t Mh = (uint64_t)((hb & 0x7fffffu) | 0x800000u) << 29;  // leading one at bit 52
    uint64_t Ml = 0;
    const int sh = eh - el;                                             // lo is sh binades below hi
    if (el != 0 && sh < 53) Ml = ((uint64_t)((lb & 0x7fffffu) | 0x800000u) << 29) >> sh;
    const bool same = ((hb ^ lb) & 0x80000000u) == 0u;
    uint64_t M = same ? Mh + Ml : Mh - Ml;
    int e = eh + 896;  // double biased exponent for a leading one at bit 52
    // a sum can carry into bit 53, a difference can drop the leading one to bit 51
    const int lz = df_clz64(M) - 11;  // 0 if the leading one is at bit 52
    if (lz < 0) {
        M >>= 1;
        e += 1;
    } else if (lz > 0) {
        M <<= lz;
        e -= lz;
    }
    return df_from_bits64((uint64_t)(hb & 0x80000000u) << 32 | (uint64_t)e << 52 | (M & 0xfffffffffffffull));
}

// ---- error-free transformations --------------------------------------------
DF_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}
DF_HD df quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return df{s, b - (s - a)};
}
DF_HD df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, df_fma(a, b, -p)};
}

DF_HD df df_add(df a, df b) {
    df s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return quick_two_sum(s.h, s.l);
}
DF_HD df df_neg(df a) { return df{-a.h, -a.l}; }
DF_HD df df_mul(df a, df b) {
    df p = two_prod(a.h, b.h);
    p.l = df_fma(a.h, b.l, p.l);
    p.l = df_fma(a.l, b.h, p.l);
    return quick_two_sum(p.h, p.l);
}

// Sum of n products a[k] * b[k] with one two-sum chain on the leading parts
// and a plain float sum of all error terms: the building block of a complex
// 2x2 update (n = 2 or 4).  Per product: the rounded head, its exact error
// (FMA) and the two cross terms; per added term one two-sum.
template <int N>
DF_HD df df_dot(const df (&a)[N], const df (&b)[N]) {
    float s = 0.0f, err = 0.0f;
#if defined(__CUDACC__)
#pragma unroll
#endif
    for (int k = 0; k < N; k++) {
        const float p = a[k].h * b[k].h;
        float e = df_fma(a[k].h, b[k].h, -p);
        e = df_fma(a[k].h, b[k].l, e);
        e = df_fma(a[k].l, b[k].h, e);
        if (k == 0) {
            s = p;
            err = e;
        } else {
            const df t = two_sum(s, p);
            s = t.h;
            err += t.l + e;
        }
    }
    return quick_two_sum(s, err);
}

// Complex double-float amplitude.
struct dcx {
    df re, im;
};

// u * a (complex)
DF_HD dcx dcx_mul(const dcx &u, const dcx &a) {
    const df ar[2] = {u.re, df_neg(u.im)}, br[2] = {a.re, a.im};
    const df ai[2] = {u.re, u.im}, bi[2] = {a.im, a.re};
    return dcx{df_dot<2>(ar, br), df_dot<2>(ai, bi)};
}
// u * a + v * b (complex)
DF_HD dcx dcx_mul2(const dcx &u, const dcx &a, const dcx &v, const dcx &b) {
    const df xr[4] = {u.re, df_neg(u.im), v.re, df_neg(v.im)}, yr[4] = {a.re, a.im, b.re, b.im};
    const df xi[4] = {u.re, u.im, v.re, v.im}, yi[4] = {a.im, a.re, b.im, b.re};
    return dcx{df_dot<4>(xr, yr), df_dot<4>(xi, yi)};
}
// real u0 * a + real u1 * b (both matrix entries real)
DF_HD dcx dcx_rmul2(const df &u, const dcx &a, const df &v, const dcx &b) {
    const df xr[2] = {u, v}, yr[2] = {a.re, b.re}, yi[2] = {a.im, b.im};
    return dcx{df_dot<2>(xr, yr), df_dot<2>(xr, yi)};
}

// ---- squared magnitudes (probabilities) ----------------------------------
DF_HD float df_fmaxf(float a, float b) {
#if defined(__CUDA_ARCH__)
    return fmaxf(a, b);
#else
    return std::fmax(a, b);
#endif
}
DF_HD float df_fminf(float a, float b) {
#if defined(__CUDA_ARCH__)
    return fminf(a, b);
#else
    return std::fmin(a, b);
#endif
}
// a + b for a, b >= 0: the heads' exact sum by Fast2Sum with the operands
// ordered by size, the tails added in float, then renormalised.
DF_HD df df_add_pos(df a, df b) {
    const float s = a.h + b.h;
    const float big = df_fmaxf(a.h, b.h), sm = df_fminf(a.h, b.h);
    const float t = (sm - (s - big)) + (a.l + b.l);
    const float h = s + t;
    return df{h, t - (h - s)};
}
// True when |d| >= 2 (biased exponent >= 1024): df_sqmag's fast split does
// not cover such values.
DF_HD bool df_mag_ge2(double d) { return ((uint32_t)(df_bits64(d) >> 32) & 0x40000000u) != 0u; }
// |d| = h + r for |d| < 2: h = the top 24 significand bits (truncated), r2 =
// 2 r with r from the remaining 29 bits rounded to a float; |d| < 2^-126 (and
// zero) gives (0, 0).  Integer operations and one int-to-float conversion.
DF_HD void df_split_mag(double d, float &h, float &r2) {
    const uint64_t b = df_bits64(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    // bits 31..23: the low 9 bits of the biased exponent e, which are e - 512
    // for 512 <= e < 1024; below them the top 23 significand bits
    const uint32_t x = (hi << 3) | (lo >> 29);
    const uint32_t hb = x - 0xC0000000u;  // (e - 896) << 23 | significand
    const bool tiny = (hi & 0x7ff00000u) < (897u << 20);
    const float hexp = df_ffrom(hb & 0x7f800000u);  // 2^(e - 1023)
    h = tiny ? 0.0f : df_ffrom(hb);
    r2 = tiny ? 0.0f : (float)(lo & 0x1fffffffu) * hexp * 0x1p-51f;
}
// re^2 + im^2 as a double-float for |re|, |im| < 2 (df_mag_ge2 false):
// (h + r)^2 = h^2 + r2 (h + r2 / 4) per component, the two h^2 as exact
// products, their sum by ordered Fast2Sum, every smaller term in float.
// Relative error below 2^-44.
DF_HD df df_sqmag(double re, double im) {
    float hr, rr2, hi, ri2;
    df_split_mag(re, hr, rr2);
    df_split_mag(im, hi, ri2);
    const float p1 = hr * hr, e1 = df_fma(hr, hr, -p1);
    const float p2 = hi * hi, e2 = df_fma(hi, hi, -p2);
    const float s = p1 + p2;
    const float big = df_fmaxf(p1, p2), sm = df_fminf(p1, p2);
    float c = (e1 + e2) + (sm - (s - big));
    c = df_fma(rr2, df_fma(0.25f, rr2, hr), c);
    c = df_fma(ri2, df_fma(0.25f, ri2, hi), c);
    const float h = s + c;
    return df{h, c - (h - s)};
}
DF_HD df df_from_double_rn(double d) {
    // for constants built on the host: hi = nearest float, lo = nearest float of the rest
    const float h = (float)d;
    return df{h, (float)(d - (double)h)};
}

}  // namespace qsim
