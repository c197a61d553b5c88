// digits.cuh -- complex128 dense blocks on the bf16 tensor cores: reals cut
// into bf16 digit slices whose products the tensor cores sum exactly (the
// Ozaki splitting scheme for error-free matrix products: Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59 (2012); its tensor-core forms: Mukunoki et
// al., ISC 2020).
//
// A dense block a' = U a (Sec. III.A's gates multiplied into one 2^k x 2^k
// matrix) is, with complex numbers as real 2x2 blocks, a real product of the
// group's 2K = 2^(k+1) reals with a 2K x 2K matrix.
//
// Digits.  Every real of a group is scaled by 2^-e, e the exponent of the
// group's largest magnitude, so |v'| < 2, and written as six digits on the
// grids w_i = 2^(-7 - 9i):
//
//     v' = sum_{i=0..5} d_i,   d_i = (integer in [-256, 256]) * w_i,
//
// up to a remainder below w_5 / 2.  Every digit is a bf16 number (at most 8
// significand bits).  The matrix entries (|u| <= 1) get six digits c_j on the
// same grids without scaling.  Then a product of slices i and j is an integer
// times 2^(-14 - 9(i + j)), and
//
//     (U a)_r = 2^e sum_L sum_{i + j = L} (A_i B_j^T)_r,   L = 0 .. 5
//
// (21 products).  Over a row of 2K = 64 products a level L sums at most
// (L + 1) 64 2^16 integer units (level 0 at most 2^18, since |c_0| <= 128
// and a unitary row has unit norm): below 2^24 for L <= 3, so the FP32
// accumulators of levels 0..3 hold their sums exactly.  Levels 4 and 5 share
// one accumulator, folded into level 3's before the combination; their
// rounding stays below 2^-50 of the result.  The dropped
// levels 6..10 and the last remainder bound an output's error by about 2^-44
// of the group's largest magnitude (typically 2^-48), the class of the
// double-float tile passes.
//
// The state is read and written in double-float form (hi + lo, two floats):
// the split runs on FP32 additions (round to the grid by adding and
// subtracting 1.5 * 2^23 * w_i, the remainder carried exactly as a pair), the
// accumulators are added in double-float (Knuth's two-sum) and scaled back by
// 2^e.  The first block of a run converts IEEE doubles to this form
// and the last one converts back, with the integer conversions of df64.cuh.
//
// Everything compiles for the host as well, so the split, the exact level
// sums and the combination are checked on the CPU against long double.
#pragma once

#include <cstdint>

#include "df64.cuh"
#include "fpair.cuh"

namespace qsim {

constexpr int kDigits = 6;          // digit slices per real
constexpr int kDigitBits = 9;       // digits are integers in [-256, 256] on their grid
constexpr int kDigitLevels = 5;     // accumulators: levels 0, 1, 2, 3 and 4-5

// ---- matrix entries (host): exact integer digits ---------------------------
// u (|u| < 2) in fixed point X = u 2^52 (truncated toward zero below 2^0),
// X = sum_j c_j 2^(45 - 9j) with c_j in [-256, 256] read from the bit fields
// of X + C, C = 256 (2^45 + 2^36 + 2^27 + 2^18 + 2^9 + 1) (field f, digit
// f - 256); slice j holds c_j 2^(-7 - 9j).
constexpr uint64_t kDigitOffset =
    (256ull << 45) | (256ull << 36) | (256ull << 27) | (256ull << 18) | (256ull << 9) | 256ull;

DF_HD void dg_split_entry(double u, float (&d)[kDigits]) {
    const uint64_t b = df_bits64(u);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t be = (hi >> 20) & 0x7ffu;  // 0: zero or subnormal, read as zero
    const uint64_t M = be ? ((uint64_t)((hi & 0xfffffu) | 0x100000u) << 32) | lo : 0ull;
    const uint32_t s = 1023u - (be < 1023u ? be : 1023u);
    uint64_t X = s < 64u ? M >> s : 0ull;
    if (hi & 0x80000000u) X = 0ull - X;
    const uint64_t XC = X + kDigitOffset;
    for (int j = 0; j < kDigits; j++) {
        const int pos = 45 - kDigitBits * j;
        const uint32_t f = j == 0 ? (uint32_t)(XC >> 45) : (uint32_t)(XC >> pos) & 511u;
        d[j] = (float)((int)f - 256) * df_ffrom((uint32_t)(127 - 7 - kDigitBits * j) << 23);
    }
}

// ---- the state: FP32 digits of double-float values ------------------------
// 2^-e and 2^e for a group whose largest hi has the float exponent field E
// (E = 0: an all-zero group, scales 1 and zero digits).
DF_HD float dg_scale_down(uint32_t E) { return df_ffrom(E ? (254u - E) << 23 : 127u << 23); }
DF_HD float dg_scale_up(uint32_t E) { return df_ffrom(E ? E << 23 : 127u << 23); }

// Digit i of the remainder (rh, rl): round rh + rl to the grid w_i, keep the
// new remainder in rh (exact).
template <int I>
DF_HD float dg_step(float &rh, float rl) {
    constexpr float M = 12582912.0f / (float)(1ull << (7 + kDigitBits * I));  // 1.5 * 2^23 * w_i
    const float s = rh + rl;
    const float d = (s + M) - M;
    if (I < kDigits - 1) rh = rh - d;
    return d;
}

// The six slices of (h + l) * scale, scale = dg_scale_down(E).
DF_HD void dg_split_df(float h, float l, float scale, float (&d)[kDigits]) {
    float rh = h * scale;
    const float rl = l * scale;
    d[0] = dg_step<0>(rh, rl);
    d[1] = dg_step<1>(rh, rl);
    d[2] = dg_step<2>(rh, rl);
    d[3] = dg_step<3>(rh, rl);
    d[4] = dg_step<4>(rh, rl);
    d[5] = dg_step<5>(rh, rl);
}

// The same for the real and imaginary parts of an amplitude at once, in
// packed FP32x2 operations (fpair.cuh: lane by lane the scalar roundings).
template <int I>
DF_HD fpair dg_step2(fpair &rh, fpair rl) {
    constexpr float M = 12582912.0f / (float)(1ull << (7 + kDigitBits * I));
    const fpair Mp = fp_splat(M);
    const fpair s = fp_add(rh, rl);
    const fpair d = fp_sub(fp_add(s, Mp), Mp);
    if (I < kDigits - 1) rh = fp_sub(rh, d);
    return d;
}
DF_HD void dg_split_df2(fpair h, fpair l, float scale, fpair (&d)[kDigits]) {
    const fpair sc = fp_splat(scale);
    fpair rh = fp_mul(h, sc);
    const fpair rl = fp_mul(l, sc);
    d[0] = dg_step2<0>(rh, rl);
    d[1] = dg_step2<1>(rh, rl);
    d[2] = dg_step2<2>(rh, rl);
    d[3] = dg_step2<3>(rh, rl);
    d[4] = dg_step2<4>(rh, rl);
    d[5] = dg_step2<5>(rh, rl);
}

// The accumulators of level 3 (exact) and levels 4-5 folded into one FP32
// value: the rounding is below 2^-24 of level 3, which is itself below 2^-27
// of the result.
DF_HD float dg_fold_high(float a3, float a45) { return a3 + a45; }

// Sum of the level accumulators (levels 0..2 exact, a3 = dg_fold_high of
// levels 3 and 4-5) as a normalised double-float, times scale =
// dg_scale_up(E).
//
// Dekker's fast two-sum (a + b = s + t, s = fl(a + b), t = b - (s - a)) is
// error free whenever a and b can be written as M_a 2^e_a and M_b 2^e_b with
// |M_a|, |M_b| < 2^24 and e_a >= e_b (Boldo and Daumas; Muller et al.,
// Handbook of Floating-Point Arithmetic, Sec. 4.3.1), whatever the
// magnitudes.  Here a0 is a multiple of 2^-14 with |a0| <= 2^4 (2^18 units),
// a1 of 2^-23 below 2^1, a2 of 2^-32 below 2^-8: fl(a0 + a1) is a multiple of
// 2^-23 and fl(of that + a2) one of 2^-32, so e_a >= -23 > -32 = e_b in the
// second step and e_a >= -32 > e_b in the third (|a3| < 2^-16, so its
// exponent is below -39).  The three heads are therefore exact; only the
// two additions of the tails round, below 2^-47 of the result.
DF_HD df dg_combine_df(float a0, float a1, float a2, float a3, float scale) {
    df s = quick_two_sum(a0, a1);
    df t = quick_two_sum(s.h, a2);
    float l = s.l + t.l;
    s = quick_two_sum(t.h, a3);
    l += s.l;
    s = quick_two_sum(s.h, l);
    return df{s.h * scale, s.l * scale};
}

// dg_combine_df for two outputs at once (packed FP32x2): heads in h, tails
// in l.
DF_HD void dg_combine_df2(fpair a0, fpair a1, fpair a2, fpair a3, float scale, fpair &h, fpair &l) {
    auto fast_two_sum = [](fpair a, fpair b, fpair &t) {
        const fpair s = fp_add(a, b);
        t = fp_sub(b, fp_sub(s, a));
        return s;
    };
    fpair l1, l2, l3;
    fpair s = fast_two_sum(a0, a1, l1);
    s = fast_two_sum(s, a2, l2);
    fpair lt = fp_add(l1, l2);
    s = fast_two_sum(s, a3, l3);
    lt = fp_add(lt, l3);
    fpair t;
    s = fast_two_sum(s, lt, t);
    const fpair sc = fp_splat(scale);
    h = fp_mul(s, sc);
    l = fp_mul(t, sc);
}

// bf16 bit pattern of a float that bf16 holds exactly (its top half).
DF_HD uint32_t dg_bf16(float v) { return df_fbits(v) >> 16; }

// Two bf16 values in one 32-bit word: lo in bits 0..15, hi in 16..31 (the
// order of consecutive K elements in a tensor-core operand).
DF_HD uint32_t dg_pack(float lo, float hi) {
#if defined(__CUDA_ARCH__)
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
#else
    return dg_bf16(lo) | (dg_bf16(hi) << 16);
#endif
}

// Accumulator of the product of slices i and j.
DF_HD int dg_level_acc(int i, int j) { return i + j < kDigitLevels - 1 ? i + j : kDigitLevels - 1; }

}  // namespace qsim
