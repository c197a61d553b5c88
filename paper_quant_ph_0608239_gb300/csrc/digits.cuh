// digits.cuh -- complex128 dense blocks on the bf16 tensor cores: IEEE
// doubles cut into bf16 digit slices whose products the tensor cores sum
// exactly (the Ozaki splitting scheme for error-free matrix products,
// Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012), and its
// tensor-core forms, Mukunoki et al., ISC 2020).
//
// A dense block a' = U a (Sec. III.A's gates multiplied into one 2^k x 2^k
// matrix) is, with complex numbers as real 2x2 blocks, a real product of the
// group's 2K = 2^(k+1) reals with a 2K x 2K matrix.  Every real x of a group
// is written in fixed point against the group's largest exponent e
// (2^e <= max |x| < 2^(e+1)):
//
//     X = x 2^(52 - e),  |X| < 2^53   (bits below 2^0 are truncated),
//     X = sum_{i=0..5} d_i 2^(45 - 9i),  d_i integers in [-256, 256],
//
// six signed base-2^9 digits obtained from the bit fields of X + C with
// C = 256 (2^45 + 2^36 + 2^27 + 2^18 + 2^9 + 1) (field value f, digit
// f - 256), so the split of X is exact.  The matrix entries (|u| <= 1) get
// the same six digits c_j against e = 0.  Slice i holds d_i 2^(-9i) as bf16,
// which is exact: |d_i| <= 256 needs at most 8 significand bits.  Then
//
//     x u = 2^(e - 14) sum_{i,j} d_i c_j 2^(-9(i + j)),
//
// and the tensor cores form the slice products A_i B_j^T (bf16 inputs, exact
// products, FP32 accumulation) grouped by level L = i + j, L <= 5 (21
// products).  Over a row of 2K = 64 products a level sums at most
// (L + 1) 64 2^16 (and level 0 at most 2^18, since |c_0| <= 128 with a unit
// row norm): below 2^24 for L <= 3, so the accumulators of levels 0..3 hold
// their sums exactly; levels 4 and 5 share one FP32 accumulator (their
// rounding is below 2^-50 of the result).  The dropped levels 6..10 and the
// truncation of X bound the error of an output by about 2^-44 of the group's
// largest magnitude (typically 2^-48), the class of the double-float tile
// passes.
//
// The epilogue adds the five accumulators in double-float (two FP32 values,
// Knuth's two-sum), converts the pair to an IEEE double with integer
// operations and scales by 2^(e - 14) through the exponent field.  Doubles
// below 2^-1022 (subnormals) are read as zero.
//
// The functions compile for the host as well, so the split, the exact level
// sums and the combination are checked on the CPU against long double.
#pragma once

#include <cstdint>

#include "df64.cuh"

namespace qsim {

constexpr int kDigits = 6;        // digit slices per real
constexpr int kDigitBits = 9;     // base 2^9, digits in [-256, 256]
constexpr int kDigitLevels = 5;   // accumulators: levels 0, 1, 2, 3 and 4-5
constexpr int kDigitExpShift = 14;  // x u = 2^(e - 14) * (level sums)
constexpr uint64_t kDigitOffset =   // 256 (2^45 + 2^36 + 2^27 + 2^18 + 2^9 + 1)
    (256ull << 45) | (256ull << 36) | (256ull << 27) | (256ull << 18) | (256ull << 9) | 256ull;

// Biased exponent field of a double from its high word (0 for zero and
// subnormals, which the split reads as zero).
DF_HD uint32_t dg_bexp(uint32_t hi) { return (hi >> 20) & 0x7ffu; }

// Fixed-point X + C of one real, the group's largest biased exponent Mg >= the
// real's own (Mg = 0: an all-zero group).  |X| < 2^53; X + C lies in
// [2^44, 2^54 + 2^45).
DF_HD uint64_t dg_fixed(uint32_t hi, uint32_t lo, uint32_t Mg) {
    const uint32_t be = dg_bexp(hi);
    const uint64_t M = be ? ((uint64_t)((hi & 0xfffffu) | 0x100000u) << 32) | lo : 0ull;
    const uint32_t s = Mg - be;  // >= 0
    uint64_t X = s < 64u ? M >> s : 0ull;
    if (hi & 0x80000000u) X = 0ull - X;
    return X + kDigitOffset;
}

// Digit i of a fixed-point value (X + C), as the bf16-exact float
// d_i 2^(-9i).
template <int I>
DF_HD float dg_digit(uint64_t XC) {
    constexpr int pos = 45 - kDigitBits * I;
    const uint32_t f = I == 0 ? (uint32_t)(XC >> 45) : (uint32_t)(XC >> pos) & 511u;
    // float(2^23 + f) by its bit pattern, then one FMA that subtracts
    // 2^23 + 256 and scales by 2^(-9i); every intermediate is exact
    constexpr float sc = 1.0f / (float)(1ull << (kDigitBits * I));
    return df_fma(df_ffrom(0x4b000000u | f), sc, -8388864.0f * sc);
}

// bf16 bit pattern of a float that bf16 holds exactly (the top half).
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

// Sum of the five level accumulators (levels 0..3 exact, level 4-5 rounded)
// times 2^(e - 14), e = Mg - 1023, as an IEEE double.
DF_HD double dg_combine(float a0, float a1, float a2, float a3, float a4, uint32_t Mg) {
    // a0 is an integer and a1 a multiple of 2^-9 with |a1| <= 2^14: either
    // |a0| >= |a1| or the sum is exact, so the quick two-sum is error free
    df s = quick_two_sum(a0, a1);
    df t = two_sum(s.h, a2);
    t.l += s.l;
    s = quick_two_sum(t.h, t.l);
    t = two_sum(s.h, a3);
    t.l += s.l + a4;
    s = quick_two_sum(t.h, t.l);
    if (s.h == 0.0f || Mg == 0u) return 0.0;
    const uint64_t b = df_bits64(df_to_double(s));
    const int e = (int)((b >> 52) & 0x7ffu) + (int)Mg - 1023 - kDigitExpShift;
    if (e <= 0) return 0.0;  // below the normal range: flushed
    return df_from_bits64((b & ~(0x7ffull << 52)) | ((uint64_t)e << 52));
}

// The six digit slices of a matrix entry u, |u| <= 1 (e = 0, Mg = 1023).
DF_HD void dg_split_entry(double u, float (&d)[kDigits]) {
    const uint64_t bits = df_bits64(u);
    const uint64_t XC = dg_fixed((uint32_t)(bits >> 32), (uint32_t)bits, 1023u);
    d[0] = dg_digit<0>(XC);
    d[1] = dg_digit<1>(XC);
    d[2] = dg_digit<2>(XC);
    d[3] = dg_digit<3>(XC);
    d[4] = dg_digit<4>(XC);
    d[5] = dg_digit<5>(XC);
}

// Accumulator of the product of slices i and j.
DF_HD int dg_level_acc(int i, int j) { return i + j < kDigitLevels - 1 ? i + j : kDigitLevels - 1; }

}  // namespace qsim
