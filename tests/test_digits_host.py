"""Digit-slice arithmetic of the complex128 tensor-core blocks, checked on the CPU.

csrc/digits.cuh compiles for the host as well.  A C++ driver takes groups of
64 doubles (in the double-float form the kernel works in) and rows of a 64 x 64
real matrix (the real form of a random 32 x 32 complex unitary), cuts them into
the six bf16 digit slices, forms the 21 slice products level by level the way
the tensor cores do (exact products, FP32 accumulation after every 16-element
K step), combines the five accumulators and compares with the exact dot
product of the original doubles in long double:

  * every digit is an integer in [-256, 256] on its grid and a bf16 number
    (its low 16 bits are zero); the digits rebuild the scaled value to half
    the last grid step, and a matrix entry to 2^-52;
  * the FP32 accumulators of levels 0..3 equal the exact level sums (the
    sums of |products| stay below 2^24), for random and adversarial inputs;
  * the combined result is within 2^-43 of max|x| * ||u_row||_1 of the exact
    dot product (the dropped levels and the fixed-point truncation), and the
    typical error is near 2^-48 of the output's magnitude scale;
  * the combination alone, for accumulators anywhere on their grids within
    their bounds (cancelling ones too), is within 2^-46 of the largest of
    them from their exact sum, as a normalised double-float;
  * the packed (FP32x2) split and combination give the scalar results lane
    by lane (on the CPU both are scalar code: this pins the order of the
    operations; the GPU parity tests pin the packed instructions).
"""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r'''
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <complex>
#include <random>
#include <vector>
#include "digits.cuh"
using namespace qsim;
typedef long double LD;

static std::mt19937_64 g(777);
static std::normal_distribution<double> N01(0.0, 1.0);
static std::uniform_real_distribution<double> U01(0.0, 1.0);

// 32 x 32 complex unitary (Gram-Schmidt of a Gaussian matrix), real form
// B[n][kk]: out_re[r] = sum_c Ure a_re - Uim a_im, out_im[r] = sum_c Uim a_re + Ure a_im
static void rand_unitary_real(std::vector<double> &B, int kind) {
    const int K = 32;
    std::vector<std::complex<double>> Q(K * K);
    if (kind == 1) {  // a permutation with phases +-1, +-i
        std::vector<int> p(K);
        for (int i = 0; i < K; i++) p[i] = i;
        std::shuffle(p.begin(), p.end(), g);
        const std::complex<double> ph[4] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
        for (int r = 0; r < K; r++) Q[r * K + p[r]] = ph[g() & 3];
    } else if (kind == 2) {  // Hadamard^5 (every entry +-2^-2.5)
        for (int r = 0; r < K; r++)
            for (int c = 0; c < K; c++) Q[r * K + c] = (__builtin_popcount(r & c) & 1 ? -1.0 : 1.0) / std::sqrt(32.0);
    } else {
        for (auto &z : Q) z = {N01(g), N01(g)};
        for (int r = 0; r < K; r++) {
            for (int q = 0; q < r; q++) {
                std::complex<double> d = 0;
                for (int c = 0; c < K; c++) d += std::conj(Q[q * K + c]) * Q[r * K + c];
                for (int c = 0; c < K; c++) Q[r * K + c] -= d * Q[q * K + c];
            }
            double nn = 0;
            for (int c = 0; c < K; c++) nn += std::norm(Q[r * K + c]);
            for (int c = 0; c < K; c++) Q[r * K + c] /= std::sqrt(nn);
        }
    }
    B.assign(64 * 64, 0.0);
    for (int r = 0; r < K; r++)
        for (int c = 0; c < K; c++) {
            const double ur = Q[r * K + c].real(), ui = Q[r * K + c].imag();
            B[(2 * r) * 64 + 2 * c] = ur;
            B[(2 * r) * 64 + 2 * c + 1] = -ui;
            B[(2 * r + 1) * 64 + 2 * c] = ui;
            B[(2 * r + 1) * 64 + 2 * c + 1] = ur;
        }
}

static void group(std::vector<double> &x, int kind) {
    x.assign(64, 0.0);
    const int e = -(int)(U01(g) * 40);
    for (int k = 0; k < 64; k++) {
        double v = N01(g) * std::ldexp(1.0, e);
        if (kind == 1) v = std::ldexp(1.0, e) * (2.0 - std::ldexp(1.0, -52)) * ((k * 7 % 3) ? 1 : -1);  // max mantissas
        if (kind == 2) v = (k == 5 ? 1.0 : std::ldexp(N01(g), -70)) * std::ldexp(1.0, e);  // one large, rest tiny
        if (kind == 3) v = (k % 4 == 0) ? 0.0 : (k % 4 == 1 ? -0.0 : v);                   // zeros
        if (kind == 4) v = std::ldexp(1.0, e - (k % 9)) * ((k & 1) ? -1 : 1);               // powers of two
        if (kind == 5) v = 0.0;                                                             // all zero
        x[k] = v;
    }
}

int main() {
    int bad_exact = 0, bad_slice = 0, bad_bound = 0, bad_err = 0, bad_pair = 0;
    double worst = 0.0, sum_typ = 0.0;
    long cnt = 0;
    std::vector<double> B, x;
    for (int trial = 0; trial < 3000; trial++) {
        rand_unitary_real(B, trial % 7 == 3 ? 1 : trial % 7 == 5 ? 2 : 0);
        group(x, trial % 11 < 6 ? 0 : trial % 11 - 5);
        // the group in double-float form (the first block's conversion), its
        // largest hi exponent, and the slices
        df v[64];
        uint32_t E = 0;
        for (int k = 0; k < 64; k++) {
            v[k] = df_from_double(x[k]);
            const uint32_t ek = (df_fbits(v[k].h) >> 23) & 0xffu;
            if (ek > E) E = ek;
        }
        const float sd = dg_scale_down(E), su = dg_scale_up(E);
        float A[kDigits][64], Bd[kDigits][64][64];
        for (int k = 0; k < 64; k++) {
            float d[kDigits];
            dg_split_df(v[k].h, v[k].l, sd, d);
            {  // the packed split of (this value, the next one) against the scalar one
                const int k2 = (k + 1) % 64;
                fpair dp[kDigits];
                float d2[kDigits];
                dg_split_df2(fpair{v[k].h, v[k2].h}, fpair{v[k].l, v[k2].l}, sd, dp);
                dg_split_df(v[k2].h, v[k2].l, sd, d2);
                for (int i = 0; i < kDigits; i++)
                    if (dp[i].x != d[i] || dp[i].y != d2[i]) bad_pair++;
            }
            LD sum = 0;
            for (int i = 0; i < kDigits; i++) {
                A[i][k] = d[i];
                const LD w = std::ldexp((LD)1, -7 - kDigitBits * i);
                const LD q = (LD)d[i] / w;
                if (q != std::floor(q) || std::fabs(q) > 256) bad_slice++;
                if ((df_fbits(d[i]) & 0xffffu) != 0u) bad_slice++;
                sum += d[i];
            }
            // the digits rebuild the scaled value up to half the last grid step
            const LD exact = ((LD)v[k].h + (LD)v[k].l) * (LD)sd;
            if (std::fabs(sum - exact) > std::ldexp((LD)1, -53) + std::ldexp((LD)1, -66)) bad_slice++;
        }
        for (int n = 0; n < 64; n++)
            for (int k = 0; k < 64; k++) {
                float d[kDigits];
                dg_split_entry(B[n * 64 + k], d);
                LD sum = 0;
                for (int j = 0; j < kDigits; j++) {
                    Bd[j][n][k] = d[j];
                    sum += d[j];
                    if ((df_fbits(d[j]) & 0xffffu) != 0u) bad_slice++;
                }
                if (std::fabs(sum - (LD)B[n * 64 + k]) > std::ldexp((LD)1, -52)) bad_slice++;
            }
        for (int n = 0; n < 64; n++) {
            // the tensor cores: 4 K steps of 16, exact products, FP32 accumulation
            float acc[kDigitLevels] = {0, 0, 0, 0, 0};
            LD exact[kDigitLevels] = {0, 0, 0, 0, 0}, mag[kDigitLevels] = {0, 0, 0, 0, 0};
            for (int ks = 0; ks < 4; ks++)
                for (int i = 0; i < kDigits; i++)
                    for (int j = 0; i + j < kDigits; j++) {
                        const int L = dg_level_acc(i, j);
                        LD part = 0;
                        for (int k = 16 * ks; k < 16 * ks + 16; k++) {
                            const LD p = (LD)A[i][k] * (LD)Bd[j][n][k];
                            part += p;
                            mag[L] += std::fabs(p);
                        }
                        exact[L] += part;
                        acc[L] = (float)((LD)acc[L] + part);
                    }
            for (int L = 0; L < 4; L++) {
                if ((LD)acc[L] != exact[L]) bad_exact++;
                // in integer units of the level, 2^(-14 - 9L)
                if (mag[L] * std::ldexp((LD)1, 14 + 9 * L) >= std::ldexp((LD)1, 24)) bad_bound++;
            }
            const df got = dg_combine_df(acc[0], acc[1], acc[2], dg_fold_high(acc[3], acc[4]), su);
            LD ref = 0, scale = 0, xmax = 0;
            for (int k = 0; k < 64; k++) {
                ref += (LD)x[k] * (LD)B[n * 64 + k];
                scale += std::fabs((LD)B[n * 64 + k]);
                if (std::fabs((LD)x[k]) > xmax) xmax = std::fabs((LD)x[k]);
            }
            const LD g = (LD)got.h + (LD)got.l;
            if (xmax == 0) {
                if (g != 0) bad_err++;
                continue;
            }
            if (std::fabs((LD)got.l) > std::fabs((LD)got.h) * std::ldexp((LD)1, -23)) bad_err++;  // normalised
            const double e = (double)(std::fabs(g - ref) / (xmax * scale));
            if (e > worst) worst = e;
            sum_typ += e;
            cnt++;
            if (e > std::ldexp(1.0, -43)) bad_err++;
        }
    }
    // the combination alone: accumulators anywhere on their grids within their
    // bounds (cancellations included), against the exact sum in long double
    int bad_comb = 0;  // (bad_pair: the packed forms differ from the scalar ones)
    std::uniform_int_distribution<int64_t> I0(-(1ll << 18), 1ll << 18), I1(-(1ll << 23), 1ll << 23),
        I2(-(3ll << 22), 3ll << 22), I3(-(1ll << 24) + 1, (1ll << 24) - 1);
    for (int trial = 0; trial < 2000000; trial++) {
        int64_t m0 = I0(g), m1 = I1(g), m2 = I2(g), m3 = I3(g);
        const int shape = trial % 8;
        if (shape == 1) m1 = -m0 * 512 + (m1 >> 12);  // a1 cancels a0 to a few units
        if (shape == 2) { m0 = 0; m1 = 0; }
        if (shape == 3) { m0 = 0; m1 >>= 16; m2 = -m1 * 512 + (m2 >> 14); }
        if (shape == 4) { m1 = -m0 * 512; m2 = 0; }
        if (m1 > (1ll << 23)) m1 = 1ll << 23;
        if (m1 < -(1ll << 23)) m1 = -(1ll << 23);
        if (m2 > (3ll << 22)) m2 = 3ll << 22;
        if (m2 < -(3ll << 22)) m2 = -(3ll << 22);
        const float a0 = std::ldexp((float)m0, -14), a1 = std::ldexp((float)m1, -23), a2 = std::ldexp((float)m2, -32);
        // a3: level 3 folded with a small rounded level 4-5 term
        const float a3 = (float)(std::ldexp((double)m3, -41) + std::ldexp(N01(g), -50));
        const df r = dg_combine_df(a0, a1, a2, a3, 1.0f);
        {  // the packed form, with the lanes swapped in the second output
            fpair h, l;
            dg_combine_df2(fpair{a0, a1}, fpair{a1, a0}, fpair{a2, a2}, fpair{a3, a3}, 1.0f, h, l);
            const df r2 = dg_combine_df(a1, a0, a2, a3, 1.0f);
            if (h.x != r.h || l.x != r.l || h.y != r2.h || l.y != r2.l) bad_pair++;
        }
        const LD exact = (LD)a0 + (LD)a1 + (LD)a2 + (LD)a3;
        const LD mag = std::max(std::max(std::fabs((LD)a0), std::fabs((LD)a1)), std::max(std::fabs((LD)a2), std::fabs((LD)a3)));
        if (std::fabs((LD)r.h + (LD)r.l - exact) > mag * std::ldexp((LD)1, -46)) bad_comb++;
        if (std::fabs((LD)r.l) > std::fabs((LD)r.h) * std::ldexp((LD)1, -24)) bad_comb++;
    }
    std::printf("%d %d %d %d %.3e %.3e %d %d\n", bad_exact, bad_slice, bad_bound, bad_err, worst, sum_typ / cnt, bad_comb,
                bad_pair);
    return 0;
}
'''


def test_digit_slices_exact_levels_and_combination():
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "drv.cpp")
        exe = os.path.join(tmp, "drv")
        open(src, "w").write(DRIVER)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc"),
                               "-o", exe, src])
        out = subprocess.check_output([exe], timeout=600).decode().split()
    bad_exact, bad_slice, bad_bound, bad_err = (int(v) for v in out[:4])
    worst, mean = float(out[4]), float(out[5])
    assert int(out[6]) == 0, out  # the combination alone
    assert int(out[7]) == 0, out  # packed FP32x2 forms = scalar forms
    print("worst %.3e (2^%.1f), mean %.3e (2^%.1f)" % (worst, __import__("math").log2(worst or 1e-300),
                                                        mean, __import__("math").log2(mean or 1e-300)))
    assert bad_slice == 0, out
    assert bad_bound == 0 and bad_exact == 0, out
    assert bad_err == 0 and worst <= 2.0 ** -43, out
    assert mean <= 2.0 ** -47, out
