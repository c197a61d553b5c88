"""Double-float arithmetic of the complex128 tile kernel, checked on the CPU.

csrc/df64.cuh compiles for the host as well; a small C++ driver feeds it
random doubles and compares against long double references:
  * double -> (hi, lo) by bit manipulation: |hi + lo - d| <= 2^-47 |d|
    (plus 2^-125 absolute where the low word underflows the float range);
  * (hi, lo) -> double by integer merging: within 1 ulp of the exact sum;
  * the complex 2x2 row u a + v b: relative error <= 2^-44;
  * the unscaled butterfly (a0 + a1, a0 - a1) of Hadamard-type gates:
    relative error <= 2^-46 of |a0| + |a1| per component.
"""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <random>
#include "df64.cuh"
using namespace qsim;
static long double ld(df x) { return (long double)x.h + (long double)x.l; }
int main() {
    std::mt19937_64 g(12345);
    std::uniform_real_distribution<double> U(-1.0, 1.0), E(-120.0, 0.0);
    int bad = 0;
    double worst_split = 0, worst_join = 0, worst_dot = 0;
    for (int i = 0; i < 200000; i++) {
        double d = U(g) * std::ldexp(1.0, (int)E(g));
        if (i % 97 == 0) d = 0.0;
        df x = df_from_double(d);
        long double err = fabsl(ld(x) - (long double)d);
        double rel = std::fabs(d) > std::ldexp(1.0, -79) ? (double)(err / fabsl((long double)d)) : 0.0;
        if (rel > worst_split) worst_split = rel;
        // below 2^-79 the low word leaves the float range and is flushed:
        // an absolute error under 2^-125, negligible next to any tolerance
        if ((double)err > std::ldexp(std::fabs(d), -47) + std::ldexp(1.0, -125)) bad++;
        if (std::fabs(x.l) > std::fabs(x.h) * std::ldexp(1.0, -23)) bad++;
        double back = df_to_double(x);
        long double exact = ld(x);
        double ulp = exact != 0 ? std::ldexp(1.0, std::ilogb((double)exact) - 52) : 0;
        double dj = (double)fabsl((long double)back - exact);
        if (ulp > 0 && dj / ulp > worst_join) worst_join = dj / ulp;
        if (dj > ulp) bad++;
    }
    // normalised pairs from arithmetic, including opposite-sign lo parts
    for (int i = 0; i < 200000; i++) {
        df a = df_from_double(U(g)), b = df_from_double(U(g) * 1e-3);
        df s = df_add(a, df_neg(b));
        double back = df_to_double(s);
        long double exact = ld(s);
        double ulp = exact != 0 ? std::ldexp(1.0, std::ilogb((double)exact) - 52) : 0;
        if ((double)fabsl((long double)back - exact) > ulp) bad++;
    }
    for (int i = 0; i < 100000; i++) {
        double ur = U(g), ui = U(g), vr = U(g), vi = U(g), ar = U(g), ai = U(g), br = U(g), bi = U(g);
        dcx u{df_from_double(ur), df_from_double(ui)}, v{df_from_double(vr), df_from_double(vi)};
        dcx a{df_from_double(ar), df_from_double(ai)}, b{df_from_double(br), df_from_double(bi)};
        dcx r = dcx_mul2(u, a, v, b);
        // reference from the same (rounded) inputs in long double
        long double Ur = ld(u.re), Ui = ld(u.im), Vr = ld(v.re), Vi = ld(v.im);
        long double Ar = ld(a.re), Ai = ld(a.im), Br = ld(b.re), Bi = ld(b.im);
        long double xr = Ur * Ar - Ui * Ai + Vr * Br - Vi * Bi;
        long double xi = Ur * Ai + Ui * Ar + Vr * Bi + Vi * Br;
        long double scale = fabsl(Ur * Ar) + fabsl(Ui * Ai) + fabsl(Vr * Br) + fabsl(Vi * Bi) +
                            fabsl(Ur * Ai) + fabsl(Ui * Ar) + fabsl(Vr * Bi) + fabsl(Vi * Br);
        double e = (double)((fabsl(ld(r.re) - xr) + fabsl(ld(r.im) - xi)) / scale);
        if (e > worst_dot) worst_dot = e;
        if (e > std::ldexp(1.0, -44)) bad++;
        dcx m = dcx_mul(u, a);
        long double mr = Ur * Ar - Ui * Ai, mi = Ur * Ai + Ui * Ar;
        long double ms = fabsl(Ur * Ar) + fabsl(Ui * Ai) + fabsl(Ur * Ai) + fabsl(Ui * Ar);
        if ((double)((fabsl(ld(m.re) - mr) + fabsl(ld(m.im) - mi)) / ms) > std::ldexp(1.0, -44)) bad++;
    }
    // the unscaled butterfly of a Hadamard-type gate: (a0 + a1, a0 - a1) by
    // double-float additions, relative to |a0| + |a1| per component
    for (int i = 0; i < 200000; i++) {
        const double e0 = E(g) / 4, e1 = E(g) / 4;
        dcx a{df_from_double(U(g) * std::ldexp(1.0, (int)e0)), df_from_double(U(g) * std::ldexp(1.0, (int)e0))};
        dcx b{df_from_double(U(g) * std::ldexp(1.0, (int)e1)), df_from_double(U(g) * std::ldexp(1.0, (int)e1))};
        const df s_re = df_add(a.re, b.re), s_im = df_add(a.im, b.im);
        const df d_re = df_add(a.re, df_neg(b.re)), d_im = df_add(a.im, df_neg(b.im));
        const long double pairs[4][3] = {{ld(s_re), ld(a.re) + ld(b.re), fabsl(ld(a.re)) + fabsl(ld(b.re))},
                                         {ld(s_im), ld(a.im) + ld(b.im), fabsl(ld(a.im)) + fabsl(ld(b.im))},
                                         {ld(d_re), ld(a.re) - ld(b.re), fabsl(ld(a.re)) + fabsl(ld(b.re))},
                                         {ld(d_im), ld(a.im) - ld(b.im), fabsl(ld(a.im)) + fabsl(ld(b.im))}};
        for (const auto &p : pairs)
            if (p[2] > 0 && (double)(fabsl(p[0] - p[1]) / p[2]) > std::ldexp(1.0, -46)) bad++;
    }
    std::printf("%d %.3e %.3e %.3e\n", bad, worst_split, worst_join, worst_dot);
    return 0;
}
'''


def test_double_float_conversions_and_arithmetic():
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "drv.cpp")
        exe = os.path.join(tmp, "drv")
        open(src, "w").write(DRIVER)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc"),
                               "-o", exe, src])
        out = subprocess.check_output([exe]).decode().split()
    bad, split, join, dot = int(out[0]), float(out[1]), float(out[2]), float(out[3])
    assert bad == 0, out
    assert split <= 2.0 ** -47 and join <= 1.0 and dot <= 2.0 ** -44


SQMAG_DRIVER = r'''
#include <cstdio>
#include <cmath>
#include <random>
#include "df64.cuh"
using namespace qsim;
static long double ld(df x) { return (long double)x.h + (long double)x.l; }
int main() {
    std::mt19937_64 g(777);
    std::uniform_real_distribution<double> U(-1.0, 1.0), E(-140.0, 1.0);
    int bad = 0;
    double worst = 0, worst_add = 0;
    for (int i = 0; i < 400000; i++) {
        double re = U(g) * std::ldexp(1.0, (int)E(g)), im = U(g) * std::ldexp(1.0, (int)E(g));
        if (i % 53 == 0) re = 0.0;
        if (i % 71 == 0) im = -0.0;
        if (i % 89 == 0) im = std::ldexp(U(g), -1000);  // far below the float range
        if (i % 101 == 0) re = std::nextafter(2.0, 0.0);  // the largest fast-path magnitude
        if (df_mag_ge2(re) || df_mag_ge2(im)) { bad++; continue; }
        const df p = df_sqmag(re, im);
        const long double ex = (long double)re * re + (long double)im * im;
        const long double err = fabsl(ld(p) - ex);
        // relative 2^-44, plus 2^-120 absolute where the squares leave the float range
        if ((double)err > std::ldexp((double)ex, -44) + std::ldexp(1.0, -120)) bad++;
        if (ex > std::ldexp(1.0, -100) && (double)(err / ex) > worst) worst = (double)(err / ex);
        if (std::fabs(p.l) > std::fabs(p.h) * std::ldexp(1.0, -23)) bad++;
        if (p.h < 0.0f) bad++;
    }
    // the magnitude test of the fast split
    const double big[] = {2.0, -2.0, 3.5, 1e300, -1e20};
    for (double d : big) if (!df_mag_ge2(d)) bad++;
    const double small[] = {0.0, -0.0, 1.0, -1.999, 1e-300, std::nextafter(2.0, 0.0)};
    for (double d : small) if (df_mag_ge2(d)) bad++;
    // sums of non-negative double-floats: 32 terms of mixed sizes
    for (int i = 0; i < 50000; i++) {
        df s{0.0f, 0.0f};
        long double ex = 0;
        for (int k = 0; k < 32; k++) {
            const double v = std::fabs(U(g)) * std::ldexp(1.0, (int)(E(g) / 8));
            const df t = df_sqmag(v, 0.0);
            s = df_add_pos(s, t);
            ex += ld(t);
        }
        const double rel = (double)(fabsl(ld(s) - ex) / ex);
        if (rel > worst_add) worst_add = rel;
        if (rel > 32 * std::ldexp(1.0, -47)) bad++;
        if (std::fabs(s.l) > std::fabs(s.h) * std::ldexp(1.0, -23)) bad++;
    }
    std::printf("%d %.3e %.3e\n", bad, worst, worst_add);
    return 0;
}
'''


def test_squared_magnitudes_and_positive_sums():
    """The complex128 marginals' arithmetic (k_reduce.cu): re^2 + im^2 as a
    double-float from the IEEE bits (relative error <= 2^-44), the |d| >= 2
    test that sends values to the FP64 branch, and sums of non-negative
    double-floats (32 terms within 32 * 2^-47), against long double."""
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "sq.cpp")
        exe = os.path.join(tmp, "sq")
        open(src, "w").write(SQMAG_DRIVER)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc"),
                               "-o", exe, src])
        out = subprocess.check_output([exe]).decode().split()
    bad, worst, worst_add = int(out[0]), float(out[1]), float(out[2])
    assert bad == 0, out
    assert worst <= 2.0 ** -44 and worst_add <= 32 * 2.0 ** -47, out
