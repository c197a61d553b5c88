"""Thread and shared-memory layout of the interchange pass, checked on the CPU.

csrc/perm_layout.hpp is host code.  A C++ driver fills the layout for many
pair sets and tile shapes and walks the kernel's index arithmetic for every
thread and group of a tile, the way k_permute.cu does it:

  * the (group, lane) -> u map covers the tile exactly once;
  * the read offset of pi(u) and the store offset of u split into a lane part
    and a group part (the kernel adds the two), and the read offset is where
    the bulk copy put element pi(u); runs do not overlap, start 16-byte
    aligned and stay inside the stage;
  * every 32-byte sector a warp store touches is written whole (for runs of
    at least 32 bytes);
  * when every pair crosses between the run bits and the run-selecting bits
    (or lies among the latter), the lanes one shared-memory wavefront serves
    (8 for 16-byte elements, 16 for 8-byte) read distinct 4-byte bank words:
    no bank conflicts; other pair sets are counted, not asserted.
"""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>
#include "perm_layout.hpp"
using namespace qsim;

static std::mt19937 rng(4242);

struct Res { long bad_cover = 0, bad_split = 0, bad_place = 0, bad_sector = 0, bad_bank = 0; long cases = 0;
             long other_conflict_cases = 0, other_cases = 0; };

static uint32_t pi(const PermPairs &pp, uint32_t u) {
    for (int k = 0; k < pp.K; k++) {
        const uint32_t t = ((u >> pp.lo[k]) ^ (u >> pp.hi[k])) & 1u;
        u ^= (t << pp.lo[k]) | (t << pp.hi[k]);
    }
    return u;
}

static void check(int E, int L, int H, PermPairs pp, bool crossing, Res &res) {
    const int T = L + H;
    perm_layout(L, H, E, pp);
    res.cases++;
    const uint32_t TS = 1u << T, emask = (1u << L) - 1u, nruns = 1u << H;
    auto run_pos = [&](uint32_t j) {
        uint32_t skew = 0;
        for (int k = 0; k < H; k++) if (pp.skew[k] >= 0) skew += ((j >> k) & 1u) << pp.skew[k];
        return j * pp.run_stride + 16u * skew;
    };
    // a stand-in for the state offsets of the runs: run bit k at state bit 20 + 3k
    auto run_off = [&](uint32_t j) { uint64_t o = 0; for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << (20 + 3 * k); return o; };
    auto read_off = [&](uint32_t v) { return run_pos(v >> L) + (v & emask) * (uint32_t)E; };
    auto store_off = [&](uint32_t u) { return run_off(u >> L) | (uint64_t)(u & emask); };
    // placement of the runs in a stage
    if (pp.run_stride % 128u) res.bad_place++;
    for (uint32_t j = 0; j < nruns; j++) {
        const uint32_t p = run_pos(j);
        if (p % 16u) res.bad_place++;
        if (p < j * pp.run_stride || p + ((uint32_t)E << L) > (j + 1) * pp.run_stride) res.bad_place++;
    }
    uint32_t lanemask = 0;
    std::set<int> lb;
    for (int i = 0; i < kPermLaneBits; i++) { if (pp.lane[i] < 0 || pp.lane[i] >= T) res.bad_cover++; lb.insert(pp.lane[i]); lanemask |= 1u << pp.lane[i]; }
    if ((int)lb.size() != kPermLaneBits) res.bad_cover++;
    std::vector<int> seen(TS, 0);
    long conflicts = 0;
    const uint32_t ngrp = TS >> 5;
    for (uint32_t r = 0; r < ngrp; r++) {
        uint32_t ur = 0, rb = r;
        for (int t = 0; t < T; t++) if (!((lanemask >> t) & 1u)) { ur |= (rb & 1u) << t; rb >>= 1; }
        std::vector<uint64_t> st(32);
        std::vector<uint32_t> rd(32);
        for (int l = 0; l < 32; l++) {
            uint32_t ul = 0;
            for (int i = 0; i < kPermLaneBits; i++) ul |= (uint32_t)((l >> i) & 1) << pp.lane[i];
            const uint32_t u = ul | ur;
            if (ul & ur) res.bad_cover++;
            seen[u]++;
            const uint32_t v = pi(pp, u);
            if (read_off(pi(pp, ul)) + read_off(pi(pp, ur)) != read_off(v)) res.bad_split++;
            if ((store_off(ul) | store_off(ur)) != store_off(u)) res.bad_split++;
            rd[l] = read_off(v);
            st[l] = store_off(u) * (uint64_t)E;
        }
        // whole sectors (a sector spans state bits 0..1 of 8-byte elements:
        // both inside a run when L >= 2)
        if (E == 16 || L >= 2) {
            std::set<uint64_t> bytes;
            for (int l = 0; l < 32; l++) for (int b = 0; b < E; b++) bytes.insert(st[l] + b);
            for (int l = 0; l < 32; l++) {
                const uint64_t s0 = st[l] & ~31ull;
                for (uint64_t b = s0; b < s0 + 32; b++) if (!bytes.count(b)) { res.bad_sector++; break; }
            }
        }
        // bank words per wavefront
        const int wl = E == 16 ? 8 : 16;
        for (int w0 = 0; w0 < 32; w0 += wl) {
            std::set<uint32_t> words;
            for (int l = w0; l < w0 + wl; l++) words.insert((rd[l] / (uint32_t)E) % (128u / (uint32_t)E));
            if ((int)words.size() != wl) conflicts++;
        }
    }
    for (uint32_t u = 0; u < TS; u++) if (seen[u] != 1) { res.bad_cover++; break; }
    if (crossing) { if (conflicts) res.bad_bank++; }
    else { res.other_cases++; if (conflicts) res.other_conflict_cases++; }
}

int main() {
    Res res;
    for (int E : {8, 16}) {
        const int Tmax = E == 8 ? 11 : 10;
        for (int trial = 0; trial < 1500; trial++) {
            const int T = 8 + (int)(rng() % (Tmax - 7));
            PermPairs pp{};
            const int kind = trial % 3;
            if (kind == 0) {  // low bits with the highest ones, the run length the host picks
                const int K = 2 + (int)(rng() % 3);
                pp.K = K;
                for (int k = 0; k < K; k++) { pp.lo[k] = (int8_t)k; pp.hi[k] = (int8_t)(T - 1 - k); }
                check(E, T - K, K, pp, true, res);
            } else if (kind == 1) {  // crossing pairs at random places
                const int H = 2 + (int)(rng() % 7), L = T - H;
                if (L < 1) continue;
                const int K = 1 + (int)(rng() % std::min(std::min(H, L), kMaxPermPairs));
                std::vector<int> lows, highs;
                for (int t = 0; t < L; t++) lows.push_back(t);
                for (int t = L; t < T; t++) highs.push_back(t);
                std::shuffle(lows.begin(), lows.end(), rng);
                std::shuffle(highs.begin(), highs.end(), rng);
                pp.K = K;
                for (int k = 0; k < K; k++) {
                    pp.lo[k] = (int8_t)lows[k];
                    pp.hi[k] = (int8_t)highs[k];
                    if (rng() & 1) std::swap(pp.lo[k], pp.hi[k]);
                }
                check(E, L, H, pp, true, res);
            } else {  // any pairs; the run length as the host picks it
                const int K = 1 + (int)(rng() % kMaxPermPairs);
                std::vector<int> bits;
                for (int t = 0; t < T; t++) bits.push_back(t);
                std::shuffle(bits.begin(), bits.end(), rng);
                if (2 * K > T) continue;
                pp.K = K;
                for (int k = 0; k < K; k++) { pp.lo[k] = (int8_t)bits[2 * k]; pp.hi[k] = (int8_t)bits[2 * k + 1]; }
                int L = T;
                auto above = [&](int l) { int a = 0; for (int k = 0; k < K; k++) a += (pp.lo[k] >= l) + (pp.hi[k] >= l); return a; };
                while (above(L) > T - L && L > 1) L--;
                if (T - L > kPermMaxH) continue;
                bool cross = true;
                for (int k = 0; k < K; k++) if (pp.lo[k] < L && pp.hi[k] < L) cross = false;
                check(E, L, T - L, pp, cross, res);
            }
        }
    }
    std::printf("%ld %ld %ld %ld %ld %ld %ld %ld\n", res.bad_cover, res.bad_split, res.bad_place, res.bad_sector,
                res.bad_bank, res.cases, res.other_conflict_cases, res.other_cases);
    return 0;
}
'''


def test_interchange_layout():
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "drv.cpp")
        exe = os.path.join(tmp, "drv")
        open(src, "w").write(DRIVER.replace("#include <cstdlib>", "#include <cstdlib>\n#include <algorithm>"))
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-I",
                               os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc"), "-o", exe, src])
        out = subprocess.check_output([exe], timeout=600).decode().split()
    bad_cover, bad_split, bad_place, bad_sector, bad_bank, cases, other_conf, other = (int(v) for v in out)
    print("cases %d; in-run pair sets with conflicts %d of %d" % (cases, other_conf, other))
    assert cases > 2000
    assert bad_cover == 0 and bad_split == 0 and bad_place == 0, out
    assert bad_sector == 0, out
    assert bad_bank == 0, out
