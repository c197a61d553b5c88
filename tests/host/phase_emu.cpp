// Host emulation of a tensor-core plan with phase passes: reads n, k, the
// run length, the precision (0: complex64, 1: complex128), the gate list
// (qsim_gate records) and a state (complex128) on stdin; plans with
// plan_fused_phases (planner.cpp); applies the dense blocks (their FP64
// matrices) and the phase passes the way k_phase.cu evaluates them (complex64:
// the rounded top 32 bits of each entry summed mod 2^32; complex128: the
// 64-bit entries summed mod 2^64; the angle from the sum); writes the state
// and (blocks, phase passes, gates in phase passes, plain block count).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../paper_quant_ph_0608239_gb300/csrc/planner.hpp"

using namespace qsim;
typedef std::complex<double> cd;

static bool rd(void *p, size_t n) { return fread(p, 1, n, stdin) == n; }

int main() {
    int32_t hdr[4];
    uint64_t ng;
    if (!rd(hdr, sizeof hdr) || !rd(&ng, sizeof ng)) return 2;
    const int n = hdr[0], k = hdr[1], minrun = hdr[2], wide = hdr[3];
    std::vector<qsim_gate> gs(ng);
    if (ng && !rd(gs.data(), ng * sizeof(qsim_gate))) return 3;
    std::vector<cd> psi((size_t)1 << n);
    if (!rd(psi.data(), psi.size() * sizeof(cd))) return 4;
    int phys[64];
    for (int q = 0; q < 64; q++) phys[q] = q;
    std::vector<PGate> pg(ng);
    std::string msg;
    for (size_t i = 0; i < ng; i++)
        if (!prepare_gate(gs[i], n, phys, pg[i], msg)) return 5;
    std::vector<FusedBlock> plain, blocks;
    std::vector<PhasePass> phases;
    if (!plan_fused(pg, n, k, plain)) return 6;
    if (!plan_fused_phases(pg, n, k, minrun, wide ? 24 : kMaxPhaseTables, blocks, phases)) return 7;
    const size_t N = psi.size();
    int pgates = 0;
    for (const FusedBlock &b : blocks) {
        if (b.phase >= 0) {
            const PhasePass &pp = phases[(size_t)b.phase];
            pgates += pp.gates;
            for (size_t x = 0; x < N; x++) {
                uint32_t ph32 = 0;
                uint64_t ph64 = 0;
                for (size_t t = 0; t < pp.ta.size(); t++) {
                    const uint32_t xa = (uint32_t)(x >> (kPhaseChunk * pp.ta[t])) & 31u;
                    const uint32_t xb = (uint32_t)(x >> (kPhaseChunk * pp.tb[t])) & 31u;
                    const uint64_t w = pp.words[t * kPhaseTableWords + (pp.ta[t] == pp.tb[t] ? xa : xa + 32u * xb)];
                    ph32 += (uint32_t)((w + (1ull << 31)) >> 32);
                    ph64 += w;
                }
                const long double ang = wide ? 2.0L * M_PI * std::ldexp((long double)(int64_t)ph64, -64)
                                             : 2.0L * M_PI * std::ldexp((long double)(int32_t)ph32, -32);
                psi[x] *= cd((double)std::cos(ang), (double)std::sin(ang));
            }
            continue;
        }
        const size_t D = (size_t)1 << b.k;
        std::vector<cd> in(D), out(D);
        for (size_t x = 0; x < N; x++) {
            bool first = true;
            for (int j = 0; j < b.k; j++)
                if ((x >> b.pos[j]) & 1u) first = false;
            if (!first) continue;  // visit each group once, from its member with the block bits 0
            for (size_t c = 0; c < D; c++) {
                size_t y = x;
                for (int j = 0; j < b.k; j++)
                    if ((c >> j) & 1u) y |= (size_t)1 << b.pos[j];
                in[c] = psi[y];
            }
            for (size_t r = 0; r < D; r++) {
                cd s = 0;
                for (size_t c = 0; c < D; c++) s += cd(b.U[2 * (r * D + c)], b.U[2 * (r * D + c) + 1]) * in[c];
                out[r] = s;
            }
            for (size_t r = 0; r < D; r++) {
                size_t y = x;
                for (int j = 0; j < b.k; j++)
                    if ((r >> j) & 1u) y |= (size_t)1 << b.pos[j];
                psi[y] = out[r];
            }
        }
    }
    fwrite(psi.data(), sizeof(cd), N, stdout);
    const int32_t st[4] = {(int32_t)blocks.size(), (int32_t)phases.size(), pgates, (int32_t)plain.size()};
    fwrite(st, sizeof st, 1, stdout);
    return 0;
}
