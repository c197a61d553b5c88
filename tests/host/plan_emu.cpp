// Host emulation of the tile planner's programs (test infrastructure).
//
// Reads a gate list and an initial state, plans the circuit with the
// library's own planner (plan_tiles, and for complex128 plans the
// butterfly / hoisting transforms), and executes the resulting tile
// programs on the host in FP64 with the documented meaning of each tile op.
// The result is compared with the oracle by tests/test_planner_host.py: it
// checks the planner's scheduling, pass capacity cuts, register phases,
// permutations, butterfly factors and per-tile factors without a GPU.  The
// CUDA kernels are not involved; the oracle shares nothing with this file.
//
// stdin (little endian): int32 n, T, RB, c128, max_ops, max_phases; uint64 ng;
// ng qsim_gate records; 2^n complex128 amplitudes.  stdout: 2^n complex128,
// then int32 passes, ops, phases, nglob total, absorbers, butterflies.
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../paper_quant_ph_0608239_gb300/csrc/planner.hpp"

using namespace qsim;
using cd = std::complex<double>;

namespace {

cd coef(const TileOp &op, int k) { return cd(op.u[2 * k], op.u[2 * k + 1]); }

uint64_t insert_zero64(uint64_t x, int pos) {
    const uint64_t lo = x & ((1ull << pos) - 1ull);
    return ((x >> pos) << (pos + 1)) | lo;
}

uint32_t swap_bits(uint32_t x, int np, const int8_t *pl, const int8_t *ph) {
    uint32_t y = x;
    for (int k = 0; k < np; k++) {
        const uint32_t bl = (x >> pl[k]) & 1u, bh = (x >> ph[k]) & 1u;
        y &= ~((1u << pl[k]) | (1u << ph[k]));
        y |= (bl << ph[k]) | (bh << pl[k]);
    }
    return y;
}

// One op over a tile t (2^T amplitudes, local indices); base = the tile's
// global bits.  `scale` multiplies the op's coefficients (per-tile factor).
bool apply_op(std::vector<cd> &t, int T, const TileOp &op, uint64_t base, cd scale = cd(1.0, 0.0)) {
    if ((base & op.gcmask) != op.gcmask) return true;
    const uint32_t TS = 1u << T, lc = op.lcmask;
    auto sel = [&](uint32_t i) { return (i & lc) == lc; };
    switch (op.kind) {
    case TOP_GENERAL:
    case TOP_ANTIDIAG:
    case TOP_EXCHANGE: {
        const uint32_t bt = 1u << op.tl;
        for (uint32_t i = 0; i < TS; i++) {
            if ((i & bt) || !sel(i)) continue;
            const cd x = t[i], y = t[i | bt];
            if (op.kind == TOP_EXCHANGE || op.pk == 3) {
                t[i] = y;
                t[i | bt] = x;
            } else if (op.kind == TOP_ANTIDIAG) {
                t[i] = scale * coef(op, 1) * y;
                t[i | bt] = scale * coef(op, 2) * x;
            } else if (op.pk == 4) {  // unscaled butterfly
                t[i] = x + y;
                t[i | bt] = x - y;
            } else {
                t[i] = scale * (coef(op, 0) * x + coef(op, 1) * y);
                t[i | bt] = scale * (coef(op, 2) * x + coef(op, 3) * y);
            }
        }
        return true;
    }
    case TOP_PHASE:
        for (uint32_t i = 0; i < TS; i++)
            if (((i >> op.tl) & 1u) && sel(i)) t[i] *= scale * coef(op, 3);
        return true;
    case TOP_DIAG:
        for (uint32_t i = 0; i < TS; i++)
            if (sel(i)) t[i] *= scale * (((i >> op.tl) & 1u) ? coef(op, 3) : coef(op, 0));
        return true;
    case TOP_DIAG_G: {
        const cd f = scale * (((base >> op.tl) & 1ull) ? coef(op, 3) : coef(op, 0));
        for (uint32_t i = 0; i < TS; i++)
            if (sel(i)) t[i] *= f;
        return true;
    }
    case TOP_SWAPGATE: {
        const uint32_t b0 = 1u << op.tl, b1 = 1u << op.tl2;
        for (uint32_t i = 0; i < TS; i++) {
            if (!(i & b0) || (i & b1) || !sel(i)) continue;
            const uint32_t j = (i & ~b0) | b1;
            std::swap(t[i], t[j]);
        }
        return true;
    }
    case TOP_PERM: {
        std::vector<cd> o(TS);
        for (uint32_t i = 0; i < TS; i++) o[swap_bits(i, op.nperm, op.pl, op.ph)] = t[i];
        t.swap(o);
        return true;
    }
    default: return false;
    }
}

}  // namespace

int main() {
    int32_t hdr[6];
    uint64_t ng = 0;
    if (fread(hdr, 4, 6, stdin) != 6 || fread(&ng, 8, 1, stdin) != 1) return 2;
    const int n = hdr[0], T0 = hdr[1], RB = hdr[2], c128 = hdr[3], max_ops = hdr[4], max_phases = hdr[5];
    std::vector<qsim_gate> g(ng);
    if (ng && fread(g.data(), sizeof(qsim_gate), ng, stdin) != ng) return 2;
    const size_t N = (size_t)1 << n;
    std::vector<cd> a(N);
    if (fread(a.data(), sizeof(cd), N, stdin) != N) return 2;

    int phys[64];
    for (int i = 0; i < 64; i++) phys[i] = i;
    std::vector<PGate> pg(ng);
    std::string msg;
    for (size_t i = 0; i < ng; i++)
        if (!prepare_gate(g[i], n, phys, pg[i], msg)) {
            fprintf(stderr, "gate %zu: %s\n", i, msg.c_str());
            return 3;
        }
    // tile geometry as the library picks it
    int T = T0, L = RB ? 5 : (c128 ? 4 : 5);
    if (T - L > 10) L = T - 10;
    if (L >= T) L = T - 2;
    if (L < 1) L = 1;
    Plan plan;
    plan_tiles(pg, n, T, L, plan, RB, max_ops, max_phases);
    if (c128) {
        defer_butterflies(plan);
        merge_local_diagonals(plan);
        hoist_global_diagonals(plan);
    }
    int32_t stats[6] = {0, 0, 0, 0, 0, 0};
    for (const PassPlan &pp : plan.passes) {
        const TileGeom &geo = pp.geom;
        const int Lg = geo.L, H = geo.H, Tg = Lg + H;
        if (pp.op_count || pp.phase_count) stats[0]++;
        stats[1] += pp.op_count;
        stats[2] += pp.phase_count;
        stats[3] += pp.nglob;
        stats[4] += pp.absorber >= 0;
        for (int i = 0; i < pp.op_count; i++) stats[5] += plan.ops[pp.op_begin + i].pk == 4;
        const uint64_t ntiles = 1ull << (n - Tg);
        std::vector<uint64_t> runoff((size_t)1 << H);
        for (uint32_t j = 0; j < (1u << H); j++) {
            uint64_t o = 0;
            for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << geo.hb[k];
            runoff[j] = o;
        }
        std::vector<cd> t((size_t)1 << Tg);
        for (uint64_t tile = 0; tile < ntiles; tile++) {
            uint64_t base = tile << Lg;
            for (int k = 0; k < H; k++) base = insert_zero64(base, geo.hb[k]);
            const uint32_t lowmask = (1u << Lg) - 1u;
            for (uint32_t i = 0; i < (1u << Tg); i++) t[i] = a[base | runoff[i >> Lg] | (i & lowmask)];
            if (pp.phase_count > 0) {
                for (int p = 0; p < pp.phase_count; p++) {
                    const TilePhase &ph = plan.phases[pp.phase_begin + p];
                    for (int o = ph.op_begin; o < ph.op_begin + ph.op_count; o++)
                        if (!apply_op(t, Tg, plan.ops[o], base)) return 4;
                    if (ph.nperm) {
                        std::vector<cd> o(t.size());
                        for (uint32_t i = 0; i < t.size(); i++) o[swap_bits(i, ph.nperm, ph.pl, ph.ph)] = t[i];
                        t.swap(o);
                    }
                }
            } else {
                const int nprog = pp.op_count - pp.nglob;
                cd f(1.0, 0.0);  // the hoisted diagonals' factor for this tile
                for (int k = 0; k < pp.nglob; k++) {
                    const TileOp &go = plan.ops[pp.op_begin + nprog + k];
                    if ((base & go.gcmask) != go.gcmask) continue;
                    f *= ((base >> go.tl) & 1ull) ? coef(go, 3) : coef(go, 0);
                }
                for (int o = 0; o < nprog; o++)
                    if (!apply_op(t, Tg, plan.ops[pp.op_begin + o], base, o == pp.absorber ? f : cd(1.0, 0.0)))
                        return 4;
                if (pp.nglob > 0 && pp.absorber < 0)
                    for (cd &v : t) v *= f;
            }
            for (uint32_t i = 0; i < (1u << Tg); i++) a[base | runoff[i >> Lg] | (i & lowmask)] = t[i];
        }
    }
    fwrite(a.data(), sizeof(cd), N, stdout);
    fwrite(stats, 4, 6, stdout);
    return 0;
}
