// planner.cpp -- gate matrices (Sec. II), validation and the tile planner.
#include "planner.hpp"

#include <algorithm>
#include <iterator>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>

namespace qsim {

namespace {

inline void set(Mat2 &M, int k, double re, double im) {
    M.u[2 * k] = re;
    M.u[2 * k + 1] = im;
}

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

bool gate_matrix(int kind, const double *p, Mat2 &M) {
    // cos(pi/4) = sin(pi/4): the pi/2 rotations e^{i pi S/2} = cos(pi/4) + i sin(pi/4) sigma
    const double c = std::sqrt(0.5);
    for (double &x : M.u) x = 0.0;
    switch (kind) {
    case QSIM_GATE_H:  // (sigma_x + sigma_z)/sqrt(2), Eq. Hadamard
        set(M, 0, c, 0); set(M, 1, c, 0); set(M, 2, c, 0); set(M, 3, -c, 0);
        return true;
    case QSIM_GATE_X:  // cos + i sin sigma_x, Eq. Xoperation
        set(M, 0, c, 0); set(M, 1, 0, c); set(M, 2, 0, c); set(M, 3, c, 0);
        return true;
    case QSIM_GATE_Y:  // cos + i sin sigma_y, Eq. Yoperation
        set(M, 0, c, 0); set(M, 1, c, 0); set(M, 2, -c, 0); set(M, 3, c, 0);
        return true;
    case QSIM_GATE_XB:  // cos - i sin sigma_x
        set(M, 0, c, 0); set(M, 1, 0, -c); set(M, 2, 0, -c); set(M, 3, c, 0);
        return true;
    case QSIM_GATE_YB:  // cos - i sin sigma_y
        set(M, 0, c, 0); set(M, 1, -c, 0); set(M, 2, c, 0); set(M, 3, c, 0);
        return true;
    case QSIM_GATE_NOT:  // sigma_x: the flip of Eqs. NUM6, NUM8
        set(M, 1, 1, 0); set(M, 2, 1, 0);
        return true;
    case QSIM_GATE_R:  // diag(1, e^{i phi}), Eq. singlephase
        set(M, 0, 1, 0); set(M, 3, std::cos(p[0]), std::sin(p[0]));
        return true;
    case QSIM_GATE_V: {  // e^{i phi/2} (cos(phi/2) - i sin(phi/2) sigma_x) = Eq. COMM4
        const double er = std::cos(p[0]), ei = std::sin(p[0]);
        set(M, 0, 0.5 * (1 + er), 0.5 * ei); set(M, 1, 0.5 * (1 - er), -0.5 * ei);
        set(M, 2, 0.5 * (1 - er), -0.5 * ei); set(M, 3, 0.5 * (1 + er), 0.5 * ei);
        return true;
    }
    case QSIM_GATE_SU2:  // quaternion (a, b, c, d)
        set(M, 0, p[0], p[1]); set(M, 1, p[2], p[3]); set(M, 2, -p[2], p[3]); set(M, 3, p[0], -p[1]);
        return true;
    case QSIM_GATE_U:
        for (int k = 0; k < 8; k++) M.u[k] = p[k];
        return true;
    default:
        return false;
    }
}

int classify(const Mat2 &M) {
    const bool off0 = M.u[2] == 0 && M.u[3] == 0 && M.u[4] == 0 && M.u[5] == 0;
    const bool diag0 = M.u[0] == 0 && M.u[1] == 0 && M.u[6] == 0 && M.u[7] == 0;
    if (off0) return (M.u[0] == 1 && M.u[1] == 0) ? GC_PHASE : GC_DIAG;
    if (diag0) return (M.u[2] == 1 && M.u[3] == 0 && M.u[4] == 1 && M.u[5] == 0) ? GC_EXCHANGE : GC_ANTIDIAG;
    const bool real = M.u[1] == 0 && M.u[3] == 0 && M.u[5] == 0 && M.u[7] == 0;
    return real ? GC_REAL : GC_GENERAL;
}

bool prepare_gate(const qsim_gate &g, int n, const int *phys, PGate &out, std::string &msg) {
    char buf[160];
    if (g.target < 0 || g.target >= n) {
        snprintf(buf, sizeof buf, "gate target %d out of range [0, %d)", g.target, n);
        msg = buf;
        return false;
    }
    if (n < 64 && (g.ctrl_mask >> n) != 0) {
        msg = "ctrl_mask names a qubit >= n";
        return false;
    }
    if ((g.ctrl_mask >> g.target) & 1ull) {
        msg = "ctrl_mask contains the target qubit";
        return false;
    }
    out.t1 = -1;
    out.cmask = 0;
    for (int q = 0; q < n; q++)
        if ((g.ctrl_mask >> q) & 1ull) out.cmask |= 1ull << phys[q];
    out.t0 = phys[g.target];
    out.kind = g.kind;
    if (g.kind == QSIM_GATE_SWAP) {
        if (g.target2 < 0 || g.target2 >= n || g.target2 == g.target) {
            msg = "SWAP needs a second, distinct target qubit";
            return false;
        }
        if ((g.ctrl_mask >> g.target2) & 1ull) {
            msg = "ctrl_mask contains a SWAP target";
            return false;
        }
        out.t1 = phys[g.target2];
        out.gc = GC_EXCHANGE;
        return true;
    }
    int np = 0;
    switch (g.kind) {
    case QSIM_GATE_R: case QSIM_GATE_V: np = 1; break;
    case QSIM_GATE_SU2: np = 4; break;
    case QSIM_GATE_U: np = 8; break;
    default: break;
    }
    for (int k = 0; k < np; k++)
        if (!std::isfinite(g.param[k])) {
            msg = "non-finite gate parameter";
            return false;
        }
    if (!gate_matrix(g.kind, g.param, out.U)) {
        snprintf(buf, sizeof buf, "unknown gate kind %d", g.kind);
        msg = buf;
        return false;
    }
    out.gc = classify(out.U);
    return true;
}

void fixed_bits_for(const PGate &g, FixedBitsHost &fb, uint64_t &pmask, bool &single) {
    std::vector<int> pos;
    uint64_t set = g.cmask;
    for (int b = 0; b < 64; b++)
        if ((g.cmask >> b) & 1ull) pos.push_back(b);
    single = false;
    pmask = 0;
    if (g.kind == QSIM_GATE_SWAP) {
        pos.push_back(g.t0);
        pos.push_back(g.t1);
        set |= 1ull << g.t0;  // visit t0 = 1, t1 = 0; the partner has them exchanged
        pmask = (1ull << g.t0) | (1ull << g.t1);
    } else if (g.gc == GC_PHASE) {
        pos.push_back(g.t0);
        set |= 1ull << g.t0;
        single = true;
    } else if (g.gc == GC_DIAG) {
        single = true;
    } else {
        pos.push_back(g.t0);
        pmask = 1ull << g.t0;
    }
    std::sort(pos.begin(), pos.end());
    fb.npos = (int)pos.size();
    for (int k = 0; k < fb.npos && k < 24; k++) fb.pos[k] = pos[k];
    fb.setmask = set;
}

double gate_flops(const PGate &g, int n) {
    double per_amp = 0.0;
    if (g.kind == QSIM_GATE_SWAP) return 0.0;
    switch (g.gc) {
    case GC_GENERAL: per_amp = 14.0; break;
    case GC_REAL: per_amp = 6.0; break;
    case GC_DIAG: per_amp = 6.0; break;
    case GC_PHASE: per_amp = 3.0; break;
    case GC_ANTIDIAG: per_amp = 6.0; break;
    default: per_amp = 0.0; break;
    }
    return per_amp * std::ldexp(1.0, n - popc(g.cmask));
}

bool make_tile_op(const PGate &pg, const TileGeom &g, TileOp &op) {
    auto local = [&](int b) -> int {
        if (b < g.L) return b;
        for (int j = 0; j < g.H; j++)
            if (g.hb[j] == b) return g.L + j;
        return -1;
    };
    op = TileOp{};
    op.tl2 = -1;
    for (int b = 0; b < 64; b++) {
        if (!((pg.cmask >> b) & 1ull)) continue;
        const int lb = local(b);
        if (lb >= 0) op.lcmask |= 1u << lb;
        else op.gcmask |= 1ull << b;
    }
    for (int k = 0; k < 8; k++) {
        op.u[k] = pg.U.u[k];
        op.uh[k] = (float)pg.U.u[k];
        op.ul[k] = (float)(pg.U.u[k] - (double)op.uh[k]);
    }
    op.regk = -1;
    op.pk = pg.gc == GC_REAL ? 1 : pg.gc == GC_ANTIDIAG ? 2 : pg.gc == GC_EXCHANGE ? 3 : 0;
    if (pg.kind == QSIM_GATE_SWAP) {
        const int a = local(pg.t0), b = local(pg.t1);
        if (a < 0 || b < 0) return false;
        op.kind = TOP_SWAPGATE;
        op.tl = a;
        op.tl2 = b;
        return true;
    }
    const int lt = local(pg.t0);
    switch (pg.gc) {
    case GC_PHASE:
    case GC_DIAG:
        if (lt >= 0) {
            op.kind = pg.gc == GC_PHASE ? TOP_PHASE : TOP_DIAG;
            op.tl = lt;
        } else {
            op.kind = TOP_DIAG_G;
            op.tl = pg.t0;
        }
        return true;
    case GC_GENERAL:
    case GC_REAL: op.kind = TOP_GENERAL; break;
    case GC_ANTIDIAG: op.kind = TOP_ANTIDIAG; break;
    default: op.kind = TOP_EXCHANGE; break;
    }
    if (lt < 0) return false;
    op.tl = lt;
    return true;
}

namespace {

// Physical bits a gate needs inside the tile (its targets, unless diagonal).
uint64_t target_bits(const PGate &g) {
    if (g.kind == QSIM_GATE_SWAP) return (1ull << g.t0) | (1ull << g.t1);
    if (g.gc == GC_PHASE || g.gc == GC_DIAG) return 0;
    return 1ull << g.t0;
}

uint64_t touched_bits(const PGate &g) {
    uint64_t m = g.cmask | (1ull << g.t0);
    if (g.t1 >= 0) m |= 1ull << g.t1;
    return m;
}

}  // namespace

namespace {

// One item of a pass program before phasing: an op, or a permutation of
// local bit pairs (an uncontrolled SWAP gate or an interchange).
struct Item {
    bool perm;
    TileOp op;
    int np;
    int8_t pl[8], ph[8];
};

bool needs_register(const TileOp &op) {
    return (op.kind == TOP_GENERAL || op.kind == TOP_ANTIDIAG || op.kind == TOP_EXCHANGE) && op.tl >= 5;
}

}  // namespace

void build_phases(const std::vector<TileOp> &pass_ops, int T, int RB, std::vector<TileOp> &ops_out,
                  std::vector<TilePhase> &phases_out) {
    // expand SWAP gates: uncontrolled ones become store permutations, controlled
    // ones three multi-controlled bit flips (each applied only where the controls
    // are 1, so the SWAP happens exactly there)
    std::vector<Item> items;
    for (const TileOp &o : pass_ops) {
        if (o.kind == TOP_SWAPGATE && o.lcmask == 0 && o.gcmask == 0) {
            Item it{};
            it.perm = true;
            it.np = 1;
            it.pl[0] = (int8_t)o.tl;
            it.ph[0] = (int8_t)o.tl2;
            items.push_back(it);
        } else if (o.kind == TOP_SWAPGATE) {
            const int a = o.tl, b = o.tl2;
            for (int r = 0; r < 3; r++) {
                Item it{};
                it.perm = false;
                it.op = o;
                it.op.kind = TOP_EXCHANGE;
                it.op.pk = 3;
                const int tgt = (r == 1) ? a : b, ctl = (r == 1) ? b : a;
                it.op.tl = tgt;
                it.op.tl2 = -1;
                it.op.lcmask = o.lcmask | (1u << ctl);
                items.push_back(it);
            }
        } else if (o.kind == TOP_PERM) {
            Item it{};
            it.perm = true;
            it.np = o.nperm;
            for (int k = 0; k < o.nperm; k++) {
                it.pl[k] = o.pl[k];
                it.ph[k] = o.ph[k];
            }
            items.push_back(it);
        } else {
            Item it{};
            it.perm = false;
            it.op = o;
            items.push_back(it);
        }
    }
    const uint32_t high = ((1u << T) - 1u) & ~31u;  // local bits 5..T-1
    size_t i = 0;
    while (i < items.size()) {
        TilePhase ph{};
        uint32_t rset = 0;
        std::vector<TileOp> pops;
        size_t j = i;
        for (; j < items.size(); j++) {
            const Item &it = items[j];
            if (it.perm) {
                ph.nperm = it.np;
                for (int k = 0; k < it.np; k++) {
                    ph.pl[k] = it.pl[k];
                    ph.ph[k] = it.ph[k];
                }
                j++;
                break;
            }
            const uint32_t need = needs_register(it.op) ? (1u << it.op.tl) : 0u;
            if (popc(rset | need) <= RB) {
                rset |= need;
                pops.push_back(it.op);
            } else {
                break;
            }
        }
        // fill the free register slots with the bits the next ops want
        for (size_t k = j; k < items.size() && popc(rset) < RB; k++) {
            if (items[k].perm) continue;
            if (needs_register(items[k].op)) rset |= 1u << items[k].op.tl;
            if (popc(rset) > RB) rset &= ~(1u << items[k].op.tl);
        }
        for (int b = 5; b < T && popc(rset) < RB; b++) rset |= 1u << b;
        int nr = 0, nw = 0;
        for (int b = 5; b < T; b++) {
            if ((rset >> b) & 1u) ph.rb[nr++] = (int8_t)b;
            else if ((high >> b) & 1u) ph.wb[nw++] = (int8_t)b;
        }
        ph.op_begin = (int)ops_out.size();
        ph.op_count = (int)pops.size();
        for (TileOp op : pops) {
            op.regk = -1;
            const bool local_target = !(op.kind == TOP_DIAG_G);
            if (local_target && op.tl >= 5)
                for (int k = 0; k < nr; k++)
                    if (ph.rb[k] == op.tl) op.regk = (int8_t)k;
            op.creg = 0;
            for (int k = 0; k < nr; k++)
                if ((op.lcmask >> ph.rb[k]) & 1u) op.creg |= 1u << k;
            op.lcthr = op.lcmask & ~rset;
            op.cslot = 0;
            const bool noctl = op.lcmask == 0;
            int fam, k = op.regk;
            if (op.kind == TOP_DIAG_G) {
                fam = RC_GLOB;
                k = 0;
            } else if (op.kind == TOP_PHASE || op.kind == TOP_DIAG) {
                if (op.regk >= 0) fam = op.kind == TOP_PHASE ? RC_PHASE : RC_DIAG;
                else {
                    fam = RC_THR;
                    k = op.kind == TOP_PHASE ? 0 : 1;
                }
            } else if (op.regk < 0) {  // pair op on a lane bit
                fam = noctl ? RC_LANE : RC_LANEC;
                k = op.pk;
            } else if (op.pk == 0) {
                fam = noctl ? RC_GEN : RC_GENC;
            } else if (op.pk == 1) {
                fam = noctl ? RC_REAL : RC_REALC;
            } else if (op.pk == 2) {
                fam = RC_ANTI;
            } else {
                fam = RC_EXCHC;
            }
            op.code = (uint8_t)(fam * 8 + k);
            ops_out.push_back(op);
        }
        phases_out.push_back(ph);
        i = j;
    }
}

void plan_tiles(const std::vector<PGate> &gates, int n, int T, int L, Plan &plan, int RB, int max_ops,
                int max_phases) {
    plan.passes.clear();
    plan.ops.clear();
    plan.dense.clear();
    plan.phases.clear();
    if (gates.empty()) return;
    if (T > n) T = n;
    if (n <= T) L = n;
    if (L > T) L = T;
    if (n > T && T - L < 2) L = T - 2;  // room for both targets of a SWAP
    if (L < 1) L = 1;
    const int H = (n > T) ? T - L : 0;
    const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
    const uint64_t low = (1ull << L) - 1;

    std::vector<int> remaining(gates.size());
    for (size_t i = 0; i < gates.size(); i++) remaining[i] = (int)i;
    std::vector<int> sched, rest;
    while (!remaining.empty()) {
        uint64_t inset = low, hmask = 0, blocked = 0;
        int hcount = 0;
        sched.clear();
        rest.clear();
        for (size_t r = 0; r < remaining.size(); r++) {
            const int gi = remaining[r];
            const PGate &g = gates[gi];
            const uint64_t qm = touched_bits(g);
            if ((blocked & all) == all || (qm & blocked)) {
                blocked |= qm;
                rest.push_back(gi);
                continue;
            }
            const uint64_t need = target_bits(g) & ~inset;
            if (hcount + popc(need) <= H) {
                inset |= need;
                hmask |= need;
                hcount += popc(need);
                sched.push_back(gi);
            } else {
                blocked |= qm;
                rest.push_back(gi);
            }
        }
        // Fill the remaining high slots with the targets of the gates that
        // come next, then with the lowest unused bits.
        for (size_t r = 0; r < rest.size() && hcount < H; r++) {
            uint64_t need = target_bits(gates[rest[r]]) & ~inset & all;
            while (need && hcount < H) {
                const uint64_t b = need & (~need + 1);
                need &= need - 1;
                inset |= b;
                hmask |= b;
                hcount++;
            }
        }
        for (int b = L; b < n && hcount < H; b++)
            if (!((inset >> b) & 1ull)) {
                inset |= 1ull << b;
                hmask |= 1ull << b;
                hcount++;
            }
        PassPlan pp{};
        pp.geom.n = n;
        pp.geom.L = L;
        pp.geom.H = hcount;
        int j = 0;
        for (int b = 0; b < 64; b++)
            if ((hmask >> b) & 1ull) pp.geom.hb[j++] = b;
        std::vector<TileOp> pass_ops;
        for (int gi : sched) {
            TileOp op;
            make_tile_op(gates[gi], pp.geom, op);  // fits by construction
            pass_ops.push_back(op);
        }
        const bool reg = RB > 0 && L + hcount == RB + 5 + kRegWarpBits && L >= 5;
        // keep the pass within the program capacity: the largest prefix of
        // its gates that fits; the others return to the remaining list
        size_t take = sched.size();
        std::vector<TileOp> rops;
        std::vector<TilePhase> rph;
        for (;;) {
            size_t nops = take, nph = 0;
            if (reg) {
                rops.clear();
                rph.clear();
                build_phases(std::vector<TileOp>(pass_ops.begin(), pass_ops.begin() + take), L + hcount, RB, rops,
                             rph);
                nops = rops.size();
                nph = rph.size();
            }
            const size_t over_o = (max_ops > 0 && nops > (size_t)max_ops) ? nops - (size_t)max_ops : 0;
            const size_t over_p = (max_phases > 0 && nph > (size_t)max_phases) ? nph - (size_t)max_phases : 0;
            if ((!over_o && !over_p) || take <= 1) break;
            const size_t cut = over_o > over_p ? over_o : over_p;
            take = cut < take ? take - cut : 1;
        }
        if (take < sched.size()) {
            // the dropped gates commute with the skipped ones before them, so
            // merging both back in program order keeps the circuit
            std::vector<int> merged;
            merged.reserve(rest.size() + sched.size() - take);
            std::merge(sched.begin() + take, sched.end(), rest.begin(), rest.end(), std::back_inserter(merged));
            rest.swap(merged);
            sched.resize(take);
            pass_ops.resize(take);
        }
        pp.flops = 0.0;
        for (int gi : sched) pp.flops += gate_flops(gates[gi], n);
        pp.op_begin = (int)plan.ops.size();
        pp.phase_begin = (int)plan.phases.size();
        if (reg) {
            build_phases(pass_ops, L + hcount, RB, plan.ops, plan.phases);
        } else {
            plan.ops.insert(plan.ops.end(), pass_ops.begin(), pass_ops.end());
        }
        pp.op_count = (int)plan.ops.size() - pp.op_begin;
        pp.phase_count = (int)plan.phases.size() - pp.phase_begin;
        pp.arith = false;
        for (int gi : sched)
            if (gates[gi].kind != QSIM_GATE_SWAP && gates[gi].gc != GC_EXCHANGE) pp.arith = true;
        plan.passes.push_back(pp);
        remaining.swap(rest);
    }
}

namespace {

// s if U = s * [[1, 1], [1, -1]] exactly (real s != 0), else 0.
double hadamard_factor(const double (&u)[8]) {
    const double s = u[0];
    if (s == 0.0 || u[1] != 0.0 || u[3] != 0.0 || u[5] != 0.0 || u[7] != 0.0) return 0.0;
    if (u[2] != s || u[4] != s || u[6] != -s) return 0.0;
    return s;
}

void scale_op(TileOp &op, double f) {
    for (int k = 0; k < 8; k++) {
        op.u[k] *= f;
        op.uh[k] = (float)op.u[k];
        op.ul[k] = (float)(op.u[k] - (double)op.uh[k]);
    }
}

}  // namespace

namespace {

// The op acts non-diagonally on local bit b (moves or mixes amplitudes along b).
bool mixes_bit(const TileOp &op, int b) {
    switch (op.kind) {
    case TOP_GENERAL:
    case TOP_ANTIDIAG:
    case TOP_EXCHANGE: return op.tl == b;
    case TOP_SWAPGATE: return op.tl == b || op.tl2 == b;
    case TOP_PERM:
    case TOP_DENSE:
        for (int k = 0; k < op.nperm; k++)
            if (op.pl[k] == b || (op.kind == TOP_PERM && op.ph[k] == b)) return true;
        return false;
    default: return false;  // diagonal ops
    }
}

bool uncontrolled(const TileOp &op) { return op.lcmask == 0 && op.gcmask == 0; }

// Row-major complex 2x2 product C = A * B (interleaved re, im).
void mat2_mul(const double (&A)[8], const double (&B)[8], double (&C)[8]) {
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 2; k++) {
                const double ar = A[2 * (2 * r + k)], ai = A[2 * (2 * r + k) + 1];
                const double br = B[2 * (2 * k + c)], bi = B[2 * (2 * k + c) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            C[2 * (2 * r + c)] = re;
            C[2 * (2 * r + c) + 1] = im;
        }
}

void set_matrix(TileOp &op, const double (&M)[8]) {
    for (int k = 0; k < 8; k++) {
        op.u[k] = M[k];
        op.uh[k] = (float)M[k];
        op.ul[k] = (float)(M[k] - (double)op.uh[k]);
    }
}

// Can `d` (an uncontrolled diagonal on local bit b) be merged into `x`, an
// uncontrolled op on the same bit that keeps its kind and cost: a dense
// complex 2x2, or another phase / diagonal.
bool merge_target(const TileOp &x, int b) {
    if (!uncontrolled(x) || x.tl != b) return false;
    if (x.kind == TOP_GENERAL) return x.pk == 0;
    return x.kind == TOP_PHASE || x.kind == TOP_DIAG;
}

}  // namespace

void merge_local_diagonals(Plan &plan) {
    for (PassPlan &pp : plan.passes) {
        if (pp.phase_count > 0 || pp.op_count < 2) continue;
        std::vector<TileOp> ops(plan.ops.begin() + pp.op_begin, plan.ops.begin() + pp.op_begin + pp.op_count);
        std::vector<bool> gone(ops.size(), false);
        for (size_t i = 0; i < ops.size(); i++) {
            TileOp &d = ops[i];
            if ((d.kind != TOP_PHASE && d.kind != TOP_DIAG) || !uncontrolled(d)) continue;
            const int b = d.tl;
            int into = -1;
            bool after = false;  // d is applied after ops[into]
            for (int j = (int)i - 1; j >= 0; j--) {  // back to the last op on bit b
                if (gone[j]) continue;
                if (merge_target(ops[j], b)) {
                    into = j;
                    after = true;
                    break;
                }
                if (mixes_bit(ops[j], b)) break;
            }
            if (into < 0)
                for (size_t j = i + 1; j < ops.size(); j++) {  // forward to the next op on bit b
                    if (merge_target(ops[j], b)) {
                        into = (int)j;
                        break;
                    }
                    if (mixes_bit(ops[j], b)) break;
                }
            if (into < 0) continue;
            TileOp &x = ops[into];
            double M[8];
            if (after) mat2_mul(d.u, x.u, M);
            else mat2_mul(x.u, d.u, M);
            if (x.kind != TOP_GENERAL)  // diagonal times diagonal
                x.kind = (x.kind == TOP_PHASE && d.kind == TOP_PHASE) ? TOP_PHASE : TOP_DIAG;
            set_matrix(x, M);
            gone[i] = true;
        }
        int k = 0;
        for (size_t i = 0; i < ops.size(); i++)
            if (!gone[i]) plan.ops[pp.op_begin + k++] = ops[i];
        // the pass shrinks in place; the tail of its old range is unused
        pp.op_count = k;
    }
}

void defer_butterflies(Plan &plan) {
    for (PassPlan &pp : plan.passes) {
        if (pp.phase_count > 0 || pp.op_count == 0) continue;
        TileOp *ops = plan.ops.data() + pp.op_begin;
        std::vector<int> bf;
        int absorber = -1;
        double S = 1.0;
        for (int i = 0; i < pp.op_count; i++) {
            TileOp &op = ops[i];
            if (op.lcmask != 0 || op.gcmask != 0) continue;  // controlled: touches a subset
            const double s = op.kind == TOP_GENERAL ? hadamard_factor(op.u) : 0.0;
            if (s != 0.0 && (int)bf.size() < kMaxDeferred) {
                bf.push_back(i);
                S *= s;
            } else if (absorber < 0 && (op.kind == TOP_GENERAL || op.kind == TOP_ANTIDIAG || op.kind == TOP_DIAG ||
                                        op.kind == TOP_DIAG_G)) {
                absorber = i;
            }
        }
        if (bf.empty()) continue;
        if (absorber < 0) {  // one Hadamard-type op takes the whole factor
            absorber = bf.back();
            bf.pop_back();
            if (bf.empty()) continue;  // a single one: nothing to defer
            scale_op(ops[absorber], S / ops[absorber].u[0]);
        } else {
            scale_op(ops[absorber], S);
        }
        for (int i : bf) {
            ops[i].pk = 4;
            scale_op(ops[i], 1.0 / ops[i].u[0]);  // the entries read +-1 (unused by the kernel)
        }
    }
}

void hoist_global_diagonals(Plan &plan) {
    for (PassPlan &pp : plan.passes) {
        if (pp.phase_count > 0 || pp.op_count == 0) continue;
        TileOp *ops = plan.ops.data() + pp.op_begin;
        std::vector<TileOp> prog, glob;
        for (int i = 0; i < pp.op_count; i++) {
            if (ops[i].kind == TOP_DIAG_G && ops[i].lcmask == 0) glob.push_back(ops[i]);
            else prog.push_back(ops[i]);
        }
        if (glob.empty()) continue;
        pp.nglob = (int)glob.size();
        pp.absorber = -1;
        for (size_t i = 0; i < prog.size(); i++) {
            const TileOp &op = prog[i];
            if (op.lcmask != 0 || op.gcmask != 0) continue;
            if ((op.kind == TOP_GENERAL && op.pk == 0) || op.kind == TOP_ANTIDIAG || op.kind == TOP_DIAG) {
                pp.absorber = (int)i;
                break;
            }
        }
        int k = 0;
        for (const TileOp &op : prog) ops[k++] = op;
        for (const TileOp &op : glob) ops[k++] = op;
    }
}

}  // namespace qsim

namespace qsim {

namespace {

// Apply one gate to the D = 2^k columns of a block matrix in block
// coordinates (bit j = pos[j]); cols holds column c at c * D.  The bit
// positions are resolved once per gate, then every column takes the same
// update.
void apply_in_block(const PGate &g, const int *pos, int k, std::complex<double> *cols) {
    auto loc = [&](int b) {
        for (int j = 0; j < k; j++)
            if (pos[j] == b) return j;
        return -1;
    };
    uint32_t cm = 0;
    for (uint64_t m = g.cmask; m; m &= m - 1) cm |= 1u << loc(__builtin_ctzll(m));
    const uint32_t D = 1u << k;
    if (g.kind == QSIM_GATE_SWAP) {
        const uint32_t b0 = 1u << loc(g.t0), b1 = 1u << loc(g.t1);
        for (uint32_t c = 0; c < D; c++) {
            std::complex<double> *v = cols + (size_t)c * D;
            for (uint32_t i = 0; i < D; i++) {
                if (!(i & b0) || (i & b1) || (i & cm) != cm) continue;
                std::swap(v[i], v[(i & ~b0) | b1]);
            }
        }
        return;
    }
    const uint32_t bt = 1u << loc(g.t0);
    const std::complex<double> u00(g.U.u[0], g.U.u[1]), u01(g.U.u[2], g.U.u[3]);
    const std::complex<double> u10(g.U.u[4], g.U.u[5]), u11(g.U.u[6], g.U.u[7]);
    for (uint32_t c = 0; c < D; c++) {
        std::complex<double> *v = cols + (size_t)c * D;
        for (uint32_t i = 0; i < D; i++) {
            if ((i & bt) || (i & cm) != cm) continue;
            const std::complex<double> a0 = v[i], a1 = v[i | bt];
            v[i] = u00 * a0 + u01 * a1;
            v[i | bt] = u10 * a0 + u11 * a1;
        }
    }
}

uint64_t block_bits(const PGate &g) {
    uint64_t m = g.cmask | (1ull << g.t0);
    if (g.t1 >= 0) m |= 1ull << g.t1;
    return m;
}

void emit_block(const std::vector<const PGate *> &gs, uint64_t mask, int n, int k, std::vector<FusedBlock> &out) {
    FusedBlock b;
    b.k = k;
    int j = 0;
    for (int q = 0; q < 64 && j < k; q++)
        if ((mask >> q) & 1ull) b.pos[j++] = q;
    for (int q = 0; q < n && j < k; q++)  // pad with the lowest other qubits
        if (!((mask >> q) & 1ull)) b.pos[j++] = q;
    std::sort(b.pos, b.pos + k);
    const uint32_t D = 1u << k;
    // column c of U = the block applied to |c>: every column starts as its
    // basis vector and takes the gates in order
    std::vector<std::complex<double>> cols((size_t)D * D, std::complex<double>(0.0, 0.0));
    for (uint32_t c = 0; c < D; c++) cols[(size_t)c * D + c] = 1.0;
    for (const PGate *g : gs) apply_in_block(*g, b.pos, k, cols.data());
    b.U.assign(2 * (size_t)D * D, 0.0);
    for (uint32_t c = 0; c < D; c++)
        for (uint32_t r = 0; r < D; r++) {
            b.U[2 * (r * D + c)] = cols[(size_t)c * D + r].real();
            b.U[2 * (r * D + c) + 1] = cols[(size_t)c * D + r].imag();
        }
    b.flops = 8.0 * D * std::ldexp(1.0, n);
    out.push_back(std::move(b));
}

}  // namespace

namespace {

// Candidate block sets of the search: the breadth of the search over the
// qubit sets a block can reach (plan_fused).
constexpr int kBlockBeam = 16;

struct BlockDraft {
    std::vector<int> picks;  // gate indices in the order they are applied
    uint64_t mask;           // the block's qubits
};

// One grouping of the circuit into blocks of at most k qubits.  A block
// starts at the earliest gate not yet placed and takes only gates whose
// earlier gates on each of their qubits are placed.  beam = 0: the greedy
// block (gates inside the block's qubits first, else the gate after which the
// fewest-qubits-first rule takes the most gates).  beam > 0: the larger of
// that block and the best one found by a beam search over the qubit sets the
// block can grow into (beam sets kept per added gate, ranked by the gates
// they hold plus those the fewest-qubits-first rule would still add).
void draft_blocks(const std::vector<uint64_t> &bits, const std::vector<std::vector<int>> &queue, int k, int beam,
                  std::vector<BlockDraft> &out) {
    const int ng = (int)bits.size();
    int nq = 0;  // qubits that have gates: the scans below stop there
    for (uint64_t b : bits) nq = std::max(nq, 64 - __builtin_clzll(b));
    using Heads = std::array<uint32_t, 64>;  // per qubit: first gate of its queue not yet placed
    auto front = [&](const Heads &hd, int q) { return hd[q] < queue[q].size() ? queue[q][hd[q]] : -1; };
    auto ready = [&](const Heads &hd, int i) {  // every earlier gate on i's qubits is placed
        for (uint64_t m = bits[i]; m; m &= m - 1)
            if (front(hd, __builtin_ctzll(m)) != i) return false;
        return true;
    };
    auto take = [&](Heads &hd, int i) {
        for (uint64_t m = bits[i]; m; m &= m - 1) hd[__builtin_ctzll(m)]++;
    };
    // the ready gate that fits a block on mask and adds the fewest qubits
    // (the earliest on ties), or -1; each gate is seen at its lowest qubit
    auto next_min = [&](const Heads &hd, uint64_t mask, int &add) {
        int pick = -1;
        add = 65;
        for (int q = 0; q < nq; q++) {
            const int i = front(hd, q);
            if (i < 0 || __builtin_ctzll(bits[i]) != q || popc(bits[i] | mask) > k) continue;
            const int a = popc(bits[i] & ~mask);
            if (a > add || (a == add && i > pick) || !ready(hd, i)) continue;
            add = a;
            pick = i;
        }
        return pick;
    };
    // gates the fewest-qubits-first rule would still add to a block (at most cap)
    constexpr int kLookCap = 1024;
    auto greedy_count = [&](Heads hd, uint64_t mask) {
        int c = 0, add;
        for (int i; c < kLookCap && (i = next_min(hd, mask, add)) >= 0; c++) {
            mask |= bits[i];
            take(hd, i);
        }
        return c;
    };
    struct Node {
        uint64_t mask;
        Heads hd;
        std::vector<int> picks;
        int score;
    };
    // every ready gate inside the node's qubits (the block's final gate set
    // depends only on its qubit set)
    auto close = [&](Node &nd) {
        int add, i;
        while ((i = next_min(nd.hd, nd.mask, add)) >= 0 && add == 0) {
            take(nd.hd, i);
            nd.picks.push_back(i);
        }
    };
    Heads head{};
    std::vector<char> placed((size_t)ng, 0);
    int first = 0;
    for (;;) {
        while (first < ng && placed[first]) first++;
        if (first == ng) break;
        Node best{0, head, {}, 0};
        int pick = first;
        while (pick >= 0) {
            best.mask |= bits[pick];
            best.picks.push_back(pick);
            take(best.hd, pick);
            int add;
            pick = next_min(best.hd, best.mask, add);  // gates inside the block's qubits come first
            if (pick < 0 || add == 0) continue;
            // a gate adding qubits: the one after which the block takes the
            // most gates (fewer added qubits, then the earliest, on ties)
            int best_cnt = -1, best_add = 65;
            for (int q = 0; q < nq; q++) {
                const int i = front(best.hd, q);
                if (i < 0 || __builtin_ctzll(bits[i]) != q || popc(bits[i] | best.mask) > k || !ready(best.hd, i))
                    continue;
                Heads h2 = best.hd;
                take(h2, i);
                const int cnt = greedy_count(h2, best.mask | bits[i]);
                const int a = popc(bits[i] & ~best.mask);
                if (cnt > best_cnt || (cnt == best_cnt && (a < best_add || (a == best_add && i < pick)))) {
                    best_cnt = cnt;
                    best_add = a;
                    pick = i;
                }
            }
        }
        if (beam > 0) {
            Node root{bits[first], head, {first}, 0};
            take(root.hd, first);
            close(root);
            root.score = (int)root.picks.size() + greedy_count(root.hd, root.mask);
            if (root.picks.size() > best.picks.size()) best = root;
            std::vector<Node> level{root}, next;
            while (!level.empty()) {
                next.clear();
                for (const Node &nd : level)
                    for (int q = 0; q < nq; q++) {
                        const int i = front(nd.hd, q);
                        if (i < 0 || __builtin_ctzll(bits[i]) != q || popc(bits[i] | nd.mask) > k || !ready(nd.hd, i))
                            continue;
                        const uint64_t m2 = nd.mask | bits[i];
                        bool seen = false;
                        for (const Node &o : next) seen = seen || o.mask == m2;
                        if (seen) continue;
                        Node c = nd;
                        c.mask = m2;
                        take(c.hd, i);
                        c.picks.push_back(i);
                        close(c);
                        c.score = (int)c.picks.size() + greedy_count(c.hd, c.mask);
                        if (c.picks.size() > best.picks.size()) best = c;
                        next.push_back(std::move(c));
                    }
                std::stable_sort(next.begin(), next.end(), [](const Node &x, const Node &y) { return x.score > y.score; });
                if ((int)next.size() > beam) next.resize((size_t)beam);
                level.swap(next);
            }
        }
        for (int i : best.picks) placed[i] = 1;
        head = best.hd;
        out.push_back(BlockDraft{std::move(best.picks), best.mask});
    }
}

}  // namespace

bool plan_fused(const std::vector<PGate> &gates, int n, int k, std::vector<FusedBlock> &out, bool search) {
    out.clear();
    const int ng = (int)gates.size();
    std::vector<uint64_t> bits((size_t)ng);
    std::vector<std::vector<int>> queue(64);  // per qubit: the gates touching it, in circuit order
    for (int i = 0; i < ng; i++) {
        bits[i] = block_bits(gates[i]);
        if (popc(bits[i]) > k) return false;
        for (uint64_t m = bits[i]; m; m &= m - 1) queue[__builtin_ctzll(m)].push_back(i);
    }
    // the greedy grouping, and with search the one that also tries the beam's
    // blocks: the one with fewer blocks is kept (the greedy one on ties)
    std::vector<BlockDraft> plan, alt;
    draft_blocks(bits, queue, k, 0, plan);
    if (search) {
        draft_blocks(bits, queue, k, kBlockBeam, alt);
        if (alt.size() < plan.size()) plan.swap(alt);
    }
    std::vector<const PGate *> cur;
    for (const BlockDraft &d : plan) {
        cur.clear();
        for (int i : d.picks) cur.push_back(&gates[i]);
        emit_block(cur, d.mask, n, k, out);
    }
    return true;
}

bool fused_geometry(int n, int k, const int *pos, TileGeom &g, FusedMap &fm) {
    const int T = k + 7;
    if (n < T || k > 8) return false;
    uint64_t F = 0;
    for (int j = 0; j < k; j++) F |= 1ull << pos[j];
    int L = T < 11 ? T : 11;  // bulk copies of at most 16 KiB
    while (L > 1 && L + __builtin_popcountll(F & ~((1ull << L) - 1ull)) > T) L--;
    uint64_t hm = F & ~((1ull << L) - 1ull);
    for (int b = L; b < n && __builtin_popcountll(hm) < T - L; b++)
        if (!((F >> b) & 1ull)) hm |= 1ull << b;
    if (__builtin_popcountll(hm) != T - L || T - L > 10) return false;
    g = TileGeom{};
    g.n = n;
    g.L = L;
    g.H = T - L;
    int h = 0;
    for (int b = 0; b < 64; b++)
        if ((hm >> b) & 1ull) g.hb[h++] = b;
    auto local = [&](int b) {
        if (b < L) return b;
        for (int j = 0; j < g.H; j++)
            if (g.hb[j] == b) return L + j;
        return -1;
    };
    uint32_t colmask = 0;
    for (int j = 0; j < k; j++) {
        fm.col[j] = (int8_t)local(pos[j]);
        colmask |= 1u << fm.col[j];
    }
    int r = 0;
    for (int b = 0; b < T; b++)
        if (!((colmask >> b) & 1u)) fm.row[r++] = (int8_t)b;
    return r == T - k;
}

bool phase_term(const PGate &g, uint64_t &turns, uint64_t &bits) {
    if (g.kind == QSIM_GATE_SWAP || popc(g.cmask) > 1) return false;
    const Mat2 &M = g.U;
    if (M.u[2] != 0.0 || M.u[3] != 0.0 || M.u[4] != 0.0 || M.u[5] != 0.0) return false;
    if (std::fabs(M.u[0] - 1.0) > 1e-15 || std::fabs(M.u[1]) > 1e-15) return false;
    if (std::fabs(std::hypot(M.u[6], M.u[7]) - 1.0) > 1e-14) return false;
    // turns in (-1/2, 1/2] as a signed 64-bit fraction of 2^63, kept mod 2^64
    const double v = std::ldexp(std::atan2(M.u[7], M.u[6]) / M_PI, 63);
    turns = v >= 9223372036854775808.0 ? (1ull << 63) : (uint64_t)(int64_t)std::llround(v);  // pi == -pi
    bits = g.cmask | (1ull << g.t0);
    return true;
}

namespace {

// The tables of one run of phase shifts.
void build_phase_pass(const std::vector<PGate> &run, PhasePass &pp) {
    std::vector<int> slot(64 * 64, -1);
    for (const PGate &g : run) {
        uint64_t turns, bits;
        phase_term(g, turns, bits);
        int b[2] = {0, 0}, nb = 0;  // a phase term has one or two bits
        for (uint64_t m = bits; m && nb < 2; m &= m - 1) b[nb++] = __builtin_ctzll(m);
        const int ca = b[0] / kPhaseChunk, cb = (nb == 2 ? b[1] : b[0]) / kPhaseChunk;  // ca <= cb
        int &t = slot[ca * 64 + cb];
        if (t < 0) {
            t = (int)pp.ta.size();
            pp.ta.push_back((int8_t)ca);
            pp.tb.push_back((int8_t)cb);
            pp.words.resize(pp.words.size() + kPhaseTableWords, 0ull);
        }
        uint64_t *w = pp.words.data() + (size_t)t * kPhaseTableWords;
        // local bit masks within the chunks; entry index xa + 32 xb (xa when ca = cb)
        uint32_t ma = 0, mb = 0;
        for (int j = 0; j < nb; j++) {
            if (b[j] / kPhaseChunk == ca) ma |= 1u << (b[j] % kPhaseChunk);
            else mb |= 1u << (b[j] % kPhaseChunk);
        }
        const int span = ca == cb ? (1 << kPhaseChunk) : kPhaseTableWords;
        for (int e = 0; e < span; e++) {
            const uint32_t xa = (uint32_t)e & 31u, xb = (uint32_t)e >> kPhaseChunk;
            if ((xa & ma) == ma && (xb & mb) == mb) w[e] += turns;
        }
        pp.gates++;
    }
}

}  // namespace

// chunk pairs of a set of phase terms
static int phase_tables(const std::vector<PGate> &run) {
    std::vector<char> seen(64 * 64, 0);
    int c = 0;
    for (const PGate &g : run) {
        uint64_t turns, bits;
        phase_term(g, turns, bits);
        const int lo = __builtin_ctzll(bits), hi = 63 - __builtin_clzll(bits);
        char &s = seen[(lo / kPhaseChunk) * 64 + hi / kPhaseChunk];
        if (!s) {
            s = 1;
            c++;
        }
    }
    return c;
}

bool plan_fused_phases(const std::vector<PGate> &gates, int n, int k, int min_gates, int max_tables,
                       std::vector<FusedBlock> &out, std::vector<PhasePass> &phases, bool search) {
    std::vector<FusedBlock> plain;
    if (!plan_fused(gates, n, k, plain, search)) return false;
    // Runs: phase shifts are held back while the gates after them commute
    // with them (none targets one of their bits); a gate that does not
    // commute releases the whole held set before it -- as one run if it is
    // long, else as ordinary gates.
    std::vector<std::vector<PGate>> segs(1), runs;
    std::vector<PGate> held;
    uint64_t held_bits = 0;
    auto release = [&]() {
        if ((int)held.size() >= min_gates && popc(held_bits) > k && phase_tables(held) <= max_tables) {
            runs.push_back(held);
            segs.emplace_back();
        } else {
            segs.back().insert(segs.back().end(), held.begin(), held.end());
        }
        held.clear();
        held_bits = 0;
    };
    for (const PGate &g : gates) {
        uint64_t turns, bits;
        if (phase_term(g, turns, bits) && (int)runs.size() < 64) {
            held.push_back(g);
            held_bits |= bits;
            continue;
        }
        uint64_t moved = 1ull << g.t0;  // the bits g changes (a diagonal g changes none)
        if (g.kind == QSIM_GATE_SWAP) moved |= 1ull << g.t1;
        else if (g.U.u[2] == 0.0 && g.U.u[3] == 0.0 && g.U.u[4] == 0.0 && g.U.u[5] == 0.0) moved = 0;
        if (moved & held_bits) release();
        segs.back().push_back(g);
    }
    release();
    if (runs.empty() || (size_t)(n + kPhaseChunk - 1) / kPhaseChunk > 8) {
        out = std::move(plain);
        return true;
    }
    std::vector<FusedBlock> with;
    std::vector<PhasePass> pps;
    for (size_t s = 0; s < segs.size(); s++) {
        std::vector<FusedBlock> part;
        if (!plan_fused(segs[s], n, k, part, search)) return false;
        for (FusedBlock &b : part) with.push_back(std::move(b));
        if (s < runs.size()) {
            PhasePass pp;
            build_phase_pass(runs[s], pp);
            FusedBlock mark;
            mark.k = k;
            for (int j = 0; j < 8; j++) mark.pos[j] = j < k ? j : 0;
            mark.flops = 8.0 * std::ldexp(1.0, n);  // one complex product per amplitude
            mark.phase = (int)pps.size();
            with.push_back(std::move(mark));
            pps.push_back(std::move(pp));
        }
    }
    if (with.size() < plain.size()) {
        out = std::move(with);
        phases = std::move(pps);
    } else {
        out = std::move(plain);
        phases.clear();
    }
    return true;
}

}  // namespace qsim
