// planner.hpp -- host-side gate preparation and pass planning.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "kernels.hpp"

namespace qsim {

// A gate after validation: physical bit positions and an FP64 matrix.
struct PGate {
    int kind;           // QSIM_GATE_SWAP or a 2x2 gate
    int t0, t1;         // physical target bit(s); t1 = -1 unless SWAP
    uint64_t cmask;     // physical control bits
    int gc;             // GateClass of the 2x2 matrix (unused for SWAP)
    Mat2 U;
};

// Build the 2x2 matrix of a gate kind from its parameters (Sec. II);
// returns false for an unknown kind.
bool gate_matrix(int kind, const double *param, Mat2 &M);
// Class of a 2x2 matrix from exact zero / one entries.
int classify(const Mat2 &M);

// Validate a logical gate against n qubits and map it to physical bits with
// phys[q] = bit of logical qubit q.  On error returns false and sets msg.
bool prepare_gate(const qsim_gate &g, int n, const int *phys, PGate &out, std::string &msg);

// Enumeration bits of a per-gate sweep: target(s) and controls as fixed bits.
void fixed_bits_for(const PGate &g, FixedBitsHost &fb, uint64_t &pmask, bool &single);

struct PassPlan {
    TileGeom geom;
    int op_begin, op_count;       // range in the plan's op array
    int phase_begin, phase_count; // range in the plan's phase array (0 phases: shared-memory kernel)
    double flops;                 // algorithmic flops of the pass
    bool arith;                   // some op does arithmetic (not only data movement)
    // complex128 shared-memory passes (hoist_global_diagonals): the last
    // nglob ops of the range are diagonal ops on bits outside the tile, one
    // factor per tile; absorber >= 0 names the op of the program whose
    // coefficients take that factor each tile (else a separate multiply)
    int nglob = 0;
    int absorber = -1;
};

// Algorithmic real flops of one gate over an n-qubit state: 14 per amplitude
// for a dense 2x2 (two complex multiply-adds per output), 6 for a diagonal or
// anti-diagonal entry (one complex multiply), 0 for pure data movement,
// times the fraction of amplitudes the controls select (and 1/2 for a phase
// shift, which leaves the bit-0 half alone).
double gate_flops(const PGate &g, int n);

struct Plan {
    std::vector<PassPlan> passes;
    std::vector<TileOp> ops;
    std::vector<TilePhase> phases;
    std::vector<double> dense;   // matrix pool for TOP_DENSE (complex, interleaved)
};

// Greedy tile planner: tiles of T bits, the L lowest always included.
// Gates are taken in order; a gate can join the current pass if it commutes
// with every gate skipped so far (no shared qubit) and its targets fit in the
// tile's bit set (diagonal gates need no target in the tile).
// RB > 0: cut each pass with T = RB + 5 + kRegWarpBits bits into register phases for the
// register-blocked kernel (k_tile2.cu); passes that do not fit that shape
// keep a flat op list for the shared-memory kernel (k_tile.cu).
// max_ops / max_phases > 0: a pass takes only as many of its gates (in order)
// as keep its op list, and the phase list of a register pass, within them;
// the rest go to later passes.
void plan_tiles(const std::vector<PGate> &gates, int n, int T, int L, Plan &plan, int RB = 0, int max_ops = 0,
                int max_phases = 0);

// complex128 shared-memory passes (k_tile_df.cu): in every pass without
// register phases, uncontrolled Hadamard-type ops s*[[1,1],[1,-1]] (at most
// kMaxDeferred of them) become unscaled butterflies (pk = 4) and the product
// of their factors s is folded into one op of the same pass that touches
// every amplitude exactly once: an uncontrolled 2x2 pair op or diagonal, else
// one of the Hadamard-type ops, which then keeps its real 2x2 form.
constexpr int kMaxDeferred = 24;  // bounds the growth of the unscaled amplitudes to 2^12
void defer_butterflies(Plan &plan);

// complex128 shared-memory passes (after defer_butterflies): an uncontrolled
// phase or diagonal on a local bit b merges into the nearest uncontrolled op
// on b before it (else after it) that keeps its kind and cost when multiplied
// by it -- a dense complex 2x2, a phase or a diagonal -- provided no op in
// between moves or mixes amplitudes along b (diagonal ops and controls on b
// commute with it).  The merged op's FP64 matrix is the product.
void merge_local_diagonals(Plan &plan);

// complex128 shared-memory passes: every op that is diagonal on a bit outside
// the tile and has no control inside it (TOP_DIAG_G, lcmask == 0) scales a
// whole tile by one factor, and commutes with every op of the pass (no op of
// a pass acts non-diagonally outside its tile).  They move to the end of the
// pass's op range (nglob of them); the kernel multiplies them into one factor
// per tile and folds it into the coefficients of one uncontrolled op that
// touches every amplitude once and stays of its kind when scaled by a complex
// number (dense 2x2, anti-diagonal or diagonal), the pass's absorber.
void hoist_global_diagonals(Plan &plan);

// Cut one pass's op list into register phases (see k_tile2.cu).
void build_phases(const std::vector<TileOp> &pass_ops, int T, int RB, std::vector<TileOp> &ops_out,
                  std::vector<TilePhase> &phases_out);

// Dense fusion: the gates grouped into blocks acting on at most k qubits;
// each block's 2^k x 2^k unitary is the FP64 product of its gates.  A block
// starts at the earliest gate not yet placed and keeps taking a gate whose
// earlier gates on each of its qubits are all placed (so it moves only past
// gates on other qubits, which commute with it): gates inside the block's
// qubits first, else the gate after which the fewest-qubits-first rule would
// add the most gates (one step of lookahead).  False if a gate acts on more
// than k qubits.
struct FusedBlock {
    int k;
    int pos[8];               // physical bits, bit j of U's index = pos[j]
    std::vector<double> U;    // 2^k x 2^k complex, row-major (re, im)
    double flops;             // algorithmic flops: 8 * 2^k per amplitude
    int phase = -1;           // >= 0: not a dense block but phase pass number `phase` (PhasePass)
};
// With search, a second grouping whose blocks may instead come from a beam
// search over the qubit sets a block can grow into (planner.cpp,
// draft_blocks) is made too, and the one with fewer blocks is kept.
bool plan_fused(const std::vector<PGate> &gates, int n, int k, std::vector<FusedBlock> &out, bool search = true);

// Phase passes.  Phase shifts with up to one control, diag(1, e^(i phi)) on
// a target with its control (Eqs. NUM5 and COMM5), commute with each other and
// with every gate whose target is none of their bits.  A long run of them
// (the controlled phases of the QFT adders between two registers, Sec. V.A)
// spreads over many dense blocks but is one diagonal operator: the phase of
// amplitude x is the sum over the gates whose bits are all 1 in x.  The index
// bits are cut into chunks of kPhaseChunk bits (kernels.hpp); a gate's bits lie in one or
// two chunks, so the sum is a sum of table entries, one table per chunk pair
// (a, b) with a <= b, indexed by x_a + 32 x_b (x_a alone when a = b).  The
// entries are fixed-point turns (phi / 2 pi times 2^64, summed mod 2^64;
// complex64 passes use their top 32 bits).
struct PhasePass {
    std::vector<int8_t> ta, tb;    // chunk pair of table t, ta <= tb
    std::vector<uint64_t> words;   // kPhaseTableWords per table
    int gates = 0;
};
// The phase-shift gate's term (turns as fixed point, bit set); false if the
// gate is not diag(1, e^(i phi)) with at most one control.
bool phase_term(const PGate &g, uint64_t &turns, uint64_t &bits);
// plan_fused, with every long run of commuting phase shifts (at least
// min_gates of them over more than k qubits, on at most max_tables chunk
// pairs) taken out as a phase pass where that gives fewer passes in all;
// blocks with phase >= 0 stand for phases[phase].
bool plan_fused_phases(const std::vector<PGate> &gates, int n, int k, int min_gates, int max_tables,
                       std::vector<FusedBlock> &out, std::vector<PhasePass> &phases, bool search = true);

// Tile geometry of a fused block on the tensor cores: T = k + 7 bits holding
// the block's qubits; false if n is too small.
bool fused_geometry(int n, int k, const int *pos, TileGeom &g, FusedMap &fm);

// Translate one gate into a tile op for a pass with geometry g.
bool make_tile_op(const PGate &pg, const TileGeom &g, TileOp &op);

}  // namespace qsim
