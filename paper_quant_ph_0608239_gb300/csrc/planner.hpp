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
void plan_tiles(const std::vector<PGate> &gates, int n, int T, int L, Plan &plan, int RB = 0);

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
};
bool plan_fused(const std::vector<PGate> &gates, int n, int k, std::vector<FusedBlock> &out);

// Tile geometry of a fused block on the tensor cores: T = k + 7 bits holding
// the block's qubits; false if n is too small.
bool fused_geometry(int n, int k, const int *pos, TileGeom &g, FusedMap &fm);

// Translate one gate into a tile op for a pass with geometry g.
bool make_tile_op(const PGate &pg, const TileGeom &g, TileOp &op);

}  // namespace qsim
