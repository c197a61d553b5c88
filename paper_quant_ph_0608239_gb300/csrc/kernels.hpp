// kernels.hpp -- launch interface between the host runtime (capi.cu,
// planner.cpp) and the CUDA kernels.  Plain structs, no CUDA types beyond
// cudaStream_t / cudaError_t.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "perm_layout.hpp"

namespace qsim {

constexpr int kMaxQubits = 34;

// How a 2x2 gate touches a pair (a0, a1) -- chosen on the host from the
// matrix entries so that no kernel does arithmetic the gate does not need.
enum GateClass : int32_t {
    GC_GENERAL = 0,   // dense 2x2
    GC_DIAG = 1,      // diag(u00, u11): every amplitude scaled, no partner
    GC_PHASE = 2,     // diag(1, u11): only the bit-1 half scaled (Eq. NUM5)
    GC_ANTIDIAG = 3,  // a'0 = u01 a1, a'1 = u10 a0
    GC_EXCHANGE = 4,  // a'0 = a1, a'1 = a0 (CNOT / Toffoli flip, Eqs. NUM6, NUM8)
    GC_REAL = 5       // dense 2x2 with real entries (H, Y, Ybar): half the multiplies
};

struct Mat2 {
    double u[8];      // row-major (re, im): u00, u01, u10, u11
};

// ------------------------------------------------------------ tile programs
// One operation applied to every tile of a tile pass.  Bit positions named
// "local" index the tile (0..T-1: first the L low bits, then the H high tile
// bits in ascending physical order); "global" masks use physical positions
// outside the tile and are tested once per tile.
enum TileOpKind : int32_t {
    TOP_GENERAL = 0,   // 2x2 on local bit tl
    TOP_DIAG = 1,      // diag on local bit tl
    TOP_PHASE = 2,     // diag(1, u11) on local bit tl
    TOP_ANTIDIAG = 3,
    TOP_EXCHANGE = 4,
    TOP_DIAG_G = 5,    // diag on a physical bit tl outside the tile: one factor per tile
    TOP_SWAPGATE = 6,  // quantum SWAP of local bits tl, tl2
    TOP_PERM = 7,      // exchange local bit pairs (pl[k], ph[k]), k < nperm: a layout change
    TOP_DENSE = 8      // dense 2^k x 2^k on local bits pl[0..k-1] (k = nperm), matrix at dense_off
};

struct TileOp {
    int32_t kind;
    int32_t tl;
    int32_t tl2;
    int32_t nperm;
    uint32_t lcmask;   // local control bits
    uint32_t dense_off;  // TOP_DENSE: offset (in complex entries) into the pass's matrix pool
    uint64_t gcmask;   // global control bits (physical)
    double u[8];
    int8_t pl[8];
    int8_t ph[8];
    // register-blocked kernel (k_tile2.cu), filled by the planner per phase
    int8_t regk;      // register slot of the target bit; -1 if it is a lane/warp bit (or outside the tile)
    int8_t pk;        // pair kind: 0 general, 1 real, 2 anti-diagonal, 3 exchange
    uint8_t code;     // register kernel dispatch: family * 8 + slot (RC_* below)
    int8_t cslot;     // unused (0)
    uint32_t creg;    // controls among the register slots (bit k = slot k)
    uint32_t lcthr;   // controls among the lane and warp bits (local index mask)
    uint32_t pad32;
    float uh[8];      // u[] rounded to float (complex64) ...
    float ul[8];      // ... and the remainders (complex128 double-float coefficients)
};
static_assert(sizeof(TileOp) == 192, "TileOp layout");

// Op families of the register kernel (TileOp::code = family * 8 + k, k = the
// target's register slot unless noted).  The host picks the family so the
// kernel applies each op with compile-time register indices.
enum RegFamily : int {
    RC_GEN = 0,     // dense 2x2, no local controls
    RC_REAL = 1,    // real 2x2, no local controls
    RC_GENC = 2,    // dense 2x2 with controls
    RC_REALC = 3,   // real 2x2 with controls
    RC_ANTI = 4,    // anti-diagonal, any controls
    RC_EXCHC = 5,   // bit flip with controls
    RC_PHASE = 6,   // diag(1, u11) on a register bit, any controls
    RC_DIAG = 7,    // diag(u00, u11) on a register bit, any controls
                    // (8: unused)
    RC_LANE = 9,    // pair op on a lane bit (tl), no local controls; k = pair kind
    RC_LANEC = 10,  // pair op on a lane bit with controls; k = pair kind
    RC_THR = 11,    // phase (k = 0) or diagonal (k = 1) on a lane/warp bit (tl)
    RC_GLOB = 12    // diagonal on a bit outside the tile (tl = physical bit)
};

// Warp bits of the register-blocked kernel (k_tile2.cu): a block has
// 2^kRegWarpBits warps, and a tile of T bits holds 5 lane bits, kRegWarpBits
// warp bits and T - 5 - kRegWarpBits register bits.
#ifndef QSIM_T2_NWB
#define QSIM_T2_NWB 3
#endif
constexpr int kRegWarpBits = QSIM_T2_NWB;

// Capacity of the shared-memory copies of one register pass's program (ops
// and phases) in k_tile2.cu and k_batch.cu.  The planner keeps every register
// pass (and every pass of a batch) within it, so the kernels read ops and
// phases from shared memory only.
constexpr int kRegMaxOps = 64;
constexpr int kRegMaxPhases = 32;

// One phase of a register-blocked tile program: which local bits are held in
// registers, the ops it applies, and an optional permutation of local bit
// pairs applied when the phase stores back (quantum SWAP gates, interchanges).
struct TilePhase {
    int32_t op_begin, op_count;
    int8_t rb[8];     // register slot k -> local bit (>= 5)
    int8_t wb[8];     // warp bit k -> local bit (>= 5)
    int32_t nperm;
    int8_t pl[8];
    int8_t ph[8];
};

constexpr int kMaxTileHigh = 16;
struct TileGeom {
    int32_t n;
    int32_t L;         // low bits 0..L-1 always in the tile
    int32_t H;         // number of high tile bits
    int32_t hb[kMaxTileHigh];  // physical positions of the high tile bits, ascending, >= L
};

// Local bit layout of a fused-gate tile (k_fused_tc.cu): row[b] = local bit
// of row-index bit b (the groups), col[j] = local bit of the gate's qubit j.
struct FusedMap {
    int8_t row[16];
    int8_t col[8];
};

// ------------------------------------------------------------ launchers
// dt: 0 = complex64, 1 = complex128.  All return the launch error.
struct FixedBitsHost {
    int npos;
    int pos[24];
    uint64_t setmask;
};

cudaError_t launch_init_basis(void *amp, int dt, int n, uint64_t x, cudaStream_t s);

// Eq. Shor2 state: zero, then a_{x + 2^X (y^x mod G)} = 2^(-X/2) for x < 2^X.
cudaError_t launch_shor_state(void *amp, int dt, int n, int X, uint64_t y, uint64_t G, cudaStream_t s);

// Pair sweep: enumerate i0 = expand(p, fb) for p < 2^(n - fb.npos), partner
// i1 = i0 ^ pmask, apply the gate class gc with matrix U.
cudaError_t launch_pairs(void *amp, int dt, int n, const FixedBitsHost &fb, uint64_t pmask, int gc,
                         const Mat2 &U, cudaStream_t s);

// Single-amplitude sweep for diagonal classes: enumerate i = expand(p, fb),
// scale by u00 (bit tbit of i is 0) or u11 (bit tbit is 1).
cudaError_t launch_diag(void *amp, int dt, int n, const FixedBitsHost &fb, int tbit, const Mat2 &U,
                        cudaStream_t s);

// Dense k-qubit gate on CUDA cores: qpos[j] = physical bit for bit j of U's
// index, U (device, 4^k complex in the state's precision, row-major).
cudaError_t launch_dense(void *amp, int dt, int n, int k, const int *qpos, const void *dU, cudaStream_t s);

// One tile pass (shared-memory program).  ops/dmat are device pointers.
// err: device word set on a bounded-wait timeout.
cudaError_t launch_tile_pass(void *amp, int dt, const TileGeom &g, const TileOp *ops, int nops,
                             const void *dmat, uint32_t *err, int sm_count, cudaStream_t s);

// Register-blocked tile pass (k_tile2.cu), complex64: T = 5 lane bits +
// kRegWarpBits warp bits + register bits = 12 or 13, L >= 5 (the lane bits
// are the physical bits 0..4).
bool tile2_supported(int dt, int T);

// complex128 tile pass in double-float arithmetic (k_tile_df.cu).  cvt_in:
// the tile arrives as IEEE doubles and is converted after the load; cvt_out:
// it is converted back to IEEE doubles before the store.  Without them the
// pass reads / writes the double-float form (re.h, re.l, im.h, im.l), which a
// run keeps in HBM between its arithmetic passes.  Passes that only move data
// take neither (bit-exact in either form).  Ops with pk == 4 are unscaled
// butterflies (a0 + a1, a0 - a1), see defer_butterflies().  ops[0, nops) is
// the program; ops[nops, nops + nglob) are diagonal ops on bits outside the
// tile, multiplied into one factor per tile and folded into the coefficients
// of program op `absorber` (or, if absorber < 0, applied as one multiply).
cudaError_t launch_tile_pass_df(void *amp, const TileGeom &g, const TileOp *ops, int nops, int nglob, int absorber,
                                bool cvt_in, bool cvt_out, uint32_t *err, int sm_count, cudaStream_t s);
// ops: the plan's op array; the pass's phases use ops[op_base, op_base + op_count).
cudaError_t launch_tile_pass2(void *amp, int dt, const TileGeom &g, const TilePhase *phases, int nphases,
                              const TileOp *ops, int op_base, int op_count, uint32_t *err, int sm_count,
                              cudaStream_t s);

// Dense k-qubit gate on the tensor cores (k_fused_tc.cu, complex64, k = 4
// or 5, n >= k + 7): tile T = k + 7 bits containing the k qubits; bmat =
// device copy of fused_tc_prepare_b's output (2 * (2^(k+1))^2 floats).
bool fused_tc_supported(int dt, int k, int n);
void fused_tc_prepare_b(int k, const double *U, float *out);
cudaError_t launch_fused_tc(void *amp, int k, const TileGeom &g, const FusedMap &fm, const float *bmat,
                            uint32_t *err, int sm_count, cudaStream_t s);

// Dense 5-qubit gate on the tensor cores for complex128 (k_fused_tc_c128.cu:
// bf16 digit slices, exact level sums; n >= 12): bmat = device copy of
// fused_tc128_prepare_b's output (fused_tc128_b_bytes() bytes), which
// returns false for a matrix the scheme cannot take exactly (an entry
// outside (-2, 2)).  in_ieee / out_ieee: the state is read / written as
// IEEE doubles, else in the double-float form kept between the blocks of a
// run (re.hi, re.lo, im.hi, im.lo as floats).
bool fused_tc128_supported(int k, int n);
size_t fused_tc128_b_bytes();
bool fused_tc128_prepare_b(const double *U, uint16_t *out);
cudaError_t launch_fused_tc128(void *amp, const TileGeom &g, const FusedMap &fm, const uint16_t *bmat,
                               uint32_t *err, int sm_count, cudaStream_t s, bool in_ieee, bool out_ieee);

// Dense 6-qubit gate on the tensor cores for complex64 (k_fused_tc6.cu: bf16
// hi/mid/lo slices, six products, FP32 accumulation; n >= 13): bmat = device
// copy of fused_tc6_prepare_b's output (fused_tc6_b_bytes() bytes).
bool fused_tc6_supported(int n);
size_t fused_tc6_b_bytes();
void fused_tc6_prepare_b(const double *U, uint16_t *out);
cudaError_t launch_fused_tc6(void *amp, const TileGeom &g, const FusedMap &fm, const uint16_t *bmat, uint32_t *err,
                             int sm_count, cudaStream_t s);

// ------------------------------------------------------------ interchange
// K pairs of local (tile) bits exchanged by the interchange pass
// (k_permute.cu): PermPairs in perm_layout.hpp; launch_permute fills its
// lane and skew layout.  Needs T = g.L + g.H >= 8, g.H <= kPermMaxH, g.L >= 1.
// Tile bits of the interchange pass for elements of elem_bytes (8 or 16).
int permute_tile_bits(int elem_bytes);
cudaError_t launch_permute(void *amp, int elem_bytes, const TileGeom &g, const PermPairs &pp, uint32_t *err,
                           int sm_count, cudaStream_t s);

// ------------------------------------------------------------ phase passes
// A run of commuting phase shifts applied in one pass (k_phase.cu; tables
// built by the planner, planner.hpp PhasePass): ntab tables of
// kPhaseTableWords fixed-point turns, table t for the chunk pair (ta[t],
// tb[t]), ta <= tb, chunk c = index bits kPhaseChunk c .. kPhaseChunk c + 4.
constexpr int kPhaseChunk = 5;
constexpr int kPhaseTableWords = 1 << (2 * kPhaseChunk);
constexpr int kMaxPhaseTables = 36;  // chunk pairs of 8 chunks (n <= 40)
struct PhaseMeta {
    int32_t ntab;
    int8_t ta[kMaxPhaseTables];
    int8_t tb[kMaxPhaseTables];
};
// n >= 10; tables: device copy of ntab * kPhaseTableWords words.
cudaError_t launch_phase_pass(void *amp, int n, const uint32_t *tables, const PhaseMeta &m, int sm_count,
                              cudaStream_t s);
// complex128, double-float arithmetic: 64-bit turns, ntab <= 24.  The state
// is read as IEEE doubles if in_ieee, else in the double-float form of the
// tensor-core blocks (re.h, re.l, im.h, im.l floats in the amplitude's 16
// bytes), and written as IEEE doubles if out_ieee, else double-float.
cudaError_t launch_phase_pass128(void *amp, int n, const uint64_t *tables, const PhaseMeta &m, int sm_count,
                                 cudaStream_t s, bool in_ieee, bool out_ieee);

// ------------------------------------------------------------ batches
struct BatchCircuit {
    void *amp;            // complex64 state of the circuit
    uint64_t x0;          // initial basis state
    int32_t pass_begin;   // first pass in the batch's pass array (and done-counter index)
    int32_t npasses;
};
struct BatchPass {
    TileGeom geom;
    int32_t op_begin, op_count;        // in the batch's op array
    uint32_t ntiles;
    int32_t phase_begin, phase_count;  // register phases (tile2_engine.cuh) in the batch's
                                       // phase array; 0 phases: the shared-memory program
};
struct BatchItem {
    uint32_t circuit, pass, tile;
};
// counters: one 64-bit item counter (zeroed before the launch); done: one
// zeroed counter per pass of the batch.  budget: SM cycles a wait may take.
cudaError_t launch_batch(const BatchCircuit *circs, const BatchPass *passes, const TileOp *ops,
                         const TilePhase *phases, const BatchItem *items, uint64_t nitems, uint32_t *counters,
                         uint32_t *done, uint32_t *err, long long budget, int sm_count, cudaStream_t s);
// register bits of the batch's 12-bit tiles (the register phases' shape)
constexpr int kBatchRB = 12 - 5 - kRegWarpBits;

// Reductions (FP64 accumulation).  scratch: device buffer of at least
// reduce_scratch_bytes(n) bytes.
size_t reduce_scratch_bytes(int n);
cudaError_t launch_norm(const void *amp, int dt, int n, double *scratch, double *dout, cudaStream_t s);
// dout[b] = P(physical bit b = 1), b < n
cudaError_t launch_bit_probs(const void *amp, int dt, int n, double *scratch, double *dout, cudaStream_t s);
// dout[j] = |a[phys(start + j)]|^2 for j < count, phys(x) = deposit of the
// logical bits of x onto physpos[q]
cudaError_t launch_probs_chunk(const void *amp, int dt, int n, const int *physpos, bool identity,
                               uint64_t start, uint64_t count, double *dout, cudaStream_t s);
// dout[j] = a[phys(start + j)] (amplitude gather to logical order)
cudaError_t launch_gather_chunk(const void *amp, int dt, int n, const int *physpos, uint64_t start,
                                uint64_t count, void *dout, cudaStream_t s);

// Per-bit marginals on the library's static scratch array instead of a
// caller buffer (no device allocation); see k_reduce.cu.
cudaError_t launch_bit_probs_noalloc(const void *amp, int dt, int n, double *dout, cudaStream_t s);

// Sampling (Sec. V.B): block sums of |a|^2 in logical order, then per-sample
// search.  scratch must hold sample_scratch_bytes(n) bytes.
size_t sample_scratch_bytes(int n);
cudaError_t launch_sample(const void *amp, int dt, int n, const int *physpos, bool identity,
                          const double *du, size_t ns, uint64_t *dout, double *scratch, cudaStream_t s);

}  // namespace qsim
