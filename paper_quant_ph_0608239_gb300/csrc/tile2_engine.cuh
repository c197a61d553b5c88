// tile2_engine.cuh -- the register-blocked gate program of one tile (used by
// the tile passes of k_tile2.cu and the batch kernel of k_batch.cu).
//
// A tile of 2^T amplitudes sits in shared memory.  A phase names RB register
// bits and kRegWarpBits warp bits (the lane bits are tile bits 0..4): every
// thread loads the 2^RB amplitudes its lane and warp bits select, applies the
// phase's ops to them in registers (pairs on a register bit inside a thread,
// pairs on a lane bit through warp shuffles, diagonal ops anywhere) and
// stores them back, optionally to permuted positions.
#pragma once

#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"

namespace qsim {
namespace t2 {

// ---------------------------------------------------------- amplitude types
template <bool C128> struct AmpT;
template <> struct AmpT<false> {
    using V = float2;
    using S = float2;  // shared-memory element
};
template <> struct AmpT<true> {
    using V = dcx;
    using S = double2;
};

// coefficients of one 2x2 entry
template <bool C128> struct Coef;
template <> struct Coef<false> { float2 c; };
template <> struct Coef<true> { dcx c; };

__device__ __forceinline__ float2 coef64(const TileOp &op, int k) { return make_float2(op.uh[2 * k], op.uh[2 * k + 1]); }
__device__ __forceinline__ dcx coef128(const TileOp &op, int k) {
    return dcx{df{op.uh[2 * k], op.ul[2 * k]}, df{op.uh[2 * k + 1], op.ul[2 * k + 1]}};
}

// ---- arithmetic on one amplitude type
__device__ __forceinline__ float2 vmul(float2 u, float2 a) { return cmul<float>(u, a); }
__device__ __forceinline__ float2 vmul2(float2 u, float2 a, float2 v, float2 b) { return cmul2<float>(u, a, v, b); }
__device__ __forceinline__ float2 vrmul2(float2 u, float2 a, float2 v, float2 b) {
    return make_float2(fmaf(u.x, a.x, v.x * b.x), fmaf(u.x, a.y, v.x * b.y));
}
__device__ __forceinline__ dcx vmul(const dcx &u, const dcx &a) { return dcx_mul(u, a); }
__device__ __forceinline__ dcx vmul2(const dcx &u, const dcx &a, const dcx &v, const dcx &b) {
    return dcx_mul2(u, a, v, b);
}
__device__ __forceinline__ dcx vrmul2(const dcx &u, const dcx &a, const dcx &v, const dcx &b) {
    return dcx_rmul2(u.re, a, v.re, b);
}

__device__ __forceinline__ float2 shfl_x(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ dcx shfl_x(const dcx &v, int m) {
    return dcx{df{__shfl_xor_sync(0xffffffffu, v.re.h, m), __shfl_xor_sync(0xffffffffu, v.re.l, m)},
               df{__shfl_xor_sync(0xffffffffu, v.im.h, m), __shfl_xor_sync(0xffffffffu, v.im.l, m)}};
}

// ---- shared-memory formats
// complex64: float2.  complex128: IEEE double2 (fmt 0) or double-float
// (fmt 1: re.h, re.l, im.h, im.l as four floats in the same 16 bytes).
__device__ __forceinline__ float2 ld_amp(const float2 *t, uint32_t i, int) { return t[i]; }
__device__ __forceinline__ void st_amp(float2 *t, uint32_t i, float2 v, int) { t[i] = v; }
__device__ __forceinline__ dcx ld_amp(const double2 *t, uint32_t i, int fmt) {
    if (fmt == 0) {
        const double2 d = t[i];
        return dcx{df_from_double(d.x), df_from_double(d.y)};
    }
    const float4 f = reinterpret_cast<const float4 *>(t)[i];
    return dcx{df{f.x, f.y}, df{f.z, f.w}};
}
__device__ __forceinline__ void st_amp(double2 *t, uint32_t i, const dcx &v, int fmt) {
    if (fmt == 0) {
        t[i] = make_double2(df_to_double(v.re), df_to_double(v.im));
    } else {
        reinterpret_cast<float4 *>(t)[i] = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
    }
}

// ---- gate application in registers
enum { PK_GENERAL = 0, PK_REAL = 1, PK_ANTI = 2, PK_EXCH = 3 };

template <int RB, int K, int PK, bool CT, typename V>
__device__ __forceinline__ void pair_reg(V (&v)[1 << RB], const V (&u)[4], bool thr_ok, uint32_t creg) {
#pragma unroll
    for (int j = 0; j < (1 << RB); j++) {
        if (j & (1 << K)) continue;
        const int j1 = j | (1 << K);
        if (CT && !(thr_ok && ((uint32_t)j & creg) == creg)) continue;
        const V a = v[j], b = v[j1];
        if (PK == PK_GENERAL) {
            v[j] = vmul2(u[0], a, u[1], b);
            v[j1] = vmul2(u[2], a, u[3], b);
        } else if (PK == PK_REAL) {
            v[j] = vrmul2(u[0], a, u[1], b);
            v[j1] = vrmul2(u[2], a, u[3], b);
        } else if (PK == PK_ANTI) {
            v[j] = vmul(u[1], b);
            v[j1] = vmul(u[2], a);
        } else {
            v[j] = b;
            v[j1] = a;
        }
    }
}

template <int RB, int PK, bool CT, typename V>
__device__ __forceinline__ void pair_reg_dispatch(int k, V (&v)[1 << RB], const V (&u)[4], bool thr_ok,
                                                  uint32_t creg) {
    switch (k) {
    case 0: pair_reg<RB, 0, PK, CT>(v, u, thr_ok, creg); break;
    case 1: pair_reg<RB, 1, PK, CT>(v, u, thr_ok, creg); break;
    case 2: pair_reg<RB, 2, PK, CT>(v, u, thr_ok, creg); break;
    case 3: pair_reg<RB, 3, PK, CT>(v, u, thr_ok, creg); break;
    default:
        if constexpr (RB > 4) pair_reg<RB, (RB > 4 ? 4 : 0), PK, CT>(v, u, thr_ok, creg);
        break;
    }
}

// target on lane bit t: partner in lane ^ 2^t; each lane computes its own
// output with the coefficients of its row.
template <int RB, int PK, bool CT, typename V>
__device__ __forceinline__ void pair_lane(int t, V (&v)[1 << RB], const V (&u)[4], bool thr_ok, uint32_t creg,
                                          int lane) {
    const bool upper = (lane >> t) & 1;
    const V c0 = upper ? u[3] : u[0];  // coefficient of the lane's own amplitude
    const V c1 = upper ? u[2] : u[1];  // coefficient of the partner's amplitude
    const int m = 1 << t;
#pragma unroll
    for (int j = 0; j < (1 << RB); j++) {
        const V w = shfl_x(v[j], m);
        if (CT && !(thr_ok && ((uint32_t)j & creg) == creg)) continue;
        if (PK == PK_GENERAL) v[j] = vmul2(c0, v[j], c1, w);
        else if (PK == PK_REAL) v[j] = vrmul2(c0, v[j], c1, w);
        else if (PK == PK_ANTI) v[j] = vmul(c1, w);
        else v[j] = w;
    }
}

template <bool C128>
__device__ __forceinline__ typename AmpT<C128>::V coef(const TileOp &op, int k);
template <> __device__ __forceinline__ float2 coef<false>(const TileOp &op, int k) { return coef64(op, k); }
template <> __device__ __forceinline__ dcx coef<true>(const TileOp &op, int k) { return coef128(op, k); }

template <int RB, int K>
__device__ __forceinline__ void phase_reg(float2 (&v)[1 << RB], float2 u, bool thr_ok, uint32_t creg) {
#pragma unroll
    for (int j = 0; j < (1 << RB); j++) {
        if (!((j >> K) & 1)) continue;
        if (!(thr_ok && ((uint32_t)j & creg) == creg)) continue;
        v[j] = vmul(u, v[j]);
    }
}

template <int RB, int K>
__device__ __forceinline__ void diag_reg(float2 (&v)[1 << RB], float2 u0, float2 u1, bool thr_ok, uint32_t creg) {
#pragma unroll
    for (int j = 0; j < (1 << RB); j++) {
        if (!(thr_ok && ((uint32_t)j & creg) == creg)) continue;
        v[j] = vmul(((j >> K) & 1) ? u1 : u0, v[j]);
    }
}

// One op of a phase.  op.code = family * 8 + k selects a code path whose
// register indices are compile-time constants.
template <int RB>
__device__ __forceinline__ void apply_rop(const TileOp &op, float2 (&v)[1 << RB], uint32_t thr_idx, int lane,
                                          uint64_t base) {
    if ((base & op.gcmask) != op.gcmask) return;  // a control outside the tile is 0 here
    const bool thr_ok = (thr_idx & op.lcthr) == op.lcthr;
    const uint32_t creg = op.creg;
    const float4 c01 = *reinterpret_cast<const float4 *>(op.uh);
    const float4 c23 = *reinterpret_cast<const float4 *>(op.uh + 4);
    const float2 u[4] = {make_float2(c01.x, c01.y), make_float2(c01.z, c01.w), make_float2(c23.x, c23.y),
                         make_float2(c23.z, c23.w)};
    switch (op.code) {
#define QSIM_K_CASES(FAM, STMT)                         \
    case FAM * 8 + 0: { constexpr int K = 0; STMT; } break; \
    case FAM * 8 + 1: { constexpr int K = 1; STMT; } break; \
    case FAM * 8 + 2: { constexpr int K = 2; STMT; } break; \
    case FAM * 8 + 3: { constexpr int K = 3; STMT; } break; \
    case FAM * 8 + 4: if constexpr (RB > 4) { constexpr int K = RB > 4 ? 4 : 0; STMT; } break;
        QSIM_K_CASES(RC_GEN, (pair_reg<RB, K, PK_GENERAL, false>(v, u, true, 0u)))
        QSIM_K_CASES(RC_REAL, (pair_reg<RB, K, PK_REAL, false>(v, u, true, 0u)))
        QSIM_K_CASES(RC_GENC, (pair_reg<RB, K, PK_GENERAL, true>(v, u, thr_ok, creg)))
        QSIM_K_CASES(RC_REALC, (pair_reg<RB, K, PK_REAL, true>(v, u, thr_ok, creg)))
        QSIM_K_CASES(RC_ANTI, (pair_reg<RB, K, PK_ANTI, true>(v, u, thr_ok, creg)))
        QSIM_K_CASES(RC_EXCHC, (pair_reg<RB, K, PK_EXCH, true>(v, u, thr_ok, creg)))
        QSIM_K_CASES(RC_PHASE, (phase_reg<RB, K>(v, u[3], thr_ok, creg)))
        QSIM_K_CASES(RC_DIAG, (diag_reg<RB, K>(v, u[0], u[3], thr_ok, creg)))
#undef QSIM_K_CASES
    case RC_LANE * 8 + PK_GENERAL: pair_lane<RB, PK_GENERAL, false>(op.tl, v, u, true, 0u, lane); break;
    case RC_LANE * 8 + PK_REAL: pair_lane<RB, PK_REAL, false>(op.tl, v, u, true, 0u, lane); break;
    case RC_LANE * 8 + PK_ANTI: pair_lane<RB, PK_ANTI, false>(op.tl, v, u, true, 0u, lane); break;
    case RC_LANE * 8 + PK_EXCH: pair_lane<RB, PK_EXCH, false>(op.tl, v, u, true, 0u, lane); break;
    case RC_LANEC * 8 + PK_GENERAL: pair_lane<RB, PK_GENERAL, true>(op.tl, v, u, thr_ok, creg, lane); break;
    case RC_LANEC * 8 + PK_REAL: pair_lane<RB, PK_REAL, true>(op.tl, v, u, thr_ok, creg, lane); break;
    case RC_LANEC * 8 + PK_ANTI: pair_lane<RB, PK_ANTI, true>(op.tl, v, u, thr_ok, creg, lane); break;
    case RC_LANEC * 8 + PK_EXCH: pair_lane<RB, PK_EXCH, true>(op.tl, v, u, thr_ok, creg, lane); break;
    case RC_THR * 8 + 0:  // phase on a lane or warp bit: the factor is uniform per thread
        if ((thr_idx >> op.tl) & 1u) {
#pragma unroll
            for (int j = 0; j < (1 << RB); j++)
                if (thr_ok && ((uint32_t)j & creg) == creg) v[j] = vmul(u[3], v[j]);
        }
        break;
    case RC_THR * 8 + 1: {
        const float2 f = ((thr_idx >> op.tl) & 1u) ? u[3] : u[0];
#pragma unroll
        for (int j = 0; j < (1 << RB); j++)
            if (thr_ok && ((uint32_t)j & creg) == creg) v[j] = vmul(f, v[j]);
        break;
    }
    case RC_GLOB * 8 + 0: {
        const float2 f = ((base >> op.tl) & 1ull) ? u[3] : u[0];
#pragma unroll
        for (int j = 0; j < (1 << RB); j++)
            if (thr_ok && ((uint32_t)j & creg) == creg) v[j] = vmul(f, v[j]);
        break;
    }
    default: break;
    }
}

// local index of register j of a thread: its lane/warp bits plus the bits
// of j scattered onto the register slots
template <int RB>
__device__ __forceinline__ uint32_t reg_index(uint32_t thr_idx, const uint32_t (&rbit)[RB], int j) {
    uint32_t x = thr_idx;
#pragma unroll
    for (int k = 0; k < RB; k++)
        if ((j >> k) & 1) x |= rbit[k];
    return x;
}

// One phase over the tile t: load this thread's registers, apply ops
// [ph.op_begin, ph.op_begin + ph.op_count) of `ops`, store back (permuted if
// the phase carries a permutation).  lfmt / sfmt: complex128 storage format
// on load / store (0 = IEEE double, 1 = double-float).  Ends with a block
// barrier.
template <bool C128, int RB>
__device__ __forceinline__ void run_phase(typename AmpT<C128>::S *t, const TilePhase &ph, const TileOp *ops,
                                          uint64_t base, int lane, int warp, int lfmt, int sfmt) {
    using V = typename AmpT<C128>::V;
    uint32_t thr_idx = (uint32_t)lane;
#pragma unroll
    for (int k = 0; k < kRegWarpBits; k++) thr_idx |= (uint32_t)((warp >> k) & 1) << ph.wb[k];
    uint32_t rbit[RB];
#pragma unroll
    for (int k = 0; k < RB; k++) rbit[k] = 1u << ph.rb[k];
    V v[1 << RB];
#pragma unroll
    for (int j = 0; j < (1 << RB); j++) v[j] = ld_amp(t, reg_index<RB>(thr_idx, rbit, j), lfmt);
    for (int o = ph.op_begin; o < ph.op_begin + ph.op_count; o++) apply_rop<RB>(ops[o], v, thr_idx, lane, base);
    if (ph.nperm) {
        __syncthreads();  // every thread has read its inputs before any permuted write
#pragma unroll
        for (int j = 0; j < (1 << RB); j++) {
            const uint32_t x = reg_index<RB>(thr_idx, rbit, j);
            uint32_t y = x;
            for (int k = 0; k < ph.nperm; k++) {
                const uint32_t bl = (x >> ph.pl[k]) & 1u, bh = (x >> ph.ph[k]) & 1u;
                y &= ~((1u << ph.pl[k]) | (1u << ph.ph[k]));
                y |= (bl << ph.ph[k]) | (bh << ph.pl[k]);
            }
            st_amp(t, y, v[j], sfmt);
        }
    } else {
#pragma unroll
        for (int j = 0; j < (1 << RB); j++) st_amp(t, reg_index<RB>(thr_idx, rbit, j), v[j], sfmt);
    }
    __syncthreads();
}

}  // namespace t2
}  // namespace qsim
