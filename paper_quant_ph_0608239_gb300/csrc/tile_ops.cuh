// tile_ops.cuh -- the gate program of a shared-memory tile: every op is one
// sweep over the tile held in shared memory (used by the tile passes of
// k_tile.cu and the batch kernel of k_batch.cu).
#pragma once

#include "common.cuh"
#include "kernels.hpp"

namespace qsim {
namespace tileops {

__device__ __forceinline__ uint32_t ins0(uint32_t i, int pos) {
    return ((i >> pos) << (pos + 1)) | (i & ((1u << pos) - 1u));
}

// Index of the p-th element whose bits at the positions in `fixed` are zero.
// Ops enumerate only the amplitudes their local controls select (control
// bits fixed at 1): a gate with c controls costs 2^-c of a sweep.
__device__ __forceinline__ uint32_t expand_fixed(uint32_t p, uint32_t fixed) {
    while (fixed) {
        p = ins0(p, __ffs(fixed) - 1);
        fixed &= fixed - 1u;
    }
    return p;
}

template <typename R>
__device__ __forceinline__ void op_pairs(amp_t<R> *t, int T, const TileOp &op) {
    const int tl = op.tl;
    const uint32_t lc = op.lcmask, bt = 1u << tl;
    const uint32_t half = 1u << (T - 1);
    amp_t<R> u[4];
#pragma unroll
    for (int k = 0; k < 4; k++) u[k] = mk<R>((R)op.u[2 * k], (R)op.u[2 * k + 1]);
    const int kind = op.kind;
    const uint32_t npair = half >> __popc(lc), fixed = bt | lc;
    for (uint32_t p = threadIdx.x; p < npair; p += blockDim.x) {
        const uint32_t i0 = lc ? expand_fixed(p, fixed) | lc : ins0(p, tl);
        const uint32_t i1 = i0 | bt;
        amp_t<R> x = t[i0], y = t[i1];
        if (kind == TOP_GENERAL) {
            t[i0] = cmul2<R>(u[0], x, u[1], y);
            t[i1] = cmul2<R>(u[2], x, u[3], y);
        } else if (kind == TOP_ANTIDIAG) {
            t[i0] = cmul<R>(u[1], y);
            t[i1] = cmul<R>(u[2], x);
        } else {
            t[i0] = y;
            t[i1] = x;
        }
    }
}

template <typename R>
__device__ __forceinline__ void op_diag(amp_t<R> *t, int T, const TileOp &op, uint64_t base) {
    const uint32_t lc = op.lcmask;
    const amp_t<R> u0 = mk<R>((R)op.u[0], (R)op.u[1]);
    const amp_t<R> u1 = mk<R>((R)op.u[6], (R)op.u[7]);
    const uint32_t TS = 1u << T;
    const uint32_t cnt = TS >> __popc(lc);  // amplitudes the controls select
    if (op.kind == TOP_PHASE) {
        const int tl = op.tl;
        const uint32_t bt = 1u << tl, fixed = bt | lc;
        for (uint32_t p = threadIdx.x; p < (cnt >> 1); p += blockDim.x) {
            const uint32_t i = (lc ? expand_fixed(p, fixed) | lc : ins0(p, tl)) | bt;
            t[i] = cmul<R>(u1, t[i]);
        }
    } else if (op.kind == TOP_DIAG) {
        const int tl = op.tl;
        for (uint32_t p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = lc ? expand_fixed(p, lc) | lc : p;
            t[i] = cmul<R>(((i >> tl) & 1u) ? u1 : u0, t[i]);
        }
    } else {  // TOP_DIAG_G: the target bit lies outside the tile
        const amp_t<R> f = ((base >> op.tl) & 1ull) ? u1 : u0;
        for (uint32_t p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = lc ? expand_fixed(p, lc) | lc : p;
            t[i] = cmul<R>(f, t[i]);
        }
    }
}

template <typename R>
__device__ __forceinline__ void op_swapgate(amp_t<R> *t, int T, const TileOp &op) {
    // visit bit tl = 1, bit tl2 = 0; partner has them exchanged
    const uint32_t b0 = 1u << op.tl, b1 = 1u << op.tl2, lc = op.lcmask;
    const uint32_t TS = 1u << T;
    for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
        if (!(i & b0) || (i & b1) || (i & lc) != lc) continue;
        const uint32_t j = (i & ~b0) | b1;
        amp_t<R> x = t[i];
        t[i] = t[j];
        t[j] = x;
    }
}

template <typename R>
__device__ __forceinline__ void op_perm(amp_t<R> *t, int T, const TileOp &op) {
    // pi exchanges local bit pl[k] with ph[k]; it is an involution, so every
    // index is in a cycle of length <= 2 and disjoint pairs swap in place.
    const uint32_t TS = 1u << T;
    const int np = op.nperm;
    for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
        uint32_t j = i;
        for (int k = 0; k < np; k++) {
            const uint32_t bl = (i >> op.pl[k]) & 1u, bh = (i >> op.ph[k]) & 1u;
            j &= ~((1u << op.pl[k]) | (1u << op.ph[k]));
            j |= (bl << op.ph[k]) | (bh << op.pl[k]);
        }
        if (j > i) {
            amp_t<R> x = t[i];
            t[i] = t[j];
            t[j] = x;
        }
    }
}

template <typename R, int K>
__device__ __forceinline__ void op_dense_k(amp_t<R> *t, int T, const TileOp &op, const amp_t<R> *__restrict__ U) {
    constexpr int D = 1 << K;
    int srt[K];
#pragma unroll
    for (int j = 0; j < K; j++) srt[j] = op.pl[j];
#pragma unroll
    for (int i = 1; i < K; i++)
#pragma unroll
        for (int j = K - 1; j >= i; j--)
            if (srt[j - 1] > srt[j]) {
                int x = srt[j];
                srt[j] = srt[j - 1];
                srt[j - 1] = x;
            }
    uint32_t off[D];
#pragma unroll
    for (int c = 0; c < D; c++) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < K; j++)
            if ((c >> j) & 1) o |= 1u << op.pl[j];
        off[c] = o;
    }
    const uint32_t lc = op.lcmask;
    const uint32_t G = 1u << (T - K);
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        uint32_t b = g;
#pragma unroll
        for (int j = 0; j < K; j++) b = ins0(b, srt[j]);
        if ((b & lc) != lc) continue;
        amp_t<R> v[D];
#pragma unroll
        for (int c = 0; c < D; c++) v[c] = t[b | off[c]];
#pragma unroll
        for (int r = 0; r < D; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                const amp_t<R> u = U[r * D + c];
                re = fma(u.x, v[c].x, re);
                re = fma(-u.y, v[c].y, re);
                im = fma(u.x, v[c].y, im);
                im = fma(u.y, v[c].x, im);
            }
            t[b | off[r]] = mk<R>(re, im);
        }
    }
}

template <typename R>
__device__ __forceinline__ void tile_apply_op(amp_t<R> *t, int T, const TileOp &op, uint64_t base,
                                              const amp_t<R> *__restrict__ dmat) {
    if ((base & op.gcmask) != op.gcmask) return;  // a control outside the tile is 0 here
    switch (op.kind) {
    case TOP_GENERAL:
    case TOP_ANTIDIAG:
    case TOP_EXCHANGE: op_pairs<R>(t, T, op); break;
    case TOP_DIAG:
    case TOP_PHASE:
    case TOP_DIAG_G: op_diag<R>(t, T, op, base); break;
    case TOP_SWAPGATE: op_swapgate<R>(t, T, op); break;
    case TOP_PERM: op_perm<R>(t, T, op); break;
    case TOP_DENSE:
        switch (op.nperm) {
        case 1: op_dense_k<R, 1>(t, T, op, dmat + op.dense_off); break;
        case 2: op_dense_k<R, 2>(t, T, op, dmat + op.dense_off); break;
        case 3: op_dense_k<R, 3>(t, T, op, dmat + op.dense_off); break;
        case 4: op_dense_k<R, 4>(t, T, op, dmat + op.dense_off); break;
        default: break;
        }
        break;
    default: break;
    }
}


}  // namespace tileops
using tileops::tile_apply_op;
}  // namespace qsim
