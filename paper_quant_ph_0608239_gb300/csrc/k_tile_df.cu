// k_tile_df.cu -- complex128 tile passes in double-float arithmetic.
//
// Same pass structure as k_tile.cu (bulk asynchronous copies of 2^T
// amplitudes = the L low index bits plus H chosen high bits; one read and one
// write of the state per pass), with the gate program applied in shared
// memory in double-float arithmetic (df64.cuh) instead of FP64: GB300 runs
// FP64 at about 1/58 of its FP32 rate.  After the tile lands it is converted
// in place from IEEE double to double-float (two floats per real, integer
// operations only); before it is stored it is converted back.  Within one
// run of a plan the state stays in double-float form in HBM between two
// arithmetic passes (same 16 bytes per amplitude: re.h, re.l, im.h, im.l), so
// only the first arithmetic pass converts on load and only the last converts
// on store.  A pass whose ops only move data (bit flips, SWAP gates,
// interchanges) moves 16-byte amplitudes in either form and stays bit-exact.
//
// Uncontrolled Hadamard-type gates s*[[1,1],[1,-1]] arrive from the planner
// as unscaled butterflies (a0 + a1, a0 - a1): the product of their factors s
// is folded into one other op of the same pass that touches every amplitude
// once (the planner's choice), which is exact as every op is linear.
// Diagonal ops on bits outside the tile without local controls come after the
// program (nglob of them): one thread multiplies them into one factor per tile
// while the tile loads, and that factor scales the coefficients of the
// pass's absorber op (or, without one, the tile in one multiply).
//
// Each op is one sweep over the tile's pairs in shared memory, with the
// target bit a runtime value, so one compact code path serves every target
// (the double-float arithmetic per pair is long enough that shared-memory
// traffic and the barrier between ops are a small share of the time).
#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"
#include "ptx.cuh"

namespace qsim {

namespace {

constexpr int kThreadsDF = 256;
constexpr int kMaxHDF = 10;
constexpr int kMaxCopyShiftDF = 14;
constexpr long long kWaitBudgetDF = 4000000000ll;
#ifndef QSIM_DF_PAIRS
#define QSIM_DF_PAIRS 2
#endif
constexpr int kPairIt = QSIM_DF_PAIRS;  // pairs a thread updates per loop iteration

__device__ __forceinline__ uint32_t ins0d(uint32_t i, int pos) {
    return ((i >> pos) << (pos + 1)) | (i & ((1u << pos) - 1u));
}

// The tile is addressed by its shared-window address t (16 bytes per amplitude).
__device__ __forceinline__ float4 ld4(uint32_t t, uint32_t i) { return lds128(t + (i << 4)); }
__device__ __forceinline__ void st4(uint32_t t, uint32_t i, float4 v) { sts128(t + (i << 4), v); }
__device__ __forceinline__ dcx ldx(uint32_t t, uint32_t i) {
    const float4 f = ld4(t, i);
    return dcx{df{f.x, f.y}, df{f.z, f.w}};
}
__device__ __forceinline__ void stx(uint32_t t, uint32_t i, const dcx &v) {
    st4(t, i, make_float4(v.re.h, v.re.l, v.im.h, v.im.l));
}
// An op as staged in shared memory: every thread reads every op of the pass
// for every tile, so the pass's ops are copied once (or once per chunk) per
// block instead of being fetched from global memory each time.
struct __align__(16) DfOp {
    float4 c[4];      // u00, u01, u10, u11 as (re.h, re.l, im.h, im.l)
    uint64_t gcmask;
    uint32_t lcmask;
    uint8_t kind, tl, pk, tl2;
};
static_assert(sizeof(DfOp) == 80, "DfOp layout");
constexpr int kStageDF = 40;  // ops per staged chunk (3.1 KiB)

__device__ __forceinline__ DfOp to_dfop(const TileOp &op) {
    DfOp d;
#pragma unroll
    for (int j = 0; j < 4; j++) d.c[j] = make_float4(op.uh[2 * j], op.ul[2 * j], op.uh[2 * j + 1], op.ul[2 * j + 1]);
    d.gcmask = op.gcmask;
    d.lcmask = op.lcmask;
    d.kind = (uint8_t)op.kind;
    d.tl = (uint8_t)op.tl;
    d.pk = (uint8_t)op.pk;
    d.tl2 = (uint8_t)op.tl2;
    return d;
}

__device__ __forceinline__ void stage_df(DfOp *dst, const TileOp *src, int cn) {
    for (int k = threadIdx.x; k < cn; k += blockDim.x) dst[k] = to_dfop(src[k]);
}

__device__ __forceinline__ dcx coefx(const DfOp &op, int k) {
    const float4 c = op.c[k];
    return dcx{df{c.x, c.y}, df{c.z, c.w}};
}

// Index of the p-th element whose bits at the positions in `fixed` are zero:
// zeros inserted at those positions in ascending order.
__device__ __forceinline__ uint32_t expand_fixed(uint32_t p, uint32_t fixed) {
    while (fixed) {
        p = ins0d(p, __ffs(fixed) - 1);
        fixed &= fixed - 1u;
    }
    return p;
}

// op: the staged copy; gop: the op in global memory (read only for the
// permutation's bit list).  An op enumerates only the amplitudes its local
// controls select (the control bits fixed at 1), so a gate with c controls
// costs 2^-c of a sweep.
__device__ void apply_df(uint32_t t, int T, const DfOp &op, const TileOp &gop, uint64_t base) {
    if ((base & op.gcmask) != op.gcmask) return;
    const uint32_t lc = op.lcmask;
    const uint32_t TS = 1u << T;
    const int kind = op.kind;
    const int nlc = __popc(lc);
    if (kind == TOP_GENERAL || kind == TOP_ANTIDIAG || kind == TOP_EXCHANGE) {
        const int tl = op.tl;
        const uint32_t bt = 1u << tl, fixed = bt | lc;
        const int pk = op.pk;
        const uint32_t npair = (TS >> 1) >> nlc;
        auto pair0 = [&](uint32_t p) { return lc ? (expand_fixed(p, fixed) | lc) : ins0d(p, tl); };
        const dcx u0 = coefx(op, 0), u1 = coefx(op, 1), u2 = coefx(op, 2), u3 = coefx(op, 3);
        if (pk == 3) {  // exchange: move the bytes
            for (uint32_t p = threadIdx.x; p < npair; p += blockDim.x) {
                const uint32_t i0 = pair0(p);
                const uint32_t i1 = i0 | bt;
                const float4 x = ld4(t, i0), y = ld4(t, i1);
                st4(t, i0, y);
                st4(t, i1, x);
            }
            return;
        }
        // kPairIt independent pairs per iteration: the two-sum chains of one
        // pair fill the latency of the others'
        const uint32_t half = npair, step = blockDim.x;
        for (uint32_t p = threadIdx.x; p < half; p += kPairIt * step) {
            uint32_t ia[kPairIt], ib[kPairIt];
            bool ok[kPairIt];
            dcx va[kPairIt], vb[kPairIt];
#pragma unroll
            for (int k = 0; k < kPairIt; k++) {
                const uint32_t pp = p + (uint32_t)k * step;
                ok[k] = pp < half;
                ia[k] = pair0(ok[k] ? pp : p);
                ib[k] = ia[k] | bt;
                va[k] = ldx(t, ia[k]);
                vb[k] = ldx(t, ib[k]);
            }
            if (pk == 0) {
#pragma unroll
                for (int k = 0; k < kPairIt; k++) {
                    const dcx x0 = dcx_mul2(u0, va[k], u1, vb[k]), x1 = dcx_mul2(u2, va[k], u3, vb[k]);
                    va[k] = x0;
                    vb[k] = x1;
                }
            } else if (pk == 4) {  // unscaled butterfly: (a0 + a1, a0 - a1)
#pragma unroll
                for (int k = 0; k < kPairIt; k++) {
                    const dcx x0{df_add(va[k].re, vb[k].re), df_add(va[k].im, vb[k].im)};
                    const dcx x1{df_add(va[k].re, df_neg(vb[k].re)), df_add(va[k].im, df_neg(vb[k].im))};
                    va[k] = x0;
                    vb[k] = x1;
                }
            } else if (pk == 1) {
#pragma unroll
                for (int k = 0; k < kPairIt; k++) {
                    const dcx x0 = dcx_rmul2(u0.re, va[k], u1.re, vb[k]), x1 = dcx_rmul2(u2.re, va[k], u3.re, vb[k]);
                    va[k] = x0;
                    vb[k] = x1;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kPairIt; k++) {
                    const dcx x0 = dcx_mul(u1, vb[k]), x1 = dcx_mul(u2, va[k]);
                    va[k] = x0;
                    vb[k] = x1;
                }
            }
#pragma unroll
            for (int k = 0; k < kPairIt; k++)
                if (ok[k]) {
                    stx(t, ia[k], va[k]);
                    stx(t, ib[k], vb[k]);
                }
        }
    } else if (kind == TOP_PHASE) {
        const uint32_t bt = 1u << op.tl, fixed = bt | lc;
        const dcx u3 = coefx(op, 3);
        const uint32_t cnt = (TS >> 1) >> nlc;
        for (uint32_t p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = (lc ? expand_fixed(p, fixed) | lc : ins0d(p, op.tl)) | bt;
            stx(t, i, dcx_mul(u3, ldx(t, i)));
        }
    } else if (kind == TOP_DIAG || kind == TOP_DIAG_G) {
        const dcx u0 = coefx(op, 0), u3 = coefx(op, 3);
        const bool global_one = kind == TOP_DIAG_G && ((base >> op.tl) & 1ull);
        const uint32_t cnt = TS >> nlc;
        for (uint32_t p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = lc ? expand_fixed(p, lc) | lc : p;
            const bool one = kind == TOP_DIAG ? ((i >> op.tl) & 1u) : global_one;
            stx(t, i, dcx_mul(one ? u3 : u0, ldx(t, i)));
        }
    } else if (kind == TOP_SWAPGATE) {
        const uint32_t b0 = 1u << op.tl, b1 = 1u << op.tl2;
        for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
            if (!(i & b0) || (i & b1) || (i & lc) != lc) continue;
            const uint32_t j = (i & ~b0) | b1;
            const float4 x = ld4(t, i), y = ld4(t, j);
            st4(t, i, y);
            st4(t, j, x);
        }
    } else if (kind == TOP_PERM) {
        const int nperm = gop.nperm;
        for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
            uint32_t j = i;
            for (int k = 0; k < nperm; k++) {
                const uint32_t bl = (i >> gop.pl[k]) & 1u, bh = (i >> gop.ph[k]) & 1u;
                j &= ~((1u << gop.pl[k]) | (1u << gop.ph[k]));
                j |= (bl << gop.ph[k]) | (bh << gop.pl[k]);
            }
            if (j > i) {
                const float4 x = ld4(t, i), y = ld4(t, j);
                st4(t, i, y);
                st4(t, j, x);
            }
        }
    }
}

// The factor of the hoisted diagonal ops for the tile at `base` (each op
// scales the tile by u00 or u11 by its bit, if its global controls are set),
// and the absorber with its coefficients multiplied by it.  One thread.
__device__ __noinline__ void tile_factor(const TileOp *ops, int nops, int nglob, int absorber, uint64_t base,
                                        DfOp &abs_out, float4 &g_out, int &one_out) {
    dcx g{df{1.0f, 0.0f}, df{0.0f, 0.0f}};
    bool one = true;
    for (int k = 0; k < nglob; k++) {
        const TileOp &go = ops[nops + k];
        if ((base & go.gcmask) != go.gcmask) continue;
        const int c = ((base >> go.tl) & 1ull) ? 3 : 0;
        const dcx f{df{go.uh[2 * c], go.ul[2 * c]}, df{go.uh[2 * c + 1], go.ul[2 * c + 1]}};
        if (f.re.h == 1.0f && f.re.l == 0.0f && f.im.h == 0.0f && f.im.l == 0.0f) continue;
        g = one ? f : dcx_mul(g, f);
        one = false;
    }
    g_out = make_float4(g.re.h, g.re.l, g.im.h, g.im.l);
    one_out = one ? 1 : 0;
    if (absorber >= 0) {
        DfOp d = to_dfop(ops[absorber]);
        if (!one)
            for (int j = 0; j < 4; j++) {
                const dcx r = dcx_mul(g, coefx(d, j));
                d.c[j] = make_float4(r.re.h, r.re.l, r.im.h, r.im.l);
            }
        abs_out = d;
    }
}

__global__ void __launch_bounds__(kThreadsDF) k_tile_df(double2 *__restrict__ a, TileGeom g,
                                                        const TileOp *__restrict__ ops, int nops, int nglob,
                                                        int absorber, int cvt_in, int cvt_out, uint32_t *err,
                                                        uint64_t ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double2 *t = reinterpret_cast<double2 *>(smem_raw);
    const uint32_t tf = smem_u32(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ DfOp s_ops[kStageDF];
    __shared__ DfOp s_abs;          // the absorber with this tile's factor folded in
    __shared__ float4 s_g;          // this tile's factor of the hoisted diagonals
    __shared__ int s_gone;          // ... which is exactly 1
    __shared__ int abort_flag;
    const int L = g.L, H = g.H, T = L + H;
    uint64_t *runoff = reinterpret_cast<uint64_t *>(smem_raw + ((size_t)16 << T));  // 2^H entries
    const bool one_stage = nops <= kStageDF;
    const uint32_t TS = 1u << T;
    const uint32_t nruns = 1u << H;
    const int sub_L = L + 4 > kMaxCopyShiftDF ? kMaxCopyShiftDF - 4 : L;
    const int sub_shift = L - sub_L;
    const uint32_t ncopies = nruns << sub_shift;
    const uint32_t copy_bytes = 1u << (sub_L + 4);

    for (uint32_t j = threadIdx.x; j < nruns; j += blockDim.x) {
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << g.hb[k];
        runoff[j] = o;
    }
    __shared__ int s_hb[kMaxHDF];  // the high tile bits, indexed at run time
    if (threadIdx.x < kMaxHDF) s_hb[threadIdx.x] = threadIdx.x < (unsigned)H ? g.hb[threadIdx.x] : 0;
    if (one_stage) stage_df(s_ops, ops, nops);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, TS * 16u);
            __syncwarp();
            for (uint32_t c = threadIdx.x; c < ncopies; c += 32) {
                const uint32_t j = c >> sub_shift, s = c & ((1u << sub_shift) - 1u);
                bulk_g2s(t + ((size_t)j << L) + ((size_t)s << sub_L), a + (base | runoff[j]) + ((size_t)s << sub_L),
                         copy_bytes, &bar);
            }
        }
        if (nglob > 0 && threadIdx.x == 0) tile_factor(ops, nops, nglob, absorber, base, s_abs, s_g, s_gone);
        if (!mbar_wait_bounded(&bar, parity, kWaitBudgetDF)) {
            atomicExch(err, kErrTimeout);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            mbar_wait_bounded(&bar, parity, kWaitBudgetDF);
            return;
        }
        parity ^= 1u;

        if (cvt_in) {
            for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
                const double2 d = t[i];
                stx(tf, i, dcx{df_from_double(d.x), df_from_double(d.y)});
            }
            __syncthreads();
        }
        for (int c0 = 0; c0 < nops; c0 += kStageDF) {
            const int cn = nops - c0 < kStageDF ? nops - c0 : kStageDF;
            if (!one_stage) {
                stage_df(s_ops, ops + c0, cn);  // the previous op ended with a barrier
                __syncthreads();
            }
            for (int o = 0; o < cn; o++) {
                apply_df(tf, T, c0 + o == absorber ? s_abs : s_ops[o], ops[c0 + o], base);
                __syncthreads();
            }
        }
        if (nglob > 0 && absorber < 0 && !s_gone) {  // no absorber: one multiply of the tile
            const dcx gf{df{s_g.x, s_g.y}, df{s_g.z, s_g.w}};
            for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) stx(tf, i, dcx_mul(gf, ldx(tf, i)));
            __syncthreads();
        }
        if (cvt_out) {
            for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
                const dcx v = ldx(tf, i);
                t[i] = make_double2(df_to_double(v.re), df_to_double(v.im));
            }
        }

        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x < 32) {
            for (uint32_t c = threadIdx.x; c < ncopies; c += 32) {
                const uint32_t j = c >> sub_shift, s = c & ((1u << sub_shift) - 1u);
                bulk_s2g(a + (base | runoff[j]) + ((size_t)s << sub_L), t + ((size_t)j << L) + ((size_t)s << sub_L),
                         copy_bytes);
            }
            bulk_commit();
            bulk_wait_read_all();
        }
        __syncthreads();
    }
    if (threadIdx.x < 32) bulk_wait_all();
}

}  // namespace

cudaError_t launch_tile_pass_df(void *amp, const TileGeom &g, const TileOp *ops, int nops, int nglob, int absorber,
                                bool cvt_in, bool cvt_out, uint32_t *err, int sm_count, cudaStream_t s) {
    const int T = g.L + g.H;
    if (g.H < 0 || g.H > kMaxHDF || T > g.n || T > 13 || g.L < 1) return cudaErrorInvalidValue;
    if (nops < 0 || nglob < 0 || absorber >= nops) return cudaErrorInvalidValue;
    const size_t smem = ((size_t)16 << T) + ((size_t)8 << g.H);  // tile + run offsets
    const uint64_t ntiles = 1ull << (g.n - T);
    cudaError_t e = cudaFuncSetAttribute(k_tile_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_df, kThreadsDF, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    k_tile_df<<<(unsigned)grid, kThreadsDF, smem, s>>>(static_cast<double2 *>(amp), g, ops, nops, nglob, absorber,
                                                      cvt_in ? 1 : 0, cvt_out ? 1 : 0, err, ntiles);
    return cudaGetLastError();
}

}  // namespace qsim
