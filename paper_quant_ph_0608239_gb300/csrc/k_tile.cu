// k_tile.cu -- shared-memory tile passes: many gates per HBM pass.
//
// The paper notes that gates on local qubits need no communication
// (Sec. III.B) and runs one sweep of the state per gate.  Here a pass holds a
// tile of 2^T amplitudes in shared memory: the L lowest index bits (contiguous
// runs of 2^L amplitudes) plus H chosen higher bits, T = L + H.  Every tile is
// fetched with bulk asynchronous copies (one cp.async.bulk per run, completing
// on an mbarrier), the pass's whole gate program is applied in shared memory,
// and the tile is written back with bulk copies: one read and one write of the
// state for any number of gates whose targets lie in the tile.  Controls may
// lie anywhere (bits outside the tile are fixed per tile and tested once), and
// diagonal gates need no target in the tile at all.
//
// Several CTAs are resident per SM; while one waits for its tile the others
// compute, which overlaps copy and compute without explicit double buffering.
#include "common.cuh"
#include "kernels.hpp"
#include "ptx.cuh"

namespace qsim {

namespace {

constexpr int kTileThreads = 256;
constexpr int kMaxH = 10;                  // at most 1024 runs per tile
constexpr int kMaxCopyShift = 14;          // bulk copies of at most 16 KiB
constexpr long long kWaitBudget = 4000000000ll;  // SM cycles (about 2 s) before a wait gives up

__device__ __forceinline__ uint32_t ins0(uint32_t i, int pos) {
    return ((i >> pos) << (pos + 1)) | (i & ((1u << pos) - 1u));
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
    for (uint32_t p = threadIdx.x; p < half; p += blockDim.x) {
        const uint32_t i0 = ins0(p, tl);
        if ((i0 & lc) != lc) continue;
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
    if (op.kind == TOP_PHASE) {
        const int tl = op.tl;
        const uint32_t bt = 1u << tl;
        for (uint32_t p = threadIdx.x; p < (TS >> 1); p += blockDim.x) {
            const uint32_t i = ins0(p, tl) | bt;
            if ((i & lc) != lc) continue;
            t[i] = cmul<R>(u1, t[i]);
        }
    } else if (op.kind == TOP_DIAG) {
        const int tl = op.tl;
        for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
            if ((i & lc) != lc) continue;
            t[i] = cmul<R>(((i >> tl) & 1u) ? u1 : u0, t[i]);
        }
    } else {  // TOP_DIAG_G: the target bit lies outside the tile
        const amp_t<R> f = ((base >> op.tl) & 1ull) ? u1 : u0;
        for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
            if ((i & lc) != lc) continue;
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
__device__ void apply_op(amp_t<R> *t, int T, const TileOp &op, uint64_t base, const amp_t<R> *__restrict__ dmat) {
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

template <typename R>
__global__ void __launch_bounds__(kTileThreads) k_tile(amp_t<R> *__restrict__ a, TileGeom g,
                                                       const TileOp *__restrict__ ops, int nops,
                                                       const amp_t<R> *__restrict__ dmat, uint32_t *err,
                                                       uint64_t ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    amp_t<R> *t = reinterpret_cast<amp_t<R> *>(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint64_t runoff[1 << kMaxH];
    __shared__ int abort_flag;
    const int L = g.L, H = g.H, T = L + H;
    const uint32_t TS = 1u << T;
    const uint32_t nruns = 1u << H;
    // each contiguous run of 2^L amplitudes is moved in copies of at most
    // kMaxCopyBytes (2^sub_L amplitudes each)
    const int amp_shift = sizeof(amp_t<R>) == 8 ? 3 : 4;
    const int sub_L = L + amp_shift > kMaxCopyShift ? kMaxCopyShift - amp_shift : L;
    const int sub_shift = L - sub_L;
    const uint32_t ncopies = nruns << sub_shift;
    const uint32_t copy_bytes = 1u << (sub_L + amp_shift);

    for (uint32_t j = threadIdx.x; j < nruns; j += blockDim.x) {
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << g.hb[k];
        runoff[j] = o;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, g.hb[k]);
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, TS * (uint32_t)sizeof(amp_t<R>));
            __syncwarp();
            for (uint32_t c = threadIdx.x; c < ncopies; c += 32) {
                const uint32_t j = c >> sub_shift, s = c & ((1u << sub_shift) - 1u);
                bulk_g2s(t + ((size_t)j << L) + ((size_t)s << sub_L), a + (base | runoff[j]) + ((size_t)s << sub_L),
                         copy_bytes, &bar);
            }
        }
        if (!mbar_wait_bounded(&bar, parity, kWaitBudget)) {
            atomicExch(err, kErrTimeout);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            // give the copies in flight one more bounded chance to land, then leave
            mbar_wait_bounded(&bar, parity, kWaitBudget);
            return;
        }
        parity ^= 1u;

        for (int o = 0; o < nops; o++) {
            apply_op<R>(t, T, ops[o], base, dmat);
            __syncthreads();
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

size_t tile_smem_bytes(int dt, int T) { return (size_t)(dt == 0 ? 8 : 16) << T; }

cudaError_t launch_tile_pass(void *amp, int dt, const TileGeom &g, const TileOp *ops, int nops, const void *dmat,
                             uint32_t *err, int sm_count, cudaStream_t s) {
    const int T = g.L + g.H;
    if (g.H < 0 || g.H > kMaxH || T > g.n || T > 14 || g.L < 1) return cudaErrorInvalidValue;
    const size_t smem = tile_smem_bytes(dt, T);
    if (smem > 200u * 1024u) return cudaErrorInvalidValue;
    const uint64_t ntiles = 1ull << (g.n - T);
    // resident CTAs per SM limited by shared memory (227 KB usable)
    int per_sm = (int)((220u * 1024u) / (smem + 9u * 1024u));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    cudaError_t e;
    if (dt == 0) {
        e = cudaFuncSetAttribute(k_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tile<float><<<(unsigned)grid, kTileThreads, smem, s>>>(static_cast<float2 *>(amp), g, ops, nops,
                                                                  static_cast<const float2 *>(dmat), err, ntiles);
    } else {
        e = cudaFuncSetAttribute(k_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tile<double><<<(unsigned)grid, kTileThreads, smem, s>>>(static_cast<double2 *>(amp), g, ops, nops,
                                                                   static_cast<const double2 *>(dmat), err, ntiles);
    }
    return cudaGetLastError();
}

}  // namespace qsim
