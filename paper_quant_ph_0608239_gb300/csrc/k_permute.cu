// k_permute.cu -- the qubit interchange of Sec. III.B as one pass over HBM.
//
// Exchanging the index bits l_i <-> h_i (i < K) moves the amplitude at index
// x to pi(x), pi swapping each pair of bits (Eq. onequbitchange and
// Eqs. twoqubitchange0-5 for K = 1, 2; any K here).  pi is an involution, so
// after the pass the amplitude at u is the one that was at pi(u).
//
// A tile holds every index bit the pairs touch: the L low bits as runs of
// 2^L contiguous amplitudes and the H high bits (the pairs' bits above L)
// selecting the run.  pi maps the tile onto itself.  One warp of each CTA
// issues bulk copies of tiles into a ring of four shared-memory stages; eight
// compute warps take a landed stage, each thread reading the elements at
// pi(u) for its output indices u and storing them to u's place in global
// memory, and give the stage back through an mbarrier.  The thread and
// shared-memory layout (perm_layout.hpp) makes the stores coalesced and the
// shared-memory reads free of bank conflicts; the address of every element a
// thread reads and writes is the sum of a per-thread and a per-group part,
// both computed once per CTA, since pi and the tile-to-memory maps are linear
// over disjoint bits.
#include "common.cuh"
#include "kernels.hpp"
#include "ptx.cuh"

namespace qsim {

namespace {

constexpr int kPermComputeWarps = 8;
constexpr int kPermThreads = 32 * (kPermComputeWarps + 1);  // compute warps + copy-issue warp
constexpr int kPermStages = 4;                                // tiles in flight per CTA
constexpr uint32_t kPermTileBytes = 16384;                   // per stage, without run padding
constexpr int kPermMaxGroups = kPermTileBytes / 8 / 32;       // groups of 32 elements per tile
constexpr long long kPermWait = 4000000000ll;

template <typename E>
__global__ void __launch_bounds__(kPermThreads)
    k_permute(E *__restrict__ a, TileGeom g, PermPairs pp, uint32_t *err, uint64_t ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kPermStages];   // stage holds its tile
    __shared__ __align__(8) uint64_t empty[kPermStages];  // stage read by every compute warp
    __shared__ uint64_t grp_g[kPermMaxGroups];            // group part of the store offset
    __shared__ uint32_t grp_r[kPermMaxGroups];            // group part of the shared-memory read offset
    __shared__ int s_hb[8];
    __shared__ int8_t s_lo[8], s_hi[8], s_skew[8];
    constexpr int kIt = kPermTileBytes / sizeof(E) / 32 / kPermComputeWarps;  // groups per warp, at most
    const int L = g.L, H = g.H, T = L + H;
    const uint32_t nruns = 1u << H, emask = (1u << L) - 1u;
    const uint32_t run_bytes = (uint32_t)sizeof(E) << L;
    const uint32_t buf_bytes = pp.run_stride * nruns;
    const uint32_t ngrp = (1u << T) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 8; k++) {  // constant indices: the parameters stay in the constant bank
            s_hb[k] = k < H ? g.hb[k] : 0;
            s_lo[k] = pp.lo[k];
            s_hi[k] = pp.hi[k];
            s_skew[k] = pp.skew[k];
        }
        for (int b = 0; b < kPermStages; b++) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kPermComputeWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    // run j: its offset in the state (the H bits deposited at hb) and its
    // place in a stage (j run strides plus the skew of its bits)
    auto run_off = [&](uint32_t j) {
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << s_hb[k];
        return o;
    };
    auto run_pos = [&](uint32_t j) {
        uint32_t skew = 0;
        for (int k = 0; k < H; k++)
            if (s_skew[k] >= 0) skew += ((j >> k) & 1u) << s_skew[k];
        return j * pp.run_stride + 16u * skew;
    };
    auto pi = [&](uint32_t u) {
        for (int k = 0; k < pp.K; k++) {
            const uint32_t t = ((u >> s_lo[k]) ^ (u >> s_hi[k])) & 1u;
            u ^= (t << s_lo[k]) | (t << s_hi[k]);
        }
        return u;
    };
    auto read_off = [&](uint32_t v) { return run_pos(v >> L) + (v & emask) * (uint32_t)sizeof(E); };
    auto store_off = [&](uint32_t u) { return run_off(u >> L) | (uint64_t)(u & emask); };
    uint32_t lanemask = 0;
    for (int i = 0; i < kPermLaneBits; i++) lanemask |= 1u << pp.lane[i];
    for (uint32_t r = threadIdx.x; r < ngrp; r += blockDim.x) {
        uint32_t u = 0, rb = r;  // r deposited at the tile bits that are not lane bits
        for (int t = 0; t < T; t++)
            if (!((lanemask >> t) & 1u)) {
                u |= (rb & 1u) << t;
                rb >>= 1;
            }
        grp_r[r] = read_off(pi(u));
        grp_g[r] = store_off(u);
    }
    __syncthreads();
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        return base;
    };
    const uint64_t stride = gridDim.x;
    // this CTA's tiles: blockIdx.x + i * stride, i < count; tile i goes
    // through stage i % kPermStages, whose j-th use completes phase j
    const uint32_t count = blockIdx.x < ntiles ? (uint32_t)((ntiles - 1 - blockIdx.x) / stride + 1) : 0u;

    if (warp == kPermComputeWarps) {
        // copy issue: tile i into stage i % kPermStages once its previous tile is read
        uint32_t i = 0;
        for (; i < count; i++) {
            const int b = (int)(i % kPermStages);
            if (i >= kPermStages &&
                !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[b], ((i / kPermStages) - 1u) & 1u, kPermWait)))
                break;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * stride);
            if (lane == 0) mbar_arrive_expect_tx(&full[b], run_bytes * nruns);
            __syncwarp();
            unsigned char *dst = smem_raw + (size_t)b * buf_bytes;
            for (uint32_t j = lane; j < nruns; j += 32)
                bulk_g2s(dst + run_pos(j), a + (base | run_off(j)), run_bytes, &full[b]);
        }
        if (i < count) {
            // gave up: the copies in flight land before the CTA leaves
            if (lane == 0) atomicExch(err, kErrTimeout);
            for (uint32_t t = i > (uint32_t)kPermStages ? i - kPermStages : 0u; t < i; t++)
                mbar_wait_bounded(&full[t % kPermStages], (t / kPermStages) & 1u, kPermWait);
        }
        return;
    }

    // compute warps: the per-thread part of the offsets (the lane bits at
    // their tile bits) added to the groups this warp takes, q = warp + 8 * it
    uint32_t ul = 0;
    for (int i = 0; i < kPermLaneBits; i++) ul |= (uint32_t)((lane >> i) & 1) << pp.lane[i];
    const uint32_t rl = read_off(pi(ul));
    const uint64_t gl = store_off(ul);
    const uint32_t nit = ngrp / kPermComputeWarps;
    uint32_t rr[kIt];
    uint64_t rg[kIt];
#pragma unroll
    for (int it = 0; it < kIt; it++) {
        const uint32_t q = (uint32_t)(warp + kPermComputeWarps * it);
        rr[it] = (uint32_t)it < nit ? grp_r[q] + rl : 0u;
        rg[it] = (uint32_t)it < nit ? grp_g[q] | gl : 0ull;
    }
    for (uint32_t i = 0; i < count; i++) {
        const int b = (int)(i % kPermStages);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[b], (i / kPermStages) & 1u, kPermWait))) {
            if (lane == 0) atomicExch(err, kErrTimeout);
            break;
        }
        const unsigned char *src = smem_raw + (size_t)b * buf_bytes;
        E *dst = a + tile_base(blockIdx.x + (uint64_t)i * stride);
        E x[kIt];
#pragma unroll
        for (int it = 0; it < kIt; it++)
            if ((uint32_t)it < nit) x[it] = *reinterpret_cast<const E *>(src + rr[it]);
#pragma unroll
        for (int it = 0; it < kIt; it++)
            if ((uint32_t)it < nit) dst[rg[it]] = x[it];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
}

}  // namespace

// Tile size of the interchange pass for elements of elem_bytes (8 or 16).
int permute_tile_bits(int elem_bytes) { return elem_bytes == 8 ? 11 : 10; }

cudaError_t launch_permute(void *amp, int elem_bytes, const TileGeom &g, const PermPairs &pairs, uint32_t *err,
                           int sm_count, cudaStream_t s) {
    const int T = g.L + g.H;
    if (g.H > kPermMaxH || g.L < 1 || T < 8 || pairs.K < 1 || pairs.K > kMaxPermPairs) return cudaErrorInvalidValue;
    if (((size_t)elem_bytes << T) > kPermTileBytes) return cudaErrorInvalidValue;
    PermPairs pp = pairs;
    perm_layout(g.L, g.H, elem_bytes, pp);
    const size_t smem = (size_t)kPermStages * pp.run_stride * ((size_t)1 << g.H);
    const uint64_t ntiles = 1ull << (g.n - T);
    auto go = [&](auto kern, auto *ptr) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPermThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)sm_count * per_sm;
        if (grid > ntiles) grid = ntiles;
        kern<<<(unsigned)grid, kPermThreads, smem, s>>>(ptr, g, pp, err, ntiles);
        return cudaGetLastError();
    };
    if (elem_bytes == 8) return go(k_permute<float2>, static_cast<float2 *>(amp));
    return go(k_permute<double2>, static_cast<double2 *>(amp));
}

}  // namespace qsim
