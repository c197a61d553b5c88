// k_fused_tc.cu -- dense k-qubit gates (k = 4, 5) on the tensor cores.
//
// A fused gate is a 2^k x 2^k unitary U (the FP64 product of the gates it
// replaces, built on the host).  For every group of 2^k amplitudes that differ
// only in the k qubits, a' = U a.  With the complex numbers embedded as real
// 2x2 blocks ([[Re, -Im], [Im, Re]]) this is the real matrix product
//
//     D (rows = groups, 2K columns) = A (groups x 2K) * B^T,  K = 2^k,
//
// where a row of A is the group's amplitudes in their memory order
// (re, im, re, im, ...).  A slot of 128 threads (see below) fetches a tile of
// 2^(k+7) amplitudes (128 groups) with bulk asynchronous copies; each thread
// takes one group and splits every value into a TF32 head and an FP32 tail
// (x = hi + lo), A_hi into the tensor cores' canonical K-major layout in
// shared memory and A_lo into tensor memory (the thread's lane).  One thread
// issues
//
//     D = A_lo B_hi^T + A_hi B_lo^T + A_hi B_hi^T      (3xTF32, FP32 accumulate)
//
// as tcgen05.mma instructions (M = 128, N = 2K, K = 8 per instruction) into
// tensor memory.  The accumulator is read back with tcgen05.ld, written into
// shared memory at the groups' positions and stored with bulk copies.
// B_hi / B_lo (from U) are prepared on the host and loaded once per CTA.
#include <cstring>

#include "common.cuh"
#include "kernels.hpp"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace qsim {

namespace {

constexpr int kMaxHTC = 10;
constexpr long long kWaitBudgetTC = 4000000000ll;

// byte offset of element (row, kk) in a canonical K-major no-swizzle operand
// with `kr` columns: 8 x 16-byte core matrices, K-adjacent ones 128 bytes
// apart, M-adjacent ones kr * 32 bytes apart
__host__ __device__ __forceinline__ uint32_t canon_off(uint32_t row, uint32_t kk, uint32_t kr) {
    return (row & 7u) * 16u + (kk & 3u) * 4u + (kk >> 2) * 128u + (row >> 3) * (kr * 32u);
}

// Slots: one CTA per SM holds NS independent pipelines of 128 threads (four
// warps = the 128 tensor-memory lanes), each with its own tile and operand
// buffers, barriers and accumulator columns, all sharing one copy of B_hi /
// B_lo.  A slot's steps (fetch, split, MMA, epilogue, store) run in order,
// the slots overlap one another.
template <int K> struct TcSlots;
template <> struct TcSlots<4> { static constexpr int NS = 4; };  // 4 x 32 KiB + 8 KiB
template <> struct TcSlots<5> { static constexpr int NS = 3; };  // 3 x 64 KiB + 32 KiB
constexpr int kSlotThreads = 128;
// Lane rotation against shared-memory bank conflicts (see the kernel).  It
// pays for 4-qubit blocks (30-qubit random circuit: 612 -> 584 ms); for
// 5-qubit blocks its register swaps cost more than the conflicts they remove
// (432 -> 496 ms), so they run without it.
template <int K> constexpr bool kRotate = (K == 4);

__device__ __forceinline__ void slot_sync(uint32_t id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// OR of v over the slot's 128 threads (a barrier as well)
__device__ __forceinline__ bool slot_any(bool v, uint32_t id) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(r) : "r"((uint32_t)v), "r"(id) : "memory");
    return r != 0;
}

template <int K>
__global__ void __launch_bounds__(kSlotThreads * TcSlots<K>::NS, 1)
    k_fused_tc(float2 *__restrict__ a, TileGeom g, FusedMap fm, const float *__restrict__ bmat, uint32_t *err,
               uint64_t ntiles) {
    constexpr int NS = TcSlots<K>::NS;
    constexpr int CK = 1 << K;              // amplitudes of a group
    constexpr int KR = 2 * CK;              // real columns = 2 * 2^K
    constexpr int N = KR;                   // output columns
    constexpr int T = K + 7;                // 128 groups per tile
    constexpr uint32_t TS = 1u << T;
    constexpr uint32_t OPB = 8u << T;       // tile / operand bytes
    constexpr uint32_t BB = (uint32_t)N * KR * 4u;
    // tensor memory per slot: the accumulator (N columns), then A_lo (KR columns)
    constexpr uint32_t SCOLS = N + KR;
    constexpr uint32_t TCOLS = NS * SCOLS <= 128 ? 128 : NS * SCOLS <= 256 ? 256 : 512;
    static_assert(NS * SCOLS <= 512, "tensor memory");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *s_bhi = smem_raw;
    unsigned char *s_blo = smem_raw + BB;
    __shared__ __align__(8) uint64_t bar_ld[NS], bar_mma[NS], bar_b;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_hb[kMaxHTC];     // the high tile bits, indexed at run time
    __shared__ uint32_t s_sink[kSlotThreads / 32 * NS];  // written, never read (see the fetch)
    const int L = g.L, H = g.H;
    const uint32_t nruns = 1u << H;
    const uint32_t run_bytes = 8u << L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = threadIdx.x / kSlotThreads, st = threadIdx.x % kSlotThreads, ws = st >> 5;
    const uint32_t bar_id = 1u + (uint32_t)slot;  // named barrier of the slot (0 is __syncthreads)
    unsigned char *s_tile = smem_raw + 2 * BB + (size_t)slot * 2 * OPB;  // the fetched tile
    unsigned char *s_ahi = s_tile + OPB;                                // A_hi, then the output tile

    if (threadIdx.x == 0) {  // (compile-time indices into the parameters: no local-memory copy)
#pragma unroll
        for (int k = 0; k < kMaxHTC; k++) s_hb[k] = k < H ? g.hb[k] : 0;
        for (int i = 0; i < NS; i++) {
            mbar_init(&bar_ld[i], 1);
            mbar_init(&bar_mma[i], 1);
        }
        mbar_init(&bar_b, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = tmem_slot + (uint32_t)slot * SCOLS;  // the slot's accumulator
    const uint32_t tmem_alo = tmem_d + N;                         // and its A_lo

    // B_hi, B_lo: 2 x BB bytes from global, once per CTA
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar_b, 2 * BB);
        bulk_g2s(s_bhi, bmat, BB, &bar_b);
        bulk_g2s(s_blo, bmat + BB / 4, BB, &bar_b);
    }
    // every abort decision goes through a vote, so the threads of a slot
    // leave its loop at the same barrier
    bool aborted = __syncthreads_or(!mbar_wait_bounded(&bar_b, 0, kWaitBudgetTC)) != 0;

    // This thread owns group (row) m = its tensor-memory lane: the tile bits
    // of m, and of the block's input / output columns.
    const uint32_t m = (uint32_t)(32 * ws + lane);
    uint32_t ibase = 0, w_col[K];
#pragma unroll
    for (int b = 0; b < T - K; b++) ibase |= ((m >> b) & 1u) << fm.row[b];
#pragma unroll
    for (int b = 0; b < K; b++) w_col[b] = 1u << fm.col[b];
    // Lane rotation against bank conflicts: the 16 lanes of a half-warp read
    // (and later write) 16 different 8-byte words of a bank row only if the
    // tile bits 0..3 of their addresses differ.  A lane bit l < 4 whose row
    // bit lies at tile bit >= 4 is paired with a gate column j at tile bit < 4
    // (there are as many of each): the lane visits column c ^ rot at step c,
    // rot = sum of (lane bit l) << j, and conditional swaps of register pairs
    // undo the order.  rmask: the rotated column bits (the same for all lanes).
    uint32_t rot = 0, rmask = 0;
    if (kRotate<K>) {
        uint32_t freecol = 0;  // gate columns at tile bits < 4 (the lowest j, col[] ascends)
#pragma unroll
        for (int j = 0; j < K; j++)
            if (fm.col[j] < 4) freecol |= 1u << j;
#pragma unroll
        for (int l = 0; l < 4; l++)
            if (fm.row[l] >= 4 && freecol) {
                const int j = __ffs(freecol) - 1;
                freecol &= freecol - 1u;
                rot |= (((uint32_t)lane >> l) & 1u) << j;
                rmask |= 1u << j;
            }
    }
    uint32_t rbase = ibase;  // the group's tile index with the rotated column bits set
#pragma unroll
    for (int b = 0; b < 4; b++)
        if ((rot >> b) & 1u) rbase |= w_col[b];
    // byte offset of row m in the canonical K-major operand (see canon_off)
    const uint32_t arow = (m & 7u) * 16u + (m >> 3) * (uint32_t)(KR * 32);
    const uint32_t lane_off = (uint32_t)(32 * ws) << 16;  // tensor-memory lane field of this warp

    auto run_off = [&](uint32_t j) {  // offset of run j: its bits deposited at the high tile bits
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << s_hb[k];
        return o;
    };
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        return base;
    };
    float2 *tin = reinterpret_cast<float2 *>(s_tile);
    auto issue_load = [&](uint64_t tile) {  // warp 0 of the slot
        const uint64_t base = tile_base(tile);
        if (lane == 0) mbar_arrive_expect_tx(&bar_ld[slot], TS * 8u);
        __syncwarp();
        for (uint32_t j = lane; j < nruns; j += 32)
            bulk_g2s(tin + ((size_t)j << L), a + (base | run_off(j)), run_bytes, &bar_ld[slot]);
    };
    uint32_t ld_parity = 0, mma_parity = 0;
    const uint64_t stride = (uint64_t)gridDim.x * NS;
    uint64_t tile = (uint64_t)blockIdx.x * NS + slot;
    // Pipeline of a slot: once every thread holds its group in registers the
    // next tile is fetched into the load buffer, under this tile's split,
    // MMAs, epilogue and store; the store's reads of the output buffer are
    // awaited only when the next split is about to overwrite it.
    if (ws == 0 && !aborted && tile < ntiles) issue_load(tile);
    for (; tile < ntiles && !aborted; tile += stride) {
        const uint64_t base = tile_base(tile);
        aborted = slot_any(!mbar_wait_bounded(&bar_ld[slot], ld_parity, kWaitBudgetTC), bar_id);
        if (aborted) {
            mbar_wait_bounded(&bar_ld[slot], ld_parity, kWaitBudgetTC);  // let the copies in flight land
            break;
        }
        ld_parity ^= 1u;

        // The group in parts of HS amplitudes: read (step c reads column
        // c ^ rot), undo the rotation, split x = hi (TF32) + lo, A_hi into the
        // canonical K-major layout in shared memory (two amplitudes = one
        // 16-byte chunk), A_lo into tensor memory (lane m, column 2c + re/im).
        // Once the last part is read the fetch buffer is free and the next
        // tile's fetch starts.
        constexpr int HS = kRotate<K> ? 16 : CK;  // the rotation's swaps want few live registers
#pragma unroll
        for (int p = 0; p < CK / HS; p++) {
            float2 x[HS];  // input columns HS p .. HS p + HS - 1
#pragma unroll
            for (int c = 0; c < HS; c++) {
                uint32_t i = rbase;
#pragma unroll
                for (int b = 0; b < K; b++)
                    if (((HS * p + c) >> b) & 1) i ^= w_col[b];
                x[c] = tin[i];
            }
            if (kRotate<K>) {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if ((rmask >> j) & 1u) {
                        const bool sw = (rot >> j) & 1u;
#pragma unroll
                        for (int c = 0; c < HS; c++)
                            if (!((c >> j) & 1)) {
                                const float2 u = x[c], v = x[c | (1 << j)];
                                x[c] = sw ? v : u;
                                x[c | (1 << j)] = sw ? u : v;
                            }
                    }
            }
            if (p == 0) {
                if (ws == 0) bulk_wait_read_all();  // the previous store has read the output buffer
                if (p < CK / HS - 1) slot_sync(bar_id);
            }
            if (p == CK / HS - 1) {
                // The fetch buffer goes back to the bulk copies: every load
                // of this part has returned (their words reduced over the
                // warp and kept by a shared-memory store -- with no rotation
                // nothing else uses them before the barrier) and is ordered
                // before the copy that overwrites the buffer.
                uint32_t fold = 0;
#pragma unroll
                for (int c = 0; c < HS; c++) fold ^= __float_as_uint(x[c].x) ^ __float_as_uint(x[c].y);
                fold = __reduce_xor_sync(0xffffffffu, fold);
                if (lane == 0) s_sink[warp] = fold;
                fence_proxy_async_smem();
                slot_sync(bar_id);
                if (ws == 0 && tile + stride < ntiles) issue_load(tile + stride);  // the fetch buffer is free
            }
#pragma unroll
            for (int h = 0; h < HS / 16; h++) {
                uint32_t lo[32];
#pragma unroll
                for (int cc = 0; cc < 16; cc += 2) {
                    const int e = 16 * h + cc, c = HS * p + e;
                    const float4 hv = make_float4(to_tf32(x[e].x), to_tf32(x[e].y), to_tf32(x[e + 1].x),
                                                  to_tf32(x[e + 1].y));
                    *reinterpret_cast<float4 *>(s_ahi + arow + (uint32_t)(c >> 1) * 128u) = hv;
                    lo[2 * cc] = __float_as_uint(x[e].x - hv.x);
                    lo[2 * cc + 1] = __float_as_uint(x[e].y - hv.y);
                    lo[2 * cc + 2] = __float_as_uint(x[e + 1].x - hv.z);
                    lo[2 * cc + 3] = __float_as_uint(x[e + 1].y - hv.w);
                }
                tmem_st32(tmem_alo + lane_off + (uint32_t)(32 * (HS / 16 * p + h)), lo);
            }
        }
        tmem_st_wait();
        fence_proxy_async_smem();  // generic-proxy writes -> tensor-core (async proxy) reads
        tc_fence_before();
        slot_sync(bar_id);
        tc_fence_after();

        if (st == 0) {
            const uint32_t ahi = smem_u32(s_ahi);
            const uint32_t bhi = smem_u32(s_bhi), blo = smem_u32(s_blo);
            const uint32_t idesc = umma_idesc_tf32(128, N);
            // Each accumulation into the FP32 accumulator loses a little
            // magnitude relative to the running sum (measured: a systematic
            // norm loss per block, not a random one): the small cross
            // products go in first, while the sum is small, and the head
            // products last, so that only one accumulation per K step rounds
            // at the output's scale.
#pragma unroll
            for (int ks = 0; ks < KR / 8; ks++) {
                const uint32_t o = (uint32_t)ks * 256u;  // 8 TF32 along K = two core matrices
                umma_tf32_ts(tmem_d, tmem_alo + (uint32_t)(8 * ks), umma_desc(bhi + o, 128, KR * 32), idesc,
                             ks > 0 ? 1u : 0u);
                umma_tf32(tmem_d, umma_desc(ahi + o, 128, KR * 32), umma_desc(blo + o, 128, KR * 32), idesc, 1u);
            }
#pragma unroll
            for (int ks = 0; ks < KR / 8; ks++) {
                const uint32_t o = (uint32_t)ks * 256u;
                umma_tf32(tmem_d, umma_desc(ahi + o, 128, KR * 32), umma_desc(bhi + o, 128, KR * 32), idesc, 1u);
            }
            umma_commit(&bar_mma[slot]);
        }
        aborted = slot_any(!mbar_wait_bounded(&bar_mma[slot], mma_parity, kWaitBudgetTC), bar_id);
        mma_parity ^= 1u;
        tc_fence_after();
        if (aborted) break;

        // epilogue: warp ws reads its 32 lanes (groups), 32 columns (16
        // outputs) at a time, into the output buffer at the groups' positions
        float2 *tout = reinterpret_cast<float2 *>(s_ahi);
#pragma unroll
        for (int chunk = 0; chunk < N / 32; chunk++) {
            uint32_t r[32];
            tmem_ld32(tmem_d + lane_off + (uint32_t)(32 * chunk), r);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 4; j++)  // output q of the chunk -> register pair q ^ rot
                if (kRotate<K> && ((rmask >> j) & 1u)) {
                    const bool sw = (rot >> j) & 1u;
#pragma unroll
                    for (int q = 0; q < 16; q++)
                        if (!((q >> j) & 1)) {
                            const int p = q | (1 << j);
                            const uint32_t u0 = r[2 * q], u1 = r[2 * q + 1], v0 = r[2 * p], v1 = r[2 * p + 1];
                            r[2 * q] = sw ? v0 : u0;
                            r[2 * q + 1] = sw ? v1 : u1;
                            r[2 * p] = sw ? u0 : v0;
                            r[2 * p + 1] = sw ? u1 : v1;
                        }
                }
            const uint32_t cb = (K == 5 && chunk) ? w_col[K - 1] : 0u;  // output bit 4 = the chunk
#pragma unroll
            for (int q = 0; q < 16; q++) {  // step q writes output q ^ rot
                uint32_t i = rbase | cb;
#pragma unroll
                for (int b = 0; b < 4; b++)
                    if ((q >> b) & 1) i ^= w_col[b];
                tout[i] = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
            }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        slot_sync(bar_id);
        if (ws == 0) {
            for (uint32_t j = lane; j < nruns; j += 32)
                bulk_s2g(a + (base | run_off(j)), tout + ((size_t)j << L), run_bytes);
            bulk_commit();
        }
    }
    if (aborted && st == 0) atomicExch(err, kErrTimeout);
    if (ws == 0) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem_slot, TCOLS);
}

template <int K>
cudaError_t launch_k(void *amp, const TileGeom &g, const FusedMap &fm, const float *bmat, uint32_t *err,
                     int sm_count, cudaStream_t s) {
    constexpr int NS = TcSlots<K>::NS;
    constexpr int KR = 2 << K;
    constexpr int T = K + 7;
    // B_hi / B_lo, then per slot a tile and an operand buffer
    const size_t smem = 2 * (size_t)KR * KR * 4 + (size_t)NS * 2 * ((size_t)8 << T);
    const uint64_t ntiles = 1ull << (g.n - T);
    cudaError_t e = cudaFuncSetAttribute(k_fused_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one CTA per SM (its slots share B); fewer when there are fewer tiles
    uint64_t grid = (ntiles + NS - 1) / NS;
    if (grid > (uint64_t)sm_count) grid = (uint64_t)sm_count;
    k_fused_tc<K><<<(unsigned)grid, kSlotThreads * NS, smem, s>>>(static_cast<float2 *>(amp), g, fm, bmat, err,
                                                                  ntiles);
    return cudaGetLastError();
}

}  // namespace

// Host: B_hi / B_lo of a fused gate in the canonical layout (see above).
// U: 2^k x 2^k complex, row-major (re, im) FP64.  out: 2 * (2K)^2 floats.
void fused_tc_prepare_b(int k, const double *U, float *out) {
    const int K = 1 << k, KR = 2 * K;
    float *hi = out, *lo = out + KR * KR;
    for (int i = 0; i < KR * KR; i++) hi[i] = lo[i] = 0.0f;
    auto tf32 = [](float x) {
        uint32_t b;
        std::memcpy(&b, &x, 4);
        b = (b + 0x1000u) & 0xFFFFE000u;  // nearest, ties away from zero, 10 significand bits
        float r;
        std::memcpy(&r, &b, 4);
        return r;
    };
    for (int r = 0; r < K; r++)
        for (int c = 0; c < K; c++) {
            const double ur = U[2 * (r * K + c)], ui = U[2 * (r * K + c) + 1];
            // output column n (2r: re, 2r+1: im) against input element kk (2c: re, 2c+1: im)
            const double v[4] = {ur, -ui, ui, ur};
            const int nn[4] = {2 * r, 2 * r, 2 * r + 1, 2 * r + 1};
            const int kk[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
            for (int e = 0; e < 4; e++) {
                const float h = tf32((float)v[e]);
                const float l = (float)(v[e] - (double)h);
                const uint32_t off = canon_off((uint32_t)nn[e], (uint32_t)kk[e], (uint32_t)KR) / 4u;
                hi[off] = h;
                lo[off] = l;
            }
        }
}

bool fused_tc_supported(int dt, int k, int n) { return dt == 0 && (k == 4 || k == 5) && n >= k + 7; }

cudaError_t launch_fused_tc(void *amp, int k, const TileGeom &g, const FusedMap &fm, const float *bmat,
                            uint32_t *err, int sm_count, cudaStream_t s) {
    if (g.L + g.H != k + 7 || g.H > kMaxHTC || g.L < 1) return cudaErrorInvalidValue;
    if (k == 4) return launch_k<4>(amp, g, fm, bmat, err, sm_count, s);
    if (k == 5) return launch_k<5>(amp, g, fm, bmat, err, sm_count, s);
    return cudaErrorInvalidValue;
}

}  // namespace qsim
