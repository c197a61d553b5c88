// k_fused_tc6.cu -- complex64 dense 6-qubit gates on the tensor cores.
//
// A fused gate is the FP64 product U of the gates it replaces (2^6 x 2^6,
// built on the host).  For every group of 64 amplitudes that differ only in
// the six qubits, a' = U a.  With complex numbers as real 2x2 blocks this is
//
//     D (rows = groups, 128 columns) = A (groups x 128) * B^T.
//
// The two operands of a 128 x 128 real product do not fit shared memory as
// TF32 pairs (B alone would take 128 KiB), so both are cut into three bf16
// slices, x = x_hi + x_mid + x_lo (each the bf16 rounding of the remainder,
// 24 significand bits in all), and the six products with the largest terms
//
//     A_hi B_hi + A_hi B_mid + A_mid B_hi + A_hi B_lo + A_mid B_mid + A_lo B_hi
//
// run as tcgen05.mma kind::f16 with FP32 accumulation in tensor memory: the
// dropped products are below 2^-24 of the result, the complex64 class.
//
// One CTA per SM, 640 threads (20 warps, five per scheduler): 16 compute
// warps -- the four warps of a tensor-memory lane quarter share its 32
// groups, each taking one quarter of a group's 64 amplitudes (two K steps of
// 16 reals) -- and one duty warp per scheduler: the MMA warp, the fetch warp
// and two idle ones.  Per tile of 128 groups (8192 amplitudes, 64 KiB):
//   1. the fetch warp copies the tile (bulk asynchronous copies) into one of
//      two shared-memory buffers once the tile two before was read out of it;
//   2. fetch: each compute thread reads its 16 amplitudes into registers;
//   3. slices: the thread writes the three bf16 slices into tensor memory;
//   4. the MMA warp issues 6 products x 8 K steps = 48 MMAs (N = 128);
//   5. the thread reads its 32 output reals from the accumulator and stores
//      them from registers to global memory.
// The A slices are double-buffered in tensor memory: tile i + 2's slices
// are written while tile i + 1's MMAs run, so the MMAs of consecutive tiles
// are separated only by the read-out of the accumulator.  Hand-offs go
// through mbarriers, every wait bounded.
// Tensor memory: the accumulator at columns 0..127, the A slices of tile t
// at 128 + 192 (t & 1) + 8 (3 ks + s) (K step ks, slice s = hi, mid, lo).
// All 512 columns.
#include <cstring>
#include <cmath>

#include "common.cuh"
#include "fpair.cuh"
#include "kernels.hpp"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace qsim {

namespace {

constexpr int kK6 = 6;
constexpr int kAmps6 = 1 << kK6;                 // 64 amplitudes of a group
constexpr int kReals6 = 2 * kAmps6;              // 128: K and N of the product
constexpr int kTileBits6 = kK6 + 7;              // 128 groups per tile
constexpr uint32_t kTileBytes6 = 8u << kTileBits6;            // 64 KiB
constexpr uint32_t kSliceBytes6 = kReals6 * kReals6 * 2;      // 32 KiB per B slice
constexpr uint32_t kBBytes6 = 3 * kSliceBytes6;               // 96 KiB
constexpr uint32_t kAcc6 = kReals6;                           // accumulator columns
constexpr uint32_t kABuf6 = 8u * 3u * 8u;                     // A slice columns of one tile (192)
constexpr uint32_t kTmemCols6 = 512;
constexpr int kCompute6 = 512;
constexpr int kThreads6 = 640;
constexpr int kMaxH6 = 10;
constexpr long long kWaitBudget6 = 4000000000ll;

// byte offset of element (n, kk) in a bf16 K-major, no-swizzle operand of 128
// K columns: core matrices of 8 rows x 16 bytes, K-adjacent ones 128 bytes
// apart, row-adjacent ones 2048 bytes apart
__host__ __device__ constexpr uint32_t bcanon6(uint32_t n, uint32_t kk) {
    return (n & 7u) * 16u + (kk & 7u) * 2u + (kk >> 3) * 128u + (n >> 3) * 2048u;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc6(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma6(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc6(128, kReals6)), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tst8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// OR vote of the 512 compute threads (named barrier 5)
__device__ __forceinline__ bool vote6(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, 5, 512, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(r) : "r"((uint32_t)v) : "memory");
    return r != 0;
}

// bf16 rounding (nearest, ties to even) of a float, as a float; the bf16
// bit pattern is its top half
__host__ __device__ __forceinline__ float bf16_rn(float x) {
#if defined(__CUDA_ARCH__)
    uint32_t b = __float_as_uint(x);
#else
    uint32_t b;
    std::memcpy(&b, &x, 4);
#endif
    b = (b + 0x7fffu + ((b >> 16) & 1u)) & 0xffff0000u;
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float r;
    std::memcpy(&r, &b, 4);
    return r;
#endif
}

// two floats rounded to bf16 (nearest, ties to even) in one word: lo in
// bits 0..15, hi in 16..31 (the order of K-adjacent operand elements)
__device__ __forceinline__ uint32_t pack_bf16_rn(float lo, float hi) {
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
    return w;
}
__device__ __forceinline__ fpair unpack_bf16(uint32_t w) {
    return fpair{__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u)};
}

// the three bf16 slices of a pair of reals (re, im) packed as K-adjacent
// words: each slice the bf16 rounding of the remainder (the remainders are
// exact), re and im together
__device__ __forceinline__ void split3(float re, float im, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
    fpair x{re, im};
    w0 = pack_bf16_rn(x.x, x.y);
    x = fp_sub(x, unpack_bf16(w0));
    w1 = pack_bf16_rn(x.x, x.y);
    x = fp_sub(x, unpack_bf16(w1));
    w2 = pack_bf16_rn(x.x, x.y);
}

__global__ void __launch_bounds__(kThreads6, 1)
    k_fused_tc6(float2 *__restrict__ a, TileGeom g, FusedMap fm, const uint16_t *__restrict__ bmat, uint32_t *err,
                uint64_t ntiles) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *s_b = smem_raw;                   // B slices hi, mid, lo
    unsigned char *s_buf0 = smem_raw + kBBytes6;     // two input buffers
    // bar_ld: tile arrived in buffer b; bar_free: the compute warps have read
    // buffer b into registers; bar_ready: the tile's A slices written and the
    // last tile's accumulator read (its MMAs may start); bar_mma: MMAs done;
    // bar_b: B loaded
    __shared__ __align__(8) uint64_t bar_ld[2], bar_free[2], bar_ready, bar_mma, bar_b;
    __shared__ uint32_t s_sink[32];  // written, never read (see the fetch)
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_hb[kMaxH6];
    const int L = g.L, H = g.H;
    const uint32_t nruns = 1u << H;
    const uint32_t run_bytes = 8u << L;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < kMaxH6; k++) s_hb[k] = k < H ? g.hb[k] : 0;
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar_ld[b], 1);
            mbar_init(&bar_free[b], kCompute6 / 32);
        }
        mbar_init(&bar_ready, kCompute6 / 32);
        mbar_init(&bar_mma, 1);
        mbar_init(&bar_b, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, kTmemCols6);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    auto run_off = [&](uint32_t j) {
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << s_hb[k];
        return o;
    };
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        return base;
    };
    auto buf = [&](int b) { return s_buf0 + (size_t)b * kTileBytes6; };
    const uint64_t stride = gridDim.x;
    const uint32_t count = blockIdx.x < ntiles ? (uint32_t)((ntiles - 1 - blockIdx.x) / stride + 1) : 0u;

    if (warp == kCompute6 / 32 && lane == 0) {
        // ---- MMA warp: 6 slice products x 8 K steps into the accumulator
        const uint64_t bdesc0 = umma_desc(smem_u32(s_b), 128, 2048);
        constexpr int PA[6] = {0, 0, 1, 0, 1, 2};  // A slice of each product
        constexpr int PB[6] = {0, 1, 0, 2, 1, 0};  // B slice
        uint32_t issued = 0;
        bool ok = mbar_wait_bounded(&bar_b, 0, kWaitBudget6);
        for (uint32_t t = 0; t < count && ok; t++) {
            ok = mbar_wait_bounded(&bar_ready, t & 1u, kWaitBudget6);
            if (!ok) break;
            tc_fence_after();
            const uint32_t abuf = tmem + kAcc6 + kABuf6 * (t & 1u);
            // Each accumulation into the FP32 accumulator loses a little
            // magnitude relative to the running sum (measured: a systematic
            // norm loss of about 1.5e-6 per block with the products in K-step
            // order, 48 accumulations at the output's scale): the five smaller
            // products of every K step go in first, while the sum is small,
            // and the head products (hi x hi) last, so that only 8
            // accumulations round at the output's scale (about 1e-7).
#pragma unroll
            for (int p = 1; p < 6; p++)
#pragma unroll
                for (int ks = 0; ks < 8; ks++)
                    mma6(tmem, abuf + 8u * (3 * ks + PA[p]),
                         bdesc0 + (uint64_t)((PB[p] * kSliceBytes6 + ks * 256) / 16), (p > 1 || ks > 0) ? 1u : 0u);
#pragma unroll
            for (int ks = 0; ks < 8; ks++)
                mma6(tmem, abuf + 8u * (3 * ks + PA[0]), bdesc0 + (uint64_t)((PB[0] * kSliceBytes6 + ks * 256) / 16),
                     1u);
            umma_commit(&bar_mma);
            issued++;
        }
        if (issued) mbar_wait_bounded(&bar_mma, (issued - 1u) & 1u, kWaitBudget6);
        if (!ok) atomicExch(err, kErrTimeout);
    } else if (warp == kCompute6 / 32 + 1) {
        // ---- fetch warp: tile k into buffer k & 1 once tile k - 2 was read
        uint32_t issued0 = 0u, issued1 = 0u;
        auto issue_load = [&](uint32_t i) {
            const int b = (int)(i & 1u);
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * stride);
            if (lane == 0) mbar_arrive_expect_tx(&bar_ld[b], kTileBytes6);
            __syncwarp();
            float2 *dst = reinterpret_cast<float2 *>(buf(b));
            for (uint32_t j = lane; j < nruns; j += 32)
                bulk_g2s(dst + ((size_t)j << L), a + (base | run_off(j)), run_bytes, &bar_ld[b]);
            if (b) issued1++; else issued0++;
        };
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar_b, kBBytes6);
            bulk_g2s(s_b, bmat, kBBytes6 / 2, &bar_b);
            bulk_g2s(s_b + kBBytes6 / 2, bmat + kBBytes6 / 4, kBBytes6 / 2, &bar_b);
        }
        bool ok = true;
        for (uint32_t k = 0; k < count && ok; k++) {
            if (k >= 2) ok = mbar_wait_bounded(&bar_free[k & 1u], ((k - 2) >> 1) & 1u, kWaitBudget6);
            if (ok) issue_load(k);
        }
        if (issued0) mbar_wait_bounded(&bar_ld[0], (issued0 - 1u) & 1u, kWaitBudget6);
        if (issued1) mbar_wait_bounded(&bar_ld[1], (issued1 - 1u) & 1u, kWaitBudget6);
    } else if (warp < kCompute6 / 32) {
        // ---- compute warps: group m (tensor-memory lane), quarter qq of its
        // 64 amplitudes (columns 16 qq .. 16 qq + 15 = K steps 2 qq, 2 qq + 1)
        const int lq = warp & 3, qq = warp >> 2;
        const uint32_t m = (uint32_t)(32 * lq + lane);
        const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
        uint32_t ibase = 0;
#pragma unroll
        for (int b = 0; b < kTileBits6 - kK6; b++) ibase |= ((m >> b) & 1u) << fm.row[b];
        uint32_t wc[kK6];
#pragma unroll
        for (int b = 0; b < kK6; b++) wc[b] = 1u << fm.col[b];
        const uint32_t qbase = ibase | ((qq & 1) ? wc[4] : 0u) | ((qq & 2) ? wc[5] : 0u);
        const uint32_t lowmask = (1u << L) - 1u;
        auto goff = [&](uint32_t t) { return (uint64_t)(t & lowmask) | run_off(t >> L); };
        const uint64_t gq = goff(qbase);
        uint64_t gc[4];
#pragma unroll
        for (int b = 0; b < 4; b++) gc[b] = goff(wc[b]);
        auto coff = [&](int j) {  // tile index of column 16 qq + j
            return qbase | ((j & 1) ? wc[0] : 0u) | ((j & 2) ? wc[1] : 0u) | ((j & 4) ? wc[2] : 0u) |
                   ((j & 8) ? wc[3] : 0u);
        };
        const uint32_t acol = tmem + lane_off + kAcc6;  // A slices of this lane (buffer 0)

        bool aborted = vote6(!mbar_wait_bounded(&bar_b, 0, kWaitBudget6));
        float2 v[16];
        // fetch(i): this thread's 16 amplitudes of tile i into registers;
        // false (for the whole warp) if the copy did not arrive in time --
        // the caller folds that into the next block-wide vote
        auto fetch = [&](uint32_t i) -> bool {
            const int b = (int)(i & 1u);
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar_ld[b], (i >> 1) & 1u, kWaitBudget6));
            const uint32_t sbuf = smem_u32(buf(b));
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                // columns j and j + 1 differ in column bit 0: two 8-byte loads
                const uint32_t p0 = sbuf + 8u * coff(j), p1 = sbuf + 8u * coff(j + 1);
                uint32_t a0, a1, b0, b1;
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(a0), "=r"(a1) : "r"(p0));
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(b0), "=r"(b1) : "r"(p1));
                v[j] = make_float2(__uint_as_float(a0), __uint_as_float(a1));
                v[j + 1] = make_float2(__uint_as_float(b0), __uint_as_float(b1));
            }
            // every load has returned (its words reduced over the warp and
            // kept by a shared-memory store) and is ordered before the bulk
            // copy that will overwrite the buffer
            uint32_t fold = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) fold ^= __float_as_uint(v[j].x) ^ __float_as_uint(v[j].y);
            fold = __reduce_xor_sync(0xffffffffu, fold);
            if (lane == 0) s_sink[warp] = fold;
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_free[b]);  // this warp's share of the buffer is read
            return ok;
        };
        // slices(t): the three bf16 slices of the held amplitudes (tile t)
        // into tile t's A buffer, K steps 2 qq and 2 qq + 1
        auto slices = [&](uint32_t t) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                uint32_t w[3][8];
#pragma unroll
                for (int j = 0; j < 8; j++) split3(v[8 * h + j].x, v[8 * h + j].y, w[0][j], w[1][j], w[2][j]);
                const uint32_t kcol = acol + kABuf6 * (t & 1u) + 8u * 3u * (uint32_t)(2 * qq + h);
#pragma unroll
                for (int s = 0; s < 3; s++) tst8(kcol + 8u * s, w[s]);
            }
        };
        auto arrive_ready = [&]() {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_ready);
        };

        // prologue: tile 0's slices (its MMAs start), tile 1's slices into
        // the other buffer
        if (!aborted && count > 0) {
            aborted = vote6(!fetch(0));
            if (!aborted) {
                slices(0);
                tmem_st_wait();
                arrive_ready();
                if (count > 1) {
                    aborted = vote6(!fetch(1));
                    if (!aborted) slices(1);
                }
            }
        }
        bool bad = false;  // a fetch of this warp gave up (voted on with the next wait)
        // steady state, tile i's MMAs in flight and tile i + 1's slices in
        // place: once the MMAs are done, the accumulator is read out and tile
        // i + 1's MMAs may start; tile i is stored and tile i + 2 fetched and
        // split into the A buffer tile i's MMAs used, while they run
        for (uint32_t i = 0; i < count && !aborted; i++) {
            const bool next = i + 1 < count;
            if (vote6(bad || !mbar_wait_bounded(&bar_mma, i & 1u, kWaitBudget6))) {
                aborted = true;
                break;
            }
            tc_fence_after();
            // tile i's 32 output reals of this thread: columns 32 qq .. 32 qq + 31
            uint32_t acc[2][16];
            tld16(tmem + lane_off + (uint32_t)(32 * qq), acc[0]);
            tld16(tmem + lane_off + (uint32_t)(32 * qq + 16), acc[1]);
            tmem_ld_wait();
            tmem_st_wait();
            if (next) arrive_ready();
            float2 *gt = a + tile_base(blockIdx.x + (uint64_t)i * stride);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint64_t go = gq | ((j & 1) ? gc[0] : 0ull) | ((j & 2) ? gc[1] : 0ull) |
                                    ((j & 4) ? gc[2] : 0ull) | ((j & 8) ? gc[3] : 0ull);
                gt[go] = make_float2(__uint_as_float(acc[j >> 3][(2 * j) & 15]),
                                     __uint_as_float(acc[j >> 3][(2 * j + 1) & 15]));
            }
            if (i + 2 < count) {
                bad = !fetch(i + 2);
                tc_fence_after();
                slices(i + 2);
            }
        }
        if (aborted && tid == 0) atomicExch(err, kErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols6);
}

}  // namespace

// Host: B_hi, B_mid, B_lo of a fused 6-qubit gate in the canonical layout.
// U: 64 x 64 complex, row-major (re, im) FP64.  out: 3 * 128 * 128 bf16 bit
// patterns.
void fused_tc6_prepare_b(const double *U, uint16_t *out) {
    std::memset(out, 0, kBBytes6);
    for (int r = 0; r < kAmps6; r++)
        for (int c = 0; c < kAmps6; c++) {
            const double ur = U[2 * (r * kAmps6 + c)], ui = U[2 * (r * kAmps6 + c) + 1];
            const double v[4] = {ur, -ui, ui, ur};
            const int nn[4] = {2 * r, 2 * r, 2 * r + 1, 2 * r + 1};
            const int kk[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
            for (int e = 0; e < 4; e++) {
                // the slices of the double entry: each the bf16 rounding of the remainder
                const float h = bf16_rn((float)v[e]);
                const double r1 = v[e] - (double)h;
                const float mdl = bf16_rn((float)r1);
                const float l = bf16_rn((float)(r1 - (double)mdl));
                const float sl[3] = {h, mdl, l};
                for (int s = 0; s < 3; s++) {
                    uint32_t b;
                    std::memcpy(&b, &sl[s], 4);
                    out[(s * kSliceBytes6 + bcanon6((uint32_t)nn[e], (uint32_t)kk[e])) / 2] = (uint16_t)(b >> 16);
                }
            }
        }
}

size_t fused_tc6_b_bytes() { return kBBytes6; }

bool fused_tc6_supported(int n) { return n >= kTileBits6; }

cudaError_t launch_fused_tc6(void *amp, const TileGeom &g, const FusedMap &fm, const uint16_t *bmat, uint32_t *err,
                             int sm_count, cudaStream_t s) {
    if (g.L + g.H != kTileBits6 || g.H > kMaxH6 || g.L < 1) return cudaErrorInvalidValue;
    const size_t smem = kBBytes6 + 2 * (size_t)kTileBytes6;
    cudaError_t e = cudaFuncSetAttribute(k_fused_tc6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t ntiles = 1ull << (g.n - kTileBits6);
    const uint64_t grid = ntiles < (uint64_t)sm_count ? ntiles : (uint64_t)sm_count;
    k_fused_tc6<<<(unsigned)grid, kThreads6, smem, s>>>(static_cast<float2 *>(amp), g, fm, bmat, err, ntiles);
    return cudaGetLastError();
}

}  // namespace qsim
