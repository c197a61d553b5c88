// k_fused_tc_c128.cu -- complex128 dense 5-qubit gates on the tensor cores.
//
// A fused gate is the FP64 product U of the gates it replaces (2^5 x 2^5,
// built on the host).  For every group of 32 amplitudes that differ only in
// the five qubits, a' = U a.  With complex numbers as real 2x2 blocks this is
//
//     D (rows = groups, 64 columns) = A (groups x 64) * B^T,
//
// a row of A being the group's 64 reals (re, im, re, im, ...).  The reals
// are cut into six bf16 digit slices against the group's largest exponent,
// and U's entries into six slices of their own (digits.cuh: the split, the
// exact level sums and the combination, with their error bounds).  The 21
// slice products A_i B_j^T with i + j <= 5 run as tcgen05.mma kind::f16
// (bf16 inputs, FP32 accumulation in tensor memory), accumulated per level
// (levels 0, 1, 2, 3 exactly, levels 4 and 5 together).
//
// Between the blocks of a run the state stays in double-float form: the same
// 16 bytes of an amplitude hold (re.hi, re.lo, im.hi, im.lo) as floats.  The
// first block of a run reads IEEE doubles (IN_IEEE) and the last one writes
// them (OUT_IEEE), converting with integer operations (df64.cuh).
//
// One CTA per SM, 608 threads (19 warps, 96 registers each): 16 compute
// warps -- the four warps of a tensor-memory lane quarter share its 32
// groups, each taking one quarter of a group's 32 amplitudes, which is one K
// step (16 reals) of the product -- and three duty warps: the MMA warp, the
// fetch warp and the store warp.  The duty warps issue work whose issue
// stalls (the tensor pipe and the bulk-copy engine take instructions only as
// fast as they execute them), so no compute warp waits for it.  Per tile of
// 128 groups (4096 amplitudes, 64 KiB):
//   1. the fetch warp copies the tile (bulk asynchronous copies, TMA engine)
//      into the input buffer as soon as the compute warps have read the tile
//      before out of it;
//   2. fetch: each compute thread reads its 8 amplitudes into registers and
//      the four threads of a group agree on its largest exponent;
//   3. split: the thread cuts its amplitudes into six bf16 digit slices,
//      kept in registers until the A slices in tensor memory are free, then
//      written there (its lane, 8 columns per slice);
//   4. the MMA warp issues the 21 products x 4 K steps of 16 as 48
//      instructions (slices of B side by side along N);
//   5. combination: each thread reads the accumulators of its 16 output
//      reals in two halves of 8, adds the levels in double-float and writes
//      the amplitudes into the output buffer at their tile positions; the
//      store warp copies the buffer's runs to global memory (bulk copies).
// The compute warps run tile i + 1's digits and tile i's combination around
// the MMAs: the MMA warp commits each K step of a tile on its own mbarrier, so
// the warps of a K quarter write the next tile's digits into their A slices
// as soon as the current tile's MMAs of that K step are done; once all are
// done and tile i's accumulators are read into registers, tile i + 1's
// MMAs start, and tile i's combination, its stores and tile i + 2's fetch and
// split run beside them.
// Shared-memory loads and stores of the amplitudes go through a per-lane
// rotation of the column index (no bank conflicts within a wavefront).
// Hand-offs go through mbarriers (tile fetched, buffer read, A slices ready,
// K step done, outputs written, outputs copied out), every wait bounded.
// Tensor memory: accumulators at columns 0..319 (level L at 64 L), the A
// slices at 320 + 48 s + 8 i (K step s, slice i): all 512 columns.
#include <cstring>
#include <cmath>

#include "common.cuh"
#include "digits.cuh"
#include "kernels.hpp"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace qsim {

namespace {

constexpr int kThreads128 = 512;            // compute threads: 16 warps
constexpr int kThreadsAll128 = 608;         // + the MMA-issue, fetch-issue and store-issue warps
constexpr int kK = 5;                          // qubits of a block
constexpr int kAmps = 1 << kK;                 // 32 amplitudes of a group
constexpr int kReals = 2 * kAmps;              // 64: K and N of the product
constexpr int kTileBits = kK + 7;              // 128 groups per tile
constexpr uint32_t kTileBytes = 16u << kTileBits;           // 64 KiB
constexpr uint32_t kSliceBytes = kReals * kReals * 2;       // 8 KiB per B slice
constexpr uint32_t kBBytes = kDigits * kSliceBytes;         // 48 KiB
constexpr uint32_t kAccCols = kDigitLevels * kReals;        // 320
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxH128 = 10;
constexpr long long kWaitBudget128 = 4000000000ll;

// byte offset of element (n, kk) in a bf16 K-major, no-swizzle operand of 64
// K columns: core matrices of 8 rows x 16 bytes, K-adjacent ones 128 bytes
// apart, row-adjacent ones 1024 bytes apart
__host__ __device__ constexpr uint32_t bcanon_off(uint32_t n, uint32_t kk) {
    return (n & 7u) * 16u + (kk & 7u) * 2u + (kk >> 3) * 128u + (n >> 3) * 1024u;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[tmem] * B[smem]^T, bf16 inputs, issued by one thread
__device__ __forceinline__ void umma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ uint4 lds_u4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

// barrier of the four warps sharing a tensor-memory lane quarter
__device__ __forceinline__ void quarter_sync(uint32_t id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// OR vote of the 512 compute threads (named barrier 5)
__device__ __forceinline__ bool compute_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, 5, 512, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(r) : "r"((uint32_t)v) : "memory");
    return r != 0;
}

template <bool IN_IEEE, bool OUT_IEEE>
__global__ void __launch_bounds__(kThreadsAll128, 1)
    k_fused_tc_c128(double2 *__restrict__ a, TileGeom g, FusedMap fm, const uint16_t *__restrict__ bmat,
                    uint32_t *err, uint64_t ntiles) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *s_b = smem_raw;                    // six B slices
    unsigned char *s_in = smem_raw + kBBytes;         // the tile being fetched
    unsigned char *s_out = s_in + kTileBytes;         // the outputs of the tile being stored
    // bar_ld: a tile arrived in s_in; bar_free: the compute warps have read
    // it into registers; bar_ready: tile's A slices written and the last
    // tile's accumulators read (MMAs may start); bar_mks[s]: the MMAs of K
    // steps 0..s done (bar_mks[3]: all); bar_out: a tile's outputs are in
    // s_out; bar_outfree: their bulk stores have read s_out; bar_b: B loaded
    __shared__ __align__(8) uint64_t bar_ld, bar_free, bar_ready, bar_mks[4], bar_out, bar_outfree, bar_b;
    __shared__ uint32_t tmem_base_s;
    __shared__ uint32_t s_max[2][4][128];  // per tile parity, K quarter, group: largest hi exponent field
    __shared__ int s_hb[kMaxH128];
    const int L = g.L, H = g.H;
    const uint32_t nruns = 1u << H;
    const uint32_t run_bytes = 16u << L;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < kMaxH128; k++) s_hb[k] = k < H ? g.hb[k] : 0;
        mbar_init(&bar_ld, 1);
        mbar_init(&bar_free, kThreads128 / 32);
        mbar_init(&bar_out, kThreads128 / 32);
        mbar_init(&bar_outfree, 1);
        mbar_init(&bar_ready, kThreads128 / 32);
        for (int ks = 0; ks < 4; ks++) mbar_init(&bar_mks[ks], 1);
        mbar_init(&bar_b, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    auto run_off = [&](uint32_t j) {  // bits of run j deposited at the high tile bits
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << s_hb[k];
        return o;
    };
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        return base;
    };
    const uint64_t stride = gridDim.x;
    // this CTA's tiles: blockIdx.x + i * stride, i < count
    const uint32_t count = blockIdx.x < ntiles ? (uint32_t)((ntiles - 1 - blockIdx.x) / stride + 1) : 0u;

    if (warp == kThreads128 / 32 && lane == 0) {
        // ---- MMA warp: tile t's products once its A slices are in place
        // One thread issues the 21 slice products, 4 K steps each.  The B
        // slices lie one after another along N (64 rows each, same layout),
        // and the accumulators of levels 0..4 one after another along the
        // columns, so slice i of A times B_0 .. B_(4-i) is a single MMA of
        // N = 64 (5 - i) into accumulators i .. 4 (two for i = 0: N <= 256);
        // the level-5 products (i + j = 5) go into accumulator 4 one by one:
        // 12 MMAs per K step.
        const uint64_t bdesc0 = umma_desc(smem_u32(s_b), 128, 1024);
        auto issue_mma = [&]() {
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                const uint32_t at = tmem + kAccCols + 48u * ks;    // A slice 0, K step ks
                const uint64_t bd = bdesc0 + (uint64_t)(ks * 256 / 16);  // B slice 0, K step ks
                const uint32_t acc0 = ks > 0 ? 1u : 0u;
                // i = 0: levels 0..3 (N = 256) and level 4 (N = 64), both start their accumulators
                umma_bf16_ts(tmem, at, bd, idesc_bf16(128, 256), acc0);
                umma_bf16_ts(tmem + 4u * kReals, at, bd + 4u * kSliceBytes / 16, idesc_bf16(128, kReals), acc0);
#pragma unroll
                for (int si = 1; si < kDigitLevels; si++)  // levels si .. 4 of slice si
                    umma_bf16_ts(tmem + (uint32_t)(si * kReals), at + 8u * si, bd,
                                 idesc_bf16(128, kReals * (kDigitLevels - si)), 1u);
#pragma unroll
                for (int si = 0; si < kDigits; si++)  // level 5 into accumulator 4
                    umma_bf16_ts(tmem + 4u * kReals, at + 8u * si, bd + (uint64_t)((kDigits - 1 - si) * kSliceBytes / 16),
                                 idesc_bf16(128, kReals), 1u);
                // K step ks read its A slices: the compute warps of that K
                // quarter may write the next tile's
                umma_commit(&bar_mks[ks]);
            }
        };

        uint32_t issued = 0;
        bool ok = mbar_wait_bounded(&bar_b, 0, kWaitBudget128);
        for (uint32_t t = 0; t < count && ok; t++) {
            ok = mbar_wait_bounded(&bar_ready, t & 1u, kWaitBudget128);
            if (!ok) break;
            tc_fence_after();
            issue_mma();
            issued++;
        }
        // the last products have finished before the CTA may free tensor memory
        if (issued) mbar_wait_bounded(&bar_mks[3], (issued - 1u) & 1u, kWaitBudget128);
        if (!ok) atomicExch(err, kErrTimeout);
    } else if (warp == kThreads128 / 32 + 1) {
        // ---- fetch warp: tile k into s_in once tile k - 1 was read out of it
        uint32_t issued = 0u;
        auto issue_load = [&](uint32_t i) {
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * stride);
            if (lane == 0) mbar_arrive_expect_tx(&bar_ld, kTileBytes);
            __syncwarp();
            double2 *dst = reinterpret_cast<double2 *>(s_in);
            for (uint32_t j = lane; j < nruns; j += 32)
                bulk_g2s(dst + ((size_t)j << L), a + (base | run_off(j)), run_bytes, &bar_ld);
            issued++;
        };
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar_b, kBBytes);
            bulk_g2s(s_b, bmat, kBBytes, &bar_b);
        }
        bool ok = true;
        for (uint32_t k = 0; k < count && ok; k++) {
            if (k >= 1) ok = mbar_wait_bounded(&bar_free, (k - 1u) & 1u, kWaitBudget128);
            if (ok) issue_load(k);
        }
        // every fetch has landed before the CTA may leave
        if (issued) mbar_wait_bounded(&bar_ld, (issued - 1u) & 1u, kWaitBudget128);
    } else if (warp == kThreads128 / 32 + 2) {
        // ---- store warp: a tile's outputs from s_out to global memory (bulk
        // copies, one per run) once the compute warps wrote them; s_out is
        // free again when the copies have read it
        bool ok = true;
        for (uint32_t i = 0; i < count && ok; i++) {
            ok = mbar_wait_bounded(&bar_out, i & 1u, kWaitBudget128);
            if (!ok) break;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * stride);
            const double2 *src = reinterpret_cast<const double2 *>(s_out);
            for (uint32_t j = lane; j < nruns; j += 32)
                bulk_s2g(a + (base | run_off(j)), src + ((size_t)j << L), run_bytes);
            bulk_commit();
            bulk_wait_read_all();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_outfree);
        }
        bulk_wait_all();  // the stores are complete before the CTA leaves
        if (!ok) atomicExch(err, kErrTimeout);
    } else if (warp < kThreads128 / 32) {
        // ---- compute warps: group m (tensor-memory lane), K quarter qq
        const int lq = warp & 3, qq = warp >> 2;
        const uint32_t m = (uint32_t)(32 * lq + lane);
        const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
        uint32_t ibase = 0;
#pragma unroll
        for (int b = 0; b < kTileBits - kK; b++) ibase |= ((m >> b) & 1u) << fm.row[b];
        uint32_t wc[kK];
#pragma unroll
        for (int b = 0; b < kK; b++) wc[b] = 1u << fm.col[b];
        // this thread's amplitudes: columns 8 qq + j, j < 8, and their tile
        // indices (the same in s_in and s_out)
        const uint32_t qbase = ibase | ((qq & 1) ? wc[3] : 0u) | ((qq & 2) ? wc[4] : 0u);
        // Shared-memory banks: the 8 lanes of one 128-byte wavefront of a
        // 16-byte access read or write 8 different 16-byte slots when tile
        // bits 0..2 vary across them.  Those that are rows vary with lane bits
        // 0..k-1 (rows are in ascending order); those that are columns 0..2 of
        // the thread are made to vary with the next lane bits by an XOR rot
        // on the column index of every load and store, undone in registers.
        uint32_t rot = 0;
        {
            uint32_t colmask = 0;
#pragma unroll
            for (int c = 0; c < kK; c++) colmask |= 1u << fm.col[c];
            int lb = 0;
#pragma unroll
            for (int b = 0; b < 3; b++) lb += ((colmask >> b) & 1u) ? 0 : 1;
#pragma unroll
            for (int c = 0; c < 3; c++)
                if (fm.col[c] <= 2) rot |= ((uint32_t)(lane >> lb++) & 1u) << c;
        }
        const bool rotated = __any_sync(0xffffffffu, rot != 0);  // the same in every warp
        auto colbits = [&](int j) {
            return ((j & 1) ? wc[0] : 0u) | ((j & 2) ? wc[1] : 0u) | ((j & 4) ? wc[2] : 0u);
        };
        // x[j] := x[j ^ rot] (after loads at rotated columns; before stores)
        auto unrot = [&](auto (&x)[8]) {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const bool sw = (rot >> b) & 1u;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (!(j & (1 << b))) {
                        const auto p = x[j], q2 = x[j | (1 << b)];
                        x[j] = sw ? q2 : p;
                        x[j | (1 << b)] = sw ? p : q2;
                    }
            }
        };
        auto coff = [&](int j) {
            return qbase | ((j & 1) ? wc[0] : 0u) | ((j & 2) ? wc[1] : 0u) | ((j & 4) ? wc[2] : 0u);
        };

        bool aborted = compute_any(!mbar_wait_bounded(&bar_b, 0, kWaitBudget128));
        uint32_t Eg_next = 0;
        const uint32_t acol = tmem + lane_off + kAccCols + 48u * (uint32_t)qq;  // this thread's A columns

        // Split of a tile in two steps.  fetch(i): wait for its copy, read
        // this thread's 8 amplitudes into registers (double-float form) and
        // agree with the group's other threads on the exponent field Eg_next
        // (false if the copy did not arrive in time).  digits(): the six
        // slices of the held amplitudes straight into the A slices (lane m,
        // K quarter qq), two amplitudes at a time.
        uint4 v[8];
        auto fetch = [&](uint32_t i) -> bool {
            const int b = (int)(i & 1u);  // s_max slot
            if (compute_any(!mbar_wait_bounded(&bar_ld, i & 1u, kWaitBudget128))) return false;
            const uint32_t sbuf = smem_u32(s_in);
            uint32_t mx = 0;
            const uint32_t cb = coff(0) | colbits((int)rot);  // coff(j ^ rot) = cb ^ colbits(j)
#pragma unroll
            for (int j = 0; j < 8; j++) {
                v[j] = lds_u4(sbuf + 16u * (cb ^ colbits(j)));
                if (IN_IEEE) {  // a double2 -> (re.h, re.l, im.h, im.l)
                    const df re = df_from_double(__hiloint2double((int)v[j].y, (int)v[j].x));
                    const df im = df_from_double(__hiloint2double((int)v[j].w, (int)v[j].z));
                    v[j] = make_uint4(__float_as_uint(re.h), __float_as_uint(re.l), __float_as_uint(im.h),
                                      __float_as_uint(im.l));
                }
                mx = max(mx, max(v[j].x & 0x7f800000u, v[j].z & 0x7f800000u));
            }
            if (rotated) unrot(v);
            s_max[b][qq][m] = mx;
            quarter_sync(1u + (uint32_t)lq);
            // this warp's amplitudes are in registers (the exponent maxima
            // above used every load): its share of the buffer is free, the
            // loads ordered before the bulk copy that overwrites it
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive(&bar_free);
            Eg_next = max(max(s_max[b][0][m], s_max[b][1][m]), max(s_max[b][2][m], s_max[b][3][m])) >> 23;
            return true;
        };
        // split(): the six slices of the held amplitudes as packed bf16
        // words (slice d, amplitude j: re and im digit), held in registers
        // until the A slices are free; put(): into the A slices (lane m,
        // K quarter qq), 8 columns per slice.
        uint32_t wd[kDigits][8];
        auto split = [&]() {
            const float sd = dg_scale_down(Eg_next);
#pragma unroll
            for (int j = 0; j < 8; j++) {  // re and im together (packed FP32x2)
                fpair dd[kDigits];
                dg_split_df2(fpair{__uint_as_float(v[j].x), __uint_as_float(v[j].z)},
                             fpair{__uint_as_float(v[j].y), __uint_as_float(v[j].w)}, sd, dd);
#pragma unroll
                for (int d = 0; d < kDigits; d++) wd[d][j] = dg_pack(dd[d].x, dd[d].y);
            }
        };
        auto put = [&]() {
#pragma unroll
            for (int d = 0; d < kDigits; d++) tmem_st8(acol + 8u * d, wd[d]);
        };
        // tile t's A slices are written (and tile t - 1's accumulators read):
        // one arrival per warp on bar_ready
        auto arrive_ready = [&]() {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_ready);
        };

        // prologue: tile 0 into tensor memory (its MMAs start), tile 1
        // fetched and split
        uint32_t Ecur = 0, Enext = 0;  // exponent fields of the tile whose MMAs run and of the next
        if (!aborted && count > 0) {
            aborted = !fetch(0);
            if (!aborted) {
                split();
                put();
                tmem_st_wait();
                arrive_ready();
                Ecur = Eg_next;
                if (count > 1) {
                    aborted = !fetch(1);
                    if (!aborted) {
                        split();
                        Enext = Eg_next;
                    }
                }
            }
        }
        // finish(i, next, bad): once tile i's MMAs are all done, its
        // accumulators are read out (then tile i + 1's MMAs may start, if
        // next), combined and stored; false if a wait gave up here or in a
        // warp (bad).
        auto finish = [&](uint32_t i, bool next, bool bad) -> bool {
            // s_out is free once the last tile's stores have read it
            const bool out_free = i == 0 || mbar_wait_bounded(&bar_outfree, (i - 1u) & 1u, kWaitBudget128);
            if (compute_any(bad || !out_free || !mbar_wait_bounded(&bar_mks[3], i & 1u, kWaitBudget128)))
                return false;
            tc_fence_after();
            // Tile i's accumulators, 16 output reals (8 amplitudes) in two
            // halves: levels 3 and 4-5 folded into one on arrival (rounding
            // below 2^-50 of the result), then levels 0, 1, 2.  Once both
            // halves are in registers, tile i + 1's MMAs may start.
            const float su = dg_scale_up(Ecur);
            const uint32_t so = smem_u32(s_out);
            uint32_t acc2[2][kDigitLevels - 1][8];
            auto drain = [&](int hf) {
                auto &acc = acc2[hf];
                uint32_t a4[8];
                const uint32_t c0 = tmem + lane_off + (uint32_t)(16 * qq + 8 * hf);
                tmem_ld8(c0 + kReals * 3, acc[3]);
                tmem_ld8(c0 + kReals * 4, a4);
                tmem_ld8(c0 + kReals * 0, acc[0]);
                tmem_ld8(c0 + kReals * 1, acc[1]);
                tmem_ld8(c0 + kReals * 2, acc[2]);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    const fpair f = fp_add(fpair{__uint_as_float(acc[3][c]), __uint_as_float(acc[3][c + 1])},
                                           fpair{__uint_as_float(a4[c]), __uint_as_float(a4[c + 1])});
                    acc[3][c] = __float_as_uint(f.x);
                    acc[3][c + 1] = __float_as_uint(f.y);
                }
            };
            // the 8 output reals of the half in acc as double-floats, the re
            // and im parts of an amplitude together (packed FP32x2)
            auto combine = [&](int hf, df (&o)[8]) {
                auto &acc = acc2[hf];
                auto pr = [&](int L, int c) {
                    return fpair{__uint_as_float(acc[L][c]), __uint_as_float(acc[L][c + 1])};
                };
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    fpair h, l;
                    dg_combine_df2(pr(0, c), pr(1, c), pr(2, c), pr(3, c), su, h, l);
                    o[c] = df{h.x, l.x};
                    o[c + 1] = df{h.y, l.y};
                }
            };
            // the 8 output amplitudes (re.h, re.l, im.h, im.l, or the IEEE
            // doubles in the last block) into s_out at their tile indices,
            // at rotated columns (the store warp copies whole runs out)
            auto amp4 = [&](const df &re, const df &im) {
                if (OUT_IEEE) {
                    const double x = df_to_double(re), y = df_to_double(im);
                    return make_float4(__uint_as_float(__double2loint(x)), __uint_as_float(__double2hiint(x)),
                                       __uint_as_float(__double2loint(y)), __uint_as_float(__double2hiint(y)));
                }
                return make_float4(re.h, re.l, im.h, im.l);
            };
            df o0[8], o1[8];
            drain(0);
            drain(1);
            tmem_st_wait();
            if (next) arrive_ready();  // tile i + 1's digits written, tile i's accumulators read
            combine(0, o0);
            combine(1, o1);
            {
                float4 w[8];
#pragma unroll
                for (int jj = 0; jj < 4; jj++) {
                    w[jj] = amp4(o0[2 * jj], o0[2 * jj + 1]);
                    w[4 + jj] = amp4(o1[2 * jj], o1[2 * jj + 1]);
                }
                if (rotated) unrot(w);
                const uint32_t cb = coff(0) | colbits((int)rot);
#pragma unroll
                for (int j = 0; j < 8; j++) sts128(so + 16u * (cb ^ colbits(j)), w[j]);
            }
            fence_proxy_async_smem();  // the outputs are visible to the bulk stores
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_out);
            return true;
        };
        // steady state, the MMAs of tile i in flight and tile i + 1 split in
        // registers: as soon as K step qq of tile i's MMAs is done, the warps
        // of K quarter qq put tile i + 1's digits into its A slices; once all
        // MMAs are done, tile i's accumulators are read out and tile i + 1's
        // MMAs may start; tile i is combined and stored, and tile i + 2
        // fetched and split, while they run.  (The loop always ends with a
        // split and always starts with a put, so the digit words are not
        // held across the combination; a split without a fetch splits zeros.)
        uint32_t i = 0;
        for (; i + 1 < count && !aborted; i++) {
            const bool bad = !__all_sync(0xffffffffu, mbar_wait_bounded(&bar_mks[qq], i & 1u, kWaitBudget128));
            tc_fence_after();
            put();
            if (!finish(i, true, bad)) {
                aborted = true;
                break;
            }
            Ecur = Enext;
            if (i + 2 < count) {
                if (!fetch(i + 2)) {
                    aborted = true;
                    break;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; j++) v[j] = make_uint4(0u, 0u, 0u, 0u);
            }
            split();
            Enext = Eg_next;
        }
        if (!aborted && count > 0 && !finish(count - 1, false, false)) aborted = true;
        if (aborted && tid == 0) atomicExch(err, kErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

// Host: the six B slices of a fused 5-qubit gate in the canonical layout.
// U: 32 x 32 complex, row-major (re, im) FP64.  out: kBBytes / 2 bf16 bit
// patterns.  Returns false when an entry is outside (-2, 2) or a row's level
// sums could leave the exact FP32 range (never for a unitary U): the caller
// then takes another path.
bool fused_tc128_prepare_b(const double *U, uint16_t *out) {
    std::memset(out, 0, kBBytes);
    double rowsum[kReals][kDigits];
    for (int n = 0; n < kReals; n++)
        for (int j = 0; j < kDigits; j++) rowsum[n][j] = 0.0;
    double unit[kDigits];  // 2^(7 + 9 j): slice j's digit times this is the integer c_j (exact)
    for (int j = 0; j < kDigits; j++) unit[j] = std::ldexp(1.0, 7 + kDigitBits * j);
    for (int r = 0; r < kAmps; r++)
        for (int c = 0; c < kAmps; c++) {
            const double ur = U[2 * (r * kAmps + c)], ui = U[2 * (r * kAmps + c) + 1];
            const double v[4] = {ur, -ui, ui, ur};
            const int nn[4] = {2 * r, 2 * r, 2 * r + 1, 2 * r + 1};
            const int kk[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
            for (int e = 0; e < 4; e++) {
                if (!(std::fabs(v[e]) < 2.0)) return false;
                float d[kDigits];
                dg_split_entry(v[e], d);
                for (int j = 0; j < kDigits; j++) {
                    out[(j * kSliceBytes + bcanon_off((uint32_t)nn[e], (uint32_t)kk[e])) / 2] = (uint16_t)dg_bf16(d[j]);
                    rowsum[nn[e]][j] += std::fabs((double)d[j] * unit[j]);  // |c_j|
                }
            }
        }
    // level L <= 3 sums at most 256 * sum_{j <= L} ||c_j||_1 (|d_i| <= 256)
    for (int n = 0; n < kReals; n++) {
        double s = 0.0;
        for (int j = 0; j < kDigitLevels - 1; j++) {
            s += rowsum[n][j];
            if (256.0 * s >= 16777216.0) return false;
        }
    }
    return true;
}

size_t fused_tc128_b_bytes() { return kBBytes; }

bool fused_tc128_supported(int k, int n) { return k == kK && n >= kTileBits; }

template <bool IN_IEEE, bool OUT_IEEE>
static cudaError_t launch_tc128(void *amp, const TileGeom &g, const FusedMap &fm, const uint16_t *bmat, uint32_t *err,
                                int sm_count, cudaStream_t s) {
    const size_t smem = kBBytes + 2 * (size_t)kTileBytes;
    cudaError_t e = cudaFuncSetAttribute(k_fused_tc_c128<IN_IEEE, OUT_IEEE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t ntiles = 1ull << (g.n - kTileBits);
    uint64_t grid = ntiles < (uint64_t)sm_count ? ntiles : (uint64_t)sm_count;
    k_fused_tc_c128<IN_IEEE, OUT_IEEE>
        <<<(unsigned)grid, kThreadsAll128, smem, s>>>(static_cast<double2 *>(amp), g, fm, bmat, err, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_fused_tc128(void *amp, const TileGeom &g, const FusedMap &fm, const uint16_t *bmat,
                               uint32_t *err, int sm_count, cudaStream_t s, bool in_ieee, bool out_ieee) {
    if (g.L + g.H != kTileBits || g.H > kMaxH128 || g.L < 1) return cudaErrorInvalidValue;
    if (in_ieee && out_ieee) return launch_tc128<true, true>(amp, g, fm, bmat, err, sm_count, s);
    if (in_ieee) return launch_tc128<true, false>(amp, g, fm, bmat, err, sm_count, s);
    if (out_ieee) return launch_tc128<false, true>(amp, g, fm, bmat, err, sm_count, s);
    return launch_tc128<false, false>(amp, g, fm, bmat, err, sm_count, s);
}

}  // namespace qsim
