// k_tile2.cu -- register-blocked tile passes.
//
// Same pass structure as k_tile.cu (a tile of 2^T amplitudes = the L low
// index bits plus H chosen high bits, fetched and written back with bulk
// asynchronous copies), but the gate program runs in registers:
//
//   local bit 0..4          lane bits: a gate on them pairs amplitudes held by
//                           lanes l and l ^ 2^t of one warp (warp shuffles)
//   RB of the bits >= 5     register bits: a gate on them pairs two registers
//                           of one thread
//   the other bits >= 5     warp bits (kRegWarpBits of them: 2^kRegWarpBits warps)
//
// The program is cut into phases; a phase loads the tile from shared memory
// into registers under its own choice of register bits, applies its gates,
// and stores back (optionally to permuted positions, which is how quantum SWAP
// gates and qubit interchanges are applied).  T = 5 + RB + kRegWarpBits.
//
// complex64 computes in FP32.  complex128 computes in double-float (FP32
// pairs, df64.cuh): the tile arrives as IEEE doubles, the first phase converts
// them with integer operations, later phases keep the double-float form in
// shared memory, and the last phase converts back.  The per-phase engine is
// in tile2_engine.cuh (shared with the batch kernel).
#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"
#include "ptx.cuh"
#include "tile2_engine.cuh"

namespace qsim {

namespace {

constexpr int kThreads2 = 32 << kRegWarpBits;
constexpr int kMaxH2 = 10;
constexpr int kMaxCopyShift2 = 14;
constexpr long long kWaitBudget2 = 4000000000ll;

#ifndef QSIM_T2_MINB
#define QSIM_T2_MINB (QSIM_T2_NWB == 4 ? 2 : 3)
#endif
constexpr int kMinBlocks2 = QSIM_T2_MINB;  // resident CTAs per SM the register budget is sized for

template <bool C128, int RB>
__global__ void __launch_bounds__(kThreads2, kMinBlocks2)
    k_tile2(typename t2::AmpT<C128>::S *__restrict__ a, TileGeom g, const TilePhase *__restrict__ phases_g, int nphases,
            const TileOp *__restrict__ ops_g, int op_base, int op_count, uint32_t *err, uint64_t ntiles) {
    using S = typename t2::AmpT<C128>::S;
    using V = typename t2::AmpT<C128>::V;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *t = reinterpret_cast<S *>(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint64_t runoff[1 << kMaxH2];
    __shared__ int abort_flag;
    const int L = g.L, H = g.H, T = L + H;
    const uint32_t TS = 1u << T;
    const uint32_t nruns = 1u << H;
    const int amp_shift = sizeof(S) == 8 ? 3 : 4;
    const int sub_L = L + amp_shift > kMaxCopyShift2 ? kMaxCopyShift2 - amp_shift : L;
    const int sub_shift = L - sub_L;
    const uint32_t ncopies = nruns << sub_shift;
    const uint32_t copy_bytes = 1u << (sub_L + amp_shift);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the pass's ops and phases, read by every thread for every tile: copied
    // to shared memory after the tile (the planner keeps a pass within
    // kRegMaxOps / kRegMaxPhases), so the op reads of the gate program are
    // shared-memory loads; phases index the ops from op_base
    TileOp *ops_s = reinterpret_cast<TileOp *>(smem_raw + (sizeof(S) << T));
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(ops_g + op_base);
        uint32_t *dst = reinterpret_cast<uint32_t *>(ops_s);
        for (uint32_t w = threadIdx.x; w < (uint32_t)op_count * (sizeof(TileOp) / 4); w += blockDim.x) dst[w] = src[w];
    }
    const TileOp *ops = ops_s - op_base;
    TilePhase *phases = reinterpret_cast<TilePhase *>(smem_raw + (sizeof(S) << T) + (size_t)op_count * sizeof(TileOp));
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(phases_g);
        uint32_t *dst = reinterpret_cast<uint32_t *>(phases);
        for (uint32_t w = threadIdx.x; w < (uint32_t)nphases * (sizeof(TilePhase) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __shared__ int s_hb[kMaxH2];  // the high tile bits, indexed at run time
    if (threadIdx.x < kMaxH2) s_hb[threadIdx.x] = threadIdx.x < (unsigned)H ? g.hb[threadIdx.x] : 0;

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
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, TS * (uint32_t)sizeof(S));
            __syncwarp();
            for (uint32_t c = threadIdx.x; c < ncopies; c += 32) {
                const uint32_t j = c >> sub_shift, s = c & ((1u << sub_shift) - 1u);
                bulk_g2s(t + ((size_t)j << L) + ((size_t)s << sub_L), a + (base | runoff[j]) + ((size_t)s << sub_L),
                         copy_bytes, &bar);
            }
        }
        if (!mbar_wait_bounded(&bar, parity, kWaitBudget2)) {
            atomicExch(err, kErrTimeout);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            mbar_wait_bounded(&bar, parity, kWaitBudget2);
            return;
        }
        parity ^= 1u;

        for (int p = 0; p < nphases; p++) {
            const int lfmt = (C128 && p == 0) ? 0 : 1, sfmt = (C128 && p == nphases - 1) ? 0 : 1;
            t2::run_phase<C128, RB>(t, phases[p], ops, base, lane, warp, lfmt, sfmt);
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

template <bool C128, int RB>
cudaError_t launch2(void *amp, const TileGeom &g, const TilePhase *phases, int nphases, const TileOp *ops,
                    int op_base, int op_count, uint32_t *err, int sm_count, cudaStream_t s) {
    using S = typename t2::AmpT<C128>::S;
    const int T = g.L + g.H;
    if (op_count > kRegMaxOps || nphases > kRegMaxPhases) return cudaErrorInvalidValue;
    const size_t smem = (sizeof(S) << T) + (size_t)op_count * sizeof(TileOp) + (size_t)nphases * sizeof(TilePhase);
    const uint64_t ntiles = 1ull << (g.n - T);
    int per_sm = (int)((220u * 1024u) / (smem + 9u * 1024u));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > kMinBlocks2) per_sm = kMinBlocks2;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    cudaError_t e = cudaFuncSetAttribute(k_tile2<C128, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile2<C128, RB><<<(unsigned)grid, kThreads2, smem, s>>>(static_cast<S *>(amp), g, phases, nphases, ops,
                                                               op_base, op_count, err, ntiles);
    return cudaGetLastError();
}

}  // namespace

bool tile2_supported(int dt, int T) { return dt == 0 && (T == 12 || T == 13); }

cudaError_t launch_tile_pass2(void *amp, int dt, const TileGeom &g, const TilePhase *phases, int nphases,
                              const TileOp *ops, int op_base, int op_count, uint32_t *err, int sm_count,
                              cudaStream_t s) {
    const int T = g.L + g.H;
    if (!tile2_supported(dt, T) || g.L < 5 || g.H > kMaxH2 || T > g.n) return cudaErrorInvalidValue;
    constexpr int RB12 = 12 - 5 - kRegWarpBits, RB13 = 13 - 5 - kRegWarpBits;
    if (T == 13) return launch2<false, RB13>(amp, g, phases, nphases, ops, op_base, op_count, err, sm_count, s);
    return launch2<false, RB12>(amp, g, phases, nphases, ops, op_base, op_count, err, sm_count, s);
}

}  // namespace qsim
