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
#include "tile_ops.cuh"

namespace qsim {

namespace {

constexpr int kTileThreads = 256;
constexpr int kMaxH = 10;                  // at most 1024 runs per tile
constexpr int kMaxCopyShift = 14;          // bulk copies of at most 16 KiB
constexpr long long kWaitBudget = 4000000000ll;  // SM cycles (about 2 s) before a wait gives up

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
            tile_apply_op<R>(t, T, ops[o], base, dmat);
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

static size_t tile_smem_bytes(int dt, int T) { return (size_t)(dt == 0 ? 8 : 16) << T; }

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
