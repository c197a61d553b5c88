// k_permute.cu -- the qubit interchange of Sec. III.B as one pass over HBM.
//
// Exchanging the index bits l_i <-> h_i (i < K) moves the amplitude at index
// x to pi(x), pi swapping each pair of bits (Eq. onequbitchange and
// Eqs. twoqubitchange0-5 for K = 1, 2; any K here).  pi is an involution, so
// after the pass the amplitude at u is the one that was at pi(u).
//
// A tile holds every index bit the pairs touch: the L low bits as runs of
// 2^L contiguous amplitudes and the H high bits (the pairs' bits above L,
// padded with further bits up to the tile size) selecting the run.  pi maps
// the tile onto itself.  A CTA fetches a tile into shared memory with bulk
// asynchronous copies (the next tile's copies in flight meanwhile), then
// every thread takes output indices u (consecutive across a warp), reads the
// element at pi(u) from shared memory and stores it to u's place in global
// memory: coalesced stores, and consecutive lanes that read from different
// runs hit different banks because each run's shared-memory copy is shifted
// by 16 bytes.
#include "common.cuh"
#include "kernels.hpp"
#include "ptx.cuh"

namespace qsim {

namespace {

constexpr int kPermThreads = 256;
constexpr int kPermMaxH = 10;
constexpr uint32_t kPermTileBytes = 32768;  // per buffer (plus 16 bytes per run)
constexpr long long kPermWait = 4000000000ll;

template <typename E>
__global__ void __launch_bounds__(kPermThreads)
    k_permute(E *__restrict__ a, TileGeom g, PermPairs pp, uint32_t *err, uint64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint64_t runoff[1 << kPermMaxH];
    __shared__ int s_hb[kPermMaxH];
    __shared__ int abort_flag;
    const int L = g.L, H = g.H, T = L + H;
    const uint32_t nruns = 1u << H, run_elems = 1u << L;
    const uint32_t run_stride = run_elems * (uint32_t)sizeof(E) + 16u;  // bytes between runs in shared memory
    const uint32_t buf_bytes = run_stride * nruns;
    const uint32_t TS = 1u << T;
    if (threadIdx.x < (unsigned)kPermMaxH) s_hb[threadIdx.x] = threadIdx.x < (unsigned)H ? g.hb[threadIdx.x] : 0;
    for (uint32_t j = threadIdx.x; j < nruns; j += blockDim.x) {
        uint64_t o = 0;
        for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << g.hb[k];
        runoff[j] = o;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    auto tile_base = [&](uint64_t tile) {
        uint64_t base = tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, s_hb[k]);
        return base;
    };
    auto issue = [&](uint64_t tile, int b) {  // warp 0
        const uint64_t base = tile_base(tile);
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar[b], TS * (uint32_t)sizeof(E));
        __syncwarp();
        unsigned char *dst = smem_raw + (size_t)b * buf_bytes;
        for (uint32_t j = threadIdx.x; j < nruns; j += 32)
            bulk_g2s(dst + (size_t)j * run_stride, a + (base | runoff[j]), run_elems * (uint32_t)sizeof(E), &bar[b]);
    };
    const uint64_t stride = gridDim.x;
    // every thread tracks the parity of each buffer's next completion and
    // whether a copy into it is outstanding (issued by warp 0, waited by all)
    uint32_t phase0 = 0u, phase1 = 0u;  // (kept in registers: no runtime-indexed arrays)
    bool pending0 = false, pending1 = false;
    uint64_t tile = blockIdx.x;
    if (tile < ntiles) {
        if (threadIdx.x < 32) issue(tile, 0);
        pending0 = true;
    }
    for (int it = 0; tile < ntiles; tile += stride, it++) {
        const int b = it & 1;
        if (tile + stride < ntiles) {
            if (threadIdx.x < 32) issue(tile + stride, b ^ 1);
            if (b) pending0 = true; else pending1 = true;
        }
        if (!mbar_wait_bounded(&bar[b], b ? phase1 : phase0, kPermWait)) atomicExch(&abort_flag, 1);
        __syncthreads();
        if (abort_flag) {
            if (threadIdx.x == 0) atomicExch(err, kErrTimeout);
            break;
        }
        if (b) phase1 ^= 1u, pending1 = false;
        else phase0 ^= 1u, pending0 = false;
        const unsigned char *src = smem_raw + (size_t)b * buf_bytes;
        const uint64_t base = tile_base(tile);
        for (uint32_t u = threadIdx.x; u < TS; u += blockDim.x) {
            uint32_t v = u;  // pi(u): the pairs' bits exchanged
#pragma unroll
            for (int i = 0; i < kMaxPermPairs; i++)
                if (i < pp.K) {
                    const uint32_t t = ((v >> pp.lo[i]) ^ (v >> pp.hi[i])) & 1u;
                    v ^= (t << pp.lo[i]) | (t << pp.hi[i]);
                }
            const E x = *reinterpret_cast<const E *>(src + (size_t)(v >> L) * run_stride + (size_t)(v & (run_elems - 1u)) * sizeof(E));
            a[base | runoff[u >> L] | (u & (run_elems - 1u))] = x;
        }
        __syncthreads();  // the buffer is read before its next copy is issued
    }
    // copies still in flight (only after an abort) land before the CTA leaves
    if (threadIdx.x == 0) {
        if (pending0) mbar_wait_bounded(&bar[0], phase0, kPermWait);
        if (pending1) mbar_wait_bounded(&bar[1], phase1, kPermWait);
    }
}

}  // namespace

// Tile size of the interchange pass for elements of elem_bytes (8 or 16).
int permute_tile_bits(int elem_bytes) { return elem_bytes == 8 ? 12 : 11; }

cudaError_t launch_permute(void *amp, int elem_bytes, const TileGeom &g, const PermPairs &pp, uint32_t *err,
                           int sm_count, cudaStream_t s) {
    const int T = g.L + g.H;
    if (g.H > kPermMaxH || g.L < 1 || pp.K < 1 || pp.K > kMaxPermPairs) return cudaErrorInvalidValue;
    if (((size_t)elem_bytes << T) > kPermTileBytes) return cudaErrorInvalidValue;
    const size_t smem = 2 * (((size_t)elem_bytes << g.L) + 16) * ((size_t)1 << g.H);
    const uint64_t ntiles = 1ull << (g.n - T);
    uint64_t grid = (uint64_t)sm_count * 3;
    if (grid > ntiles) grid = ntiles;
    if (elem_bytes == 8) {
        cudaError_t e = cudaFuncSetAttribute(k_permute<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_permute<float2><<<(unsigned)grid, kPermThreads, smem, s>>>(static_cast<float2 *>(amp), g, pp, err, ntiles);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_permute<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_permute<double2><<<(unsigned)grid, kPermThreads, smem, s>>>(static_cast<double2 *>(amp), g, pp, err, ntiles);
    }
    return cudaGetLastError();
}

}  // namespace qsim
