// k_batch.cu -- many independent circuits in one persistent launch.
//
// Every circuit of the batch is planned into tile passes (k_tile.cu's op
// programs, complex64).  The host lists the work as items (circuit, pass,
// tile), ordered by pass, then circuit, then tile.  The CTAs of one
// cooperative launch take items in that order from an atomic counter.  An item
// of pass p > 0 waits until every tile of pass p - 1 of its circuit is done
// (per-pass counters, acquire loads, bounded spin); since an item only waits
// for items earlier in the order, and those are held by running CTAs, the
// scheme cannot deadlock.  A circuit of at most 12 qubits is one tile: it runs
// entirely in one CTA's shared memory, from a basis state generated there, and
// touches global memory once, to store its result.
//
// A pass with register phases (12-bit tiles) runs the register-blocked
// program of tile2_engine.cuh on the tile; other passes run the shared-memory
// program of tile_ops.cuh.
//
// A wait that exceeds its budget sets an error word and the kernel returns;
// the host reports QSIM_ETIMEOUT.
#include "common.cuh"
#include "kernels.hpp"
#include "tile2_engine.cuh"
#include "tile_ops.cuh"

namespace qsim {

namespace {

constexpr int kThreadsB = 256;
constexpr int kMaxHB = 10;
constexpr int kMaxTB = 12;                            // tiles of at most 2^12 amplitudes
constexpr int kLoadIt = (1 << kMaxTB) / kThreadsB;    // amplitudes a thread loads per tile
constexpr int kStageOpsB = kRegMaxOps;                // ops of one pass staged in shared memory (12 KiB)
constexpr int kStagePhB = kRegMaxPhases;              // phases of one pass staged (1.4 KiB)

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

static_assert(kThreadsB == (32 << kRegWarpBits), "the register program's block shape");

__global__ void __launch_bounds__(kThreadsB, 3) k_batch(const BatchCircuit *__restrict__ circs,
                                                     const BatchPass *__restrict__ passes,
                                                     const TileOp *__restrict__ ops,
                                                     const TilePhase *__restrict__ phases,
                                                     const BatchItem *__restrict__ items, uint64_t nitems,
                                                     uint32_t *counters, uint32_t *done, uint32_t *err,
                                                     long long budget) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *t = reinterpret_cast<float2 *>(smem_raw);
    __shared__ uint64_t runoff[1 << kMaxHB];
    __shared__ __align__(16) TileOp s_ops[kStageOpsB];
    __shared__ TilePhase s_ph[kStagePhB];
    __shared__ uint64_t sh_item;
    __shared__ int sh_abort;
    // The pass whose run offsets, ops and phases are in shared memory: items
    // of one pass follow one another, so a block mostly reuses them.  Every
    // thread tracks the same value.
    uint32_t staged_pass = 0xffffffffu;
    for (;;) {
        if (threadIdx.x == 0) {
            sh_item = atomicAdd(reinterpret_cast<unsigned long long *>(counters), 1ull);
            sh_abort = 0;
        }
        __syncthreads();
        const uint64_t it = sh_item;
        if (it >= nitems) break;
        const BatchItem item = items[it];
        const BatchCircuit &c = circs[item.circuit];
        const BatchPass &ps = passes[c.pass_begin + item.pass];
        if (threadIdx.x == 0 && item.pass > 0) {
            // every tile of the previous pass of this circuit must be done
            const uint32_t *flag = done + c.pass_begin + item.pass - 1;
            const uint32_t need = (uint32_t)ps.ntiles;
            if (ld_acquire(flag) < need) {
                const long long t0 = clock64();
                while (ld_acquire(flag) < need) {
                    if (clock64() - t0 > budget) {
                        atomicExch(err, kErrTimeout);
                        sh_abort = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __syncthreads();
        if (sh_abort) return;
        const TileGeom &g = ps.geom;
        const int L = g.L, H = g.H, T = L + H;
        const uint32_t TS = 1u << T, lowmask = (1u << L) - 1u;
        const uint32_t pass_id = (uint32_t)(c.pass_begin + item.pass);
        // (the host checked that every pass fits the staged copies)
        if (pass_id != staged_pass) {
            // (the previous item ended with a barrier: nobody reads the old copies)
            for (uint32_t j = threadIdx.x; j < (1u << H); j += blockDim.x) {
                uint64_t o = 0;
                for (int k = 0; k < H; k++) o |= (uint64_t)((j >> k) & 1u) << g.hb[k];
                runoff[j] = o;
            }
            {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(ops + ps.op_begin);
                uint32_t *dst = reinterpret_cast<uint32_t *>(s_ops);
                for (uint32_t w = threadIdx.x; w < (uint32_t)ps.op_count * (sizeof(TileOp) / 4); w += blockDim.x)
                    dst[w] = src[w];
            }
            {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(phases + ps.phase_begin);
                uint32_t *dst = reinterpret_cast<uint32_t *>(s_ph);
                for (uint32_t w = threadIdx.x; w < (uint32_t)ps.phase_count * (sizeof(TilePhase) / 4); w += blockDim.x)
                    dst[w] = src[w];
            }
            staged_pass = pass_id;
        }
        // ops indexed by their position in the batch's op array (shared-memory copies only)
        const TileOp *ops_p = s_ops - ps.op_begin;
        uint64_t base = (uint64_t)item.tile << L;
        for (int k = 0; k < H; k++) base = insert_zero(base, g.hb[k]);
        __syncthreads();
        float2 *a = reinterpret_cast<float2 *>(c.amp);
        if (item.pass == 0) {  // the circuit's initial basis state, generated in place
            for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) {
                const uint64_t gi = base | runoff[i >> L] | (i & lowmask);
                t[i] = make_float2(gi == c.x0 ? 1.0f : 0.0f, 0.0f);
            }
        } else {  // written by other CTAs: read through L2, four loads of a thread in flight at once
            for (int k0 = 0; k0 < kLoadIt; k0 += 4) {
                float2 buf[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t i = threadIdx.x + (uint32_t)(k0 + k) * kThreadsB;
                    if (i < TS) buf[k] = __ldcg(a + (base | runoff[i >> L] | (i & lowmask)));
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t i = threadIdx.x + (uint32_t)(k0 + k) * kThreadsB;
                    if (i < TS) t[i] = buf[k];
                }
            }
        }
        __syncthreads();
        if (ps.phase_count > 0) {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int p = 0; p < ps.phase_count; p++)
                t2::run_phase<false, kBatchRB>(t, s_ph[p], ops_p, base, lane, warp, 1, 1);
        } else {
            for (int o = ps.op_begin; o < ps.op_begin + ps.op_count; o++) {
                tile_apply_op<float>(t, T, ops_p[o], base, nullptr);
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) a[base | runoff[i >> L] | (i & lowmask)] = t[i];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + c.pass_begin + item.pass, 1u);
    }
}

}  // namespace

static size_t batch_smem_bytes() { return (size_t)8 << kMaxTB; }

cudaError_t launch_batch(const BatchCircuit *circs, const BatchPass *passes, const TileOp *ops,
                         const TilePhase *phases, const BatchItem *items, uint64_t nitems, uint32_t *counters,
                         uint32_t *done, uint32_t *err, long long budget, int sm_count, cudaStream_t s) {
    const size_t smem = batch_smem_bytes();
    // the staged programs sit in static shared memory, so the tile needs the
    // opt-in beyond the default 48 KiB per block
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreadsB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned grid = (unsigned)(sm_count * per_sm);
    if ((uint64_t)grid > nitems) grid = (unsigned)(nitems ? nitems : 1);
    void *args[] = {(void *)&circs, (void *)&passes, (void *)&ops, (void *)&phases, (void *)&items,
                    (void *)&nitems, (void *)&counters, (void *)&done, (void *)&err, (void *)&budget};
    // cooperative: every CTA resident at once, so a waiting CTA never blocks
    // the one it waits for from being scheduled
    return cudaLaunchCooperativeKernel((const void *)k_batch, dim3(grid), dim3(kThreadsB), args, smem, s);
}

}  // namespace qsim
