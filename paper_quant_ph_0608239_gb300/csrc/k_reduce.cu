// k_reduce.cu -- read-only sweeps: norm (Eq. STAT1), per-bit marginals
// <Q_q> (Eq. Shor7, the DO MEASUREMENT of App. A), probabilities |a_i|^2 and
// amplitudes in logical order, and basis-state sampling (Sec. V.B).
//
// Accumulation is FP64.  For complex64 states the squares of up to 16
// amplitudes are summed in FP32 before they enter an FP64 accumulator (the
// FP32 partial sums of non-negative terms carry at most 16 ulp of relative
// error, far below the precision of the amplitudes themselves); complex128
// states are summed in FP64.  The per-bit marginals for n >= 13 of either
// precision run their inner sums in double-float (k_bits_partial_df).
//
// The partial sums of each block go to a caller-provided scratch buffer in
// global memory and a second kernel adds them up.

#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"

namespace qsim {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;
constexpr int kChunkBits = 9;  // 32 lanes x 16 amplitudes per warp chunk

template <typename R>
__device__ __forceinline__ R sq(amp_t<R> v) { return v.x * v.x + v.y * v.y; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum v over the block; result valid in thread 0.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_norm_partial(const amp_t<R> *__restrict__ a, uint64_t D,
                                                              double *__restrict__ partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 7 * stride < D; i += 8 * stride) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) s += sq<R>(a[i + k * stride]);
        acc += (double)s;
    }
    for (; i < D; i += stride) acc += (double)sq<R>(a[i]);
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// out[j] = sum over blocks b of partial[b * stride + j], j < count
__global__ void k_sum_columns(const double *__restrict__ partial, int nblocks, int count, int stride,
                              double *__restrict__ out) {
    __shared__ double sh[32];
    for (int j = 0; j < count; j++) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += partial[(size_t)b * stride + j];
        const double r = block_sum(acc, sh);
        if (threadIdx.x == 0) out[j] = r;
    }
}

// Per-bit marginals P(bit b = 1), b < n, n >= kChunkBits.  A warp works on
// chunks of 512 consecutive amplitudes; lane l holds amplitudes l + 32 k,
// k < 16, so bits 0..4 of every amplitude a lane sees equal l, bits 5..8 equal
// k (known at compile time) and the higher bits are those of the chunk.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_bits_partial(const amp_t<R> *__restrict__ a, int n,
                                                              double *__restrict__ partial) {
    __shared__ double sh[32];
    double acc[kMaxQubits];
#pragma unroll
    for (int b = 0; b < kMaxQubits; b++) acc[b] = 0.0;
    double lane_tot = 0.0;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t nch = 1ull << (n - kChunkBits);
    for (uint64_t ch = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < nch; ch += warps) {
        const amp_t<R> *p = a + (ch << kChunkBits) + lane;
        R v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = sq<R>(p[32 * k]);
        R tot = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            tot += v[k];
            if (k & 1) m0 += v[k];
            if (k & 2) m1 += v[k];
            if (k & 4) m2 += v[k];
            if (k & 8) m3 += v[k];
        }
        const double t = (double)tot;
        lane_tot += t;
        acc[5] += (double)m0;
        acc[6] += (double)m1;
        acc[7] += (double)m2;
        acc[8] += (double)m3;
#pragma unroll
        for (int b = kChunkBits; b < kMaxQubits; b++)
            if (b < n && ((ch >> (b - kChunkBits)) & 1ull)) acc[b] += t;
    }
#pragma unroll
    for (int b = 0; b < 5; b++) acc[b] = ((lane >> b) & 1) ? lane_tot : 0.0;
#pragma unroll
    for (int b = 0; b < kMaxQubits; b++) {
        if (b < n) {  // uniform across the block
            const double r = block_sum(acc[b], sh);
            if (threadIdx.x == 0) partial[(size_t)blockIdx.x * n + b] = r;
        }
    }
}

// Per-bit marginals, n >= kGroupBits, with no FP64 in the inner loop (GB300
// issues FP64 at about 2 instructions per clock per SM, fewer than reading
// the state at full bandwidth needs).  A warp takes groups of 8192
// consecutive amplitudes: lane l holds amplitudes l + 32 j, j < 256, read in
// chunks of 8 (j = 8 c + k), so bits 0..4 of an index are the lane, bits 5..7
// are k, bits 8..12 are the chunk c and the higher bits are the group's.
// Each |a|^2 of a complex128 state is a double-float from the IEEE bits
// (df_sqmag, relative error below 2^-44; a chunk holding a magnitude >= 2
// takes the FP64 branch); of a complex64 state it is an FP32 square, and a
// chunk's 8 squares are summed in FP32.  Per group and lane the sums run in
// double-float over at most 32 terms: per k (bits 5..7), per set bit of c
// (bits 8..12, from the chunk sums) and the group total.  At the end of the
// group they are added to FP64 accumulators; the group total, summed over the
// warp, is added by lane b - 13 to bit b's accumulator when bit b of the
// group index is set.
constexpr int kGroupBits = 13;

__device__ __forceinline__ double df_sum_d(df x) { return (double)x.h + (double)x.l; }  // exact

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_bits_partial_df(const amp_t<R> *__restrict__ a, int n,
                                                                  double *__restrict__ partial) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    double A[8], B[5], L = 0.0, H = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) A[k] = 0.0;
#pragma unroll
    for (int i = 0; i < 5; i++) B[i] = 0.0;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t ngroups = 1ull << (n - kGroupBits);
    for (uint64_t gi = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < ngroups; gi += warps) {
        const amp_t<R> *p = a + (gi << kGroupBits) + lane;
        df ak[8], bc[5], tg{0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < 8; k++) ak[k] = df{0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 5; i++) bc[i] = df{0.0f, 0.0f};
#pragma unroll 2
        for (int c = 0; c < 32; c++) {
            amp_t<R> v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = p[32 * (8 * c + k)];
            df q[8];
            if constexpr (sizeof(R) == 4) {
                // complex64: the square in FP32 (the precision of the state)
#pragma unroll
                for (int k = 0; k < 8; k++) q[k] = df{fmaf(v[k].x, v[k].x, v[k].y * v[k].y), 0.0f};
            } else {
                uint32_t any = 0;
#pragma unroll
                for (int k = 0; k < 8; k++)
                    any |= (uint32_t)(df_bits64(v[k].x) >> 32) | (uint32_t)(df_bits64(v[k].y) >> 32);
                if (__any_sync(0xffffffffu, (any & 0x40000000u) != 0u)) {
                    // a magnitude >= 2 in the chunk: the squares in FP64
#pragma unroll
                    for (int k = 0; k < 8; k++) q[k] = df_from_double(fma(v[k].x, v[k].x, v[k].y * v[k].y));
                } else {
#pragma unroll
                    for (int k = 0; k < 8; k++) q[k] = df_sqmag(v[k].x, v[k].y);
                }
            }
#pragma unroll
            for (int k = 0; k < 8; k++) ak[k] = df_add_pos(ak[k], q[k]);
            df cs;
            if constexpr (sizeof(R) == 4) {  // complex64: the chunk's 8 squares summed in FP32
                cs = df{((q[0].h + q[1].h) + (q[2].h + q[3].h)) + ((q[4].h + q[5].h) + (q[6].h + q[7].h)), 0.0f};
            } else {
                cs = df_add_pos(df_add_pos(df_add_pos(q[0], q[1]), df_add_pos(q[2], q[3])),
                                df_add_pos(df_add_pos(q[4], q[5]), df_add_pos(q[6], q[7])));
            }
            tg = df_add_pos(tg, cs);
#pragma unroll
            for (int i = 0; i < 5; i++)
                if ((c >> i) & 1) bc[i] = df_add_pos(bc[i], cs);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) A[k] += df_sum_d(ak[k]);
#pragma unroll
        for (int i = 0; i < 5; i++) B[i] += df_sum_d(bc[i]);
        const double t = df_sum_d(tg);
        L += t;
        const double G = warp_sum(t);
        if (lane < n - kGroupBits && ((gi >> lane) & 1ull)) H += G;
    }
    for (int b = 0; b < n; b++) {  // uniform across the block
        double v;
        if (b < 5) {
            v = ((lane >> b) & 1) ? L : 0.0;
        } else if (b < 8) {
            v = 0.0;
#pragma unroll
            for (int k = 0; k < 8; k++)
                if ((k >> (b - 5)) & 1) v += A[k];
        } else if (b < kGroupBits) {
            v = 0.0;
#pragma unroll
            for (int i = 0; i < 5; i++)
                if (i == b - 8) v = B[i];
        } else {
            v = lane == b - kGroupBits ? H : 0.0;
        }
        const double r = block_sum(v, sh);
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * n + b] = r;
    }
}

// Small states: one amplitude per thread iteration.
template <typename R>
__global__ void k_bits_small(const amp_t<R> *__restrict__ a, int n, double *__restrict__ out) {
    __shared__ double sh[32];
    const uint64_t D = 1ull << n;
    for (int b = 0; b < n; b++) {
        double acc = 0.0;
        for (uint64_t i = threadIdx.x; i < D; i += blockDim.x)
            if ((i >> b) & 1ull) acc += (double)sq<R>(a[i]);
        const double r = block_sum(acc, sh);
        if (threadIdx.x == 0) out[b] = r;
    }
}

struct PhysPos {
    int8_t p[kMaxQubits];
};

__device__ __forceinline__ uint64_t phys_of(uint64_t x, const PhysPos &pp, int n) {
    uint64_t r = 0;
    for (int q = 0; q < n; q++) r |= ((x >> q) & 1ull) << pp.p[q];
    return r;
}

template <typename R>
__global__ void k_probs_chunk(const amp_t<R> *__restrict__ a, int n, PhysPos pp, bool ident, uint64_t start,
                              uint64_t count, double *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
        const uint64_t x = start + j;
        const amp_t<R> v = a[ident ? x : phys_of(x, pp, n)];
        out[j] = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
}

template <typename R>
__global__ void k_gather_chunk(const amp_t<R> *__restrict__ a, int n, PhysPos pp, uint64_t start, uint64_t count,
                               amp_t<R> *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride)
        out[j] = a[phys_of(start + j, pp, n)];
}

// ---- sampling ------------------------------------------------------------
constexpr int kSampleBlockBits = 12;

// bsum[b] = sum of |a_x|^2 over logical x in [b 2^S, (b+1) 2^S), FP64.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_block_sums(const amp_t<R> *__restrict__ a, int n, PhysPos pp,
                                                            bool ident, int S, double *__restrict__ bsum,
                                                            uint64_t nb) {
    __shared__ double sh[32];
    for (uint64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        double acc = 0.0;
        for (uint64_t j = threadIdx.x; j < (1ull << S); j += blockDim.x) {
            const uint64_t x = (b << S) + j;
            const amp_t<R> v = a[ident ? x : phys_of(x, pp, n)];
            acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        const double r = block_sum(acc, sh);
        if (threadIdx.x == 0) bsum[b] = r;
        __syncthreads();
    }
}

// In-place inclusive prefix sum of nb values by one block (sequential over
// segments of blockDim.x values).
__global__ void k_prefix(double *__restrict__ v, uint64_t nb) {
    __shared__ double sh[1024];
    __shared__ double carry;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    for (uint64_t s0 = 0; s0 < nb; s0 += blockDim.x) {
        const uint64_t i = s0 + threadIdx.x;
        sh[threadIdx.x] = i < nb ? v[i] : 0.0;
        __syncthreads();
        for (unsigned o = 1; o < blockDim.x; o <<= 1) {
            double t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0.0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) v[i] = sh[threadIdx.x] + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[blockDim.x - 1];
        __syncthreads();
    }
}

// One warp per sample: find the block by binary search over the inclusive
// prefix sums, then the index inside the block by a warp scan.
template <typename R>
__global__ void k_draw(const amp_t<R> *__restrict__ a, int n, PhysPos pp, bool ident, int S,
                       const double *__restrict__ cum, uint64_t nb, const double *__restrict__ u, uint64_t ns,
                       uint64_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const double total = cum[nb - 1];
    const uint64_t D = 1ull << n;
    for (uint64_t s = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < ns; s += warps) {
        const double target = u[s] * total;
        // smallest b with target < cum[b]
        uint64_t lo = 0, hi = nb;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (target < cum[mid]) hi = mid;
            else lo = mid + 1;
        }
        if (lo >= nb) {  // rounding put the target past the total: last state with weight
            if (lane == 0) out[s] = D - 1;
            continue;
        }
        double before = lo ? cum[lo - 1] : 0.0;
        // values per lane; blocks of fewer than 32 values (registers of fewer
        // than 5 qubits) give one value to each of the first 2^S lanes
        const uint64_t blk = 1ull << S;
        const uint64_t per = blk >= 32 ? blk / 32 : 1;
        const int nlanes = blk >= 32 ? 32 : (int)blk;
        const bool active = lane < nlanes;
        const uint64_t x0 = (lo << S) + (uint64_t)lane * per;
        double mine = 0.0;
        for (uint64_t j = 0; active && j < per; j++) {
            const amp_t<R> v = a[ident ? (x0 + j) : phys_of(x0 + j, pp, n)];
            mine += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        // inclusive scan of lane sums
        double incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, active && target < before + incl);
        int owner = ball ? __ffs(ball) - 1 : nlanes - 1;
        double c = before + __shfl_sync(0xffffffffu, incl - mine, owner);
        if (lane == owner) {
            uint64_t pick = x0 + per - 1;
            for (uint64_t j = 0; j < per; j++) {
                const amp_t<R> v = a[ident ? (x0 + j) : phys_of(x0 + j, pp, n)];
                c += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
                if (target < c) {
                    pick = x0 + j;
                    break;
                }
            }
            out[s] = pick;
        }
    }
}

PhysPos to_pp(const int *physpos, int n) {
    PhysPos pp{};
    for (int q = 0; q < n; q++) pp.p[q] = (int8_t)physpos[q];
    return pp;
}

}  // namespace

size_t reduce_scratch_bytes(int n) { return (size_t)kRedBlocks * (size_t)(n + 1) * sizeof(double) + 64; }

cudaError_t launch_norm(const void *amp, int dt, int n, double *scratch, double *dout, cudaStream_t s) {
    const uint64_t D = 1ull << n;
    if (dt == 0)
        k_norm_partial<float><<<kRedBlocks, kRedThreads, 0, s>>>(static_cast<const float2 *>(amp), D, scratch);
    else
        k_norm_partial<double><<<kRedBlocks, kRedThreads, 0, s>>>(static_cast<const double2 *>(amp), D, scratch);
    k_sum_columns<<<1, 256, 0, s>>>(scratch, kRedBlocks, 1, 1, dout);
    return cudaGetLastError();
}

cudaError_t launch_bit_probs(const void *amp, int dt, int n, double *scratch, double *dout, cudaStream_t s) {
    if (n < kChunkBits + 1) {
        if (dt == 0)
            k_bits_small<float><<<1, 256, 0, s>>>(static_cast<const float2 *>(amp), n, dout);
        else
            k_bits_small<double><<<1, 256, 0, s>>>(static_cast<const double2 *>(amp), n, dout);
        return cudaGetLastError();
    }
    if (n >= kGroupBits) {
        uint64_t blocks = ((1ull << (n - kGroupBits)) + 7) / 8;
        if (blocks > (uint64_t)kRedBlocks) blocks = kRedBlocks;
        if (dt == 0)
            k_bits_partial_df<float><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const float2 *>(amp), n,
                                                                         scratch);
        else
            k_bits_partial_df<double><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const double2 *>(amp), n,
                                                                          scratch);
        k_sum_columns<<<1, 256, 0, s>>>(scratch, (int)blocks, n, n, dout);
        return cudaGetLastError();
    }
    uint64_t nch = 1ull << (n - kChunkBits);
    uint64_t blocks = (nch + 7) / 8;
    if (blocks > (uint64_t)kRedBlocks) blocks = kRedBlocks;
    if (dt == 0)
        k_bits_partial<float><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const float2 *>(amp), n, scratch);
    else
        k_bits_partial<double><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const double2 *>(amp), n, scratch);
    k_sum_columns<<<1, 256, 0, s>>>(scratch, (int)blocks, n, n, dout);
    return cudaGetLastError();
}

cudaError_t launch_probs_chunk(const void *amp, int dt, int n, const int *physpos, bool identity, uint64_t start,
                               uint64_t count, double *dout, cudaStream_t s) {
    const PhysPos pp = to_pp(physpos, n);
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    if (blocks < 1) blocks = 1;
    if (dt == 0)
        k_probs_chunk<float><<<(int)blocks, 256, 0, s>>>(static_cast<const float2 *>(amp), n, pp, identity, start,
                                                          count, dout);
    else
        k_probs_chunk<double><<<(int)blocks, 256, 0, s>>>(static_cast<const double2 *>(amp), n, pp, identity,
                                                           start, count, dout);
    return cudaGetLastError();
}

cudaError_t launch_gather_chunk(const void *amp, int dt, int n, const int *physpos, uint64_t start, uint64_t count,
                                void *dout, cudaStream_t s) {
    const PhysPos pp = to_pp(physpos, n);
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    if (blocks < 1) blocks = 1;
    if (dt == 0)
        k_gather_chunk<float><<<(int)blocks, 256, 0, s>>>(static_cast<const float2 *>(amp), n, pp, start, count,
                                                           static_cast<float2 *>(dout));
    else
        k_gather_chunk<double><<<(int)blocks, 256, 0, s>>>(static_cast<const double2 *>(amp), n, pp, start, count,
                                                            static_cast<double2 *>(dout));
    return cudaGetLastError();
}

size_t sample_scratch_bytes(int n) {
    const uint64_t nb = n > kSampleBlockBits ? (1ull << (n - kSampleBlockBits)) : 1ull;
    return (size_t)nb * sizeof(double) + 64;
}

cudaError_t launch_sample(const void *amp, int dt, int n, const int *physpos, bool identity, const double *du,
                          size_t ns, uint64_t *dout, double *scratch, cudaStream_t s) {
    // blocks of 2^S values
    const int S = n >= kSampleBlockBits ? kSampleBlockBits : n;
    const uint64_t nb = 1ull << (n - S);
    const PhysPos pp = to_pp(physpos, n);
    uint64_t g = nb < 152ull * 8 ? nb : 152ull * 8;
    if (dt == 0)
        k_block_sums<float><<<(int)g, kRedThreads, 0, s>>>(static_cast<const float2 *>(amp), n, pp, identity, S,
                                                            scratch, nb);
    else
        k_block_sums<double><<<(int)g, kRedThreads, 0, s>>>(static_cast<const double2 *>(amp), n, pp, identity, S,
                                                             scratch, nb);
    k_prefix<<<1, 1024, 0, s>>>(scratch, nb);
    uint64_t dg = (ns + 7) / 8;
    if (dg > 152ull * 8) dg = 152ull * 8;
    if (dg < 1) dg = 1;
    if (dt == 0)
        k_draw<float><<<(int)dg, 256, 0, s>>>(static_cast<const float2 *>(amp), n, pp, identity, S, scratch, nb, du,
                                               ns, dout);
    else
        k_draw<double><<<(int)dg, 256, 0, s>>>(static_cast<const double2 *>(amp), n, pp, identity, S, scratch, nb,
                                                du, ns, dout);
    return cudaGetLastError();
}

}  // namespace qsim

// ---- allocation-free per-qubit marginals ----------------------------------
// Some callers may not allocate device memory at all: code running while a
// framework owns the whole device through its own memory pool, latency-bound
// measurement loops that cannot absorb the implicit device synchronisation of
// cudaMalloc/cudaFree, and embedders that forbid allocation after start-up.
// For them the per-qubit marginal reduction can run on a fixed scratch array
// that the library places in device memory when it is loaded.  Every GPU that
// loads the library keeps this array until the process exits.
namespace qsim {

namespace {

constexpr int kNoAllocBlocks = kRedBlocks;                    // 608 blocks
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocBlocks * kMaxQubits;  // 161.5 KiB

// Block partials of the last call: [block][bit], kNoAllocBlocks x n used.
static __device__ __align__(256) double g_noalloc_partial[kNoAllocDoubles];

}  // namespace


cudaError_t launch_bit_probs_noalloc(const void *amp, int dt, int n, double *dout, cudaStream_t s) {
    // The array's name is not a device address in host code: look the address
    // up on every call, with the caller's device current.  The lookup is a
    // host-side query, and doing it each time keeps the address right after a
    // context was torn down and the module loaded again (cudaDeviceReset).
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    double *scratch = static_cast<double *>(p);
    if (n < kChunkBits + 1) {  // small registers reduce in one block, no scratch
        if (dt == 0)
            k_bits_small<float><<<1, 256, 0, s>>>(static_cast<const float2 *>(amp), n, dout);
        else
            k_bits_small<double><<<1, 256, 0, s>>>(static_cast<const double2 *>(amp), n, dout);
        return cudaGetLastError();
    }
    // Every partial the second kernel reads is written first by this call's
    // first kernel (each block writes all n of its slots), so nothing left by
    // an earlier call is read and no clearing is needed.
    const uint64_t nch = 1ull << (n - kChunkBits);
    uint64_t blocks = (nch + 7) / 8;
    if (blocks > (uint64_t)kNoAllocBlocks) blocks = kNoAllocBlocks;
    if (dt == 0)
        k_bits_partial<float><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const float2 *>(amp), n, scratch);
    else
        k_bits_partial<double><<<(int)blocks, kRedThreads, 0, s>>>(static_cast<const double2 *>(amp), n, scratch);
    k_sum_columns<<<1, 256, 0, s>>>(scratch, (int)blocks, n, n, dout);
    return cudaGetLastError();
}

}  // namespace qsim
