// k_phase.cu -- a run of commuting phase shifts (Eqs. NUM5 and COMM5: the
// controlled phases of the QFT adders of Sec. V.A) as one pass over the
// state, complex64 (k_phase) and complex128 (k_phase128, in IEEE or in the
// double-float form of the tensor-core blocks).
//
// The phase of amplitude x is a sum of table entries, one table per chunk
// pair (a, b) of the index bits (planner.hpp, PhasePass), in fixed-point
// turns summed mod 2^32 (complex64) or 2^64 (complex128).  A warp takes rows
// of 1024 amplitudes: chunk 0 (bits 0..4) is the lane, chunk 1 (bits 5..9)
// the step j of its loop, the higher chunks are fixed for the row.  So the tables of two high chunks are read
// once per row, those of chunk 0 with a high chunk once per row and lane, and
// per amplitude only the tables of chunk 1 (the same word for the whole warp)
// and the table of chunks 0 and 1 (consecutive words across the warp): no
// bank conflicts.  The phase becomes e^(i 2 pi turns) (complex64 through
// sincospif) and multiplies the amplitude in place: one read and one write of
// the state.
#include <cmath>

#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"

namespace qsim {

namespace {

constexpr int kPhThreads = 256;
constexpr int kPhMaxUni = 8;  // tables of chunk 1 with chunk 1..7

__global__ void __launch_bounds__(kPhThreads)
    k_phase(float2 *__restrict__ a, uint64_t nrows, const uint32_t *__restrict__ tab, PhaseMeta m) {
    extern __shared__ uint32_t s_tab[];  // m.ntab tables of kPhaseTableWords
    __shared__ int8_t s_ta[kMaxPhaseTables], s_tb[kMaxPhaseTables];
    const uint32_t nw = (uint32_t)m.ntab * kPhaseTableWords;
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) s_tab[w] = tab[w];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < kMaxPhaseTables; t++) {
            s_ta[t] = m.ta[t];
            s_tb[t] = m.tb[t];
        }
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (kPhThreads / 32);
    for (uint64_t row = (uint64_t)blockIdx.x * (kPhThreads / 32) + (threadIdx.x >> 5); row < nrows; row += warps) {
        const uint64_t hi = row << (2 * kPhaseChunk);
        auto chunk = [&](int c) { return (uint32_t)(hi >> (kPhaseChunk * c)) & 31u; };
        // per row and lane: the tables without chunk 1; per step j: the
        // offsets (row part) of the tables with chunk 1
        uint32_t base = 0, nuni = 0, lan = 0xffffffffu;
        uint32_t uoff[kPhMaxUni];
#pragma unroll
        for (int u = 0; u < kPhMaxUni; u++) uoff[u] = 0u;
        for (int t = 0; t < m.ntab; t++) {
            const int ca = s_ta[t], cb = s_tb[t];
            const uint32_t tb0 = (uint32_t)t * kPhaseTableWords;
            if (ca == 1 || (ca == 0 && cb == 1)) {
                if (ca == 0) {
                    lan = tb0;  // table of chunks 0 and 1: index lane + 32 j
                } else {
                    // chunk 1 with chunk cb >= 1: index j + 32 x_cb (j alone for cb = 1)
                    const uint32_t o = tb0 + (cb == 1 ? 0u : 32u * chunk(cb));
#pragma unroll
                    for (int u = 0; u < kPhMaxUni; u++)
                        if ((uint32_t)u == nuni) uoff[u] = o;
                    nuni++;
                }
            } else if (ca == 0) {
                base += s_tab[tb0 + lane + (cb == 0 ? 0u : 32u * chunk(cb))];
            } else {
                base += s_tab[tb0 + chunk(ca) + (ca == cb ? 0u : 32u * chunk(cb))];
            }
        }
        float2 *ar = a + hi + lane;
#pragma unroll 4
        for (uint32_t j = 0; j < 32u; j++) {
            uint32_t ph = base;
#pragma unroll
            for (int u = 0; u < kPhMaxUni; u++)
                if ((uint32_t)u < nuni) ph += s_tab[uoff[u] + j];
            if (lan != 0xffffffffu) ph += s_tab[lan + lane + 32u * j];
            // 2 pi turns = pi (turns as a signed 32-bit fraction of 2^31)
            float s, c;
            sincospif((float)(int32_t)ph * 4.656612873077393e-10f, &s, &c);
            const float2 v = ar[32u * j];
            ar[32u * j] = make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
        }
    }
}

// complex128: 64-bit turns; the factor e^(2 pi i t) from a table of the
// 1024 multiples of 2 pi / 1024 (double-float, computed at the start from
// FP64 sincospi) times e^(i delta) for the remaining delta < 2 pi / 1024 as a
// short Taylor series in double-float (terms past delta^7 below 1e-22); the
// amplitude is multiplied in double-float.  When no table pairs chunk 0 with
// chunk 1, the phase of amplitude (row, j, lane) is F(row, lane) + G(row, j):
// each lane then builds the two factors e^(2 pi i F) and e^(2 pi i G) with
// j = lane once per row, and each amplitude takes F times G (from lane j) --
// two complex products per amplitude instead of a factor of its own.  The
// state is read and written as IEEE doubles (IN_IEEE, OUT_IEEE: the first or
// last step of a plan) or in the double-float form of the tensor-core blocks.
constexpr int kPhE = 1024;

struct TurnsConst {
    df K;      // 2 pi / 2^64
    df SIXTH;  // 1/6
};

// e^(2 pi i ph / 2^64), ph = k 2^54 + r: table entry k times e^(i delta),
// delta = r 2 pi / 2^64 < 2 pi / 1024
__device__ __forceinline__ dcx turns_factor(uint64_t ph, const float4 *s_e, const TurnsConst &tc) {
    const uint32_t k = (uint32_t)(ph >> 54);
    const uint64_t r = ph & ((1ull << 54) - 1ull);
    const df rr = quick_two_sum(ldexpf((float)(uint32_t)(r >> 30), 30), (float)(uint32_t)(r & 0x3fffffffu));
    const df d = df_mul(rr, tc.K);
    const df d2 = df_mul(d, d);
    const float f2 = d2.h;
    df cv = df_add(df{1.0f, 0.0f}, df{-0.5f * d2.h, -0.5f * d2.l});
    cv = df_add(cv, df{f2 * f2 * (1.0f / 24.0f) - f2 * f2 * f2 * (1.0f / 720.0f), 0.0f});
    const df d3 = df_mul(d2, d);
    df sv = df_add(d, df_neg(df_mul(d3, tc.SIXTH)));
    sv = df_add(sv, df{d3.h * f2 * (1.0f / 120.0f) - d3.h * f2 * f2 * (1.0f / 5040.0f), 0.0f});
    const float4 e4 = s_e[k];
    return dcx_mul(dcx{df{e4.x, e4.y}, df{e4.z, e4.w}}, dcx{cv, sv});
}

template <bool IN_IEEE>
__device__ __forceinline__ dcx ld_amp128(const double2 *p) {
    if (IN_IEEE) {
        const double2 v = *p;
        return dcx{df_from_double(v.x), df_from_double(v.y)};
    }
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return dcx{df{v.x, v.y}, df{v.z, v.w}};
}

template <bool OUT_IEEE>
__device__ __forceinline__ void st_amp128(double2 *p, const dcx &w) {
    if (OUT_IEEE)
        *p = make_double2(df_to_double(w.re), df_to_double(w.im));
    else
        *reinterpret_cast<float4 *>(p) = make_float4(w.re.h, w.re.l, w.im.h, w.im.l);
}

template <bool IN_IEEE, bool OUT_IEEE>
__global__ void __launch_bounds__(kPhThreads)
    k_phase128(double2 *__restrict__ a, uint64_t nrows, const uint64_t *__restrict__ tab, PhaseMeta m) {
    extern __shared__ __align__(16) unsigned char smem128[];
    uint64_t *s_tab = reinterpret_cast<uint64_t *>(smem128);
    float4 *s_e = reinterpret_cast<float4 *>(smem128 + (size_t)m.ntab * kPhaseTableWords * sizeof(uint64_t));
    __shared__ int8_t s_ta[kMaxPhaseTables], s_tb[kMaxPhaseTables];
    const uint32_t nw = (uint32_t)m.ntab * kPhaseTableWords;
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) s_tab[w] = tab[w];
    for (int e = threadIdx.x; e < kPhE; e += blockDim.x) {
        double sn, cs;
        sincospi((double)e / (kPhE / 2), &sn, &cs);
        const df c = df_from_double_rn(cs), sv = df_from_double_rn(sn);
        s_e[e] = make_float4(c.h, c.l, sv.h, sv.l);
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < kMaxPhaseTables; t++) {
            s_ta[t] = m.ta[t];
            s_tb[t] = m.tb[t];
        }
    }
    __syncthreads();
    // 2 pi / 2^64 and 1/6 as double-floats
    const double twopi = 6.283185307179586476925286766559;
    const float kph = (float)twopi;
    const float s6h = 1.0f / 6.0f;
    const TurnsConst tc{df{ldexpf(kph, -64), ldexpf((float)(twopi - (double)kph), -64)},
                        df{s6h, (float)(1.0 / 6.0 - (double)s6h)}};
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (kPhThreads / 32);
    for (uint64_t row = (uint64_t)blockIdx.x * (kPhThreads / 32) + (threadIdx.x >> 5); row < nrows; row += warps) {
        const uint64_t hi = row << (2 * kPhaseChunk);
        auto chunk = [&](int c) { return (uint32_t)(hi >> (kPhaseChunk * c)) & 31u; };
        uint64_t base = 0;
        uint32_t nuni = 0, lan = 0xffffffffu;
        uint32_t uoff[kPhMaxUni];
#pragma unroll
        for (int u = 0; u < kPhMaxUni; u++) uoff[u] = 0u;
        for (int t = 0; t < m.ntab; t++) {
            const int ca = s_ta[t], cb = s_tb[t];
            const uint32_t tb0 = (uint32_t)t * kPhaseTableWords;
            if (ca == 1 || (ca == 0 && cb == 1)) {
                if (ca == 0) {
                    lan = tb0;
                } else {
                    const uint32_t o = tb0 + (cb == 1 ? 0u : 32u * chunk(cb));
#pragma unroll
                    for (int u = 0; u < kPhMaxUni; u++)
                        if ((uint32_t)u == nuni) uoff[u] = o;
                    nuni++;
                }
            } else if (ca == 0) {
                base += s_tab[tb0 + lane + (cb == 0 ? 0u : 32u * chunk(cb))];
            } else {
                base += s_tab[tb0 + chunk(ca) + (ca == cb ? 0u : 32u * chunk(cb))];
            }
        }
        double2 *ar = a + hi + lane;
        if (lan == 0xffffffffu) {
            // separable: F for this lane, G for j = lane
            uint64_t phj = 0;
#pragma unroll
            for (int u = 0; u < kPhMaxUni; u++)
                if ((uint32_t)u < nuni) phj += s_tab[uoff[u] + lane];
            const dcx F = turns_factor(base, s_e, tc);
            const dcx Gl = turns_factor(phj, s_e, tc);
            // eight amplitudes in flight per lane
#pragma unroll 1
            for (uint32_t j0 = 0; j0 < 32u; j0 += 8u) {
                dcx v[8];
#pragma unroll
                for (uint32_t jj = 0; jj < 8u; jj++) v[jj] = ld_amp128<IN_IEEE>(ar + 32u * (j0 + jj));
#pragma unroll
                for (uint32_t jj = 0; jj < 8u; jj++) {
                    const uint32_t j = j0 + jj;
                    const dcx G{df{__shfl_sync(0xffffffffu, Gl.re.h, j), __shfl_sync(0xffffffffu, Gl.re.l, j)},
                                df{__shfl_sync(0xffffffffu, Gl.im.h, j), __shfl_sync(0xffffffffu, Gl.im.l, j)}};
                    st_amp128<OUT_IEEE>(ar + 32u * j, dcx_mul(dcx_mul(F, G), v[jj]));
                }
            }
        } else {
#pragma unroll 1
            for (uint32_t j0 = 0; j0 < 32u; j0 += 4u) {
                dcx v[4];
#pragma unroll
                for (uint32_t jj = 0; jj < 4u; jj++) v[jj] = ld_amp128<IN_IEEE>(ar + 32u * (j0 + jj));
#pragma unroll
                for (uint32_t jj = 0; jj < 4u; jj++) {
                    const uint32_t j = j0 + jj;
                    uint64_t ph = base;
#pragma unroll
                    for (int u = 0; u < kPhMaxUni; u++)
                        if ((uint32_t)u < nuni) ph += s_tab[uoff[u] + j];
                    ph += s_tab[lan + lane + 32u * j];
                    st_amp128<OUT_IEEE>(ar + 32u * j, dcx_mul(turns_factor(ph, s_e, tc), v[jj]));
                }
            }
        }
    }
}

template <bool IN_IEEE, bool OUT_IEEE>
cudaError_t launch_k_phase128(void *amp, uint64_t nrows, const uint64_t *tables, const PhaseMeta &m, size_t smem,
                              int sm_count, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_phase128<IN_IEEE, OUT_IEEE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase128<IN_IEEE, OUT_IEEE>, kPhThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t need = (nrows + kPhThreads / 32 - 1) / (kPhThreads / 32);
    if (grid > need) grid = need;
    k_phase128<IN_IEEE, OUT_IEEE>
        <<<(unsigned)grid, kPhThreads, smem, s>>>(static_cast<double2 *>(amp), nrows, tables, m);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_phase_pass128(void *amp, int n, const uint64_t *tables, const PhaseMeta &m, int sm_count,
                                 cudaStream_t s, bool in_ieee, bool out_ieee) {
    if (n < 2 * kPhaseChunk || m.ntab < 1 || m.ntab > 24) return cudaErrorInvalidValue;
    int nuni = 0;
    for (int t = 0; t < m.ntab; t++) {
        if (m.ta[t] > m.tb[t] || (int)m.tb[t] * kPhaseChunk >= n) return cudaErrorInvalidValue;
        if (m.ta[t] == 1) nuni++;
    }
    if (nuni > kPhMaxUni) return cudaErrorInvalidValue;
    const size_t smem = (size_t)m.ntab * kPhaseTableWords * sizeof(uint64_t) + kPhE * sizeof(float4);
    const uint64_t nrows = 1ull << (n - 2 * kPhaseChunk);
    if (in_ieee && out_ieee) return launch_k_phase128<true, true>(amp, nrows, tables, m, smem, sm_count, s);
    if (in_ieee) return launch_k_phase128<true, false>(amp, nrows, tables, m, smem, sm_count, s);
    if (out_ieee) return launch_k_phase128<false, true>(amp, nrows, tables, m, smem, sm_count, s);
    return launch_k_phase128<false, false>(amp, nrows, tables, m, smem, sm_count, s);
}

cudaError_t launch_phase_pass(void *amp, int n, const uint32_t *tables, const PhaseMeta &m, int sm_count,
                              cudaStream_t s) {
    if (n < 2 * kPhaseChunk || m.ntab < 1 || m.ntab > kMaxPhaseTables) return cudaErrorInvalidValue;
    int nuni = 0;
    for (int t = 0; t < m.ntab; t++) {
        if (m.ta[t] > m.tb[t] || (int)m.tb[t] * kPhaseChunk >= n) return cudaErrorInvalidValue;
        if (m.ta[t] == 1) nuni++;
    }
    if (nuni > kPhMaxUni) return cudaErrorInvalidValue;
    const size_t smem = (size_t)m.ntab * kPhaseTableWords * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase, kPhThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t nrows = 1ull << (n - 2 * kPhaseChunk);
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t need = (nrows + kPhThreads / 32 - 1) / (kPhThreads / 32);
    if (grid > need) grid = need;
    k_phase<<<(unsigned)grid, kPhThreads, smem, s>>>(static_cast<float2 *>(amp), nrows, tables, m);
    return cudaGetLastError();
}

}  // namespace qsim
