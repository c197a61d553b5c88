// k_gates.cu -- per-gate sweeps over the whole state (the one-gate-per-sweep
// execution of Sec. III.A, Eqs. NUM2-NUM8) and the basis-state initialiser.
//
// A gate touches either pairs (a0, a1) of amplitudes whose indices differ in
// the target bit, or single amplitudes (diagonal gates).  The host inserts the
// fixed bits (target = 0, controls = 1) into a compact enumeration index, so a
// kernel visits exactly the amplitudes the gate changes: 2^(n-1-c) pairs for a
// c-controlled gate (Eqs. NUM6, NUM8), 2^(n-1-c) single amplitudes for a phase
// shift (Eq. NUM5).  Consecutive threads get consecutive enumeration indices,
// so both members of the pair are read with coalesced accesses for every
// target bit; the low target bits fall inside one 32-byte sector and are
// merged by L1.
#include <cmath>

#include "common.cuh"
#include "df64.cuh"
#include "kernels.hpp"

namespace qsim {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

inline FixedBits to_dev(const FixedBitsHost &h) {
    FixedBits f;
    f.npos = h.npos;
    for (int i = 0; i < kMaxFixed; i++) f.pos[i] = i < h.npos ? h.pos[i] : 0;
    f.setmask = h.setmask;
    return f;
}

inline int grid_for(uint64_t work, int per_thread) {
    uint64_t b = (work + (uint64_t)kThreads * per_thread - 1) / ((uint64_t)kThreads * per_thread);
    const uint64_t cap = 152ull * 32ull;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename R, int GC>
__device__ __forceinline__ void pair_update(amp_t<R> &x, amp_t<R> &y, const amp_t<R> (&u)[4]) {
    if (GC == GC_GENERAL) {
        amp_t<R> a = cmul2<R>(u[0], x, u[1], y);
        amp_t<R> b = cmul2<R>(u[2], x, u[3], y);
        x = a;
        y = b;
    } else if (GC == GC_REAL) {
        amp_t<R> a = mk<R>(fma(u[0].x, x.x, u[1].x * y.x), fma(u[0].x, x.y, u[1].x * y.y));
        amp_t<R> b = mk<R>(fma(u[2].x, x.x, u[3].x * y.x), fma(u[2].x, x.y, u[3].x * y.y));
        x = a;
        y = b;
    } else if (GC == GC_ANTIDIAG) {
        amp_t<R> a = cmul<R>(u[1], y);
        amp_t<R> b = cmul<R>(u[2], x);
        x = a;
        y = b;
    } else {  // GC_EXCHANGE
        amp_t<R> t = x;
        x = y;
        y = t;
    }
}

template <typename R, int GC, int NP>
__global__ void __launch_bounds__(kThreads) k_pairs(amp_t<R> *__restrict__ a, uint64_t W, FixedBits fb,
                                                    uint64_t pmask, Mat2 M) {
    amp_t<R> u[4];
#pragma unroll
    for (int k = 0; k < 4; k++) u[k] = mk<R>((R)M.u[2 * k], (R)M.u[2 * k + 1]);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    uint64_t p = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; p + (kUnroll - 1) * stride < W; p += kUnroll * stride) {
        uint64_t i0[kUnroll];
        amp_t<R> x[kUnroll], y[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; k++) {
            i0[k] = expand_n<NP>(p + k * stride, fb);
            x[k] = a[i0[k]];
            y[k] = a[i0[k] ^ pmask];
        }
#pragma unroll
        for (int k = 0; k < kUnroll; k++) {
            pair_update<R, GC>(x[k], y[k], u);
            a[i0[k]] = x[k];
            a[i0[k] ^ pmask] = y[k];
        }
    }
    for (; p < W; p += stride) {
        const uint64_t i = expand_n<NP>(p, fb);
        amp_t<R> x = a[i], y = a[i ^ pmask];
        pair_update<R, GC>(x, y, u);
        a[i] = x;
        a[i ^ pmask] = y;
    }
}

template <typename R, int NP>
__global__ void __launch_bounds__(kThreads) k_diag(amp_t<R> *__restrict__ a, uint64_t W, FixedBits fb, int tbit,
                                                   Mat2 M) {
    const amp_t<R> u0 = mk<R>((R)M.u[0], (R)M.u[1]);
    const amp_t<R> u1 = mk<R>((R)M.u[6], (R)M.u[7]);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    uint64_t p = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; p + (kUnroll - 1) * stride < W; p += kUnroll * stride) {
        uint64_t i[kUnroll];
        amp_t<R> x[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; k++) {
            i[k] = expand_n<NP>(p + k * stride, fb);
            x[k] = a[i[k]];
        }
#pragma unroll
        for (int k = 0; k < kUnroll; k++) a[i[k]] = cmul<R>(((i[k] >> tbit) & 1) ? u1 : u0, x[k]);
    }
    for (; p < W; p += stride) {
        const uint64_t i = expand_n<NP>(p, fb);
        a[i] = cmul<R>(((i >> tbit) & 1) ? u1 : u0, a[i]);
    }
}

// ---- complex128 sweeps in double-float arithmetic ---------------------------
// GB300 runs FP64 at about 1/58 of its FP32 rate, which makes an FP64 dense
// 2x2 sweep arithmetic-bound at well under the memory bandwidth.  The
// amplitudes stay IEEE double in memory; each sweep converts them to
// double-float with integer operations (df64.cuh), applies the gate on the
// FP32 pipes and converts back.  Pure exchanges never get here: they move
// bytes and stay bit-exact.
struct DfMat {
    float h[8], l[8];
};

__device__ __forceinline__ dcx df_coef(const DfMat &M, int k) {
    return dcx{df{M.h[2 * k], M.l[2 * k]}, df{M.h[2 * k + 1], M.l[2 * k + 1]}};
}
__device__ __forceinline__ dcx to_dcx(double2 v) { return dcx{df_from_double(v.x), df_from_double(v.y)}; }
__device__ __forceinline__ double2 from_dcx(const dcx &v) {
    return make_double2(df_to_double(v.re), df_to_double(v.im));
}

template <int GC, int NP>
__global__ void __launch_bounds__(kThreads) k_pairs_df(double2 *__restrict__ a, uint64_t W, FixedBits fb,
                                                       uint64_t pmask, DfMat M) {
    const dcx u0 = df_coef(M, 0), u1 = df_coef(M, 1), u2 = df_coef(M, 2), u3 = df_coef(M, 3);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t p = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p < W; p += 2 * stride) {
        const bool two = p + stride < W;
        const uint64_t i = expand_n<NP>(p, fb), j = two ? expand_n<NP>(p + stride, fb) : i;
        const double2 ra = a[i], rb = a[i ^ pmask], rc = a[j], rd = a[j ^ pmask];
        const dcx x0 = to_dcx(ra), y0 = to_dcx(rb), x1 = to_dcx(rc), y1 = to_dcx(rd);
        dcx o0, o1, o2, o3;
        if (GC == GC_GENERAL) {
            o0 = dcx_mul2(u0, x0, u1, y0);
            o1 = dcx_mul2(u2, x0, u3, y0);
            o2 = dcx_mul2(u0, x1, u1, y1);
            o3 = dcx_mul2(u2, x1, u3, y1);
        } else if (GC == GC_REAL) {
            o0 = dcx_rmul2(u0.re, x0, u1.re, y0);
            o1 = dcx_rmul2(u2.re, x0, u3.re, y0);
            o2 = dcx_rmul2(u0.re, x1, u1.re, y1);
            o3 = dcx_rmul2(u2.re, x1, u3.re, y1);
        } else {  // anti-diagonal
            o0 = dcx_mul(u1, y0);
            o1 = dcx_mul(u2, x0);
            o2 = dcx_mul(u1, y1);
            o3 = dcx_mul(u2, x1);
        }
        a[i] = from_dcx(o0);
        a[i ^ pmask] = from_dcx(o1);
        if (two) {
            a[j] = from_dcx(o2);
            a[j ^ pmask] = from_dcx(o3);
        }
    }
}

template <int NP>
__global__ void __launch_bounds__(kThreads) k_diag_df(double2 *__restrict__ a, uint64_t W, FixedBits fb, int tbit,
                                                      DfMat M) {
    const dcx u0 = df_coef(M, 0), u3 = df_coef(M, 3);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t p = (uint64_t)blockIdx.x * kThreads + threadIdx.x; p < W; p += 2 * stride) {
        const bool two = p + stride < W;
        const uint64_t i = expand_n<NP>(p, fb), j = two ? expand_n<NP>(p + stride, fb) : i;
        const double2 ra = a[i], rc = a[j];
        const dcx x0 = dcx_mul(((i >> tbit) & 1) ? u3 : u0, to_dcx(ra));
        const dcx x1 = dcx_mul(((j >> tbit) & 1) ? u3 : u0, to_dcx(rc));
        a[i] = from_dcx(x0);
        if (two) a[j] = from_dcx(x1);
    }
}

DfMat to_dfmat(const Mat2 &U) {
    DfMat d;
    for (int k = 0; k < 8; k++) {
        d.h[k] = (float)U.u[k];
        d.l[k] = (float)(U.u[k] - (double)d.h[k]);
    }
    return d;
}

template <int NP>
cudaError_t pairs_df_np(void *amp, uint64_t W, const FixedBits &fb, uint64_t pmask, int gc, const Mat2 &U,
                        cudaStream_t s) {
    const int grid = grid_for(W, 2);
    double2 *a = static_cast<double2 *>(amp);
    const DfMat M = to_dfmat(U);
    switch (gc) {
    case GC_GENERAL: k_pairs_df<GC_GENERAL, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, M); break;
    case GC_REAL: k_pairs_df<GC_REAL, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, M); break;
    case GC_ANTIDIAG: k_pairs_df<GC_ANTIDIAG, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, M); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t pairs_df(void *amp, uint64_t W, const FixedBits &fb, uint64_t pmask, int gc, const Mat2 &U,
                     cudaStream_t s) {
    if (fb.npos <= 2) return pairs_df_np<2>(amp, W, fb, pmask, gc, U, s);
    if (fb.npos <= 4) return pairs_df_np<4>(amp, W, fb, pmask, gc, U, s);
    if (fb.npos <= 8) return pairs_df_np<8>(amp, W, fb, pmask, gc, U, s);
    return pairs_df_np<kMaxFixed>(amp, W, fb, pmask, gc, U, s);
}

cudaError_t diag_df(void *amp, uint64_t W, const FixedBits &fb, int tbit, const Mat2 &U, cudaStream_t s) {
    const int grid = grid_for(W, 2);
    double2 *a = static_cast<double2 *>(amp);
    const DfMat M = to_dfmat(U);
    if (fb.npos <= 2) k_diag_df<2><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, M);
    else if (fb.npos <= 4) k_diag_df<4><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, M);
    else if (fb.npos <= 8) k_diag_df<8><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, M);
    else k_diag_df<kMaxFixed><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, M);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_init_basis(amp_t<R> *__restrict__ a, uint64_t D, uint64_t x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += stride)
        a[i] = mk<R>(i == x ? (R)1 : (R)0, (R)0);
}

// Eq. Shor2: a_{x + 2^X f(x)} = amp for x < 2^X, f(x) = y^x mod G (square and
// multiply; G < 2^32, so every product fits in 64 bits).  The other
// amplitudes are zeroed by the caller.
template <class R>
__global__ void k_shor_state(amp_t<R> *__restrict__ a, int X, uint64_t y, uint64_t G, R amp) {
    const uint64_t D = 1ull << X;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += stride) {
        uint64_t f = 1 % G, b = y % G, e = x;
        while (e) {
            if (e & 1ull) f = (f * b) % G;
            b = (b * b) % G;
            e >>= 1;
        }
        a[x | (f << X)] = mk<R>(amp, (R)0);
    }
}

struct Qpos {
    int p[8];
};

// Dense 2^k x 2^k gate on CUDA cores: one thread per group of 2^k amplitudes.
// The matrix is staged in shared memory; groups are enumerated by inserting
// zeros at the k (sorted) positions, so consecutive threads read consecutive
// addresses whenever the low bits are free.
template <typename R, int K>
__global__ void __launch_bounds__(128) k_dense(amp_t<R> *__restrict__ a, uint64_t W, FixedBits fb, Qpos q,
                                               const amp_t<R> *__restrict__ U) {
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    amp_t<R> *sU = reinterpret_cast<amp_t<R> *>(smem_raw);
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) sU[e] = U[e];
    __syncthreads();
    uint64_t off[D];
#pragma unroll
    for (int c = 0; c < D; c++) {
        uint64_t o = 0;
#pragma unroll
        for (int j = 0; j < K; j++)
            if ((c >> j) & 1) o |= 1ull << q.p[j];
        off[c] = o;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < W; g += stride) {
        const uint64_t base = expand(g, fb);
        amp_t<R> v[D];
#pragma unroll
        for (int c = 0; c < D; c++) v[c] = a[base | off[c]];
#pragma unroll 1
        for (int r = 0; r < D; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                const amp_t<R> u = sU[r * D + c];
                re = fma(u.x, v[c].x, re);
                re = fma(-u.y, v[c].y, re);
                im = fma(u.x, v[c].y, im);
                im = fma(u.y, v[c].x, im);
            }
            a[base | off[r]] = mk<R>(re, im);
        }
    }
}

template <typename R, int K>
cudaError_t dense_k(void *amp, uint64_t W, const FixedBits &fb, const Qpos &q, const void *dU, cudaStream_t s) {
    const size_t smem = sizeof(amp_t<R>) * (1u << (2 * K));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_dense<R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    uint64_t b = (W + 127) / 128;
    if (b > 152ull * 16) b = 152ull * 16;
    if (b < 1) b = 1;
    k_dense<R, K><<<(int)b, 128, smem, s>>>(static_cast<amp_t<R> *>(amp), W, fb, q,
                                              static_cast<const amp_t<R> *>(dU));
    return cudaGetLastError();
}

template <typename R>
cudaError_t dense_dispatch(void *amp, int k, uint64_t W, const FixedBits &fb, const Qpos &q, const void *dU,
                           cudaStream_t s) {
    switch (k) {
    case 1: return dense_k<R, 1>(amp, W, fb, q, dU, s);
    case 2: return dense_k<R, 2>(amp, W, fb, q, dU, s);
    case 3: return dense_k<R, 3>(amp, W, fb, q, dU, s);
    case 4: return dense_k<R, 4>(amp, W, fb, q, dU, s);
    case 5: return dense_k<R, 5>(amp, W, fb, q, dU, s);
    case 6: return dense_k<R, 6>(amp, W, fb, q, dU, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename R, int NP>
cudaError_t pairs_np(void *amp, uint64_t W, const FixedBits &fb, uint64_t pmask, int gc, const Mat2 &U,
                     cudaStream_t s) {
    const int grid = grid_for(W, kUnroll);
    amp_t<R> *a = static_cast<amp_t<R> *>(amp);
    switch (gc) {
    case GC_GENERAL: k_pairs<R, GC_GENERAL, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, U); break;
    case GC_REAL: k_pairs<R, GC_REAL, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, U); break;
    case GC_ANTIDIAG: k_pairs<R, GC_ANTIDIAG, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, U); break;
    case GC_EXCHANGE: k_pairs<R, GC_EXCHANGE, NP><<<grid, kThreads, 0, s>>>(a, W, fb, pmask, U); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t pairs_dispatch(void *amp, uint64_t W, const FixedBits &fb, uint64_t pmask, int gc, const Mat2 &U,
                           cudaStream_t s) {
    if (fb.npos <= 2) return pairs_np<R, 2>(amp, W, fb, pmask, gc, U, s);
    if (fb.npos <= 4) return pairs_np<R, 4>(amp, W, fb, pmask, gc, U, s);
    if (fb.npos <= 8) return pairs_np<R, 8>(amp, W, fb, pmask, gc, U, s);
    return pairs_np<R, kMaxFixed>(amp, W, fb, pmask, gc, U, s);
}

template <typename R>
cudaError_t diag_dispatch(void *amp, uint64_t W, const FixedBits &fb, int tbit, const Mat2 &U, cudaStream_t s) {
    const int grid = grid_for(W, kUnroll);
    amp_t<R> *a = static_cast<amp_t<R> *>(amp);
    if (fb.npos <= 2) k_diag<R, 2><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, U);
    else if (fb.npos <= 4) k_diag<R, 4><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, U);
    else if (fb.npos <= 8) k_diag<R, 8><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, U);
    else k_diag<R, kMaxFixed><<<grid, kThreads, 0, s>>>(a, W, fb, tbit, U);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_basis(void *amp, int dt, int n, uint64_t x, cudaStream_t s) {
    const uint64_t D = 1ull << n;
    const int grid = grid_for(D, 4);
    if (dt == 0)
        k_init_basis<float><<<grid, kThreads, 0, s>>>(static_cast<float2 *>(amp), D, x);
    else
        k_init_basis<double><<<grid, kThreads, 0, s>>>(static_cast<double2 *>(amp), D, x);
    return cudaGetLastError();
}

cudaError_t launch_shor_state(void *amp, int dt, int n, int X, uint64_t y, uint64_t G, cudaStream_t s) {
    if (X < 1 || X >= n || G < 2 || G >= (1ull << 32) || G > (1ull << (n - X))) return cudaErrorInvalidValue;
    const size_t bytes = (size_t)(dt == 0 ? 8 : 16) << n;
    cudaError_t e = cudaMemsetAsync(amp, 0, bytes, s);  // all-zero bits are +0.0
    if (e != cudaSuccess) return e;
    const uint64_t D = 1ull << X;
    const int grid = grid_for(D, 4);
    const double v = std::sqrt(std::ldexp(1.0, -X));  // 2^(-X/2), correctly rounded
    if (dt == 0)
        k_shor_state<float><<<grid, kThreads, 0, s>>>(static_cast<float2 *>(amp), X, y, G, (float)v);
    else
        k_shor_state<double><<<grid, kThreads, 0, s>>>(static_cast<double2 *>(amp), X, y, G, v);
    return cudaGetLastError();
}

cudaError_t launch_pairs(void *amp, int dt, int n, const FixedBitsHost &fbh, uint64_t pmask, int gc,
                         const Mat2 &U, cudaStream_t s) {
    if (fbh.npos > n || fbh.npos > kMaxFixed) return cudaErrorInvalidValue;
    const uint64_t W = 1ull << (n - fbh.npos);
    const FixedBits fb = to_dev(fbh);
    if (dt == 1 && gc != GC_EXCHANGE) return pairs_df(amp, W, fb, pmask, gc, U, s);
    return dt == 0 ? pairs_dispatch<float>(amp, W, fb, pmask, gc, U, s)
                   : pairs_dispatch<double>(amp, W, fb, pmask, gc, U, s);
}

cudaError_t launch_diag(void *amp, int dt, int n, const FixedBitsHost &fbh, int tbit, const Mat2 &U,
                        cudaStream_t s) {
    if (fbh.npos > n || fbh.npos > kMaxFixed) return cudaErrorInvalidValue;
    const uint64_t W = 1ull << (n - fbh.npos);
    const FixedBits fb = to_dev(fbh);
    if (dt == 1) return diag_df(amp, W, fb, tbit, U, s);
    return dt == 0 ? diag_dispatch<float>(amp, W, fb, tbit, U, s) : diag_dispatch<double>(amp, W, fb, tbit, U, s);
}

cudaError_t launch_dense(void *amp, int dt, int n, int k, const int *qpos, const void *dU, cudaStream_t s) {
    if (k < 1 || k > 6 || k > n) return cudaErrorInvalidValue;
    FixedBitsHost h{};
    int sorted[8];
    for (int j = 0; j < k; j++) sorted[j] = qpos[j];
    for (int i = 1; i < k; i++)
        for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; j--) {
            int t = sorted[j];
            sorted[j] = sorted[j - 1];
            sorted[j - 1] = t;
        }
    h.npos = k;
    for (int j = 0; j < k; j++) h.pos[j] = sorted[j];
    h.setmask = 0;
    Qpos q{};
    for (int j = 0; j < k; j++) q.p[j] = qpos[j];
    const uint64_t W = 1ull << (n - k);
    const FixedBits fb = to_dev(h);
    return dt == 0 ? dense_dispatch<float>(amp, k, W, fb, q, dU, s) : dense_dispatch<double>(amp, k, W, fb, q, dU, s);
}

}  // namespace qsim
