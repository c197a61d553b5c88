// common.cuh -- device helpers shared by the sm_103a kernels of the simulator.
//
// Amplitude storage is interleaved (re, im): float2 for complex64, double2 for
// complex128.  Index conventions follow Sec. II.A (qubit q = bit q, qubit 0 the
// least significant bit).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qsim {

// ---------------------------------------------------------------- amplitudes
template <typename R> struct Amp;
template <> struct Amp<float>  { using V = float2;  };
template <> struct Amp<double> { using V = double2; };

template <typename R> using amp_t = typename Amp<R>::V;

template <typename R>
__device__ __forceinline__ amp_t<R> mk(R x, R y) { amp_t<R> v; v.x = x; v.y = y; return v; }

// (u * a): complex product
template <typename R>
__device__ __forceinline__ amp_t<R> cmul(amp_t<R> u, amp_t<R> a) {
    return mk<R>(u.x * a.x - u.y * a.y, u.x * a.y + u.y * a.x);
}
// (u * a + v * b): the row of a 2x2 complex matrix times a pair
template <typename R>
__device__ __forceinline__ amp_t<R> cmul2(amp_t<R> u, amp_t<R> a, amp_t<R> v, amp_t<R> b) {
    R re = u.x * a.x;
    re = fma(-u.y, a.y, re);
    re = fma(v.x, b.x, re);
    re = fma(-v.y, b.y, re);
    R im = u.x * a.y;
    im = fma(u.y, a.x, im);
    im = fma(v.x, b.y, im);
    im = fma(v.y, b.x, im);
    return mk<R>(re, im);
}

// ------------------------------------------------------------- index algebra
// Insert a zero bit at position pos (the bits at and above pos move up by one).
__device__ __host__ __forceinline__ uint64_t insert_zero(uint64_t i, int pos) {
    const uint64_t lo = i & ((1ull << pos) - 1ull);
    return ((i >> pos) << (pos + 1)) | lo;
}

// Fixed bits inserted into a compact enumeration index: positions must be
// ascending; after insertion the bits of setmask are forced to 1.  Used to
// enumerate only the amplitudes a gate touches (target bit 0, controls 1).
constexpr int kMaxFixed = 24;
struct FixedBits {
    int npos;
    int pos[kMaxFixed];
    uint64_t setmask;
};

__device__ __forceinline__ uint64_t expand(uint64_t p, const FixedBits &fb) {
#pragma unroll 1
    for (int k = 0; k < fb.npos; k++) p = insert_zero(p, fb.pos[k]);
    return p | fb.setmask;
}

// Same, with the loop unrolled to a compile-time bound NP >= fb.npos so the
// positions stay in registers.
template <int NP>
__device__ __forceinline__ uint64_t expand_n(uint64_t p, const FixedBits &fb) {
#pragma unroll
    for (int k = 0; k < NP; k++)
        if (k < fb.npos) p = insert_zero(p, fb.pos[k]);
    return p | fb.setmask;
}

// Scatter the low bits of j onto the positions listed in pos[0..cnt-1].
__device__ __host__ __forceinline__ uint64_t deposit(uint64_t j, const int *pos, int cnt) {
    uint64_t r = 0;
    for (int k = 0; k < cnt; k++) r |= ((j >> k) & 1ull) << pos[k];
    return r;
}

// ------------------------------------------------------- bounded waits / error
// Error word written by a kernel whose bounded wait expired; the host reads it
// back and reports QSIM_ETIMEOUT.
enum : uint32_t { kErrNone = 0, kErrTimeout = 1, kErrBadOp = 2 };

}  // namespace qsim
