// fpair.cuh -- two FP32 values in one packed operation.
//
// sm_100 and later execute add, sub, mul and fma on a pair of FP32 values
// held in a 64-bit register pair (PTX add/sub/mul/fma.rn.f32x2) as one
// instruction.  Each lane rounds exactly as the scalar .rn operation does
// (IEEE round to nearest even, subnormals kept), so error-free
// transformations built from scalar operations stay error free lane by lane.
// The host versions are the scalar operations, so the same code compiles and
// gives the same results on the CPU.
#pragma once

#if defined(__CUDACC__)
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif

namespace qsim {

struct fpair {
    float x, y;
};

#if defined(__CUDA_ARCH__)
#define QSIM_FP2_OP(NAME, OP)                                                                               \
    __device__ __forceinline__ fpair NAME##_dev(fpair a, fpair b) {                                         \
        fpair r;                                                                                            \
        asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t" OP           \
            " pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"                                                    \
            : "=f"(r.x), "=f"(r.y)                                                                          \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                      \
        return r;                                                                                           \
    }
QSIM_FP2_OP(fp_add, "add.rn.f32x2")
QSIM_FP2_OP(fp_sub, "sub.rn.f32x2")
QSIM_FP2_OP(fp_mul, "mul.rn.f32x2")
#undef QSIM_FP2_OP
#endif

FP_HD fpair fp_add(fpair a, fpair b) {
#if defined(__CUDA_ARCH__)
    return fp_add_dev(a, b);
#else
    return fpair{a.x + b.x, a.y + b.y};
#endif
}
FP_HD fpair fp_sub(fpair a, fpair b) {
#if defined(__CUDA_ARCH__)
    return fp_sub_dev(a, b);
#else
    return fpair{a.x - b.x, a.y - b.y};
#endif
}
FP_HD fpair fp_mul(fpair a, fpair b) {
#if defined(__CUDA_ARCH__)
    return fp_mul_dev(a, b);
#else
    return fpair{a.x * b.x, a.y * b.y};
#endif
}
FP_HD fpair fp_splat(float v) { return fpair{v, v}; }

}  // namespace qsim
