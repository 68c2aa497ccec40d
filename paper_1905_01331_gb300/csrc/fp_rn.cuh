// Round-to-nearest FP32 add, subtract and multiply that the compiler may not
// fuse into an FMA.  The error-free transformations of the pair arithmetic
// (two-sum, product residual) are exact only if every operation rounds once
// as written: nvcc contracts a*b + c into one FMA by default, which would
// break them.  Device code uses the _rn intrinsics (never contracted); host
// code (the tests' drivers) is compiled with -ffp-contract=off.
#pragma once

#ifdef __CUDACC__
#define RN_HD __host__ __device__ __forceinline__
#else
#define RN_HD inline
#endif

namespace ttn {
namespace rn {

RN_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
RN_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
RN_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
RN_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

}  // namespace rn
}  // namespace ttn
