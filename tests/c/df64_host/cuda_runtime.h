/* Host stand-in for the few CUDA declarations df64.cuh uses, so that its
 * double-float arithmetic compiles with g++ and can be checked on the CPU:
 * the _rn intrinsics are IEEE single-precision operations with round to
 * nearest (compiled with -ffp-contract=off, so no product and sum fuse),
 * fmaf is the correctly rounded fused multiply-add, and the qualifiers expand
 * to nothing.  Found before the real header through -I. */
#ifndef DF64_HOST_CUDA_RUNTIME_H
#define DF64_HOST_CUDA_RUNTIME_H
#include <cmath>
#include <cstring>

#define __device__
#define __host__
#define __forceinline__ inline
#define __constant__

struct float2 {
  float x, y;
};
inline float2 make_float2(float a, float b) { return {a, b}; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
inline int __float_as_int(float f) {
  int i;
  std::memcpy(&i, &f, sizeof i);
  return i;
}
inline float __int_as_float(int i) {
  float f;
  std::memcpy(&f, &i, sizeof f);
  return f;
}
using std::log1pf;
#endif
