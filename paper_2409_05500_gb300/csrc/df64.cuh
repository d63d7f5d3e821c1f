// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the
// FP32 pipes (this part issues FP32 at ~80x its FP64 rate).
//
// Error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker) and the
// product error from a fused multiply-add; the sums and products of pairs
// follow the double-double algorithms of Hida, Li and Bailey (2001) in their
// "sloppy" form (relative error about 2^-46 of the operands' magnitudes).
// Every step uses the _rn intrinsics so that the compiler cannot contract a
// product and a sum into one FMA, which would break the transformations.
//
// exp: Cody-Waite reduction x = (32 m + j) ln2 / 32 + r, |r| <= ln2 / 64, with
// ln2 / 32 as a float pair; e^r by its Taylor series to r^6 (the r^4..r^6
// terms in FP32, the rest in pairs); the result T_j e^r 2^m with T_j =
// 2^(j / 32) as a float pair.  log1p: one Newton step on e^L = 1 + y from the
// FP32 log1pf.  The constants are the float pairs nearest to 1 / k!, ln2 / 32,
// 32 / ln2 and 2^(j / 32) (hi the nearest float, lo the nearest float to the
// remainder).
#pragma once

#include <cuda_runtime.h>

namespace vl {
namespace df {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 add(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}

// x + y when |x.hi| >= |y.hi| is known (a constant term of a series plus a
// smaller remainder): FastTwoSum in place of the first TwoSum
__device__ __forceinline__ F2 add_big(F2 x, F2 y) {
  F2 s = fast_two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ F2 neg(F2 x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ F2 mul(F2 x, F2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ F2 mul_f(F2 x, float b) {
  const float p = __fmul_rn(x.hi, b);
  float e = __fmaf_rn(x.hi, b, -p);
  e = __fmaf_rn(x.lo, b, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ F2 sqr(F2 x) {
  const float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(__fmul_rn(2.0f, x.hi), x.lo, e);
  return fast_two_sum(p, e);
}

// multiply by a power of two (exact unless the result leaves the normal range)
__device__ __forceinline__ F2 scale(F2 x, float p2) { return {__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)}; }

__host__ __device__ __forceinline__ F2 from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

__host__ __device__ __forceinline__ double to_double(F2 x) { return (double)x.hi + (double)x.lo; }

// 2^(j / 32), j = 0..31, as float pairs (staged into shared memory by the
// kernels that use dexp, whose lanes index it at random)
static __constant__ float2 kExp2Frac[32] = {
    {1.0f, 0.0f}, {1.0218971967697144f, -4.811559861650494e-08f},
    {1.0442737340927124f, 4.8334701574503924e-08f}, {1.0671404600143433f, -5.9337519786595294e-08f},
    {1.0905077457427979f, -1.3077539939843064e-08f}, {1.114386796951294f, -5.435540018083884e-08f},
    {1.1387885808944702f, 5.386222312608879e-08f}, {1.1637248992919922f, -4.051441493402308e-08f},
    {1.1892070770263672f, 3.797635272917432e-08f}, {1.215247392654419f, -3.267394887984665e-08f},
    {1.2418577671051025f, 4.496838101886169e-08f}, {1.2690509557724f, 1.419333317542737e-09f},
    {1.2968395948410034f, -4.018999533172973e-08f}, {1.3252366781234741f, -3.496373324196611e-08f},
    {1.3542555570602417f, -1.0123349269974824e-08f}, {1.3839099407196045f, -5.875577357983275e-08f},
    {1.4142135381698608f, 2.4203234971764687e-08f}, {1.4451807737350464f, 3.324199937537742e-08f},
    {1.4768261909484863f, -4.500898853621038e-08f}, {1.5091644525527954f, -2.4959373234878512e-08f},
    {1.5422108173370361f, 8.070904833346049e-09f}, {1.5759809017181396f, -5.661025426206834e-08f},
    {1.610490322113037f, 9.836217174097328e-09f}, {1.6457555294036865f, -5.124972091152813e-08f},
    {1.6817928552627563f, -2.4755326677450284e-08f}, {1.7186193466186523f, -4.8496175963919086e-08f},
    {1.7562521696090698f, -9.235770370707996e-09f}, {1.7947090864181519f, -1.141504490931311e-08f},
    {1.8340080976486206f, -1.1239277952768134e-08f}, {1.8741676807403564f, -4.663005626071026e-08f},
    {1.9152065515518188f, 9.845328108326612e-09f}, {1.9571441411972046f, -1.7021804410433106e-08f},
};

constexpr float LN2_32_HI = 0.021660849452018738f;  // ln2 / 32
constexpr float LN2_32_LO = -5.952044412893542e-11f;
constexpr float INV_LN2_32 = 46.16624069213867f;    // 32 / ln2 (only rounds the index)
constexpr float C3_HI = 0.1666666716337204f, C3_LO = -4.967053879312289e-09f;  // 1/3!
constexpr float C4 = 0.0416666679084301f;   // 1/4!
constexpr float C5 = 0.008333333767950535f;  // 1/5!
constexpr float C6 = 0.0013888889225199819f;  // 1/6!

// e^x for x.hi in [-87, 87]; 0 below -87 (e^-87 ~ 1.6e-38: the callers'
// terms there are far below their sums' resolution).  tab: kExp2Frac, usually
// staged in shared memory.
__device__ __forceinline__ F2 dexp(F2 x, const float2* tab) {
  if (x.hi < -87.0f) return {0.0f, 0.0f};
  // k = nearest integer to x 32/ln2: adding 1.5 2^23 leaves the rounded
  // integer in the low mantissa bits (|x 32/ln2| < 2^22), which avoids the
  // slower round and float-to-int conversion instructions
  constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
  const float kb = __fmaf_rn(x.hi, INV_LN2_32, kRound);
  const int k = __float_as_int(kb) - __float_as_int(kRound);
  const float kf = __fsub_rn(kb, kRound);
  // r = x - k ln2/32: k * hi exactly as a pair, x.hi - p exact (Sterbenz)
  const float p = __fmul_rn(kf, LN2_32_HI);
  const float pe = __fmaf_rn(kf, LN2_32_HI, -p);
  const float t = __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, LN2_32_LO));
  const F2 r = two_sum(__fsub_rn(x.hi, p), t);
  // e^r = 1 + r + r^2/2 + r^3/6 + r^4/24 + r^5/120 + r^6/720; with |r| < 0.011
  // every Horner step adds a remainder smaller than its constant
  const float q = __fmaf_rn(r.hi, __fmaf_rn(r.hi, C6, C5), C4);
  F2 s = add_big(F2{C3_HI, C3_LO}, mul_f(r, q));
  s = add_big(F2{0.5f, 0.0f}, mul(r, s));
  s = add_big(F2{1.0f, 0.0f}, mul(r, s));
  s = add_big(F2{1.0f, 0.0f}, mul(r, s));
  const float2 tj = tab[k & 31];
  s = mul(s, F2{tj.x, tj.y});
  const int m2 = k >> 5;  // floor(k / 32)
  return scale(s, __int_as_float((m2 + 127) << 23));
}

// log(1 + y) for y in [0, 1]
__device__ __forceinline__ F2 dlog1p(F2 y, const float2* tab) {
  const float l0 = log1pf(y.hi);
  const F2 e = dexp(F2{-l0, 0.0f}, tab);  // e^{-l0}
  F2 z = fast_two_sum(1.0f, y.hi);  // y <= 1
  z.lo = __fadd_rn(z.lo, y.lo);
  const F2 q = mul(z, e);  // (1 + y) e^{-l0} = 1 + w
  const float w = __fadd_rn(__fsub_rn(q.hi, 1.0f), q.lo);
  return two_sum(l0, __fmaf_rn(-0.5f * w, w, w));  // l0 + log(1 + w)
}

}  // namespace df
}  // namespace vl
