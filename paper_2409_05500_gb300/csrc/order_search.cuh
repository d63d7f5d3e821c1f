// Device pieces of Algorithm 1's search (Eq. 3 argmin over the remaining
// set), shared by the plain search (k_order.cu) and the search resumed after
// an FP64 re-evaluation of a near tie (k_certify.cu).
//
// The running sums S_i = sum_{j in U, j != i} min(0, D_ij)^2 are double-float
// pairs (hi + lo, two FP32 numbers, ~48-bit significand) updated with TwoSum,
// because FP64 issues at 1/64 of the FP32 rate on this part.  The argmin
// compares an order-preserving 64-bit integer key built from (hi, lo) and the
// index with two warp reduction instructions and no branch.
#pragma once

#include "vl_internal.cuh"

namespace vl {
namespace search {

constexpr int OTH = 1024;  // threads of the one-CTA search

// order-preserving map float -> uint32 (valid for every non-NaN value)
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// (hi, lo) -= (ph, pl) in double-float, renormalised so |lo| <= ulp(hi)/2
// (then the pair order equals the order of (key(hi), key(lo))).
__device__ __forceinline__ void df_sub(float& hi, float& lo, float ph, float pl) {
  float s = hi - ph;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (-ph - bp);
  float l = lo - pl + err;
  float h2 = s + l;
  lo = l - (h2 - s);
  hi = h2;
}

// clock64 read ordered after `dep` is available
__device__ __forceinline__ long long clock_after(float dep) {
  long long t;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(t) : "f"(dep));
  return t;
}

// Search key of a live variable: (fkey(hi), fkey(lo) with its low 12 bits
// replaced by the index).  Compared as a 64-bit integer it orders by the
// double-float score and then by index; dropping 12 bits of lo merges
// scores closer than about 2^-35 relative into index order, far below any
// gap the method distinguishes.  A dead variable is (~0, ~0).
__device__ __forceinline__ uint2 skey(float hi, float lo, int i) {
  return make_uint2(fkey(hi), (fkey(lo) & 0xfffff000u) | (uint32_t)i);
}
// The score a key encodes (lo without its 12 index bits).
__device__ __forceinline__ double skey_score(uint2 k) {
  return (double)fkey_inv(k.x) + (double)fkey_inv(k.y & 0xfffff000u);
}
// warp-wide minimum key, in every lane (two REDUX, no branches)
__device__ __forceinline__ uint2 warp_kmin(uint2 k) {
  const uint32_t full = 0xffffffffu;
  const uint32_t h = __reduce_min_sync(full, k.x);
  const uint32_t l = __reduce_min_sync(full, k.x == h ? k.y : 0xffffffffu);
  return make_uint2(h, l);
}

// order-preserving map double -> uint64
__device__ __forceinline__ unsigned long long dkey(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Steps kbeg .. m-1 of the search, one CTA of up to 1024 threads, each owning
// PER variables (i = tid + q*nthr).  A step: every warp reduces its keys
// (warp_kmin) and lane 0 writes the warp minimum to a shared slot of the
// step's parity; one barrier; every warp then reduces the warp minima itself,
// so all threads learn the pick c without a second barrier (slots alternate by
// parity: a warp can run at most one step ahead of the slowest); S_i -=
// P_{i,c}.  forced >= 0 makes step kbeg pick that variable without a search
// (its score is then not recorded).  spick (optional): the winning score of
// every searched step.  fetch(c, i, h, l) loads P_{i,c} as the double-float
// pair (h, l).  prof (optional): clock64 stamps of thread 0, five per step:
// start, warp minimum written, after the barrier, pick known, update done.
template <int PER, class Fetch>
__device__ __forceinline__ void search_steps(float (&hi)[PER], float (&lo)[PER],
                                             bool (&alive)[PER], int m, int kbeg, int forced,
                                             int32_t* __restrict__ order,
                                             double* __restrict__ spick,
                                             long long* __restrict__ prof, Fetch fetch) {
  __shared__ uint2 wb[2][32];
  const int nthr = blockDim.x, nw = (nthr + 31) >> 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint2 dead = make_uint2(0xffffffffu, 0xffffffffu);
  for (int k = kbeg; k < m; ++k) {
    const int ph = k & 1;
    int c;
    if (k == kbeg && forced >= 0) {
      c = forced;
    } else {
      if (prof && threadIdx.x == 0) prof[5 * k] = clock64();
      uint2 b = dead;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const uint2 cq = alive[q] ? skey(hi[q], lo[q], (int)threadIdx.x + q * nthr) : dead;
        if (cq.x < b.x || (cq.x == b.x && cq.y < b.y)) b = cq;
      }
      const uint2 w = warp_kmin(b);
      if (lane == 0) wb[ph][wid] = w;
      if (prof && threadIdx.x == 0) prof[5 * k + 1] = clock64();
      __syncthreads();
      if (prof && threadIdx.x == 0) prof[5 * k + 2] = clock64();
      // block level, redundantly in every warp
      const uint2 a = lane < nw ? wb[ph][lane] : dead;
      const uint2 g = warp_kmin(a);
      c = (int)(g.y & 0xfffu);
      if (prof && threadIdx.x == 0) prof[5 * k + 3] = clock64();
      if (spick && threadIdx.x == 0) spick[k] = skey_score(g);
    }
    if (threadIdx.x == 0) order[k] = c;
    float ch[PER], cl[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      ch[q] = cl[q] = 0.f;
      if (alive[q]) fetch(c, (int)threadIdx.x + q * nthr, ch[q], cl[q]);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = threadIdx.x + q * nthr;
      if (!alive[q]) continue;
      if (i == c)
        alive[q] = false;
      else
        df_sub(hi[q], lo[q], ch[q], cl[q]);
    }
    if (prof && threadIdx.x == 0) prof[5 * k + 4] = clock_after(hi[0]);
  }
}

}  // namespace search
}  // namespace vl
