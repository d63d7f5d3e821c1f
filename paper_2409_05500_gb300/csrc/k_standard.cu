// The iterative search of Sec. 3 (steps 1-5) on the device: after the
// pairwise measure of the remaining variables (the library's pairwise
// kernels), one kernel scores every candidate by Eq. 3 and picks the
// minimiser, and one kernel removes the pick and replaces every other
// remaining variable by its residual on it (Eq. 4).  The pick never leaves
// the device: the host only enqueues the m - 1 iterations.
//
// Data layout: the remaining variables are kept compacted, u rows of one
// FP64 buffer in their original relative order, so the local index of a
// variable orders the same way as its original index (the tie rule) and the
// pairwise kernels see a plain u x n matrix; idx maps local to original.
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int SC_WARPS = 8;  // rows scored per CTA (one warp per row)
constexpr int RF_TH = 256;   // threads of a refinement CTA (a row is 1-8 CTAs)

// smallest score, its index (lowest among equal scores) and the second
// smallest score (equal values counted separately)
struct Best {
  double v1;
  int i1;
  double v2;
};

__device__ __forceinline__ Best merge(Best a, Best b) {
  const bool take_b = b.v1 < a.v1 || (b.v1 == a.v1 && b.i1 < a.i1);
  Best o;
  if (take_b) {
    o.v1 = b.v1;
    o.i1 = b.i1;
    o.v2 = fmin(a.v1, b.v2);
  } else {
    o.v1 = a.v1;
    o.i1 = a.i1;
    o.v2 = fmin(a.v2, b.v1);
  }
  return o;
}

__device__ __forceinline__ Best shfl_best(Best b, int o) {
  Best r;
  r.v1 = __shfl_xor_sync(0xffffffffu, b.v1, o);
  r.i1 = __shfl_xor_sync(0xffffffffu, b.i1, o);
  r.v2 = __shfl_xor_sync(0xffffffffu, b.v2, o);
  return r;
}

// Eq. 3 for every remaining candidate a: S_a = sum_{b != a} min(0, D_ab)^2
// over the u x u measure of this iteration (one warp per row, FP64).  The
// last CTA to finish takes the argmin (ties: lowest index), writes
// order[k] = idx[pick], gap[k] = (S_(2) - S_(1)) / max(|S_(1)|, |S_(2)|) and
// the pick, and re-arms the counter for the next iteration.
__global__ void __launch_bounds__(SC_WARPS * 32)
    std_score_pick_kernel(const double* __restrict__ D, int u, double* __restrict__ S,
                          unsigned* __restrict__ counter, const int32_t* __restrict__ idx,
                          int32_t* __restrict__ order, double* __restrict__ gap, int k,
                          int* __restrict__ pick, int* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.x * SC_WARPS + warp;
  if (a < u) {
    const double* row = D + (int64_t)a * u;
    double s = 0.0;
    for (int b = lane; b < u; b += 32) {
      const double d = row[b];
      if (b != a && d < 0.0) s = fma(d, d, s);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) S[a] = s;
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double INF = __longlong_as_double(0x7ff0000000000000LL);
  Best b{INF, 0x7fffffff, INF};
  for (int i = threadIdx.x; i < u; i += blockDim.x) b = merge(b, Best{__ldcg(S + i), i, INF});
#pragma unroll
  for (int o = 16; o; o >>= 1) b = merge(b, shfl_best(b, o));
  __shared__ Best wb[SC_WARPS];
  if (lane == 0) wb[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    Best r = wb[0];
    for (int w = 1; w < SC_WARPS; ++w) r = merge(r, wb[w]);
    if (r.i1 >= u) {  // no finite score: D was not finite
      set_status(st, VL_ERR_NONFINITE);
      r.i1 = 0;
    }
    *pick = r.i1;
    order[k] = idx ? idx[r.i1] : r.i1;
    if (gap) {
      const double den = fmax(fmax(fabs(r.v1), fabs(r.v2)), 1e-300);
      gap[k] = r.v2 == INF ? INF : (r.v2 - r.v1) / den;
    }
    *counter = 0u;
  }
}

// Eq. 4 for output row an (0..u-2): source row a = an, skipping the pick;
// x_a <- x_a - (C_a,pick / C_pick,pick) x_pick, where C (u x u) holds the
// centred cross products of this iteration's data that the measure computed
// for its correlations, so the ratio is cov(x_a, x_pick) / var(x_pick)
// (ddof cancels).  FP64.  Writes the compacted row, idx_next[an] = idx[a]
// and, when one variable is left, its order entry.
__global__ void __launch_bounds__(RF_TH)
    std_refine_kernel(const double* __restrict__ W, int64_t ldw, int u, int n,
                      const double* __restrict__ C, const int* __restrict__ pick,
                      const int32_t* __restrict__ idx, double* __restrict__ Wn, int64_t ldn,
                      int32_t* __restrict__ idx_next, int32_t* __restrict__ order,
                      double* __restrict__ gap, int k) {
  const int pk = *pick;
  const int an = blockIdx.y;
  const int a = an + (an >= pk ? 1 : 0);
  const double slope = C[(int64_t)a * u + pk] / C[(int64_t)pk * u + pk];
  const double* xa = W + (int64_t)a * ldw;
  const double* xp = W + (int64_t)pk * ldw;
  double* dst = Wn + (int64_t)an * ldn;
  for (int t = blockIdx.x * RF_TH + threadIdx.x; t < n; t += gridDim.x * RF_TH)
    dst[t] = fma(-slope, xp[t], xa[t]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int32_t orig = idx ? idx[a] : a;
    idx_next[an] = orig;
    if (u == 2) {  // the last variable closes the order
      order[k + 1] = orig;
      if (gap) gap[k + 1] = __longlong_as_double(0x7ff0000000000000LL);
    }
  }
}

}  // namespace

void launch_std_score_pick(const double* D, int u, double* S, unsigned* counter,
                           const int32_t* idx, int32_t* order, double* gap, int k, int* pick,
                           int* st, cudaStream_t s) {
  note_launch();
  std_score_pick_kernel<<<(u + SC_WARPS - 1) / SC_WARPS, SC_WARPS * 32, 0, s>>>(
      D, u, S, counter, idx, order, gap, k, pick, st);
}

void launch_std_refine(const double* W, int64_t ldw, int u, int n, const double* C,
                       const int* pick, const int32_t* idx, double* Wn, int64_t ldn,
                       int32_t* idx_next, int32_t* order, double* gap, int k, cudaStream_t s) {
  const int chunks = std::min(8, std::max(1, (n + 4 * RF_TH - 1) / (4 * RF_TH)));
  note_launch();
  std_refine_kernel<<<dim3(chunks, u - 1), RF_TH, 0, s>>>(W, ldw, u, n, C, pick, idx, Wn, ldn,
                                                          idx_next, order, gap, k);
}

}  // namespace vl
