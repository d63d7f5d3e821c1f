// Algorithm 1: the accelerated causal-order search over the static
// precomputed matrix.  For k = 1..m the candidate c_k in U minimising
//     M_i = sum_{j in U, j != i} min(0, D_ij)^2            (Eq. 3)
// is appended to the order and removed from U.  The kernel keeps the running
// sums S_i = M_i in FP64 registers and subtracts P_{i,c} = min(0, D_ic)^2
// after each pick, which equals the literal recomputation over U up to FP64
// rounding.  Ties pick the lowest index.  One CTA: the m steps are strictly
// sequential, each one a block-wide argmin.
#include <cfloat>
#include <climits>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int OTH = 1024;
constexpr int PER = (VL_MAX_M + OTH - 1) / OTH;

// Pt[c * m + i] = min(0, D[i * m + c])^2, zero on the diagonal.
__global__ void pt_kernel(const double* __restrict__ D, int m, double* __restrict__ Pt, int* st) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    int i = i0 + r, c = c0 + tx;
    double v = 0.0;
    if (i < m && c < m) {
      double d = D[(int64_t)i * m + c];
      if (!isfinite(d)) set_status(st, VL_ERR_NONFINITE);
      v = (i != c && d < 0.0) ? d * d : 0.0;
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int c = c0 + r, i = i0 + tx;
    if (c < m && i < m) Pt[(int64_t)c * m + i] = tile[tx][r];
  }
}

struct Best {
  double v1;
  int i1;
  double v2;
};

__device__ __forceinline__ Best merge(Best a, Best b) {
  const bool bfirst = (b.v1 < a.v1) || (b.v1 == a.v1 && b.i1 < a.i1);
  Best r;
  if (bfirst) {
    r.v1 = b.v1;
    r.i1 = b.i1;
    r.v2 = fmin(a.v1, fmin(a.v2, b.v2));
  } else {
    r.v1 = a.v1;
    r.i1 = a.i1;
    r.v2 = fmin(b.v1, fmin(a.v2, b.v2));
  }
  return r;
}

__device__ __forceinline__ Best warp_merge(Best b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Best x;
    x.v1 = __shfl_xor_sync(0xffffffffu, b.v1, o);
    x.i1 = __shfl_xor_sync(0xffffffffu, b.i1, o);
    x.v2 = __shfl_xor_sync(0xffffffffu, b.v2, o);
    b = merge(b, x);
  }
  return b;
}

__global__ void __launch_bounds__(OTH) order_kernel(const double* __restrict__ Pt, int m,
                                                    int32_t* __restrict__ order,
                                                    double* __restrict__ gap) {
  __shared__ Best wb[32];
  __shared__ int s_c;
  const int nthr = blockDim.x;
  double S[PER];
  bool alive[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = threadIdx.x + q * nthr;
    alive[q] = i < m;
    double s = 0.0;
    if (alive[q])
      for (int j = 0; j < m; ++j) s += Pt[(int64_t)j * m + i];
    S[q] = s;
  }
  const int nw = (nthr + 31) >> 5;
  for (int k = 0; k < m; ++k) {
    Best b{DBL_MAX, INT_MAX, DBL_MAX};
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = threadIdx.x + q * nthr;
      if (alive[q]) b = merge(b, Best{S[q], i, DBL_MAX});
    }
    b = warp_merge(b);
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
      Best x = (threadIdx.x < nw) ? wb[threadIdx.x] : Best{DBL_MAX, INT_MAX, DBL_MAX};
      x = warp_merge(x);
      if (threadIdx.x == 0) {
        s_c = x.i1;
        order[k] = x.i1;
        if (gap) {
          double g;
          if (x.v2 == DBL_MAX) {
            g = __longlong_as_double(0x7ff0000000000000LL);  // +inf: one candidate left
          } else {
            double den = fmax(fmax(fabs(x.v1), fabs(x.v2)), 1e-300);
            g = (x.v2 - x.v1) / den;
          }
          gap[k] = g;
        }
      }
    }
    __syncthreads();
    const int c = s_c;
    const double* row = Pt + (int64_t)c * m;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = threadIdx.x + q * nthr;
      if (!alive[q]) continue;
      if (i == c)
        alive[q] = false;
      else
        S[q] -= row[i];
    }
  }
}

}  // namespace

void launch_causal_order(const double* D, int m, double* Pt, int32_t* order, double* gap,
                         int* st, cudaStream_t s) {
  dim3 grid((m + 31) / 32, (m + 31) / 32), block(32, 8);
  note_launch();
  pt_kernel<<<grid, block, 0, s>>>(D, m, Pt, st);
  int nthr = ((m + PER - 1) / PER + 31) / 32 * 32;
  if (nthr < 32) nthr = 32;
  if (nthr > OTH) nthr = OTH;
  note_launch();
  order_kernel<<<1, nthr, 0, s>>>(Pt, m, order, gap);
}

}  // namespace vl
