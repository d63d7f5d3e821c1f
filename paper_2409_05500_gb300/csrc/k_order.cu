// Algorithm 1: the accelerated causal-order search over the static
// precomputed matrix.  For k = 1..m the candidate c_k in U minimising
//     M_i = sum_{j in U, j != i} min(0, D_ij)^2            (Eq. 3)
// is appended to the order and removed from U (ties: lowest index).
//
// GB300 design.  The m steps are strictly sequential, so the search is one
// CTA and its cost is latency per step.  FP64 issues at 1/64 of the FP32 rate
// on this part, so the running sums S_i = M_i are kept as double-float pairs
// (hi + lo, two FP32 numbers, ~48-bit significand) and updated with TwoSum
// after each pick, S_i -= P_{i,c}.  The argmin compares an order-preserving
// 64-bit integer key built from (hi, lo) with the warp reduction instruction
// (__reduce_min_sync), so no floating-point compare sits on the critical path.
// The initial sums are computed in FP64 by a parallel kernel; the per-step
// relative gaps are computed after the search by another.  Subtracting the
// removed column instead of re-summing over U gives the same sums as the
// literal recomputation up to rounding (~1e-14 relative).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>

#include "vl_internal.cuh"


namespace vl {

namespace {

constexpr int OTH = 1024;
static_assert(VL_MAX_M <= 4 * OTH, "ordering holds at most four variables per thread");

// Pt_hi/lo[c * m + i] = min(0, D[i * m + c])^2 as a double-float pair.
__global__ void pt_kernel(const double* __restrict__ D, int m, float* __restrict__ pth,
                          float* __restrict__ ptl, int* st) {
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
    if (c < m && i < m) {
      double v = tile[tx][r];
      float hi = (float)v;
      pth[(int64_t)c * m + i] = hi;
      ptl[(int64_t)c * m + i] = (float)(v - (double)hi);
    }
  }
}

// S_i = sum_{j != i} min(0, D_ij)^2 in FP64, one warp per row, fixed order.
__global__ void rowsum_kernel(const double* __restrict__ D, int m, float* __restrict__ sh,
                              float* __restrict__ sl) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) {
    double d = D[(int64_t)i * m + j];
    if (j != i && d < 0.0) s += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    float hi = (float)s;
    sh[i] = hi;
    sl[i] = (float)(s - (double)hi);
  }
}

// order-preserving map float -> uint32 (valid for every non-NaN value)
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
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

struct Cand {
  uint32_t kh, kl;  // key of (hi, lo)
  int idx;
};

__device__ __forceinline__ bool cless(const Cand& a, const Cand& b) {
  if (a.kh != b.kh) return a.kh < b.kh;
  if (a.kl != b.kl) return a.kl < b.kl;
  return a.idx < b.idx;
}

// lexicographic warp-wide minimum of (kh, kl, idx) with REDUX
__device__ __forceinline__ Cand warp_min(Cand c) {
  const uint32_t full = 0xffffffffu;
  uint32_t mh = __reduce_min_sync(full, c.kh);
  uint32_t kl = (c.kh == mh) ? c.kl : 0xffffffffu;
  uint32_t ml = __reduce_min_sync(full, kl);
  uint32_t id = (c.kh == mh && c.kl == ml) ? (uint32_t)c.idx : 0xffffffffu;
  uint32_t mi = __reduce_min_sync(full, id);
  return Cand{mh, ml, (int)mi};
}

__device__ __forceinline__ Cand none() { return Cand{0xffffffffu, 0xffffffffu, INT_MAX}; }

// Warp-wide lexicographic minimum of (kh, kl, idx), in every lane.  A real
// score never has the key 0xffffffff (that is a NaN pattern), so a warp whose
// minimum kh is 0xffffffff holds no live candidate.  Fast path: one lane holds
// the minimum kh (REDUX + VOTE + SHFL); ties on kh take the full three-key
// reduction.  *src returns the winning lane (-1 if none).
__device__ __forceinline__ Cand warp_argmin(const Cand& c, int* src) {
  const uint32_t full = 0xffffffffu;
  const uint32_t mh = __reduce_min_sync(full, c.kh);
  if (mh == 0xffffffffu) {
    *src = -1;
    return none();
  }
  const uint32_t bal = __ballot_sync(full, c.kh == mh);
  if (__popc(bal) == 1) {
    const int l = __ffs(bal) - 1;
    *src = l;
    return Cand{mh, __shfl_sync(full, c.kl, l), __shfl_sync(full, c.idx, l)};
  }
  const Cand w = warp_min(c);
  *src = __ffs(__ballot_sync(full, c.idx == w.idx && c.kh == w.kh && c.kl == w.kl)) - 1;
  return w;
}

// One CTA of up to 1024 threads, each owning PER variables (i = tid + q*nthr).
// A step: every warp finds its best and runner-up (warp_argmin), writes them
// to a shared slot of the step's parity, one barrier, then every warp reduces
// the warp winners itself, so all threads learn the pick c and the runner-up
// r without a second barrier (slots alternate by parity: a warp can run at
// most one step ahead of the slowest).  Then S_i -= P_{i,c}.  The P column of
// the pick is loaded together with the column of the runner-up; when the
// runner-up wins the next step (about 60% of the steps on the workloads
// measured) that step uses the prefetched registers and skips the L2 round
// trip.
template <int PER>
__global__ void __launch_bounds__(OTH) order_kernel(const float* __restrict__ pth,
                                                    const float* __restrict__ ptl,
                                                    const float* __restrict__ sh0,
                                                    const float* __restrict__ sl0, int m,
                                                    int32_t* __restrict__ order,
                                                    float4* __restrict__ best2) {
  __shared__ Cand wb1[2][32], wb2[2][32];
  const int nthr = blockDim.x, nw = (nthr + 31) >> 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float hi[PER], lo[PER], nh[PER], nl[PER];
  bool alive[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = threadIdx.x + q * nthr;
    alive[q] = i < m;
    hi[q] = alive[q] ? sh0[i] : 0.f;
    lo[q] = alive[q] ? sl0[i] : 0.f;
    nh[q] = nl[q] = 0.f;
  }
  int pre = -1;
  for (int k = 0; k < m; ++k) {
    const int ph = k & 1;
    // this thread's best and runner-up
    Cand b1 = none(), b2 = none();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      if (!alive[q]) continue;
      const Cand c{fkey(hi[q]), fkey(lo[q]), (int)threadIdx.x + q * nthr};
      if (PER == 1) {
        b1 = c;
      } else if (cless(c, b1)) {
        b2 = b1;
        b1 = c;
      } else if (cless(c, b2)) {
        b2 = c;
      }
    }
    // warp level: the winning lane writes its own candidate
    int l1, l2;
    warp_argmin(b1, &l1);
    const Cand s2 = (lane == l1) ? b2 : b1;
    warp_argmin(s2, &l2);
    if (lane == 0 && l1 < 0) wb1[ph][wid] = none();
    if (lane == l1) wb1[ph][wid] = b1;
    if (lane == 0 && l2 < 0) wb2[ph][wid] = none();
    if (lane == l2) wb2[ph][wid] = s2;
    __syncthreads();
    // block level, redundantly in every warp
    const Cand a1 = lane < nw ? wb1[ph][lane] : none();
    const Cand a2 = lane < nw ? wb2[ph][lane] : none();
    int g1l, g2l;
    const Cand g1 = warp_argmin(a1, &g1l);
    const int c = g1.idx;
    const Cand g2 = warp_argmin((lane == g1l) ? a2 : a1, &g2l);
    const int r = g2.idx;
    if (threadIdx.x == 0) {
      order[k] = c;
      best2[k] = make_float4(fkey_inv(g1.kh), fkey_inv(g1.kl),
                             r == INT_MAX ? __int_as_float(0x7f800000) : fkey_inv(g2.kh),
                             r == INT_MAX ? 0.f : fkey_inv(g2.kl));
    }
    float ch[PER], cl[PER];
    if (c == pre) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        ch[q] = nh[q];
        cl[q] = nl[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x + q * nthr;
        ch[q] = alive[q] ? pth[(int64_t)c * m + i] : 0.f;
        cl[q] = alive[q] ? ptl[(int64_t)c * m + i] : 0.f;
      }
    }
    if (r != INT_MAX) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x + q * nthr;
        nh[q] = alive[q] ? pth[(int64_t)r * m + i] : 0.f;
        nl[q] = alive[q] ? ptl[(int64_t)r * m + i] : 0.f;
      }
      pre = r;
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
  }
}

__global__ void gap_kernel(const float4* __restrict__ best2, int m, double* __restrict__ gap) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  float4 b = best2[k];
  if (isinf(b.z)) {
    gap[k] = __longlong_as_double(0x7ff0000000000000LL);
    return;
  }
  double s1 = (double)b.x + (double)b.y;
  double s2 = (double)b.z + (double)b.w;
  double den = fmax(fmax(fabs(s1), fabs(s2)), 1e-300);
  gap[k] = (s2 - s1) / den;
}

}  // namespace

size_t order_ws_bytes(int m) {
  return (size_t)m * m * 2 * sizeof(float) + (size_t)m * 2 * sizeof(float) +
         (size_t)m * sizeof(float4) + 1024;
}

void launch_causal_order(const double* D, int m, void* ws, int32_t* order, double* gap, int* st,
                         cudaStream_t s) {
  char* p = static_cast<char*>(ws);
  float* pth = reinterpret_cast<float*>(p);
  float* ptl = pth + (size_t)m * m;
  float* sh = ptl + (size_t)m * m;
  float* sl = sh + m;
  float4* best2 = reinterpret_cast<float4*>(((uintptr_t)(sl + m) + 15) & ~(uintptr_t)15);
  dim3 grid((m + 31) / 32, (m + 31) / 32), block(32, 8);
  note_launch();
  pt_kernel<<<grid, block, 0, s>>>(D, m, pth, ptl, st);
  note_launch();
  rowsum_kernel<<<(m + 7) / 8, 256, 0, s>>>(D, m, sh, sl);
  // variables per thread: PER = 1 up to 1024 variables, then 2 and 4
  const int per = m <= OTH ? 1 : (m <= 2 * OTH ? 2 : 4);
  const int nthr = std::min(OTH, ((m + per - 1) / per + 31) / 32 * 32);
  note_launch();
  if (per == 1)
    order_kernel<1><<<1, nthr, 0, s>>>(pth, ptl, sh, sl, m, order, best2);
  else if (per == 2)
    order_kernel<2><<<1, nthr, 0, s>>>(pth, ptl, sh, sl, m, order, best2);
  else
    order_kernel<4><<<1, nthr, 0, s>>>(pth, ptl, sh, sl, m, order, best2);
  if (gap) {
    note_launch();
    gap_kernel<<<(m + 255) / 256, 256, 0, s>>>(best2, m, gap);
  }
}

}  // namespace vl

// ------------------------------------------------------------------------
// Allocation-free variant of the search, for callers that must not allocate
// device memory after start-up.  Its scratch is this file-scope array; every
// GPU that loads the library holds it until the process exits.
namespace vl {
namespace {

constexpr size_t kNoallocBytes =
    (size_t)VL_NOALLOC_MAX_M * VL_NOALLOC_MAX_M * 2 * sizeof(float) +
    (size_t)VL_NOALLOC_MAX_M * 2 * sizeof(float) + (size_t)VL_NOALLOC_MAX_M * sizeof(float4) +
    1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

}  // namespace

}  // namespace vl

extern "C" vl_status vl_causal_order_noalloc(void* cuda_stream, const double* D, int m,
                                             int32_t* order, double* gap) {
  using namespace vl;
  if (!D || !order) return VL_ERR_ARG;
  if (m < 1) return VL_ERR_SHAPE;
  if (m > VL_NOALLOC_MAX_M) return VL_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return VL_ERR_CUDA;
  }
  void* scratch;
  {
    // first call on this device: resolve the array's device address (host
    // code cannot use the symbol itself: on the host it names a stand-in)
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return VL_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (order_ws_bytes(m) > kNoallocBytes) return VL_ERR_UNSUPPORTED;
  launch_causal_order(D, m, scratch, order, gap, nullptr, static_cast<cudaStream_t>(cuda_stream));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VL_OK : VL_ERR_CUDA;
}
