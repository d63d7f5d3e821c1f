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
// 64-bit integer key built from (hi, lo) and the index with two warp
// reduction instructions (__reduce_min_sync) and no branch, so no
// floating-point compare sits on the critical path; scores closer than about
// 2^-35 relative are taken as tied and go by index.
// The initial sums are computed in FP64 by a parallel kernel; the per-step
// relative gaps are computed after the search by another.  Subtracting the
// removed column instead of re-summing over U gives the same sums as the
// literal recomputation up to rounding (~1e-14 relative).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>

#include "order_search.cuh"


namespace vl {

namespace {

using namespace search;
static_assert(VL_MAX_M <= 4 * OTH, "ordering holds at most four variables per thread");
static_assert(VL_MAX_M <= 4096, "the search key holds the variable index in 12 bits");

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

// Search with P in global memory (L2): Pt_hi/lo[c * m + i] = P_{i,c}.
template <int PER>
__global__ void __launch_bounds__(OTH) order_kernel(const float* __restrict__ pth,
                                                    const float* __restrict__ ptl,
                                                    const float* __restrict__ sh0,
                                                    const float* __restrict__ sl0, int m,
                                                    int32_t* __restrict__ order,
                                                    double* __restrict__ spick,
                                                    long long* __restrict__ prof) {
  float hi[PER], lo[PER];
  bool alive[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = threadIdx.x + q * blockDim.x;
    alive[q] = i < m;
    hi[q] = alive[q] ? sh0[i] : 0.f;
    lo[q] = alive[q] ? sl0[i] : 0.f;
  }
  search_steps<PER>(hi, lo, alive, m, 0, -1, order, spick, prof,
                    [&](int c, int i, float& h, float& l) {
    h = pth[(int64_t)c * m + i];
    l = ptl[(int64_t)c * m + i];
  });
}

// The same search with P held in distributed shared memory: a cluster of
// OC_CTAS CTAs, CTA t keeping the rows i in [t R, (t+1) R) of P for every
// column c (R = ceil(m / OC_CTAS), layout [c][i - t R] as (hi, lo) pairs).  CTA 0
// runs the search; the others only hold their rows until it is done.  A
// step's load of P_{i,c} is then a distributed-shared-memory load (about 200
// clocks) instead of an L2 load of Pt (about 750 clocks on this part, two
// thirds of a step at m = 400).  The only synchronisation is a cluster barrier
// after the rows are loaded and one at the end, so no CTA leaves while its
// rows can still be read.
constexpr int OC_CTAS = 8;
constexpr int OC_MAX_M = 448;  // R m (hi, lo) pairs must fit one CTA's shared memory

inline size_t oc_smem(int m) {
  const int R = (m + OC_CTAS - 1) / OC_CTAS;
  return (size_t)R * m * sizeof(float2);
}

__global__ void __launch_bounds__(OTH) order_cluster_kernel(const float* __restrict__ pth,
                                                            const float* __restrict__ ptl,
                                                            const float* __restrict__ sh0,
                                                            const float* __restrict__ sl0, int m,
                                                            int32_t* __restrict__ order,
                                                            double* __restrict__ spick) {
  extern __shared__ __align__(16) float2 oc_rows[];
  unsigned rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int R = (m + OC_CTAS - 1) / OC_CTAS;
  const int i0 = (int)rank * R;
  for (int idx = threadIdx.x; idx < R * m; idx += blockDim.x) {
    const int c = idx / R, il = idx - c * R, i = i0 + il;
    oc_rows[idx] = i < m ? make_float2(pth[(int64_t)c * m + i], ptl[(int64_t)c * m + i])
                         : make_float2(0.f, 0.f);
  }
  __syncthreads();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
  if (rank == 0) {
    const int i = threadIdx.x;
    float hi[1], lo[1];
    bool alive[1];
    alive[0] = i < m;
    hi[0] = alive[0] ? sh0[i] : 0.f;
    lo[0] = alive[0] ? sl0[i] : 0.f;
    // this thread's row: owner CTA and local index, as a shared::cluster base
    const int own = min(i / R, OC_CTAS - 1);
    uint32_t base = (uint32_t)__cvta_generic_to_shared(oc_rows) + 8u * (uint32_t)(i - own * R);
    asm volatile("mapa.shared::cluster.u32 %0, %0, %1;" : "+r"(base) : "r"(own));
    const uint32_t stride = 8u * (uint32_t)R;
    search_steps<1>(hi, lo, alive, m, 0, -1, order, spick, nullptr,
                    [&](int c, int, float& h, float& l) {
      asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];"
                   : "=f"(h), "=f"(l)
                   : "r"(base + stride * (uint32_t)c)
                   : "memory");
    });
  }
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Launch the cluster search; false if m is out of its range or the cluster
// cannot be launched (the caller then runs order_kernel).
bool launch_order_cluster(const OrderWs& w, int m, int32_t* order, double* spick,
                          cudaStream_t s) {
  if (m < 64 || m > OC_MAX_M) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(order_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)oc_smem(OC_MAX_M)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(OC_CTAS, 1, 1);
  cfg.blockDim = dim3((m + 31) / 32 * 32, 1, 1);
  cfg.dynamicSmemBytes = oc_smem(m);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = OC_CTAS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  if (cudaLaunchKernelEx(&cfg, order_cluster_kernel, (const float*)w.pth, (const float*)w.ptl,
                         (const float*)w.sh, (const float*)w.sl, m, order, spick) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Gaps after the search, from the order: variable i replays its score
// S_i = sum_{j in U} P_ij step by step in FP64; at the step that picks it, it
// records its score as the minimum s1[k]; at earlier steps it offers its
// score to the step's runner-up s2[k] (atomic minimum of an ordered key).
// Steps are taken eight at a time so that their loads overlap.
__global__ void gap_scores_kernel(const float* __restrict__ pth, const float* __restrict__ ptl,
                                  const float* __restrict__ sh0, const float* __restrict__ sl0,
                                  const int32_t* __restrict__ order, int m,
                                  double* __restrict__ s1, unsigned long long* __restrict__ s2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = (double)sh0[i] + (double)sl0[i];
  for (int t0 = 0; t0 < m; t0 += 8) {
    int cs[8];
    double p[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) cs[u] = t0 + u < m ? order[t0 + u] : i;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      p[u] = (double)pth[(int64_t)cs[u] * m + i] + (double)ptl[(int64_t)cs[u] * m + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (cs[u] == i) {
        if (t0 + u < m) s1[t0 + u] = s;
        return;
      }
      atomicMin(&s2[t0 + u], dkey(s));
      s -= p[u];
    }
  }
}

__global__ void gap_kernel(const double* __restrict__ s1, const unsigned long long* __restrict__ s2,
                           int m, double* __restrict__ gap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  if (s2[k] == ~0ull) {
    gap[k] = __longlong_as_double(0x7ff0000000000000LL);
    return;
  }
  const double a = s1[k], b = dkey_inv(s2[k]);
  const double den = fmax(fmax(fabs(a), fabs(b)), 1e-300);
  gap[k] = (b - a) / den;
}

}  // namespace

OrderWs order_ws_layout(void* ws, int m) {
  OrderWs w;
  char* p = static_cast<char*>(ws);
  w.pth = reinterpret_cast<float*>(p);
  w.ptl = w.pth + (size_t)m * m;
  w.sh = w.ptl + (size_t)m * m;
  w.sl = w.sh + m;
  w.s1 = reinterpret_cast<double*>(((uintptr_t)(w.sl + m) + 15) & ~(uintptr_t)15);
  w.s2 = reinterpret_cast<unsigned long long*>(w.s1 + m);
  return w;
}

void launch_order_gaps(void* ws, int m, const int32_t* order, double* gap, cudaStream_t s) {
  const OrderWs w = order_ws_layout(ws, m);
  cudaMemsetAsync(w.s2, 0xff, (size_t)m * sizeof(unsigned long long), s);
  note_launch();
  gap_scores_kernel<<<(m + 127) / 128, 128, 0, s>>>(w.pth, w.ptl, w.sh, w.sl, order, m, w.s1,
                                                      w.s2);
  note_launch();
  gap_kernel<<<(m + 255) / 256, 256, 0, s>>>(w.s1, w.s2, m, gap);
}

size_t order_ws_bytes(int m) {
  return (size_t)m * m * 2 * sizeof(float) + (size_t)m * 2 * sizeof(float) +
         (size_t)m * sizeof(float4) + 1024;
}

void launch_causal_order(const double* D, int m, void* ws, int32_t* order, double* gap, int* st,
                         cudaStream_t s, long long* prof, double* spick) {
  const OrderWs w = order_ws_layout(ws, m);
  dim3 grid((m + 31) / 32, (m + 31) / 32), block(32, 8);
  note_launch();
  pt_kernel<<<grid, block, 0, s>>>(D, m, w.pth, w.ptl, st);
  note_launch();
  rowsum_kernel<<<(m + 7) / 8, 256, 0, s>>>(D, m, w.sh, w.sl);
  // P in distributed shared memory (64 <= m <= 448), unless profiling
  if (!prof && launch_order_cluster(w, m, order, spick, s)) {
    if (gap) launch_order_gaps(ws, m, order, gap, s);
    return;
  }
  // variables per thread: PER = 1 up to 1024 variables, then 2 and 4
  const int per = m <= OTH ? 1 : (m <= 2 * OTH ? 2 : 4);
  const int nthr = std::min(OTH, ((m + per - 1) / per + 31) / 32 * 32);
  note_launch();
  if (per == 1)
    order_kernel<1><<<1, nthr, 0, s>>>(w.pth, w.ptl, w.sh, w.sl, m, order, spick, prof);
  else if (per == 2)
    order_kernel<2><<<1, nthr, 0, s>>>(w.pth, w.ptl, w.sh, w.sl, m, order, spick, prof);
  else
    order_kernel<4><<<1, nthr, 0, s>>>(w.pth, w.ptl, w.sh, w.sl, m, order, spick, prof);
  if (gap) launch_order_gaps(ws, m, order, gap, s);
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
  // an error the caller left pending is not this call's: report only an
  // error that the launches below raise (and clear only that one)
  const cudaError_t before = cudaPeekAtLastError();
  launch_causal_order(D, m, scratch, order, gap, nullptr, static_cast<cudaStream_t>(cuda_stream));
  const cudaError_t after = cudaPeekAtLastError();
  if (after == cudaSuccess || after == before) return VL_OK;
  cudaGetLastError();
  return VL_ERR_CUDA;
}
