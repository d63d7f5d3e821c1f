// Diagnostics: the special-function unit's throughput on this part, for the
// roofline of the pairwise kernel (whose per-sample cost is its exponentials
// and logarithms).
//
// One CTA of 1024 threads per SM; every thread runs 8 independent chains of
// the instruction under test (ex2.approx or lg2.approx), so each SM sub-
// partition has far more independent warp instructions in flight than the
// unit's latency; thread 0 reads the SM clock (clock64) around the loop.
// Rate = results per clock per SM = 1024 x 8 x iterations / cycles, the
// median over the CTAs.
#include <algorithm>
#include <vector>

#include "vl_internal.cuh"

namespace vl {

namespace {

template <bool LG2>
__global__ void __launch_bounds__(1024, 1) sfu_rate_kernel(int iters, long long* cycles,
                                                             float* sink) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1.0f + 0.001f * (threadIdx.x + j);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float y;
      if (LG2) {
        // lg2 of a value in [1, 2): the chain stays in [1, 2)
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
        x[j] = 1.0f + 0.5f * y;
      } else {
        // ex2 of a value in (-1, 0]: the chain stays in (0.5, 1]
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[j] * 0.5f));
        x[j] = y;
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 12345.f) sink[threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

}  // namespace vl

extern "C" vl_status vl_sfu_rate(int device, double* ex2_per_clk_sm, double* lg2_per_clk_sm) {
  using namespace vl;
  if (!ex2_per_clk_sm || !lg2_per_clk_sm) return VL_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return VL_ERR_CUDA;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  long long* cyc = nullptr;
  float* sink = nullptr;
  vl_status st = VL_OK;
  if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(float) * 1024) != cudaSuccess) {
    cudaGetLastError();
    st = VL_ERR_NOMEM;
  }
  const int iters = 4096;
  for (int which = 0; which < 2 && st == VL_OK; ++which) {
    std::vector<long long> h(sms);
    double rate = 0.0;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
      note_launch();
      if (which == 0)
        sfu_rate_kernel<false><<<sms, 1024>>>(iters, cyc, sink);
      else
        sfu_rate_kernel<true><<<sms, 1024>>>(iters, cyc, sink);
      if (cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
        cudaGetLastError();
        st = VL_ERR_CUDA;
        break;
      }
      std::sort(h.begin(), h.end());
      rate = 1024.0 * 8.0 * iters / (double)std::max(1LL, h[sms / 2]);
    }
    (which == 0 ? *ex2_per_clk_sm : *lg2_per_clk_sm) = rate;
  }
  if (cyc) cudaFree(cyc);
  if (sink) cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
