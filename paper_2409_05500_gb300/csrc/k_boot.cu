// Bootstrap of the whole method (no counterpart in the paper's experiments;
// the moving-block resampling of Kuensch 1989 for dependent series).
//
// Resample b of an m x n series is the concatenation of blocks of block_len
// consecutive time points, block k starting at
//   s_k = floor(u_k (n - block_len + 1) / 2^64),
//   u_k = SplitMix64 output number b 2^32 + k + 1 for the seed
// (Steele, Lea and Flood 2014: output number c of the generator seeded with
// `seed` is mix(seed + c * 0x9E3779B97F4A7C15), mix being two
// multiply-xorshift rounds and a final xorshift), cut to n.  The generator
// is counter based, so any thread computes any draw with no shared state and
// a resample does not depend on how resamples are grouped into launches.
//
// After the fits: the inverse permutation of every resample's causal order
// (pos[order[k]] = k), then per pair (i, j) the number of resamples with
// |B0[i][j]| > threshold and with i before j, accumulated as doubles (exact
// integers) and divided by the number of resamples at the end.
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int kBootThreads = 256;
constexpr int kBootRows = 16;  // rows of X gathered by one CTA

__device__ __forceinline__ unsigned long long splitmix64_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// grid (ceil(n / 256), ceil(m / 16), nb): thread t of resample b0 + z finds
// its source time point once and gathers it for 16 rows.  Within a block of
// the resample consecutive threads read consecutive time points, so the
// loads coalesce except where a warp spans a block boundary.
__global__ void __launch_bounds__(kBootThreads) boot_resample_kernel(
    const double* __restrict__ X, int64_t ldx, int m, int n, int block_len,
    unsigned long long seed, long long b0, double* __restrict__ out) {
  const int t = blockIdx.x * kBootThreads + threadIdx.x;
  if (t >= n) return;
  const unsigned long long b = (unsigned long long)(b0 + blockIdx.z);
  const int k = t / block_len, off = t - k * block_len;
  const unsigned long long counter = (b << 32) + (unsigned long long)k + 1ull;
  const unsigned long long u = splitmix64_mix(seed + counter * 0x9E3779B97F4A7C15ull);
  const unsigned long long span = (unsigned long long)(n - block_len + 1);
  const int src = (int)__umul64hi(u, span) + off;
  const int i0 = blockIdx.y * kBootRows, i1 = min(m, i0 + kBootRows);
  double* o = out + ((int64_t)blockIdx.z * m) * n + t;
  for (int i = i0; i < i1; ++i) o[(int64_t)i * n] = X[(int64_t)i * ldx + src];
}

// pos[z m + order[z m + k]] = k; an entry out of range (not a permutation)
// sets VL_ERR_ARG and is skipped.
__global__ void boot_inverse_kernel(const int32_t* __restrict__ order, int m,
                                    int32_t* __restrict__ pos, int* st) {
  const int32_t* o = order + (int64_t)blockIdx.x * m;
  int32_t* q = pos + (int64_t)blockIdx.x * m;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int v = o[k];
    if (v < 0 || v >= m) {
      set_status(st, VL_ERR_ARG);
      continue;
    }
    q[v] = k;
  }
}

// One thread per (i, j), looping over the nb resamples of a chunk.
__global__ void __launch_bounds__(kBootThreads) boot_count_kernel(
    const double* __restrict__ B0, const int32_t* __restrict__ pos, int m, int nb,
    double threshold, double* __restrict__ edge, double* __restrict__ before) {
  const int64_t mm = (int64_t)m * m;
  const int64_t e = (int64_t)blockIdx.x * kBootThreads + threadIdx.x;
  if (e >= mm) return;
  const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
  int ce = 0, cb = 0;
  for (int z = 0; z < nb; ++z) {
    ce += fabs(B0[z * mm + e]) > threshold;
    cb += pos[(int64_t)z * m + i] < pos[(int64_t)z * m + j];
  }
  edge[e] += (double)ce;
  before[e] += (double)cb;
}

__global__ void boot_normalize_kernel(double* __restrict__ edge, double* __restrict__ before,
                                      int64_t mm, double count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mm;
       e += (int64_t)gridDim.x * blockDim.x) {
    edge[e] = edge[e] / count;
    before[e] = before[e] / count;
  }
}

}  // namespace

void launch_boot_resample(const double* X, int64_t ldx, int m, int n, int block_len,
                          unsigned long long seed, long long b0, int nb, double* out,
                          cudaStream_t s) {
  constexpr int kMaxZ = 65535;  // grid.z limit
  for (int z0 = 0; z0 < nb; z0 += kMaxZ) {
    note_launch();
    dim3 grid((n + kBootThreads - 1) / kBootThreads, (m + kBootRows - 1) / kBootRows,
              std::min(kMaxZ, nb - z0));
    boot_resample_kernel<<<grid, kBootThreads, 0, s>>>(X, ldx, m, n, block_len, seed, b0 + z0,
                                                       out + (int64_t)z0 * m * n);
  }
}

void launch_boot_count(const int32_t* order, const double* B0, int m, int nb, double threshold,
                       int32_t* pos, double* edge, double* before, int* st, cudaStream_t s) {
  note_launch();
  boot_inverse_kernel<<<nb, 256, 0, s>>>(order, m, pos, st);
  note_launch();
  const int64_t mm = (int64_t)m * m;
  boot_count_kernel<<<(unsigned)((mm + kBootThreads - 1) / kBootThreads), kBootThreads, 0, s>>>(
      B0, pos, m, nb, threshold, edge, before);
}

void launch_boot_normalize(double* edge, double* before, int m, int count, cudaStream_t s) {
  note_launch();
  const int64_t mm = (int64_t)m * m;
  const int blocks = (int)std::min<int64_t>((mm + 255) / 256, 4096);
  boot_normalize_kernel<<<blocks, 256, 0, s>>>(edge, before, mm, (double)count);
}

}  // namespace vl
