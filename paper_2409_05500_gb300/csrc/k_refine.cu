// One step of iterative refinement of the VAR least-squares coefficients
// (Sec. 4.1) on the mixed-precision path.
//
// The normal equations G_zz beta = G_zy (centred lagged Gram, from the
// tensor-core product, FP64) are factored and solved in FP32 (Cholesky,
// triangular solves), which leaves beta0 with a relative error of about
// cond(G_zz) 2^-24.  One refinement step
//     r = G_zy - G_zz beta0           (= Z^T (Y - Z beta0), double-float)
//     G_zz delta = r                  (the FP32 factor again)
//     beta = beta0 + delta            (FP64)
// removes the factorisation's error to first order: the residual is formed
// with the normal equations split into FP32 (hi, lo) pairs and every product
// and sum kept as an exact or compensated double-float (about 2^-44
// relative), so only beta's own rounding and the Gram's error remain.
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int RT = 32;   // output tile (rows of r) x (columns of r): m = 400 gives 169 CTAs
constexpr int RK = 32;   // k-chunk staged in shared memory
constexpr int RTH = 128; // threads: 8 x 16, each 4 rows x 2 columns (one float2)

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Partial sums sum_{c in split z} NE[a][m + c] beta0[c][i], a < mp, i < m,
// with NE = (hi + lo) the centred normal equations (mp x q, q = m (p + 1))
// and beta0 (FP32, mp x m), as double-float pairs (the two columns of a
// thread as one float2, on the paired FP32 instructions).  The K range (c) is
// split over blockIdx.z in chunks of kchunk so that the grid fills the GPU;
// part[z][a][i] = (hi, lo) of split z.
__global__ void __launch_bounds__(RTH, 4)
    refine_residual_kernel(const float* __restrict__ nhi, const float* __restrict__ nlo, int m,
                           int mp, const float* __restrict__ beta0, int kchunk,
                           float2* __restrict__ part) {
  __shared__ float Ah[RK][RT + 1], Al[RK][RT + 1];
  __shared__ __align__(8) float Bs[RK][RT];
  const int q = m + mp;
  const int a0 = blockIdx.y * RT, i0 = blockIdx.x * RT;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const float2 mone = f2(-1.f, -1.f);
  float2 sh[4], sl[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) sh[u] = sl[u] = f2(0.f, 0.f);
  const int cbeg = blockIdx.z * kchunk, cend = min(mp, cbeg + kchunk);
  for (int c0 = cbeg; c0 < cend; c0 += RK) {
    for (int idx = threadIdx.x; idx < RK * RT; idx += RTH) {
      const int kk = idx % RK, rr = idx / RK;  // A: rows a, consecutive k per thread group
      const int a = a0 + rr, c = c0 + kk;
      const bool ok = a < mp && c < cend;
      Ah[kk][rr] = ok ? nhi[(int64_t)a * q + m + c] : 0.f;
      Al[kk][rr] = ok ? nlo[(int64_t)a * q + m + c] : 0.f;
      const int kb = idx / RT, ii = idx % RT;  // B: rows c, consecutive i
      const int cb = c0 + kb, i = i0 + ii;
      Bs[kb][ii] = (cb < cend && i < m) ? beta0[(int64_t)cb * m + i] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < RK; ++kk) {
      const float2 b = *reinterpret_cast<const float2*>(&Bs[kk][tx * 2]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float ahs = Ah[kk][ty * 4 + u], als = Al[kk][ty * 4 + u];
        const float2 ah = f2(ahs, ahs), al = f2(als, als);
        // exact product ah b = p + e, plus al b; added to (sh, sl) by TwoSum
        const float2 p = __fmul2_rn(ah, b);
        const float2 e = __ffma2_rn(al, b, __ffma2_rn(ah, b, __fmul2_rn(p, mone)));
        const float2 s = __fadd2_rn(sh[u], p);
        const float2 bp = __ffma2_rn(sh[u], mone, s);                  // s - sh
        const float2 t = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, mone, s), mone, sh[u]),
                                    __ffma2_rn(bp, mone, p));         // (sh - (s - bp)) + (p - bp)
        sh[u] = s;
        sl[u] = __fadd2_rn(sl[u], __fadd2_rn(t, e));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = a0 + ty * 4 + u;
    if (a >= mp) continue;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + tx * 2 + v;
      if (i >= m) continue;
      part[((int64_t)blockIdx.z * mp + a) * m + i] =
          v ? make_float2(sh[u].y, sl[u].y) : make_float2(sh[u].x, sl[u].x);
    }
  }
}

// r[a][i] = NE[a][i] - sum_z part[z][a][i]: the split partials added in
// double-float (TwoSum), the difference with the right-hand side likewise;
// r rounded to FP32 at the end (it is small, and only feeds the FP32
// correction solve).
__global__ void refine_reduce_kernel(const float* __restrict__ nhi, const float* __restrict__ nlo,
                                     int m, int mp, const float2* __restrict__ part, int splits,
                                     float* __restrict__ r) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)mp * m) return;
  const int a = (int)(idx / m), i = (int)(idx % m);
  float h = 0.f, l = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float2 v = part[(int64_t)z * mp * m + idx];
    const float s = h + v.x;
    const float bp = s - h;
    const float err = (h - (s - bp)) + (v.x - bp);
    h = s;
    l += err + v.y;
  }
  // r = (yh + yl) - (h + l)
  const int q = m + mp;
  const float yh = nhi[(int64_t)a * q + i], yl = nlo[(int64_t)a * q + i];
  const float d = yh - h;
  const float bp = d - yh;
  const float err = (yh - (d - bp)) + (-h - bp);
  r[idx] = d + (err + (yl - l));
}

// beta = beta0 + delta: M[tau][i][k] in FP64 from beta[(tau-1) m + k][i], and
// beta0 replaced by its FP32 rounding (for the residuals of the VAR).
__global__ void refine_apply_kernel(float* __restrict__ beta, const float* __restrict__ delta,
                                    int m, int p, double* __restrict__ M) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p * m * m) return;
  const int a = (int)(idx / m), i = (int)(idx % m);  // a = tau m + k (0-based tau)
  const double v = (double)beta[idx] + (double)delta[idx];
  const int tau = a / m, k = a % m;
  M[((int64_t)tau * m + i) * m + k] = v;
  beta[idx] = (float)v;
}

}  // namespace

int refine_splits(int m, int p, int num_sms) {
  const int mp = m * p;
  const int base = ((m + RT - 1) / RT) * ((mp + RT - 1) / RT);
  // about four CTAs per SM, each K chunk at least two staging rounds
  return std::max(1, std::min({REFINE_MAX_SPLITS, (4 * num_sms + base - 1) / base,
                               (mp + 2 * RK - 1) / (2 * RK)}));
}

void launch_refine_residual(const float* nhi, const float* nlo, int m, int p, const float* beta0,
                            float* r, float2* part, int num_sms, cudaStream_t s) {
  const int mp = m * p, splits = refine_splits(m, p, num_sms);
  const int kchunk = ((mp + splits - 1) / splits + RK - 1) / RK * RK;
  const int nz = (mp + kchunk - 1) / kchunk;
  dim3 grid((m + RT - 1) / RT, (mp + RT - 1) / RT, nz);
  note_launch();
  refine_residual_kernel<<<grid, RTH, 0, s>>>(nhi, nlo, m, mp, beta0, kchunk, part);
  const int64_t tot = (int64_t)mp * m;
  note_launch();
  refine_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nhi, nlo, m, mp, part, nz, r);
}

void launch_refine_apply(float* beta, const float* delta, int m, int p, double* M,
                         cudaStream_t s) {
  const int64_t tot = (int64_t)p * m * m;
  note_launch();
  refine_apply_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(beta, delta, m, p, M);
}

}  // namespace vl
