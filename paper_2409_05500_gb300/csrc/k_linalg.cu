// Small dense linear algebra on the CUDA cores: a tiled GEMM over strided
// views, a compensated hi/lo split product for covariances, and a blocked
// Cholesky factorisation with blocked triangular solves built from them.
//
// Precision: with T = float every product is an FP32 FMA; partial sums are
// flushed every `kFlush` steps of k into a double-float (hi, lo) accumulator
// (TwoSum), so the error does not grow with K.  With T = double everything is
// FP64.  Split-K partials are combined in FP64 in a fixed order (deterministic).
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int NTH = 256;
constexpr int KC = 8;  // k-depth of one shared-memory stage

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

// Reciprocal and square root for the factorisations: the single-instruction
// approximations in FP32 (a few ulp; the FP32 factorisation's own rounding
// dominates), IEEE in FP64.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_fast(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// Register-staged loads of one BM x KC stage of a view.  With ks == 1
// consecutive threads read consecutive k of a row, otherwise consecutive rows.
template <class T, int BM>
struct StageLoader {
  static constexpr int TOT = BM * KC;
  static constexpr int PER = (TOT + NTH - 1) / NTH;  // the last slot may be partial
  T v[PER];
  __device__ __forceinline__ static void slot(int idx, int ks, int& r, int& k) {
    if (ks == 1) {
      r = idx / KC;
      k = idx % KC;
    } else {
      r = idx % BM;
      k = idx / BM;
    }
  }
  __device__ __forceinline__ void load(const View<T>& w, int r0, int rows, int k0, int kmax) {
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * NTH;
      if (TOT % NTH != 0 && idx >= TOT) break;
      int r, k;
      slot(idx, w.ks, r, k);
      const int gr = r0 + r, gk = k0 + k;
      v[e] = (gr < rows && gk < kmax) ? w.base[(int64_t)gr * w.rs + (int64_t)gk * w.ks] : T(0);
    }
  }
  __device__ __forceinline__ void store(T* sm, int ks) const {  // sm[k * (BM + 4) + r]
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + e * NTH;
      if (TOT % NTH != 0 && idx >= TOT) break;
      int r, k;
      slot(idx, ks, r, k);
      sm[k * (BM + 4) + r] = v[e];
    }
  }
};

// mode: 0 = full, 1 = lower (c <= r), 2 = upper (c >= r, mirrored into C[c, r]).
// C[r, c] = alpha * sum_k A(r, k) B(c, k) + beta * C[r, c], or, with split-K
// (gridDim.z > 1), slice z's partial into part[z][r][c].  The next k-stage is
// loaded into registers while the current one is consumed (double buffer).
// SPLIT: A and B come as (hi, lo) FP32 pairs; each step adds hi*hi + hi*lo +
// lo*hi and the FP32 sum is flushed every 32 steps into a double-float pair.
template <class T, class TC, int TMt, int TNt, bool SPLIT>
__global__ void __launch_bounds__(NTH) gemm_kernel(int M, int N, int K, int kchunk,
                                                   double alpha, View<T> A, View<T> Al, View<T> B,
                                                   View<T> Bl, double beta, TC* __restrict__ C,
                                                   int64_t ldc, int mode,
                                                   double* __restrict__ part) {
  constexpr int BM = 16 * TMt, BN = 16 * TNt;
  constexpr int NOP = SPLIT ? 2 : 1;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  if (mode == 1 && c0 > r0 + BM - 1) return;
  if (mode == 2 && r0 > c0 + BN - 1) return;
  __shared__ __align__(16) T As[2][NOP][KC * (BM + 4)];
  __shared__ __align__(16) T Bs[2][NOP][KC * (BN + 4)];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  T acc[TMt][TNt];
  float hi[SPLIT ? TMt : 1][SPLIT ? TNt : 1], lo[SPLIT ? TMt : 1][SPLIT ? TNt : 1];
#pragma unroll
  for (int a = 0; a < TMt; ++a)
#pragma unroll
    for (int b = 0; b < TNt; ++b) acc[a][b] = T(0);
  if constexpr (SPLIT) {
#pragma unroll
    for (int a = 0; a < TMt; ++a)
#pragma unroll
      for (int b = 0; b < TNt; ++b) hi[a][b] = lo[a][b] = 0.f;
  }
  StageLoader<T, BM> la, lal;
  StageLoader<T, BN> lb, lbl;
  const int nst = kend > kbeg ? (kend - kbeg + KC - 1) / KC : 0;
  if (nst > 0) {
    la.load(A, r0, M, kbeg, kend);
    lb.load(B, c0, N, kbeg, kend);
    la.store(As[0][0], A.ks);
    lb.store(Bs[0][0], B.ks);
    if constexpr (SPLIT) {
      lal.load(Al, r0, M, kbeg, kend);
      lbl.load(Bl, c0, N, kbeg, kend);
      lal.store(As[0][NOP - 1], Al.ks);
      lbl.store(Bs[0][NOP - 1], Bl.ks);
    }
  }
  __syncthreads();
  for (int t = 0; t < nst; ++t) {
    const int buf = t & 1;
    const bool more = t + 1 < nst;
    if (more) {
      const int k1 = kbeg + (t + 1) * KC;
      la.load(A, r0, M, k1, kend);
      lb.load(B, c0, N, k1, kend);
      if constexpr (SPLIT) {
        lal.load(Al, r0, M, k1, kend);
        lbl.load(Bl, c0, N, k1, kend);
      }
    }
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T a[TMt], b[TNt];
#pragma unroll
      for (int q = 0; q < TMt; ++q) a[q] = As[buf][0][kk * (BM + 4) + ty * TMt + q];
#pragma unroll
      for (int q = 0; q < TNt; ++q) b[q] = Bs[buf][0][kk * (BN + 4) + tx * TNt + q];
      if constexpr (SPLIT) {
        T al[TMt], bl[TNt];
#pragma unroll
        for (int q = 0; q < TMt; ++q) al[q] = As[buf][NOP - 1][kk * (BM + 4) + ty * TMt + q];
#pragma unroll
        for (int q = 0; q < TNt; ++q) bl[q] = Bs[buf][NOP - 1][kk * (BN + 4) + tx * TNt + q];
#pragma unroll
        for (int x = 0; x < TMt; ++x)
#pragma unroll
          for (int y = 0; y < TNt; ++y) {
            T tt = fma(a[x], bl[y], al[x] * b[y]);
            acc[x][y] = fma(a[x], b[y], acc[x][y] + tt);
          }
      } else {
#pragma unroll
        for (int x = 0; x < TMt; ++x)
#pragma unroll
          for (int y = 0; y < TNt; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
      }
    }
    if constexpr (SPLIT) {
      if ((t & 3) == 3) {  // every 32 steps of k
#pragma unroll
        for (int x = 0; x < TMt; ++x)
#pragma unroll
          for (int y = 0; y < TNt; ++y) {
            two_sum_acc(hi[x][y], lo[x][y], (float)acc[x][y]);
            acc[x][y] = T(0);
          }
      }
    }
    if (more) {
      la.store(As[buf ^ 1][0], A.ks);
      lb.store(Bs[buf ^ 1][0], B.ks);
      if constexpr (SPLIT) {
        lal.store(As[buf ^ 1][NOP - 1], Al.ks);
        lbl.store(Bs[buf ^ 1][NOP - 1], Bl.ks);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TMt; ++x)
#pragma unroll
    for (int y = 0; y < TNt; ++y) {
      const int r = r0 + ty * TMt + x, c = c0 + tx * TNt + y;
      if (r >= M || c >= N) continue;
      if (mode == 1 && c > r) continue;
      if (mode == 2 && c < r) continue;
      if constexpr (!SPLIT && sizeof(T) == 4) {
        // all-FP32 epilogue (FP64 conversions run at 1/64 rate on this part):
        // split-K slices leave FP32 partials, reduced by splitk_reduce_f32
        if (part) {
          reinterpret_cast<float*>(part)[((int64_t)blockIdx.z * M + r) * N + c] =
              (float)alpha * acc[x][y];
          continue;
        }
        if constexpr (sizeof(TC) == 4) {
          float v = (float)alpha * acc[x][y];
          if (beta != 0.0) v = fmaf((float)beta, C[(int64_t)r * ldc + c], v);
          C[(int64_t)r * ldc + c] = v;
          if (mode == 2 && c != r) C[(int64_t)c * ldc + r] = v;
          continue;
        }
      }
      double v;
      if constexpr (SPLIT)
        v = ((double)hi[x][y] + (double)lo[x][y]) + (double)acc[x][y];
      else
        v = (double)acc[x][y];
      v *= alpha;
      if (part) {
        part[((int64_t)blockIdx.z * M + r) * N + c] = v;
      } else {
        if (beta != 0.0) v += beta * (double)C[(int64_t)r * ldc + c];
        C[(int64_t)r * ldc + c] = (TC)v;
        if (mode == 2 && c != r) C[(int64_t)c * ldc + r] = (TC)v;
      }
    }
}

// FP32 partials of the plain FP32 GEMM: summed as a double-float pair, one
// conversion per output.
template <class TC>
__global__ void splitk_reduce_f32_kernel(const float* __restrict__ part, int ksplit, int M,
                                         int N, double beta, TC* __restrict__ C, int64_t ldc,
                                         int mode) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  int r = (int)(idx / N), c = (int)(idx % N);
  if (mode == 1 && c > r) return;
  if (mode == 2 && c < r) return;
  float hi = 0.f, lo = 0.f;
  for (int z = 0; z < ksplit; ++z) two_sum_acc(hi, lo, part[((int64_t)z * M + r) * N + c]);
  TC v;
  if constexpr (sizeof(TC) == 4) {
    float f = hi + lo;
    if (beta != 0.0) f = fmaf((float)beta, C[(int64_t)r * ldc + c], f);
    v = f;
  } else {
    double d = (double)hi + (double)lo;
    if (beta != 0.0) d += beta * (double)C[(int64_t)r * ldc + c];
    v = d;
  }
  C[(int64_t)r * ldc + c] = v;
  if (mode == 2 && c != r) C[(int64_t)c * ldc + r] = v;
}

template <class TC>
__global__ void splitk_reduce_kernel(const double* __restrict__ part, int ksplit, int M, int N,
                                     double beta, TC* __restrict__ C, int64_t ldc, int mode) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  int r = (int)(idx / N), c = (int)(idx % N);
  if (mode == 1 && c > r) return;
  if (mode == 2 && c < r) return;
  double v = 0.0;
  for (int z = 0; z < ksplit; ++z) v += part[((int64_t)z * M + r) * N + c];
  if (beta != 0.0) v += beta * (double)C[(int64_t)r * ldc + c];
  C[(int64_t)r * ldc + c] = (TC)v;
  if (mode == 2 && c != r) C[(int64_t)c * ldc + r] = (TC)v;
}

// ---- Cholesky of one nb x nb diagonal block, plus the inverse of the factor.
// Right-looking elimination with the block in registers: thread (ty, tx)
// owns rows 4ty..4ty+3 x columns 4tx..4tx+3.  At step j the owners of column j
// publish it (unscaled) to a double-buffered shared vector, one barrier, then
// every thread updates its own elements a_ik -= a_ij a_kj / a_jj (j < k <= i)
// and the owners scale column j by 1/sqrt(a_jj).  The factor then goes to
// shared memory for the inverse, which is built row by row.
template <class T>
__global__ void __launch_bounds__(NTH) chol_diag_kernel(T* __restrict__ A, int64_t lda, int nb,
                                                        T* __restrict__ dinv,
                                                        const double* __restrict__ diag0,
                                                        double rel_tol, int* st) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T(*L)[CHOL_NB + 1] = reinterpret_cast<T(*)[CHOL_NB + 1]>(chol_smem);
  T(*Li)[CHOL_NB + 1] = L + CHOL_NB;
  __shared__ T colj[2][CHOL_NB];
  __shared__ T thr[CHOL_NB];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  if (tid == 0) bad = 0;
  // pivot thresholds, converted once (FP64 issues at 1/64 rate on this part)
  if (tid < CHOL_NB) thr[tid] = tid < nb ? (T)(rel_tol * diag0[tid]) : T(0);
  T r[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ty * 4 + a, k = tx * 4 + b;
      T v = T(0);
      if (i < nb && k <= i) v = A[(int64_t)i * lda + k];
      if (i >= nb && i == k) v = T(1);  // pad with identity
      r[a][b] = v;
    }
  for (int j = 0; j < CHOL_NB; ++j) {
    const int buf = j & 1;
    if (tx == (j >> 2)) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T v = r[a][0];
#pragma unroll
        for (int b = 1; b < 4; ++b)
          if ((j & 3) == b) v = r[a][b];
        colj[buf][ty * 4 + a] = v;
      }
    }
    __syncthreads();
    T d = colj[buf][j];
    bool ok = d > thr[j];
    if (!ok) d = T(1);
    if (!ok && tid == 0 && j < nb) bad = 1;
    const T inv_d = recip(d);
    T ci[4], ck[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ci[q] = colj[buf][ty * 4 + q];
      ck[q] = colj[buf][tx * 4 + q];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ty * 4 + a;
      const T lij = ci[a] * inv_d;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int k = tx * 4 + b;
        if (k > j && k <= i) r[a][b] -= lij * ck[b];
      }
    }
    if (tx == (j >> 2)) {
      const T pv = sqrt_fast(d);
      const T ipv = recip(pv);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = ty * 4 + a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if ((j & 3) != b) continue;
          if (i > j) r[a][b] *= ipv;
          if (i == j) r[a][b] = pv;
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ty * 4 + a, k = tx * 4 + b;
      L[i][k] = k <= i ? r[a][b] : T(0);
    }
  __syncthreads();
  if (tid == 0 && bad) set_status(st, VL_ERR_RANK);
  // Li = L^{-1}: row i from rows < i, every column c <= i in parallel:
  // Li[i][c] = (delta_ic - sum_{c <= k < i} L[i][k] Li[k][c]) / L[i][i]
  // 4 threads per column split the k range and combine with shuffles.
  const int col = tid >> 2, part = tid & 3;
  for (int i = 0; i < CHOL_NB; ++i) {
    T sacc = T(0);
    if (col < i) {
      for (int k = col + part; k < i; k += 4) sacc += L[i][k] * Li[k][col];
    }
    sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
    sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
    if (part == 0) {
      const T rdiag = recip(L[i][i]);
      if (col < i)
        Li[i][col] = -sacc * rdiag;
      else if (col == i)
        Li[i][col] = rdiag;
      else
        Li[i][col] = T(0);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < CHOL_NB * CHOL_NB; idx += NTH) {
    int r = idx / CHOL_NB, c = idx % CHOL_NB;
    if (r < nb && c <= r) A[(int64_t)r * lda + c] = L[r][c];
    dinv[idx] = Li[r][c];
  }
}

// ---- Whole Cholesky factorisation in one CTA (FP32, n <= SINGLE_MAX).
// 32-wide blocks; for each block column k0:
//  1. warp 0 factors the 32 x 32 diagonal block in registers (lane r holds
//     row r; the pivot column travels by shuffles) and inverts it;
//  2. all warps form the panel L[i, k0:k0+32] = A[i, k0:k0+32] Linv^T for the
//     rows below, kept in shared memory and written back;
//  3. all warps update the trailing lower triangle in 32 x 32 tiles,
//     A[i, j] -= sum_q P[i, q] P[j, q] (read-modify-write, L2 resident).
// Finally the inverses of consecutive 32-blocks are combined into the 64 x 64
// diagonal-block inverses the blocked solves use:
//     [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}].
constexpr int SB = 32;
constexpr int SBP = SB + 4;  // panel row stride in shared memory (16-byte aligned rows)
constexpr int SINGLE_MAX = 512;
constexpr int STH = 512;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// prof (optional, NULL in the library): three globaltimer stamps per block
// column (after the diagonal block, the panel and the trailing update).
__global__ void __launch_bounds__(STH) chol_single_kernel(float* __restrict__ A, int64_t lda,
                                                          int n, float* __restrict__ dinv,
                                                          const double* __restrict__ diag0,
                                                          float rel_tol, int* st,
                                                          unsigned long long* prof = nullptr) {
  extern __shared__ __align__(16) float cs_smem[];
  const int nblk = (n + SB - 1) / SB;
  float* P = cs_smem;                      // [max(n, SB)][SBP] panel; rows 0..31 also
                                           // stage the diagonal tile
  float* Li = P + (size_t)max(n, SB) * SBP;  // [nblk][SB][SB + 1] block inverses
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned full = 0xffffffffu;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int b = 0; b < nblk; ++b) {
    const int k0 = b * SB;
    const int nb = min(SB, n - k0);
    float* Lib = Li + (size_t)b * SB * (SB + 1);
    if (warp == 0) {
      {  // stage the tile through shared memory: coalesced rows, all in flight
        float rowv[SB];
#pragma unroll
        for (int r = 0; r < SB; ++r)
          rowv[r] = (r < nb && lane <= r) ? A[(int64_t)(k0 + r) * lda + k0 + lane] : 0.f;
#pragma unroll
        for (int r = 0; r < SB; ++r) P[(size_t)r * SBP + lane] = rowv[r];
      }
      __syncwarp();
      float a[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        float v = (c == lane) ? 1.f : 0.f;  // identity padding
        if (lane < nb && c < nb && c <= lane) v = P[(size_t)lane * SBP + c];
        a[c] = v;
      }
      const float thr = lane < nb ? (float)(rel_tol * diag0[k0 + lane]) : 0.f;
      bool lbad = false;
#pragma unroll
      for (int j = 0; j < SB; ++j) {
        float d = __shfl_sync(full, a[j], j);
        const float tj = __shfl_sync(full, thr, j);
        if (!(d > tj)) {
          lbad |= (j < nb);
          d = 1.f;
        }
        const float ipiv = rsqrtf(d);  // one MUFU op: 1/sqrt(d), then 1/d and sqrt(d)
        const float inv = ipiv * ipiv;
        const float piv = d * ipiv;
        const float lrj = a[j];  // (lane, j), not yet scaled
#pragma unroll
        for (int c = j + 1; c < SB; ++c) {
          const float lcj = __shfl_sync(full, a[j], c);  // (c, j)
          a[c] -= lrj * lcj * inv;
        }
        a[j] = (lane == j) ? piv : (lane > j ? lrj * ipiv : 0.f);
      }
      if (lbad) bad = 1;
      // inverse of the block: lane r builds row r of Linv, rows in order
      float li[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) li[c] = 0.f;
#pragma unroll
      for (int k = 0; k < SB; ++k) {
        const float rd = recip(__shfl_sync(full, a[k], k));
#pragma unroll
        for (int c = 0; c <= k; ++c)
          if (lane == k) li[c] = ((c == k ? 1.f : 0.f) - li[c]) * rd;
#pragma unroll
        for (int c = 0; c <= k; ++c) {
          const float v = __shfl_sync(full, li[c], k);
          if (lane > k) li[c] += a[k] * v;
        }
      }
      __syncwarp();
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        Lib[lane * (SB + 1) + c] = c <= lane ? li[c] : 0.f;
        P[(size_t)lane * SBP + c] = a[c];
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < SB; ++r)  // write the factor back, coalesced
        if (r < nb && lane <= r) A[(int64_t)(k0 + r) * lda + k0 + lane] = P[(size_t)r * SBP + lane];
    }
    __syncthreads();
    if (prof && tid == 0) prof[3 * b] = gtimer();
    // panel rows below the block: P[i][c] = sum_{q <= c} A[i][k0+q] Linv[c][q]
    const int r0 = k0 + SB;
    for (int i0 = r0 + 4 * warp; i0 < n; i0 += 4 * (STH / 32)) {  // four rows per warp
      float av[4], pv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = (lane < nb && i0 + u < n) ? A[(int64_t)(i0 + u) * lda + k0 + lane] : 0.f;
        pv[u] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        const float l = Lib[lane * (SB + 1) + q];
#pragma unroll
        for (int u = 0; u < 4; ++u) pv[u] = fmaf(__shfl_sync(full, av[u], q), l, pv[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i0 + u >= n) continue;
        P[(size_t)(i0 + u) * SBP + lane] = pv[u];
        if (lane < nb) A[(int64_t)(i0 + u) * lda + k0 + lane] = pv[u];
      }
    }
    __syncthreads();
    if (prof && tid == 0) prof[3 * b + 1] = gtimer();
    // trailing update, lower triangle, 32 x 32 tiles over rows/cols >= r0
    const int nt = (n - r0 + SB - 1) / SB;
    const int ntiles = nt * (nt + 1) / 2;
    for (int t = warp; t < ntiles; t += STH / 32) {
      int I = 0, rem = t;  // tile (I, J), J <= I, row-major over the triangle
      while (rem > I) {
        rem -= I + 1;
        ++I;
      }
      const int J = rem;
      const int j = r0 + J * SB + lane;
      float pj[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q) pj[q] = j < n ? P[(size_t)j * SBP + q] : 0.f;
      const int ibeg = r0 + I * SB;
      const int iend = min(n, ibeg + SB);
      for (int i = ibeg; i < iend; i += 4) {  // four independent rows at a time
        float old[4];  // issued before the FMAs so their latency overlaps them
#pragma unroll
        for (int u = 0; u < 4; ++u)
          old[u] = (i + u < iend && j < n && j <= i + u) ? A[(int64_t)(i + u) * lda + j] : 0.f;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* prow[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) prow[u] = P + (size_t)min(i + u, n - 1) * SBP;
#pragma unroll
        for (int q = 0; q < SB; q += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 v = *reinterpret_cast<const float4*>(prow[u] + q);  // broadcast
            acc[u] = fmaf(v.x, pj[q], acc[u]);
            acc[u] = fmaf(v.y, pj[q + 1], acc[u]);
            acc[u] = fmaf(v.z, pj[q + 2], acc[u]);
            acc[u] = fmaf(v.w, pj[q + 3], acc[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i + u < iend && j < n && j <= i + u) A[(int64_t)(i + u) * lda + j] = old[u] - acc[u];
      }
    }
    __syncthreads();
    if (prof && tid == 0) prof[3 * b + 2] = gtimer();
  }
  if (tid == 0 && bad) set_status(st, VL_ERR_RANK);
  // 64 x 64 diagonal-block inverses for the blocked solves
  const int nb64 = (n + CHOL_NB - 1) / CHOL_NB;
  for (int b = warp; b < nb64; b += STH / 32) {
    float* out = dinv + (size_t)b * CHOL_NB * CHOL_NB;
    const int b0 = 2 * b, b1 = 2 * b + 1;
    const float* Ai = Li + (size_t)b0 * SB * (SB + 1);
    const bool has1 = b1 < nblk;
    const float* Ci = has1 ? Li + (size_t)b1 * SB * (SB + 1) : nullptr;
    // row `lane` of each quadrant
    for (int c = 0; c < SB; ++c) {
      out[lane * CHOL_NB + c] = Ai[lane * (SB + 1) + c];                 // A^{-1}
      out[lane * CHOL_NB + SB + c] = 0.f;                                // 0
      out[(SB + lane) * CHOL_NB + SB + c] =
          has1 ? Ci[lane * (SB + 1) + c] : (c == lane ? 1.f : 0.f);      // C^{-1}
    }
    // X = -C^{-1} (B A^{-1}), B[r][q] = L[k0 + 32 + r][k0 + q]
    float tmp[SB];
    const int k0 = b0 * SB;
#pragma unroll
    for (int c = 0; c < SB; ++c) tmp[c] = 0.f;
    if (has1) {
      const int r = k0 + SB + lane;  // row of B held by this lane
      for (int q = 0; q < SB; ++q) {
        const float bq = r < n ? A[(int64_t)r * lda + k0 + q] : 0.f;
#pragma unroll
        for (int c = 0; c < SB; ++c) tmp[c] += bq * Ai[q * (SB + 1) + c];
      }
    }
    // out row (32 + lane): -sum_r Ci[lane][r] tmp_r[c], tmp_r is lane r's tmp
#pragma unroll
    for (int c = 0; c < SB; ++c) {
      float x = 0.f;
      for (int r = 0; r < SB; ++r) {
        const float t = __shfl_sync(full, tmp[c], r);
        x += (has1 ? Ci[lane * (SB + 1) + r] : 0.f) * t;
      }
      out[(SB + lane) * CHOL_NB + c] = -x;
    }
  }
}

size_t chol_single_smem(int n) {
  const int nblk = (n + SB - 1) / SB;
  return sizeof(float) * ((size_t)std::max(n, SB) * SBP + (size_t)nblk * SB * (SB + 1));
}

// ---- Column-parallel blocked triangular solves.  Each CTA owns SC
// right-hand-side columns and sweeps all block rows: forward
//     Y_b = Linv_bb (R_b - L_{b,<b} Y_{<b}),
// then (optionally) backward
//     X_b = Linv_bb^T (Y_b - L_{>b,b}^T X_{>b}),
// streaming 64 x 64 pieces of L (and the matching rows of R) through shared
// memory with cp.async, double-buffered so a piece loads while the previous
// one is consumed.  Results overwrite R.
constexpr int SC = 8;
constexpr int LSW = CHOL_NB + 1;  // padded row of a shared L piece

template <class T>
__device__ __forceinline__ void cp_async_el(T* smem, const T* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <class T>
__global__ void __launch_bounds__(NTH) trsm_cols_kernel(const T* __restrict__ L, int64_t lda,
                                                        const T* __restrict__ dinv, int n,
                                                        T* __restrict__ R, int64_t ldr, int nrhs,
                                                        int backward) {
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  T* Lbuf = reinterpret_cast<T*>(trsm_smem);          // [2][64][LSW]
  T* Dbuf = Lbuf + 2 * CHOL_NB * LSW;                  // [64][LSW]  inverse block
  T* Ybuf = Dbuf + CHOL_NB * LSW;                      // [2][64][SC]
  T* Acc = Ybuf + 2 * CHOL_NB * SC;                    // [64][SC]
  const int tid = threadIdx.x;
  const int r = tid >> 2;        // row within the block, 0..63
  const int cc = (tid & 3) * 2;  // two columns per thread
  const int c0 = blockIdx.x * SC;
  const int nblk = (n + CHOL_NB - 1) / CHOL_NB;
  for (int pass = 0; pass < (backward ? 2 : 1); ++pass) {
    for (int bi = 0; bi < nblk; ++bi) {
      const int b = pass == 0 ? bi : nblk - 1 - bi;
      const int k0 = b * CHOL_NB;
      const int nb = min(CHOL_NB, n - k0);
      const int jb = pass == 0 ? 0 : k0 + nb;  // forward 0..k0, backward k0+nb..n
      const int je = pass == 0 ? k0 : n;
      const int nch = (je - jb + CHOL_NB - 1) / CHOL_NB;
      // issue piece c into buffer c & 1 (zero outside the matrix)
      auto issue = [&](int c) {
        const int j0 = jb + c * CHOL_NB;
        const int jn = min(CHOL_NB, je - j0);
        T* Ls = Lbuf + (c & 1) * CHOL_NB * LSW;
        T* Ys = Ybuf + (c & 1) * CHOL_NB * SC;
        for (int idx = tid; idx < CHOL_NB * CHOL_NB; idx += NTH) {
          const int a = idx / CHOL_NB, bc = idx % CHOL_NB;
          if (pass == 0) {  // Ls[a][bc] = L[k0 + a][j0 + bc]
            if (a < nb && bc < jn)
              cp_async_el(&Ls[a * LSW + bc], &L[(int64_t)(k0 + a) * lda + j0 + bc]);
            else
              Ls[a * LSW + bc] = T(0);
          } else {  // Ls[bc][a] = L[j0 + a][k0 + bc]  (transposed slab)
            if (a < jn && bc < nb)
              cp_async_el(&Ls[bc * LSW + a], &L[(int64_t)(j0 + a) * lda + k0 + bc]);
            else
              Ls[bc * LSW + a] = T(0);
          }
        }
        for (int idx = tid; idx < CHOL_NB * SC; idx += NTH) {
          const int a = idx / SC, c = idx % SC;
          if (a < jn && c0 + c < nrhs)
            cp_async_el(&Ys[a * SC + c], &R[(int64_t)(j0 + a) * ldr + c0 + c]);
          else
            Ys[a * SC + c] = T(0);
        }
      };
      // the inverse of the diagonal block (transposed for the backward pass)
      // travels with the first piece
      for (int idx = tid; idx < CHOL_NB * CHOL_NB; idx += NTH) {
        const int a = idx / CHOL_NB, bc = idx % CHOL_NB;
        T* dst = pass == 0 ? &Dbuf[a * LSW + bc] : &Dbuf[bc * LSW + a];
        cp_async_el(dst, &dinv[(int64_t)b * CHOL_NB * CHOL_NB + idx]);
      }
      T acc[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int col = c0 + cc + q;
        acc[q] = (r < nb && col < nrhs) ? R[(int64_t)(k0 + r) * ldr + col] : T(0);
      }
      if (nch > 0) issue(0);
      cp_commit();
      for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
          issue(c + 1);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncthreads();
        const T* Ls = Lbuf + (c & 1) * CHOL_NB * LSW;
        const T* Ys = Ybuf + (c & 1) * CHOL_NB * SC;
#pragma unroll 8
        for (int jj = 0; jj < CHOL_NB; ++jj) {
          const T l = Ls[r * LSW + jj];
          acc[0] -= l * Ys[jj * SC + cc];
          acc[1] -= l * Ys[jj * SC + cc + 1];
        }
        __syncthreads();
      }
      cp_wait<0>();
      Acc[r * SC + cc] = acc[0];
      Acc[r * SC + cc + 1] = acc[1];
      __syncthreads();
      T o0 = T(0), o1 = T(0);
#pragma unroll 8
      for (int q = 0; q < CHOL_NB; ++q) {
        const T l = Dbuf[r * LSW + q];
        o0 += l * Acc[q * SC + cc];
        o1 += l * Acc[q * SC + cc + 1];
      }
      if (r < nb) {
        if (c0 + cc < nrhs) R[(int64_t)(k0 + r) * ldr + c0 + cc] = o0;
        if (c0 + cc + 1 < nrhs) R[(int64_t)(k0 + r) * ldr + c0 + cc + 1] = o1;
      }
      __syncthreads();
    }
  }
}

template <class T>
size_t trsm_smem_bytes() {
  return sizeof(T) * (3 * CHOL_NB * LSW + 3 * CHOL_NB * SC);
}

template <class TI, class TO>
__global__ void convert_kernel(const TI* __restrict__ in, int64_t ldi, TO* __restrict__ out,
                               int64_t ldo, int rows, int cols) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int r = (int)(idx / cols), c = (int)(idx % cols);
  out[(int64_t)r * ldo + c] = (TO)in[(int64_t)r * ldi + c];
}

template <class T>
__global__ void save_diag_kernel(const T* __restrict__ A, int64_t lda, int n,
                                 double* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (double)A[(int64_t)i * lda + i];
}

template <class T>
__global__ void set_identity_kernel(T* A, int64_t lda, int n) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int r = (int)(idx / n), c = (int)(idx % n);
  A[(int64_t)r * lda + c] = (r == c) ? T(1) : T(0);
}

// Split-K factor: about two CTAs per SM, FP32 slices of at most max_chunk
// steps of k (the FP64 reduction of the slices bounds the accumulation error).
int pick_ksplit(int tiles, int K, int num_sms, int max_chunk) {
  int want = std::max(1, 2 * num_sms / std::max(tiles, 1));
  int need = (K + max_chunk - 1) / max_chunk;
  int ks = std::max(want, need);
  ks = std::min(ks, std::max(1, K / 64));
  return std::min(ks, 64);
}

template <class T, class TC, int TMt, int TNt, bool SPLIT>
void gemm_launch(const Ctx& cx, int M, int N, int K, double alpha, View<T> A, View<T> Al,
                 View<T> B, View<T> Bl, double beta, TC* C, int64_t ldc, int mode,
                 int max_chunk) {
  if (M <= 0 || N <= 0) return;
  constexpr int BM = 16 * TMt, BN = 16 * TNt;
  const int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  int tiles = gm * gn;
  if (mode != 0) tiles = (tiles + std::min(gm, gn)) / 2;
  int ks = pick_ksplit(tiles, K, cx.num_sms, max_chunk);
  if (ks > 1 && (!cx.part || (size_t)ks * M * N > cx.part_cap))
    ks = cx.part ? std::max(1, (int)std::min<size_t>(ks, cx.part_cap / ((size_t)M * N))) : 1;
  int kchunk = ks > 1 ? (((K + ks - 1) / ks + 31) / 32) * 32 : std::max(K, 1);
  ks = ks > 1 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid(gn, gm, ks);
  note_launch();
  gemm_kernel<T, TC, TMt, TNt, SPLIT><<<grid, NTH, 0, cx.s>>>(
      M, N, K, kchunk, alpha, A, Al, B, Bl, beta, C, ldc, mode, ks > 1 ? cx.part : nullptr);
  if (ks > 1) {
    int64_t tot = (int64_t)M * N;
    note_launch();
    if constexpr (!SPLIT && sizeof(T) == 4)
      splitk_reduce_f32_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, cx.s>>>(
          reinterpret_cast<const float*>(cx.part), ks, M, N, beta, C, ldc, mode);
    else
      splitk_reduce_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, cx.s>>>(
          cx.part, ks, M, N, beta, C, ldc, mode);
  }
}

// Padded work of an M x N product in BM x BN tiles (relative to M N).
double tile_waste(int M, int N, int BM, int BN) {
  const double gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  return gm * BM * gn * BN / ((double)M * N);
}

}  // namespace

size_t gemm_part_need(int M, int N, int K) {
  (void)K;
  return (size_t)64 * M * N;
}

template <class T, class TC>
void launch_gemm(const Ctx& cx, int M, int N, int K, double alpha, View<T> A, View<T> B,
                 double beta, TC* C, int64_t ldc, bool lower_only) {
  const int mode = lower_only ? 1 : 0;
  if constexpr (sizeof(T) == 4) {
    // largest micro-tile whose padded work stays within 10% of the best
    if ((int64_t)M * N >= 256 * 256) {
      const double w8 = tile_waste(M, N, 128, 128), w5 = tile_waste(M, N, 80, 80);
      const double w4 = tile_waste(M, N, 64, 64);
      if (w8 <= 1.1 * std::min(w5, w4))
        gemm_launch<T, TC, 8, 8, false>(cx, M, N, K, alpha, A, A, B, B, beta, C, ldc, mode, 512);
      else if (w5 <= 1.1 * w4)
        gemm_launch<T, TC, 5, 5, false>(cx, M, N, K, alpha, A, A, B, B, beta, C, ldc, mode, 512);
      else
        gemm_launch<T, TC, 4, 4, false>(cx, M, N, K, alpha, A, A, B, B, beta, C, ldc, mode, 512);
    } else {
      gemm_launch<T, TC, 4, 4, false>(cx, M, N, K, alpha, A, A, B, B, beta, C, ldc, mode, 512);
    }
  } else {
    gemm_launch<T, TC, 4, 4, false>(cx, M, N, K, alpha, A, A, B, B, beta, C, ldc, mode,
                                    1 << 30);
  }
}
template void launch_gemm<float, float>(const Ctx&, int, int, int, double, View<float>,
                                        View<float>, double, float*, int64_t, bool);
template void launch_gemm<float, double>(const Ctx&, int, int, int, double, View<float>,
                                         View<float>, double, double*, int64_t, bool);
template void launch_gemm<double, double>(const Ctx&, int, int, int, double, View<double>,
                                          View<double>, double, double*, int64_t, bool);

void launch_gemm_split(const Ctx& cx, int M, int N, int K, View<float> Ahi, View<float> Alo,
                       View<float> Bhi, View<float> Blo, double* C, int64_t ldc,
                       bool upper_only) {
  // a 32 x 32 tile when the whole product fits one: a 64 x 64 tile would
  // spend three quarters of its arithmetic on padding
  if (std::max(M, N) <= 32)
    gemm_launch<float, double, 2, 2, true>(cx, M, N, K, 1.0, Ahi, Alo, Bhi, Blo, 0.0, C, ldc,
                                           upper_only ? 2 : 0, 1 << 30);
  else
    gemm_launch<float, double, 4, 4, true>(cx, M, N, K, 1.0, Ahi, Alo, Bhi, Blo, 0.0, C, ldc,
                                           upper_only ? 2 : 0, 1 << 30);
}

template <class T>
void chol_blocked(const Ctx& cx, T* A, int64_t lda, int n, T* dinv, double* diag0,
                  double pivot_floor) {
  const int NB = CHOL_NB;
  cudaStream_t s = cx.s;
  const double rel_tol = pivot_floor > 0 ? pivot_floor : (sizeof(T) == 4 ? 1e-6 : 1e-12);
  if constexpr (sizeof(T) == 4) {
    if (n <= SINGLE_MAX) {
      const size_t smem1 = chol_single_smem(SINGLE_MAX);
      static bool attr1 = false;
      if (!attr1) {
        cudaFuncSetAttribute(chol_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem1);
        attr1 = true;
      }
      note_launch();
      save_diag_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(A, lda, n, diag0);
      if (launch_chol_cluster(A, lda, n, dinv, diag0, (float)rel_tol, cx.st, s)) return;
      note_launch();
      chol_single_kernel<<<1, STH, chol_single_smem(n), s>>>(A, lda, n, dinv, diag0,
                                                            (float)rel_tol, cx.st);
      return;
    }
  }
  const size_t smem = 2 * CHOL_NB * (CHOL_NB + 1) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  note_launch();
  save_diag_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(A, lda, n, diag0);
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = std::min(NB, n - k0);
    T* dblk = dinv + (int64_t)(k0 / NB) * NB * NB;
    note_launch();
    chol_diag_kernel<T><<<1, NTH, smem, s>>>(A + (int64_t)k0 * lda + k0, lda, nb, dblk,
                                             diag0 + k0, rel_tol, cx.st);
    const int rest = n - k0 - nb;
    if (rest <= 0) break;
    // panel: L[i, k0:k0+nb] = A[i, k0:k0+nb] * Linv_kk^T
    View<T> Ap{A + (int64_t)(k0 + nb) * lda + k0, lda, 1};
    View<T> Bi{dblk, NB, 1};
    launch_gemm<T, T>(cx, rest, nb, nb, 1.0, Ap, Bi, 0.0, A + (int64_t)(k0 + nb) * lda + k0,
                      lda, false);
    // trailing update (lower triangle): A22 -= L21 L21^T
    View<T> L21{A + (int64_t)(k0 + nb) * lda + k0, lda, 1};
    launch_gemm<T, T>(cx, rest, rest, nb, -1.0, L21, L21, 1.0,
                      A + (int64_t)(k0 + nb) * (lda + 1), lda, true);
  }
}
template void chol_blocked<float>(const Ctx&, float*, int64_t, int, float*, double*, double);
template void chol_blocked<double>(const Ctx&, double*, int64_t, int, double*, double*, double);

template <class T>
void chol_solve_blocked(const Ctx& cx, const T* L, int64_t lda, const T* dinv, int n, T* R,
                        int64_t ldr, int nrhs, bool backward) {
  if (launch_trsm_ring<T>(L, lda, dinv, n, R, ldr, nrhs, backward, cx.s)) return;
  const size_t smem = trsm_smem_bytes<T>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(trsm_cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  note_launch();
  trsm_cols_kernel<T><<<(nrhs + SC - 1) / SC, NTH, smem, cx.s>>>(L, lda, dinv, n, R, ldr, nrhs,
                                                                 backward ? 1 : 0);
}
template void chol_solve_blocked<float>(const Ctx&, const float*, int64_t, const float*, int,
                                        float*, int64_t, int, bool);
template void chol_solve_blocked<double>(const Ctx&, const double*, int64_t, const double*, int,
                                         double*, int64_t, int, bool);

template <class TI, class TO>
void launch_convert(const TI* in, int64_t ldi, TO* out, int64_t ldo, int rows, int cols,
                    cudaStream_t s) {
  int64_t tot = (int64_t)rows * cols;
  if (tot <= 0) return;
  note_launch();
  convert_kernel<TI, TO><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(in, ldi, out, ldo, rows,
                                                                      cols);
}
template void launch_convert<double, float>(const double*, int64_t, float*, int64_t, int, int,
                                            cudaStream_t);
template void launch_convert<float, double>(const float*, int64_t, double*, int64_t, int, int,
                                            cudaStream_t);
template void launch_convert<double, double>(const double*, int64_t, double*, int64_t, int, int,
                                             cudaStream_t);

template <class T>
void launch_set_identity(T* A, int64_t lda, int n, cudaStream_t s) {
  int64_t tot = (int64_t)n * n;
  note_launch();
  set_identity_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, lda, n);
}
template void launch_set_identity<float>(float*, int64_t, int, cudaStream_t);
template void launch_set_identity<double>(double*, int64_t, int, cudaStream_t);

}  // namespace vl
