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

constexpr int TM = 64, TN = 64, KC = 16, NTH = 256;
constexpr int kFlush = 256;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

template <class T>
__device__ __forceinline__ void load_tile(T (*sm)[TM + 4], View<T> v, int r0, int rows, int k0,
                                          int kmax) {
  // sm[k][r] = v(r0 + r, k0 + k), zero outside.
  if (v.ks == 1) {
    for (int idx = threadIdx.x; idx < TM * KC; idx += NTH) {
      int r = idx / KC, k = idx % KC;
      int gr = r0 + r, gk = k0 + k;
      sm[k][r] = (gr < rows && gk < kmax) ? v.base[(int64_t)gr * v.rs + gk] : T(0);
    }
  } else {
    for (int idx = threadIdx.x; idx < TM * KC; idx += NTH) {
      int r = idx % TM, k = idx / TM;
      int gr = r0 + r, gk = k0 + k;
      sm[k][r] = (gr < rows && gk < kmax) ? v.base[(int64_t)gr * v.rs + (int64_t)gk * v.ks]
                                          : T(0);
    }
  }
}

// mode: 0 = full, 1 = lower (c <= r), 2 = upper (c >= r, mirrored into C[c, r])
template <class T, class TC>
__global__ void __launch_bounds__(NTH) gemm_kernel(int M, int N, int K, int kchunk,
                                                   double alpha, View<T> A, View<T> B,
                                                   double beta, TC* __restrict__ C,
                                                   int64_t ldc, int mode,
                                                   double* __restrict__ part) {
  const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
  if (mode == 1 && c0 > r0 + TM - 1) return;
  if (mode == 2 && r0 > c0 + TN - 1) return;
  __shared__ __align__(16) T As[KC][TM + 4];
  __shared__ __align__(16) T Bs[KC][TN + 4];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  T acc[4][4];
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = T(0);
      hi[a][b] = 0.f;
      lo[a][b] = 0.f;
    }
  int since_flush = 0;
  for (int k0 = kbeg; k0 < kend; k0 += KC) {
    load_tile<T>(As, A, r0, M, k0, kend);
    load_tile<T>(Bs, B, c0, N, k0, kend);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      since_flush += KC;
      if (since_flush >= kFlush) {
        since_flush = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            two_sum_acc(hi[x][y], lo[x][y], (float)acc[x][y]);
            acc[x][y] = T(0);
          }
      }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int r = r0 + ty * 4 + x, c = c0 + tx * 4 + y;
      if (r >= M || c >= N) continue;
      if (mode == 1 && c > r) continue;
      if (mode == 2 && c < r) continue;
      double v;
      if constexpr (sizeof(T) == 4)
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

// Compensated covariance product: (Ahi + Alo)(Bhi + Blo)^T ~ Ahi Bhi + Ahi Blo
// + Alo Bhi, FP32 FMAs flushed every 32 steps into a double-float accumulator.
__global__ void __launch_bounds__(NTH) gemm_split_kernel(int M, int N, int K, int kchunk,
                                                         View<float> Ah, View<float> Al,
                                                         View<float> Bh, View<float> Bl,
                                                         double* __restrict__ C, int64_t ldc,
                                                         int mode, double* __restrict__ part) {
  const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
  if (mode == 2 && r0 > c0 + TN - 1) return;
  __shared__ __align__(16) float Ahs[KC][TM + 4], Als[KC][TM + 4];
  __shared__ __align__(16) float Bhs[KC][TN + 4], Bls[KC][TN + 4];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  float acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = hi[a][b] = lo[a][b] = 0.f;
  int since = 0;
  for (int k0 = kbeg; k0 < kend; k0 += KC) {
    load_tile<float>(Ahs, Ah, r0, M, k0, kend);
    load_tile<float>(Als, Al, r0, M, k0, kend);
    load_tile<float>(Bhs, Bh, c0, N, k0, kend);
    load_tile<float>(Bls, Bl, c0, N, k0, kend);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[q] = Ahs[kk][ty * 4 + q];
        al[q] = Als[kk][ty * 4 + q];
        bh[q] = Bhs[kk][tx * 4 + q];
        bl[q] = Bls[kk][tx * 4 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          float t = fmaf(ah[x], bl[y], al[x] * bh[y]);
          acc[x][y] = fmaf(ah[x], bh[y], acc[x][y] + t);
        }
    }
    __syncthreads();
    since += KC;
    if (since >= 32) {
      since = 0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          two_sum_acc(hi[x][y], lo[x][y], acc[x][y]);
          acc[x][y] = 0.f;
        }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int r = r0 + ty * 4 + x, c = c0 + tx * 4 + y;
      if (r >= M || c >= N) continue;
      if (mode == 2 && c < r) continue;
      double v = ((double)hi[x][y] + (double)lo[x][y]) + (double)acc[x][y];
      if (part) {
        part[((int64_t)blockIdx.z * M + r) * N + c] = v;
      } else {
        C[(int64_t)r * ldc + c] = v;
        if (mode == 2 && c != r) C[(int64_t)c * ldc + r] = v;
      }
    }
}

// ---- Cholesky of one nb x nb diagonal block in shared memory, plus the
// inverse of the factor.
// A pivot below rel_tol times the matrix's original diagonal entry marks the
// system as (numerically) singular.
template <class T>
__global__ void __launch_bounds__(NTH) chol_diag_kernel(T* __restrict__ A, int64_t lda, int nb,
                                                        T* __restrict__ dinv,
                                                        const double* __restrict__ diag0,
                                                        double rel_tol, int* st) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T(*L)[CHOL_NB + 1] = reinterpret_cast<T(*)[CHOL_NB + 1]>(chol_smem);
  T(*Li)[CHOL_NB + 1] = L + CHOL_NB;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int idx = threadIdx.x; idx < CHOL_NB * CHOL_NB; idx += NTH) {
    int r = idx / CHOL_NB, c = idx % CHOL_NB;
    T v = T(0);
    if (r < nb && c <= r) v = A[(int64_t)r * lda + c];
    if (r >= nb && r == c) v = T(1);  // pad with identity
    L[r][c] = v;
    Li[r][c] = T(0);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      T d = L[j][j];
      if (!((double)d > rel_tol * diag0[j])) {
        bad = 1;
        d = T(1);
      }
      L[j][j] = sqrt(d);
    }
    __syncthreads();
    const T dj = L[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += NTH) L[i][j] /= dj;
    __syncthreads();
    // trailing update of the lower triangle (i >= k > j)
    const int w = nb - j - 1;
    for (int idx = threadIdx.x; idx < w * w; idx += NTH) {
      int i = j + 1 + idx / w, k = j + 1 + idx % w;
      if (k <= i) L[i][k] -= L[i][j] * L[k][j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) set_status(st, VL_ERR_RANK);
  // inverse of the lower-triangular factor: column c of L^{-1} by forward
  // substitution, one thread per column
  for (int c = threadIdx.x; c < CHOL_NB; c += NTH) {
    for (int i = 0; i < CHOL_NB; ++i) {
      T s = (i == c) ? T(1) : T(0);
      for (int k = c; k < i; ++k) s -= L[i][k] * Li[k][c];
      Li[i][c] = (i >= c) ? s / L[i][i] : T(0);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CHOL_NB * CHOL_NB; idx += NTH) {
    int r = idx / CHOL_NB, c = idx % CHOL_NB;
    if (r < nb && c <= r) A[(int64_t)r * lda + c] = L[r][c];
    dinv[idx] = Li[r][c];
  }
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

int pick_ksplit(int M, int N, int K, int mode, int num_sms) {
  int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  if (mode != 0) tiles = (tiles + ((M + TM - 1) / TM)) / 2;
  int want = std::max(1, 2 * num_sms / std::max(tiles, 1));
  int maxk = std::max(1, K / 512);
  return std::min(std::min(want, maxk), 16);
}

}  // namespace

size_t gemm_part_need(int M, int N, int K) {
  (void)K;
  return (size_t)16 * M * N;
}

template <class T, class TC>
void launch_gemm(const Ctx& cx, int M, int N, int K, double alpha, View<T> A, View<T> B,
                 double beta, TC* C, int64_t ldc, bool lower_only) {
  if (M <= 0 || N <= 0) return;
  cudaStream_t s = cx.s;
  const int mode = lower_only ? 1 : 0;
  int ks = pick_ksplit(M, N, K, mode, cx.num_sms);
  double* part = nullptr;
  if (ks > 1) {
    if ((size_t)ks * M * N <= cx.part_cap && cx.part)
      part = cx.part;
    else
      ks = 1;
  }
  int kchunk = ks > 1 ? (((K + ks - 1) / ks + KC - 1) / KC) * KC : std::max(K, 1);
  ks = ks > 1 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, ks);
  note_launch();
  gemm_kernel<T, TC><<<grid, NTH, 0, s>>>(M, N, K, kchunk, alpha, A, B, beta, C, ldc, mode,
                                          ks > 1 ? part : nullptr);
  if (ks > 1) {
    int64_t tot = (int64_t)M * N;
    note_launch();
    splitk_reduce_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, ks, M, N, beta,
                                                                          C, ldc, mode);
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
  cudaStream_t s = cx.s;
  const int mode = upper_only ? 2 : 0;
  int ks = pick_ksplit(M, N, K, mode, cx.num_sms);
  double* part = nullptr;
  if (ks > 1) {
    if ((size_t)ks * M * N <= cx.part_cap && cx.part)
      part = cx.part;
    else
      ks = 1;
  }
  int kchunk = ks > 1 ? (((K + ks - 1) / ks + 31) / 32) * 32 : std::max(K, 1);
  ks = ks > 1 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, ks);
  note_launch();
  gemm_split_kernel<<<grid, NTH, 0, s>>>(M, N, K, kchunk, Ahi, Alo, Bhi, Blo, C, ldc, mode,
                                         ks > 1 ? part : nullptr);
  if (ks > 1) {
    int64_t tot = (int64_t)M * N;
    note_launch();
    splitk_reduce_kernel<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        part, ks, M, N, 0.0, C, ldc, mode);
  }
}

template <class T>
void chol_blocked(const Ctx& cx, T* A, int64_t lda, int n, T* dinv, double* diag0) {
  const int NB = CHOL_NB;
  cudaStream_t s = cx.s;
  const size_t smem = 2 * CHOL_NB * (CHOL_NB + 1) * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(chol_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  const double rel_tol = sizeof(T) == 4 ? 1e-6 : 1e-12;
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
template void chol_blocked<float>(const Ctx&, float*, int64_t, int, float*, double*);
template void chol_blocked<double>(const Ctx&, double*, int64_t, int, double*, double*);

template <class T>
void chol_solve_blocked(const Ctx& cx, const T* L, int64_t lda, const T* dinv, int n, T* R,
                        int64_t ldr, int nrhs, bool backward) {
  const int NB = CHOL_NB;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = std::min(NB, n - k0);
    if (k0 > 0) {
      View<T> Lr{L + (int64_t)k0 * lda, lda, 1};
      View<T> Y{R, 1, ldr};
      launch_gemm<T, T>(cx, nb, nrhs, k0, -1.0, Lr, Y, 1.0, R + (int64_t)k0 * ldr, ldr, false);
    }
    View<T> Di{dinv + (int64_t)(k0 / NB) * NB * NB, NB, 1};
    View<T> Rk{R + (int64_t)k0 * ldr, 1, ldr};
    launch_gemm<T, T>(cx, nb, nrhs, nb, 1.0, Di, Rk, 0.0, R + (int64_t)k0 * ldr, ldr, false);
  }
  if (!backward) return;
  const int nblk = (n + NB - 1) / NB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * NB;
    const int nb = std::min(NB, n - k0);
    const int rest = n - k0 - nb;
    if (rest > 0) {
      View<T> Lt{L + (int64_t)(k0 + nb) * lda + k0, 1, lda};
      View<T> X{R + (int64_t)(k0 + nb) * ldr, 1, ldr};
      launch_gemm<T, T>(cx, nb, nrhs, rest, -1.0, Lt, X, 1.0, R + (int64_t)k0 * ldr, ldr, false);
    }
    View<T> DiT{dinv + (int64_t)b * NB * NB, 1, NB};
    View<T> Rk{R + (int64_t)k0 * ldr, 1, ldr};
    launch_gemm<T, T>(cx, nb, nrhs, nb, 1.0, DiT, Rk, 0.0, R + (int64_t)k0 * ldr, ldr, false);
  }
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
