// Per-variable statistics and data layout kernels.
//
//  * var_prep     : full-series mean of each variable, the centred copy the VAR
//                   Gram reads, and the mean of every lag window (Sec. 4.1;
//                   the VAR intercept is equivalent to centring each window).
//  * standardize  : mean, 1/std (population) and the two entropy moments of
//                   each standardized variable (Sec. 3 step 1; Sec. 4.2 item 1
//                   precomputes H(x_i) once).
//  * split_center : centred residuals as an FP32 hi/lo pair for the
//                   compensated covariance product.
//  * transpose_std: standardized residuals, time-major, zero padded, in the
//                   layout the pairwise kernel stages into shared memory.
#include <cmath>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int kStatThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

template <class T>
__global__ void __launch_bounds__(kStatThreads) var_prep_kernel(
    const double* __restrict__ X, int64_t ldx, int m, int n, int p, T* __restrict__ Xc,
    int64_t ldc, double* __restrict__ mu_out, double* __restrict__ wbar, int* st) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const double* x = X + (int64_t)i * ldx;
  double s = 0.0;
  bool finite = true;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double v = x[t];
    finite &= isfinite(v);
    s += v;
  }
  if (__syncthreads_or(!finite)) {
    if (threadIdx.x == 0) set_status(st, VL_ERR_NONFINITE);
    return;
  }
  const double mu = block_sum(s, red) / n;
  if (threadIdx.x == 0) mu_out[i] = mu;
  T* xc = Xc + (int64_t)i * ldc;
  for (int t = threadIdx.x; t < ldc; t += blockDim.x) xc[t] = (t < n) ? T(x[t] - mu) : T(0);
  const int n_eff = n - p;
  for (int b = 0; b <= p; ++b) {
    double w = 0.0;
    for (int t = threadIdx.x; t < n_eff; t += blockDim.x) w += x[p - b + t] - mu;
    w = block_sum(w, red);
    if (threadIdx.x == 0) wbar[(int64_t)b * m + i] = w / n_eff;
  }
}

// Centred normal equations of the VAR: G holds, for the Z rows a = (tau-1) m + k
// against every W row b (W = [Y; Z_1; ..; Z_p], windows of the series centred
// by its full mean), the raw cross-product; the intercept is removed by the
// rank-one window-mean correction n_eff * wbar_a * wbar_b.
template <class T>
__global__ void var_normal_eq_kernel(const double* __restrict__ G, int m, int p, int n_eff,
                                     const double* __restrict__ wbar, T* __restrict__ Gzz,
                                     T* __restrict__ Gzy, float* __restrict__ nhi,
                                     float* __restrict__ nlo) {
  const int mp = m * p, q = m * (p + 1);
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)mp * q) return;
  const int a = (int)(idx / q), b = (int)(idx % q);
  const double v = G[idx] - (double)n_eff * wbar[m + a] * wbar[b];
  if (nhi) {  // the same values as an FP32 pair, for the refinement residual
    const float h = (float)v;
    nhi[idx] = h;
    nlo[idx] = (float)(v - (double)h);
  }
  if (b < m)
    Gzy[(int64_t)a * m + b] = (T)v;
  else
    Gzz[(int64_t)a * mp + (b - m)] = (T)v;
}

template <class T>
__global__ void var_coef_kernel(const T* __restrict__ beta, int m, int p, double* __restrict__ M) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p * m * m) return;
  const int tau = (int)(idx / ((int64_t)m * m));
  const int rem = (int)(idx % ((int64_t)m * m));
  const int i = rem / m, k = rem % m;
  M[idx] = (double)beta[((int64_t)tau * m + k) * m + i];
}

// One warp per row: cst[i] = wbar0_i - sum_a beta[a][i] wbar_{Z,a}.
template <class T>
__global__ void var_cst_kernel(const T* __restrict__ beta, int m, int p,
                               const double* __restrict__ wbar, double* __restrict__ cst) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double c = 0.0;
  for (int a = lane; a < m * p; a += 32) c += (double)beta[(int64_t)a * m + i] * wbar[m + a];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cst[i] = wbar[i] - c;
}

__global__ void var_resid_init_kernel(const double* __restrict__ X, int64_t ldx, int n_eff, int p,
                                      const double* __restrict__ mu,
                                      const double* __restrict__ cst, double* __restrict__ E,
                                      int64_t lde) {
  const int i = blockIdx.y;
  const double off = mu[i] + cst[i];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_eff; t += gridDim.x * blockDim.x)
    E[(int64_t)i * lde + t] = X[(int64_t)i * ldx + p + t] - off;
}

// Sample moments of the standardized variable for H(x_i):
// A = mean log cosh u, B = mean u exp(-u^2/2).
__device__ __forceinline__ void moments_one(double u, double& a, double& b) {
  // FP64 path of the moments
  double au = fabs(u);
  a += au + log1p(exp(-2.0 * au)) - LN2;
  b += u * exp(-0.5 * u * u);
}
__device__ __forceinline__ void kahan_f(float& S, float& C, float x) {
  float y = x - C;
  float t = S + y;
  C = (t - S) - y;
  S = t;
}

template <class T>
__global__ void __launch_bounds__(kStatThreads) standardize_kernel(
    const double* __restrict__ E, int64_t lde, int m, int n, double* __restrict__ mu_out,
    double* __restrict__ isd_out, double* __restrict__ mom, int* st) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const double* e = E + (int64_t)i * lde;
  double s = 0.0;
  bool finite = true;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double v = e[t];
    finite &= isfinite(v);
    s += v;
  }
  if (__syncthreads_or(!finite)) {
    if (threadIdx.x == 0) set_status(st, VL_ERR_NONFINITE);
    return;
  }
  const double mu = block_sum(s, red) / n;
  double q = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double d = e[t] - mu;
    q += d * d;
  }
  const double var = block_sum(q, red) / n;
  if (!(var > 1e-300)) {
    if (threadIdx.x == 0) {
      set_status(st, VL_ERR_DEGENERATE);
      mu_out[i] = mu;
      isd_out[i] = 0.0;
      mom[2 * i] = 0.0;
      mom[2 * i + 1] = 0.0;
    }
    return;
  }
  const double isd = 1.0 / sqrt(var);
  double a = 0.0, b = 0.0;
  if (sizeof(T) == 8) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) moments_one((e[t] - mu) * isd, a, b);
  } else {
    // FP32 per-sample functions (CUDA's accurate expf / log1pf), Kahan sums
    // of log cosh u + ln 2 (= |u| + log1p(e^{-2|u|})) and u e^{-u^2/2}
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    int cnt = 0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const float u = (float)((e[t] - mu) * isd);
      const float au = fabsf(u);
      kahan_f(sa, ca, au + log1pf(expf(-2.0f * au)));
      kahan_f(sb, cb, u * expf(-0.5f * u * u));
      ++cnt;
    }
    a = ((double)sa - (double)ca) - LN2 * cnt;
    b = (double)sb - (double)cb;
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    mu_out[i] = mu;
    isd_out[i] = isd;
    mom[2 * i] = a / n;
    mom[2 * i + 1] = b / n;
  }
}

__global__ void split_center_kernel(const double* __restrict__ E, int64_t lde, int n,
                                    const double* __restrict__ mu, float* __restrict__ hi,
                                    float* __restrict__ lo, int64_t ldc) {
  const int i = blockIdx.y;
  const double mi = mu[i];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ldc;
       t += (int64_t)gridDim.x * blockDim.x) {
    double v = (t < n) ? E[(int64_t)i * lde + t] - mi : 0.0;
    float h = (float)v;
    hi[(int64_t)i * ldc + t] = h;
    lo[(int64_t)i * ldc + t] = (float)(v - (double)h);
  }
}

__global__ void center64_kernel(const double* __restrict__ E, int64_t lde, int n,
                                const double* __restrict__ mu, double* __restrict__ out,
                                int64_t ldc) {
  const int i = blockIdx.y;
  const double mi = mu[i];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ldc;
       t += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)i * ldc + t] = (t < n) ? E[(int64_t)i * lde + t] - mi : 0.0;
}

// 32 x 32 tiled transpose: xt[t * m_pad + i] = (E[i, t] - mu_i) / sd_i.
template <class T>
__global__ void transpose_std_kernel(const double* __restrict__ E, int64_t lde, int m, int n,
                                     const double* __restrict__ mu,
                                     const double* __restrict__ isd, T* __restrict__ xt,
                                     int m_pad, int n_pad) {
  __shared__ T tile[32][33];
  const int t0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    int i = i0 + r, t = t0 + tx;
    T v = T(0);
    if (i < m && t < n) v = T((E[(int64_t)i * lde + t] - mu[i]) * isd[i]);
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int t = t0 + r, i = i0 + tx;
    if (t < n_pad && i < m_pad) xt[(int64_t)t * m_pad + i] = tile[tx][r];
  }
}

}  // namespace

template <class T>
void launch_var_prep(const double* X, int64_t ldx, int m, int n, int p, T* Xc, int64_t ldc,
                     double* mu, double* wbar, int* st, cudaStream_t s) {
  note_launch();
  var_prep_kernel<T><<<m, kStatThreads, 0, s>>>(X, ldx, m, n, p, Xc, ldc, mu, wbar, st);
}
template void launch_var_prep<float>(const double*, int64_t, int, int, int, float*, int64_t,
                                     double*, double*, int*, cudaStream_t);
template void launch_var_prep<double>(const double*, int64_t, int, int, int, double*, int64_t,
                                      double*, double*, int*, cudaStream_t);

template <class T>
void launch_var_normal_eq(const double* G, int m, int p, int n_eff, const double* wbar, T* Gzz,
                          T* Gzy, cudaStream_t s, float* nhi, float* nlo) {
  const int mp = m * p;
  const int64_t tot = (int64_t)mp * (mp + m);
  note_launch();
  var_normal_eq_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, m, p, n_eff, wbar,
                                                                        Gzz, Gzy, nhi, nlo);
}
template void launch_var_normal_eq<float>(const double*, int, int, int, const double*, float*,
                                          float*, cudaStream_t, float*, float*);
template void launch_var_normal_eq<double>(const double*, int, int, int, const double*,
                                           double*, double*, cudaStream_t, float*, float*);

template <class T>
void launch_var_coef(const T* beta, int m, int p, const double* wbar, double* M, double* cst,
                     cudaStream_t s) {
  const int64_t tot = (int64_t)p * m * m;
  note_launch();
  var_coef_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(beta, m, p, M);
  note_launch();
  var_cst_kernel<T><<<(m + 7) / 8, 256, 0, s>>>(beta, m, p, wbar, cst);
}
template void launch_var_coef<float>(const float*, int, int, const double*, double*, double*,
                                     cudaStream_t);

template <class T>
void launch_var_cst(const T* beta, int m, int p, const double* wbar, double* cst, cudaStream_t s) {
  note_launch();
  var_cst_kernel<T><<<(m + 7) / 8, 256, 0, s>>>(beta, m, p, wbar, cst);
}
template void launch_var_cst<float>(const float*, int, int, const double*, double*, cudaStream_t);
template void launch_var_coef<double>(const double*, int, int, const double*, double*, double*,
                                      cudaStream_t);

void launch_var_resid_init(const double* X, int64_t ldx, int m, int n, int p, const double* mu,
                           const double* cst, double* E, int64_t lde, cudaStream_t s) {
  const int n_eff = n - p;
  dim3 grid((unsigned)((n_eff + 255) / 256 < 64 ? (n_eff + 255) / 256 : 64), m);
  note_launch();
  var_resid_init_kernel<<<grid, 256, 0, s>>>(X, ldx, n_eff, p, mu, cst, E, lde);
}

template <class T>
void launch_standardize(const double* E, int64_t lde, int m, int n, double* mu, double* inv_sd,
                        double* hx_mom, int* st, cudaStream_t s) {
  note_launch();
  standardize_kernel<T><<<m, kStatThreads, 0, s>>>(E, lde, m, n, mu, inv_sd, hx_mom, st);
}
template void launch_standardize<float>(const double*, int64_t, int, int, double*, double*,
                                        double*, int*, cudaStream_t);
template void launch_standardize<double>(const double*, int64_t, int, int, double*, double*,
                                         double*, int*, cudaStream_t);

void launch_split_center(const double* E, int64_t lde, int m, int n, const double* mu,
                         float* hi, float* lo, int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)((ldc + 255) / 256 < 64 ? (ldc + 255) / 256 : 64), m);
  note_launch();
  split_center_kernel<<<grid, 256, 0, s>>>(E, lde, n, mu, hi, lo, ldc);
}

void launch_center64(const double* E, int64_t lde, int m, int n, const double* mu, double* out,
                     int64_t ldc, cudaStream_t s) {
  dim3 grid((unsigned)((ldc + 255) / 256 < 64 ? (ldc + 255) / 256 : 64), m);
  note_launch();
  center64_kernel<<<grid, 256, 0, s>>>(E, lde, n, mu, out, ldc);
}

template <class T>
void launch_transpose_std(const double* E, int64_t lde, int m, int n, const double* mu,
                          const double* inv_sd, T* xt, int m_pad, int n_pad, cudaStream_t s) {
  dim3 grid((n_pad + 31) / 32, (m_pad + 31) / 32), block(32, 8);
  note_launch();
  transpose_std_kernel<T><<<grid, block, 0, s>>>(E, lde, m, n, mu, inv_sd, xt, m_pad, n_pad);
}
template void launch_transpose_std<float>(const double*, int64_t, int, int, const double*,
                                          const double*, float*, int, int, cudaStream_t);
template void launch_transpose_std<double>(const double*, int64_t, int, int, const double*,
                                           const double*, double*, int, int, cudaStream_t);

namespace {

// One CTA: 2 sum ln L[i][i] in FP64 (a fixed-order block reduction).
__global__ void logdet_value_kernel(const double* __restrict__ L, int64_t ldl, int m,
                                    double penalty, double* __restrict__ value, int* st) {
  __shared__ double red[32];
  double s = 0.0;
  bool bad = false;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double d = L[(int64_t)i * ldl + i];
    bad |= !(d > 0.0);
    s += d > 0.0 ? log(d) : 0.0;
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) set_status(st, VL_ERR_RANK);
    return;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) *value = 2.0 * s + penalty;
}

__global__ void argmin_p_kernel(const double* __restrict__ values, int p_max,
                                int32_t* __restrict__ p_best) {
  int best = 0;
  for (int i = 1; i < p_max; ++i)
    if (values[i] < values[best]) best = i;
  *p_best = best + 1;
}

}  // namespace

void launch_logdet_value(const double* L, int64_t ldl, int m, double penalty, double* value,
                         int* st, cudaStream_t s) {
  note_launch();
  logdet_value_kernel<<<1, kStatThreads, 0, s>>>(L, ldl, m, penalty, value, st);
}

void launch_argmin_p(const double* values, int p_max, int32_t* p_best, cudaStream_t s) {
  note_launch();
  argmin_p_kernel<<<1, 1, 0, s>>>(values, p_max, p_best);
}

}  // namespace vl
