// B0 from a causal order (Sec. 4: VarLiNGAM's instantaneous matrix, taken as
// the predecessor least-squares regression) and B_tau = (I - B0) M_tau.
//
// With the residual covariance S permuted into the causal order,
// S_perm = Lc Lc^T (Cholesky) and L = Lc diag(1/d), d = diag(Lc), is the
// unit-lower factor of S_perm = L diag(d^2) L^T.  Row k of I - L^{-1} holds
// the coefficients of the regression of variable c_k on c_1..c_{k-1}, so
//     B0_perm = I - diag(d) Lc^{-1}.
#include "vl_internal.cuh"

namespace vl {

namespace {

template <class T>
__global__ void permute_cov_kernel(const double* __restrict__ C, int m, double scale,
                                   const int32_t* __restrict__ order, T* __restrict__ out,
                                   int64_t ldo) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  out[(int64_t)a * ldo + b] = (T)(C[(int64_t)order[a] * m + order[b]] * scale);
}

template <class T>
__global__ void b0_from_linv_kernel(const T* __restrict__ Linv, int64_t ld,
                                    const T* __restrict__ L, int64_t ldl, int m,
                                    const int32_t* __restrict__ order, double* __restrict__ B0) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  double v = 0.0;
  if (b < a) v = -(double)L[(int64_t)a * ldl + a] * (double)Linv[(int64_t)a * ld + b];
  B0[(int64_t)order[a] * m + order[b]] = v;
}

__global__ void identity_minus_kernel(const double* __restrict__ B0, int m,
                                      double* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  out[idx] = (a == b ? 1.0 : 0.0) - B0[idx];
}

}  // namespace

template <class T>
void launch_permute_cov(const double* C, int m, double scale, const int32_t* order, T* out,
                        int64_t ldo, cudaStream_t s) {
  int64_t tot = (int64_t)m * m;
  note_launch();
  permute_cov_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C, m, scale, order, out,
                                                                      ldo);
}
template void launch_permute_cov<float>(const double*, int, double, const int32_t*, float*,
                                        int64_t, cudaStream_t);
template void launch_permute_cov<double>(const double*, int, double, const int32_t*, double*,
                                         int64_t, cudaStream_t);

template <class T>
void launch_b0_from_linv(const T* Linv, int64_t ld, const T* L, int64_t ldl, int m,
                         const int32_t* order, double* B0, cudaStream_t s) {
  int64_t tot = (int64_t)m * m;
  note_launch();
  b0_from_linv_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Linv, ld, L, ldl, m,
                                                                      order, B0);
}
template void launch_b0_from_linv<float>(const float*, int64_t, const float*, int64_t, int,
                                         const int32_t*, double*, cudaStream_t);
template void launch_b0_from_linv<double>(const double*, int64_t, const double*, int64_t, int,
                                          const int32_t*, double*, cudaStream_t);

void launch_identity_minus(const double* B0, int m, double* out, cudaStream_t s) {
  int64_t tot = (int64_t)m * m;
  note_launch();
  identity_minus_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B0, m, out);
}

}  // namespace vl
