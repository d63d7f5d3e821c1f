// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/varlingam_gb300.h"

namespace vl {

// ---------------------------------------------------------------- status
// Device-side sticky status word: kernels record the first error with
// atomicCAS(0 -> code); the host reads and clears it in vl_sync().
__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

constexpr double LOG2E = 1.4426950408889634;
constexpr double LN2 = 0.6931471805599453;
constexpr double H_GAUSS = 1.4189385332046727;  // (1 + log 2 pi) / 2
constexpr double ENT_K1 = 79.047;
constexpr double ENT_K2 = 7.4129;
constexpr double ENT_GAMMA = 0.37457;
constexpr double DEGENERATE_1MR2 = 1e-12;  // 1 - rho^2 below this: r_{i<-j} == 0

// H(u) from the two sample moments A = mean log cosh u, B = mean u e^{-u^2/2}.
__host__ __device__ __forceinline__ double entropy_from_moments(double A, double B) {
  double a = A - ENT_GAMMA;
  return H_GAUSS - ENT_K1 * a * a - ENT_K2 * B * B;
}

// ------------------------------------------------------------ workspace
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    size_t a = (off + 255) & ~size_t(255);
    off = a + count * sizeof(T);
    return reinterpret_cast<T*>(base + a);
  }
};

template <class T>
inline size_t ws_bytes(size_t count) {
  return ((count * sizeof(T) + 255) & ~size_t(255)) + 256;
}

}  // namespace vl

namespace vl {
// One stream of the batched path with its own workspace and series buffers.
struct PoolSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* ws = nullptr;
  size_t ws_cap = 0;
  void* buf = nullptr;
  size_t buf_cap = 0;
};
constexpr int BATCH_STREAMS = 8;
}  // namespace vl

struct vl_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;  // device workspace
  size_t ws_cap = 0;
  int* status = nullptr;  // device sticky status word (own allocation)
  int num_sms = 0;
  void* sbuf = nullptr;  // per-series buffers (E, C, D) of vl_fit
  size_t sbuf_cap = 0;
  std::vector<vl::PoolSlot> pool;  // batched path
  int* bstatus = nullptr;          // per-instance status words of a batch
  size_t bstatus_cap = 0;
  cudaEvent_t prof_start = nullptr;  // optional: recorded around the pairwise kernel
  cudaEvent_t prof_stop = nullptr;
  std::string last_error;
};

namespace vl {

// What every launcher needs: the stream, the sticky status word, the split-K
// scratch of the handle (FP64 partial products) and the SM count.
struct Ctx {
  cudaStream_t s;
  int* st;
  double* part;
  size_t part_cap;  // in doubles
  int num_sms;
};

// Count of kernel launches issued by the library in this process.
void note_launch();

// Make sure the handle owns at least `bytes` of workspace.
vl_status ensure_ws(vl_handle h, size_t bytes);
vl_status fail(vl_handle h, vl_status code, const std::string& msg);
vl_status check_launch(vl_handle h, const char* what);

// ------------------------------------------------------- kernel launchers
// Statistics / layout kernels (k_stats.cu)
template <class T>
void launch_var_prep(const double* X, int64_t ldx, int m, int n, int p, T* Xc, int64_t ldc,
                     double* mu, double* wbar, int* st, cudaStream_t s);
// VAR normal equations from the lagged Gram G (mp x m(p+1), FP64, uncentred
// in the windows): Gzz = centred Z Z^T (T, mp x mp), Gzy = centred Z Y^T
// (T, mp x m).
template <class T>
void launch_var_normal_eq(const double* G, int m, int p, int n_eff, const double* wbar, T* Gzz,
                          T* Gzy, cudaStream_t s);
// M[tau][i][k] = beta[(tau-1) m + k][i]; cst[i] = intercept offset of row i;
// E[i][t] = X[i][p + t] - mu_i - cst_i (the GEMM then subtracts sum M Z).
template <class T>
void launch_var_coef(const T* beta, int m, int p, const double* wbar, double* M, double* cst,
                     cudaStream_t s);
void launch_var_resid_init(const double* X, int64_t ldx, int m, int n, int p, const double* mu,
                           const double* cst, double* E, int64_t lde, cudaStream_t s);
template <class T>
void launch_standardize(const double* E, int64_t lde, int m, int n, double* mu, double* inv_sd,
                        double* hx_mom, int* st, cudaStream_t s);
void launch_split_center(const double* E, int64_t lde, int m, int n, const double* mu,
                         float* hi, float* lo, int64_t ldc, cudaStream_t s);
void launch_center64(const double* E, int64_t lde, int m, int n, const double* mu, double* out,
                     int64_t ldc, cudaStream_t s);
template <class T>
void launch_transpose_std(const double* E, int64_t lde, int m, int n, const double* mu,
                          const double* inv_sd, T* xt, int m_pad, int n_pad, cudaStream_t s);

// Dense linear algebra (k_linalg.cu).  A "view" addresses element (r, k) at
// base[r * rs + k * ks].  gemm computes C[r, c] = alpha * sum_k A(r,k) B(c,k)
// + beta * C[r, c] for r < M, c < N (C row-major, ldc), accumulating in T
// with a double-float flush every `flush` steps of k when T is float.
template <class T>
struct View {
  const T* base;
  int64_t rs, ks;
};
template <class T, class TC>
void launch_gemm(const Ctx& c, int M, int N, int K, double alpha, View<T> A, View<T> B,
                 double beta, TC* C, int64_t ldc, bool lower_only);
void launch_gemm_split(const Ctx& c, int M, int N, int K, View<float> Ahi, View<float> Alo,
                       View<float> Bhi, View<float> Blo, double* C, int64_t ldc,
                       bool upper_only);
// Split-K scratch (doubles) the GEMMs of an (M x N) product may use.
size_t gemm_part_need(int M, int N, int K);
// Cholesky of the n x n SPD matrix A (T, row-major, lda, lower part used) in
// place; the inverse of every nb x nb diagonal block of L is written to
// dinv (T, ceil(n/nb) blocks of nb*nb).  diag0 (n doubles) receives the
// original diagonal; a pivot below 1e-6 (FP32) / 1e-12 (FP64) of it sets
// VL_ERR_RANK.
// Triangular solves with the solution panel in shared memory (n <= 1024);
// false if not launched (the caller then uses trsm_cols_kernel).
template <class T>
bool launch_trsm_ring(const T* L, int64_t lda, const T* dinv, int n, T* R, int64_t ldr, int nrhs,
                      bool backward, cudaStream_t s);
// Cholesky of an FP32 matrix with n <= 512 on one thread-block cluster; false
// if not launched (n out of range or no cluster resources).
bool launch_chol_cluster(float* A, int64_t lda, int n, float* dinv, const double* diag0,
                         float rel_tol, int* st, cudaStream_t s,
                         unsigned long long* prof = nullptr);
template <class T>
void chol_blocked(const Ctx& c, T* A, int64_t lda, int n, T* dinv, double* diag0);
// Solve L Y = R (forward) then optionally L^T X = Y (backward) for nrhs
// right-hand sides held in R (n x nrhs, row-major, ldr), in place.
template <class T>
void chol_solve_blocked(const Ctx& c, const T* L, int64_t lda, const T* dinv, int n, T* R,
                        int64_t ldr, int nrhs, bool backward);
constexpr int CHOL_NB = 64;

template <class TI, class TO>
void launch_convert(const TI* in, int64_t ldi, TO* out, int64_t ldo, int rows, int cols,
                    cudaStream_t s);

// Pairwise measure (k_pairwise.cu)
struct PairPlan {
  int m, n, m_pad, n_pad, tiles, splits, t_per_split;
};
PairPlan plan_pairwise(int m, int n, int num_sms, bool fp64);
void launch_pair_consts(const double* C, int m, float* rho32, float* c32, double* rho64, int* st,
                        cudaStream_t s);
void launch_pairwise_f32(const float* xt, const PairPlan& pl, const float* rho32,
                         const float* c32, float* part, cudaStream_t s);
void launch_pairwise_f64(const double* xt, const PairPlan& pl, const double* rho64,
                         double* part, cudaStream_t s);
void launch_measure_finalize(const void* part, const PairPlan& pl, const double* hx_mom,
                             double* Hx, double* Hr, double* D, bool fp32_parts, cudaStream_t s);

// Ordering (k_order.cu)
size_t order_ws_bytes(int m);
void launch_causal_order(const double* D, int m, void* ws, int32_t* order, double* gap, int* st,
                         cudaStream_t s, long long* prof = nullptr);

// Iterative search of Sec. 3 (k_standard.cu).  score_pick: Eq. 3 over the
// u x u measure D, argmin (ties: lowest index) into *pick, order[k] =
// idx[pick] (idx NULL: identity), gap[k]; counter: a zeroed device word the
// kernel re-arms.  refine: Eq. 4 on the pick with the slopes C_a,pick /
// C_pick,pick of the centred cross products C (u x u), rows compacted into
// Wn (u - 1 rows), idx_next; at u == 2 also order[k + 1].
void launch_std_score_pick(const double* D, int u, double* S, unsigned* counter,
                           const int32_t* idx, int32_t* order, double* gap, int k, int* pick,
                           int* st, cudaStream_t s);
void launch_std_refine(const double* W, int64_t ldw, int u, int n, const double* C,
                       const int* pick, const int32_t* idx, double* Wn, int64_t ldn,
                       int32_t* idx_next, int32_t* order, double* gap, int k, cudaStream_t s);

// B0 / B_tau helpers (k_fitb.cu)
template <class T>
void launch_permute_cov(const double* C, int m, double scale, const int32_t* order, T* out,
                        int64_t ldo, cudaStream_t s);
template <class T>
void launch_b0_from_linv(const T* Linv, int64_t ld, const T* L, int64_t ldl, int m,
                         const int32_t* order, double* B0, cudaStream_t s);
void launch_identity_minus(const double* B0, int m, double* out, cudaStream_t s);
template <class T>
void launch_set_identity(T* A, int64_t lda, int n, cudaStream_t s);

}  // namespace vl
