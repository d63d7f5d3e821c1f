// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
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
constexpr int BATCH_STREAMS = 32;
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
  // phase-major batches (mixed precision): per-instance buffers, the device
  // list of pairwise work items of the last batch layout and its signature,
  // and the autotuner's cache (batch signature -> samples per split)
  void* bbuf = nullptr;
  size_t bbuf_cap = 0;
  void* selbuf = nullptr;  // lag selection: coefficients and residuals of the fits
  size_t selbuf_cap = 0;
  void* bootbuf = nullptr;  // bootstrap: a chunk of resamples and their fits
  size_t bootbuf_cap = 0;
  void* blist = nullptr;
  size_t blist_cap = 0;
  unsigned long long blist_sig = 0;
  int blist_items = 0;
  std::unordered_map<unsigned long long, int> split_tune;
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
// nhi / nlo (optional, mp x m(p+1)): the centred normal equations as FP32
// pairs, for the refinement residual (k_refine.cu).
template <class T>
void launch_var_normal_eq(const double* G, int m, int p, int n_eff, const double* wbar, T* Gzz,
                          T* Gzy, cudaStream_t s, float* nhi = nullptr, float* nlo = nullptr);
// M[tau][i][k] = beta[(tau-1) m + k][i]; cst[i] = intercept offset of row i;
// E[i][t] = X[i][p + t] - mu_i - cst_i (the GEMM then subtracts sum M Z).
template <class T>
void launch_var_coef(const T* beta, int m, int p, const double* wbar, double* M, double* cst,
                     cudaStream_t s);
template <class T>
void launch_var_cst(const T* beta, int m, int p, const double* wbar, double* cst, cudaStream_t s);
// One refinement step of the VAR coefficients (k_refine.cu): r = G_zy -
// G_zz beta0 in double-float from the FP32 pairs (nhi, nlo); after the FP32
// correction solve, beta = beta0 + delta into M (FP64) and beta0 (FP32).
// The refinement residual's K range is split over up to REFINE_MAX_SPLITS
// CTAs per output tile (refine_splits(m, p, num_sms) of them); part holds
// that many m p x m blocks of float2 partial sums.
constexpr int REFINE_MAX_SPLITS = 8;
// Lag selection: values[0] = 2 sum_i ln L[i][i] + penalty for the Cholesky
// factor L (lower part of L, row stride ldl) of the residual covariance; a
// non-positive diagonal sets VL_ERR_RANK.  Then p_best = 1 + argmin of the
// p_max values (ties: smaller p).
void launch_logdet_value(const double* L, int64_t ldl, int m, double penalty, double* value,
                         int* st, cudaStream_t s);
void launch_argmin_p(const double* values, int p_max, int32_t* p_best, cudaStream_t s);
int refine_splits(int m, int p, int num_sms);
void launch_refine_residual(const float* nhi, const float* nlo, int m, int p, const float* beta0,
                            float* r, float2* part, int num_sms, cudaStream_t s);
void launch_refine_apply(float* beta, const float* delta, int m, int p, double* M,
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
// original diagonal; a pivot below 1e-6 (FP32) / 1e-12 (FP64) of it (or
// below pivot_floor of it) sets VL_ERR_RANK.
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
// pivot_floor > 0 replaces the default relative pivot floor.
void chol_blocked(const Ctx& c, T* A, int64_t lda, int n, T* dinv, double* diag0,
                  double pivot_floor = -1.0);
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
// FP32 plan with sample splits of about split_len samples (batched launches,
// where many instances fill the GPU together)
PairPlan plan_pairwise_split(int m, int n, int split_len);
void launch_pair_consts(const double* C, int m, float* rho32, float* c32, double* rho64, int* st,
                        cudaStream_t s);
void launch_pairwise_f32(const float* xt, const PairPlan& pl, const float* rho32,
                         const float* c32, float* part, cudaStream_t s);
void launch_pairwise_f64(const double* xt, const PairPlan& pl, const double* rho64,
                         double* part, cudaStream_t s);
// One instance of the FP32 pairwise kernel in a multi-instance launch.
struct PairJob {
  const float* xt;
  const float* rho32;
  const float* c32;
  float* part;
  int m, m_pad, T, n_run, tps;
};
PairJob make_pair_job(const float* xt, const PairPlan& pl, const float* rho32, const float* c32,
                      float* part);
// items: (job, tile, split, 0), largest first; grid: CTAs (about one per SM)
void launch_pairwise_f32_list(const PairJob* jobs, const int4* items, int nitems, int grid,
                              cudaStream_t s);
void launch_measure_finalize(const void* part, const PairPlan& pl, const double* hx_mom,
                             double* Hx, double* Hr, double* D, bool fp32_parts, cudaStream_t s);

// Ordering (k_order.cu).  Its workspace: P^T as double-float (pth, ptl),
// the initial row sums (sh, sl) and the gap scratch (s1, s2).
struct OrderWs {
  float *pth, *ptl, *sh, *sl;
  double* s1;
  unsigned long long* s2;
};
OrderWs order_ws_layout(void* ws, int m);
size_t order_ws_bytes(int m);
// per-step relative gaps of an order over the workspace's P (after a search)
void launch_order_gaps(void* ws, int m, const int32_t* order, double* gap, cudaStream_t s);
// spick (optional): the winning score of every step, for the certification
// of near ties (k_certify.cu).
void launch_causal_order(const double* D, int m, void* ws, int32_t* order, double* gap, int* st,
                         cudaStream_t s, long long* prof = nullptr, double* spick = nullptr);

// Tensor-core exact-slice Gram products (k_tcgram.cu).  Operands are three
// bf16 slice planes S[z][r][k] (k < Kpad = tg_kpad(K), a multiple of 64; row
// stride Kpad, plane stride `plane` elements) with a power-of-two exponent
// per row.  slice_center: rows E[r] - mu[r] (FP64); slice_lags: the lag
// windows of the centred FP32 series Xc, row b m + k = Xc[k][p - b + t].
// launch_tcgram_sym: C = (S S^T) scaled back, N x N FP64 symmetric, using
// the context's split-K scratch; false if the tensor maps cannot be made.
int64_t tg_kpad(int K);
void launch_slice_center(const double* E, int64_t lde, const double* mu, int m, int K,
                         int64_t Kpad, void* S, int64_t plane, int* exps, cudaStream_t s);
void launch_slice_lags(const float* Xc, int64_t ldc, int m, int n, int p, int64_t Kpad, void* S,
                       int64_t plane, int* exps, cudaStream_t s);
bool launch_tcgram_sym(const Ctx& cx, const void* S, int N, int Kpad, int64_t ldo, int64_t plane,
                       const int* exps, double* C, int64_t ldc);
// The VAR residuals E = X[:, p:] - mu - cst - sum_tau M_tau Z_tau as one
// tensor-core product (beta: FP32 mp x m; vexp: the variables' slice
// exponents of launch_slice_lags); false if the tensor maps cannot be made or
// the split-K buffer is smaller than m (n - p).
bool launch_tc_var_resid(const Ctx& cx, const float* Xc, int64_t ldc, const double* X,
                         int64_t ldx, int m, int n, int p, const float* beta, const int* vexp,
                         const double* mu, const double* cst, void* St, void* Sb, int* aexp,
                         double* E);

// Certified ordering (k_certify.cu): after a search on an FP32-measure D
// (launch_causal_order with spick = certify_spick(cert_ws, m)), near ties
// are re-decided on entries of D recomputed to FP64 accuracy from E (m x n,
// lde); the workspace holds E's standardized rows as double-float pairs.
// stats_out (device, 4 ints, may be NULL): flagged steps, pairs re-evaluated,
// picks changed, steps left unverified.
size_t certify_ws_bytes(int m, int n);
double* certify_spick(void* cert_ws, int m);
void launch_certify(const double* D, const double* E, int64_t lde, int m, int n, void* order_ws,
                    void* cert_ws, int32_t* order, int32_t* stats_out, int num_sms,
                    cudaStream_t s);

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

// Bootstrap (k_boot.cu).  resample: out[z] (m x n, row stride n) = moving-
// block resample b0 + z of X for z < nb.  count: with pos (nb x m scratch),
// edge[i][j] += #{z : |B0_z[i][j]| > threshold}, before[i][j] += #{z : i
// precedes j in order_z} over the nb fits (order nb x m, B0 nb x m x m).
// normalize: both tables divided by count.
void launch_boot_resample(const double* X, int64_t ldx, int m, int n, int block_len,
                          unsigned long long seed, long long b0, int nb, double* out,
                          cudaStream_t s);
void launch_boot_count(const int32_t* order, const double* B0, int m, int nb, double threshold,
                       int32_t* pos, double* edge, double* before, int* st, cudaStream_t s);
void launch_boot_normalize(double* edge, double* before, int m, int count, cudaStream_t s);

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
