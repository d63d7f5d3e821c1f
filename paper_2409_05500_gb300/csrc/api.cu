// C ABI of the library: handle, validation, workspace and the orchestration
// of each step of the method on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vl_internal.cuh"

using namespace vl;

namespace vl {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

vl_status fail(vl_handle h, vl_status code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

vl_status check_launch(vl_handle h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(h, VL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return VL_OK;
}

vl_status ensure_ws(vl_handle h, size_t bytes) {
  if (bytes <= h->ws_cap) return VL_OK;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_cap = 0;
  }
  size_t cap = std::max(bytes, (size_t)8 << 20);
  if (cudaMalloc(&h->ws, cap) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, VL_ERR_NOMEM, "workspace allocation of " + std::to_string(cap) + " bytes failed");
  }
  h->ws_cap = cap;
  return VL_OK;
}

}  // namespace vl

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Where one step of the method runs: a stream, the status word its kernels
// report to, and a device workspace it may overwrite.  Single calls use the
// handle's own; a batch gives every stream of its pool one of these.
struct Exec {
  vl_handle h;
  cudaStream_t s;
  int* st;
  void** ws;       // workspace pointer owned by the handle
  size_t* ws_cap;  // and its capacity
  bool measure;    // true: only accumulate the workspace size in `need`
  size_t need;
};

Exec handle_exec(vl_handle h) {
  return Exec{h, h->stream, h->status, &h->ws, &h->ws_cap, false, 0};
}

vl_status grow(vl_handle h, void** ws, size_t* cap, size_t bytes, cudaStream_t s) {
  if (bytes <= *cap) return VL_OK;
  if (*ws) {
    cudaStreamSynchronize(s);
    cudaFree(*ws);
    *ws = nullptr;
    *cap = 0;
  }
  size_t c = std::max(bytes, (size_t)8 << 20);
  if (cudaMalloc(ws, c) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, VL_ERR_NOMEM, "workspace allocation of " + std::to_string(c) + " bytes failed");
  }
  *cap = c;
  return VL_OK;
}

// Carve a workspace layout twice: once to measure, once for real.  In
// measure mode only the size is recorded and the caller launches nothing.
template <class F>
vl_status with_workspace(Exec& x, F&& carve) {
  Arena probe;
  probe.base = nullptr;
  carve(probe);
  if (x.measure) {
    x.need = std::max(x.need, probe.off + 512);
    return VL_OK;
  }
  vl_status s = grow(x.h, x.ws, x.ws_cap, probe.off + 512, x.s);
  if (s != VL_OK) return s;
  Arena a;
  a.base = static_cast<char*>(*x.ws);
  a.cap = *x.ws_cap;
  carve(a);
  return VL_OK;
}

Ctx make_ctx(const Exec& x, double* part, size_t part_cap) {
  return Ctx{x.s, x.st, part, part_cap, x.h->num_sms};
}

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------- VAR fit
template <class T>
vl_status var_fit_impl(Exec& x, const double* X, int64_t ldx, int m, int n, int p, double* M,
                       double* E) {
  const int n_eff = n - p, mp = m * p, q = m * (p + 1);
  const int64_t ldc = round_up(n, 4);
  const int nblk = (mp + CHOL_NB - 1) / CHOL_NB;
  const size_t part_cap =
      (size_t)16 * std::max((size_t)m * m, (size_t)mp * mp) +
      (sizeof(T) == 4 ? (size_t)4 * m * (p + 1) * m * (p + 1) + (size_t)m * (n - p)
                      : 0);  // tensor-core split-K and residual partials
  const bool tc = sizeof(T) == 4;  // mixed: the Gram on the tensor cores
  const int64_t kp = tg_kpad(n_eff), plane = (int64_t)q * kp;
  T *Xc, *Gzz, *Gzy, *dinv;
  double *mu, *wbar, *G, *cst, *Ew, *part, *diag0;
  char* S = nullptr;
  int* exps = nullptr;
  float *nhi = nullptr, *nlo = nullptr, *rr = nullptr;
  float2* rpart = nullptr;
  char *St = nullptr, *Sb = nullptr;
  int* aexp = nullptr;
  vl_status s = with_workspace(x, [&](Arena& a) {
    Xc = a.take<T>((size_t)m * ldc);
    mu = a.take<double>(m);
    wbar = a.take<double>((size_t)(p + 1) * m);
    if (tc) {
      G = a.take<double>((size_t)q * q) + (size_t)m * q;  // rows m.. of the full W W^T
      S = a.take<char>(3 * (size_t)plane * 2);
      exps = a.take<int>(q);
      nhi = a.take<float>((size_t)mp * q);
      nlo = a.take<float>((size_t)mp * q);
      rr = a.take<float>((size_t)mp * m);
      rpart = a.take<float2>((size_t)refine_splits(m, p, x.h->num_sms) * mp * m);
      St = a.take<char>(3 * (size_t)n * tg_kpad(m) * 2);
      Sb = a.take<char>(3 * (size_t)m * p * tg_kpad(m) * 2);
      aexp = a.take<int>(m);
    } else {
      G = a.take<double>((size_t)mp * q);
    }
    Gzz = a.take<T>((size_t)mp * mp);
    Gzy = a.take<T>((size_t)mp * m);
    dinv = a.take<T>((size_t)nblk * CHOL_NB * CHOL_NB);
    cst = a.take<double>(m);
    diag0 = a.take<double>(mp);
    Ew = E ? nullptr : a.take<double>((size_t)m * n_eff);
    part = a.take<double>(part_cap);
  });
  if (s != VL_OK || x.measure) return s;
  if (!E) E = Ew;
  Ctx cx = make_ctx(x, part, part_cap);
  cudaStream_t st = x.s;
  launch_var_prep<T>(X, ldx, m, n, p, Xc, ldc, mu, wbar, x.st, st);
  if constexpr (sizeof(T) == 4) {
    // W W^T on the tensor cores: the lag windows sliced once, the symmetric
    // q x q product; its rows m.. (the Z rows) are G
    launch_slice_lags(Xc, ldc, m, n, p, kp, S, plane, exps, st);
    if (!launch_tcgram_sym(cx, S, q, (int)kp, kp, plane, exps, G - (size_t)m * q, q))
      return fail(x.h, VL_ERR_CUDA, "vl_var_fit: tensor map encoding unavailable");
  } else {
    // lagged Gram: rows of Z (lags 1..p) against rows of W = [Y; Z]
    for (int t1 = 1; t1 <= p; ++t1)
      for (int b2 = 0; b2 <= p; ++b2) {
        View<T> A{Xc + (p - t1), ldc, 1};
        View<T> B{Xc + (p - b2), ldc, 1};
        launch_gemm<T, double>(cx, m, m, n_eff, 1.0, A, B, 0.0,
                               G + (int64_t)(t1 - 1) * m * q + (int64_t)b2 * m, q, false);
      }
  }
  launch_var_normal_eq<T>(G, m, p, n_eff, wbar, Gzz, Gzy, st, nhi, nlo);
  // Mixed: the FP32 lag Gram is accurate to about FP32 rounding, so a lag
  // variable explained by the earlier ones to within 1e-3 of its variance
  // (relative pivot below 1e-3) leaves coefficients whose error exceeds the
  // tolerances; the fit reports VL_ERR_RANK instead (VL_PREC_FP64 fits it).
  chol_blocked<T>(cx, Gzz, mp, mp, dinv, diag0, sizeof(T) == 4 ? 1e-3 : -1.0);
  chol_solve_blocked<T>(cx, Gzz, mp, dinv, mp, Gzy, m, m, true);
  if constexpr (sizeof(T) == 4) {
    // one step of iterative refinement: r = G_zy - G_zz beta0 in
    // double-float, the correction from the same FP32 factor
    launch_refine_residual(nhi, nlo, m, p, Gzy, rr, rpart, cx.num_sms, st);
    chol_solve_blocked<T>(cx, Gzz, mp, dinv, mp, rr, m, m, true);
    launch_refine_apply(Gzy, rr, m, p, M, st);
    launch_var_cst<T>(Gzy, m, p, wbar, cst, st);
  } else {
    launch_var_coef<T>(Gzy, m, p, wbar, M, cst, st);
  }
  if constexpr (sizeof(T) == 4) {
    // residuals on the tensor cores (exact slices of beta and the series)
    if (!launch_tc_var_resid(cx, Xc, ldc, X, ldx, m, n, p, Gzy, exps, mu, cst, St, Sb, aexp, E))
      return fail(x.h, VL_ERR_CUDA, "vl_var_fit: tensor map encoding unavailable");
  } else {
    launch_var_resid_init(X, ldx, m, n, p, mu, cst, E, n_eff, st);
    for (int tau = 1; tau <= p; ++tau) {
      View<T> A{Gzy + (int64_t)(tau - 1) * m * m, 1, m};  // A(i, k) = M_tau[i][k]
      View<T> B{Xc + (p - tau), 1, ldc};                 // B(t, k) = Xc[k][p - tau + t]
      launch_gemm<T, double>(cx, m, n_eff, m, -1.0, A, B, 1.0, E, n_eff, false);
    }
  }
  return check_launch(x.h, "vl_var_fit");
}

// ------------------------------------------------------- pairwise measure
struct CovOut {
  double* C;  // m x m centred cross products
  double* mu;
  double* isd;
  double* hx;  // 2m moments of the standardized variables
};

// Statistics of the standardization and the centred cross products C of E.
// Mixed precision: C on the tensor cores from exact bf16 slices
// (k_tcgram.cu); FP64: the FP64 GEMM.
template <class T>
vl_status cov_and_stats(const Ctx& cx, const double* E, int64_t lde, int m, int n,
                        const CovOut& o, void* scratch) {
  cudaStream_t st = cx.s;
  launch_standardize<T>(E, lde, m, n, o.mu, o.isd, o.hx, cx.st, st);
  if constexpr (sizeof(T) == 4) {
    const int64_t kp = tg_kpad(n), plane = (int64_t)m * kp;
    char* S = static_cast<char*>(scratch);
    int* exps = reinterpret_cast<int*>(S + round_up(3 * plane * 2, 256));
    launch_slice_center(E, lde, o.mu, m, n, kp, S, plane, exps, st);
    if (!launch_tcgram_sym(cx, S, m, (int)kp, kp, plane, exps, o.C, m)) return VL_ERR_CUDA;
  } else {
    const int64_t ldc = round_up(n, 4);
    double* ec = static_cast<double*>(scratch);
    launch_center64(E, lde, m, n, o.mu, ec, ldc, st);
    View<double> V{ec, ldc, 1};
    launch_gemm<double, double>(cx, m, m, n, 1.0, V, V, 0.0, o.C, m, false);
  }
  return VL_OK;
}

template <class T>
size_t cov_scratch_bytes(int m, int n) {
  if (sizeof(T) == 4)
    return (size_t)round_up(3 * (int64_t)m * tg_kpad(n) * 2, 256) + sizeof(int) * (size_t)m;
  return sizeof(double) * (size_t)m * round_up(n, 4);
}

template <class T>
vl_status pairwise_impl(Exec& x, const double* E, int64_t lde, int m, int n, double* Hx,
                        double* Hr, double* D, double* C_out) {
  const bool f32 = sizeof(T) == 4;
  PairPlan pl = plan_pairwise(m, n, x.h->num_sms, !f32);
  // split-K scratch of the covariance: 16 m^2, at least 64 m^2 up to 8 MB, so
  // that a small product still splits its long K over enough CTAs
  const size_t part_cap =
      std::max((size_t)16 * m * m, std::min((size_t)64 * m * m, (size_t)1 << 20));
  // FP32 path: 4 floats (2 double-float sums) per residual per split;
  // FP64 path: 2 doubles
  const size_t nparts = (size_t)pl.splits * 2 * m * m;  // in 8-byte units
  CovOut o;
  void* scratch;
  float *rho32 = nullptr, *c32 = nullptr;
  double* rho64 = nullptr;
  T* xt;
  double *pparts, *gpart, *Hr_w, *D_w;
  vl_status s = with_workspace(x, [&](Arena& a) {
    o.C = C_out ? C_out : a.take<double>((size_t)m * m);
    o.mu = a.take<double>(m);
    o.isd = a.take<double>(m);
    o.hx = a.take<double>(2 * (size_t)m);
    scratch = a.take<char>(cov_scratch_bytes<T>(m, n));
    if (f32) {
      rho32 = a.take<float>((size_t)m * m);
      c32 = a.take<float>((size_t)m * m);
    } else {
      rho64 = a.take<double>((size_t)m * m);
    }
    xt = a.take<T>((size_t)pl.n_pad * pl.m_pad);
    pparts = a.take<double>(nparts);
    gpart = a.take<double>(part_cap);
    Hr_w = Hr ? nullptr : a.take<double>((size_t)m * m);
    D_w = D ? nullptr : a.take<double>((size_t)m * m);
  });
  if (s != VL_OK || x.measure) return s;
  if (!Hr) Hr = Hr_w;
  if (!D) D = D_w;
  vl_handle h = x.h;
  Ctx cx = make_ctx(x, gpart, part_cap);
  cudaStream_t st = x.s;
  if (cov_and_stats<T>(cx, E, lde, m, n, o, scratch) != VL_OK)
    return fail(h, VL_ERR_CUDA, "vl_pairwise_measure: tensor map encoding unavailable");
  launch_pair_consts(o.C, m, rho32, c32, rho64, x.st, st);
  launch_transpose_std<T>(E, lde, m, n, o.mu, o.isd, xt, pl.m_pad, pl.n_pad, st);
  if (h->prof_start) cudaEventRecord(h->prof_start, st);
  if constexpr (sizeof(T) == 4)
    launch_pairwise_f32(xt, pl, rho32, c32, reinterpret_cast<float*>(pparts), st);
  else
    launch_pairwise_f64(xt, pl, rho64, pparts, st);
  if (h->prof_stop) cudaEventRecord(h->prof_stop, st);
  launch_measure_finalize(pparts, pl, o.hx, Hx, Hr, D, f32, st);
  return check_launch(h, "vl_pairwise_measure");
}

// ---------------------------------------------------------------- B0
template <class T>
vl_status fit_b_impl(Exec& x, const double* E, int64_t lde, int m, int n,
                     const int32_t* order, const double* M, int p, double* B0, double* Btau,
                     const double* C_in) {
  const int nblk = (m + CHOL_NB - 1) / CHOL_NB;
  const size_t part_cap = (size_t)16 * m * m;
  CovOut o{};
  void* scratch = nullptr;
  T *Sp, *dinv, *R, *IBt = nullptr, *Mt = nullptr;
  double *IB, *gpart, *diag0;
  vl_status s = with_workspace(x, [&](Arena& a) {
    if (!C_in) {
      o.C = a.take<double>((size_t)m * m);
      o.mu = a.take<double>(m);
      o.isd = a.take<double>(m);
      o.hx = a.take<double>(2 * (size_t)m);
      scratch = a.take<char>(cov_scratch_bytes<T>(m, n));
    }
    Sp = a.take<T>((size_t)m * m);
    dinv = a.take<T>((size_t)nblk * CHOL_NB * CHOL_NB);
    R = a.take<T>((size_t)m * m);
    IB = a.take<double>((size_t)m * m);
    diag0 = a.take<double>(m);
    if (sizeof(T) == 4) {
      IBt = a.take<T>((size_t)m * m);
      Mt = a.take<T>((size_t)std::max(p, 1) * m * m);
    }
    gpart = a.take<double>(part_cap);
  });
  if (s != VL_OK || x.measure) return s;
  Ctx cx = make_ctx(x, gpart, part_cap);
  cudaStream_t st = x.s;
  const double* C = C_in;
  if (!C) {
    if (cov_and_stats<T>(cx, E, lde, m, n, o, scratch) != VL_OK)
      return fail(x.h, VL_ERR_CUDA, "vl_fit_b: tensor map encoding unavailable");
    C = o.C;
  }
  launch_permute_cov<T>(C, m, 1.0 / n, order, Sp, m, st);
  chol_blocked<T>(cx, Sp, m, m, dinv, diag0);
  launch_set_identity<T>(R, m, m, st);
  chol_solve_blocked<T>(cx, Sp, m, dinv, m, R, m, m, false);
  launch_b0_from_linv<T>(R, m, Sp, m, m, order, B0, st);
  if (p > 0 && Btau && M) {
    launch_identity_minus(B0, m, IB, st);
    if constexpr (sizeof(T) == 4) {
      launch_convert<double, float>(IB, m, IBt, m, m, m, st);
      launch_convert<double, float>(M, m, Mt, m, p * m, m, st);
      for (int tau = 0; tau < p; ++tau) {
        View<float> A{IBt, m, 1};
        View<float> B{Mt + (int64_t)tau * m * m, 1, m};
        launch_gemm<float, double>(cx, m, m, m, 1.0, A, B, 0.0, Btau + (int64_t)tau * m * m, m,
                                   false);
      }
    } else {
      for (int tau = 0; tau < p; ++tau) {
        View<double> A{IB, m, 1};
        View<double> B{M + (int64_t)tau * m * m, 1, m};
        launch_gemm<double, double>(cx, m, m, m, 1.0, A, B, 0.0, Btau + (int64_t)tau * m * m,
                                    m, false);
      }
    }
  }
  return check_launch(x.h, "vl_fit_b");
}

vl_status order_impl(Exec& x, const double* D, int m, int32_t* order, double* gap) {
  char* ows;
  vl_status s = with_workspace(x, [&](Arena& a) { ows = a.take<char>(order_ws_bytes(m)); });
  if (s != VL_OK || x.measure) return s;
  launch_causal_order(D, m, ows, order, gap, x.st, x.s);
  return check_launch(x.h, "vl_causal_order");
}

// Algorithm 1 on an FP32-measure D with its near ties re-decided in FP64
// from E (k_certify.cu).
vl_status order_certified_impl(Exec& x, const double* D, const double* E, int64_t lde, int m,
                               int n, int32_t* order, double* gap, int32_t* stats) {
  char *ows, *cws;
  vl_status s = with_workspace(x, [&](Arena& a) {
    ows = a.take<char>(order_ws_bytes(m));
    cws = a.take<char>(certify_ws_bytes(m, n));
  });
  if (s != VL_OK || x.measure) return s;
  launch_causal_order(D, m, ows, order, nullptr, x.st, x.s, nullptr, certify_spick(cws, m));
  launch_certify(D, E, lde, m, n, ows, cws, order, stats, x.h->num_sms, x.s);
  if (gap) launch_order_gaps(ows, m, order, gap, x.s);
  return check_launch(x.h, "vl_causal_order_certified");
}

// The iterative search of Sec. 3: m - 1 iterations of (pairwise measure of
// the u remaining variables, Eq. 3 score + pick, Eq. 4 refinement with
// compaction), all queued on the stream; the pick stays on the device.
template <class T>
vl_status order_standard_impl(Exec& x, const double* E, int64_t lde, int m, int n,
                              int32_t* order, double* gap) {
  vl_handle h = x.h;
  // workspace of the largest measure (every later one is smaller in all
  // terms except the split count, so take the maximum over all of them)
  Exec probe{h, nullptr, nullptr, nullptr, nullptr, true, 0};
  for (int u = m; u >= 2; --u)
    pairwise_impl<T>(probe, E, lde, u, n, nullptr, nullptr, nullptr, nullptr);
  vl_status s = grow(h, x.ws, x.ws_cap, probe.need, x.s);
  if (s != VL_OK) return s;
  const int64_t ldw = round_up(n, 4);
  double *W0, *W1, *D, *C, *S;
  int32_t *idx0, *idx1;
  int* pick;
  unsigned* counter;
  auto carve = [&](Arena& a) {
    W0 = a.take<double>((size_t)m * ldw);
    W1 = a.take<double>((size_t)m * ldw);
    D = a.take<double>((size_t)m * m);
    C = a.take<double>((size_t)m * m);
    S = a.take<double>(m);
    idx0 = a.take<int32_t>(m);
    idx1 = a.take<int32_t>(m);
    pick = a.take<int>(1);
    counter = a.take<unsigned>(1);
  };
  Arena sz;
  carve(sz);
  s = grow(h, &h->sbuf, &h->sbuf_cap, sz.off + 512, x.s);
  if (s != VL_OK) return s;
  Arena a;
  a.base = static_cast<char*>(h->sbuf);
  a.cap = h->sbuf_cap;
  carve(a);
  cudaMemsetAsync(counter, 0, sizeof(unsigned), x.s);
  const double* src = E;
  int64_t lds = lde;
  const int32_t* isrc = nullptr;  // identity at the first iteration
  double* Wdst = W0;
  int32_t* idst = idx0;
  for (int k = 0; k + 1 < m; ++k) {
    const int u = m - k;
    s = pairwise_impl<T>(x, src, lds, u, n, nullptr, nullptr, D, C);
    if (s != VL_OK) return s;
    launch_std_score_pick(D, u, S, counter, isrc, order, gap, k, pick, x.st, x.s);
    launch_std_refine(src, lds, u, n, C, pick, isrc, Wdst, ldw, idst, order, gap, k, x.s);
    src = Wdst;
    lds = ldw;
    isrc = idst;
    Wdst = Wdst == W0 ? W1 : W0;
    idst = idst == idx0 ? idx1 : idx0;
  }
  return check_launch(h, "vl_causal_order_standard");
}

// The whole method on one series, on one execution context.  E, C and D are
// per-series buffers of the caller (E: m x (n-p), C, D: m x m).
template <class T>
vl_status fit_one(Exec& x, const vl_instance& I, double* E, double* C, double* D,
                  bool certified = false) {
  const int m = I.m, n_eff = I.n - I.p;
  vl_status s = var_fit_impl<T>(x, I.X, I.ldx, m, I.n, I.p, I.M, E);
  if (s == VL_OK) s = pairwise_impl<T>(x, E, n_eff, m, n_eff, nullptr, nullptr, D, C);
  if (s == VL_OK)
    s = certified ? order_certified_impl(x, D, E, n_eff, m, n_eff, I.order, nullptr, nullptr)
                  : order_impl(x, D, m, I.order, nullptr);
  if (s == VL_OK) s = fit_b_impl<T>(x, E, n_eff, m, n_eff, I.order, I.M, I.p, I.B0, I.Btau, C);
  return s;
}

vl_status validate_prec(vl_handle h, vl_precision prec) {
  if (prec != VL_PREC_FP64 && prec != VL_PREC_MIXED && prec != VL_PREC_MIXED_CERTIFIED)
    return fail(h, VL_ERR_ARG,
                "precision must be VL_PREC_FP64, VL_PREC_MIXED or VL_PREC_MIXED_CERTIFIED");
  return VL_OK;
}

vl_status check_instance(vl_handle h, const vl_instance& I) {
  if (!I.X || !I.order || !I.B0 || !I.M || !I.Btau)
    return fail(h, VL_ERR_ARG, "vl_fit_batched: NULL pointer in instance");
  if (I.m < 2 || I.p < 1 || I.n < 2 || I.m > VL_MAX_M || I.ldx < I.n)
    return fail(h, VL_ERR_SHAPE, "vl_fit_batched: bad sizes");
  if ((int64_t)I.n - I.p <= (int64_t)I.m * I.p + 1)
    return fail(h, VL_ERR_RANK, "vl_fit_batched: n - p <= m p + 1");
  return VL_OK;
}

// ------------------------------------------------ phase-major mixed batches
// A mixed-precision batch runs in three phases: (A) every instance's VAR fit
// and the measure's preparation (statistics, tensor-core covariance, pair
// constants, time-major standardized data) on a pool of streams; (B) ONE
// launch of the pairwise kernel over a device list of (instance, pair tile,
// sample split) work items of all instances, largest first; (C) every
// instance's finalisation of the measure, ordering and B0 / B_tau on the
// pool.  The per-instance buffers live in one handle-owned allocation; the
// work list is uploaded once per batch layout, so after a first call the
// whole batch can be captured into one CUDA graph (vl_fit_batched_async).
// The length of the sample splits of phase B is chosen by an autotuner: on
// the first uncaptured call of a batch shape every candidate length is timed
// (CUDA events) and the fastest is cached in the handle.

struct InstBufs {
  PairPlan pl;  // the plan phase B and the finalisation use
  double *E, *C, *D, *mu, *isd, *hx;
  float *rho32, *c32, *xt, *parts;
};

constexpr int SPLIT_CANDIDATES[] = {256, 512, 1024, 2048, 4096};
constexpr int SPLIT_MIN = 256;      // buffers hold the partials of the shortest split
constexpr int SPLIT_DEFAULT = 1024;  // used under capture before any tuning

void carve_inst(Arena& a, const vl_instance& I, InstBufs& b) {
  const size_t m = I.m, ne = I.n - I.p;
  const PairPlan big = plan_pairwise_split(I.m, I.n - I.p, SPLIT_MIN);
  b.E = a.take<double>(m * ne);
  b.C = a.take<double>(m * m);
  b.D = a.take<double>(m * m);
  b.mu = a.take<double>(m);
  b.isd = a.take<double>(m);
  b.hx = a.take<double>(2 * m);
  b.rho32 = a.take<float>(m * m);
  b.c32 = a.take<float>(m * m);
  b.xt = a.take<float>((size_t)big.n_pad * big.m_pad);
  b.parts = a.take<float>((size_t)big.splits * 4 * m * m);
}

// Phase A of one instance.
vl_status batch_prep(Exec& x, const vl_instance& I, InstBufs& b) {
  const int m = I.m, n_eff = I.n - I.p;
  vl_status s = var_fit_impl<float>(x, I.X, I.ldx, m, I.n, I.p, I.M, b.E);
  if (s != VL_OK) return s;
  const size_t part_cap =
      std::max((size_t)16 * m * m, std::min((size_t)64 * m * m, (size_t)1 << 20));
  void* scratch;
  double* gpart;
  s = with_workspace(x, [&](Arena& a) {
    scratch = a.take<char>(cov_scratch_bytes<float>(m, n_eff));
    gpart = a.take<double>(part_cap);
  });
  if (s != VL_OK || x.measure) return s;
  Ctx cx = make_ctx(x, gpart, part_cap);
  CovOut o{b.C, b.mu, b.isd, b.hx};
  if (cov_and_stats<float>(cx, b.E, n_eff, m, n_eff, o, scratch) != VL_OK)
    return fail(x.h, VL_ERR_CUDA, "vl_fit_batched: tensor map encoding unavailable");
  launch_pair_consts(b.C, m, b.rho32, b.c32, nullptr, x.st, x.s);
  launch_transpose_std<float>(b.E, n_eff, m, n_eff, b.mu, b.isd, b.xt, b.pl.m_pad, b.pl.n_pad,
                              x.s);
  return VL_OK;
}

// Phase C of one instance.
vl_status batch_finish(Exec& x, const vl_instance& I, const InstBufs& b, bool certified) {
  const int m = I.m, n_eff = I.n - I.p;
  double* Hr;
  vl_status s = with_workspace(x, [&](Arena& a) { Hr = a.take<double>((size_t)m * m); });
  if (s != VL_OK) return s;
  double* D = I.D ? I.D : b.D;
  if (!x.measure) launch_measure_finalize(b.parts, b.pl, b.hx, nullptr, Hr, D, true, x.s);
  s = certified ? order_certified_impl(x, D, b.E, n_eff, m, n_eff, I.order, nullptr, nullptr)
                : order_impl(x, D, m, I.order, nullptr);
  if (s == VL_OK) s = fit_b_impl<float>(x, b.E, n_eff, m, n_eff, I.order, I.M, I.p, I.B0, I.Btau,
                                        b.C);
  return s;
}

unsigned long long mix64(unsigned long long h, unsigned long long v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// The work items of phase B for split length `len`, largest first; the plans
// of the instances are set to that length.
void build_items(const vl_instance* inst, const std::vector<int>& idx, std::vector<InstBufs>& B,
                 int len, std::vector<PairJob>& jobs, std::vector<int4>& items) {
  jobs.clear();
  items.clear();
  std::vector<std::pair<double, int4>> w;
  for (size_t j = 0; j < idx.size(); ++j) {
    const vl_instance& I = inst[idx[j]];
    InstBufs& b = B[j];
    b.pl = plan_pairwise_split(I.m, I.n - I.p, len);
    jobs.push_back(make_pair_job(b.xt, b.pl, b.rho32, b.c32, b.parts));
    const int T = b.pl.m_pad / 32;
    for (int t = 0, q = 0; t < T; ++t)
      for (int u = t; u < T; ++u, ++q) {
        // pairs with i < j < m in tile (t, u)
        const int i0 = 32 * t, j0 = 32 * u;
        double pairs = 0;
        for (int i = i0; i < std::min(i0 + 32, I.m); ++i)
          pairs += std::max(0, std::min(j0 + 32, I.m) - std::max(j0, i + 1));
        for (int z = 0; z < b.pl.splits; ++z) {
          const int n_run = ((I.n - I.p + 15) / 16) * 16;
          const int len_z = std::min(b.pl.t_per_split, n_run - z * b.pl.t_per_split);
          w.push_back({pairs * std::max(len_z, 0) + 1e-3, make_int4((int)j, q, z, 0)});
        }
      }
  }
  std::stable_sort(w.begin(), w.end(),
                   [](const std::pair<double, int4>& a, const std::pair<double, int4>& b) {
                     return a.first > b.first;
                   });
  for (auto& e : w) items.push_back(e.second);
}

// The phase-major batch over the valid instances idx (already checked on the
// host).  dstat: per-instance device status words (count of the caller's
// array, indexed by instance).  Allocates only if a buffer must grow, uploads
// the work list only when the batch layout changed, and tunes the split
// length only outside stream capture.
vl_status batched_mixed(vl_handle h, const vl_instance* inst, const std::vector<int>& idx,
                        bool certified, int* dstat) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(h->stream, &cap);
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  const int S = (int)std::min<size_t>(idx.size(), (size_t)BATCH_STREAMS);
  if (S == 0) return VL_OK;
  // per-instance buffers, one allocation
  std::vector<InstBufs> B(idx.size());
  Arena sz;
  for (size_t j = 0; j < idx.size(); ++j) carve_inst(sz, inst[idx[j]], B[j]);
  if (sz.off + 512 > h->bbuf_cap && capturing)
    return fail(h, VL_ERR_UNSUPPORTED, "vl_fit_batched_async: call once outside capture first");
  vl_status s = grow(h, &h->bbuf, &h->bbuf_cap, sz.off + 512, h->stream);
  if (s != VL_OK) return s;
  Arena ar;
  ar.base = static_cast<char*>(h->bbuf);
  ar.cap = h->bbuf_cap;
  for (size_t j = 0; j < idx.size(); ++j) {
    carve_inst(ar, inst[idx[j]], B[j]);
    B[j].pl = plan_pairwise_split(inst[idx[j]].m, inst[idx[j]].n - inst[idx[j]].p, SPLIT_DEFAULT);
  }
  // per-stream workspace: the largest need of phases A and C
  size_t ws_need = 0;
  for (size_t j = 0; j < idx.size(); ++j) {
    Exec probe{h, nullptr, nullptr, nullptr, nullptr, true, 0};
    batch_prep(probe, inst[idx[j]], B[j]);
    batch_finish(probe, inst[idx[j]], B[j], certified);
    ws_need = std::max(ws_need, probe.need);
  }
  if ((int)h->pool.size() < S) h->pool.resize(S);
  for (int q = 0; q < S; ++q) {
    PoolSlot& ps = h->pool[q];
    if ((!ps.stream || !ps.done || ps.ws_cap < ws_need) && capturing)
      return fail(h, VL_ERR_UNSUPPORTED, "vl_fit_batched_async: call once outside capture first");
    if (!ps.stream && cudaStreamCreateWithFlags(&ps.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, VL_ERR_CUDA, "vl_fit_batched: stream creation failed");
    }
    if (!ps.done && cudaEventCreateWithFlags(&ps.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, VL_ERR_CUDA, "vl_fit_batched: event creation failed");
    }
    s = grow(h, &ps.ws, &ps.ws_cap, ws_need, ps.stream);
    if (s != VL_OK) return s;
  }
  // split length: tuned once per batch shape
  unsigned long long shape = mix64(0, idx.size());
  for (int k : idx) shape = mix64(mix64(mix64(shape, inst[k].m), inst[k].n), inst[k].p);
  auto tuned = h->split_tune.find(shape);
  const bool tune = tuned == h->split_tune.end() && !capturing;
  int len = tuned != h->split_tune.end() ? tuned->second : SPLIT_DEFAULT;
  std::vector<PairJob> jobs;
  std::vector<int4> items;
  // upload the work list of `len` if the layout differs from the device copy
  auto upload = [&](int L) -> vl_status {
    build_items(inst, idx, B, L, jobs, items);
    const unsigned long long sig =
        mix64(mix64(mix64(shape, (unsigned long long)(uintptr_t)h->bbuf), L), items.size());
    if (sig == h->blist_sig) return VL_OK;
    if (capturing)
      return fail(h, VL_ERR_UNSUPPORTED, "vl_fit_batched_async: call once outside capture first");
    const size_t bytes = jobs.size() * sizeof(PairJob) + 256 + items.size() * sizeof(int4);
    vl_status r = grow(h, &h->blist, &h->blist_cap, bytes, h->stream);
    if (r != VL_OK) return r;
    char* d = static_cast<char*>(h->blist);
    const size_t joff = ((jobs.size() * sizeof(PairJob)) + 255) & ~size_t(255);
    if (cudaMemcpyAsync(d, jobs.data(), jobs.size() * sizeof(PairJob), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(d + joff, items.data(), items.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, VL_ERR_CUDA, "vl_fit_batched: work list upload failed");
    }
    h->blist_sig = sig;
    h->blist_items = (int)items.size();
    return VL_OK;
  };
  auto list_ptrs = [&](const PairJob*& J, const int4*& It) {
    char* d = static_cast<char*>(h->blist);
    J = reinterpret_cast<const PairJob*>(d);
    It = reinterpret_cast<const int4*>(
        d + (((jobs.size() * sizeof(PairJob)) + 255) & ~size_t(255)));
  };
  if (!tune) {
    s = upload(len);
    if (s != VL_OK) return s;
  }
  // fork: every pool stream waits for the handle stream
  auto fork = [&]() {
    cudaEventRecord(h->pool[0].done, h->stream);
    for (int q = 0; q < S; ++q) cudaStreamWaitEvent(h->pool[q].stream, h->pool[0].done, 0);
  };
  auto join = [&]() {
    for (int q = 0; q < S; ++q) {
      cudaEventRecord(h->pool[q].done, h->pool[q].stream);
      cudaStreamWaitEvent(h->stream, h->pool[q].done, 0);
    }
  };
  // phase A, instances largest first (idx is sorted so), dealt round robin
  fork();
  for (size_t j = 0; j < idx.size(); ++j) {
    PoolSlot& ps = h->pool[j % S];
    Exec x{h, ps.stream, dstat + idx[j], &ps.ws, &ps.ws_cap, false, 0};
    s = batch_prep(x, inst[idx[j]], B[j]);
    if (s != VL_OK) break;
  }
  join();
  if (s != VL_OK) return s;
  // phase B
  const int grid = h->num_sms;  // one CTA per SM (the kernel's occupancy)
  const PairJob* J;
  const int4* It;
  if (tune) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int L : SPLIT_CANDIDATES) {
      s = upload(L);
      if (s != VL_OK) break;
      list_ptrs(J, It);
      cudaEventRecord(e0, h->stream);
      launch_pairwise_f32_list(J, It, (int)items.size(), grid, h->stream);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        len = L;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != VL_OK) return s;
    h->split_tune[shape] = len;
    s = upload(len);
    if (s != VL_OK) return s;
  }
  build_items(inst, idx, B, len, jobs, items);  // the plans of the chosen length
  list_ptrs(J, It);
  launch_pairwise_f32_list(J, It, h->blist_items, grid, h->stream);
  // phase C
  fork();
  for (size_t j = 0; j < idx.size(); ++j) {
    PoolSlot& ps = h->pool[j % S];
    Exec x{h, ps.stream, dstat + idx[j], &ps.ws, &ps.ws_cap, false, 0};
    s = batch_finish(x, inst[idx[j]], B[j], certified);
    if (s != VL_OK) break;
  }
  join();
  if (s != VL_OK) return s;
  return check_launch(h, "vl_fit_batched");
}


// Wait for the batch and merge the per-instance device statuses into the
// host statuses; returns the first non-OK status.
vl_status read_batch_status(vl_handle h, const std::vector<int>& idx, int count,
                            vl_status* inst_status) {
  std::vector<int> dev(count, 0);
  cudaError_t e = cudaMemcpyAsync(dev.data(), h->bstatus, sizeof(int) * count,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    for (int k : idx) inst_status[k] = VL_ERR_CUDA;
    return fail(h, VL_ERR_CUDA, std::string("vl_fit_batched: ") + cudaGetErrorString(e));
  }
  for (int k : idx)
    if (inst_status[k] == VL_OK && dev[k] != 0) inst_status[k] = (vl_status)dev[k];
  vl_status err = VL_OK;
  for (int k = 0; k < count; ++k)
    if (err == VL_OK && inst_status[k] != VL_OK) err = inst_status[k];
  if (err != VL_OK && h->last_error.empty()) h->last_error = "vl_fit_batched: an instance failed";
  return err;
}

// A batch: instances are dealt, largest first, to a pool of streams forked
// from the handle's stream; every stream has its own workspace and per-series
// buffers, and every instance its own status word.  Nothing allocates while
// kernels are queued unless a buffer must grow; the host waits once, at the
// end, to read the statuses.
vl_status batched_impl(vl_handle h, const vl_instance* inst, int count, vl_precision prec,
                       vl_status* inst_status) {
  std::vector<int> idx;
  for (int k = 0; k < count; ++k) {
    inst_status[k] = check_instance(h, inst[k]);
    if (inst_status[k] == VL_OK) idx.push_back(k);
  }
  // largest first (cost ~ m^2 n) so the streams finish together
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return (double)inst[a].m * inst[a].m * inst[a].n > (double)inst[b].m * inst[b].m * inst[b].n;
  });
  const int S = (int)std::min<size_t>(idx.size(), (size_t)BATCH_STREAMS);
  vl_status err = VL_OK;
  if (S > 0) {
    // per-stream sizes: workspace of every step + E, C, D of its largest series
    size_t ws_need = 0, buf_need = 0;
    for (int k : idx) {
      const vl_instance& I = inst[k];
      Exec probe{h, nullptr, nullptr, nullptr, nullptr, true, 0};
      double* dummy = nullptr;
      if (prec != VL_PREC_FP64)
        fit_one<float>(probe, I, dummy, dummy, dummy, prec == VL_PREC_MIXED_CERTIFIED);
      else
        fit_one<double>(probe, I, dummy, dummy, dummy);
      ws_need = std::max(ws_need, probe.need);
      const size_t m = I.m, ne = I.n - I.p;
      buf_need = std::max(buf_need, sizeof(double) * (m * ne + 2 * m * m) + 1024);
    }
    vl_status s = VL_OK;
    if ((int)h->pool.size() < S) h->pool.resize(S);
    if (h->bstatus_cap < (size_t)count) {
      if (h->bstatus) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->bstatus);
      }
      h->bstatus = nullptr;
      h->bstatus_cap = 0;
      if (cudaMalloc(&h->bstatus, sizeof(int) * count) != cudaSuccess) {
        cudaGetLastError();
        for (int k : idx) inst_status[k] = VL_ERR_NOMEM;
        return fail(h, VL_ERR_NOMEM, "vl_fit_batched: status array allocation failed");
      }
      h->bstatus_cap = count;
    }
    if (prec != VL_PREC_FP64) {  // mixed precisions: the phase-major batch
      cudaMemsetAsync(h->bstatus, 0, sizeof(int) * count, h->stream);
      s = batched_mixed(h, inst, idx, prec == VL_PREC_MIXED_CERTIFIED, h->bstatus);
      if (s != VL_OK) {
        for (int k : idx) inst_status[k] = s;
        return s;
      }
      return read_batch_status(h, idx, count, inst_status);
    }
    for (int q = 0; q < S && s == VL_OK; ++q) {
      PoolSlot& ps = h->pool[q];
      if (!ps.stream && cudaStreamCreateWithFlags(&ps.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s = fail(h, VL_ERR_CUDA, "vl_fit_batched: stream creation failed");
        break;
      }
      if (!ps.done && cudaEventCreateWithFlags(&ps.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        s = fail(h, VL_ERR_CUDA, "vl_fit_batched: event creation failed");
        break;
      }
      s = grow(h, &ps.ws, &ps.ws_cap, ws_need, ps.stream);
      if (s == VL_OK) s = grow(h, &ps.buf, &ps.buf_cap, buf_need, ps.stream);
    }
    if (s != VL_OK) {  // nothing ran: every valid instance reports the call's error
      for (int k : idx) inst_status[k] = s;
      return s;
    }
    cudaMemsetAsync(h->bstatus, 0, sizeof(int) * count, h->stream);
    // fork: every pool stream waits for the handle stream
    cudaEvent_t fork = h->pool[0].done;
    cudaEventRecord(fork, h->stream);
    for (int q = 0; q < S; ++q) cudaStreamWaitEvent(h->pool[q].stream, fork, 0);
    for (size_t t = 0; t < idx.size(); ++t) {
      const int k = idx[t];
      PoolSlot& ps = h->pool[t % S];
      const vl_instance& I = inst[k];
      Exec x{h, ps.stream, h->bstatus + k, &ps.ws, &ps.ws_cap, false, 0};
      double* E = static_cast<double*>(ps.buf);
      double* C = E + (size_t)I.m * (I.n - I.p);
      double* D = I.D ? I.D : C + (size_t)I.m * I.m;
      vl_status r = prec != VL_PREC_FP64 ? fit_one<float>(x, I, E, C, D, prec == VL_PREC_MIXED_CERTIFIED)
                                          : fit_one<double>(x, I, E, C, D);
      if (r != VL_OK) inst_status[k] = r;
    }
    // join
    for (int q = 0; q < S; ++q) {
      cudaEventRecord(h->pool[q].done, h->pool[q].stream);
      cudaStreamWaitEvent(h->stream, h->pool[q].done, 0);
    }
    return read_batch_status(h, idx, count, inst_status);
  }
  for (int k = 0; k < count; ++k)
    if (err == VL_OK && inst_status[k] != VL_OK) err = inst_status[k];
  if (err != VL_OK && h->last_error.empty()) h->last_error = "vl_fit_batched: an instance failed";
  return err;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

vl_status vl_create(vl_handle* out, int device, void* cuda_stream, size_t workspace_bytes) {
  if (!out) return VL_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return VL_ERR_CUDA;
  }
  vl_handle h = new (std::nothrow) vl_handle_s();
  if (!h) return VL_ERR_NOMEM;
  h->device = device;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&h->status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return VL_ERR_NOMEM;
  }
  cudaMemset(h->status, 0, sizeof(int));
  if (workspace_bytes > 0 && ensure_ws(h, workspace_bytes) != VL_OK) {
    cudaFree(h->status);
    delete h;
    return VL_ERR_NOMEM;
  }
  cudaDeviceSynchronize();
  *out = h;
  return VL_OK;
}

vl_status vl_destroy(vl_handle h) {
  if (!h) return VL_ERR_ARG;
  {
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto& ps : h->pool) {
      if (ps.stream) cudaStreamSynchronize(ps.stream);
      if (ps.ws) cudaFree(ps.ws);
      if (ps.buf) cudaFree(ps.buf);
      if (ps.done) cudaEventDestroy(ps.done);
      if (ps.stream) cudaStreamDestroy(ps.stream);
    }
    if (h->bstatus) cudaFree(h->bstatus);
    if (h->sbuf) cudaFree(h->sbuf);
    if (h->bbuf) cudaFree(h->bbuf);
    if (h->selbuf) cudaFree(h->selbuf);
    if (h->bootbuf) cudaFree(h->bootbuf);
    if (h->blist) cudaFree(h->blist);
    if (h->ws) cudaFree(h->ws);
    if (h->status) cudaFree(h->status);
  }
  delete h;
  return VL_OK;
}

vl_status vl_set_stream(vl_handle h, void* cuda_stream) {
  if (!h) return VL_ERR_ARG;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return VL_OK;
}

vl_status vl_reserve(vl_handle h, int m, int n, int p) {
  if (!h) return VL_ERR_ARG;
  if (m < 2 || n < 2 || p < 0 || m > VL_MAX_M) return fail(h, VL_ERR_SHAPE, "vl_reserve: bad sizes");
  // generous upper bound of the largest per-call layout
  const size_t mm = (size_t)m * m, mp = (size_t)m * std::max(p, 1);
  const size_t ln = (size_t)round_up(n, 64) + 64;
  const size_t mpad = (size_t)round_up(m, 32);
  size_t b = 0;
  b += 8 * (mp * (mp + m) * 2 + 16 * std::max(mm, mp * mp) + (size_t)m * ln * 3);
  b += 8 * (mm * 8 + mpad * ln + (size_t)64 * mm);
  // pairwise partials of a problem too small to fill one wave: shorter
  // splits, at most one CTA per SM, 4096 doubles per CTA beyond the m^2 terms
  b += 8 * (size_t)4096 * h->num_sms;
  // mixed path: the tensor-core Grams (full W W^T, its split-K partials, the
  // bf16 slices of W and of E) and the certified ordering's FP64 cache and
  // standardized rows
  const size_t q = (size_t)m * (std::max(p, 1) + 1);
  b += 8 * 5 * q * q + 6 * (q + (size_t)m) * ln + 24 * mm + 8 * (size_t)m * ln;
  // the residual product's slices and partials
  b += 6 * ln * (mpad + 64) + 6 * mp * (mpad + 64) + 8 * (size_t)m * ln;
  DeviceGuard g(h->device);
  return ensure_ws(h, b);
}

vl_status vl_sync(vl_handle h) {
  if (!h) return VL_ERR_ARG;
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, VL_ERR_CUDA, std::string("vl_sync: ") + cudaGetErrorString(e));
  int code = 0;
  e = cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(h, VL_ERR_CUDA, std::string("vl_sync: ") + cudaGetErrorString(e));
  if (code != 0) {
    cudaMemset(h->status, 0, sizeof(int));
    static const char* names[] = {"ok", "argument", "shape", "rank deficient (non-SPD system)",
                                  "degenerate (zero variance or |rho| = 1)", "non-finite input",
                                  "cuda", "out of memory", "timeout", "unsupported"};
    const char* nm = (code >= 0 && code <= 9) ? names[code] : "unknown";
    return fail(h, (vl_status)code, std::string("device reported: ") + nm);
  }
  return VL_OK;
}

vl_status vl_profile_events(vl_handle h, void* start_event, void* stop_event) {
  if (!h) return VL_ERR_ARG;
  if ((start_event == nullptr) != (stop_event == nullptr))
    return fail(h, VL_ERR_ARG, "vl_profile_events: give both events or neither");
  h->prof_start = static_cast<cudaEvent_t>(start_event);
  h->prof_stop = static_cast<cudaEvent_t>(stop_event);
  return VL_OK;
}

unsigned long long vl_kernel_launches(void) { return g_launches.load(); }

const char* vl_last_error(vl_handle h) {
  if (!h) return "null handle";
  return h->last_error.c_str();
}

vl_status vl_var_fit(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                     vl_precision prec, double* M, double* E) {
  if (!h) return VL_ERR_ARG;
  if (!X || !M) return fail(h, VL_ERR_ARG, "vl_var_fit: X and M must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (m < 2 || p < 1 || n < 2 || m > VL_MAX_M || ldx < n)
    return fail(h, VL_ERR_SHAPE, "vl_var_fit: need m >= 2, p >= 1, ldx >= n");
  if ((int64_t)n - p <= (int64_t)m * p + 1)
    return fail(h, VL_ERR_RANK, "vl_var_fit: n - p <= m p + 1, the VAR has no unique fit");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return prec != VL_PREC_FP64 ? var_fit_impl<float>(x, X, ldx, m, n, p, M, E)
                               : var_fit_impl<double>(x, X, ldx, m, n, p, M, E);
}

vl_status vl_var_select(vl_handle h, const double* X, int64_t ldx, int m, int n, int p_max,
                        vl_criterion crit, vl_precision prec, double* values, int32_t* p_best) {
  if (!h) return VL_ERR_ARG;
  if (!X || !values || !p_best)
    return fail(h, VL_ERR_ARG, "vl_var_select: X, values and p_best must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (crit != VL_IC_AIC && crit != VL_IC_BIC && crit != VL_IC_HQ)
    return fail(h, VL_ERR_ARG, "vl_var_select: unknown criterion");
  if (m < 2 || p_max < 1 || n < 2 || m > VL_MAX_M || ldx < n)
    return fail(h, VL_ERR_SHAPE, "vl_var_select: need m >= 2, p_max >= 1, ldx >= n");
  const int64_t T = (int64_t)n - p_max;
  if (T <= (int64_t)m * (p_max + 1))
    return fail(h, VL_ERR_RANK,
                "vl_var_select: n - p_max <= m (p_max + 1), the residual covariance of the "
                "largest VAR cannot be of full rank");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  // the candidates' coefficients and residuals (reused from p to p)
  const size_t mb = (size_t)p_max * m * m, eb = (size_t)m * T;
  vl_status s = grow(h, &h->selbuf, &h->selbuf_cap, sizeof(double) * (mb + eb) + 512, x.s);
  if (s != VL_OK) return s;
  double* Mb = static_cast<double*>(h->selbuf);
  double* Eb = Mb + mb;
  const double lt = std::log((double)T);
  const double pen = crit == VL_IC_AIC ? 2.0 : (crit == VL_IC_BIC ? lt : 2.0 * std::log(lt));
  const int nblk = (m + CHOL_NB - 1) / CHOL_NB;
  const size_t part_cap = std::max((size_t)16 * m * m, gemm_part_need(m, m, (int)T));
  for (int p = 1; p <= p_max; ++p) {
    // candidate p on the columns p_max - p .. n-1: residuals for t = p_max .. n-1
    const double* Xp = X + (p_max - p);
    const int np = (int)T + p;
    s = prec != VL_PREC_FP64 ? var_fit_impl<float>(x, Xp, ldx, m, np, p, Mb, Eb)
                             : var_fit_impl<double>(x, Xp, ldx, m, np, p, Mb, Eb);
    if (s != VL_OK) return s;
    // S = E E^T / T and its Cholesky factor, in FP64; ln det S from the diagonal
    double *S, *dinv, *diag0, *part;
    s = with_workspace(x, [&](Arena& a) {
      S = a.take<double>((size_t)m * m);
      dinv = a.take<double>((size_t)nblk * CHOL_NB * CHOL_NB);
      diag0 = a.take<double>(m);
      part = a.take<double>(part_cap);
    });
    if (s != VL_OK) return s;
    Ctx cx = make_ctx(x, part, part_cap);
    View<double> Ev{Eb, T, 1};
    launch_gemm<double, double>(cx, m, m, (int)T, 1.0 / (double)T, Ev, Ev, 0.0, S, m, false);
    chol_blocked<double>(cx, S, m, m, dinv, diag0);
    launch_logdet_value(S, m, m, pen * p * (double)m * m / (double)T, values + (p - 1), x.st, x.s);
  }
  launch_argmin_p(values, p_max, p_best, x.s);
  return check_launch(h, "vl_var_select");
}

vl_status vl_pairwise_measure(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                              vl_precision prec, double* Hx, double* Hr, double* D) {
  if (!h) return VL_ERR_ARG;
  if (!E) return fail(h, VL_ERR_ARG, "vl_pairwise_measure: E must not be NULL");
  if (!Hx && !Hr && !D) return fail(h, VL_ERR_ARG, "vl_pairwise_measure: no output requested");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (m < 2 || n_eff < 2 || m > VL_MAX_M || lde < n_eff)
    return fail(h, VL_ERR_SHAPE, "vl_pairwise_measure: need 2 <= m <= VL_MAX_M, n_eff >= 2, lde >= n_eff");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return prec != VL_PREC_FP64 ? pairwise_impl<float>(x, E, lde, m, n_eff, Hx, Hr, D, nullptr)
                               : pairwise_impl<double>(x, E, lde, m, n_eff, Hx, Hr, D, nullptr);
}

vl_status vl_causal_order(vl_handle h, const double* D, int m, int32_t* order, double* gap) {
  if (!h) return VL_ERR_ARG;
  if (!D || !order) return fail(h, VL_ERR_ARG, "vl_causal_order: D and order must not be NULL");
  if (m < 1 || m > VL_MAX_M) return fail(h, VL_ERR_SHAPE, "vl_causal_order: need 1 <= m <= VL_MAX_M");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return order_impl(x, D, m, order, gap);
}

vl_status vl_causal_order_certified(vl_handle h, const double* D, const double* E, int64_t lde,
                                    int m, int n_eff, int32_t* order, double* gap,
                                    int32_t* stats) {
  if (!h) return VL_ERR_ARG;
  if (!D || !E || !order)
    return fail(h, VL_ERR_ARG, "vl_causal_order_certified: D, E and order must not be NULL");
  if (m < 2 || n_eff < 2 || m > VL_MAX_M || lde < n_eff)
    return fail(h, VL_ERR_SHAPE,
                "vl_causal_order_certified: need 2 <= m <= VL_MAX_M, n_eff >= 2, lde >= n_eff");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return order_certified_impl(x, D, E, lde, m, n_eff, order, gap, stats);
}

vl_status vl_causal_order_standard(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                                   vl_precision prec, int32_t* order, double* gap) {
  if (!h) return VL_ERR_ARG;
  if (!E || !order)
    return fail(h, VL_ERR_ARG, "vl_causal_order_standard: E and order must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (m < 2 || n_eff < 2 || m > VL_MAX_M || lde < n_eff)
    return fail(h, VL_ERR_SHAPE,
                "vl_causal_order_standard: need 2 <= m <= VL_MAX_M, n_eff >= 2, lde >= n_eff");
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return prec != VL_PREC_FP64 ? order_standard_impl<float>(x, E, lde, m, n_eff, order, gap)
                               : order_standard_impl<double>(x, E, lde, m, n_eff, order, gap);
}

vl_status vl_fit_b(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                   const int32_t* order, const double* M, int p, vl_precision prec, double* B0,
                   double* Btau) {
  if (!h) return VL_ERR_ARG;
  if (!E || !order || !B0) return fail(h, VL_ERR_ARG, "vl_fit_b: E, order and B0 must not be NULL");
  if (p > 0 && Btau && !M) return fail(h, VL_ERR_ARG, "vl_fit_b: Btau requested without M");
  if (m < 2 || n_eff < 2 || p < 0 || m > VL_MAX_M || lde < n_eff)
    return fail(h, VL_ERR_SHAPE, "vl_fit_b: bad sizes");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  DeviceGuard g(h->device);
  Exec x = handle_exec(h);
  return prec == VL_PREC_MIXED
             ? fit_b_impl<float>(x, E, lde, m, n_eff, order, M, p, B0, Btau, nullptr)
             : fit_b_impl<double>(x, E, lde, m, n_eff, order, M, p, B0, Btau, nullptr);
}

vl_status vl_fit(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                 vl_precision prec, double* M, int32_t* order, double* B0, double* Btau,
                 double* D) {
  if (!h) return VL_ERR_ARG;
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  vl_instance I{X, ldx, m, n, p, order, B0, Btau, M, D};
  vl_status s = check_instance(h, I);
  if (s != VL_OK) return s;
  DeviceGuard g(h->device);
  const size_t mm = (size_t)m * m, ne = (size_t)(n - p);
  s = grow(h, &h->sbuf, &h->sbuf_cap, sizeof(double) * (m * ne + 2 * mm) + 1024, h->stream);
  if (s != VL_OK) return s;
  double* E = static_cast<double*>(h->sbuf);
  double* C = E + m * ne;
  if (!D) D = C + mm;
  Exec x = handle_exec(h);
  return prec != VL_PREC_FP64 ? fit_one<float>(x, I, E, C, D, prec == VL_PREC_MIXED_CERTIFIED)
                               : fit_one<double>(x, I, E, C, D);
}

vl_status vl_fit_batched_async(vl_handle h, const vl_instance* inst, int count,
                               vl_precision prec, int32_t* dev_status) {
  if (!h) return VL_ERR_ARG;
  if (count < 0 || (count > 0 && (!inst || !dev_status)))
    return fail(h, VL_ERR_ARG, "vl_fit_batched_async: inst and dev_status must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (prec == VL_PREC_FP64)
    return fail(h, VL_ERR_UNSUPPORTED, "vl_fit_batched_async: mixed precisions only");
  if (count == 0) return VL_OK;
  std::vector<int> idx;
  for (int k = 0; k < count; ++k) {
    const vl_status s = check_instance(h, inst[k]);
    if (s != VL_OK) return s;
    idx.push_back(k);
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return (double)inst[a].m * inst[a].m * inst[a].n > (double)inst[b].m * inst[b].m * inst[b].n;
  });
  DeviceGuard g(h->device);
  cudaMemsetAsync(dev_status, 0, sizeof(int32_t) * count, h->stream);
  return batched_mixed(h, inst, idx, prec == VL_PREC_MIXED_CERTIFIED, dev_status);
}

vl_status vl_fit_batched(vl_handle h, const vl_instance* inst, int count, vl_precision prec,
                         vl_status* inst_status) {
  if (!h) return VL_ERR_ARG;
  if (count < 0 || (count > 0 && (!inst || !inst_status)))
    return fail(h, VL_ERR_ARG, "vl_fit_batched: inst and inst_status must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (count == 0) return VL_OK;
  DeviceGuard g(h->device);
  return batched_impl(h, inst, count, prec, inst_status);
}

vl_status vl_bootstrap_resample(vl_handle h, const double* X, int64_t ldx, int m, int n,
                                int block_len, uint64_t seed, int64_t b0, int nb, double* Xb) {
  if (!h) return VL_ERR_ARG;
  if (!X || !Xb) return fail(h, VL_ERR_ARG, "vl_bootstrap_resample: X and Xb must not be NULL");
  if (m < 1 || n < 1 || nb < 0 || ldx < n || block_len < 1 || block_len > n)
    return fail(h, VL_ERR_SHAPE, "vl_bootstrap_resample: need m, n >= 1, 1 <= block_len <= n");
  if (b0 < 0 || b0 + nb > ((int64_t)1 << 32))
    return fail(h, VL_ERR_SHAPE, "vl_bootstrap_resample: need 0 <= b0, b0 + nb <= 2^32");
  if (nb == 0) return VL_OK;
  DeviceGuard g(h->device);
  launch_boot_resample(X, ldx, m, n, block_len, seed, b0, nb, Xb, h->stream);
  return check_launch(h, "vl_bootstrap_resample");
}

vl_status vl_bootstrap(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                       int n_resamples, int block_len, uint64_t seed, double threshold,
                       vl_precision prec, double* edge_prob, double* order_prob) {
  if (!h) return VL_ERR_ARG;
  if (!X || !edge_prob || !order_prob)
    return fail(h, VL_ERR_ARG, "vl_bootstrap: X, edge_prob and order_prob must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  if (!(threshold >= 0.0)) return fail(h, VL_ERR_ARG, "vl_bootstrap: threshold must be >= 0");
  if (m < 2 || p < 1 || n < 2 || m > VL_MAX_M || ldx < n || block_len < 1 || block_len > n ||
      n_resamples < 1)
    return fail(h, VL_ERR_SHAPE,
                "vl_bootstrap: need m >= 2, p >= 1, 1 <= block_len <= n, n_resamples >= 1");
  if ((int64_t)n - p <= (int64_t)m * p + 1)
    return fail(h, VL_ERR_RANK, "vl_bootstrap: n - p <= m p + 1, the VAR has no unique fit");
  DeviceGuard g(h->device);
  // a chunk of resamples with their fits: X_b, B0, B_tau, M, order, pos
  const size_t mm = (size_t)m * m;
  const size_t per = sizeof(double) * ((size_t)m * n + mm * (1 + 2 * (size_t)p)) +
                     2 * sizeof(int32_t) * m + 4 * 256;
  const size_t budget = (size_t)2 << 30;
  const int chunk = (int)std::min<size_t>({(size_t)n_resamples, (size_t)256,
                                           std::max<size_t>(1, budget / per)});
  vl_status s = grow(h, &h->bootbuf, &h->bootbuf_cap, per * chunk + 1024, h->stream);
  if (s != VL_OK) return s;
  Arena a;
  a.base = static_cast<char*>(h->bootbuf);
  a.cap = h->bootbuf_cap;
  double* Xb = a.take<double>((size_t)chunk * m * n);
  double* B0 = a.take<double>((size_t)chunk * mm);
  double* Bt = a.take<double>((size_t)chunk * p * mm);
  double* M = a.take<double>((size_t)chunk * p * mm);
  int32_t* order = a.take<int32_t>((size_t)chunk * m);
  int32_t* pos = a.take<int32_t>((size_t)chunk * m);
  cudaMemsetAsync(edge_prob, 0, sizeof(double) * mm, h->stream);
  cudaMemsetAsync(order_prob, 0, sizeof(double) * mm, h->stream);
  std::vector<vl_instance> inst(chunk);
  std::vector<vl_status> ist(chunk);
  for (int b0 = 0; b0 < n_resamples; b0 += chunk) {
    const int nb = std::min(chunk, n_resamples - b0);
    launch_boot_resample(X, ldx, m, n, block_len, seed, b0, nb, Xb, h->stream);
    for (int z = 0; z < nb; ++z)
      inst[z] = vl_instance{Xb + (size_t)z * m * n, n, m, n, p, order + (size_t)z * m,
                            B0 + z * mm, Bt + z * p * mm, M + z * p * mm, nullptr};
    s = batched_impl(h, inst.data(), nb, prec, ist.data());
    if (s != VL_OK) return s;
    launch_boot_count(order, B0, m, nb, threshold, pos, edge_prob, order_prob, h->status,
                      h->stream);
  }
  launch_boot_normalize(edge_prob, order_prob, m, n_resamples, h->stream);
  return check_launch(h, "vl_bootstrap");
}

}  // extern "C"
