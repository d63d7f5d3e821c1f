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

// Carve a workspace layout twice: once to measure, once for real.
template <class F>
vl_status with_workspace(vl_handle h, F&& carve) {
  Arena probe;
  probe.base = nullptr;
  carve(probe);
  vl_status s = ensure_ws(h, probe.off + 512);
  if (s != VL_OK) return s;
  Arena a;
  a.base = static_cast<char*>(h->ws);
  a.cap = h->ws_cap;
  carve(a);
  return VL_OK;
}

Ctx make_ctx(vl_handle h, double* part, size_t part_cap) {
  return Ctx{h->stream, h->status, part, part_cap, h->num_sms};
}

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------- VAR fit
template <class T>
vl_status var_fit_impl(vl_handle h, const double* X, int64_t ldx, int m, int n, int p, double* M,
                       double* E) {
  const int n_eff = n - p, mp = m * p, q = m * (p + 1);
  const int64_t ldc = round_up(n, 4);
  const int nblk = (mp + CHOL_NB - 1) / CHOL_NB;
  const size_t part_cap = (size_t)16 * std::max((size_t)m * m, (size_t)mp * mp);
  T *Xc, *Gzz, *Gzy, *dinv;
  double *mu, *wbar, *G, *cst, *Ew, *part, *diag0;
  vl_status s = with_workspace(h, [&](Arena& a) {
    Xc = a.take<T>((size_t)m * ldc);
    mu = a.take<double>(m);
    wbar = a.take<double>((size_t)(p + 1) * m);
    G = a.take<double>((size_t)mp * q);
    Gzz = a.take<T>((size_t)mp * mp);
    Gzy = a.take<T>((size_t)mp * m);
    dinv = a.take<T>((size_t)nblk * CHOL_NB * CHOL_NB);
    cst = a.take<double>(m);
    diag0 = a.take<double>(mp);
    Ew = E ? nullptr : a.take<double>((size_t)m * n_eff);
    part = a.take<double>(part_cap);
  });
  if (s != VL_OK) return s;
  if (!E) E = Ew;
  Ctx cx = make_ctx(h, part, part_cap);
  cudaStream_t st = h->stream;
  launch_var_prep<T>(X, ldx, m, n, p, Xc, ldc, mu, wbar, h->status, st);
  // lagged Gram: rows of Z (lags 1..p) against rows of W = [Y; Z]
  for (int t1 = 1; t1 <= p; ++t1)
    for (int b2 = 0; b2 <= p; ++b2) {
      View<T> A{Xc + (p - t1), ldc, 1};
      View<T> B{Xc + (p - b2), ldc, 1};
      launch_gemm<T, double>(cx, m, m, n_eff, 1.0, A, B, 0.0,
                             G + (int64_t)(t1 - 1) * m * q + (int64_t)b2 * m, q, false);
    }
  launch_var_normal_eq<T>(G, m, p, n_eff, wbar, Gzz, Gzy, st);
  chol_blocked<T>(cx, Gzz, mp, mp, dinv, diag0);
  chol_solve_blocked<T>(cx, Gzz, mp, dinv, mp, Gzy, m, m, true);
  launch_var_coef<T>(Gzy, m, p, wbar, M, cst, st);
  launch_var_resid_init(X, ldx, m, n, p, mu, cst, E, n_eff, st);
  for (int tau = 1; tau <= p; ++tau) {
    View<T> A{Gzy + (int64_t)(tau - 1) * m * m, 1, m};  // A(i, k) = M_tau[i][k]
    View<T> B{Xc + (p - tau), 1, ldc};                 // B(t, k) = Xc[k][p - tau + t]
    launch_gemm<T, double>(cx, m, n_eff, m, -1.0, A, B, 1.0, E, n_eff, false);
  }
  return check_launch(h, "vl_var_fit");
}

// ------------------------------------------------------- pairwise measure
struct CovOut {
  double* C;  // m x m centred cross products
  double* mu;
  double* isd;
  double* hx;  // 2m moments of the standardized variables
};

template <class T>
void cov_and_stats(vl_handle h, const Ctx& cx, const double* E, int64_t lde, int m, int n,
                   const CovOut& o, void* scratch) {
  cudaStream_t st = h->stream;
  launch_standardize<T>(E, lde, m, n, o.mu, o.isd, o.hx, h->status, st);
  const int64_t ldc = round_up(n, 4);
  if constexpr (sizeof(T) == 4) {
    float* hi = static_cast<float*>(scratch);
    float* lo = hi + (size_t)m * ldc;
    launch_split_center(E, lde, m, n, o.mu, hi, lo, ldc, st);
    View<float> Vh{hi, ldc, 1}, Vl{lo, ldc, 1};
    launch_gemm_split(cx, m, m, n, Vh, Vl, Vh, Vl, o.C, m, true);
  } else {
    double* ec = static_cast<double*>(scratch);
    launch_center64(E, lde, m, n, o.mu, ec, ldc, st);
    View<double> V{ec, ldc, 1};
    launch_gemm<double, double>(cx, m, m, n, 1.0, V, V, 0.0, o.C, m, false);
  }
}

template <class T>
size_t cov_scratch_bytes(int m, int n) {
  const int64_t ldc = round_up(n, 4);
  return sizeof(T) == 4 ? 2 * sizeof(float) * (size_t)m * ldc : sizeof(double) * (size_t)m * ldc;
}

template <class T>
vl_status pairwise_impl(vl_handle h, const double* E, int64_t lde, int m, int n, double* Hx,
                        double* Hr, double* D, double* C_out) {
  const bool f32 = sizeof(T) == 4;
  PairPlan pl = plan_pairwise(m, n, h->num_sms, !f32);
  const size_t part_cap = (size_t)16 * m * m;
  const size_t nparts = (size_t)pl.splits * (f32 ? 3 : 2) * m * m;
  CovOut o;
  void* scratch;
  float *rho32 = nullptr, *c32 = nullptr;
  double* rho64 = nullptr;
  T* xt;
  double *pparts, *gpart, *Hr_w, *D_w;
  vl_status s = with_workspace(h, [&](Arena& a) {
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
  if (s != VL_OK) return s;
  if (!Hr) Hr = Hr_w;
  if (!D) D = D_w;
  Ctx cx = make_ctx(h, gpart, part_cap);
  cudaStream_t st = h->stream;
  cov_and_stats<T>(h, cx, E, lde, m, n, o, scratch);
  launch_pair_consts(o.C, m, rho32, c32, rho64, h->status, st);
  launch_transpose_std<T>(E, lde, m, n, o.mu, o.isd, xt, pl.m_pad, pl.n_pad, st);
  if (h->prof_start) cudaEventRecord(h->prof_start, st);
  if constexpr (sizeof(T) == 4)
    launch_pairwise_f32(xt, pl, rho32, c32, pparts, st);
  else
    launch_pairwise_f64(xt, pl, rho64, pparts, st);
  if (h->prof_stop) cudaEventRecord(h->prof_stop, st);
  launch_measure_finalize(pparts, pl, o.hx, Hx, Hr, D, f32, st);
  return check_launch(h, "vl_pairwise_measure");
}

// ---------------------------------------------------------------- B0
template <class T>
vl_status fit_b_impl(vl_handle h, const double* E, int64_t lde, int m, int n,
                     const int32_t* order, const double* M, int p, double* B0, double* Btau,
                     const double* C_in) {
  const int nblk = (m + CHOL_NB - 1) / CHOL_NB;
  const size_t part_cap = (size_t)16 * m * m;
  CovOut o{};
  void* scratch = nullptr;
  T *Sp, *dinv, *R, *IBt = nullptr, *Mt = nullptr;
  double *IB, *gpart, *diag0;
  vl_status s = with_workspace(h, [&](Arena& a) {
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
  if (s != VL_OK) return s;
  Ctx cx = make_ctx(h, gpart, part_cap);
  cudaStream_t st = h->stream;
  const double* C = C_in;
  if (!C) {
    cov_and_stats<T>(h, cx, E, lde, m, n, o, scratch);
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
  return check_launch(h, "vl_fit_b");
}

vl_status validate_prec(vl_handle h, vl_precision prec) {
  if (prec != VL_PREC_FP64 && prec != VL_PREC_MIXED)
    return fail(h, VL_ERR_ARG, "precision must be VL_PREC_FP64 or VL_PREC_MIXED");
  return VL_OK;
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
  return prec == VL_PREC_MIXED ? var_fit_impl<float>(h, X, ldx, m, n, p, M, E)
                               : var_fit_impl<double>(h, X, ldx, m, n, p, M, E);
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
  return prec == VL_PREC_MIXED ? pairwise_impl<float>(h, E, lde, m, n_eff, Hx, Hr, D, nullptr)
                               : pairwise_impl<double>(h, E, lde, m, n_eff, Hx, Hr, D, nullptr);
}

vl_status vl_causal_order(vl_handle h, const double* D, int m, int32_t* order, double* gap) {
  if (!h) return VL_ERR_ARG;
  if (!D || !order) return fail(h, VL_ERR_ARG, "vl_causal_order: D and order must not be NULL");
  if (m < 1 || m > VL_MAX_M) return fail(h, VL_ERR_SHAPE, "vl_causal_order: need 1 <= m <= VL_MAX_M");
  DeviceGuard g(h->device);
  double* Pt;
  vl_status s = with_workspace(h, [&](Arena& a) { Pt = a.take<double>((size_t)m * m); });
  if (s != VL_OK) return s;
  launch_causal_order(D, m, Pt, order, gap, h->status, h->stream);
  return check_launch(h, "vl_causal_order");
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
  return prec == VL_PREC_MIXED
             ? fit_b_impl<float>(h, E, lde, m, n_eff, order, M, p, B0, Btau, nullptr)
             : fit_b_impl<double>(h, E, lde, m, n_eff, order, M, p, B0, Btau, nullptr);
}

vl_status vl_fit_batched(vl_handle h, const vl_instance* inst, int count, vl_precision prec,
                         vl_status* inst_status) {
  if (!h) return VL_ERR_ARG;
  if (count < 0 || (count > 0 && (!inst || !inst_status)))
    return fail(h, VL_ERR_ARG, "vl_fit_batched: inst and inst_status must not be NULL");
  if (validate_prec(h, prec) != VL_OK) return VL_ERR_ARG;
  DeviceGuard g(h->device);
  vl_status first = VL_OK;
  for (int k = 0; k < count; ++k) {
    const vl_instance& I = inst[k];
    vl_status s = VL_OK;
    if (!I.X || !I.order || !I.B0 || !I.M || (I.p > 0 && !I.Btau))
      s = fail(h, VL_ERR_ARG, "vl_fit_batched: NULL pointer in instance");
    else if (I.m < 2 || I.p < 1 || I.n < 2 || I.m > VL_MAX_M || I.ldx < I.n)
      s = fail(h, VL_ERR_SHAPE, "vl_fit_batched: bad sizes");
    else if ((int64_t)I.n - I.p <= (int64_t)I.m * I.p + 1)
      s = fail(h, VL_ERR_RANK, "vl_fit_batched: n - p <= m p + 1");
    if (s == VL_OK) {
      const int m = I.m, n_eff = I.n - I.p;
      // per-instance buffers that the caller does not provide live at the
      // top of the workspace growth: allocate them separately
      double *E = nullptr, *D = I.D, *C = nullptr;
      size_t bytes = sizeof(double) * ((size_t)m * n_eff + (I.D ? 0 : (size_t)m * m) + (size_t)m * m);
      void* blk = nullptr;
      if (cudaMalloc(&blk, bytes) != cudaSuccess) {
        cudaGetLastError();
        s = fail(h, VL_ERR_NOMEM, "vl_fit_batched: instance buffer allocation failed");
      } else {
        E = static_cast<double*>(blk);
        C = E + (size_t)m * n_eff;
        if (!D) D = C + (size_t)m * m;
        if (prec == VL_PREC_MIXED) {
          s = var_fit_impl<float>(h, I.X, I.ldx, m, I.n, I.p, I.M, E);
          if (s == VL_OK) s = pairwise_impl<float>(h, E, n_eff, m, n_eff, nullptr, nullptr, D, C);
        } else {
          s = var_fit_impl<double>(h, I.X, I.ldx, m, I.n, I.p, I.M, E);
          if (s == VL_OK) s = pairwise_impl<double>(h, E, n_eff, m, n_eff, nullptr, nullptr, D, C);
        }
        if (s == VL_OK) {
          double* Pt;
          s = with_workspace(h, [&](Arena& a) { Pt = a.take<double>((size_t)m * m); });
          if (s == VL_OK) launch_causal_order(D, m, Pt, I.order, nullptr, h->status, h->stream);
        }
        if (s == VL_OK) {
          if (prec == VL_PREC_MIXED)
            s = fit_b_impl<float>(h, E, n_eff, m, n_eff, I.order, I.M, I.p, I.B0, I.Btau, C);
          else
            s = fit_b_impl<double>(h, E, n_eff, m, n_eff, I.order, I.M, I.p, I.B0, I.Btau, C);
        }
        vl_status sy = vl_sync(h);
        if (s == VL_OK) s = sy;
        cudaFree(blk);
      }
    }
    inst_status[k] = s;
    if (first == VL_OK && s != VL_OK) first = s;
  }
  return first;
}

}  // extern "C"
