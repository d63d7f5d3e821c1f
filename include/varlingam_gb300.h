/*
 * varlingam_gb300.h -- C ABI of the GB300 (sm_103a) approximate-ordering
 * VarLiNGAM library (Jiao, Guo, Luk: "Scalable Time-Series Causal Discovery
 * with Approximate Causal Ordering").
 *
 * The method (one series):
 *   1. fit a VAR(p) by least squares and keep its residuals E     (Sec. 4.1)
 *   2. precompute, once, the variable entropies E_x and the entropies E_r of
 *      all m(m-1) standardized pairwise regression residuals, giving the
 *      m x m likelihood-ratio matrix D                   (Sec. 4.2, Eqs. 1-2)
 *   3. order the variables by m greedy argmins of Eq. 3 over that static
 *      matrix                                                  (Algorithm 1)
 *   4. estimate B0 from the order and B_tau = (I - B0) M_tau       (Sec. 4)
 * and, for comparison, the iterative search that step 3 approximates, which
 * re-measures the remaining variables after every pick      (Sec. 3, Eq. 4)
 *
 * Conventions shared by every call:
 *   - All array arguments are DEVICE pointers owned by the caller; the library
 *     never frees or retains them after the call returns.  Matrices are dense,
 *     row-major, FP64 unless stated.
 *   - Calls are asynchronous on the handle's CUDA stream.  Errors detectable on
 *     the host (NULL pointers, bad sizes) return at once and launch nothing.
 *     Errors found on the device (non-finite data, zero variance, a singular
 *     system) are recorded in a sticky status word and returned by vl_sync().
 *   - Outputs are undefined when a call returns an error or when vl_sync()
 *     reports one.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - vl_precision selects the internal arithmetic; user-visible arrays are
 *     FP64 either way.  VL_PREC_MIXED runs the O(m^2 n) and O(m^3) work in
 *     FP32 with compensated FP32 sums and FP64 cross-block reductions;
 *     VL_PREC_FP64 runs every step in FP64 (the plain comparison path).
 *   - The handle grows its device workspace on demand (cudaMalloc).  Call
 *     vl_reserve() first to make later calls allocation-free.
 */
#ifndef VARLINGAM_GB300_H
#define VARLINGAM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vl_handle_s* vl_handle;

typedef enum {
  VL_OK = 0,
  VL_ERR_ARG = 1,         /* NULL pointer or invalid enum                        */
  VL_ERR_SHAPE = 2,       /* sizes out of range (m < 2, p < 1, ld too small ...) */
  VL_ERR_RANK = 3,        /* VAR or B0 normal equations not positive definite,
                             or n - p <= m p + 1 (no unique VAR fit)            */
  VL_ERR_DEGENERATE = 4,  /* a zero-variance variable or a pair with
                             1 - rho^2 < 1e-12 (residual identically zero)      */
  VL_ERR_NONFINITE = 5,   /* NaN or Inf in the input                            */
  VL_ERR_CUDA = 6,        /* a CUDA runtime call failed                         */
  VL_ERR_NOMEM = 7,       /* workspace allocation failed                        */
  VL_ERR_TIMEOUT = 8,     /* a bounded device wait gave up                      */
  VL_ERR_UNSUPPORTED = 9  /* size beyond the library's fixed limits            */
} vl_status;

/* VL_PREC_MIXED_CERTIFIED computes like VL_PREC_MIXED and, in the calls that
 * order (vl_fit, vl_fit_batched), decides every near tie of Eq. 3 on entries
 * of D re-evaluated to FP64 accuracy (see vl_causal_order_certified). */
typedef enum { VL_PREC_FP64 = 0, VL_PREC_MIXED = 1, VL_PREC_MIXED_CERTIFIED = 2 } vl_precision;

/* Largest m any call accepts (the ordering kernel keeps m scores per CTA). */
#define VL_MAX_M 4096

/* Create a handle on CUDA device `device` that issues its work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * workspace_bytes > 0 preallocates that much device workspace.
 * Returns VL_ERR_CUDA if the device cannot be selected. */
vl_status vl_create(vl_handle* out, int device, void* cuda_stream, size_t workspace_bytes);

/* Release the handle and its workspace (synchronises its stream first). */
vl_status vl_destroy(vl_handle h);

/* Change the stream subsequent calls are issued on. */
vl_status vl_set_stream(vl_handle h, void* cuda_stream);

/* Grow the workspace so that every single-series call on sizes up to
 * (m, n, p) runs without allocating. */
vl_status vl_reserve(vl_handle h, int m, int n, int p);

/* Wait for the stream, then return and clear the first device-side error
 * recorded since the last vl_sync (VL_OK if none). */
vl_status vl_sync(vl_handle h);

/* Diagnostics.  vl_profile_events: when both are non-NULL, later calls
 * record start_event / stop_event (cudaEvent_t) on the handle's stream
 * immediately before and after the pairwise-moment kernel, so a caller can
 * time that kernel alone; NULL, NULL turns it off.  vl_kernel_launches:
 * number of CUDA kernels this library has launched in the process. */
vl_status vl_profile_events(vl_handle h, void* start_event, void* stop_event);
unsigned long long vl_kernel_launches(void);

/* Diagnostic, no counterpart in the paper: the measured throughput of the
 * special-function unit on device `device`, in results per clock per SM, of
 * ex2.approx.f32 and lg2.approx.f32 (the instructions the pairwise kernel's
 * exponentials and logarithms use).  Synchronous; allocates two small
 * buffers.  VL_ERR_ARG for NULL outputs. */
vl_status vl_sfu_rate(int device, double* ex2_per_clk_sm, double* lg2_per_clk_sm);

/* Human-readable text of the last error on this handle (never NULL). */
const char* vl_last_error(vl_handle h);

/*
 * VAR(p) least-squares fit with intercept (Sec. 4.1; Sec. 2.1: VarLiNGAM
 * fits a VAR first and passes its residuals on):
 *     x_t = c + sum_{tau=1..p} M_tau x_{t-tau} + e_t ,   t = p .. n-1.
 * X   : m x n, row i = variable i over time, row stride ldx >= n (elements).
 * M   : output, p*m*m, M[(tau-1)*m*m + i*m + k] = effect of x_k(t-tau) on x_i(t).
 * E   : output, m x (n-p) residuals, row stride n-p.  May be NULL.
 * Requires m >= 2, p >= 1, n - p > m p + 1 (else VL_ERR_RANK).
 */
vl_status vl_var_fit(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                     vl_precision prec, double* M, double* E);

/*
 * Lag order of the VAR by an information criterion (the paper takes p as
 * given, Sec. 4.1; the criteria are standard VAR practice).  Every candidate
 * p = 1..p_max is fitted as by vl_var_fit (precision prec) on the same
 * T = n - p_max equations t = p_max..n-1, so the fits compare the same data;
 * its ML residual covariance S(p) = E E^T / T is formed and factored in FP64,
 * and
 *     AIC(p) = ln det S(p) + 2 p m^2 / T
 *     BIC(p) = ln det S(p) + ln(T) p m^2 / T
 *     HQ(p)  = ln det S(p) + 2 ln(ln T) p m^2 / T
 * (the m intercepts, common to every p, are left out).  The smallest value
 * wins; ties pick the smaller p.
 * X      : m x n, row stride ldx (device).
 * values : output, p_max doubles (device): the criterion for p = 1..p_max.
 * p_best : output, one int32 (device): the chosen p.
 * Requires m >= 2, p_max >= 1 and n - p_max > m (p_max + 1), so that the
 * largest candidate's residual covariance can be of full rank (else
 * VL_ERR_RANK).
 * A residual covariance that is not positive definite sets VL_ERR_RANK on
 * the device (reported by vl_sync).  The fits' residuals and coefficients
 * live in a buffer of the handle, allocated on the first call of a size.
 */
typedef enum { VL_IC_AIC = 0, VL_IC_BIC = 1, VL_IC_HQ = 2 } vl_criterion;
vl_status vl_var_select(vl_handle h, const double* X, int64_t ldx, int m, int n, int p_max,
                        vl_criterion crit, vl_precision prec, double* values, int32_t* p_best);

/*
 * One-time pairwise precomputation (Sec. 4.2 items 1-2; Algorithm 1, the two
 * precompute calls; Eqs. 1-2 of Sec. 3).  Each row of E is standardized
 * (population variance).  For every ordered pair (i, j), i != j, the residual
 * r_{i<-j} = x_i - rho_ij x_j (Eq. 1) is rescaled to unit variance and its
 * entropy approximated by
 *     H(u) = (1 + log 2 pi)/2 - k1 (E log cosh u - gamma)^2 - k2 (E u e^{-u^2/2})^2
 * with k1 = 79.047, k2 = 7.4129, gamma = 0.37457.
 * E   : m x n_eff, row stride lde >= n_eff.
 * Hx  : output m,   Hx[i] = H(x_i)                       (may be NULL)
 * Hr  : output m*m, Hr[i*m+j] = H(r_{i<-j}), diagonal 0  (may be NULL)
 * D   : output m*m, D[i*m+j] = Hx[j] + Hr[i*m+j] - Hx[i] - Hr[j*m+i]
 *       (= T_{j<-i} - T_{i<-j}; > 0 favours i -> j; antisymmetric).
 * Requires m >= 2, n_eff >= 2.
 */
vl_status vl_pairwise_measure(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                              vl_precision prec, double* Hx, double* Hr, double* D);

/*
 * Algorithm 1 over the static matrix D: for k = 1..m pick
 *     c_k = argmin_{i in U} sum_{j in U, j != i} min(0, D[i*m+j])^2      (Eq. 3)
 * (ties -> lowest index), append it, remove it from U.
 * order : output m int32 (causes first).
 * gap   : output m doubles or NULL; gap[k] = (S_2nd - S_min) / max(|S_min|,
 *         |S_2nd|, 1e-300) at step k (+inf when one candidate is left).
 */
vl_status vl_causal_order(vl_handle h, const double* D, int m, int32_t* order, double* gap);

/*
 * Algorithm 1 over a D measured in VL_PREC_MIXED, with its near ties decided
 * to FP64 accuracy (Algorithm 1 and Eq. 3; Eqs. 1-2 for the re-evaluated
 * entries).
 * The FP32 measure carries errors of about 1e-6 of max|D|, which move the
 * scores of Eq. 3 by about 5e-5 relative; two candidates closer than that may
 * swap.  After the search on D, every step whose picked score and some other
 * candidate's score overlap within their error bands
 *     band(S) = 1e-3 S + 1e-5 max|D| sqrt(S) + u (1e-5 max|D|)^2
 * (u = variables remaining) is re-decided on exact scores: the entries D_ij
 * of its candidates against the remaining variables are recomputed from E:
 * the standardization in FP64, rho, both standardized residuals and the
 * per-sample functions of their entropies in double-float arithmetic (pairs
 * of FP32 numbers, about 48 bits; the per-sample values within 3e-14 of
 * FP64), the sums, entropies and scores in FP64, and the argmin taken (ties:
 * lowest index).  If a
 * pick changes, the search resumes from that step with the corrected pick and
 * the steps after it are checked again (up to three rounds).  The result is
 * then the order Algorithm 1 gives on the FP64 measure wherever the FP64
 * scores of a step differ by more than the bands.
 * D     : m x m, as vl_pairwise_measure wrote it from E (VL_PREC_MIXED).
 * E     : the m x n_eff data D was measured from, row stride lde >= n_eff.
 * order : output m int32.   gap : output m doubles or NULL (as vl_causal_order,
 *         from the FP32 scores of the final order).
 * stats : output 4 int32 (device) or NULL: steps re-decided, pairs re-evaluated,
 *         picks changed, steps left as the FP32 search took them
 *         (more than 16 candidates, or after a change in the last round).
 * Asynchronous, no host synchronisation; workspace about 12 m^2 + 8 m n_eff
 * bytes plus the ordering's.  Requires 2 <= m <= VL_MAX_M, n_eff >= 2.
 */
vl_status vl_causal_order_certified(vl_handle h, const double* D, const double* E, int64_t lde,
                                    int m, int n_eff, int32_t* order, double* gap,
                                    int32_t* stats);

/*
 * Allocation-free variant of vl_causal_order (same search, same results).
 * This entry point has no counterpart in the paper; it exists for callers that
 * cannot allocate device memory when they need the ordering: frameworks and
 * serving runtimes that own all device memory through their own pooling
 * allocator (a stray cudaMalloc would bypass their accounting, or fail when
 * the pool has already taken the free memory), and latency-bound loops that
 * must not pay for an allocation, which synchronises the device.  It needs no handle and
 * allocates nothing: its scratch is a fixed device array inside the library
 * (about 2.1 MB, held on every GPU that loads the library until the process
 * exits), so it accepts 1 <= m <= VL_NOALLOC_MAX_M and returns
 * VL_ERR_UNSUPPORTED above that.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress); make this first call before any stream capture.
 *  - All calls share the one array: calls that may overlap on the GPU (on
 *    different streams without ordering between them) race.  A call needs no
 *    zeroed scratch: it writes every scratch element before reading it.
 *  - Work is queued on cuda_stream (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns without waiting.  Only host-side argument
 *    errors are reported; non-finite entries of D are not detected here (use
 *    vl_causal_order when D is not known to be finite).
 */
#define VL_NOALLOC_MAX_M 512
vl_status vl_causal_order_noalloc(void* cuda_stream, const double* D, int m, int32_t* order,
                                  double* gap);

/*
 * The iterative DirectLiNGAM search (Sec. 3, steps 1-5), the method that
 * Algorithm 1 approximates: with U = all variables, repeat until one is left
 *   1. standardize every x_i, i in U (population variance);
 *   2-3. the pairwise measure D over U, as vl_pairwise_measure computes it
 *        (Eqs. 1-2), on the CURRENT data;
 *   4. pick c = argmin_{i in U} sum_{j in U, j != i} min(0, D_ij)^2 (Eq. 3;
 *      ties -> lowest index), append it to the order, remove it from U;
 *   5. replace every x_j, j in U, by its residual on the pick,
 *      x_j - cov(x_j, x_c) / var(x_c) x_c (Eq. 4).
 * The last variable closes the order.  Cost: sum over u = m..2 of the
 * measure of u variables, about m/3 times the pairwise work of Algorithm 1.
 * E     : m x n_eff data (the VAR residuals), row stride lde >= n_eff; read only.
 * prec  : the precision of each pairwise measure (as vl_pairwise_measure).
 *         Step 5 is applied in FP64 with the slopes taken from the centred
 *         cross products the measure computes for its correlations (FP64,
 *         or in VL_PREC_MIXED split-FP32 products summed in double-float,
 *         relative error about 1e-8).
 * order : output m int32 (causes first).
 * gap   : output m doubles or NULL; gap[k] = relative gap between the two
 *         smallest scores of iteration k, as in vl_causal_order (+inf last).
 * Runs asynchronously on the handle's stream with no host synchronisation
 * (the picks stay on the device); its buffers are the handle's series
 * buffers (shared with vl_fit, about 2 m n_eff + 2 m^2 + 2 m doubles) and workspace,
 * so after a first call of the same or larger size it allocates nothing.
 * Device errors (degenerate or non-finite data at any iteration) surface at
 * vl_sync().  Requires 2 <= m <= VL_MAX_M, n_eff >= 2.
 */
vl_status vl_causal_order_standard(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                                   vl_precision prec, int32_t* order, double* gap);

/*
 * B0 and B_tau from a causal order (Sec. 4: the instantaneous matrix of
 * VarLiNGAM): row order[k] of B0 holds the least-squares coefficients of
 * e_{order[k]} on e_{order[0..k-1]}; then B_tau = (I - B0) M_tau.
 * E     : m x n_eff residuals, row stride lde.   order : m int32 (device).
 * M     : p*m*m as produced by vl_var_fit (may be NULL when Btau is NULL).
 * prec  : VL_PREC_MIXED factors the permuted covariance in FP32 (B0 error
 *         ~1e-6 for well-conditioned residuals), VL_PREC_FP64 in FP64.
 * B0    : output m*m, B0[i*m+j] = effect of j on i.
 * Btau  : output p*m*m (may be NULL when p == 0 or not wanted).
 */
vl_status vl_fit_b(vl_handle h, const double* E, int64_t lde, int m, int n_eff,
                   const int32_t* order, const double* M, int p, vl_precision prec,
                   double* B0, double* Btau);

/*
 * The whole method (steps 1-4 above) for one series, asynchronously on the
 * handle's stream: VAR fit, pairwise measure, Algorithm 1, B0 and B_tau.  The
 * residual covariance is computed once and shared by the measure and B0
 * steps.  No host synchronisation; device errors surface at vl_sync().  After
 * a first call has sized the workspace, later calls with the same or smaller
 * sizes allocate nothing (they can then be captured in a CUDA graph).
 * X : m x n (row stride ldx).  Outputs: M p*m*m, order m, B0 m*m, Btau p*m*m,
 * D m*m (may be NULL).
 */
vl_status vl_fit(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                 vl_precision prec, double* M, int32_t* order, double* B0, double* Btau,
                 double* D);

/* One series for the batched call.  Device pointers; D may be NULL. */
typedef struct {
  const double* X;  /* m x n, row stride ldx                 */
  int64_t ldx;
  int m, n, p;
  int32_t* order;   /* out: m                                 */
  double* B0;       /* out: m*m                               */
  double* Btau;     /* out: p*m*m                             */
  double* M;        /* out: p*m*m                             */
  double* D;        /* out: m*m or NULL                       */
} vl_instance;

/*
 * The whole method (steps 1-4 above) for `count` independent series of
 * possibly different (m, n, p).  Mixed precisions run the phase-major batch
 * of vl_fit_batched_async; VL_PREC_FP64 deals the series, largest first, to a
 * pool of up to 32 streams forked from the handle's stream and joined back
 * into it; each stream has its own workspace.  inst and inst_status are HOST
 * arrays of length count; inst_status[k] receives the instance's own status
 * after the call has completed (the call synchronises the stream).  An
 * instance that fails the host checks reports that error and is skipped; when
 * the call fails as a whole (workspace or stream creation, a CUDA error),
 * every other instance reports that error.  Returns the first non-OK
 * instance status, or a host-side error.
 */
vl_status vl_fit_batched(vl_handle h, const vl_instance* inst, int count, vl_precision prec,
                         vl_status* inst_status);

/*
 * The whole method for `count` series in a mixed precision (VL_PREC_MIXED or
 * VL_PREC_MIXED_CERTIFIED), enqueued on the handle's stream without any host
 * synchronisation (the batched form of vl_fit).  Phase-major: (A) every
 * series' VAR fit and the measure's preparation on a pool of streams forked
 * from the handle's stream, (B) ONE launch of the pairwise-moment kernel over
 * a device list of (series, pair tile, sample split) work items of all
 * series, largest first, (C) every series' finalisation of the measure,
 * ordering and B0 / B_tau on the pool, joined back into the handle's stream.
 * The length of the sample splits of (B) is tuned on the first call of a
 * batch shape (every candidate timed, the fastest cached in the handle).
 * dev_status: DEVICE array of count int32, zeroed by the call, receiving each
 * series' device-detected status (vl_status codes).  Host-side errors of any
 * series fail the call as a whole (nothing is launched).  After one call with
 * the same instances, sizes and precision, a call allocates nothing, uploads
 * nothing and can be captured into a CUDA graph; a call under capture that
 * would need either returns VL_ERR_UNSUPPORTED.  VL_PREC_FP64 is not
 * accepted (use vl_fit_batched).
 */
vl_status vl_fit_batched_async(vl_handle h, const vl_instance* inst, int count,
                               vl_precision prec, int32_t* dev_status);

/*
 * Bootstrap (no counterpart in the paper, which reports single fits): the
 * moving-block bootstrap of Kuensch (1989), which keeps the serial
 * dependence a VAR model relies on within blocks of block_len consecutive
 * time points.  Resample b (0 <= b < 2^32) of the m x n series is the
 * concatenation of blocks k = 0, 1, ... starting at time
 *   s_k = floor(u_k (n - block_len + 1) / 2^64),
 * cut to n points, where u_k is output number b 2^32 + k + 1 of SplitMix64
 * (Steele, Lea and Flood 2014) seeded with `seed`:
 *   u = mix(seed + c * 0x9E3779B97F4A7C15) mod 2^64 for output number c.
 * The generator is counter based, so resample b is the same however many
 * resamples a call asks for.
 *
 * vl_bootstrap_resample: resamples b0 .. b0 + nb - 1 of X (device, m x n,
 * row stride ldx) into Xb (device, nb blocks of m x n, row stride n, block z
 * = resample b0 + z).  Needs 1 <= block_len <= n and b0 + nb <= 2^32 (else
 * VL_ERR_SHAPE).  Asynchronous on the handle's stream; allocates nothing.
 *
 * vl_bootstrap: the whole method (vl_fit, steps 1-4) on resamples
 * 0 .. n_resamples - 1 and, over them (device outputs, m x m row-major),
 *   edge_prob[i][j]  = fraction of resamples with |B0[i][j]| > threshold,
 *   order_prob[i][j] = fraction of resamples whose causal order puts i
 *                      before j (0 on the diagonal).
 * The resamples are fitted in chunks through the batched path
 * (vl_fit_batched) in the given precision, in a handle-owned buffer of at
 * most about 2 GiB; the call synchronises the stream after every chunk.
 * The first failed fit of a resample fails the call with its status.
 * Needs m >= 2, p >= 1, n - p > m p + 1 (else VL_ERR_RANK), threshold >= 0
 * (else VL_ERR_ARG).
 */
vl_status vl_bootstrap_resample(vl_handle h, const double* X, int64_t ldx, int m, int n,
                                int block_len, uint64_t seed, int64_t b0, int nb, double* Xb);
vl_status vl_bootstrap(vl_handle h, const double* X, int64_t ldx, int m, int n, int p,
                       int n_resamples, int block_len, uint64_t seed, double threshold,
                       vl_precision prec, double* edge_prob, double* order_prob);

#ifdef __cplusplus
}
#endif

#endif /* VARLINGAM_GB300_H */
