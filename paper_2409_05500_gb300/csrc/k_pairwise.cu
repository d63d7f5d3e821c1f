// The one-time O(m^2 n) pairwise precomputation (Sec. 4.2 items 1-2 and
// Algorithm 1's two precompute calls; Eqs. 1-2 of Sec. 3).
//
// For every unordered pair i < j and every sample t the two standardized
// regression residuals are
//     u_t = s (x_i[t] - rho x_j[t]),   v_t = s (x_j[t] - rho x_i[t]),
//     s = (1 - rho^2)^{-1/2},
// and H needs, per residual, A = mean log cosh u and B = mean u exp(-u^2/2).
//
// FP32 kernel arithmetic (per residual stream, per sample):
//     w    = kappa s r                  kappa = 2 log2(e), so 2^{-|w|} = e^{-2|u|}
//     y    = ex2(-|w|)                  (MUFU)
//     prod = prod * (1 + y)             log cosh u = |u| + ln(1 + y) - ln 2
//     ra  += |w|
//     g    = ex2(-w^2 / (8 log2 e))     = e^{-u^2/2}   (MUFU)
//     rb  += w g
// Every KRUN = 16 samples the run's log-cosh sum
//     sum_t log cosh u_t = ra / kappa + ln 2 (log2(prod) - 16)
// (one MUFU lg2 per run) and its sb are Kahan-added into FP32 (sum, comp)
// pairs.  The two j's of a thread's micro-tile are processed as one float2
// with the paired FP32 instructions of this architecture (fma/mul/add .f32x2),
// which halves the FP32 instruction count; the exponentials stay scalar MUFU.
// The split partials are combined in double-float arithmetic by
// measure_finalize.
//
// Padding: x is zero beyond n (time) and beyond m (variables).  A zero sample
// gives |w| = 0, 1 + y = 2 (log2 adds exactly 1, cancelled by the -16 per
// run) and w g = 0, i.e. it contributes exactly 0: padding needs no masking.
#include <algorithm>
#include <cmath>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int TB = 32;        // variables per tile side
constexpr int TT = 128;       // samples per shared-memory stage
constexpr int KRUN = 16;      // samples per product/Kahan run (product <= 2^16)
constexpr int NTH = 256;      // FP64 kernel threads: 16 x 16, each a 2 x 2 pair micro-tile
constexpr float KAPPA = 2.8853900817779268f;       // 2 log2(e)
constexpr float GAUSS_K = -0.08664339756999316f;   // -1 / (8 log2 e)

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// tile index -> (I, J), I <= J, row-major over the upper triangle
__device__ __forceinline__ void tile_coords(int q, int T, int& I, int& J) {
  int i = 0, rem = q;
  while (rem >= T - i) {
    rem -= T - i;
    ++i;
  }
  I = i;
  J = i + rem;
}

// State of two residual streams (the two j's of a micro-tile row), as float2.
struct Pair2 {
  float2 prod, ra, rb;      // current 16-sample run
  float2 sa, ca, sb, cb;    // Kahan (sum, compensation) of the run sums
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// (S, C) += x, Kahan, both lanes at once
__device__ __forceinline__ void kahan2(float2& S, float2& C, float2 x) {
  const float2 mone = f2(-1.f, -1.f);
  const float2 y = __ffma2_rn(C, mone, x);  // x - C
  const float2 t = __fadd2_rn(S, y);
  C = __ffma2_rn(y, mone, __ffma2_rn(S, mone, t));  // (t - S) - y
  S = t;
}

// Thread -> MTI x 2 pair micro-tile (ti, tj) of tile (I, J), enumerating only
// micro-tiles holding at least one pair i < j < m; returns false for threads
// beyond that count.  Micro-tile (ti, tj) covers i = MTI ti + a, j = 2 tj + b.
template <int MTI>
__device__ __forceinline__ bool micro_tile(int s, int I, int J, int m, int& ti, int& tj) {
  constexpr int R = TB / MTI;                     // micro-rows
  const int lim = min(16, (m - J * TB + 1) / 2);  // micro-columns with some j < m
  if (I < J) {
    ti = s / lim;
    tj = s % lim;
    if (ti < R) return true;
  } else {
    // diagonal tile: row ti needs 2 tj + 1 > MTI ti, i.e. tj >= (MTI ti + 1) / 2
    for (int r = 0; r < R; ++r) {
      const int st = (MTI * r + 1) / 2;
      const int len = lim - st;
      if (len <= 0) break;
      if (s < len) {
        ti = r;
        tj = st + s;
        return true;
      }
      s -= len;
    }
  }
  ti = 0;
  tj = 0;
  return false;
}

// One sample of one stream pair: residual R (both lanes), scale C.
__device__ __forceinline__ void step2(Pair2& q, float2 R, float2 C, float2 KK) {
  const float2 W = __fmul2_rn(C, R);
  const float2 Y = f2(ex2_approx(-fabsf(W.x)), ex2_approx(-fabsf(W.y)));
  q.prod = __ffma2_rn(q.prod, Y, q.prod);
  q.ra.x += fabsf(W.x);
  q.ra.y += fabsf(W.y);
  const float2 E = __fmul2_rn(__fmul2_rn(W, KK), W);
  const float2 G = f2(ex2_approx(E.x), ex2_approx(E.y));
  q.rb = __ffma2_rn(W, G, q.rb);
}

__device__ __forceinline__ void end_run2(Pair2& q) {
  const float2 L = f2(lg2_approx(q.prod.x), lg2_approx(q.prod.y));
  const float ik = 1.f / KAPPA;
  const float m16 = -16.f * 0.69314718055994531f;
  // sum log cosh over the run = ra / kappa + ln 2 (log2 prod - 16)
  const float2 run =
      __ffma2_rn(L, f2(0.69314718055994531f, 0.69314718055994531f),
                 __ffma2_rn(q.ra, f2(ik, ik), f2(m16, m16)));
  kahan2(q.sa, q.ca, run);
  kahan2(q.sb, q.cb, q.rb);
  q.prod = f2(1.f, 1.f);
  q.ra = f2(0.f, 0.f);
  q.rb = f2(0.f, 0.f);
}

// MTI x 2 pair micro-tiles, (32 / MTI) x 16 threads per 32 x 32 tile, TTS
// samples per shared-memory stage, MINB CTAs per SM.
// One work item: pair tile `tile` of the upper triangle, sample split `split`.
template <int MTI, int TTS>
__device__ __forceinline__ void pairwise_f32_item(int tile, int split,
                                                  const float* __restrict__ xt, int m, int m_pad,
                                                  int T, int n_run, int tps,
                                                  const float* __restrict__ rho32,
                                                  const float* __restrict__ c32,
                                                  float* __restrict__ part) {
  constexpr int NT = TB / MTI * 16;
  extern __shared__ __align__(16) float pw_smem[];
  float(*sx)[TTS][2 * TB] = reinterpret_cast<float(*)[TTS][2 * TB]>(pw_smem);  // [3][TTS][64]
  int I, J;
  tile_coords(tile, T, I, J);
  const int t0 = split * tps;
  const int t1 = min(n_run, t0 + tps);

  // Valid micro-tiles first: on a diagonal tile only those with some i < j,
  // on the last tile column only j < m; threads past the valid count (whole
  // warps, at the end) skip the arithmetic and only help stage the samples.
  int ti, tj;
  const bool active = micro_tile<MTI>(threadIdx.x, I, J, m, ti, tj);
  const int li = MTI * ti, lj = 2 * tj;
  const int gi0 = I * TB + li, gj0 = J * TB + lj;

  // pair (a, b) = (i0 + a, j0 + b); constants as float2 over b
  float2 NR[MTI], C[MTI];
  bool valid[MTI][2];
#pragma unroll
  for (int a = 0; a < MTI; ++a) {
    float r2[2], c2[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int gi = gi0 + a, gj = gj0 + b;
      valid[a][b] = active && (gi < gj) && (gj < m);
      r2[b] = valid[a][b] ? rho32[(int64_t)gi * m + gj] : 0.f;
      c2[b] = valid[a][b] ? c32[(int64_t)gi * m + gj] : KAPPA;
    }
    NR[a] = f2(-r2[0], -r2[1]);
    C[a] = f2(c2[0], c2[1]);
  }
  const float2 KK = f2(GAUSS_K, GAUSS_K);
  // stream pairs: 2a = residuals of i_a on (j0, j1), 2a + 1 = of (j0, j1) on i_a
  Pair2 q[2 * MTI];
#pragma unroll
  for (int k = 0; k < 2 * MTI; ++k)
    q[k] = Pair2{f2(1.f, 1.f), f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f),
                 f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};

  // stage loader: TTS rows x (32 + 32) floats = TTS * 16 chunks of 16 B
  auto load_stage = [&](int buf, int tb) {
    for (int idx = threadIdx.x; idx < TTS * 16; idx += NT) {
      const int r = idx >> 4, c = idx & 15;  // c: 0-7 I block, 8-15 J block
      const int t = tb + r;
      if (t < t1) {
        const int col = (c < 8) ? (I * TB + 4 * c) : (J * TB + 4 * (c - 8));
        cp_async16(&sx[buf][r][4 * c], xt + (int64_t)t * m_pad + col);
      }
    }
    cp_async_commit();
  };

  // three-stage ring: stage s+2 is copied while stage s is consumed, and the
  // one barrier per stage both publishes stage s and frees the buffer of
  // stage s-1 for the copy of stage s+2
  const int nst = t1 > t0 ? (t1 - t0 + TTS - 1) / TTS : 0;
  if (nst > 0) load_stage(0, t0);
  if (nst > 1) load_stage(1, t0 + TTS);
  for (int st = 0; st < nst; ++st) {
    const int tb = t0 + st * TTS, buf = st % 3;
    const int rows = min(TTS, t1 - tb);
    if (st + 1 < nst)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    __syncthreads();
    if (st + 2 < nst) load_stage((st + 2) % 3, tb + 2 * TTS);
    for (int r0 = 0; active && r0 < rows; r0 += KRUN) {
#pragma unroll
      for (int k = 0; k < KRUN; ++k) {
        const float2 xj = *reinterpret_cast<const float2*>(&sx[buf][r0 + k][TB + lj]);
        float xi[MTI];
        if constexpr (MTI == 2) {
          const float2 v = *reinterpret_cast<const float2*>(&sx[buf][r0 + k][li]);
          xi[0] = v.x;
          xi[1] = v.y;
        } else {
          xi[0] = sx[buf][r0 + k][li];
        }
#pragma unroll
        for (int a = 0; a < MTI; ++a) {
          const float2 xa = f2(xi[a], xi[a]);
          step2(q[2 * a], __ffma2_rn(NR[a], xj, xa), C[a], KK);      // x_i - rho x_j
          step2(q[2 * a + 1], __ffma2_rn(NR[a], xa, xj), C[a], KK);  // x_j - rho x_i
        }
      }
#pragma unroll
      for (int k = 0; k < 2 * MTI; ++k) end_run2(q[k]);
    }
  }

  // partials of this split as exact double-float pairs (sum, -comp):
  // part[(split*4 + k) * m*m + a*m + b] for the residual of a on b, k = 0, 1:
  // sum of log cosh u; k = 2, 3: sum of w e^{-u^2/2}.  No FP64 arithmetic here.
  const int64_t mm = (int64_t)m * m;
#pragma unroll
  for (int a = 0; a < MTI; ++a) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (!valid[a][b]) continue;
      const int gi = gi0 + a, gj = gj0 + b;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const Pair2& st = q[2 * a + d];
        const int64_t off = d ? ((int64_t)gj * m + gi) : ((int64_t)gi * m + gj);
        float* base = part + (int64_t)split * 4 * mm + off;
        base[0] = b ? st.sa.y : st.sa.x;
        base[mm] = -(b ? st.ca.y : st.ca.x);
        base[2 * mm] = b ? st.sb.y : st.sb.x;
        base[3 * mm] = -(b ? st.cb.y : st.cb.x);
      }
    }
  }
}

template <int MTI, int TTS, int MINB>
__global__ void __launch_bounds__(TB / MTI * 16, MINB)
    pairwise_f32_kernel(const float* __restrict__ xt, int m, int m_pad, int T, int n_run,
                        int tps, const float* __restrict__ rho32,
                        const float* __restrict__ c32, float* __restrict__ part) {
  pairwise_f32_item<MTI, TTS>(blockIdx.x, blockIdx.y, xt, m, m_pad, T, n_run, tps, rho32, c32,
                              part);
}

// Many instances in one launch: a device list of (job, tile, split) items,
// ordered by cost (largest first), dealt round-robin to a grid of about one
// CTA per SM; each CTA runs its items one after another.
template <int MTI, int TTS, int MINB>
__global__ void __launch_bounds__(TB / MTI * 16, MINB)
    pairwise_f32_list_kernel(const PairJob* __restrict__ jobs, const int4* __restrict__ items,
                             int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const PairJob& j = jobs[w.x];
    pairwise_f32_item<MTI, TTS>(w.y, w.z, j.xt, j.m, j.m_pad, j.T, j.n_run, j.tps, j.rho32,
                                j.c32, j.part);
    __syncthreads();  // the sample stages are reused by the next item
  }
}

// Plain FP64 comparison kernel: per sample log cosh u = |u| + log1p(e^{-2|u|})
// - ln 2 and u e^{-u^2/2} with CUDA's double-precision exp/log1p, FP64 sums.
// Partials: k = 0 sum log cosh u, k = 1 sum u e^{-u^2/2}.
__global__ void __launch_bounds__(NTH)
    pairwise_f64_kernel(const double* __restrict__ xt, int m, int m_pad, int T, int n_real,
                        int tps, const double* __restrict__ rho64, double* __restrict__ part) {
  int I, J;
  tile_coords(blockIdx.x, T, I, J);
  const int split = blockIdx.y;
  const int t0 = split * tps;
  const int t1 = min(n_real, t0 + tps);
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  const int gi0 = I * TB + 2 * ti, gj0 = J * TB + 2 * tj;
  double rho[4], sc[4];
  bool valid[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int a = gi0 + (p >> 1), b = gj0 + (p & 1);
    valid[p] = (a < b) && (b < m);
    rho[p] = valid[p] ? rho64[(int64_t)a * m + b] : 0.0;
    sc[p] = 1.0 / sqrt(1.0 - rho[p] * rho[p]);
  }
  double sA[8], sB[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) sA[q] = sB[q] = 0.0;
  for (int t = t0; t < t1; ++t) {
    const double* row = xt + (int64_t)t * m_pad;
    const double xa[2] = {row[gi0], row[gi0 + 1]};
    const double xb[2] = {row[gj0], row[gj0 + 1]};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (!valid[p]) continue;
      const double a = xa[p >> 1], b = xb[p & 1];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const double self = d ? b : a, other = d ? a : b;
        const double u = sc[p] * (self - rho[p] * other);
        const double au = fabs(u);
        sA[2 * p + d] += au + log1p(exp(-2.0 * au)) - LN2;
        sB[2 * p + d] += u * exp(-0.5 * u * u);
      }
    }
  }
  const int64_t mm = (int64_t)m * m;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    if (!valid[p]) continue;
    const int a = gi0 + (p >> 1), b = gj0 + (p & 1);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int64_t off = d ? ((int64_t)b * m + a) : ((int64_t)a * m + b);
      double* base = part + (int64_t)split * 2 * mm + off;
      base[0] = sA[2 * p + d];
      base[mm] = sB[2 * p + d];
    }
  }
}

// rho_ij = C_ij / sqrt(C_ii C_jj) from the centred cross-product matrix C.
__global__ void pair_consts_kernel(const double* __restrict__ C, int m,
                                   float* __restrict__ rho32, float* __restrict__ c32,
                                   double* __restrict__ rho64, int* st) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  double r = 0.0;
  if (a != b) {
    r = C[idx] / sqrt(C[(int64_t)a * m + a] * C[(int64_t)b * m + b]);
    if (!(1.0 - r * r >= DEGENERATE_1MR2)) {
      set_status(st, VL_ERR_DEGENERATE);
      r = 0.0;
    }
  }
  if (rho32) {
    rho32[idx] = (float)r;
    c32[idx] = (float)((double)KAPPA / sqrt(1.0 - r * r));
  }
  if (rho64) rho64[idx] = r;
}

// double-float accumulate (hi, lo) += x (TwoSum)
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

__global__ void measure_finalize_kernel(const void* __restrict__ part_v, int m, int splits,
                                        int n_real, const double* __restrict__ hx,
                                        double* __restrict__ Hx, double* __restrict__ Hr,
                                        double* __restrict__ D, int fp32_parts) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t mm = (int64_t)m * m;
  if (idx >= mm) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  if (Hx && b == 0) Hx[a] = entropy_from_moments(hx[2 * a], hx[2 * a + 1]);
  if (a == b) {
    Hr[idx] = 0.0;
    D[idx] = 0.0;
    return;
  }
  // H of the residual of a on b and of b on a
  double h[2];
  for (int d = 0; d < 2; ++d) {
    const int64_t off = d ? ((int64_t)b * m + a) : idx;
    double A, B;
    if (fp32_parts) {
      // splits combined in double-float FP32 arithmetic, one FP64 conversion
      const float* part = static_cast<const float*>(part_v);
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      for (int s = 0; s < splits; ++s) {
        const float* p = part + (int64_t)s * 4 * mm + off;
        df_add(h0, l0, p[0]);
        df_add(h0, l0, p[mm]);
        df_add(h1, l1, p[2 * mm]);
        df_add(h1, l1, p[3 * mm]);
      }
      const double s0 = (double)h0 + (double)l0;  // sum of log cosh u
      const double s1 = (double)h1 + (double)l1;  // sum of w e^{-u^2/2}
      const double kappa = 2.0 * LOG2E;
      A = s0 / n_real;
      B = s1 / (kappa * n_real);
    } else {
      const double* part = static_cast<const double*>(part_v);
      double s0 = 0.0, s1 = 0.0;
      for (int s = 0; s < splits; ++s) {
        const double* p = part + (int64_t)s * 2 * mm + off;
        s0 += p[0];
        s1 += p[mm];
      }
      A = s0 / n_real;
      B = s1 / n_real;
    }
    h[d] = entropy_from_moments(A, B);
  }
  Hr[idx] = h[0];
  const double hxa = entropy_from_moments(hx[2 * a], hx[2 * a + 1]);
  const double hxb = entropy_from_moments(hx[2 * b], hx[2 * b + 1]);
  D[idx] = hxb + h[0] - hxa - h[1];
}

}  // namespace

// FP32 kernel configuration: micro-tile rows, samples per stage, CTAs per SM.
// 1 x 2 micro-tiles, 512 threads and one CTA per SM: measured at m = 400,
// n = 2500 against 2 x 2 micro-tiles with 256 threads (one or two CTAs per SM)
// and 64-192 sample stages, this was the fastest (148 vs 150-164 us).
constexpr int F32_MTI = 1;
constexpr int F32_TTS = 128;
constexpr int F32_MINB = 1;

// Sample splits for `slots` resident CTAs: the CTA count should fill whole
// waves (about 3-6 of them), each split at least two stages of `tts` long.
PairPlan plan_pairwise_slots(int m, int n, int slots, int tts, bool fp64, int num_sms) {
  PairPlan pl{};
  pl.m = m;
  pl.n = n;
  pl.m_pad = ((m + TB - 1) / TB) * TB;
  const int Tside = pl.m_pad / TB;
  pl.tiles = Tside * (Tside + 1) / 2;
  const int n_run = ((n + KRUN - 1) / KRUN) * KRUN;
  int max_split = std::max(1, n_run / (2 * tts));
  // a small problem that does not fill one wave even at this split count gets
  // shorter splits (down to 4 runs of samples each), up to one CTA per slot
  if ((long)pl.tiles * max_split < slots)
    max_split = std::max(max_split, std::min(n_run / (4 * KRUN), (slots + pl.tiles - 1) / pl.tiles));
  int splits = 1;
  double best = -1.0;
  for (int sp = 1; sp <= max_split; ++sp) {
    const long ctas = (long)pl.tiles * sp;
    const long waves = (ctas + slots - 1) / slots;
    if (waves > 8) break;
    const double eff = (double)ctas / (double)(waves * slots);
    // prefer full waves; among equals, at least 3 waves for load balance
    const double score = eff - (waves < 3 ? 0.05 * (3 - waves) : 0.0);
    if (score > best + 1e-9) {
      best = score;
      splits = sp;
    }
  }
  if (fp64) splits = std::min(std::max(1, (4 * num_sms + pl.tiles - 1) / pl.tiles), n);
  int tps = (n_run + splits - 1) / splits;
  tps = ((tps + KRUN - 1) / KRUN) * KRUN;
  pl.splits = (n_run + tps - 1) / tps;
  pl.t_per_split = tps;
  pl.n_pad = ((n_run + 255) / 256) * 256;  // whole stages of any configuration
  return pl;
}

PairPlan plan_pairwise_split(int m, int n, int split_len) {
  PairPlan pl{};
  pl.m = m;
  pl.n = n;
  pl.m_pad = ((m + TB - 1) / TB) * TB;
  const int Tside = pl.m_pad / TB;
  pl.tiles = Tside * (Tside + 1) / 2;
  const int n_run = ((n + KRUN - 1) / KRUN) * KRUN;
  int tps = std::max(KRUN, ((std::min(split_len, n_run) + KRUN - 1) / KRUN) * KRUN);
  pl.splits = (n_run + tps - 1) / tps;
  tps = ((n_run + pl.splits - 1) / pl.splits + KRUN - 1) / KRUN * KRUN;  // even splits
  pl.splits = (n_run + tps - 1) / tps;
  pl.t_per_split = tps;
  pl.n_pad = ((n_run + 255) / 256) * 256;
  return pl;
}

PairPlan plan_pairwise(int m, int n, int num_sms, bool fp64) {
  return plan_pairwise_slots(m, n, F32_MINB * num_sms, F32_TTS, fp64, num_sms);
}

void launch_pair_consts(const double* C, int m, float* rho32, float* c32, double* rho64, int* st,
                        cudaStream_t s) {
  int64_t tot = (int64_t)m * m;
  note_launch();
  pair_consts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C, m, rho32, c32, rho64, st);
}

template <int MTI, int TTS, int MINB>
void launch_pairwise_f32_cfg(const float* xt, const PairPlan& pl, const float* rho32,
                             const float* c32, float* part, cudaStream_t s) {
  const int n_run = ((pl.n + KRUN - 1) / KRUN) * KRUN;
  dim3 grid(pl.tiles, pl.splits);
  const size_t smem = sizeof(float) * 3 * TTS * 2 * TB;  // three stages of TTS x 64 samples
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(pairwise_f32_kernel<MTI, TTS, MINB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  note_launch();
  pairwise_f32_kernel<MTI, TTS, MINB><<<grid, TB / MTI * 16, smem, s>>>(
      xt, pl.m, pl.m_pad, pl.m_pad / TB, n_run, pl.t_per_split, rho32, c32, part);
}

void launch_pairwise_f32(const float* xt, const PairPlan& pl, const float* rho32,
                         const float* c32, float* part, cudaStream_t s) {
  launch_pairwise_f32_cfg<F32_MTI, F32_TTS, F32_MINB>(xt, pl, rho32, c32, part, s);
}

PairJob make_pair_job(const float* xt, const PairPlan& pl, const float* rho32, const float* c32,
                      float* part) {
  PairJob j;
  j.xt = xt;
  j.rho32 = rho32;
  j.c32 = c32;
  j.part = part;
  j.m = pl.m;
  j.m_pad = pl.m_pad;
  j.T = pl.m_pad / TB;
  j.n_run = ((pl.n + KRUN - 1) / KRUN) * KRUN;
  j.tps = pl.t_per_split;
  return j;
}

void launch_pairwise_f32_list(const PairJob* jobs, const int4* items, int nitems, int grid,
                              cudaStream_t s) {
  constexpr int MTI = F32_MTI, TTS = F32_TTS, MINB = F32_MINB;
  const size_t smem = sizeof(float) * 3 * TTS * 2 * TB;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(pairwise_f32_list_kernel<MTI, TTS, MINB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  note_launch();
  pairwise_f32_list_kernel<MTI, TTS, MINB><<<std::max(1, std::min(grid, nitems)), TB / MTI * 16,
                                             smem, s>>>(jobs, items, nitems);
}

void launch_pairwise_f64(const double* xt, const PairPlan& pl, const double* rho64,
                         double* part, cudaStream_t s) {
  dim3 grid(pl.tiles, pl.splits);
  note_launch();
  pairwise_f64_kernel<<<grid, NTH, 0, s>>>(xt, pl.m, pl.m_pad, pl.m_pad / TB, pl.n,
                                           pl.t_per_split, rho64, part);
}

void launch_measure_finalize(const void* part, const PairPlan& pl, const double* hx_mom,
                             double* Hx, double* Hr, double* D, bool fp32_parts,
                             cudaStream_t s) {
  const int64_t tot = (int64_t)pl.m * pl.m;
  note_launch();
  measure_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      part, pl.m, pl.splits, pl.n, hx_mom, Hx, Hr, D, fp32_parts ? 1 : 0);
}

}  // namespace vl
