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
//     sa  += |w|
//     g    = ex2(-w^2 / (8 log2 e))     = e^{-u^2/2}   (MUFU)
//     sb  += w g
// Every KRUN = 16 samples the run sums are Kahan-added into FP32 (sum, comp)
// pairs and log2(prod) (one MUFU lg2 per run) is Kahan-added as well, so
// sum_t ln(1 + y_t) = ln 2 * sum_runs log2(prod_run).  The split partials are
// written as FP64 and combined in a fixed order by measure_finalize.
//
// Padding: x is zero beyond n (time) and beyond m (variables).  A zero sample
// gives |w| = 0, 1 + y = 2, w g = 0, i.e. exactly log cosh 0 = 0 once the
// ln 2 per processed sample is removed, so padding needs no masking.
#include <algorithm>
#include <cmath>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int TB = 32;        // variables per tile side
constexpr int TT = 128;       // samples per shared-memory stage
constexpr int KRUN = 16;      // samples per product/Kahan run (product <= 2^16)
constexpr int NTH = 256;      // threads: 16 x 16, each a 2 x 2 pair micro-tile
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
__device__ __forceinline__ void kahan_add(float& S, float& C, float x) {
  float y = x - C;
  float t = S + y;
  C = (t - S) - y;
  S = t;
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

struct Stream {
  float sa, ca, sb, cb, sl, cl;
};

// Thread -> 2 x 2 pair micro-tile (ti, tj) of tile (I, J), enumerating only
// micro-tiles holding at least one pair i < j < m; returns false for threads
// beyond that count.
__device__ __forceinline__ bool micro_tile(int s, int I, int J, int m, int& ti, int& tj) {
  const int lim = min(16, (m - J * TB + 1) / 2);  // micro-columns with some j < m
  if (I < J) {
    ti = s / lim;
    tj = s % lim;
    if (ti < 16) return true;
  } else {
    // upper triangle ti <= tj < lim, row by row
    for (int r = 0; r < lim; ++r) {
      const int len = lim - r;
      if (s < len) {
        ti = r;
        tj = r + s;
        return true;
      }
      s -= len;
    }
  }
  ti = 0;
  tj = 0;
  return false;
}

__global__ void __launch_bounds__(NTH, 2)
    pairwise_f32_kernel(const float* __restrict__ xt, int m, int m_pad, int T, int n_run,
                        int tps, const float* __restrict__ rho32,
                        const float* __restrict__ c32, float* __restrict__ part) {
  extern __shared__ __align__(16) float pw_smem[];
  float(*sx)[TT][2 * TB] = reinterpret_cast<float(*)[TT][2 * TB]>(pw_smem);  // [2][TT][64]
  int I, J;
  tile_coords(blockIdx.x, T, I, J);
  const int split = blockIdx.y;
  const int t0 = split * tps;
  const int t1 = min(n_run, t0 + tps);

  // Valid 2 x 2 pair micro-tiles first: on a diagonal tile only ti <= tj,
  // on the last tile column only j < m; threads past the valid count (whole
  // warps, at the end) skip the arithmetic and only help stage the samples.
  int ti, tj;
  const bool active = micro_tile(threadIdx.x, I, J, m, ti, tj);
  const int li = 2 * ti, lj = 2 * tj;
  const int gi0 = I * TB + li, gj0 = J * TB + lj;

  float rho[4], cc[4];
  bool valid[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int a = gi0 + (p >> 1), b = gj0 + (p & 1);
    valid[p] = active && (a < b) && (b < m);
    rho[p] = valid[p] ? rho32[(int64_t)a * m + b] : 0.f;
    cc[p] = valid[p] ? c32[(int64_t)a * m + b] : KAPPA;
  }
  Stream st[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) st[q] = Stream{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

  // stage loader: TT rows x (32 + 32) floats = TT * 16 chunks of 16 B
  auto load_stage = [&](int buf, int tb) {
    for (int idx = threadIdx.x; idx < TT * 16; idx += NTH) {
      const int r = idx >> 4, c = idx & 15;  // c: 0-7 I block, 8-15 J block
      const int t = tb + r;
      if (t < t1) {
        const int col = (c < 8) ? (I * TB + 4 * c) : (J * TB + 4 * (c - 8));
        cp_async16(&sx[buf][r][4 * c], xt + (int64_t)t * m_pad + col);
      }
    }
    cp_async_commit();
  };

  int buf = 0;
  if (t0 < t1) load_stage(0, t0);
  for (int tb = t0; tb < t1; tb += TT) {
    const int rows = min(TT, t1 - tb);
    if (tb + TT < t1) {
      load_stage(buf ^ 1, tb + TT);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int r0 = 0; active && r0 < rows; r0 += KRUN) {
      float ra[8], rb[8], pr[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ra[q] = 0.f;
        rb[q] = 0.f;
        pr[q] = 1.f;
      }
#pragma unroll
      for (int k = 0; k < KRUN; ++k) {
        const float2 xi = *reinterpret_cast<const float2*>(&sx[buf][r0 + k][li]);
        const float2 xj = *reinterpret_cast<const float2*>(&sx[buf][r0 + k][TB + lj]);
        const float xa[2] = {xi.x, xi.y}, xb[2] = {xj.x, xj.y};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float a = xa[p >> 1], b = xb[p & 1];
#pragma unroll
          for (int d = 0; d < 2; ++d) {
            const int q = 2 * p + d;
            const float self = d ? b : a, other = d ? a : b;
            const float r = fmaf(-rho[p], other, self);
            const float w = cc[p] * r;
            const float y = ex2_approx(-fabsf(w));
            pr[q] = fmaf(pr[q], y, pr[q]);
            ra[q] += fabsf(w);
            const float g = ex2_approx((w * GAUSS_K) * w);
            rb[q] = fmaf(w, g, rb[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        kahan_add(st[q].sa, st[q].ca, ra[q]);
        kahan_add(st[q].sb, st[q].cb, rb[q]);
        kahan_add(st[q].sl, st[q].cl, lg2_approx(pr[q]));
      }
    }
    __syncthreads();
    buf ^= 1;
  }

  // partial sums of this split as exact double-float pairs (sum, -comp):
  // part[(split*6 + k) * m*m + a*m + b] for the residual of a on b.  No FP64
  // arithmetic here: FP64 issues at 1/64 rate on this part, and a CTA covers
  // only a few hundred samples.
  const int64_t mm = (int64_t)m * m;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    if (!valid[p]) continue;
    const int a = gi0 + (p >> 1), b = gj0 + (p & 1);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const Stream& s = st[2 * p + d];
      const int64_t off = d ? ((int64_t)b * m + a) : ((int64_t)a * m + b);
      float* base = part + (int64_t)split * 6 * mm + off;
      base[0] = s.sa;
      base[mm] = -s.ca;
      base[2 * mm] = s.sl;
      base[3 * mm] = -s.cl;
      base[4 * mm] = s.sb;
      base[5 * mm] = -s.cb;
    }
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
                                        int n_real, int n_proc, const double* __restrict__ hx,
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
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
      for (int s = 0; s < splits; ++s) {
        const float* p = part + (int64_t)s * 6 * mm + off;
        df_add(h0, l0, p[0]);
        df_add(h0, l0, p[mm]);
        df_add(h1, l1, p[2 * mm]);
        df_add(h1, l1, p[3 * mm]);
        df_add(h2, l2, p[4 * mm]);
        df_add(h2, l2, p[5 * mm]);
      }
      const double s0 = (double)h0 + (double)l0;
      const double s1 = (double)h1 + (double)l1;
      const double s2 = (double)h2 + (double)l2;
      const double kappa = 2.0 * LOG2E;
      A = (s0 / kappa + LN2 * (s1 - (double)n_proc)) / n_real;
      B = s2 / (kappa * n_real);
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

PairPlan plan_pairwise(int m, int n, int num_sms, bool fp64) {
  PairPlan pl{};
  pl.m = m;
  pl.n = n;
  pl.m_pad = ((m + TB - 1) / TB) * TB;
  const int Tside = pl.m_pad / TB;
  pl.tiles = Tside * (Tside + 1) / 2;
  const int n_run = ((n + KRUN - 1) / KRUN) * KRUN;
  // Split the samples so that the CTA count fills whole waves of 2 CTAs per
  // SM (about 3-6 waves), each split at least 2 stages long.
  const int slots = 2 * num_sms;
  const int max_split = std::max(1, n_run / (2 * TT));
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
  pl.n_pad = ((n_run + TT - 1) / TT) * TT;
  return pl;
}

void launch_pair_consts(const double* C, int m, float* rho32, float* c32, double* rho64, int* st,
                        cudaStream_t s) {
  int64_t tot = (int64_t)m * m;
  note_launch();
  pair_consts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C, m, rho32, c32, rho64, st);
}

void launch_pairwise_f32(const float* xt, const PairPlan& pl, const float* rho32,
                         const float* c32, float* part, cudaStream_t s) {
  const int n_run = ((pl.n + KRUN - 1) / KRUN) * KRUN;
  dim3 grid(pl.tiles, pl.splits);
  const size_t smem = sizeof(float) * 2 * TT * 2 * TB;  // two stages of TT x 64 samples
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(pairwise_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  note_launch();
  pairwise_f32_kernel<<<grid, NTH, smem, s>>>(xt, pl.m, pl.m_pad, pl.m_pad / TB, n_run,
                                              pl.t_per_split, rho32, c32, part);
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
  const int n_run = ((pl.n + KRUN - 1) / KRUN) * KRUN;
  note_launch();
  measure_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      part, pl.m, pl.splits, pl.n, n_run, hx_mom, Hx, Hr, D, fp32_parts ? 1 : 0);
}

}  // namespace vl
