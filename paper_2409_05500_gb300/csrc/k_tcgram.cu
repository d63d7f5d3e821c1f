// Tensor-core Gram products of the mixed-precision path: the lagged VAR Gram
// W W^T (Sec. 4.1; W = [Y; Z_1; ..; Z_p]) and the residual covariance E E^T
// whose correlations rho_ij enter Eq. 1 (Sec. 3, Sec. 4.2).
//
// Arithmetic (exact-slice split).  Every row r of an operand is scaled by a
// power of two 2^(e_r - 7) so that its entries lie in (-128, 128), and each
// scaled entry y is split into three bf16 slices holding integers,
//     y = a0 + a1 2^-8 + a2 2^-16 + (remainder below 2^-17),   |a_s| <= 128,
// which bf16 (8-bit significand) represents exactly.  The product of two
// entries is the sum over slice pairs (s, s') of a_s a'_s' 2^-8(s+s'); the
// pairs with s + s' <= 3 are kept, grouped in four levels L = s + s':
//     L0: (0,0)   L1: (0,1) (1,0)   L2: (0,2) (1,1) (2,0)   L3: (1,2) (2,1),
// eight bf16 tensor-core products per K-block.  Each product is an integer of
// magnitude <= 2^14 and each level sums at most 3 of them per k, so over a
// segment of 256 values of k every level's sum stays below 2^24 and the FP32
// accumulators in tensor memory hold it EXACTLY (no rounding, whatever the
// accumulation order or rounding mode).  After each segment the four level
// sums are combined, L0 + L1 2^-8 + L2 2^-16 + L3 2^-24, into a double-float
// (two FP32) register accumulator; split-K partials are added in double-float
// and the final value is scaled by 2^(e_i + e_j - 14) in FP64.  The only
// errors are the slicing remainder (2^-24 of the row's largest entry per
// entry) and the dropped level-4 pair (same order): about FP32 rounding of
// each entry relative to its row maximum, random across k, so the products
// are accurate to ~1e-8 relative after the sum -- comparable to or better
// than a compensated FP32 SIMT product, on the tensor pipe.
//
// Data path (sm_103a).  One CTA computes a 128 x 64 output tile over a range
// of K: warp 0 issues TMA loads (cp.async.bulk.tensor, 128-byte swizzle, one
// 3-D box per operand holding all three slices of a 64-wide K-block) into a
// three-stage shared-memory ring; warp 1 owns the tensor memory (512 columns:
// two buffers x four levels x 64) and one of its threads issues the
// tcgen05.mma instructions (M = 128, N = 64, K = 16 each) and commits them to
// mbarriers; warps 2-5 drain a finished segment's levels from tensor memory
// (tcgen05.ld) into their double-float accumulators while the next segment
// accumulates into the other buffer.  All waits are bounded: a wait that
// runs out sets VL_ERR_TIMEOUT, the CTA stops issuing work, lets its copies
// and products in flight complete, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"
#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int TG_M = 128;        // tile rows (MMA M)
constexpr int TG_N = 64;         // tile columns (MMA N)
constexpr int TG_K = 64;         // K per stage: one 128-byte swizzle row of bf16
constexpr int TG_SL = 3;         // slices per operand
constexpr int TG_LEV = 4;        // product levels kept
constexpr int TG_STAGES = 3;
constexpr int TG_SEG = 4;        // K-blocks per exact segment (256 values of k)
constexpr int TG_THREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 drain
constexpr int A_SLICE = TG_M * TG_K * 2;               // 16 KB
constexpr int B_SLICE = TG_N * TG_K * 2;               // 8 KB
constexpr int STAGE_BYTES = TG_SL * (A_SLICE + B_SLICE);  // 72 KB
constexpr int TMEM_COLS = 2 * TG_LEV * TG_N;             // 512
constexpr size_t TG_SMEM = (size_t)TG_STAGES * STAGE_BYTES + 1024 /*barriers*/ +
                           1024 /*alignment*/;
constexpr uint32_t WAIT_LIMIT = 1u << 20;  // bounded polls of one mbarrier wait

static_assert(TG_SEG * TG_K * 3 * 128 * 128 < (1 << 24), "a level sum must stay exact in FP32");

// ------------------------------------------------------------- slicing
// Exponent e with max < 2^e from the bits of a non-negative double (0 -> 0),
// clamped so that the FP32 scale 2^(7 - e) is finite and normal (rows whose
// largest entry is below 2^-100 are treated as zero-ish; the mixed path
// takes no entries above 2^120).
__device__ __forceinline__ int clamp_exp(int e) { return min(120, max(-100, e)); }
__device__ __forceinline__ int exp_above(unsigned long long bits) {
  if (bits == 0) return 0;
  return clamp_exp((int)((bits >> 52) & 0x7ff) - 1022);
}

// Three integer slices of y in (-128, 128) given as an FP32 pair (yh + yl).
__device__ __forceinline__ void slice3(float yh, float yl, __nv_bfloat16& s0, __nv_bfloat16& s1,
                                       __nv_bfloat16& s2) {
  const float a0 = rintf(yh);
  const float r1 = ((yh - a0) + yl) * 256.f;
  const float a1 = rintf(r1);
  const float a2 = rintf((r1 - a1) * 256.f);
  s0 = __float2bfloat16_rn(a0);
  s1 = __float2bfloat16_rn(a1);
  s2 = __float2bfloat16_rn(a2);
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b = red[q] > b ? red[q] : b;
    red[0] = b;
  }
  __syncthreads();
  return red[0];
}

// Centred FP64 rows (E[r][k] - mu[r], k < K) into three slice planes
// S[z][r][k] (row stride ldo, plane stride plane; zeros for K <= k < Kpad)
// and the row exponent.  One block per row.
__global__ void slice_center_kernel(const double* __restrict__ E, int64_t lde,
                                    const double* __restrict__ mu, int K, int Kpad,
                                    __nv_bfloat16* __restrict__ S, int64_t ldo, int64_t plane,
                                    int* __restrict__ exps) {
  __shared__ unsigned long long red[32];
  const int r = blockIdx.x;
  const double* e = E + (int64_t)r * lde;
  const double m = mu[r];
  unsigned long long mx = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(e[k] - m) & 0x7fffffffffffffffull;
    mx = b > mx ? b : mx;
  }
  const int ex = exp_above(block_max_u64(mx, red));
  if (threadIdx.x == 0) exps[r] = ex;
  const float sc = ldexpf(1.f, 7 - ex);
  __nv_bfloat16* o = S + (int64_t)r * ldo;
  for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
    __nv_bfloat16 s0, s1, s2;
    if (k < K) {
      const double d = e[k] - m;
      const float h = (float)d;
      const float l = (float)(d - (double)h);
      slice3(h * sc, l * sc, s0, s1, s2);
    } else {
      s0 = s1 = s2 = __float2bfloat16_rn(0.f);
    }
    o[k] = s0;
    o[plane + k] = s1;
    o[2 * plane + k] = s2;
  }
}

// The lag windows of the centred FP32 series Xc (m rows, stride ldc): row
// b m + k of W is Xc[k][p - b + t], t < n_eff, for b = 0..p (b = 0 is Y, b =
// tau is Z_tau).  One block per variable k; one exponent per variable for all
// of its windows.
__global__ void slice_lags_kernel(const float* __restrict__ Xc, int64_t ldc, int m, int n,
                                  int p, int Kpad, __nv_bfloat16* __restrict__ S, int64_t ldo,
                                  int64_t plane, int* __restrict__ exps) {
  __shared__ unsigned long long red[32];
  const int k = blockIdx.x;
  const float* x = Xc + (int64_t)k * ldc;
  const int n_eff = n - p;
  unsigned long long mx = 0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const unsigned long long b = __float_as_uint(x[t]) & 0x7fffffffu;
    mx = b > mx ? b : mx;
  }
  // float bits: f < 2^(E - 126) for biased exponent E (0 -> 0)
  const unsigned long long fb = block_max_u64(mx, red);
  const int ex = fb == 0 ? 0 : clamp_exp((int)((fb >> 23) & 0xff) - 126);
  const float sc = ldexpf(1.f, 7 - ex);
  if (threadIdx.x <= p) exps[threadIdx.x * m + k] = ex;
  for (int t = threadIdx.x; t < Kpad; t += blockDim.x) {
    for (int b = 0; b <= p; ++b) {
      __nv_bfloat16 s0, s1, s2;
      if (t < n_eff) {
        slice3(x[p - b + t] * sc, 0.f, s0, s1, s2);
      } else {
        s0 = s1 = s2 = __float2bfloat16_rn(0.f);
      }
      __nv_bfloat16* o = S + (int64_t)(b * m + k) * ldo;
      o[t] = s0;
      o[plane + t] = s1;
      o[2 * plane + t] = s2;
    }
  }
}

// The VAR residual product (Sec. 4.1, E = Y - sum_tau M_tau Z_tau) as one
// Gram-type product over K = (tau, k): A = beta' (m rows), B = the time-major
// series (rows t).  The per-variable scale of the series moves into A, so
// that every row of B shares one scale: A[i][(tau-1) mp + k] = M_tau[i][k]
// 2^(e_k) and B[s][k] = Xc[k][s] 2^(-e_k), whose product is M_tau[i][k]
// Xc[k][s] exactly.
// Time-major slices of the normalised series: St[z][s][k], k < kp (zeros for
// k >= m), from Xc (m rows, stride ldc) and the variables' exponents.
__global__ void slice_time_kernel(const float* __restrict__ Xc, int64_t ldc, int m, int n,
                                  int kp, const int* __restrict__ vexp,
                                  __nv_bfloat16* __restrict__ St, int64_t plane) {
  __shared__ float tile[32][33];
  const int s0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, t = s0 + tx;
    tile[r][tx] = (k < m && t < n) ? ldexpf(Xc[(int64_t)k * ldc + t], 7 - vexp[k]) : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int t = s0 + r, k = k0 + tx;
    if (t >= n || k >= kp) continue;
    __nv_bfloat16 a, b, c;
    slice3(tile[tx][r], 0.f, a, b, c);
    __nv_bfloat16* o = St + (int64_t)t * kp + k;
    o[0] = a;
    o[plane] = b;
    o[2 * plane] = c;
  }
}

// Slices of beta' (m rows, K = p kp): row i, column (tau-1) kp + k holds
// beta[(tau-1) m + k][i] 2^(e_k) (zeros for k >= m), with the row exponent.
__global__ void slice_beta_kernel(const float* __restrict__ beta, int m, int p, int kp,
                                  const int* __restrict__ vexp, __nv_bfloat16* __restrict__ Sb,
                                  int64_t plane, int* __restrict__ aexp) {
  __shared__ unsigned long long red[32];
  const int i = blockIdx.x, K = p * kp;
  unsigned long long mx = 0;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const int tau = c / kp, k = c % kp;
    if (k >= m) continue;
    const float a = ldexpf(beta[((int64_t)tau * m + k) * m + i], vexp[k]);
    const unsigned long long b = __float_as_uint(a) & 0x7fffffffu;
    mx = b > mx ? b : mx;
  }
  const unsigned long long fb = block_max_u64(mx, red);
  const int ex = fb == 0 ? 0 : clamp_exp((int)((fb >> 23) & 0xff) - 126);
  if (threadIdx.x == 0) aexp[i] = ex;
  __nv_bfloat16* o = Sb + (int64_t)i * K;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const int tau = c / kp, k = c % kp;
    const float a = k < m ? ldexpf(beta[((int64_t)tau * m + k) * m + i], vexp[k] + 7 - ex) : 0.f;
    __nv_bfloat16 s0, s1, s2;
    slice3(a, 0.f, s0, s1, s2);
    o[c] = s0;
    o[plane + c] = s1;
    o[2 * plane + c] = s2;
  }
}

// E[i][t] = X[i][p + t] - (mu_i + cst_i) - 2^(a_i - 14) (product), t < n_eff.
__global__ void resid_apply_kernel(const double* __restrict__ X, int64_t ldx, int m, int n_eff,
                                   int p, const double* __restrict__ mu,
                                   const double* __restrict__ cst, const float2* __restrict__ part,
                                   const int* __restrict__ aexp, double* __restrict__ E) {
  const int i = blockIdx.y;
  const double off = mu[i] + cst[i];
  const int ex = aexp[i] - 14;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_eff; t += gridDim.x * blockDim.x) {
    const float2 v = part[(int64_t)i * n_eff + t];
    E[(int64_t)i * n_eff + t] =
        X[(int64_t)i * ldx + p + t] - off - ldexp((double)v.x + (double)v.y, ex);
  }
}

// --------------------------------------------------------- the product
struct TgParams {
  int M, N;            // output rows / columns
  int nkb;             // K-blocks (of 64) over the whole K
  int kb_per_split;    // K-blocks per CTA (the last CTA may have fewer)
  int tiles_n;         // 64-wide column tiles
  int sym;             // 1: only tiles reaching the upper triangle (A == B)
  int lag_kb;          // > 0: B is read as lag windows (see tcgram_kernel)
  int lag_p;
  float2* part;        // [split][M][N] double-float partials
  int* st;             // sticky status word
};

// exact double-float s + x (x an FP32 value)
__device__ __forceinline__ void df_add1(float& h, float& l, float x) {
  const float s = h + x;
  const float bp = s - h;
  const float e = (h - (s - bp)) + (x - bp);
  h = s;
  l += e;
}
__device__ __forceinline__ void df_norm(float& h, float& l) {
  const float s = h + l;
  l = l - (s - h);
  h = s;
}

// tile index -> (I, J): row tile I (128 rows), column tile J (64 columns); in
// symmetric mode only J >= 2 I (the tiles holding entries with column >= row)
__device__ __forceinline__ void tg_tile(int q, const TgParams& P, int& I, int& J) {
  if (!P.sym) {
    I = q / P.tiles_n;
    J = q % P.tiles_n;
    return;
  }
  int i = 0;
  for (;;) {
    const int cnt = P.tiles_n - 2 * i;
    if (q < cnt) break;
    q -= cnt;
    ++i;
  }
  I = i;
  J = 2 * i + q;
}

__global__ void __launch_bounds__(TG_THREADS, 1)
    tcgram_kernel(const __grid_constant__ CUtensorMap mapA,
                  const __grid_constant__ CUtensorMap mapB, TgParams P) {
  extern __shared__ unsigned char tg_raw[];
  // 1024-byte aligned base for the swizzled tiles
  unsigned char* smem = tg_raw + ((1024 - (tc::smem_u32(tg_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TG_STAGES * STAGE_BYTES);
  uint64_t* empty = full + TG_STAGES;
  uint64_t* tfull = empty + TG_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int I, J;
  tg_tile(blockIdx.x, P, I, J);
  const int row0 = I * TG_M, col0 = J * TG_N;
  const int kb0 = blockIdx.y * P.kb_per_split;
  const int nkb = min(P.kb_per_split, P.nkb - kb0);
  const int nseg = (nkb + TG_SEG - 1) / TG_SEG;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 4);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tc::tma_prefetch_map(&mapA);
    tc::tma_prefetch_map(&mapB);
  }
  __syncwarp();
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // TMA K-blocks issued (warp 0, lane 0)
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nkb; ++it) {
        const int s = it % TG_STAGES, u = it / TG_STAGES;
        if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag, WAIT_LIMIT)) break;
        tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
        unsigned char* st = smem + s * STAGE_BYTES;
        const int kb = kb0 + it, kx = kb * TG_K;
        tc::tma_load_3d(st, &mapA, &full[s], kx, row0, 0);
        if (P.lag_kb > 0) {
          // K-block kb belongs to lag tau = kb / lag_kb + 1: rows t of B are
          // the time-major slices at time p - tau + t (a row offset: no
          // alignment rule), columns the variables of that K-block
          const int tau = kb / P.lag_kb + 1;
          tc::tma_load_3d(st + TG_SL * A_SLICE, &mapB, &full[s], (kb % P.lag_kb) * TG_K,
                          col0 + P.lag_p - tau, 0);
        } else {
          tc::tma_load_3d(st + TG_SL * A_SLICE, &mapB, &full[s], kx, col0, 0);
        }
        ++issued;
      }
      if (issued < nkb) *abort_flag = 1;
    }
    __syncwarp();  // the warp reaches the final barrier converged
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(TG_M, TG_N);
      // slice pairs (a, b) and their level a + b
      const int pa[8] = {0, 0, 1, 0, 1, 2, 1, 2};
      const int pb[8] = {0, 1, 0, 2, 1, 0, 2, 1};
      bool ok = true;
      int it = 0;
      for (int seg = 0; seg < nseg && ok; ++seg) {
        const int b = seg & 1, u = seg >> 1;
        if (u > 0 && !tc::mbar_wait(&tempty[b], (u - 1) & 1, abort_flag, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const int send = min(nkb, (seg + 1) * TG_SEG);
        bool started[TG_LEV] = {false, false, false, false};
        for (; it < send; ++it) {
          const int s = it % TG_STAGES;
          if (!tc::mbar_wait(&full[s], (it / TG_STAGES) & 1, abort_flag, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * STAGE_BYTES);
          const uint32_t sb = sa + TG_SL * A_SLICE;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int lev = pa[q] + pb[q];
            const uint32_t d = tmem + (uint32_t)(b * TG_LEV * TG_N + lev * TG_N);
#pragma unroll
            for (int kk = 0; kk < TG_K / 16; ++kk) {
              const uint64_t da = tc::desc_kmajor_sw128(sa + pa[q] * A_SLICE + kk * 32);
              const uint64_t db = tc::desc_kmajor_sw128(sb + pb[q] * B_SLICE + kk * 32);
              tc::mma_bf16(d, da, db, idesc, started[lev] ? 1u : 0u);
              started[lev] = true;
            }
          }
          tc::commit(&empty[s]);  // the stage is free once these products finish
        }
        if (!ok) break;
        tc::commit(&tfull[b]);  // this segment's levels are complete
      }
      if (!ok) *abort_flag = 1;
      // every product issued has finished before tensor memory is released
      tc::commit(drain);
      tc::mbar_wait(drain, 0, nullptr, WAIT_LIMIT);
    }
    __syncwarp();
  } else {
    // drain warps: quadrant q of the tensor-memory lanes = tile rows 32q..32q+31
    const int q = warp & 3;
    float ah[TG_N], al[TG_N];
#pragma unroll
    for (int c = 0; c < TG_N; ++c) ah[c] = al[c] = 0.f;
    bool ok = true;
    for (int seg = 0; seg < nseg; ++seg) {
      const int b = seg & 1;
      // one lane polls; the warp then continues converged, as the
      // .sync.aligned tensor-memory loads and barriers below require
      int got = 1;
      if (lane == 0) got = tc::mbar_wait(&tfull[b], (seg >> 1) & 1, abort_flag, WAIT_LIMIT);
      __syncwarp();
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int c16 = 0; c16 < TG_N / 16; ++c16) {
        uint32_t v0[16], v1[16], v2[16], v3[16];
        const uint32_t base =
            tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * TG_LEV * TG_N + c16 * 16);
        tc::tmem_ld16(base, v0);
        tc::tmem_ld16(base + TG_N, v1);
        tc::tmem_ld16(base + 2 * TG_N, v2);
        tc::tmem_ld16(base + 3 * TG_N, v3);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          // exact integers: L0 + L1 2^-8 + L2 2^-16 + L3 2^-24 as a double-float
          float h = __uint_as_float(v0[j]), l = 0.f;
          df_add1(h, l, __uint_as_float(v1[j]) * 0x1p-8f);
          df_add1(h, l, __uint_as_float(v2[j]) * 0x1p-16f);
          df_add1(h, l, __uint_as_float(v3[j]) * 0x1p-24f);
          const int c = c16 * 16 + j;
          df_add1(ah[c], al[c], h);
          al[c] += l;
          df_norm(ah[c], al[c]);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
    }
    // stage the 128 x 64 tile in the (now idle) first pipeline stage, then
    // store it row by row with consecutive threads on consecutive columns
    float2* tile = reinterpret_cast<float2*>(smem);  // [128][TG_N + 1]
    if (!ok) {
      *abort_flag = 1;
    } else {
      const int r = 32 * q + lane;
#pragma unroll
      for (int c = 0; c < TG_N; ++c) tile[r * (TG_N + 1) + c] = make_float2(ah[c], al[c]);
    }
    __syncwarp();
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the four drain warps, always
    if (!*abort_flag) {
      const int t = threadIdx.x - 64;
      float2* base = P.part + (int64_t)blockIdx.y * P.M * P.N;
      for (int idx = t; idx < TG_M * TG_N; idx += 128) {
        const int rr = idx / TG_N, cc = idx % TG_N;
        if (row0 + rr < P.M && col0 + cc < P.N)
          base[(int64_t)(row0 + rr) * P.N + col0 + cc] = tile[rr * (TG_N + 1) + cc];
      }
    }
    __syncwarp();
  }
  // teardown: TMA copies still in flight (only after an abort) land before
  // the CTA exits; then tensor memory is released
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int it = max(0, issued - TG_STAGES); it < issued; ++it)
      tc::mbar_wait(&full[it % TG_STAGES], (it / TG_STAGES) & 1, nullptr, WAIT_LIMIT);
  }
  __syncwarp();
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) set_status(P.st, VL_ERR_TIMEOUT);
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Split-K partials (double-float) -> FP64, scaled by 2^(e_i + e_j - 14), into
// C[i][j] and C[j][i] for i <= j (symmetric mode).
__global__ void tg_reduce_sym_kernel(const float2* __restrict__ part, int splits, int N,
                                     const int* __restrict__ exps, double* __restrict__ C,
                                     int64_t ldc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int i = (int)(idx / N), j = (int)(idx % N);
  if (j < i) return;
  float h = 0.f, l = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float2 v = part[((int64_t)z * N + i) * N + j];
    df_add1(h, l, v.x);
    l += v.y;
  }
  const double v = ldexp((double)h + (double)l, exps[i] + exps[j] - 14);
  C[(int64_t)i * ldc + j] = v;
  C[(int64_t)j * ldc + i] = v;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of three bf16 slice planes S[z][r][k] (k < Kpad, a multiple of
// 64; r < rows; row stride ldo, plane stride plane, in elements), box of 64
// values of k x box_rows rows x 3 planes, 128-byte swizzle; rows beyond
// `rows` read as zeros.
bool make_slice_map(CUtensorMap* map, const void* S, int Kpad, int rows, int64_t ldo,
                    int64_t plane, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)TG_SL};
  const cuuint64_t strides[2] = {(cuuint64_t)ldo * 2, (cuuint64_t)plane * 2};
  const cuuint32_t box[3] = {(cuuint32_t)TG_K, (cuuint32_t)box_rows, (cuuint32_t)TG_SL};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(S), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int sym_tiles(int N, int& tiles_n) {
  const int tiles_m = (N + TG_M - 1) / TG_M;
  tiles_n = (N + TG_N - 1) / TG_N;
  int t = 0;
  for (int I = 0; I < tiles_m; ++I) t += std::max(0, tiles_n - 2 * I);
  return t;
}

}  // namespace

int64_t tg_kpad(int K) { return ((int64_t)K + TG_K - 1) / TG_K * TG_K; }

// Symmetric exact-slice Gram C = S S^T (N x N, FP64, ldc) of the N sliced
// rows in S.  Returns false if the tensor maps cannot be made (the caller
// then has no tensor-core path); launch errors surface at check_launch.
bool launch_tcgram_sym(const Ctx& cx, const void* S, int N, int Kpad, int64_t ldo, int64_t plane,
                       const int* exps, double* C, int64_t ldc) {
  CUtensorMap mA, mB;
  if (!make_slice_map(&mA, S, Kpad, N, ldo, plane, TG_M) ||
      !make_slice_map(&mB, S, Kpad, N, ldo, plane, TG_N))
    return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tcgram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TG_SMEM) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  TgParams P{};
  P.M = P.N = N;
  P.sym = 1;
  const int tiles = sym_tiles(N, P.tiles_n);
  P.nkb = Kpad / TG_K;
  // split K so that tiles x splits roughly fills the SMs, in whole segments,
  // within the partial buffer
  const int nseg = (P.nkb + TG_SEG - 1) / TG_SEG;
  // (one CTA per SM: a partial second wave would double the time)
  int splits = std::max(1, std::min(nseg, cx.num_sms / std::max(1, tiles)));
  const size_t per = (size_t)N * N;
  splits = (int)std::max<size_t>(1, std::min<size_t>(splits, cx.part_cap / per));
  P.kb_per_split = (P.nkb + splits - 1) / splits;  // a CTA forms its own segments
  splits = (P.nkb + P.kb_per_split - 1) / P.kb_per_split;
  P.part = reinterpret_cast<float2*>(cx.part);
  P.st = cx.st;
  note_launch();
  tcgram_kernel<<<dim3(tiles, splits), TG_THREADS, TG_SMEM, cx.s>>>(mA, mB, P);
  note_launch();
  tg_reduce_sym_kernel<<<(unsigned)((per + 255) / 256), 256, 0, cx.s>>>(P.part, splits, N, exps,
                                                                       C, ldc);
  return true;
}

// The VAR residuals on the tensor cores: E = X[:, p:] - mu - cst - sum_tau
// M_tau Z_tau with beta (FP32, mp x m) and the centred FP32 series Xc;
// vexp: the variables' exponents (those of the lag slicing).  Scratch: St
// (3 n kp bf16), Sb (3 m p kp bf16), aexp (m ints); the partials in the
// context's split-K buffer (m n_eff float2).  kp = tg_kpad(m).
bool launch_tc_var_resid(const Ctx& cx, const float* Xc, int64_t ldc, const double* X,
                         int64_t ldx, int m, int n, int p, const float* beta, const int* vexp,
                         const double* mu, const double* cst, void* St, void* Sb, int* aexp,
                         double* E) {
  const int kp = (int)tg_kpad(m), n_eff = n - p, K = p * kp;
  const int64_t plane_t = (int64_t)n * kp, plane_b = (int64_t)m * K;
  if ((size_t)m * n_eff > cx.part_cap) return false;
  note_launch();
  slice_time_kernel<<<dim3((n + 31) / 32, kp / 32), dim3(32, 8), 0, cx.s>>>(
      Xc, ldc, m, n, kp, vexp, static_cast<__nv_bfloat16*>(St), plane_t);
  note_launch();
  slice_beta_kernel<<<m, 256, 0, cx.s>>>(beta, m, p, kp, vexp, static_cast<__nv_bfloat16*>(Sb),
                                          plane_b, aexp);
  CUtensorMap mA, mB;
  if (!make_slice_map(&mA, Sb, K, m, K, plane_b, TG_M) ||
      !make_slice_map(&mB, St, kp, n, kp, plane_t, TG_N))
    return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tcgram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TG_SMEM) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  TgParams P{};
  P.M = m;
  P.N = n_eff;
  P.sym = 0;
  P.tiles_n = (n_eff + TG_N - 1) / TG_N;
  const int tiles = ((m + TG_M - 1) / TG_M) * P.tiles_n;
  P.nkb = K / TG_K;
  P.kb_per_split = P.nkb;  // one split: the tiles fill the GPU
  P.lag_kb = kp / TG_K;
  P.lag_p = p;
  P.part = reinterpret_cast<float2*>(cx.part);
  P.st = cx.st;
  note_launch();
  tcgram_kernel<<<dim3(tiles, 1), TG_THREADS, TG_SMEM, cx.s>>>(mA, mB, P);
  note_launch();
  resid_apply_kernel<<<dim3((n_eff + 255) / 256 < 16 ? (n_eff + 255) / 256 : 16, m), 256, 0,
                       cx.s>>>(X, ldx, m, n_eff, p, mu, cst, P.part, aexp, E);
  return true;
}

void launch_slice_center(const double* E, int64_t lde, const double* mu, int m, int K,
                         int64_t Kpad, void* S, int64_t plane, int* exps, cudaStream_t s) {
  note_launch();
  slice_center_kernel<<<m, 256, 0, s>>>(E, lde, mu, K, (int)Kpad,
                                         static_cast<__nv_bfloat16*>(S), Kpad, plane, exps);
}

void launch_slice_lags(const float* Xc, int64_t ldc, int m, int n, int p, int64_t Kpad, void* S,
                       int64_t plane, int* exps, cudaStream_t s) {
  note_launch();
  slice_lags_kernel<<<m, 256, 0, s>>>(Xc, ldc, m, n, p, (int)Kpad,
                                       static_cast<__nv_bfloat16*>(S), Kpad, plane, exps);
}

}  // namespace vl
