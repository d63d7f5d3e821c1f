// Certified Algorithm 1 under an FP32 measure: near ties of Eq. 3 are decided
// on entries of D re-evaluated to FP64 accuracy.
//
// The mixed-precision measure gives D to about 1e-6 of max|D| (the per-sample
// functions run in FP32), which moves the scores S_i = sum_{j in U, j != i}
// min(0, D_ij)^2 of Eq. 3 by about 5e-5 relative (4e-4 at the 99th
// percentile, measured against the FP64 path on 260 series).  Where two
// candidates of a step lie closer than that, the FP32 measure may pick the
// other one.  After the search on the FP32 D:
//   1. flag: every variable replays its score over the steps of the found
//      order; step k is flagged when some other candidate's score, lowered by
//      its error band, reaches the picked score raised by its band.  The band
//      of a score S over u remaining variables is
//          tau S + c dmax sqrt(S) + u (eta dmax)^2,
//      tau = 1e-3, c = 1e-5, eta = 1e-5, dmax = max|D| (a relative part, a
//      part for the spread of small scores, and a floor for scores near zero;
//      on the 260 calibration series no score error exceeded its band and
//      every differing pick was flagged).
//   2. mark: for the candidates of every flagged step, the pairs (i, j) with
//      j still remaining are queued once (a bitset dedups them across steps
//      and rounds), except entries D_ij so clearly positive that their exact
//      value is positive too (they add nothing to Eq. 3).
//   3. re-evaluate the queued pairs from the data E: the rows standardized in
//      FP64 and kept as double-float pairs (df64.cuh, about 48 bits), rho, both
//      standardized residuals and the per-sample functions of their entropies
//      in double-float arithmetic, the sums and D_ij = H(x_j) + H(r_i<-j) -
//      H(x_i) - H(r_j<-i) in FP64.  The per-sample log cosh and u e^{-u^2/2}
//      agree with FP64 to 3e-14 absolute (measured over 2M samples with light
//      and heavy tails), six orders of magnitude below the smallest score gap
//      the decision has to resolve, at a thirteenth of the FP64 cost on this part.
//   4. decide: every flagged step recomputes its candidates' exact scores over
//      its remaining set and takes the argmin (ties: lowest index).  The first
//      step whose pick changes is resumed: the search restarts there with the
//      corrected pick and runs to the end on the FP32 scores.
// Steps 1-4 repeat from the step after a changed pick (at most CERT_ROUNDS
// times).  Everything stays on the device: no host synchronisation, a fixed
// launch sequence (rounds with nothing to do exit at once).
#include <algorithm>

#include "df64.cuh"
#include "order_search.cuh"

namespace vl {

namespace {

using namespace search;

constexpr int CMAX = 16;         // candidates recorded per flagged step
constexpr int CERT_ROUNDS = 3;   // flag / re-evaluate / decide / resume rounds
constexpr double CERT_TAU = 1e-3;
constexpr double CERT_C = 1e-5;
constexpr double CERT_ETA = 1e-5;
constexpr int RTH = 256;         // threads of the block-per-item kernels

// control words
enum { C_ACTIVE = 0, C_K0, C_FIRST, C_ANY, C_NPAIRS, C_HXREADY, C_NCTRL };

__device__ __forceinline__ double cert_band(double S, int u, double dmax) {
  const double e = CERT_ETA * dmax;
  return CERT_TAU * fabs(S) + CERT_C * dmax * sqrt(fmax(S, 0.0)) + (double)u * e * e;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
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

// max |D| (as the bits of a non-negative double, which order like integers)
// and the control words of round 0.
__global__ void cert_init_kernel(const double* __restrict__ D, int m, int* ctrl,
                                 unsigned long long* dmax_bits) {
  __shared__ double red[32];
  double v = 0.0;
  const int64_t tot = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x)
    v = fmax(v, fabs(D[idx]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b = fmax(b, red[q]);
    atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(b));
    if (blockIdx.x == 0) {
      ctrl[C_ACTIVE] = 1;
      ctrl[C_K0] = 0;
      ctrl[C_FIRST] = m;
      ctrl[C_ANY] = 0;
      ctrl[C_NPAIRS] = 0;
      ctrl[C_HXREADY] = 0;
    }
  }
}

// Start of a round: positions of the current order, cleared step flags; from
// round 1 on, the round runs only if the previous one changed a pick, from
// the step after it.
__global__ void cert_round_kernel(const int32_t* __restrict__ order, int m, int round, int* ctrl,
                                  int* __restrict__ pos, int* __restrict__ flag,
                                  int* __restrict__ ccount, const double* __restrict__ spick,
                                  const unsigned long long* __restrict__ dmax_bits,
                                  float* __restrict__ thr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) {
    pos[order[t]] = t;
    flag[t] = 0;
    ccount[t] = 0;
    // the picked score of step t raised by its band, rounded up to FP32
    const double dmax = __longlong_as_double((long long)*dmax_bits);
    const double sc = spick[t];
    thr[t] = __double2float_ru(sc + cert_band(sc, m - t, dmax));
  }
  if (t == 0 && round > 0) {
    const int fc = ctrl[C_FIRST];
    ctrl[C_ACTIVE] = fc < m ? 1 : 0;
    ctrl[C_K0] = fc + 1;
    ctrl[C_FIRST] = m;
    ctrl[C_ANY] = 0;
    ctrl[C_NPAIRS] = 0;
  }
}

// 1. flag.  Variable i replays its FP32-measure score over the steps before
// its own pick (as a double-float pair, the search's own arithmetic) and, at
// every step k >= k0, compares its score lowered by its band with thr[k], the
// picked score raised by its band.  The lowered score is formed in FP32 with
// the band widened by 1e-3 of itself (at least 1e-6 of the score, several
// times FP32's rounding error), so the test flags every step the exact
// comparison would.  One warp per block, so the m independent replays spread
// over ceil(m / 32) SMs; the order and the thresholds are staged in shared
// memory (a threshold load from L2 on every step put ~400 clocks of latency
// on each step's branch) and the P entries of the next eight steps are
// loaded while the current eight are replayed.
constexpr int FLAG_GROUP = 8;

__device__ __forceinline__ void flag_load(const float* __restrict__ pth,
                                          const float* __restrict__ ptl, const int* ord, int m,
                                          int i, int pi, int t0, float* h, float* l) {
#pragma unroll
  for (int u = 0; u < FLAG_GROUP; ++u) {
    const int c = t0 + u < pi ? ord[t0 + u] : i;
    h[u] = pth[(int64_t)c * m + i];
    l[u] = ptl[(int64_t)c * m + i];
  }
}

__global__ void __launch_bounds__(32)
    cert_flag_kernel(const float* __restrict__ pth, const float* __restrict__ ptl,
                     const float* __restrict__ sh0, const float* __restrict__ sl0,
                     const int32_t* __restrict__ order, const int* __restrict__ pos,
                     const float* __restrict__ thr, int m, int* ctrl,
                     const unsigned long long* __restrict__ dmax_bits, int* __restrict__ flag,
                     int* __restrict__ ccount, int* __restrict__ cand) {
  extern __shared__ int ord_s[];  // m order entries, then m thresholds
  float* thr_s = reinterpret_cast<float*>(ord_s + m);
  if (!ctrl[C_ACTIVE]) return;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    ord_s[t] = order[t];
    thr_s[t] = thr[t];
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int k0 = ctrl[C_K0], pi = pos[i];
  const float dmax = (float)__longlong_as_double((long long)*dmax_bits);
  const float bc = (float)CERT_C * dmax, be = (float)CERT_ETA * dmax;
  df::F2 s{sh0[i], sl0[i]};
  float ph[FLAG_GROUP], pl[FLAG_GROUP], nh[FLAG_GROUP], nl[FLAG_GROUP];
  if (pi > 0) flag_load(pth, ptl, ord_s, m, i, pi, 0, ph, pl);
  for (int t0 = 0; t0 < pi; t0 += FLAG_GROUP) {
    if (t0 + FLAG_GROUP < pi) flag_load(pth, ptl, ord_s, m, i, pi, t0 + FLAG_GROUP, nh, nl);
    // the group's scores first (the only dependent chain), then its tests
    float sf[FLAG_GROUP];
#pragma unroll
    for (int u = 0; u < FLAG_GROUP; ++u) {
      sf[u] = s.hi + s.lo;
      s = df::add(s, df::F2{-ph[u], -pl[u]});
    }
#pragma unroll
    for (int u = 0; u < FLAG_GROUP; ++u) {
      const int k = t0 + u;
      if (k >= pi) break;
      if (k >= k0) {
        const float band = ((float)CERT_TAU * fabsf(sf[u]) + bc * sqrtf(fmaxf(sf[u], 0.0f)) +
                            (float)(m - k) * be * be) * 1.001f;
        if (sf[u] - band <= thr_s[k]) {
          flag[k] = 1;
          ctrl[C_ANY] = 1;
          const int slot = atomicAdd(&ccount[k], 1);
          if (slot < CMAX) cand[(int64_t)k * CMAX + slot] = i;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < FLAG_GROUP; ++u) {
      ph[u] = nh[u];
      pl[u] = nl[u];
    }
  }
}

// 2. mark.  Block k (a flagged step): for the pick and every candidate i, the
// pairs (i, j) with j still remaining at step k are queued once, except those
// whose entry D_ij exceeds CERT_POS max|D| (five times the largest FP32-measure
// error seen): their exact entry is positive as well and adds nothing to
// i's score.
constexpr double CERT_POS = 5e-5;
__global__ void __launch_bounds__(RTH)
    cert_mark_kernel(const double* __restrict__ D, const int32_t* __restrict__ order,
                     const int* __restrict__ pos, int m, int* ctrl,
                     const unsigned long long* __restrict__ dmax_bits,
                     const int* __restrict__ flag, const int* __restrict__ ccount,
                     const int* __restrict__ cand, unsigned* __restrict__ need,
                     const unsigned* __restrict__ done, int2* __restrict__ pairs,
                     int* __restrict__ stats) {
  const int k = blockIdx.x;
  const double pos_thr = CERT_POS * __longlong_as_double((long long)*dmax_bits);
  if (!ctrl[C_ACTIVE] || k < ctrl[C_K0] || !flag[k]) return;
  const int cnt = ccount[k];
  if (cnt > CMAX) {  // too many candidates: this step is left as the FP32 search took it
    if (threadIdx.x == 0) atomicAdd(&stats[3], 1);
    return;
  }
  if (threadIdx.x == 0) atomicAdd(&stats[0], 1);
  for (int q = 0; q <= cnt; ++q) {
    const int i = q == 0 ? order[k] : cand[(int64_t)k * CMAX + q - 1];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      if (j == i || pos[j] < k || D[(int64_t)i * m + j] > pos_thr) continue;
      const int a = min(i, j), b = max(i, j);
      const int64_t bit = (int64_t)a * m + b;
      const unsigned mask = 1u << (bit & 31);
      if (done[bit >> 5] & mask) continue;
      const unsigned old = atomicOr(&need[bit >> 5], mask);
      if (!(old & mask)) pairs[atomicAdd(&ctrl[C_NPAIRS], 1)] = make_int2(a, b);
    }
  }
}

// Moments of one standardized sample u in double-float: |u| + log1p(e^{-2|u|})
// (= log cosh u + ln 2; the ln 2 is taken off the mean in FP64) into a, and
// u e^{-u^2/2} into b.  tab: the exp table in shared memory.
__device__ __forceinline__ void moments_df(df::F2 u, df::F2& a, df::F2& b, const float2* tab) {
  const df::F2 au = u.hi < 0.0f ? df::neg(u) : u;
  const df::F2 y = df::dexp(df::scale(au, -2.0f), tab);
  a = df::add(a, df::add(au, df::dlog1p(y, tab)));
  b = df::add(b, df::mul(u, df::dexp(df::scale(df::sqr(u), -0.5f), tab)));
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 3a. Block i, once per call and only when some step was flagged: FP64 mean
// and 1/std of row i of E, the standardized row x_i as double-float pairs
// (xs, row stride n) for the pair kernel, and the entropy H(x_i).
__global__ void __launch_bounds__(RTH)
    cert_stats_kernel(const double* __restrict__ E, int64_t lde, int m, int n, const int* ctrl,
                      float2* __restrict__ xs, double* __restrict__ hx) {
  __shared__ double red[32];
  __shared__ float2 tab[32];
  if (!ctrl[C_ACTIVE] || !ctrl[C_ANY] || ctrl[C_HXREADY]) return;
  if (threadIdx.x < 32) tab[threadIdx.x] = df::kExp2Frac[threadIdx.x];
  const int i = blockIdx.x;
  const double* e = E + (int64_t)i * lde;
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += e[t];
  const double mean = block_sum_d(s, red) / n;
  double q = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double d = e[t] - mean;
    q += d * d;
  }
  const double var = block_sum_d(q, red) / n;
  const double is = var > 1e-300 ? 1.0 / sqrt(var) : 0.0;
  df::F2 a{0.0f, 0.0f}, b{0.0f, 0.0f};
  float2* xr = xs + (int64_t)i * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const df::F2 x = df::from_double((e[t] - mean) * is);
    xr[t] = make_float2(x.hi, x.lo);
    moments_df(x, a, b, tab);
  }
  const double sa = block_sum_d(df::to_double(a), red);
  const double sb = block_sum_d(df::to_double(b), red);
  if (threadIdx.x == 0) hx[i] = entropy_from_moments(sa / n - LN2, sb / n);
}

// 3b. Re-evaluation of the queued pairs, one warp per pair (a, b): rho =
// mean(x_a x_b) of the standardized rows, the moments of both standardized
// residuals u = (x_a - rho x_b) / sqrt(1 - rho^2) and v (roles swapped) in
// double-float, their sums and entropies in FP64, and D_ab = -D_ba into the
// cache D64.
__global__ void __launch_bounds__(RTH)
    cert_pairs_kernel(const float2* __restrict__ xs, int m, int n, const int* ctrl,
                      const double* __restrict__ hx, const int2* __restrict__ pairs,
                      double* __restrict__ D64, unsigned* __restrict__ done,
                      int* __restrict__ stats) {
  __shared__ float2 tab[32];
  if (!ctrl[C_ACTIVE] || !ctrl[C_ANY]) return;
  if (threadIdx.x < 32) tab[threadIdx.x] = df::kExp2Frac[threadIdx.x];
  __syncthreads();
  const int np = ctrl[C_NPAIRS];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < np; w += nwarps) {
    const int2 pr = pairs[w];
    const int a = pr.x, b = pr.y;
    const float2* xa = xs + (int64_t)a * n;
    const float2* xb = xs + (int64_t)b * n;
    df::F2 c{0.0f, 0.0f};
    for (int t = lane; t < n; t += 32) {
      const float2 p = xa[t], q = xb[t];
      c = df::add(c, df::mul(df::F2{p.x, p.y}, df::F2{q.x, q.y}));
    }
    const double rho = warp_sum_d(df::to_double(c)) / n;
    double dab = 0.0;
    if (1.0 - rho * rho >= DEGENERATE_1MR2) {
      const df::F2 r = df::from_double(rho);
      const df::F2 sc = df::from_double(1.0 / sqrt(1.0 - rho * rho));
      df::F2 au{0.0f, 0.0f}, bu{0.0f, 0.0f}, av{0.0f, 0.0f}, bv{0.0f, 0.0f};
      for (int t = lane; t < n; t += 32) {
        const float2 p = xa[t], q = xb[t];
        const df::F2 fa{p.x, p.y}, fb{q.x, q.y};
        moments_df(df::mul(sc, df::add(fa, df::neg(df::mul(r, fb)))), au, bu, tab);
        moments_df(df::mul(sc, df::add(fb, df::neg(df::mul(r, fa)))), av, bv, tab);
      }
      const double sau = warp_sum_d(df::to_double(au)), sbu = warp_sum_d(df::to_double(bu));
      const double sav = warp_sum_d(df::to_double(av)), sbv = warp_sum_d(df::to_double(bv));
      const double hab = entropy_from_moments(sau / n - LN2, sbu / n);  // H(r_{a<-b})
      const double hba = entropy_from_moments(sav / n - LN2, sbv / n);  // H(r_{b<-a})
      dab = hx[b] + hab - hx[a] - hba;
    }
    if (lane == 0) {
      D64[(int64_t)a * m + b] = dab;
      D64[(int64_t)b * m + a] = -dab;
      const int64_t bit = (int64_t)a * m + b;
      atomicOr(&done[bit >> 5], 1u << (bit & 31));
      atomicAdd(&stats[1], 1);
    }
  }
}

// 4a. decide.  Block k (a flagged step): exact scores of the pick and its
// candidates over the variables remaining at step k from the FP64 entries
// (an entry that was not re-evaluated is certainly positive and adds 0); the
// argmin (ties: lowest index).  A different pick is recorded and the first
// such step becomes the resume point.
__global__ void __launch_bounds__(RTH)
    cert_decide_kernel(const int32_t* __restrict__ order, const int* __restrict__ pos, int m,
                       int* ctrl, const int* __restrict__ flag, const int* __restrict__ ccount,
                       const int* __restrict__ cand, const double* __restrict__ D64,
                       const unsigned* __restrict__ done, int* __restrict__ pick) {
  __shared__ double red[32];
  __shared__ double sc[CMAX + 1];
  const int k = blockIdx.x;
  if (!ctrl[C_ACTIVE] || k < ctrl[C_K0] || !flag[k]) return;
  if (threadIdx.x == 0) ctrl[C_HXREADY] = 1;  // the entropies and standardized rows exist from now on
  const int cnt = ccount[k];
  if (cnt > CMAX) return;
  for (int q = 0; q <= cnt; ++q) {
    const int i = q == 0 ? order[k] : cand[(int64_t)k * CMAX + q - 1];
    double s = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      if (j == i || pos[j] < k) continue;
      const int64_t bit = (int64_t)min(i, j) * m + max(i, j);
      if (!(done[bit >> 5] & (1u << (bit & 31)))) continue;
      const double d = D64[(int64_t)i * m + j];
      if (d < 0.0) s += d * d;
    }
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) sc[q] = s;
  }
  if (threadIdx.x == 0) {
    int best = order[k];
    double bs = sc[0];
    for (int q = 1; q <= cnt; ++q) {
      const int i = cand[(int64_t)k * CMAX + q - 1];
      if (sc[q] < bs || (sc[q] == bs && i < best)) {
        bs = sc[q];
        best = i;
      }
    }
    if (best != order[k]) {
      pick[k] = best;
      atomicMin(&ctrl[C_FIRST], k);
    }
  }
}

// 4b. resume.  If a pick changed, the search restarts at the first such step
// k*: every remaining variable rebuilds its double-float score by the same
// subtractions the first search made over steps 0 .. k*-1, step k* takes the
// corrected pick, and the remaining steps search as before.
template <int PER>
__global__ void __launch_bounds__(OTH)
    cert_resume_kernel(const float* __restrict__ pth, const float* __restrict__ ptl,
                       const float* __restrict__ sh0, const float* __restrict__ sl0, int m,
                       int32_t* __restrict__ order, const int* __restrict__ pos,
                       const int* __restrict__ pick, const int* ctrl,
                       double* __restrict__ spick, int* __restrict__ stats) {
  if (!ctrl[C_ACTIVE]) return;
  const int ks = ctrl[C_FIRST];
  if (ks >= m) return;
  if (threadIdx.x == 0) atomicAdd(&stats[2], 1);
  float hi[PER], lo[PER];
  bool alive[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = threadIdx.x + q * blockDim.x;
    alive[q] = i < m && pos[i] >= ks;
    hi[q] = alive[q] ? sh0[i] : 0.f;
    lo[q] = alive[q] ? sl0[i] : 0.f;
  }
  for (int l = 0; l < ks; ++l) {
    const int c = order[l];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = threadIdx.x + q * blockDim.x;
      if (alive[q]) df_sub(hi[q], lo[q], pth[(int64_t)c * m + i], ptl[(int64_t)c * m + i]);
    }
  }
  // every thread has read order[0 .. ks-1] before thread 0 overwrites order[ks ..]
  __syncthreads();
  search_steps<PER>(hi, lo, alive, m, ks, pick[ks], order, spick, nullptr,
                    [&](int c, int i, float& h, float& l) {
                      h = pth[(int64_t)c * m + i];
                      l = ptl[(int64_t)c * m + i];
                    });
}

// Steps after a pick changed in the last round were not verified again.
__global__ void cert_tail_kernel(int m, const int* ctrl, int* stats) {
  if (ctrl[C_ACTIVE] && ctrl[C_FIRST] < m) atomicAdd(&stats[3], 1);
}

}  // namespace

namespace {

// Device layout of the certification's workspace (base NULL: sizes only).
struct CertWs {
  int* ctrl;
  unsigned long long* dmax;
  int* stats;
  int *pos, *flag, *ccount, *cand, *pick;
  double *spick, *hx, *D64;
  float* thr;
  unsigned *need, *done;
  int2* pairs;
  float2* xs;
  size_t bits_words;
  size_t bytes;
};

// n: samples of the standardized rows kept for the pair kernel (they come
// last, so the other fields do not depend on n)
CertWs cert_layout(void* base, int m, int n) {
  Arena a;
  a.base = static_cast<char*>(base);
  CertWs w{};
  const size_t mm = (size_t)m * m;
  w.ctrl = a.take<int>(C_NCTRL);
  w.dmax = a.take<unsigned long long>(1);
  w.stats = a.take<int>(4);
  w.bits_words = (mm + 31) / 32;
  w.need = a.take<unsigned>(w.bits_words);
  w.done = a.take<unsigned>(w.bits_words);
  w.pos = a.take<int>(m);
  w.flag = a.take<int>(m);
  w.ccount = a.take<int>(m);
  w.cand = a.take<int>((size_t)m * CMAX);
  w.pick = a.take<int>(m);
  w.spick = a.take<double>(m);
  w.thr = a.take<float>(m);
  w.hx = a.take<double>(m);
  w.D64 = a.take<double>(mm);
  w.pairs = a.take<int2>(mm / 2 + 1);
  w.xs = a.take<float2>((size_t)m * n);
  w.bytes = a.off + 256;
  return w;
}

}  // namespace

size_t certify_ws_bytes(int m, int n) { return cert_layout(nullptr, m, n).bytes; }

double* certify_spick(void* cert_ws, int m) { return cert_layout(cert_ws, m, 0).spick; }

void launch_certify(const double* D, const double* E, int64_t lde, int m, int n, void* order_ws,
                    void* cert_ws, int32_t* order, int32_t* stats_out, int num_sms,
                    cudaStream_t s) {
  const OrderWs ow = order_ws_layout(order_ws, m);
  CertWs w = cert_layout(cert_ws, m, n);
  // the control words, counters and bitsets start at zero (they are laid out
  // first, contiguously)
  cudaMemsetAsync(w.ctrl, 0, reinterpret_cast<char*>(w.pos) - reinterpret_cast<char*>(w.ctrl), s);
  const int gb = (m + 255) / 256;
  note_launch();
  cert_init_kernel<<<std::min(1024, std::max(1, (int)(((size_t)m * m + 255) / 256))), 256, 0, s>>>(
      D, m, w.ctrl, w.dmax);
  const int per = m <= OTH ? 1 : (m <= 2 * OTH ? 2 : 4);
  const int nthr = std::min(OTH, ((m + per - 1) / per + 31) / 32 * 32);
  for (int r = 0; r < CERT_ROUNDS; ++r) {
    note_launch();
    cert_round_kernel<<<gb, 256, 0, s>>>(order, m, r, w.ctrl, w.pos, w.flag, w.ccount, w.spick,
                                         w.dmax, w.thr);
    note_launch();
    cert_flag_kernel<<<(m + 31) / 32, 32, 8 * (size_t)m, s>>>(ow.pth, ow.ptl, ow.sh, ow.sl, order, w.pos,
                                                   w.thr, m, w.ctrl, w.dmax, w.flag, w.ccount,
                                                   w.cand);
    note_launch();
    cert_mark_kernel<<<m, RTH, 0, s>>>(D, order, w.pos, m, w.ctrl, w.dmax, w.flag, w.ccount,
                                      w.cand, w.need, w.done, w.pairs, w.stats);
    note_launch();
    cert_stats_kernel<<<m, RTH, 0, s>>>(E, lde, m, n, w.ctrl, w.xs, w.hx);
    note_launch();
    cert_pairs_kernel<<<4 * num_sms, RTH, 0, s>>>(w.xs, m, n, w.ctrl, w.hx, w.pairs, w.D64,
                                                  w.done, w.stats);
    note_launch();
    cert_decide_kernel<<<m, RTH, 0, s>>>(order, w.pos, m, w.ctrl, w.flag, w.ccount, w.cand,
                                        w.D64, w.done, w.pick);
    note_launch();
    if (per == 1)
      cert_resume_kernel<1><<<1, nthr, 0, s>>>(ow.pth, ow.ptl, ow.sh, ow.sl, m, order, w.pos,
                                               w.pick, w.ctrl, w.spick, w.stats);
    else if (per == 2)
      cert_resume_kernel<2><<<1, nthr, 0, s>>>(ow.pth, ow.ptl, ow.sh, ow.sl, m, order, w.pos,
                                               w.pick, w.ctrl, w.spick, w.stats);
    else
      cert_resume_kernel<4><<<1, nthr, 0, s>>>(ow.pth, ow.ptl, ow.sh, ow.sl, m, order, w.pos,
                                               w.pick, w.ctrl, w.spick, w.stats);
  }
  note_launch();
  cert_tail_kernel<<<1, 1, 0, s>>>(m, w.ctrl, w.stats);
  if (stats_out)
    cudaMemcpyAsync(stats_out, w.stats, 4 * sizeof(int), cudaMemcpyDeviceToDevice, s);
}

}  // namespace vl
