// Cholesky factorisation A = L L^T of an FP32 SPD matrix (n <= 512) by one
// thread-block cluster: the normal-equation matrix of the VAR fit (Sec. 4.1)
// and the causally ordered residual covariance whose factor gives B0 (Sec. 4.2
// item 5) are both factored here on the mixed-precision path.
//
// GB300 design.  n <= 512 is far too small to fill the GPU, and one CTA
// alone spends most of its time on the trailing updates, so the factorisation
// runs on a cluster of up to 8 CTAs (one per SM) that keep the whole matrix in
// their shared memory: the 32-wide block columns are dealt round-robin to the
// CTAs.  Block column k is factored by its owner (diagonal block by one warp,
// its inverse, then the panel below it); the other CTAs read the finished
// panel straight out of the owner's shared memory (distributed shared memory)
// and apply it to their own block columns.  One hardware cluster barrier per
// block column orders the two.  Look-ahead: the owner of block column k + 1
// applies panel k to that column first, factors it and signals, and only then
// applies panel k to its other columns, so the serial chain per block column
// is: copy panel, update one block column, factor 32 x 32, invert, panel.
//
// Outputs follow the multi-kernel path: L in the lower triangle of A (the
// strict upper triangle is left as it was) and, per 64-block of rows, the
// inverse of the 64 x 64 diagonal block of L (dinv), built from the two 32 x 32
// inverses as [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}].
// A pivot at or below rel_tol * (its original diagonal) sets VL_ERR_RANK.
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int CB = 32;        // block column width
constexpr int RS = CB + 4;    // shared row stride: 16-byte rows, conflict-free float4 columns
constexpr int CL_MAX = 8;     // CTAs per cluster (portable maximum)
constexpr int CTH = 512;      // threads per CTA
constexpr int CL_NMAX = 512;  // largest n handled
#ifndef VL_CHOL_RB
#define VL_CHOL_RB 4
#endif
constexpr int RB = VL_CHOL_RB;  // rows per warp pass in the panel and update

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// shared::cta address of this CTA -> shared::cluster address in CTA `rank`
__device__ __forceinline__ unsigned map_rank(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float4 ld_cluster4(unsigned addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// Shared-memory layout of one CTA (floats):
//   own   owned block columns, each rows k0 .. n-1 of 32 columns (stride RS)
//   pbuf  copy of the current panel, rows (k+1)*32 .. n-1 (stride RS)
//   li    32 x 32 inverses of the owned diagonal blocks (stride RS)
//   scr   64 rows of scratch: the diagonal factor's columns, then its rows;
//         the partner inverse and B A^{-1} when combining 64-blocks
struct Layout {
  int n, nblk, cl, rank;
  // offset (in rows) of owned block b inside `own`
  __host__ __device__ int own_row0(int b) const {
    int r = 0;
    for (int c = rank; c < b; c += cl) r += n - c * CB;
    return r;
  }
  __host__ __device__ int own_rows() const {
    int r = 0;
    for (int c = rank; c < nblk; c += cl) r += n - c * CB;
    return r;
  }
  __host__ __device__ int n_owned() const { return nblk > rank ? (nblk - 1 - rank) / cl + 1 : 0; }
};

// rows of shared memory (each RS floats): own, pbuf, li, scr (64 rows)
inline size_t cluster_chol_smem(int n, int cl, int rank) {
  Layout L{n, (n + CB - 1) / CB, cl, rank};
  const size_t rows = (size_t)L.own_rows() + std::max(0, n - CB) + (size_t)L.n_owned() * CB + 2 * CB;
  return rows * RS * sizeof(float);
}

// Warp 0: factor the diagonal block (rows of `blk`, nb valid rows/columns;
// identity padding beyond nb) in place; its rows also go to scr.  Lane r
// holds row r in registers; column j of the factor is published through
// shared memory (scr row j) and read back as float4 broadcasts for the rank-1
// update of the remaining columns.  Returns true if a pivot failed the
// relative threshold.
__device__ __noinline__ bool factor_diag(float* blk, int nb, const double* diag0k,
                                         float rel_tol, float* scr) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  float a[CB];
#pragma unroll
  for (int c4 = 0; c4 < CB; c4 += 4) {
    const float4 v = lane < nb ? *reinterpret_cast<const float4*>(blk + lane * RS + c4)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    a[c4] = v.x;
    a[c4 + 1] = v.y;
    a[c4 + 2] = v.z;
    a[c4 + 3] = v.w;
  }
#pragma unroll
  for (int c = 0; c < CB; ++c)
    if (!(lane < nb && c < nb && c <= lane)) a[c] = (c == lane) ? 1.f : 0.f;
  const float thr = lane < nb ? (float)(rel_tol * diag0k[lane]) : 0.f;
  bool lbad = false;
  float* ip = scr + (2 * CB - 1) * RS;  // 1 / L[j][j]
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    float d = __shfl_sync(full, a[j], j);
    const float tj = __shfl_sync(full, thr, j);
    if (!(d > tj)) {
      lbad |= (j < nb);
      d = 1.f;
    }
    const float ipv = rsqrtf(d);
    if (lane == 0) ip[j] = ipv;
    const float l = (lane > j) ? a[j] * ipv : (lane == j ? d * ipv : 0.f);
    scr[j * RS + lane] = l;  // column j of L
    __syncwarp();
#pragma unroll
    for (int c4 = ((j + 1) & ~3); c4 < CB; c4 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(scr + j * RS + c4);
      if (c4 > j) a[c4] = fmaf(-l, v.x, a[c4]);
      if (c4 + 1 > j) a[c4 + 1] = fmaf(-l, v.y, a[c4 + 1]);
      if (c4 + 2 > j) a[c4 + 2] = fmaf(-l, v.z, a[c4 + 2]);
      if (c4 + 3 > j) a[c4 + 3] = fmaf(-l, v.w, a[c4 + 3]);
    }
    a[j] = l;
  }
  __syncwarp();
  // rows of L (strict upper part zero) to scr and, for rows that exist, to blk
#pragma unroll
  for (int c4 = 0; c4 < CB; c4 += 4) {
    const float4 v = make_float4(c4 <= lane ? a[c4] : 0.f, c4 + 1 <= lane ? a[c4 + 1] : 0.f,
                                 c4 + 2 <= lane ? a[c4 + 2] : 0.f, c4 + 3 <= lane ? a[c4 + 3] : 0.f);
    *reinterpret_cast<float4*>(scr + lane * RS + c4) = v;
    if (lane < nb) *reinterpret_cast<float4*>(blk + lane * RS + c4) = v;
  }
  __syncwarp();
  return __any_sync(full, lbad);
}

// Warp 0: inverse of the factored diagonal block whose rows are in scr (and
// 1 / L[r][r] in scr row 63): lane c solves L x = e_c by forward substitution
// (no exchange between lanes); x[r] = Linv[r][c] goes to li.
__device__ __noinline__ void invert_diag(const float* scr, float* li) {
  const int lane = threadIdx.x & 31;
  const float* ip = scr + (2 * CB - 1) * RS;
  float x[CB];
#pragma unroll
  for (int r = 0; r < CB; ++r) {
    float s0 = (r == lane) ? 1.f : 0.f, s1 = 0.f;
#pragma unroll
    for (int q4 = 0; q4 < r; q4 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(scr + r * RS + q4);
      float& s = ((q4 >> 2) & 1) ? s1 : s0;
      s = fmaf(-v.x, x[q4], s);
      if (q4 + 1 < r) s = fmaf(-v.y, x[q4 + 1], s);
      if (q4 + 2 < r) s = fmaf(-v.z, x[q4 + 2], s);
      if (q4 + 3 < r) s = fmaf(-v.w, x[q4 + 3], s);
    }
    x[r] = (s0 + s1) * ip[r];
  }
#pragma unroll
  for (int r = 0; r < CB; ++r) li[r * RS + lane] = x[r];
}

// All warps: panel rows below the diagonal block of block column b,
// P[i][c] = sum_{q <= c} A[i][q] Linv[c][q], in place (rows 32 .. rows-1 of blk).
__device__ __forceinline__ void panel_rows(float* blk, int rows, const float* li) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float lr[CB];  // row `lane` of Linv
#pragma unroll
  for (int q4 = 0; q4 < CB; q4 += 4) {
    const float4 v = *reinterpret_cast<const float4*>(li + lane * RS + q4);
    lr[q4] = v.x;
    lr[q4 + 1] = v.y;
    lr[q4 + 2] = v.z;
    lr[q4 + 3] = v.w;
  }
  for (int i0 = CB + RB * warp; i0 < rows; i0 += RB * (CTH / 32)) {
    float acc[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) acc[u] = 0.f;
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const float* row = blk + (size_t)min(i0 + u, rows - 1) * RS;
#pragma unroll
      for (int q4 = 0; q4 < CB; q4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + q4);
        acc[u] = fmaf(v.x, lr[q4], acc[u]);
        acc[u] = fmaf(v.y, lr[q4 + 1], acc[u]);
        acc[u] = fmaf(v.z, lr[q4 + 2], acc[u]);
        acc[u] = fmaf(v.w, lr[q4 + 3], acc[u]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < RB; ++u)
      if (i0 + u < rows) blk[(size_t)(i0 + u) * RS + lane] = acc[u];
  }
}

// All warps: block column j (rows j0 .. n-1 in blk) minus the panel product,
// A_j[i][c] -= sum_q P[i][q] P[j0 + c][q]; panel row i is P + (i - prow0) * RS.
__device__ __noinline__ void update_block(float* blk, int j0, int n, const float* P,
                                             int prow0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float pj[CB];
  {
    const bool ok = j0 + lane < n;
    const float* row = P + (size_t)(min(j0 + lane, n - 1) - prow0) * RS;
#pragma unroll
    for (int q4 = 0; q4 < CB; q4 += 4) {
      const float4 v = ok ? *reinterpret_cast<const float4*>(row + q4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      pj[q4] = v.x;
      pj[q4 + 1] = v.y;
      pj[q4 + 2] = v.z;
      pj[q4 + 3] = v.w;
    }
  }
  const int rows = n - j0;
  for (int i0 = RB * warp; i0 < rows; i0 += RB * (CTH / 32)) {
    float old[RB], acc[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) acc[u] = 0.f;
#pragma unroll
    for (int u = 0; u < RB; ++u) old[u] = blk[(size_t)min(i0 + u, rows - 1) * RS + lane];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const float* row = P + (size_t)(j0 + min(i0 + u, rows - 1) - prow0) * RS;
#pragma unroll
      for (int q4 = 0; q4 < CB; q4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + q4);
        acc[u] = fmaf(v.x, pj[q4], acc[u]);
        acc[u] = fmaf(v.y, pj[q4 + 1], acc[u]);
        acc[u] = fmaf(v.z, pj[q4 + 2], acc[u]);
        acc[u] = fmaf(v.w, pj[q4 + 3], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < RB; ++u)
      if (i0 + u < rows) blk[(size_t)(i0 + u) * RS + lane] = old[u] - acc[u];
  }
}

// Factor block column b owned by this CTA: warp 0 factors and inverts the
// diagonal block, then all warps form the panel below it.
__device__ __noinline__ void factor_block(const Layout& L, float* own, float* li_all,
                                          float* scr, int b, const double* diag0,
                                          float rel_tol, int* bad, unsigned long long* pf) {
  const int k0 = b * CB, nb = min(CB, L.n - k0);
  float* blk = own + (size_t)L.own_row0(b) * RS;
  float* li = li_all + (size_t)((b - L.rank) / L.cl) * CB * RS;
  if ((threadIdx.x >> 5) == 0) {
    const bool fail = factor_diag(blk, nb, diag0 + k0, rel_tol, scr);
    if (fail && (threadIdx.x & 31) == 0) *bad = 1;
    if (pf && threadIdx.x == 0) pf[0] = gtime();
    invert_diag(scr, li);
    if (pf && threadIdx.x == 0) pf[1] = gtime();
  }
  __syncthreads();
  panel_rows(blk, L.n - k0, li);
  __syncthreads();
  if (pf && threadIdx.x == 0) pf[2] = gtime();
}

// Warp 0 of the owner of an even block column b: lower-left quadrant
// -C^{-1} (B A^{-1}) of the 64 x 64 inverse (C^{-1} = I and a zero quadrant
// when b has no partner).  A^{-1} and B are local, C^{-1} is copied from the
// partner's shared memory.
__device__ __noinline__ void combine_64(const Layout& L, const float* own, float* li_all,
                                        float* scr, int b, float* out) {
  const int lane = threadIdx.x & 31, n = L.n, nblk = L.nblk, cl = L.cl, rank = L.rank;
  const int k0 = b * CB;
  const float* li = li_all + (size_t)((b - rank) / cl) * CB * RS;
  float x[CB];
  if (b + 1 < nblk) {
    const int pr = (b + 1) % cl;
    const Layout Lp{n, nblk, cl, pr};
    const size_t li_row = (size_t)Lp.own_rows() + max(0, n - CB) + (size_t)((b + 1 - pr) / cl) * CB;
    const unsigned src = map_rank(own, pr) + (unsigned)(li_row * RS * sizeof(float));
    float* ci = scr;  // partner inverse C^{-1}
#pragma unroll
    for (int q4 = 0; q4 < CB; q4 += 4)
      *reinterpret_cast<float4*>(ci + lane * RS + q4) =
          ld_cluster4(src + (unsigned)((lane * RS + q4) * sizeof(float)));
    // t = B A^{-1}, row `lane`: B[lane][q] = L[k0 + 32 + lane][k0 + q]
    const bool okr = k0 + CB + lane < n;
    const float* brow = own + ((size_t)L.own_row0(b) + CB + (okr ? lane : 0)) * RS;
    float t[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) t[c] = 0.f;
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const float bq = okr ? brow[q] : 0.f;
#pragma unroll
      for (int c4 = 0; c4 < CB; c4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(li + q * RS + c4);
        t[c4] = fmaf(bq, v.x, t[c4]);
        t[c4 + 1] = fmaf(bq, v.y, t[c4 + 1]);
        t[c4 + 2] = fmaf(bq, v.z, t[c4 + 2]);
        t[c4 + 3] = fmaf(bq, v.w, t[c4 + 3]);
      }
    }
    float* tb = scr + CB * RS;
#pragma unroll
    for (int c4 = 0; c4 < CB; c4 += 4)
      *reinterpret_cast<float4*>(tb + lane * RS + c4) = make_float4(t[c4], t[c4 + 1], t[c4 + 2], t[c4 + 3]);
    __syncwarp();
    // x = -C^{-1} t, row `lane`
#pragma unroll
    for (int c = 0; c < CB; ++c) x[c] = 0.f;
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const float cq = ci[lane * RS + q];
#pragma unroll
      for (int c4 = 0; c4 < CB; c4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(tb + q * RS + c4);
        x[c4] = fmaf(-cq, v.x, x[c4]);
        x[c4 + 1] = fmaf(-cq, v.y, x[c4 + 1]);
        x[c4 + 2] = fmaf(-cq, v.z, x[c4 + 2]);
        x[c4 + 3] = fmaf(-cq, v.w, x[c4 + 3]);
      }
    }
  } else {
    // no partner: C^{-1} = I, lower-left quadrant zero
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      out[(CB + lane) * CHOL_NB + CB + c] = (c == lane) ? 1.f : 0.f;
      x[c] = 0.f;
    }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c) out[(CB + lane) * CHOL_NB + c] = x[c];
}

// One cluster of cl = min(8, ceil(n/32)) CTAs factors A (n <= 512) in place.
__global__ void __launch_bounds__(CTH, 1)
    chol_cluster_kernel(float* __restrict__ A, int64_t lda, int n, float* __restrict__ dinv,
                        const double* __restrict__ diag0, float rel_tol, int* st,
                        unsigned long long* prof) {
  extern __shared__ __align__(16) float cc_smem[];
  const int nblk = (n + CB - 1) / CB;
  const Layout L{n, nblk, (int)cluster_size(), (int)cluster_rank()};
  const int rank = L.rank, cl = L.cl;
  float* own = cc_smem;
  float* pbuf = own + (size_t)L.own_rows() * RS;
  float* li_all = pbuf + (size_t)max(0, n - CB) * RS;
  float* scr = li_all + (size_t)L.n_owned() * CB * RS;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  // owned block columns from global memory (rows k0 .. n-1; columns >= n read as 0)
  for (int b = rank; b < nblk; b += cl) {
    const int k0 = b * CB;
    float* blk = own + (size_t)L.own_row0(b) * RS;
    const int tot = (n - k0) * CB;
    for (int idx = tid; idx < tot; idx += CTH) {
      const int r = idx >> 5, c = idx & 31;
      blk[(size_t)r * RS + c] = (k0 + c < n) ? A[(int64_t)(k0 + r) * lda + k0 + c] : 0.f;
    }
  }
  __syncthreads();
  // prof (optional, NULL in the library): globaltimer stamps, 8 per CTA and
  // block column: wait done, panel copied, look-ahead update, diagonal factor,
  // inverse, panel, end of the step
  unsigned long long* pf = prof ? prof + (size_t)rank * nblk * 8 : nullptr;
  if (rank == 0) factor_block(L, own, li_all, scr, 0, diag0, rel_tol, &bad, pf ? pf + 3 : nullptr);
  __syncthreads();
  cluster_arrive();
  for (int k = 0; k < nblk; ++k) {
    cluster_wait();  // block column k is factored and visible cluster-wide
    if (pf && tid == 0) pf[8 * k] = gtime();
    const int ok = k % cl;
    int jn = rank;  // first owned block column after k
    while (jn <= k) jn += cl;
    const float* P;
    int prow0;
    if (ok == rank) {
      P = own + (size_t)L.own_row0(k) * RS;
      prow0 = k * CB;
    } else {
      prow0 = (k + 1) * CB;
      P = pbuf;
      if (jn < nblk) {
        // copy panel rows jn*32 .. n-1 of block column k out of its owner
        const Layout Lo{n, nblk, cl, ok};
        const unsigned src = map_rank(own, ok) +
                             (unsigned)(((size_t)Lo.own_row0(k) + (size_t)(jn - k) * CB) * RS *
                                        sizeof(float));
        float* dst = pbuf + (size_t)(jn - k - 1) * CB * RS;
        const int tot = (n - jn * CB) * (CB / 4);
        for (int base = tid; base < tot; base += 4 * CTH) {
          float4 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int idx = base + u * CTH;
            if (idx < tot)
              v[u] = ld_cluster4(src + (unsigned)(((idx >> 3) * RS + (idx & 7) * 4) * sizeof(float)));
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int idx = base + u * CTH;
            if (idx < tot) *reinterpret_cast<float4*>(dst + (idx >> 3) * RS + (idx & 7) * 4) = v[u];
          }
        }
      }
    }
    __syncthreads();
    if (pf && tid == 0) pf[8 * k + 1] = gtime();
    if (k + 1 < nblk && (k + 1) % cl == rank) {  // look-ahead: next block column first
      update_block(own + (size_t)L.own_row0(k + 1) * RS, (k + 1) * CB, n, P, prow0);
      __syncthreads();
      if (pf && tid == 0) pf[8 * k + 2] = gtime();
      factor_block(L, own, li_all, scr, k + 1, diag0, rel_tol, &bad,
                   pf ? pf + 8 * (k + 1) + 3 : nullptr);
    }
    if (k + 1 < nblk) cluster_arrive();
    for (int j = jn; j < nblk; j += cl)
      if (j != k + 1) update_block(own + (size_t)L.own_row0(j) * RS, j * CB, n, P, prow0);
    __syncthreads();
    if (pf && tid == 0) pf[8 * k + 6] = gtime();
  }

  // 64 x 64 inverses: each owner writes its 32 x 32 inverses into their
  // quadrants; the owner of an even block column adds the lower-left one.
  const int warp = tid >> 5;
  for (int b = rank; b < nblk; b += cl) {
    const float* li = li_all + (size_t)((b - rank) / cl) * CB * RS;
    float* out = dinv + (size_t)(b >> 1) * CHOL_NB * CHOL_NB;
    const int qo = (b & 1) * CB;
    // own inverse into its quadrant; zero the upper-right quadrant
    for (int idx = tid; idx < CB * CB; idx += CTH) {
      const int r = idx >> 5, c = idx & 31;
      out[(qo + r) * CHOL_NB + qo + c] = li[r * RS + c];
      if (qo == 0) out[r * CHOL_NB + CB + c] = 0.f;
    }
    if ((b & 1) || warp != 0) continue;
    combine_64(L, own, li_all, scr, b, out);
  }
  // factor back to global memory: lower triangle of the owned block columns
  for (int b = rank; b < nblk; b += cl) {
    const int k0 = b * CB;
    const float* blk = own + (size_t)L.own_row0(b) * RS;
    const int tot = (n - k0) * CB;
    for (int idx = tid; idx < tot; idx += CTH) {
      const int r = idx >> 5, c = idx & 31;
      if (k0 + c < n && (r >= CB || c <= r)) A[(int64_t)(k0 + r) * lda + k0 + c] = blk[(size_t)r * RS + c];
    }
  }
  if (tid == 0 && bad) set_status(st, VL_ERR_RANK);
  // no CTA may leave while a partner may still read its shared memory
  cluster_arrive();
  cluster_wait();
}

}  // namespace

// Launch the cluster factorisation; false if n is out of range or the cluster
// cannot be launched (the caller then uses the single-CTA kernel).
bool launch_chol_cluster(float* A, int64_t lda, int n, float* dinv, const double* diag0,
                         float rel_tol, int* st, cudaStream_t s, unsigned long long* prof) {
  if (n < 1 || n > CL_NMAX) return false;
  const int nblk = (n + CB - 1) / CB;
  const int cl = std::min(CL_MAX, nblk);
  const size_t smem = cluster_chol_smem(n, cl, 0);  // rank 0 owns the most rows
  static int attr_smem = 0;
  if ((int)smem > attr_smem) {
    if (cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cluster_chol_smem(CL_NMAX, CL_MAX, 0)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_smem = (int)cluster_chol_smem(CL_NMAX, CL_MAX, 0);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(CTH, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  if (cudaLaunchKernelEx(&cfg, chol_cluster_kernel, A, lda, n, dinv, diag0, rel_tol, st, prof) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace vl
