// Cholesky factorisation A = L L^T of an FP32 SPD matrix (n <= 512) by one
// thread-block cluster: the normal-equation matrix of the VAR fit (Sec. 4.1)
// and the causally ordered residual covariance whose factor gives B0 (Sec. 4.2
// item 5) are both factored here on the mixed-precision path.
//
// GB300 design.  n <= 512 is far too small to fill the GPU and one CTA alone
// spends most of its time in the trailing updates, so the factorisation runs
// on a cluster of up to 8 CTAs (one per SM) that keep the whole lower
// triangle in their shared memory, dealt out by 32-row blocks round-robin:
// CTA t owns row blocks R_b with b = t (mod cl), columns 0 .. 32(b+1)-1.
// Step k (block column C_k):
//   - the owner of R_k has factored the diagonal block A[R_k][C_k] and
//     inverted it (two warps: one factors, the other builds the inverse one
//     column behind);
//   - every CTA copies that 32 x 32 inverse out of the owner's shared memory
//     (distributed shared memory) and forms the panel rows of its own row
//     blocks, L[R_b][C_k] = A[R_b][C_k] Linv^T, in place;
//   - the trailing update A[R_b][C_j] -= L[R_b][C_k] L[R_j][C_k]^T needs the
//     panel rows of every row block j <= b: they are gathered from their
//     owners at the start of step k + 1.
// Look-ahead: the owner of R_{k+1} applies panel k to its diagonal block
// right after forming its own panel rows and factors it, so the chain from
// one diagonal block to the next is: copy inverse, a few 32 x 32 products,
// factor and invert 32 x 32.  Updates that no one waits for run after the
// CTA has signalled the step (split cluster barrier arrive / wait).
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
constexpr int CTH = 384;      // threads per CTA (measured against 512 and 256)
constexpr int CL_NMAX = 512;  // largest n handled

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
//   own   owned row blocks: R_b as 32 rows x ldb(b) = 32(b+1) + 4 floats
//         (columns 0 .. 32(b+1)-1; the 4-float pad makes a lane-per-row
//         float4 read conflict-free)
//   gbuf  gathered panel rows of the previous block column, rows 32k .. n-1
//         of step k (stride RS)
//   li    32 x 32 inverses of the owned diagonal blocks (stride RS)
//   lcur  copy of the current diagonal inverse (stride RS)
//   scr   64 rows of scratch for the diagonal factor and the 64-block combine
struct Layout {
  int n, nblk, cl, rank;
  __host__ __device__ static int ldb(int b) { return CB * (b + 1) + 4; }
  __host__ __device__ int owner(int b) const { return b % cl; }
  // offset (floats) of owned row block b inside `own`
  __host__ __device__ int own_off(int b) const {
    int o = 0;
    for (int c = rank; c < b; c += cl) o += CB * ldb(c);
    return o;
  }
  __host__ __device__ int own_floats() const {
    int o = 0;
    for (int c = rank; c < nblk; c += cl) o += CB * ldb(c);
    return o;
  }
  __host__ __device__ int n_owned() const { return nblk > rank ? (nblk - 1 - rank) / cl + 1 : 0; }
  __host__ __device__ int gbuf_off() const { return own_floats(); }
  __host__ __device__ int li_off() const { return gbuf_off() + (n > CB ? n - CB : 0) * RS; }
  __host__ __device__ int lcur_off() const { return li_off() + n_owned() * CB * RS; }
  __host__ __device__ int scr_off() const { return lcur_off() + CB * RS; }
  __host__ __device__ int total() const { return scr_off() + 2 * CB * RS; }
};

inline size_t cluster_chol_smem(int n, int cl, int rank) {
  Layout L{n, (n + CB - 1) / CB, cl, rank};
  return (size_t)L.total() * sizeof(float);
}

// Warps 0 and 1: warp 0 factors the block (rows of blk, stride ldb, nb valid)
// in place and writes the rows of L to scr (stride RS); warp 1 builds L^{-1}
// into li (stride RS) one column behind, from the multipliers warp 0 hands
// over through a two-row column buffer (col, 2 x 33 floats: 32 multipliers
// and 1 / L[j][j]) and the 64-thread named barrier 3.
__device__ __noinline__ bool factor_invert2(float* blk, int ldb, int nb, const double* diag0k,
                                            float rel_tol, float* scr, float* li, float* col) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  bool lbad = false;
  if (warp == 0) {
    float a[CB];
#pragma unroll
    for (int c4 = 0; c4 < CB; c4 += 4) {
      const float4 v = lane < nb ? *reinterpret_cast<const float4*>(blk + lane * ldb + c4)
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
    float piv = a[0];
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      float d = __shfl_sync(full, piv, j);
      const float tj = __shfl_sync(full, thr, j);
      if (!(d > tj)) {
        lbad |= (j < nb);
        d = 1.f;
      }
      const float rs = rsqrtf(d);
      const float l = lane > j ? a[j] * rs : (lane == j ? d * rs : 0.f);
      float* cj = col + (j & 1) * (CB + 4);
      cj[lane] = l;
      if (lane == 0) cj[CB] = rs;
      a[j] = l;
      if (j + 1 < CB) {
        piv = fmaf(-l, l, a[j + 1]);
        const float l1 = __shfl_sync(full, l, j + 1);
        a[j + 1] = fmaf(-l, l1, a[j + 1]);
      }
      __syncwarp();
      asm volatile("bar.sync 3, 64;" ::: "memory");
#pragma unroll
      for (int c4 = (j + 2) & ~3; c4 < CB; c4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(cj + c4);
        if (c4 >= j + 2) a[c4] = fmaf(-l, v.x, a[c4]);
        if (c4 + 1 >= j + 2) a[c4 + 1] = fmaf(-l, v.y, a[c4 + 1]);
        if (c4 + 2 >= j + 2) a[c4 + 2] = fmaf(-l, v.z, a[c4 + 2]);
        if (c4 + 3 >= j + 2) a[c4 + 3] = fmaf(-l, v.w, a[c4 + 3]);
      }
    }
#pragma unroll
    for (int c4 = 0; c4 < CB; c4 += 4) {
      const float4 v = make_float4(c4 <= lane ? a[c4] : 0.f, c4 + 1 <= lane ? a[c4 + 1] : 0.f,
                                   c4 + 2 <= lane ? a[c4 + 2] : 0.f, c4 + 3 <= lane ? a[c4 + 3] : 0.f);
      *reinterpret_cast<float4*>(scr + lane * RS + c4) = v;
      if (lane < nb) *reinterpret_cast<float4*>(blk + lane * ldb + c4) = v;
    }
  } else {
    // lane c: column c of L^{-1}; s[i] = sum_{q < i} L[i][q] x_q
    float s[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) s[i] = 0.f;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      asm volatile("bar.sync 3, 64;" ::: "memory");
      const float* cj = col + (j & 1) * (CB + 4);
      const float rs = cj[CB];
      const float x = ((lane == j ? 1.f : 0.f) - s[j]) * rs;
      li[j * RS + lane] = x;
#pragma unroll
      for (int c4 = (j + 1) & ~3; c4 < CB; c4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(cj + c4);
        if (c4 > j) s[c4] = fmaf(v.x, x, s[c4]);
        if (c4 + 1 > j) s[c4 + 1] = fmaf(v.y, x, s[c4 + 1]);
        if (c4 + 2 > j) s[c4 + 2] = fmaf(v.z, x, s[c4 + 2]);
        if (c4 + 3 > j) s[c4 + 3] = fmaf(v.w, x, s[c4 + 3]);
      }
    }
  }
  __syncwarp();
  return __any_sync(full, lbad);
}

// One warp: rows [r0, r1) of a 32-row tile, out[r][c] -= sum_q P[r][q] Q[c][q]
// for lane c; Q rows c >= qrows count as zero.  P rows are read as float4
// broadcasts, Q row c by lane c (stride ldq, conflict-free for ldq = 4 mod 32).
__device__ __forceinline__ void tile_rows(float* out, int ldo, const float* P, int ldp,
                                          const float* Q, int ldq, int qrows, int r0, int r1) {
  const int lane = threadIdx.x & 31;
  float q[CB];
  {
    const bool ok = lane < qrows;
    const float* row = Q + (size_t)(ok ? lane : 0) * ldq;
#pragma unroll
    for (int q4 = 0; q4 < CB; q4 += 4) {
      const float4 v = ok ? *reinterpret_cast<const float4*>(row + q4) : make_float4(0.f, 0.f, 0.f, 0.f);
      q[q4] = v.x;
      q[q4 + 1] = v.y;
      q[q4 + 2] = v.z;
      q[q4 + 3] = v.w;
    }
  }
  for (int r = r0; r < r1; r += 4) {
    float old[4], acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) old[u] = out[(size_t)min(r + u, r1 - 1) * ldo + lane];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float* prow = P + (size_t)min(r + u, r1 - 1) * ldp;
#pragma unroll
      for (int q4 = 0; q4 < CB; q4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(prow + q4);
        acc[u] = fmaf(v.x, q[q4], acc[u]);
        acc[u] = fmaf(v.y, q[q4 + 1], acc[u]);
        acc[u] = fmaf(v.z, q[q4 + 2], acc[u]);
        acc[u] = fmaf(v.w, q[q4 + 3], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r + u < r1) out[(size_t)(r + u) * ldo + lane] = old[u] - acc[u];
  }
}

// One warp: panel rows [r0, r1), X[r][c] = sum_{q <= c} X[r][q] Linv[c][q] in
// place (lane c; Linv lower triangular, stride RS).
__device__ __forceinline__ void panel_tile_rows(float* X, int ldx, const float* linv, int r0,
                                                int r1) {
  const int lane = threadIdx.x & 31;
  float lr[CB];
#pragma unroll
  for (int q4 = 0; q4 < CB; q4 += 4) {
    const float4 v = *reinterpret_cast<const float4*>(linv + lane * RS + q4);
    lr[q4] = v.x;
    lr[q4 + 1] = v.y;
    lr[q4 + 2] = v.z;
    lr[q4 + 3] = v.w;
  }
  for (int r = r0; r < r1; r += 4) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float* row = X + (size_t)min(r + u, r1 - 1) * ldx;
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
    for (int u = 0; u < 4; ++u)
      if (r + u < r1) X[(size_t)(r + u) * ldx + lane] = acc[u];
    __syncwarp();
  }
}

// Copy rows [g0, g1) of block column kc (panel rows, 32 floats each) from
// their owners' shared memory into gbuf (row g at (g - gbase) * RS).
__device__ __forceinline__ void gather_rows(const Layout& L, const float* smem_base, float* gbuf,
                                            int gbase, int kc, int g0, int g1) {
  const int tot = (g1 - g0) * (CB / 4);
  for (int base = threadIdx.x; base < tot; base += 4 * CTH) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * CTH;
      if (idx < tot) {
        const int g = g0 + (idx >> 3), rb = g / CB, o = L.owner(rb);
        const Layout Lo{L.n, L.nblk, L.cl, o};
        const size_t off = (size_t)Lo.own_off(rb) + (size_t)(g - rb * CB) * Layout::ldb(rb) +
                           (size_t)kc * CB + (idx & 7) * 4;
        v[u] = ld_cluster4(map_rank(smem_base + off, o));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * CTH;
      if (idx < tot)
        *reinterpret_cast<float4*>(gbuf + (size_t)(g0 + (idx >> 3) - gbase) * RS + (idx & 7) * 4) = v[u];
    }
  }
}

// Warp 0 of the owner of an odd row block b: lower-left quadrant
// -C^{-1} (B A^{-1}) of the 64 x 64 inverse for row blocks b-1, b.  B (its
// panel rows of block column b-1) and C^{-1} are local; A^{-1} is copied from
// the owner of b-1.
__device__ __noinline__ void combine_64(const Layout& L, const float* smem_base, const float* Xb,
                                        int ldxb, const float* cinv, float* scr, int b,
                                        float* out) {
  const int lane = threadIdx.x & 31;
  const int o = L.owner(b - 1);
  const Layout Lo{L.n, L.nblk, L.cl, o};
  const size_t off = (size_t)Lo.li_off() + (size_t)((b - 1 - o) / L.cl) * CB * RS;
  float* ai = scr;  // A^{-1}
#pragma unroll
  for (int q4 = 0; q4 < CB; q4 += 4)
    *reinterpret_cast<float4*>(ai + lane * RS + q4) =
        ld_cluster4(map_rank(smem_base + off + lane * RS + q4, o));
  __syncwarp();
  // t = B A^{-1}, row `lane` (rows beyond n are zero in shared memory)
  const float* brow = Xb + (size_t)lane * ldxb + (b - 1) * CB;
  float t[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) t[c] = 0.f;
#pragma unroll
  for (int q = 0; q < CB; ++q) {
    const float bq = brow[q];
#pragma unroll
    for (int c4 = 0; c4 < CB; c4 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(ai + q * RS + c4);
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
  float x[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = 0.f;
#pragma unroll
  for (int q = 0; q < CB; ++q) {
    const float cq = cinv[lane * RS + q];
#pragma unroll
    for (int c4 = 0; c4 < CB; c4 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(tb + q * RS + c4);
      x[c4] = fmaf(-cq, v.x, x[c4]);
      x[c4 + 1] = fmaf(-cq, v.y, x[c4 + 1]);
      x[c4 + 2] = fmaf(-cq, v.z, x[c4 + 2]);
      x[c4 + 3] = fmaf(-cq, v.w, x[c4 + 3]);
    }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c) out[(CB + lane) * CHOL_NB + c] = x[c];
}

// One cluster of cl = min(8, ceil(n/32)) CTAs factors A (n <= 512) in place.
// prof (optional, NULL in the library): globaltimer stamps, 8 per CTA and
// step: wait done, first rows gathered, priority updates, panel rows,
// look-ahead update, diagonal factored and inverted, end of the step,
// diagonal factored (before its inverse).
__global__ void __launch_bounds__(CTH, 1)
    chol_cluster_kernel(float* __restrict__ A, int64_t lda, int n, float* __restrict__ dinv,
                        const double* __restrict__ diag0, float rel_tol, int* st,
                        unsigned long long* prof) {
  extern __shared__ __align__(16) float cc_smem[];
  const int nblk = (n + CB - 1) / CB;
  const Layout L{n, nblk, (int)cluster_size(), (int)cluster_rank()};
  const int rank = L.rank, cl = L.cl;
  float* own = cc_smem;
  float* gbuf = cc_smem + L.gbuf_off();
  float* li_all = cc_smem + L.li_off();
  float* lcur = cc_smem + L.lcur_off();
  float* scr = cc_smem + L.scr_off();
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, nwarp = CTH / 32;
  if (tid == 0) bad = 0;
  unsigned long long* pf = prof ? prof + (size_t)rank * nblk * 8 : nullptr;
  auto blk = [&](int b) { return own + L.own_off(b); };
  auto nbr = [&](int b) { return min(CB, n - b * CB); };
  auto lib = [&](int b) { return li_all + (size_t)((b - rank) / cl) * CB * RS; };
  auto first_after = [&](int k) {  // first owned row block > k
    int b = rank;
    while (b <= k) b += cl;
    return b;
  };
  int bmax = -1;
  for (int b = rank; b < nblk; b += cl) bmax = b;
  // owned row blocks: rows 32b .. 32b+31 (zero beyond n), columns 0 .. 32(b+1)-1
  for (int b = rank; b < nblk; b += cl) {
    float* X = blk(b);
    const int ld = Layout::ldb(b), w = CB * (b + 1);
    for (int idx = tid; idx < CB * w; idx += CTH) {
      const int r = idx / w, c = idx - r * w, g = b * CB + r;
      X[(size_t)r * ld + c] = (g < n && c < n) ? A[(int64_t)g * lda + c] : 0.f;
    }
  }
  __syncthreads();
  if (rank == 0 && warp < 2) {  // diagonal block 0
    if (factor_invert2(blk(0), Layout::ldb(0), nbr(0), diag0, rel_tol, scr, lib(0),
                       scr + CB * RS) &&
        tid == 0)
      bad = 1;
  }
  __syncthreads();
  cluster_arrive();
  for (int k = 0; k < nblk; ++k) {
    cluster_wait();  // diagonal block k and the panel rows of block column k-1 are ready
    if (pf && tid == 0) pf[8 * k] = gtime();
    const int ok = L.owner(k);
    const bool below = bmax > k;  // owns a row block below k
    const bool next_owner = k + 1 < nblk && L.owner(k + 1) == rank;
    const int jb = first_after(k);
    const int gbase = k * CB;
    const int gend = below ? min(n, CB * (bmax + 1)) : gbase;
    // (a) inverse of diagonal block k
    const float* linv = (ok == rank) ? lib(k) : lcur;
    if (ok != rank && below) {
      const Layout Lo{n, nblk, cl, ok};
      const size_t off = (size_t)Lo.li_off() + (size_t)((k - ok) / cl) * CB * RS;
      for (int idx = tid; idx < CB * CB / 4; idx += CTH) {
        const int r = idx >> 3, q4 = (idx & 7) * 4;
        *reinterpret_cast<float4*>(lcur + r * RS + q4) =
            ld_cluster4(map_rank(cc_smem + off + r * RS + q4, ok));
      }
    }
    // (b) panel rows of block column k-1 for row blocks k and k+1
    if (k >= 1 && below) gather_rows(L, cc_smem, gbuf, gbase, k - 1, gbase, min(gend, gbase + 2 * CB));
    __syncthreads();
    if (pf && tid == 0) pf[8 * k + 1] = gtime();
    // (c) panel k-1 on block column k of the owned row blocks below k, and on
    //     diagonal block k+1 if owned; (d) panel rows of block column k for the
    //     owned row blocks below k.  Both act row by row, so the warp that
    //     updates 8 rows in (c) forms the same 8 panel rows in (d) right after,
    //     with no CTA barrier between the two.
    {
      int ntile = 0;
      for (int b = jb; b < nblk; b += cl) ++ntile;
      const int ntask = 4 * (ntile + (k >= 1 && next_owner ? 1 : 0));
      for (int t = warp; t < ntask; t += nwarp) {
        const int tile = t >> 2, qr = t & 3;
        if (k >= 1) {
          const int b = tile < ntile ? jb + tile * cl : k + 1;
          const int j = tile < ntile ? k : k + 1;
          float* X = blk(b);
          const int ld = Layout::ldb(b);
          tile_rows(X + j * CB, ld, X + (k - 1) * CB, ld, gbuf + (size_t)(j * CB - gbase) * RS,
                    RS, min(CB, n - j * CB), qr * 8, qr * 8 + 8);
        }
        if (tile < ntile) {
          __syncwarp();
          const int b = jb + tile * cl;
          panel_tile_rows(blk(b) + k * CB, Layout::ldb(b), linv, qr * 8, qr * 8 + 8);
        }
      }
      __syncthreads();
    }
    if (pf && tid == 0) pf[8 * k + 3] = gtime();
    // (e) look-ahead: panel k on diagonal block k+1, then factor and invert it
    if (next_owner) {
      float* X = blk(k + 1);
      const int ld = Layout::ldb(k + 1);
      if (warp < 4) tile_rows(X + (k + 1) * CB, ld, X + k * CB, ld, X + k * CB, ld, nbr(k + 1),
                              warp * 8, warp * 8 + 8);
      __syncthreads();
      if (pf && tid == 0) pf[8 * k + 4] = gtime();
      if (warp < 2) {
        if (factor_invert2(X + (k + 1) * CB, ld, nbr(k + 1), diag0 + (k + 1) * CB, rel_tol, scr,
                           lib(k + 1), scr + CB * RS) &&
            tid == 0)
          bad = 1;
        if (pf && tid == 0) pf[8 * k + 7] = gtime();
      }
      __syncthreads();
      if (pf && tid == 0) pf[8 * k + 5] = gtime();
    }
    if (k + 1 < nblk) cluster_arrive();
    // (f) remaining rows of block column k-1, then panel k-1 on blocks (b, j),
    //     b > k+1 owned, k+1 <= j <= b
    if (k >= 1 && below) {
      if (gend > gbase + 2 * CB) {
        gather_rows(L, cc_smem, gbuf, gbase, k - 1, gbase + 2 * CB, gend);
        __syncthreads();
      }
      const int b0 = first_after(k + 1);
      int ntile = 0;
      for (int b = b0; b < nblk; b += cl) ntile += b - k;
      for (int t = warp; t < 4 * ntile; t += nwarp) {
        int tile = t >> 2, b = b0;
        while (tile >= b - k) {
          tile -= b - k;
          b += cl;
        }
        const int j = k + 1 + tile, qr = t & 3;
        float* X = blk(b);
        const int ld = Layout::ldb(b);
        tile_rows(X + j * CB, ld, X + (k - 1) * CB, ld, gbuf + (size_t)(j * CB - gbase) * RS, RS,
                  min(CB, n - j * CB), qr * 8, qr * 8 + 8);
      }
    }
    __syncthreads();
    if (pf && tid == 0) pf[8 * k + 6] = gtime();
  }

  // 64 x 64 inverses of the diagonal blocks of L
  for (int b = rank; b < nblk; b += cl) {
    float* out = dinv + (size_t)(b >> 1) * CHOL_NB * CHOL_NB;
    const int qo = (b & 1) * CB;
    const float* li = lib(b);
    for (int idx = tid; idx < CB * CB; idx += CTH) {
      const int r = idx >> 5, c = idx & 31;
      out[(qo + r) * CHOL_NB + qo + c] = li[r * RS + c];
      if (qo == 0) {
        out[r * CHOL_NB + CB + c] = 0.f;
        if (b + 1 == nblk) {  // no partner: C^{-1} = I, lower-left zero
          out[(CB + r) * CHOL_NB + CB + c] = (r == c) ? 1.f : 0.f;
          out[(CB + r) * CHOL_NB + c] = 0.f;
        }
      }
    }
    if ((b & 1) && warp == 0) combine_64(L, cc_smem, blk(b), Layout::ldb(b), li, scr, b, out);
  }
  // factor back to global memory: lower triangle of the owned row blocks
  for (int b = rank; b < nblk; b += cl) {
    const float* X = blk(b);
    const int ld = Layout::ldb(b), w = min(n, CB * (b + 1));
    for (int idx = tid; idx < CB * w; idx += CTH) {
      const int r = idx / w, c = idx - r * w, g = b * CB + r;
      if (g < n && c <= g) A[(int64_t)g * lda + c] = X[(size_t)r * ld + c];
    }
  }
  if (tid == 0 && bad) set_status(st, VL_ERR_RANK);
  // no CTA may leave while a peer may still read its shared memory
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
  size_t smem = 0;
  for (int r = 0; r < cl; ++r) smem = std::max(smem, cluster_chol_smem(n, cl, r));
  static size_t attr_smem = 0;
  if (smem > attr_smem) {
    size_t need = 0;
    for (int r = 0; r < CL_MAX; ++r) need = std::max(need, cluster_chol_smem(CL_NMAX, CL_MAX, r));
    if (cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)need) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_smem = need;
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
