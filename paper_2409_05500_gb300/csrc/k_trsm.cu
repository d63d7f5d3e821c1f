// Blocked triangular solves with a Cholesky factor L (64 x 64 blocks, the
// inverses of the diagonal blocks given): forward Y = L^{-1} R and, on
// request, backward X = L^{-T} Y, for the VAR normal equations (Sec. 4.1) and
// for L^{-1} itself, which gives B0 (Sec. 4.2 item 5).
//
// GB300 design.  Each CTA owns 4 right-hand-side columns (100 CTAs for 400
// columns) and keeps its whole solution panel (n x 4) in shared memory, so a
// block row never waits for its own earlier results to come back from memory.
// A thread computes one row of the block row for all four columns over a
// 16-wide slice of each piece (vector loads of the piece's row and of the
// solution rows): a piece costs about 20 shared-memory loads per thread, not
// 128, which is what limited the scalar one-column-per-thread form; the four
// slices are added once per block row.  The 64 x 64 pieces of L (and
// the diagonal-block inverses) flow through an NS-stage cp.async ring in one
// stream over both passes, so the next pieces are in flight while the current
// one is applied: the solve is paced by the L2 bandwidth of the pieces rather
// than by one round trip per piece.
#include <algorithm>

#include "vl_internal.cuh"

namespace vl {

namespace {

constexpr int TB = CHOL_NB;   // block size (64)
constexpr int TSC = 4;        // right-hand sides per CTA
constexpr int TTH = 256;      // threads: 64 rows x 4 columns
constexpr int TNMAX = 1024;   // largest n with the solution panel in shared memory

template <class T>
struct Ring;
template <>
struct Ring<float> {
  static constexpr int NS = 4, LS = TB + 4;  // 16-byte rows, conflict-free access
};
template <>
struct Ring<double> {
  static constexpr int NS = 3, LS = TB + 2;
};

__device__ __forceinline__ void cp16(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes));
}
template <int N>
__device__ __forceinline__ void cp_el(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(N),
               "r"(bytes));
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void wait_groups() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Four consecutive elements from shared memory (16-byte aligned for float,
// two 16-byte loads for double).
template <class T>
struct V4 {
  T v[4];
};
__device__ __forceinline__ V4<float> ld_v4(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return V4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld_v4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return V4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Position in the piece stream: pass 0 (forward) then pass 1 (backward);
// block rows in solve order; per block row its off-diagonal pieces, then the
// inverse of its diagonal block (c == pieces(b)).
struct Cursor {
  int pass, bi, c;
  __device__ int block(int nblk) const { return pass == 0 ? bi : nblk - 1 - bi; }
  __device__ int pieces(int nblk) const {
    const int b = block(nblk);
    return pass == 0 ? b : nblk - 1 - b;
  }
  __device__ void advance(int nblk) {
    if (++c > pieces(nblk)) {
      c = 0;
      if (++bi == nblk) {
        bi = 0;
        ++pass;
      }
    }
  }
};

template <class T>
__global__ void __launch_bounds__(TTH) trsm_ring_kernel(const T* __restrict__ L, int64_t lda,
                                                        const T* __restrict__ dinv, int n,
                                                        T* __restrict__ R, int64_t ldr, int nrhs,
                                                        int npass, int vec) {
  constexpr int NS = Ring<T>::NS, LS = Ring<T>::LS;
  constexpr int EPC = 16 / sizeof(T);  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char trsm_ring_smem[];
  const int nblk = (n + TB - 1) / TB;
  T* ring = reinterpret_cast<T*>(trsm_ring_smem);  // [NS][TB][LS]
  T* Acc = ring + NS * TB * LS;                     // [TB][TSC], then [4][TB][TSC] slices
  T* Ysol = Acc + 5 * TB * TSC;                     // [nblk * TB][TSC]
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * TSC;

  // this CTA's columns of the right-hand side (zero beyond n and nrhs)
  for (int idx = tid; idx < nblk * TB * TSC; idx += TTH) {
    const int row = idx / TSC, col = c0 + idx % TSC;
    Ysol[idx] = (row < n && col < nrhs) ? R[(int64_t)row * ldr + col] : T(0);
  }

  // copy one piece into ring slot `slot`
  auto issue = [&](const Cursor& q, int slot) {
    T* S = ring + slot * TB * LS;
    const int b = q.block(nblk), k0 = b * TB;
    const T* src;
    int64_t ld;
    int rows, cols;
    if (q.c == q.pieces(nblk)) {  // inverse of the diagonal block, 64 x 64 dense
      src = dinv + (int64_t)b * TB * TB;
      ld = TB;
      rows = cols = TB;
    } else if (q.pass == 0) {     // L[k0 + a][j0 + e]
      const int j0 = q.c * TB;
      src = L + (int64_t)k0 * lda + j0;
      ld = lda;
      rows = min(TB, n - k0);
      cols = min(TB, n - j0);
    } else {                      // L[j0 + a][k0 + e], used transposed
      const int j0 = (b + 1 + q.c) * TB;
      src = L + (int64_t)j0 * lda + k0;
      ld = lda;
      rows = min(TB, n - j0);
      cols = min(TB, n - k0);
    }
    if (vec) {
      for (int idx = tid; idx < TB * (TB / EPC); idx += TTH) {
        const int a = idx / (TB / EPC), e = (idx % (TB / EPC)) * EPC;
        const int ok = a < rows ? max(0, min(EPC, cols - e)) : 0;
        cp16(S + a * LS + e, ok ? (const void*)(src + (int64_t)a * ld + e) : (const void*)src,
             ok * (int)sizeof(T));
      }
    } else {
      for (int idx = tid; idx < TB * TB; idx += TTH) {
        const int a = idx / TB, e = idx % TB;
        const int ok = a < rows && e < cols;
        cp_el<sizeof(T)>(S + a * LS + e, ok ? (const void*)(src + (int64_t)a * ld + e)
                                            : (const void*)src,
                         ok ? (int)sizeof(T) : 0);
      }
    }
  };

  const int total = npass * (nblk * (nblk + 1) / 2);  // pieces incl. diagonal inverses
  Cursor qi{0, 0, 0}, qc{0, 0, 0};
  for (int s = 0; s < NS - 1; ++s) {
    if (s < total) {
      issue(qi, s);
      qi.advance(nblk);
    }
    commit();
  }
  // Thread (rr = tid % 64, ks = tid / 64): row rr of the block row, all TSC
  // right-hand sides, over the k-slice [16 ks, 16 ks + 16) of every piece;
  // the four slices are added once per block row, at its diagonal piece.
  const int rr = tid & (TB - 1), ks = tid >> 6;
  constexpr int KS = TB / 4;  // k-slice length
  T part[TSC];
#pragma unroll
  for (int c = 0; c < TSC; ++c) part[c] = T(0);
  for (int i = 0; i < total; ++i) {
    wait_groups<NS - 2>();
    __syncthreads();
    if (i + NS - 1 < total) {
      issue(qi, (i + NS - 1) % NS);
      qi.advance(nblk);
    }
    commit();
    const T* S = ring + (i % NS) * TB * LS;
    const int b = qc.block(nblk), k0 = b * TB, nb = min(TB, n - k0);
    if (qc.c < qc.pieces(nblk)) {
      const int j0 = (qc.pass == 0 ? qc.c : b + 1 + qc.c) * TB;
      const T* Y = Ysol + (j0 + KS * ks) * TSC;
      if (qc.pass == 0) {  // S[rr][jj]: row rr, four consecutive jj per vector load
#pragma unroll
        for (int j4 = 0; j4 < KS; j4 += 4) {
          const V4<T> sv = ld_v4(S + rr * LS + KS * ks + j4);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const V4<T> y = ld_v4(Y + (j4 + e) * TSC);
#pragma unroll
            for (int c = 0; c < TSC; ++c) part[c] = fma_t(sv.v[e], y.v[c], part[c]);
          }
        }
      } else {  // S[jj][rr] (the piece used transposed): consecutive rr across lanes
#pragma unroll
        for (int jj = 0; jj < KS; ++jj) {
          const T sv = S[(KS * ks + jj) * LS + rr];
          const V4<T> y = ld_v4(Y + jj * TSC);
#pragma unroll
          for (int c = 0; c < TSC; ++c) part[c] = fma_t(sv, y.v[c], part[c]);
        }
      }
    } else {
      // end of the block row: Acc = R - (the four slices' sums), then the
      // inverse of the diagonal block (transposed when backward), again in
      // four k-slices added through shared memory
      T* red = Acc + TB * TSC;  // [4][TB][TSC]
#pragma unroll
      for (int c = 0; c < TSC; ++c) red[(ks * TB + rr) * TSC + c] = part[c];
      __syncthreads();
      {
        const int r2 = tid >> 2, c2 = tid & 3;  // one (row, column) per thread
        T sum = Ysol[(k0 + r2) * TSC + c2];
#pragma unroll
        for (int z = 0; z < 4; ++z) sum -= red[(z * TB + r2) * TSC + c2];
        Acc[r2 * TSC + c2] = sum;
      }
      __syncthreads();
      T o[TSC];
#pragma unroll
      for (int c = 0; c < TSC; ++c) o[c] = T(0);
      const T* A = Acc + KS * ks * TSC;
      if (qc.pass == 0) {
#pragma unroll
        for (int q4 = 0; q4 < KS; q4 += 4) {
          const V4<T> sv = ld_v4(S + rr * LS + KS * ks + q4);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const V4<T> a = ld_v4(A + (q4 + e) * TSC);
#pragma unroll
            for (int c = 0; c < TSC; ++c) o[c] = fma_t(sv.v[e], a.v[c], o[c]);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < KS; ++q) {
          const T sv = S[(KS * ks + q) * LS + rr];
          const V4<T> a = ld_v4(A + q * TSC);
#pragma unroll
          for (int c = 0; c < TSC; ++c) o[c] = fma_t(sv, a.v[c], o[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < TSC; ++c) red[(ks * TB + rr) * TSC + c] = o[c];
      __syncthreads();
      {
        const int r2 = tid >> 2, c2 = tid & 3;
        T sum = T(0);
#pragma unroll
        for (int z = 0; z < 4; ++z) sum += red[(z * TB + r2) * TSC + c2];
        Ysol[(k0 + r2) * TSC + c2] = r2 < nb ? sum : T(0);
      }
#pragma unroll
      for (int c = 0; c < TSC; ++c) part[c] = T(0);
    }
    qc.advance(nblk);
  }
  wait_groups<0>();
  __syncthreads();
  for (int idx = tid; idx < n * TSC; idx += TTH) {
    const int row = idx / TSC, col = c0 + idx % TSC;
    if (col < nrhs) R[(int64_t)row * ldr + col] = Ysol[idx];
  }
}

template <class T>
size_t ring_smem(int n) {
  const int nblk = (n + TB - 1) / TB;
  return sizeof(T) *
         ((size_t)Ring<T>::NS * TB * Ring<T>::LS + 5 * TB * TSC + (size_t)nblk * TB * TSC);
}

}  // namespace

template <class T>
bool launch_trsm_ring(const T* L, int64_t lda, const T* dinv, int n, T* R, int64_t ldr, int nrhs,
                      bool backward, cudaStream_t s) {
  if (n < 1 || n > TNMAX || nrhs < 1) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(trsm_ring_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ring_smem<T>(TNMAX)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  const int vec = ((uintptr_t)L % 16 == 0) && ((uintptr_t)dinv % 16 == 0) &&
                  ((lda * (int64_t)sizeof(T)) % 16 == 0);
  note_launch();
  trsm_ring_kernel<T><<<(nrhs + TSC - 1) / TSC, TTH, ring_smem<T>(n), s>>>(
      L, lda, dinv, n, R, ldr, nrhs, backward ? 2 : 1, vec);
  return true;
}
template bool launch_trsm_ring<float>(const float*, int64_t, const float*, int, float*, int64_t,
                                      int, bool, cudaStream_t);
template bool launch_trsm_ring<double>(const double*, int64_t, const double*, int, double*,
                                       int64_t, int, bool, cudaStream_t);

}  // namespace vl
