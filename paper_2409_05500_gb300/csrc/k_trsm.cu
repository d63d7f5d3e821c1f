// Blocked triangular solves with a Cholesky factor L (64 x 64 blocks, the
// inverses of the diagonal blocks given): forward Y = L^{-1} R and, on
// request, backward X = L^{-T} Y, for the VAR normal equations (Sec. 4.1) and
// for L^{-1} itself, which gives B0 (Sec. 4.2 item 5).
//
// GB300 design.  Each CTA owns 4 right-hand-side columns (one per thread of a
// row; 100 CTAs for 400 columns) and keeps its whole solution panel (n x 4) in
// shared memory, so a block row never waits for its own earlier results to
// come back from memory.  The 64 x 64 pieces of L (and
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
  T* Acc = ring + NS * TB * LS;                     // [TB][TSC]
  T* Ysol = Acc + TB * TSC;                         // [nblk * TB][TSC]
  const int tid = threadIdx.x, r = tid >> 2, cc = tid & 3;
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
  T acc = T(0);
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
    if (qc.c == 0) acc = Ysol[(k0 + r) * TSC + cc];  // start of a block row
    if (qc.c < qc.pieces(nblk)) {
      const int j0 = (qc.pass == 0 ? qc.c : b + 1 + qc.c) * TB;
      const T* Y = Ysol + j0 * TSC + cc;
      // four independent partial sums: the dot product is not one long chain
      T a[4] = {T(0), T(0), T(0), T(0)};
      if (qc.pass == 0) {
#pragma unroll 16
        for (int jj = 0; jj < TB; ++jj) a[jj & 3] += S[r * LS + jj] * Y[jj * TSC];
      } else {
#pragma unroll 16
        for (int jj = 0; jj < TB; ++jj) a[jj & 3] += S[jj * LS + r] * Y[jj * TSC];
      }
      acc -= (a[0] + a[1]) + (a[2] + a[3]);
    } else {  // apply the inverse of the diagonal block (transposed when backward)
      Acc[r * TSC + cc] = acc;
      __syncthreads();
      T o[4] = {T(0), T(0), T(0), T(0)};
      if (qc.pass == 0) {
#pragma unroll 16
        for (int q = 0; q < TB; ++q) o[q & 3] += S[r * LS + q] * Acc[q * TSC + cc];
      } else {
#pragma unroll 16
        for (int q = 0; q < TB; ++q) o[q & 3] += S[q * LS + r] * Acc[q * TSC + cc];
      }
      Ysol[(k0 + r) * TSC + cc] = r < nb ? (o[0] + o[1]) + (o[2] + o[3]) : T(0);
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
  return sizeof(T) * ((size_t)Ring<T>::NS * TB * Ring<T>::LS + TB * TSC + (size_t)nblk * TB * TSC);
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
