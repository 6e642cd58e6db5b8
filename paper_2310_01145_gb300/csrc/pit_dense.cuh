// Block-level dense linear algebra for the large-state solver (D = d (q+1) up to 256).
//
// Every routine here is executed by all NT threads of one thread block and works on row-major
// matrices in global memory (a per-block scratch area that stays resident in L2), staging tiles
// through the block's shared memory.  Each routine ends with __syncthreads(), so its outputs are
// visible to the whole block on return; inputs must be visible on entry.
//
//  * cta_gemm      C = alpha op(A) op(B) + beta C       (64 x 64 tiles, 4 x 2 outputs a thread)
//  * cta_lq        tria of Section 3.1.2: the lower-triangular factor L of M = L Q, computed by
//                  Householder reflections from the right in blocks of NB rows (compact WY form
//                  I - V T V^T, trailing rows updated with two register-tiled products).  Only the
//                  first `rf` rows are triangularised; rows below receive the same reflections.
//                  Columns [0, ctri) may be declared lower-triangular for rows < ctri, in which
//                  case reflection k acts on column k and the dense columns [ctri, ncols) only.
//  * cta_trsm_*    blocked triangular solves with a lower-triangular factor.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pit_tc.cuh"

namespace pit {
namespace dn {

constexpr int NT = 512;              // threads per block of every large-state kernel
constexpr int NWARPS = NT / 32;
constexpr int NB = 32;               // reflections per LQ panel
constexpr int MAXCH = 9;             // 32-wide chunks of a panel row held per lane
constexpr int MAXWS = MAXCH * 32;    // widest panel (compact columns) the LQ accepts: 288
constexpr int GBM = 64, GBN = 64, GBK = 16, GLD = 68;  // GEMM tile and its shared row stride

// Trailing-row tile of the LQ update (shared memory: RT x ldv values).
template <typename T>
struct LqTile {
  static constexpr int RT = sizeof(T) == 4 ? 64 : 32;
};

// Shared memory (elements of T) the LQ needs for compact panel width up to `ws`.
template <typename T>
__host__ __device__ constexpr int lq_ldv(int ws) {
  return (ws + 3) & ~3;
}
template <typename T>
__host__ __device__ constexpr size_t lq_smem_elems(int wsmax) {
  return static_cast<size_t>(NB) * lq_ldv<T>(wsmax)           // V (panel reflections)
         + static_cast<size_t>(LqTile<T>::RT) * lq_ldv<T>(wsmax)  // trailing tile
         + NB * (NB + 1) * 2                                     // T and Gram
         + static_cast<size_t>(NB) * (LqTile<T>::RT + 4)         // (W T)^T
         + static_cast<size_t>(LqTile<T>::RT) * (NB + 1)         // W
         + NB;                                                   // tau
}
// Shared memory (bytes) of the LQ with its trailing rows updated on the tensor cores (FP64): the
// panel's reflections, T, Gram and tau, then the digit staging area at a 128-byte boundary.
__host__ __device__ constexpr size_t lq_tc_smem_bytes(int wsmax) {
  return (static_cast<size_t>(NB) * lq_ldv<double>(wsmax) + 2 * NB * (NB + 1) + NB) * 8 + 128 +
         tc::stage_bytes();   // + 128: the staging area starts at the next 128-byte boundary
}
template <typename T>
__host__ __device__ constexpr size_t gemm_smem_elems() {
  return 2 * GBK * GLD;
}

// ---- small helpers ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// 4 consecutive values from shared memory (16-byte aligned for float, 2 x 16 bytes for double)
__device__ __forceinline__ void ld4s(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4s(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld2s(const float* p, float (&o)[2]) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void ld2s(const double* p, double (&o)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x; o[1] = v.y;
}

// dst[r][c] = src[r][c] for r < m, c < n
template <typename T>
__device__ __forceinline__ void cta_copy(int m, int n, const T* src, int lds, T* dst, int ldd) {
  for (int i = threadIdx.x; i < m * n; i += NT) {
    const int r = i / n, c = i - r * n;
    dst[static_cast<size_t>(r) * ldd + c] = src[static_cast<size_t>(r) * lds + c];
  }
  __syncthreads();
}
// dst[c][r] = src[r][c]  (src m x n, dst n x m)
template <typename T>
__device__ __forceinline__ void cta_copy_t(int m, int n, const T* src, int lds, T* dst, int ldd) {
  for (int i = threadIdx.x; i < m * n; i += NT) {
    const int c = i / m, r = i - c * m;
    dst[static_cast<size_t>(c) * ldd + r] = src[static_cast<size_t>(r) * lds + c];
  }
  __syncthreads();
}
// A[r][c] = (r == c) ? diag : 0
template <typename T>
__device__ __forceinline__ void cta_set(int m, int n, T* A, int lda, T diag) {
  for (int i = threadIdx.x; i < m * n; i += NT) {
    const int r = i / n, c = i - r * n;
    A[static_cast<size_t>(r) * lda + c] = (r == c) ? diag : T(0);
  }
  __syncthreads();
}

// y[r] = beta y[r] + alpha sum_c op(A)[r][c] x[c], r < m, c < n   (one warp per row)
// TRANS: op(A)[r][c] = A[c][r] (A stored n x m).  y must not alias x.
template <typename T, bool TRANS>
__device__ __forceinline__ void cta_gemv(int m, int n, T alpha, const T* A, int lda, const T* x,
                                         T beta, T* y) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (!TRANS) {
    for (int r = warp; r < m; r += NWARPS) {
      T acc = T(0);
      for (int c = lane; c < n; c += 32) acc += A[static_cast<size_t>(r) * lda + c] * x[c];
      acc = warp_sum(acc);
      if (lane == 0) y[r] = (beta == T(0) ? T(0) : beta * y[r]) + alpha * acc;
    }
  } else {
    for (int r = threadIdx.x; r < m; r += NT) {
      T acc = T(0);
      for (int c = 0; c < n; ++c) acc += A[static_cast<size_t>(c) * lda + r] * x[c];
      y[r] = (beta == T(0) ? T(0) : beta * y[r]) + alpha * acc;
    }
  }
  __syncthreads();
}

// ---- GEMM ------------------------------------------------------------------------------------
// C[m x n] = alpha op(A)[m x k] op(B)[k x n] + beta C.  op(A)[i][l] = TA ? A[l][i] : A[i][l],
// op(B)[l][j] = TB ? B[j][l] : B[l][j].  beta == 0 does not read C.  C must not alias A or B.
// sm: gemm_smem_elems<T>() elements of shared memory.
template <typename T, bool TA, bool TB>
__device__ void cta_gemm(int m, int n, int k, T alpha, const T* A, int lda, const T* B, int ldb,
                         T beta, T* C, int ldc, T* sm) {
  T* As = sm;                // [GBK][GLD], As[l][i]
  T* Bs = sm + GBK * GLD;    // [GBK][GLD], Bs[l][j]
  const int tid = threadIdx.x;
  const int tr = tid >> 5;   // rows 4 tr .. 4 tr + 3 of the tile
  const int tc = tid & 31;   // cols 2 tc, 2 tc + 1
  const int tm = (m + GBM - 1) / GBM, tn = (n + GBN - 1) / GBN;
  for (int tile = 0; tile < tm * tn; ++tile) {
    const int i0 = (tile / tn) * GBM, j0 = (tile % tn) * GBN;
    T acc[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
    for (int l0 = 0; l0 < k; l0 += GBK) {
      // stage op(A)[i0 .. i0+63][l0 .. l0+15] -> As[l][i]
#pragma unroll
      for (int e = 0; e < (GBM * GBK) / NT; ++e) {
        const int idx = tid + e * NT;
        int i, l;
        if constexpr (TA) { l = idx >> 6; i = idx & 63; }   // contiguous along i
        else { i = idx >> 4; l = idx & 15; }                 // contiguous along l
        const int gi = i0 + i, gl = l0 + l;
        T v = T(0);
        if (gi < m && gl < k)
          v = TA ? A[static_cast<size_t>(gl) * lda + gi] : A[static_cast<size_t>(gi) * lda + gl];
        As[l * GLD + i] = v;
      }
      // stage op(B)[l0 .. l0+15][j0 .. j0+63] -> Bs[l][j]
#pragma unroll
      for (int e = 0; e < (GBN * GBK) / NT; ++e) {
        const int idx = tid + e * NT;
        int j, l;
        if constexpr (TB) { j = idx >> 4; l = idx & 15; }
        else { l = idx >> 6; j = idx & 63; }
        const int gj = j0 + j, gl = l0 + l;
        T v = T(0);
        if (gj < n && gl < k)
          v = TB ? B[static_cast<size_t>(gj) * ldb + gl] : B[static_cast<size_t>(gl) * ldb + gj];
        Bs[l * GLD + j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int l = 0; l < GBK; ++l) {
        T a[4], b[2];
        ld4s(As + l * GLD + 4 * tr, a);
        ld2s(Bs + l * GLD + 2 * tc, b);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          acc[x][0] += a[x] * b[0];
          acc[x][1] += a[x] * b[1];
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int gi = i0 + 4 * tr + x;
      if (gi >= m) continue;
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int gj = j0 + 2 * tc + y;
        if (gj >= n) continue;
        T* c = C + static_cast<size_t>(gi) * ldc + gj;
        *c = (beta == T(0) ? T(0) : beta * *c) + alpha * acc[x][y];
      }
    }
  }
  __syncthreads();
}

// ---- triangular solves -------------------------------------------------------------------------
// X op(L) = B in place (X: m x n, overwritten; L: n x n lower-triangular, full rank).
//   TRANS = false:  X L = B;   TRANS = true: X L^T = B.
// Blocks of NB columns: the coupling to solved blocks is one GEMM, the diagonal block is solved
// row by row (one thread per row of X, the block of L in shared memory).
// FP64 with tcx: the coupling products run as exact digit products on the tensor cores (their
// staging area at sm, which then needs tc::stage_bytes() bytes).
template <typename T, bool TRANS>
__device__ void cta_trsm_right(int m, int n, const T* L, int ldl, T* X, int ldx, T* sm,
                               const tc::TcCtx* tcx = nullptr) {
  T* Lb = sm + gemm_smem_elems<T>();  // [NB][NB + 1] diagonal block (after the coupling)

  const int nblk = (n + NB - 1) / NB;
  for (int bi = 0; bi < nblk; ++bi) {
    // X L: columns are resolved from the right;  X L^T: from the left
    const int blk = TRANS ? bi : nblk - 1 - bi;
    const int j0 = blk * NB, j1 = min(n, j0 + NB), bj = j1 - j0;
    if (!TRANS && j1 < n) {
      // X[:, J] -= X[:, j1:n] L[j1:n, J]
      bool done = false;
      if constexpr (std::is_same<T, double>::value) {
        if (tcx) {
          const tc::TcCtx c{reinterpret_cast<unsigned char*>(sm), tcx->gstatus, tcx->wait_ns};
          tc::cta_dgemm<false, false>(c, m, bj, n - j1, -1.0, X + j1, ldx,
                                      L + static_cast<size_t>(j1) * ldl + j0, ldl, 1.0, X + j0, ldx);
          done = true;
        }
      }
      if (!done)
        cta_gemm<T, false, false>(m, bj, n - j1, T(-1), X + j1, ldx, L + static_cast<size_t>(j1) * ldl + j0,
                                  ldl, T(1), X + j0, ldx, sm);
    }
    if (TRANS && j0 > 0) {
      // X[:, J] -= X[:, 0:j0] L[J, 0:j0]^T
      bool done = false;
      if constexpr (std::is_same<T, double>::value) {
        if (tcx) {
          const tc::TcCtx c{reinterpret_cast<unsigned char*>(sm), tcx->gstatus, tcx->wait_ns};
          tc::cta_dgemm<false, true>(c, m, bj, j0, -1.0, X, ldx, L + static_cast<size_t>(j0) * ldl,
                                     ldl, 1.0, X + j0, ldx);
          done = true;
        }
      }
      if (!done)
        cta_gemm<T, false, true>(m, bj, j0, T(-1), X, ldx, L + static_cast<size_t>(j0) * ldl, ldl,
                                 T(1), X + j0, ldx, sm);
    }
    for (int i = threadIdx.x; i < NB * NB; i += NT) {
      const int r = i / NB, c = i % NB;
      Lb[r * (NB + 1) + c] = (r < bj && c < bj) ? L[static_cast<size_t>(j0 + r) * ldl + j0 + c] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += NT) {
      T x[NB];
      T* xr = X + static_cast<size_t>(r) * ldx + j0;
#pragma unroll
      for (int c = 0; c < NB; ++c) x[c] = c < bj ? xr[c] : T(0);
      if (!TRANS) {
        // x[c] = (x[c] - sum_{k > c} x[k] L[k][c]) / L[c][c], c descending
#pragma unroll
        for (int c = NB - 1; c >= 0; --c) {
          if (c < bj) {
            T acc = x[c];
#pragma unroll
            for (int kk = c + 1; kk < NB; ++kk) acc -= x[kk] * Lb[kk * (NB + 1) + c];
            x[c] = acc / Lb[c * (NB + 1) + c];
          }
        }
      } else {
        // x[c] = (x[c] - sum_{k < c} x[k] L[c][k]) / L[c][c], c ascending
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < bj) {
            T acc = x[c];
#pragma unroll
            for (int kk = 0; kk < c; ++kk) acc -= x[kk] * Lb[c * (NB + 1) + kk];
            x[c] = acc / Lb[c * (NB + 1) + c];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < bj) xr[c] = x[c];
    }
    __syncthreads();
  }
}

// L X = B in place (L: n x n lower-triangular, full rank; X: n x m, overwritten).
template <typename T>
__device__ void cta_trsm_left(int n, int m, const T* L, int ldl, T* X, int ldx, T* sm) {
  T* Lb = sm + gemm_smem_elems<T>();
  const int nblk = (n + NB - 1) / NB;
  for (int blk = 0; blk < nblk; ++blk) {
    const int i0 = blk * NB, i1 = min(n, i0 + NB), bi = i1 - i0;
    if (i0 > 0) {
      // X[I, :] -= L[I, 0:i0] X[0:i0, :]
      cta_gemm<T, false, false>(bi, m, i0, T(-1), L + static_cast<size_t>(i0) * ldl, ldl, X, ldx, T(1),
                                X + static_cast<size_t>(i0) * ldx, ldx, sm);
    }
    for (int i = threadIdx.x; i < NB * NB; i += NT) {
      const int r = i / NB, c = i % NB;
      Lb[r * (NB + 1) + c] = (r < bi && c < bi) ? L[static_cast<size_t>(i0 + r) * ldl + i0 + c] : T(0);
    }
    __syncthreads();
    for (int col = threadIdx.x; col < m; col += NT) {
      T x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = r < bi ? X[static_cast<size_t>(i0 + r) * ldx + col] : T(0);
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        if (r < bi) {
          T acc = x[r];
#pragma unroll
          for (int kk = 0; kk < r; ++kk) acc -= Lb[r * (NB + 1) + kk] * x[kk];
          x[r] = acc / Lb[r * (NB + 1) + r];
        }
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < bi) X[static_cast<size_t>(i0 + r) * ldx + col] = x[r];
    }
    __syncthreads();
  }
}

// ---- LQ (tria) ---------------------------------------------------------------------------------
// Compact column set of one panel: position p < kb is column k0 + p, position p >= kb is column
// c1 + (p - kb).
struct PanelCols {
  int k0, kb, c1;
  __device__ __forceinline__ int col(int p) const { return p < kb ? k0 + p : c1 + (p - kb); }
};

// Householder reflection of one row held by a warp (LAPACK larfg convention: H = I - tau v v^T,
// v[j] = 1, [alpha, x] H = [beta, 0]).  The row is first scaled by an exact power of two so that
// its largest entry lies in [0.5, 1): no intermediate overflows or underflows, whatever the
// magnitude of the entries (FP32 rows of rank-deficient factors carry subnormal round-off, whose
// reciprocal would overflow).  Entries negligible against 2^-149 of the row maximum are dropped.
// Writes v (zeros before position j and beyond ws, up to ldv) to vrow and returns tau; the row
// becomes [.., beta, 0, ..].
template <typename T>
__device__ __forceinline__ T make_reflection(T (&x)[MAXCH], int j, int ws, int ldv, T* vrow) {
  const int lane = threadIdx.x & 31;
  const int nch = (ldv + 31) >> 5;  // chunks that hold positions < ldv
  const int cj = j >> 5, lj = j & 31;
  T xa = T(0);
#pragma unroll
  for (int c = 0; c < MAXCH; ++c)
    if (c == cj) xa = x[c];
  const T alpha = __shfl_sync(0xffffffffu, xa, lj);
  T amax = T(0);
#pragma unroll
  for (int c = 0; c < MAXCH; ++c) {
    if (c >= nch) break;
    const int p = lane + 32 * c;
    if (p >= j && p < ws) amax = fmax(amax, fabs(x[c]));
  }
  amax = warp_max(amax);
  int e = 0;
  if (amax > T(0)) frexp(amax, &e);
  T ssq = T(0);
#pragma unroll
  for (int c = 0; c < MAXCH; ++c) {
    if (c >= nch) break;
    const int p = lane + 32 * c;
    if (p > j && p < ws) {
      const T t = ldexp(x[c], -e);
      ssq += t * t;
    }
  }
  ssq = warp_sum(ssq);
  T tau = T(0), beta = alpha, scale = T(0);
  if (ssq > T(0)) {
    const T as = ldexp(alpha, -e);
    const T nrm = sqrt(as * as + ssq);
    const T bs = as >= T(0) ? -nrm : nrm;
    tau = (bs - as) / bs;
    scale = T(1) / (as - bs);
    beta = ldexp(bs, e);
  }
#pragma unroll
  for (int c = 0; c < MAXCH; ++c) {
    if (c >= nch) break;
    const int p = lane + 32 * c;
    const T v = (p == j) ? T(1) : ((p > j && p < ws) ? ldexp(x[c], -e) * scale : T(0));
    if (p < ldv) vrow[p] = v;
    x[c] = (p == j) ? beta : ((p > j) ? T(0) : x[c]);
  }
  return tau;
}

// In-place LQ of the first rf rows of M (rows x ncols, row stride ld); see the file header.
// Requires rf <= rows, rf <= ncols, and either ctri == 0 (dense) or rf <= ctri <= ncols with
// rows < ctri lower-triangular in columns [0, ctri).  The compact panel width
// kb + (ncols - max(k0 + kb, ctri)) must not exceed MAXWS.
// sm: lq_smem_elems<T>(wsmax) elements with wsmax >= every panel width of this call.
// FP64 with tcx: the trailing rows' two products run as exact digit products on the tensor
// cores (pit_tc.cuh); sm then needs lq_tc_smem_bytes(wsmax) bytes and wbuf (global memory of
// the block) 2 (rows - 1) NB values.
template <typename T>
__device__ __noinline__ void cta_lq(T* M, int ld, int rows, int rf, int ctri, int ncols, T* sm,
                                   int wsmax, const tc::TcCtx* tcx = nullptr, T* wbuf = nullptr) {
  constexpr int RT = LqTile<T>::RT;
  constexpr bool kF64 = std::is_same<T, double>::value;
  const bool use_tc = kF64 && tcx != nullptr;
  const int ldvmax = lq_ldv<T>(wsmax);
  T* Vs = sm;                                           // [NB][ldv]
  T* Xs = Vs + NB * ldvmax;                             // [RT][ldv] (FP64 pipes only)
  T* Tm = use_tc ? Xs : Xs + RT * ldvmax;               // [NB][NB + 1]
  T* Gm = Tm + NB * (NB + 1);                           // [NB][NB + 1] Gram v_i . v_j (i < j)
  T* W2t = Gm + NB * (NB + 1);                          // [NB][RT + 4] (FP64 pipes only)
  T* Ws = W2t + NB * (RT + 4);                          // [RT][NB + 1] (FP64 pipes only)
  T* tau = use_tc ? W2t : Ws + RT * (NB + 1);           // [NB]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tid = threadIdx.x;

  for (int k0 = 0; k0 < rf; k0 += NB) {
    const int kb = min(NB, rf - k0);
    const int c1 = max(k0 + kb, ctri);
    const int ws = kb + max(0, ncols - c1);
    const int ldv = lq_ldv<T>(ws);
    const PanelCols pc{k0, kb, c1};
    // unused reflection rows are zero (the trailing products read all NB rows)
    for (int i = kb * ldv + tid; i < NB * ldv; i += NT) Vs[i] = T(0);

    // ---- panel: rows k0 .. k0+kb-1 in registers, two per warp (rows warp, warp + 16)
    T x[2][MAXCH];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = warp + s * NWARPS;
#pragma unroll
      for (int c = 0; c < MAXCH; ++c) {
        const int p = lane + 32 * c;
        x[s][c] = (i < kb && p < ws) ? M[static_cast<size_t>(k0 + i) * ld + pc.col(p)] : T(0);
      }
    }
    const int nch = (ldv + 31) >> 5;
    for (int j = 0; j < kb; ++j) {
      if (warp == (j % NWARPS)) {
        const int s_own = j / NWARPS;
        T tj;
        if (s_own == 0) tj = make_reflection<T>(x[0], j, ws, ldv, Vs + j * ldv);
        else tj = make_reflection<T>(x[1], j, ws, ldv, Vs + j * ldv);
        if (lane == 0) tau[j] = tj;
      }
      __syncthreads();
      const T tj = tau[j];
      T vr[MAXCH];
#pragma unroll
      for (int c = 0; c < MAXCH; ++c) {
        const int p = lane + 32 * c;
        vr[c] = (c < nch && p < ldv) ? Vs[j * ldv + p] : T(0);
      }
      // apply H_j to the panel rows below j held by this warp (warp-uniform conditions)
      const int i0 = warp, i1 = warp + NWARPS;
      const bool a0 = i0 > j && i0 < kb, a1 = i1 > j && i1 < kb;
      if (a0 || a1) {
        T acc0 = T(0), acc1 = T(0);
#pragma unroll
        for (int c = 0; c < MAXCH; ++c) {
          if (c >= nch) break;
          if (a0) acc0 += x[0][c] * vr[c];
          if (a1) acc1 += x[1][c] * vr[c];
        }
        acc0 = warp_sum(acc0);
        acc1 = warp_sum(acc1);
        const T f0 = tj * acc0, f1 = tj * acc1;
#pragma unroll
        for (int c = 0; c < MAXCH; ++c) {
          if (c >= nch) break;
          if (a0) x[0][c] -= f0 * vr[c];
          if (a1) x[1][c] -= f1 * vr[c];
        }
      }
      // Gram entries G[i][j] = v_i . v_j for i < j (rows i = warp, warp + 16)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int i = warp + s * NWARPS;
        if (i < j) {
          T g = T(0);
#pragma unroll
          for (int c = 0; c < MAXCH; ++c) {
            if (c >= nch) break;
            const int p = lane + 32 * c;
            if (p < ldv) g += Vs[i * ldv + p] * vr[c];
          }
          g = warp_sum(g);
          if (lane == 0) Gm[i * (NB + 1) + j] = g;
        }
      }
    }
    // write the triangularised panel rows back
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = warp + s * NWARPS;
      if (i < kb) {
#pragma unroll
        for (int c = 0; c < MAXCH; ++c) {
          const int p = lane + 32 * c;
          if (p < ws) M[static_cast<size_t>(k0 + i) * ld + pc.col(p)] = x[s][c];
        }
      }
    }
    __syncthreads();
    if (k0 + kb >= rows) continue;  // no trailing rows

    // ---- T of the compact WY form H_0 ... H_{kb-1} = I - V T V^T (upper-triangular):
    // T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V^T v_j)[0:j].  Thread i owns row i.
    if (warp == 0) {
      const int i = lane;
      for (int j = 0; j < NB; ++j) {
        T t = T(0);
        if (j < kb) {
          if (i == j) {
            t = tau[j];
          } else if (i < j) {
            T a0 = T(0), a1 = T(0);
            int kk = i;
            for (; kk + 1 < j; kk += 2) {
              a0 += Tm[i * (NB + 1) + kk] * Gm[kk * (NB + 1) + j];
              a1 += Tm[i * (NB + 1) + kk + 1] * Gm[(kk + 1) * (NB + 1) + j];
            }
            if (kk < j) a0 += Tm[i * (NB + 1) + kk] * Gm[kk * (NB + 1) + j];
            t = -tau[j] * (a0 + a1);
          }
        }
        Tm[i * (NB + 1) + j] = t;
      }
    }
    __syncthreads();

    if constexpr (kF64) {
      if (use_tc) {
        // ---- trailing rows on the tensor cores: W = X V^T, W2 = W T, X <- X - W2 V
        const int r0 = k0 + kb, R = rows - r0;
        unsigned char* stage = reinterpret_cast<unsigned char*>(
            (reinterpret_cast<uintptr_t>(tau + NB) + 127) & ~static_cast<uintptr_t>(127));
        const tc::TcCtx c{stage, tcx->gstatus, tcx->wait_ns};
        double* W = wbuf;                                   // [R][NB]
        double* W2 = wbuf + static_cast<size_t>(R) * NB;   // [R][NB]
        tc::cta_dgemm_f(
            c, R, NB, ws,
            [=](int i, int l) { return M[static_cast<size_t>(r0 + i) * ld + pc.col(l)]; },
            [=](int l, int j) { return Vs[j * ldv + l]; },
            [=](int i, int j, double v, bool first) {
              double* w = W + static_cast<size_t>(i) * NB + j;
              *w = first ? v : *w + v;
            });
        tc::cta_dgemm_f(
            c, R, NB, NB, [=](int i, int l) { return W[static_cast<size_t>(i) * NB + l]; },
            [=](int l, int j) { return l <= j ? Tm[l * (NB + 1) + j] : 0.0; },
            [=](int i, int j, double v, bool first) {
              double* w = W2 + static_cast<size_t>(i) * NB + j;
              *w = first ? v : *w + v;
            });
        tc::cta_dgemm_f(
            c, R, ws, NB, [=](int i, int l) { return W2[static_cast<size_t>(i) * NB + l]; },
            [=](int l, int j) { return Vs[l * ldv + j]; },
            [=](int i, int j, double v, bool) {
              M[static_cast<size_t>(r0 + i) * ld + pc.col(j)] -= v;
            });
        continue;
      }
    }

    // ---- trailing rows: X <- X - ((X V) T) V^T on the panel's columns, RT rows at a time
    for (int r0 = k0 + kb; r0 < rows; r0 += RT) {
      const int nr = min(RT, rows - r0);
      for (int i = tid; i < RT * ldv; i += NT) {
        const int r = i / ldv, p = i - r * ldv;
        Xs[r * ldv + p] = (r < nr && p < ws) ? M[static_cast<size_t>(r0 + r) * ld + pc.col(p)] : T(0);
      }
      __syncthreads();
      // W = Xs V^T  (RT x NB): 4 x 4 tiles, the p range split over KS lanes
      {
        constexpr int TILES = (RT / 4) * (NB / 4);
        constexpr int KS = NT / TILES;
        const int tile = tid / KS, ks = tid % KS;
        const int rg = tile / (NB / 4), jg = tile % (NB / 4);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int pq = ks; pq < ldv / 4; pq += KS) {
          T xv[4][4], vv[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a) ld4s(Xs + (4 * rg + a) * ldv + 4 * pq, xv[a]);
#pragma unroll
          for (int b = 0; b < 4; ++b) ld4s(Vs + (4 * jg + b) * ldv + 4 * pq, vv[b]);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[a][b] += xv[a][e] * vv[b][e];
        }
#pragma unroll
        for (int o = 1; o < KS; o <<= 1)
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += __shfl_xor_sync(0xffffffffu, acc[a][b], o);
        if (ks == 0) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Ws[(4 * rg + a) * (NB + 1) + 4 * jg + b] = acc[a][b];
        }
      }
      __syncthreads();
      // W2 = W T, stored transposed: W2t[j][r]
      for (int i = tid; i < RT * NB; i += NT) {
        const int r = i / NB, j = i % NB;
        T acc = T(0);
        for (int kk = 0; kk <= j; ++kk) acc += Ws[r * (NB + 1) + kk] * Tm[kk * (NB + 1) + j];
        W2t[j * (RT + 4) + r] = acc;
      }
      __syncthreads();
      // Xs - W2 V, written straight to M: 4 rows x 4 positions per thread-tile
      {
        const int nq = (ws + 3) / 4;
        const int ntile = (RT / 4) * nq;
        for (int t = tid; t < ntile; t += NT) {
          const int rg = t / nq, pq = t - rg * nq;
          T acc[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a) ld4s(Xs + (4 * rg + a) * ldv + 4 * pq, acc[a]);
          for (int j = 0; j < kb; ++j) {
            T w[4], v[4];
            ld4s(W2t + j * (RT + 4) + 4 * rg, w);
            ld4s(Vs + j * ldv + 4 * pq, v);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] -= w[a] * v[b];
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int r = 4 * rg + a;
            if (r >= nr) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int p = 4 * pq + b;
              if (p < ws) M[static_cast<size_t>(r0 + r) * ld + pc.col(p)] = acc[a][b];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

}  // namespace dn
}  // namespace pit
