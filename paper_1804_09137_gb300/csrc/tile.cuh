// Tile views and CTA-level float64 building blocks shared by the factor,
// inverse and solve kernels.
//
// Off-diagonal tile t = i(i-1)/2 + j (i > j) is either
//   low rank: U_t V_t^T, U_t, V_t in slot t (nb x kcap, column-major, ld nb), rank rank[t];
//   dense:    A_t in dense-pool slot dslot[t] (nb x nb, column-major, ld nb).
// Diagonal tiles are always dense (D + i nb^2).
#pragma once
#include "common.cuh"

struct TlrView {
  int nb, nt, kcap;
  double* D;      // nt diagonal tiles
  double* U;      // low-rank slots
  double* V;
  int* rank;      // per off-diagonal tile
  int* dslot;     // dense-pool slot or -1
  double* dpool;  // dense pool
};

static inline TlrView view_of(const tlr_ctx* h) {
  TlrView v;
  v.nb = h->nb; v.nt = h->nt; v.kcap = h->kcap;
  v.D = h->D; v.U = h->U; v.V = h->V; v.rank = h->rank; v.dslot = h->dslot; v.dpool = h->dpool;
  return v;
}

struct GemmDesc {  // C -= P Q^T (nb x nb), inner dimension r; lower: only the lower triangle
  const double* P;
  const double* Q;
  double* C;
  int r;
  int lower;
};

__device__ __forceinline__ size_t lr_slot(const TlrView& v) { return (size_t)v.nb * v.kcap; }
__device__ __forceinline__ double* tileU(const TlrView& v, int64_t t) { return v.U + t * lr_slot(v); }
__device__ __forceinline__ double* tileV(const TlrView& v, int64_t t) { return v.V + t * lr_slot(v); }
__device__ __forceinline__ double* tileA(const TlrView& v, int64_t t) {
  return v.dpool + (size_t)v.dslot[t] * v.nb * v.nb;
}
__device__ __forceinline__ double* diagT(const TlrView& v, int i) { return v.D + (size_t)i * v.nb * v.nb; }

// C[0:m, 0:n] = beta C + alpha op(A) op(B); op(A) is m x k, op(B) is k x n; column-major.
// tA / tB: 0 no transpose, 1 transpose.  Whole CTA (256 threads) cooperates; the
// output is processed in 64 x 64 blocks, block ids [blk0, blk0 + nblk_step, ...).
__device__ __forceinline__ void cta_gemm_blocks(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                int lda, int tA, const double* __restrict__ B, int ldb, int tB,
                                                double beta, double* __restrict__ C, int ldc, int blk0,
                                                int nblk_step, int lower_only) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int mb = (m + 63) / 64, nbk = (n + 63) / 64;
  for (int blk = blk0; blk < mb * nbk; blk += nblk_step) {
    const int bi = blk % mb, bj = blk / mb;
    const int r0 = bi * 64, c0 = bj * 64;
    if (lower_only && r0 + 63 < c0) continue;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
      __syncthreads();
      for (int id = threadIdx.x; id < 64 * 16; id += 256) {
        int a, kk;
        // coalesced mapping depends on the storage direction
        if (!tA) { a = id & 63; kk = id >> 6; } else { kk = id & 15; a = id >> 4; }
        const int ra = r0 + a, kc = k0 + kk;
        double v = 0.0;
        if (ra < m && kc < k) v = tA ? A[(size_t)ra * lda + kc] : A[(size_t)kc * lda + ra];
        As[kk][a] = v;
        if (!tB) { kk = id & 15; a = id >> 4; } else { a = id & 63; kk = id >> 6; }
        const int cb = c0 + a, kc2 = k0 + kk;
        double w = 0.0;
        if (cb < n && kc2 < k) w = tB ? B[(size_t)kc2 * ldb + cb] : B[(size_t)cb * ldb + kc2];
        Bs[kk][a] = w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
        if (r < m && c < n && (!lower_only || r >= c)) {
          double* cp = C + (size_t)c * ldc + r;
          *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * acc[i][j];
        }
      }
  }
  __syncthreads();
}

__device__ __forceinline__ void cta_gemm(int m, int n, int k, double alpha, const double* A, int lda, int tA,
                                         const double* B, int ldb, int tB, double beta, double* C, int ldc) {
  cta_gemm_blocks(m, n, k, alpha, A, lda, tA, B, ldb, tB, beta, C, ldc, 0, 1, 0);
}

__device__ __forceinline__ void decode_lower(int64_t t, int* i, int* j) {
  int ii = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while ((int64_t)ii * (ii - 1) / 2 > t) --ii;
  while ((int64_t)(ii + 1) * ii / 2 <= t) ++ii;
  *i = ii;
  *j = (int)(t - (int64_t)ii * (ii - 1) / 2);
}

// Work item of a batched tile operation (built on the host from the tile kinds).
struct TileItem {
  int i, j, k;  // target (i, j); source index k (meaning depends on the operation)
  int kind;     // operation-specific case code
};
