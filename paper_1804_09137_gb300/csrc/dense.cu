// Dense float64 Cholesky of one diagonal tile: blocked right-looking over
// 32-column panels (panel POTRF in shared memory, row-parallel panel TRSM,
// 64 x 64-blocked SYRK of the trailing lower triangle).
#include "common.cuh"

namespace {

constexpr int PB = 32;  // panel width of the tile Cholesky

// unblocked Cholesky of the w x w diagonal block at (c0, c0), in shared memory
__global__ void k_potrf_diag(double* __restrict__ A, int lda, int c0, int w, int64_t col0,
                             long long* __restrict__ st) {
  __shared__ double S[PB][PB + 1];
  for (int id = threadIdx.x; id < w * w; id += blockDim.x) {
    const int r = id % w, c = id / w;
    S[r][c] = A[(size_t)(c0 + c) * lda + c0 + r];
  }
  __syncthreads();
  for (int c = 0; c < w; ++c) {
    if (threadIdx.x == 0) {
      double d = S[c][c];
      if (!(d > 0.0)) {  // non-positive or NaN pivot
        set_status(st, TLR_ERR_NOT_SPD, col0 + c0 + c + 1);
        d = 1.0;
      }
      S[c][c] = sqrt(d);
    }
    __syncthreads();
    const double inv = 1.0 / S[c][c];
    for (int r = c + 1 + threadIdx.x; r < w; r += blockDim.x) S[r][c] *= inv;
    __syncthreads();
    for (int id = threadIdx.x; id < w * w; id += blockDim.x) {
      const int r = id % w, q = id / w;
      if (q > c && r >= q) S[r][q] -= S[r][c] * S[q][c];
    }
    __syncthreads();
  }
  for (int id = threadIdx.x; id < w * w; id += blockDim.x) {
    const int r = id % w, c = id / w;
    A[(size_t)(c0 + c) * lda + c0 + r] = (r >= c) ? S[r][c] : 0.0;
  }
}

// rows r >= c0 + w of the panel: A[r, c0:c0+w] <- A[r, c0:c0+w] L_pp^{-T}
__global__ void k_trsm_panel(double* __restrict__ A, int lda, int nrows, int c0, int w) {
  __shared__ double L[PB][PB + 1];
  for (int id = threadIdx.x; id < w * w; id += blockDim.x) {
    const int r = id % w, c = id / w;
    L[r][c] = A[(size_t)(c0 + c) * lda + c0 + r];
  }
  __syncthreads();
  const int r = c0 + w + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  double xr[PB];
#pragma unroll
  for (int c = 0; c < PB; ++c) xr[c] = (c < w) ? A[(size_t)(c0 + c) * lda + r] : 0.0;
#pragma unroll
  for (int c = 0; c < PB; ++c) {
    if (c < w) {
      double s = xr[c];
#pragma unroll
      for (int l = 0; l < PB; ++l)
        if (l < c) s -= xr[l] * L[c][l];
      xr[c] = s / L[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < PB; ++c)
    if (c < w) A[(size_t)(c0 + c) * lda + r] = xr[c];
}

// C[r0:r0+64, q0:q0+64] -= A[r0:.., 0:K] * B[q0:.., 0:K]^T  (column major, 256 threads)
// rows >= mrows / cols >= mcols are ignored
__device__ __forceinline__ void tile_gemm_nt_sub(const double* __restrict__ A, int lda, const double* __restrict__ B,
                                                 int ldb, double* __restrict__ C, int ldc, int r0, int q0, int mrows,
                                                 int mcols, int K, bool lower_only) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int id = threadIdx.x; id < 64 * 16; id += 256) {
      const int a = id & 63, kk = id >> 6;
      const int ra = r0 + a, qb = q0 + a, kc = k0 + kk;
      As[kk][a] = (ra < mrows && kc < K) ? A[(size_t)kc * lda + ra] : 0.0;
      Bs[kk][a] = (qb < mcols && kc < K) ? B[(size_t)kc * ldb + qb] : 0.0;
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
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, q = q0 + tx + 16 * j;
      if (r < mrows && q < mcols && (!lower_only || r >= q)) C[(size_t)q * ldc + r] -= acc[i][j];
    }
}

// trailing update of the tile Cholesky: lower blocks of A[c1:, c1:] -= P P^T, P = A[c1:, c0:c1]
__global__ void k_syrk_trailing(double* __restrict__ A, int lda, int nrows, int c0, int w) {
  const int c1 = c0 + w;
  // decode lower block (bi >= bj) from blockIdx.x
  const int t = blockIdx.x;
  int bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  const int bj = t - bi * (bi + 1) / 2;
  const double* P = A + (size_t)c0 * lda + c1;
  double* C = A + (size_t)c1 * lda + c1;
  tile_gemm_nt_sub(P, lda, P, lda, C, lda, 64 * bi, 64 * bj, nrows - c1, nrows - c1, w, true);
}

}  // namespace

int tlr_potrf_tile(tlr_ctx* h, double* A, int lda, int nb, int64_t col0, cudaStream_t s) {
  for (int c0 = 0; c0 < nb; c0 += PB) {
    const int w = nb - c0 < PB ? nb - c0 : PB;
    k_potrf_diag<<<1, 256, 0, s>>>(A, lda, c0, w, col0, h->d_stat);
    TLR_LAUNCH_CHECK();
    const int below = nb - c0 - w;
    if (below > 0) {
      k_trsm_panel<<<(below + 127) / 128, 128, 0, s>>>(A, lda, nb, c0, w);
      TLR_LAUNCH_CHECK();
      const int T = (below + 63) / 64;
      k_syrk_trailing<<<T * (T + 1) / 2, 256, 0, s>>>(A, lda, nb, c0, w);
      TLR_LAUNCH_CHECK();
    }
  }
  return TLR_OK;
}

