// Dense float64 tile kernels: Cholesky of one diagonal tile (blocked, right
// looking, 32-column panels), the batched triangular solve L^{-1} X applied to
// the V factors of a tile column, and the batched C -= A B^T update used by the
// low-rank SYRK into the diagonal tiles.
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

// batched X_i <- L^{-1} X_i, L: nb x nb lower (ld nb), X_i: nb x k_i (ld nb), 32 columns per block
// items: V slots of tiles (i, k) for i = k+1 .. nt-1
__global__ void k_trsm_v(const double* __restrict__ L, int nb, double* __restrict__ Vbase, size_t slot_elems,
                         const int* __restrict__ rank, int k, int kcap) {
  const int i = k + 1 + blockIdx.y;
  const int64_t t = dtile_index(i, k);
  const int kr = rank[t];
  const int cb = blockIdx.x * 32;
  if (cb >= kr) return;
  const int ncol = min(32, kr - cb);
  double* X = Vbase + (size_t)t * slot_elems + (size_t)cb * nb;
  __shared__ double Ls[32][33];
  __shared__ double Xs[32][33];
  for (int rb0 = 0; rb0 < nb; rb0 += 32) {
    const int w = min(32, nb - rb0);
    for (int id = threadIdx.x; id < 32 * 32; id += blockDim.x) {
      const int r = id & 31, c = id >> 5;
      Ls[r][c] = (r < w && c < w) ? L[(size_t)(rb0 + c) * nb + rb0 + r] : 0.0;
      Xs[r][c] = (r < w && c < ncol) ? X[(size_t)c * nb + rb0 + r] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < ncol) {  // forward substitution, one column per thread
      const int c = threadIdx.x;
      for (int r = 0; r < w; ++r) {
        double s = Xs[r][c];
        for (int l = 0; l < r; ++l) s -= Ls[r][l] * Xs[l][c];
        Xs[r][c] = s / Ls[r][r];
      }
    }
    __syncthreads();
    for (int id = threadIdx.x; id < 32 * 32; id += blockDim.x) {
      const int r = id & 31, c = id >> 5;
      if (r < w && c < ncol) X[(size_t)c * nb + rb0 + r] = Xs[r][c];
    }
    // rows below: X[r, :] -= L[r, rb0:rb0+w] Xs
    for (int r = rb0 + w + threadIdx.x; r < nb; r += blockDim.x) {
      double acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0.0;
      for (int l = 0; l < w; ++l) {
        const double lv = L[(size_t)(rb0 + l) * nb + r];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fma(lv, Xs[l][c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < ncol) X[(size_t)c * nb + r] -= acc[c];
    }
    __syncthreads();
  }
}

// batched D_i -= T_i U_i^T (lower blocks), T_i in workspace (nb x kcap per item), U_i = U slot of (i, k)
__global__ void k_syrk_lr_update(double* __restrict__ D, int nb, const double* __restrict__ T, size_t t_elems,
                                 const double* __restrict__ Ubase, size_t slot_elems, const int* __restrict__ rank,
                                 int k, int i_first) {
  const int i = i_first + blockIdx.y;
  const int64_t t = dtile_index(i, k);
  const int kr = rank[t];
  if (kr == 0) return;
  const int b = blockIdx.x;
  int bi = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
  while (bi * (bi + 1) / 2 > b) --bi;
  const int bj = b - bi * (bi + 1) / 2;
  tile_gemm_nt_sub(T + (size_t)blockIdx.y * t_elems, nb, Ubase + (size_t)t * slot_elems, nb,
                   D + (size_t)i * nb * nb, nb, 64 * bi, 64 * bj, nb, nb, kr, true);
}

// T_i = U_i (V_i^T V_i) for the SYRK of step k; one block per item
__global__ void k_syrk_lr_prep(int nb, const double* __restrict__ Ubase, const double* __restrict__ Vbase,
                               size_t slot_elems, const int* __restrict__ rank, int k, int i_first,
                               double* __restrict__ T, size_t t_elems, double* __restrict__ G, size_t g_elems) {
  const int i = i_first + blockIdx.x;
  const int64_t t = dtile_index(i, k);
  const int kr = rank[t];
  if (kr == 0) return;
  const double* U = Ubase + (size_t)t * slot_elems;
  const double* V = Vbase + (size_t)t * slot_elems;
  double* Gi = G + (size_t)blockIdx.x * g_elems;
  double* Ti = T + (size_t)blockIdx.x * t_elems;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // G = V^T V (kr x kr), warp per entry (upper incl. diagonal), mirrored
  for (int e = warp; e < kr * kr; e += blockDim.x / 32) {
    const int a = e % kr, c = e / kr;
    if (a > c) continue;
    double s = 0.0;
    for (int r = lane; r < nb; r += 32) s = fma(V[(size_t)a * nb + r], V[(size_t)c * nb + r], s);
    s = warp_sum(s);
    if (lane == 0) { Gi[(size_t)c * kr + a] = s; Gi[(size_t)a * kr + c] = s; }
  }
  __syncthreads();
  // T = U G (nb x kr)
  for (int e = threadIdx.x; e < nb * kr; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    double s = 0.0;
    for (int l = 0; l < kr; ++l) s = fma(U[(size_t)l * nb + r], Gi[(size_t)c * kr + l], s);
    Ti[(size_t)c * nb + r] = s;
  }
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

// launchers used by the factorization driver
int tlr_launch_trsm_v(tlr_ctx* h, int k, cudaStream_t s) {
  const int items = h->nt - k - 1;
  if (items <= 0) return TLR_OK;
  dim3 grid((h->kcap + 31) / 32, items);
  k_trsm_v<<<grid, 256, 0, s>>>(h->D + (size_t)k * h->nb * h->nb, h->nb, h->V, (size_t)h->nb * h->kcap, h->rank, k,
                                h->kcap);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

int tlr_launch_syrk_lr(tlr_ctx* h, int k, cudaStream_t s) {
  const int items = h->nt - k - 1;
  if (items <= 0) return TLR_OK;
  const size_t nb = h->nb, kc = h->kcap;
  const size_t t_elems = nb * kc, g_elems = kc * kc;
  // workspace: items * (T + G); chunk so that it fits
  const size_t per = t_elems + g_elems;
  int chunk = (int)(h->scratch_elems / per);
  if (chunk > 65535) chunk = 65535;
  for (int i0 = 0; i0 < items; i0 += chunk) {
    const int cnt = items - i0 < chunk ? items - i0 : chunk;
    double* T = h->scratch;
    double* G = h->scratch + (size_t)cnt * t_elems;
    k_syrk_lr_prep<<<cnt, 256, 0, s>>>(h->nb, h->U, h->V, nb * kc, h->rank, k, k + 1 + i0, T, t_elems, G, g_elems);
    TLR_LAUNCH_CHECK();
    const int Tb = (h->nb + 63) / 64;
    dim3 grid(Tb * (Tb + 1) / 2, cnt);
    k_syrk_lr_update<<<grid, 256, 0, s>>>(h->D, h->nb, T, t_elems, h->U, nb * kc, h->rank, k, k + 1 + i0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}
