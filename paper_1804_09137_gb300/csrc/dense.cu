// Dense Cholesky of one diagonal tile in one launch: a cooperative grid (every CTA
// resident) walks the tile's 32-column panels right-looking, with two grid barriers
// per panel:
//   1. the CTAs that own rows below the panel (and CTA 0) factor the panel's 32 x 32
//      diagonal block in float64 (one warp, a row per lane, in shared memory),
//      CTA 0 stores it, and each CTA solves its share of the panel rows
//      (A[r, panel] <- A[r, panel] L_pp^{-T}, a row per warp, float64);
//   2. the trailing lower triangle is updated in 64 x 64 blocks spread over the CTAs
//      (A22 <- A22 - P P^T with the products in double-float on the float32 pipe).
// Only the lower triangle of the tile is read or defined afterwards; the strict upper
// part of each 32 x 32 diagonal block is written as zero.  Every barrier wait is
// bounded (about two seconds): a CTA that gives up records TLR_ERR_TIMEOUT and returns.
#include "common.cuh"
#include "recompress.cuh"

namespace {

constexpr int PB = 32;  // panel width of the tile Cholesky

__global__ void __launch_bounds__(256, 2) k_potrf_tile(double* __restrict__ A, int lda, int nb, int64_t col0,
                                                       long long* __restrict__ st, unsigned int* __restrict__ bar) {
  __shared__ double Ls[PB][PB + 1];
  __shared__ double Linv[PB];  // reciprocals of the diagonal block's pivots
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned int target = 0;
  for (int c0 = 0; c0 < nb; c0 += PB) {
    const int w = nb - c0 < PB ? nb - c0 : PB;
    const int c1 = c0 + w;
    const int below = nb - c1;
    const int per = (below + gridDim.x - 1) / gridDim.x;  // panel rows per CTA
    const int r_lo = blockIdx.x * per;
    const int r_hi = below < r_lo + per ? below : r_lo + per;
    if (blockIdx.x == 0 || r_lo < r_hi) {
      if (warp == 0) {
        // lane r owns row r of the diagonal block in shared memory (identity beyond w)
        for (int q = 0; q < PB; ++q)
          Ls[lane][q] = (lane < w && q < w) ? A[(size_t)(c0 + q) * lda + c0 + lane] : (lane == q ? 1.0 : 0.0);
        __syncwarp();
        for (int c = 0; c < w; ++c) {
          double d = Ls[c][c];
          if (!(d > 0.0)) {  // non-positive or NaN pivot
            if (blockIdx.x == 0 && lane == 0) set_status(st, TLR_ERR_NOT_SPD, col0 + c0 + c + 1);
            d = 1.0;
          }
          const double l = sqrt(d);
          __syncwarp();
          if (lane == c) Ls[c][c] = l;
          else if (lane > c && lane < w) Ls[lane][c] /= l;
          __syncwarp();
          if (lane > c && lane < w) {
            const double lrc = Ls[lane][c];
            for (int q = c + 1; q <= lane; ++q) Ls[lane][q] = fma(-lrc, Ls[q][c], Ls[lane][q]);
          }
          __syncwarp();
        }
        for (int q = lane + 1; q < PB; ++q) Ls[lane][q] = 0.0;
        Linv[lane] = 1.0 / Ls[lane][lane];
      }
      __syncthreads();
      if (blockIdx.x == 0)
        for (int id = threadIdx.x; id < w * w; id += blockDim.x) {
          const int r = id % w, c = id / w;
          A[(size_t)(c0 + c) * lda + c0 + r] = Ls[r][c];
        }
      // panel rows of this CTA, a warp per row: lane c holds column c, forward substitution over the columns
      for (int rr = r_lo + warp; rr < r_hi; rr += blockDim.x >> 5) {
        const int r = c1 + rr;
        double x = lane < w ? A[(size_t)(c0 + lane) * lda + r] : 0.0;
        for (int c = 0; c < w; ++c) {
          const double xc = __shfl_sync(0xffffffffu, x, c) * Linv[c];
          if (lane == c) x = xc;
          else if (lane > c) x = fma(-xc, Ls[lane][c], x);
        }
        if (lane < w) A[(size_t)(c0 + lane) * lda + r] = x;
      }
    }
    if (below <= 0) break;
    if (!grid_barrier(bar, target, st)) return;
    // A22 -= P P^T over the lower blocks of the trailing matrix, P = A[c1:, c0:c1]
    const double* P = A + (size_t)c0 * lda + c1;
    cta_gemm_df_blocks(below, below, w, -1.0, P, lda, 0, P, lda, 1, 1.0, A + (size_t)c1 * lda + c1, lda, blockIdx.x,
                       gridDim.x, 1);
    if (!grid_barrier(bar, target, st)) return;
  }
}

// resident CTAs of k_potrf_tile on the current device (cached per device)
int potrf_max_grid() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev] > 0) return cached[dev];
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_potrf_tile, 256, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cached[dev] = per_sm * sms;
  return cached[dev];
}

}  // namespace

int tlr_potrf_tile(tlr_ctx* h, double* A, int lda, int nb, int64_t col0, cudaStream_t s) {
  if (nb <= 0) return TLR_OK;
  const int maxg = potrf_max_grid();
  if (maxg < 1) return TLR_ERR_CUDA;
  // one CTA per 64 x 64 block of the first panel's trailing update, within what stays resident
  const int t = (nb - PB + 63) / 64;
  int grid = t > 0 ? t * (t + 1) / 2 : 1;
  if (grid > maxg) grid = maxg;
  long long* st = h->d_stat;
  unsigned int* bar = reinterpret_cast<unsigned int*>(h->d_stat + ST_BAR);
  TLR_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned int), s));
  void* args[] = {&A, &lda, &nb, &col0, &st, &bar};
  TLR_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_potrf_tile, dim3(grid), dim3(256), args, 0, s));
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}
