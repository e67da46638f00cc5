// Triangular solves on the TLR factor, log-determinant and quadratic form of
// eq. 1, z = L e (Sec. VIII-D), kriging of eq. 4 and its prediction variance.  Reductions are two-stage (per-block partials summed in
// a fixed order) so results are bitwise reproducible run to run.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "tile.cuh"
#include "tileops.h"

namespace {

__global__ void k_perm_in(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ perm,
                          int64_t n, int64_t npad) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < npad; s += (int64_t)gridDim.x * blockDim.x)
    dst[s] = (s < n) ? src[perm[s]] : 0.0;
}

__global__ void k_perm_out(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ perm,
                           int64_t n) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    dst[perm[s]] = src[s];
}

// r <- L^{-1} r for one dense lower tile (one CTA)
__global__ void k_trsv_lower(const double* __restrict__ L, int nb, double* __restrict__ r) {
  __shared__ double xs[32];
  const int lane = threadIdx.x & 31;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int w = min(32, nb - b0);
    if (threadIdx.x < 32) {
      double xl = 0.0;
      for (int c = 0; c < w; ++c) {
        const double part = (lane < c) ? L[(size_t)(b0 + lane) * nb + b0 + c] * xl : 0.0;
        const double s = warp_sum(part);
        const double v = (r[b0 + c] - s) / L[(size_t)(b0 + c) * nb + b0 + c];
        if (lane == c) xl = v;
      }
      if (lane < w) { xs[lane] = xl; r[b0 + lane] = xl; }
    }
    __syncthreads();
    for (int row = b0 + w + threadIdx.x; row < nb; row += blockDim.x) {
      double acc = 0.0;
      for (int l = 0; l < w; ++l) acc = fma(L[(size_t)(b0 + l) * nb + row], xs[l], acc);
      r[row] -= acc;
    }
    __syncthreads();
  }
}

// r <- L^{-T} r for one dense lower tile (one CTA), backward over row blocks
__global__ void k_trsv_lower_t(const double* __restrict__ L, int nb, double* __restrict__ r) {
  __shared__ double xs[32];
  const int lane = threadIdx.x & 31;
  const int nblk = (nb + 31) / 32;
  for (int bb = nblk - 1; bb >= 0; --bb) {
    const int b0 = bb * 32, w = min(32, nb - b0);
    if (threadIdx.x < 32) {
      double xl = 0.0;
      for (int c = w - 1; c >= 0; --c) {
        // (L^T x)_c = sum_{l >= c} L[l, c] x_l
        const double part = (lane > c && lane < w) ? L[(size_t)(b0 + c) * nb + b0 + lane] * xl : 0.0;
        const double s = warp_sum(part);
        const double v = (r[b0 + c] - s) / L[(size_t)(b0 + c) * nb + b0 + c];
        if (lane == c) xl = v;
      }
      if (lane < w) { xs[lane] = xl; r[b0 + lane] = xl; }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < b0; a += blockDim.x) {
      double acc = 0.0;
      const double* col = L + (size_t)a * nb + b0;
      for (int l = 0; l < w; ++l) acc = fma(col[l], xs[l], acc);
      r[a] -= acc;
    }
    __syncthreads();
  }
}

// rows r0 .. r0 + 31 of xo = op(M) r for the explicit inverse M = L_kk^{-1} of a diagonal tile
// (op(M) = M^T when trans), one CTA of 256 threads
__device__ void diag_inv_rows(const double* __restrict__ M, int nb, int trans, const double* __restrict__ r,
                              double* __restrict__ xo, int r0) {
  __shared__ double part[8][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!trans) {  // (M r)_a = sum_b M[b * nb + a] r[b]: lanes over rows (coalesced), warps split b
    const int a = r0 + lane;
    double acc = 0.0;
    if (a < nb)
      for (int b = warp; b <= a; b += 8) acc = fma(M[(size_t)b * nb + a], r[b], acc);
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && a < nb) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += part[w][lane];
      xo[a] = t;
    }
    __syncthreads();  // part is rewritten by the CTA's next call
  } else {  // (M^T r)_a = sum_{b >= a} M[a * nb + b] r[b]: warp per row, lanes over b
    for (int q = warp; q < 32; q += 8) {
      const int a = r0 + q;
      if (a >= nb) break;
      double t = 0.0;
      for (int b = a + lane; b < nb; b += 32) t = fma(M[(size_t)a * nb + b], r[b], t);
      t = warp_sum(t);
      if (lane == 0) xo[a] = t;
    }
  }
}

// rows [c0, c1) of  r_i -= L_ik x  (forward, tile (i, k)) or  r_j -= L_kj^T x  (backward, tile (k, j))
__device__ void tile_gemv_sub(const TlrView& v, int64_t t, int bwd, const double* __restrict__ x,
                              double* __restrict__ out, int c0, int c1, double* tv) {
  const int nb = v.nb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (v.dslot[t] >= 0) {
    const double* A = tileA(v, t);
    if (!bwd) {  // (A x)_a = sum_b A[b * nb + a] x[b]
      for (int a = c0 + threadIdx.x; a < c1; a += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc = fma(A[(size_t)b * nb + a], x[b], acc);
        out[a] -= acc;
      }
    } else {  // (A^T x)_a = sum_b A[a * nb + b] x[b]
      for (int a = c0 + warp; a < c1; a += nw) {
        double acc = 0.0;
        for (int b = lane; b < nb; b += 32) acc = fma(A[(size_t)a * nb + b], x[b], acc);
        acc = warp_sum(acc);
        if (lane == 0) out[a] -= acc;
      }
    }
    return;
  }
  const int kr = v.rank[t];
  if (kr <= 0) return;
  // forward: out -= U (V^T x); backward: out -= V (U^T x)
  const double* P = bwd ? tileV(v, t) : tileU(v, t);
  const double* Q = bwd ? tileU(v, t) : tileV(v, t);
  for (int l = warp; l < kr; l += nw) {
    double acc = 0.0;
    for (int q = lane; q < nb; q += 32) acc = fma(Q[(size_t)l * nb + q], x[q], acc);
    acc = warp_sum(acc);
    if (lane == 0) tv[l] = acc;
  }
  __syncthreads();
  for (int a = c0 + threadIdx.x; a < c1; a += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < kr; ++l) acc = fma(P[(size_t)l * nb + a], tv[l], acc);
    out[a] -= acc;
  }
}

// Work item q of step k of a solve, after x_k = op(L_kk^{-1}) r_k is in xk: item 0 stores x_k into
// r_k; the others update the remaining blocks, GEMV_SPLIT row chunks per tile (a dense tile's
// nb^2 multiply-adds are spread over the chunks; a low-rank tile is one chunk's work)
#define GEMV_SPLIT 16
__device__ void gemv_item(const TlrView& v, int k, int bwd, const double* __restrict__ xk, double* __restrict__ r,
                          int q, double* tv) {
  const int nb = v.nb;
  if (q == 0) {
    for (int a = threadIdx.x; a < nb; a += blockDim.x) r[(size_t)k * nb + a] = xk[a];
    return;
  }
  --q;
  const int tix = q / GEMV_SPLIT, c = q % GEMV_SPLIT;
  const int other = bwd ? tix : k + 1 + tix;  // block row i (forward) or column j (backward)
  const int64_t t = bwd ? dtile_index(k, other) : dtile_index(other, k);
  const bool dense = v.dslot[t] >= 0;
  int c0, c1;
  if (dense) {
    const int w = (nb + GEMV_SPLIT - 1) / GEMV_SPLIT;
    c0 = min(nb, c * w);
    c1 = min(nb, c0 + w);
  } else {
    if (c != 0) return;
    c0 = 0;
    c1 = nb;
  }
  if (c0 >= c1) return;
  tile_gemv_sub(v, t, bwd, xk, r + (size_t)other * nb, c0, c1, tv);
}

// A whole tile triangular solve in one launch, r <- L^{-1} r (forward) or L^{-T} r (backward): a
// cooperative grid walks the block columns (rows), each step in two phases separated by grid
// barriers: x_k = op(L_kk^{-1}) r_k into xk (32-row chunks over the CTAs), then the work items of
// gemv_item over the CTAs in turn.  tv: kcap doubles of dynamic shared memory.
__global__ void __launch_bounds__(256) k_solve_tiles(TlrView v, const double* __restrict__ linv, int bwd,
                                                     double* __restrict__ r, double* __restrict__ xk,
                                                     long long* __restrict__ st, unsigned int* __restrict__ bar) {
  extern __shared__ double tv[];
  const int nb = v.nb, nt = v.nt;
  const int nchunk = (nb + 31) / 32;
  unsigned int target = 0;
  for (int step = 0; step < nt; ++step) {
    const int k = bwd ? nt - 1 - step : step;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x)
      diag_inv_rows(linv + (size_t)k * nb * nb, nb, bwd, r + (size_t)k * nb, xk, 32 * c);
    if (!grid_barrier(bar, target, st)) return;
    const int items = 1 + (bwd ? k : nt - k - 1) * GEMV_SPLIT;
    for (int q = blockIdx.x; q < items; q += gridDim.x) gemv_item(v, k, bwd, xk, r, q, tv);
    if (!grid_barrier(bar, target, st)) return;
  }
}

// z_i = L_ii e_i + sum_{j<i} L_ij e_j   (one CTA per tile row i)
__global__ void k_lmul(TlrView v, const double* __restrict__ e, double* __restrict__ z) {
  extern __shared__ double tv[];
  const int i = blockIdx.x, nb = v.nb;
  const double* Li = diagT(v, i);
  const double* ei = e + (size_t)i * nb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* zi = z + (size_t)i * nb;
  for (int a = threadIdx.x; a < nb; a += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b <= a; ++b) acc = fma(Li[(size_t)b * nb + a], ei[b], acc);
    zi[a] = acc;
  }
  for (int j = 0; j < i; ++j) {
    const int64_t t = dtile_index(i, j);
    const double* ej = e + (size_t)j * nb;
    if (v.dslot[t] >= 0) {
      const double* A = tileA(v, t);
      for (int a = threadIdx.x; a < nb; a += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc = fma(A[(size_t)b * nb + a], ej[b], acc);
        zi[a] += acc;
      }
      continue;
    }
    const int kr = v.rank[t];
    if (kr <= 0) continue;
    const double* Ut = tileU(v, t);
    const double* Vt = tileV(v, t);
    __syncthreads();
    for (int l = warp; l < kr; l += nw) {
      double s = 0.0;
      for (int q = lane; q < nb; q += 32) s = fma(Vt[(size_t)l * nb + q], ej[q], s);
      s = warp_sum(s);
      if (lane == 0) tv[l] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      double acc = 0.0;
      for (int l = 0; l < kr; ++l) acc = fma(Ut[(size_t)l * nb + a], tv[l], acc);
      zi[a] += acc;
    }
  }
}

// per-tile partial of log|L| (sum of log of the diagonal) and of sum w^2
__global__ void k_partials(const double* __restrict__ D, int nb, const double* __restrict__ w,
                           double* __restrict__ part) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  const int k = blockIdx.x;
  const double* Lk = D + (size_t)k * nb * nb;
  double ld = 0.0, q = 0.0;
  for (int a = threadIdx.x; a < nb; a += blockDim.x) {
    ld += log(Lk[(size_t)a * nb + a]);
    const double v = w[(size_t)k * nb + a];
    q = fma(v, v, q);
  }
  ld = block_sum(ld, sh);
  q = block_sum(q, sh);
  if (threadIdx.x == 0) { part[2 * k] = ld; part[2 * k + 1] = q; }
}

__global__ void k_finish_loglik(const double* __restrict__ part, int nt, int64_t n, double* __restrict__ out3) {
  if (threadIdx.x != 0) return;
  double ld = 0.0, q = 0.0;
  for (int k = 0; k < nt; ++k) { ld += part[2 * k]; q += part[2 * k + 1]; }
  ld *= 2.0;
  out3[0] = -0.5 * (double)n * 1.83787706640934548356 - 0.5 * ld - 0.5 * q;  // log(2 pi)
  out3[1] = ld;
  out3[2] = q;
}

// kriging: zn[a] = sum_b C(|new_a - s_b|) alpha_b, one CTA per new point
__global__ void k_krige(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                        const double* __restrict__ y, int64_t n, const double* __restrict__ alpha,
                        const double* __restrict__ xn, const double* __restrict__ yn, double* __restrict__ zn) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  const int64_t a = blockIdx.x;
  const double px = xn[a], py = yn[a];
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < n; b += blockDim.x) {
    acc = fma(matern_tab(tab, mp, 0, pt_dist(mp, px, py, x[b], y[b])), alpha[b], acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) zn[a] = acc;
}

// B[i * ldb + b] = C(|s_b - p_i|) for sorted point b < n, 0 on the padded rows (b < npad)
__global__ void k_cov_block(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                            const double* __restrict__ y, int64_t n, int64_t npad, const double* __restrict__ xn,
                            const double* __restrict__ yn, double* __restrict__ B, int64_t ldb) {
  const int64_t i = blockIdx.y;
  const double px = xn[i], py = yn[i];
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < npad; b += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (b < n) {
      v = matern_tab(tab, mp, 0, pt_dist(mp, px, py, x[b], y[b]));
    }
    B[i * ldb + b] = v;
  }
}

// var[i] = sigma2 - sum_b W[b, i]^2 (one CTA per column)
__global__ void k_colvar(const double* __restrict__ W, int64_t ldw, int64_t rows, double sigma2,
                         double* __restrict__ var) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  const double* w = W + (int64_t)blockIdx.x * ldw;
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < rows; b += blockDim.x) acc = fma(w[b], w[b], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) var[blockIdx.x] = sigma2 - acc;
}

// Step k of the batched forward solve W = L^{-1} C (C consumed, both npad x mb, column-major, ld):
// d0: W_k = L_kk^{-1} C_k with the diagonal tile's explicit inverse; for the block rows i > k
// (thread i - k - 1): low rank  d1: T_i = V_ik^T W_k (rank x mb in Tb, ld kcap), d2: C_i -= U_ik T_i;
// dense  d1 empty, d2: C_i -= A_ik W_k.  Every product writes a block of its own (no operand is
// written by a product of the same stage).
__global__ void k_msolve_desc(TlrView v, int k, const double* __restrict__ linv_k, int mb, double* __restrict__ C,
                              double* __restrict__ W, int64_t ld, double* __restrict__ Tb, GemmGen* __restrict__ d0,
                              GemmGen* __restrict__ d1, GemmGen* __restrict__ d2) {
  const int nb = v.nb;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  GemmGen g;
  g.A = g.B = nullptr; g.C = nullptr; g.m = g.n = g.k = 0; g.lda = g.ldb = nb; g.ldc = (int)ld;
  g.tA = g.tB = 0; g.alpha = 1.0; g.beta = 0.0; g.lower = 0;
  if (q == 0) {
    GemmGen x = g;
    x.A = linv_k; x.B = C + (size_t)k * nb; x.ldb = (int)ld; x.C = W + (size_t)k * nb;
    x.m = nb; x.n = mb; x.k = nb;
    *d0 = x;
  }
  const int i = k + 1 + q;
  if (i >= v.nt) return;
  const int64_t t = dtile_index(i, k);
  const double* Wk = W + (size_t)k * nb;
  double* Ci = C + (size_t)i * nb;
  GemmGen a = g, b = g;
  b.C = Ci; b.m = nb; b.n = mb; b.alpha = -1.0; b.beta = 1.0; b.ldb = (int)ld;
  if (v.dslot[t] >= 0) {
    b.A = tileA(v, t); b.B = Wk; b.k = nb;
  } else {
    const int r = v.rank[t];
    double* Ti = Tb + (size_t)(i - k - 1) * v.kcap * mb;
    if (r > 0) {
      a.A = tileV(v, t); a.tA = 1; a.B = Wk; a.ldb = (int)ld; a.C = Ti; a.ldc = v.kcap; a.m = r; a.n = mb; a.k = nb;
      b.A = tileU(v, t); b.B = Ti; b.ldb = v.kcap; b.k = r;
    }
  }
  d1[q] = a;
  d2[q] = b;
}

}  // namespace

int tlr_permute_in(tlr_ctx* h, const double* src, double* dst, cudaStream_t s) {
  k_perm_in<<<(unsigned)((h->npad + 255) / 256), 256, 0, s>>>(src, dst, h->perm, h->n, h->npad);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

int tlr_permute_out(tlr_ctx* h, const double* src, double* dst, cudaStream_t s) {
  k_perm_out<<<(unsigned)((h->n + 255) / 256), 256, 0, s>>>(src, dst, h->perm, h->n);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

// Tile solves: one cooperative launch each (k_solve_tiles), the diagonal blocks applied as GEMVs with
// the explicit inverses L_kk^{-1} (all formed by tlr_factor).  A single tile (also the allocation-free
// context, which keeps no inverse) is solved by substitution.
namespace {
int solve_max_grid(size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = memo.find({dev, smem});
  if (it != memo.end()) return it->second;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_tiles, 256, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  memo[{dev, smem}] = per_sm * sms;
  return per_sm * sms;
}

int solve_tiles(tlr_ctx* h, int bwd, double* r, cudaStream_t s) {
  const size_t sm = (size_t)h->kcap * sizeof(double);
  const int maxg = solve_max_grid(sm);
  if (maxg < 1) return TLR_ERR_CUDA;
  const int grid = std::min(maxg, 1 + (h->nt - 1) * GEMV_SPLIT);
  TlrView v = view_of(h);
  const double* linv = h->linv;
  double* xk = h->d_xk;
  long long* st = h->d_stat;
  unsigned int* bar = reinterpret_cast<unsigned int*>(h->d_stat + ST_BAR);
  TLR_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned int), s));
  void* args[] = {&v, &linv, &bwd, &r, &xk, &st, &bar};
  TLR_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_solve_tiles, dim3(grid), dim3(256), args, sm, s));
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}
}  // namespace

int tlr_fwd_solve(tlr_ctx* h, double* r, cudaStream_t s) {
  if (h->nt == 1 || !h->d_xk) {  // one tile (also the allocation-free context)
    k_trsv_lower<<<1, 256, 0, s>>>(h->D, h->nb, r);
    TLR_LAUNCH_CHECK();
    return TLR_OK;
  }
  return solve_tiles(h, 0, r, s);
}

int tlr_bwd_solve(tlr_ctx* h, double* r, cudaStream_t s) {
  if (h->nt == 1 || !h->d_xk) {
    k_trsv_lower_t<<<1, 256, 0, s>>>(h->D, h->nb, r);
    TLR_LAUNCH_CHECK();
    return TLR_OK;
  }
  return solve_tiles(h, 1, r, s);
}

int tlr_lmul(tlr_ctx* h, const double* e, double* z, cudaStream_t s) {
  const size_t sm = (size_t)h->kcap * sizeof(double);
  k_lmul<<<h->nt, 256, sm, s>>>(view_of(h), e, z);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

int tlr_reduce_loglik(tlr_ctx* h, const double* w, double* out3, cudaStream_t s) {
  k_partials<<<h->nt, 256, 0, s>>>(h->D, h->nb, w, h->d_red);
  TLR_LAUNCH_CHECK();
  k_finish_loglik<<<1, 32, 0, s>>>(h->d_red, h->nt, h->n, out3);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

int tlr_krige(tlr_ctx* h, const double* a, int64_t m, const double* xn, const double* yn, double* zn,
              cudaStream_t s) {
  for (int64_t a0 = 0; a0 < m; a0 += 65535) {
    const int64_t cnt = m - a0 < 65535 ? m - a0 : 65535;
    k_krige<<<(unsigned)cnt, 256, 0, s>>>(h->tab, h->mp, h->x, h->y, h->n, a, xn + a0, yn + a0, zn + a0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}


#define TRY_RC(x)                  \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != TLR_OK) return rc_; \
  } while (0)

// Prediction variance at m new points (sorted-order observations), mb points at a time: the
// covariances C = Sigma_{obs,new} (npad x mb, generated), W = L^{-1} C by the batched tile forward solve
// (three batched GEMM launches per block column), var_j = sigma2 - |W[:, j]|^2.
int tlr_predict_var_sorted(tlr_ctx* h, int64_t m, const double* xn, const double* yn, double* var, cudaStream_t s) {
  const int nt = h->nt, nb = h->nb;
  const int64_t npad = h->npad;
  const size_t nn = (size_t)nb * nb;  // (the Cholesky formed every L_kk^{-1})
  // workspace: descriptors, then per right-hand side C, W (npad each) and the thin products (nt kcap)
  const size_t gd = (sizeof(GemmGen) + 7) / 8;
  const size_t desc = (1 + 2 * (size_t)nt) * gd + 16;
  const size_t per = 2 * (size_t)npad + (size_t)nt * h->kcap;
  if (h->scratch_elems <= desc + per) TLR_RETURN_OOM();
  const int64_t mb = std::min<int64_t>(std::min<int64_t>(m, 1024), (int64_t)((h->scratch_elems - desc) / per));
  GemmGen* d0 = (GemmGen*)h->scratch;
  GemmGen* d1 = (GemmGen*)(h->scratch + gd);
  GemmGen* d2 = (GemmGen*)(h->scratch + (1 + (size_t)nt) * gd);
  double* C = h->scratch + desc;
  double* W = C + (size_t)npad * mb;
  double* Tb = W + (size_t)npad * mb;
  const TlrView v = view_of(h);
  for (int64_t j0 = 0; j0 < m; j0 += mb) {
    const int cnt = (int)std::min<int64_t>(mb, m - j0);
    k_cov_block<<<dim3((unsigned)std::min<int64_t>((npad + 255) / 256, 64), (unsigned)cnt), 256, 0, s>>>(
        h->tab, h->mp, h->x, h->y, h->n, npad, xn + j0, yn + j0, C, npad);
    TLR_LAUNCH_CHECK();
    for (int k = 0; k < nt; ++k) {
      const int rows = nt - k - 1;
      k_msolve_desc<<<(unsigned)(rows / 128 + 1), 128, 0, s>>>(v, k, h->linv + (size_t)k * nn, cnt, C, W, npad, Tb,
                                                                d0, d1, d2);
      TLR_LAUNCH_CHECK();
      TRY_RC(tops_gemm(d0, 1, nb, cnt, s));
      if (rows > 0) {
        TRY_RC(tops_gemm(d1, rows, h->kcap, cnt, s));
        TRY_RC(tops_gemm(d2, rows, nb, cnt, s));
      }
    }
    k_colvar<<<(unsigned)cnt, 256, 0, s>>>(W, npad, npad, h->mp.sigma2, var + j0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}
