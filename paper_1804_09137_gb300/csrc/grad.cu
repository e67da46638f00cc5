// Gradient of eq. 1 in theta (not in the paper), from a = Sigma^{-1} z and the
// TLR inverse Z:
//   dl/dtheta_p = 1/2 a^T dSigma_p a - 1/2 tr(Z dSigma_p)
//               = sum_{a > b} (a_a a_b - Z_ab) dC_p(r_ab)      for p = beta, nu
// (dC_beta(0) = dC_nu(0) = 0).  For sigma2, dSigma = Sigma / sigma2 exactly, so
// dl/dsigma2 = (q - n) / (2 sigma2) with q = z^T Sigma^{-1} z (no trace needed).
// One pass over the strictly lower triangle regenerates the three derivative
// entries from the Matérn table (dSigma is never stored) and reads Z's tile:
// dense tiles directly, low-rank tiles as U V^T formed 64 x 64 at a time in
// registers.  Per-CTA partial sums are reduced in a fixed order.
#include "tile.cuh"
#include "df.cuh"

namespace {

// acc = (U[r0:r0+64, :k] V[c0:c0+64, :k]^T) for this thread's 4 x 4 entries
__device__ __forceinline__ void cta_lr_block(const double* __restrict__ U, const double* __restrict__ V, int nb,
                                             int k, int r0, int c0, double acc[4][4]) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int k0 = 0; k0 < k; k0 += 16) {
    __syncthreads();
    for (int id = threadIdx.x; id < 64 * 16; id += 256) {
      const int a = id & 63, kk = id >> 6;
      const int kc = k0 + kk;
      As[kk][a] = (r0 + a < nb && kc < k) ? U[(size_t)kc * nb + r0 + a] : 0.0;
      Bs[kk][a] = (c0 + a < nb && kc < k) ? V[(size_t)kc * nb + c0 + a] : 0.0;
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
}

__global__ void k_grad_fused(TlrView z, const double* __restrict__ tab, const MaternParams mp,
                             const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                             const double* __restrict__ al, double* __restrict__ part) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  const int nb = z.nb;
  const int mb = (nb + 63) / 64;
  const int64_t pair = blockIdx.y;  // I(I+1)/2 + J, I >= J
  int I = (int)((sqrt(8.0 * (double)pair + 1.0) - 1.0) * 0.5);
  while ((int64_t)(I + 1) * (I + 2) / 2 <= pair) ++I;
  while ((int64_t)I * (I + 1) / 2 > pair) --I;
  const int J = (int)(pair - (int64_t)I * (I + 1) / 2);
  const int bi = blockIdx.x % mb, bj = blockIdx.x / mb;
  const int r0 = bi * 64, c0 = bj * 64;
  double g1 = 0.0, g2 = 0.0;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool skip = (I == J && r0 + 63 < c0) || ((int64_t)I * nb + r0 >= n) || ((int64_t)J * nb + c0 >= n);
  if (!skip) {
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const double* Zd = nullptr;  // dense source (diagonal or dense tile)
    if (I == J) {
      Zd = diagT(z, I);
    } else {
      const int64_t t = dtile_index(I, J);
      if (z.dslot[t] >= 0) Zd = tileA(z, t);
      else cta_lr_block(tileU(z, t), tileV(z, t), nb, z.rank[t], r0, c0, acc);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = r0 + ty + 16 * i;
      const int64_t pa = (int64_t)I * nb + a;
      if (a >= nb || pa >= n) continue;
      const double xa = x[pa], ya = y[pa], wa = al[pa];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = c0 + tx + 16 * j;
        const int64_t pb = (int64_t)J * nb + b;
        if (b >= nb || pb >= n) continue;
        if (I == J && b > a) continue;
        const double zab = Zd ? Zd[(size_t)b * nb + a] : acc[i][j];
        if (I == J && a == b) continue;  // dC_beta(0) = dC_nu(0) = 0
        const double r = pt_dist(mp, xa, ya, x[pb], y[pb]);
        const double w = wa * al[pb] - zab;
        if (r > 0.0) {
          double t;
          const int jt = tab_locate(r, mp.e_lo, &t);
          if (jt >= 0 && jt < TAB_NINT) {  // below the table the derivatives vanish
            g1 = fma(w, tab_poly(tab + (size_t)(TAB_NINT + jt) * TAB_NC, t), g1);
            g2 = fma(w, tab_poly(tab + (size_t)(2 * TAB_NINT + jt) * TAB_NC, t), g2);
          }
        }
      }
    }
  }
  g1 = block_sum(g1, sh);
  g2 = block_sum(g2, sh);
  if (threadIdx.x == 0) {
    const size_t id = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[3 * id] = 0.0;
    part[3 * id + 1] = g1;
    part[3 * id + 2] = g2;
  }
}

// p(t) of one table interval with the coefficients as double-float pairs (Horner in double-float, about
// 2^-44 relative; the float32 pipe issues 64 times the float64 rate on this GPU)
__device__ __forceinline__ double tab_poly_df(const float2* __restrict__ c, dfloat t) {
  dfloat s = c[TAB_DEG];
#pragma unroll
  for (int d = TAB_DEG - 1; d >= 0; --d) s = df_add(df_mul(s, t), c[d]);
  return df_to_scaled(s, 0);
}

// The same sums over a batch of dense tiles of Z = Sigma^{-1} (the LAUUM's products, nb x nb each,
// column-major, tile t of the batch at Z + t nb^2, target (m, n) = tg[t]): CTA (blk, t) takes the
// 64 x 64 block blk of tile t, thread (row a, column parity) its 32 entries (a, c0 + parity + 2 j), so
// each warp reads 32 consecutive rows of one column.  The partial pair goes to part[2 (slot0 + t mb^2 +
// blk)], written even for a block with nothing to add.  The derivative polynomials run in double-float
// (coefficient pairs tabf), the distance, the weights and the sums in float64.
__global__ void __launch_bounds__(128) k_grad_tiles(const int2* __restrict__ tg, const double* __restrict__ Z, int nb,
                                                    int64_t slot0, const float2* __restrict__ tabf,
                                                    const MaternParams mp, const double* __restrict__ x,
                                                    const double* __restrict__ y, int64_t n,
                                                    const double* __restrict__ al, double* __restrict__ part) {
  __shared__ double sh[4][2];
  const int mb = (nb + 63) / 64;
  const int t = blockIdx.y;
  const int2 mn = tg[t];
  const int bi = blockIdx.x % mb, bj = blockIdx.x / mb;
  const int r0 = bi * 64, c0 = bj * 64;
  const bool diag = mn.x == mn.y;
  double g1 = 0.0, g2 = 0.0;
  const int a = r0 + (threadIdx.x & 63);
  const int64_t pa = (int64_t)mn.x * nb + a;
  if (!(diag && r0 + 63 < c0) && a < nb && pa < n) {
    const double* Zt = Z + (size_t)t * nb * nb;
    const double xa = x[pa], ya = y[pa], wa = al[pa];
    for (int j = 0; j < 32; ++j) {
      const int b = c0 + (threadIdx.x >> 6) + 2 * j;
      const int64_t pb = (int64_t)mn.y * nb + b;
      if (b >= nb || pb >= n || (diag && b >= a)) continue;  // dC_beta(0) = dC_nu(0) = 0
      const double r = pt_dist(mp, xa, ya, x[pb], y[pb]);
      if (!(r > 0.0)) continue;
      double tt;
      const int jt = tab_locate(r, mp.e_lo, &tt);
      if (jt < 0 || jt >= TAB_NINT) continue;  // below the table the derivatives vanish
      const double w = wa * al[pb] - Zt[(size_t)b * nb + a];
      const dfloat td = df_from_scaled(tt, 0);
      g1 = fma(w, tab_poly_df(tabf + (size_t)(TAB_NINT + jt) * TAB_NC, td), g1);
      g2 = fma(w, tab_poly_df(tabf + (size_t)(2 * TAB_NINT + jt) * TAB_NC, td), g2);
    }
  }
  g1 = warp_sum(g1);
  g2 = warp_sum(g2);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[warp][0] = g1; sh[warp][1] = g2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < 4; ++i) { s1 += sh[i][0]; s2 += sh[i][1]; }
    double* p = part + 2 * (slot0 + (int64_t)t * mb * mb + blockIdx.x);
    p[0] = s1;
    p[1] = s2;
  }
}

__global__ void k_sum3_stage(const double* __restrict__ part, int64_t cnt, double* __restrict__ out) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int64_t per = (cnt + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(cnt, b0 + per);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    s0 += part[3 * i]; s1 += part[3 * i + 1]; s2 += part[3 * i + 2];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) { out[3 * blockIdx.x] = s0; out[3 * blockIdx.x + 1] = s1; out[3 * blockIdx.x + 2] = s2; }
}

__global__ void k_sum2_stage(const double* __restrict__ part, int64_t cnt, double* __restrict__ out) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  double s0 = 0.0, s1 = 0.0;
  const int64_t per = (cnt + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(cnt, b0 + per);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) { out[2 * blockIdx.x] = s0; out[2 * blockIdx.x + 1] = s1; }
}

}  // namespace

int tlr_sum_pairs(const double* part, int64_t count, double* out2, double* ws, cudaStream_t s) {
  const int nstage = 256;
  k_sum2_stage<<<nstage, TLR_THREADS, 0, s>>>(part, count, ws);
  TLR_LAUNCH_CHECK();
  k_sum2_stage<<<1, TLR_THREADS, 0, s>>>(ws, nstage, out2);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

// out3 = (dl/dsigma2, dl/dbeta, dl/dnu); alpha = Sigma^{-1} z in sorted order
int tlr_grad_fused(tlr_ctx* h, const double* alpha, double* out3, cudaStream_t s) {
  TlrView z;
  z.nb = h->nb; z.nt = h->nt; z.kcap = h->kcap;
  z.D = h->Dz; z.U = h->Uz; z.V = h->Vz; z.rank = h->rankz; z.dslot = h->dslotz; z.dpool = h->dpoolz;
  z.off = h->offz; z.cap = h->capz; z.top = h->topz; z.arena = h->arenaz;
  const int mb = (h->nb + 63) / 64;
  const int64_t pairs = (int64_t)h->nt * (h->nt + 1) / 2;
  const int64_t cnt = pairs * mb * mb;
  const int nstage = 256;
  if ((size_t)(3 * cnt + 3 * nstage) > h->scratch_elems) TLR_RETURN_OOM();
  double* part = h->scratch;
  double* stage = h->scratch + 3 * cnt;
  if (pairs > 65535) return TLR_ERR_STATE;  // nt up to 361
  k_grad_fused<<<dim3(mb * mb, (unsigned)pairs), TLR_THREADS, 0, s>>>(z, h->tab, h->mp, h->x, h->y, h->n, alpha,
                                                                      part);
  TLR_LAUNCH_CHECK();
  k_sum3_stage<<<nstage, TLR_THREADS, 0, s>>>(part, cnt, stage);
  TLR_LAUNCH_CHECK();
  k_sum3_stage<<<1, TLR_THREADS, 0, s>>>(stage, nstage, out3);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

int tlr_grad_tiles(const tlr_ctx* h, const int2* tg, int cnt, const double* Z, int64_t slot0, const double* alpha,
                   double* part, cudaStream_t s) {
  if (cnt <= 0) return TLR_OK;
  if (cnt > 65535 || !h->tabf) return TLR_ERR_STATE;
  const int mb = (h->nb + 63) / 64;
  k_grad_tiles<<<dim3(mb * mb, cnt), 128, 0, s>>>(tg, Z, h->nb, slot0, h->tabf, h->mp, h->x, h->y, h->n, alpha, part);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}
