// Low-rank tile kernels (Sec. V and the TLR Cholesky updates).
//
//  * k_aca_compress: one CTA per off-diagonal tile.  Adaptive cross
//    approximation with partial pivoting generates only the rows and columns
//    it pivots on (each a row/column of Sigma_ij from the Matérn table),
//    stopping once two successive rank-one terms have ||u|| ||v|| <= eps / 8,
//    then recompresses the cross factors to the eps-truncated SVD.
//  * k_lr_update: one CTA per tile (i, j), i > j > k, of panel step k:
//    A_ij <- trunc_eps([U_ij, -U_ik W] [V_ij, U_jk]^T), W = V_ik^T V_jk
//    (or the mirrored grouping when k_ik < k_jk), the TLR GEMM of Sec. VIII-C.
//  * recompression (cta_recompress): Householder QR of both factors, product
//    of the triangular factors, one-sided Jacobi SVD of that core, keep the
//    singular values > eps, apply the orthogonal factors back.
#include "common.cuh"

namespace {

struct ItemWs {  // per-item workspace layout (doubles)
  double* Up;    // nb x Kmax
  double* Vp;    // nb x Kmax
  double* W;     // kcap x kcap
  double* M;     // Kmax x Kmax
  double* Y;     // Kmax x Kmax
  double* tu;    // Kmax
  double* tv;    // Kmax
  double* s;     // Kmax
};

__device__ __forceinline__ ItemWs item_ws(double* base, size_t item_elems, int slot, int nb, int Kmax, int kcap) {
  ItemWs w;
  double* p = base + (size_t)slot * item_elems;
  w.Up = p; p += (size_t)nb * Kmax;
  w.Vp = p; p += (size_t)nb * Kmax;
  w.W = p; p += (size_t)kcap * kcap;
  w.M = p; p += (size_t)Kmax * Kmax;
  w.Y = p; p += (size_t)Kmax * Kmax;
  w.tu = p; p += Kmax;
  w.tv = p; p += Kmax;
  w.s = p;
  return w;
}

// Householder QR in place (R on/above the diagonal, reflector v below it with v0 = 1)
__device__ void cta_geqr2(double* __restrict__ A, int lda, int m, int K, double* __restrict__ tau, double* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nref = K < m ? K : m;
  for (int c = 0; c < nref; ++c) {
    double* a = A + (size_t)c * lda;
    double p = 0.0;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) p = fma(a[r], a[r], p);
    const double sig = block_sum(p, sh);
    const double alpha = a[c];
    double beta = alpha, tc = 0.0, scal = 1.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
      tc = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    if (sig > 0.0)
      for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) a[r] *= scal;
    __syncthreads();
    if (threadIdx.x == 0) { a[c] = beta; tau[c] = tc; }
    if (tc != 0.0) {
      for (int j = c + 1 + warp; j < K; j += nw) {
        double* b = A + (size_t)j * lda;
        double d = (lane == 0) ? b[c] : 0.0;
        for (int r = c + 1 + lane; r < m; r += 32) d = fma(a[r], b[r], d);
        d = warp_sum(d) * tc;
        if (lane == 0) b[c] -= d;
        for (int r = c + 1 + lane; r < m; r += 32) b[r] = fma(-d, a[r], b[r]);
      }
    }
    __syncthreads();
  }
}

// B <- Q B for Q = H_0 ... H_{K-1} stored by cta_geqr2; B: m x ncol (ld ldb). Warp per column.
__device__ void cta_apply_q(const double* __restrict__ A, int lda, int m, int K, const double* __restrict__ tau,
                            double* __restrict__ B, int ldb, int ncol) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < ncol; j += nw) {
    double* b = B + (size_t)j * ldb;
    for (int c = K - 1; c >= 0; --c) {
      const double tc = tau[c];
      if (tc == 0.0) continue;
      const double* v = A + (size_t)c * lda;
      double d = (lane == 0) ? b[c] : 0.0;
      for (int r = c + 1 + lane; r < m; r += 32) d = fma(v[r], b[r], d);
      d = warp_sum(d) * tc;
      if (lane == 0) b[c] -= d;
      for (int r = c + 1 + lane; r < m; r += 32) b[r] = fma(-d, v[r], b[r]);
    }
  }
}

// round-robin pairing: round rr of K2-1, pair pi of K2/2
__device__ __forceinline__ void rr_pair(int K2, int rr, int pi, int* p, int* q) {
  const int L = K2 - 1;
  auto el = [&](int pos) { return ((pos - rr) % L + L) % L + 1; };
  if (pi == 0) { *p = 0; *q = el(0); }
  else { *p = el(pi); *q = el(L - pi); }
}

// one-sided Jacobi: M (K x K, ld K) <- M Y with orthogonal columns, Y (K x K) accumulated
__device__ void cta_jacobi(double* __restrict__ M, double* __restrict__ Y, int K, int* sh_flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) Y[e] = ((e % K) == (e / K)) ? 1.0 : 0.0;
  __syncthreads();
  if (K < 2) return;
  const int K2 = K + (K & 1);
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) *sh_flag = 0;
    __syncthreads();
    int rotated = 0;
    for (int rr = 0; rr < K2 - 1; ++rr) {
      for (int pi = warp; pi < K2 / 2; pi += nw) {
        int p, q;
        rr_pair(K2, rr, pi, &p, &q);
        if (p >= K || q >= K) continue;
        double* mp = M + (size_t)p * K;
        double* mq = M + (size_t)q * K;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < K; r += 32) {
          const double a = mp[r], b = mq[r];
          al = fma(a, a, al);
          be = fma(b, b, be);
          ga = fma(a, b, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > 0.0 && be > 0.0 && fabs(ga) > 1e-15 * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int r = lane; r < K; r += 32) {
            const double a = mp[r], b = mq[r];
            mp[r] = c * a - s * b;
            mq[r] = s * a + c * b;
          }
          double* yp = Y + (size_t)p * K;
          double* yq = Y + (size_t)q * K;
          for (int r = lane; r < K; r += 32) {
            const double a = yp[r], b = yq[r];
            yp[r] = c * a - s * b;
            yq[r] = s * a + c * b;
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (rotated && lane == 0) atomicOr(sh_flag, 1);
    __syncthreads();
    if (*sh_flag == 0) break;
    __syncthreads();
  }
}

// Recompress Up Vp^T (nb x K each, destroyed) into Uo Vo^T (nb x k, ld nb) with
// singular values > eps.  Returns k (same in all threads).
__device__ int cta_recompress(const ItemWs& w, int nb, int K, double eps, int kcap, int trunc_cap, double* Uo,
                              double* Vo, long long* st, long long info, double* sh, int* shi) {
  if (K == 0) return 0;
  cta_geqr2(w.Up, nb, nb, K, w.tu, sh);
  cta_geqr2(w.Vp, nb, nb, K, w.tv, sh);
  const int Ke = K < nb ? K : nb;  // rows of the trapezoidal R factors
  // M = R_u R_v^T (Ke x Ke)
  for (int e = threadIdx.x; e < Ke * Ke; e += blockDim.x) {
    const int a = e % Ke, b = e / Ke;
    const int c0 = a > b ? a : b;
    double s = 0.0;
    for (int c = c0; c < K; ++c) s = fma(w.Up[(size_t)c * nb + a], w.Vp[(size_t)c * nb + b], s);
    w.M[(size_t)b * Ke + a] = s;
  }
  __syncthreads();
  cta_jacobi(w.M, w.Y, Ke, shi);
  // singular values = column norms of M
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = warp; l < Ke; l += nw) {
    double s = 0.0;
    for (int r = lane; r < Ke; r += 32) s = fma(w.M[(size_t)l * Ke + r], w.M[(size_t)l * Ke + r], s);
    s = warp_sum(s);
    if (lane == 0) w.s[l] = sqrt(s);
  }
  __syncthreads();
  // rank of each kept value in descending order; count kept
  int cnt_local = 0;
  for (int l = threadIdx.x; l < Ke; l += blockDim.x) cnt_local += (w.s[l] > eps);
  const int kept = (int)block_sum((double)cnt_local, sh);
  int k = kept;
  if (k > kcap) {
    if (!trunc_cap) set_status(st, TLR_ERR_RANK_CAP, info);
    k = kcap;
  }
  // output columns: position of l among kept values sorted by (s desc, l asc)
  for (int j = 0; j < k; ++j)
    for (int r = threadIdx.x; r < nb; r += blockDim.x) { Uo[(size_t)j * nb + r] = 0.0; Vo[(size_t)j * nb + r] = 0.0; }
  __syncthreads();
  for (int l = threadIdx.x; l < Ke; l += blockDim.x) {
    const double sl = w.s[l];
    if (!(sl > eps)) continue;
    int pos = 0;
    for (int l2 = 0; l2 < Ke; ++l2) {
      const double s2 = w.s[l2];
      pos += (s2 > sl) || (s2 == sl && l2 < l);
    }
    if (pos < k) {
      for (int r = 0; r < Ke; ++r) {
        Uo[(size_t)pos * nb + r] = w.M[(size_t)l * Ke + r];
        Vo[(size_t)pos * nb + r] = w.Y[(size_t)l * Ke + r];
      }
    }
  }
  __syncthreads();
  cta_apply_q(w.Up, nb, nb, Ke, w.tu, Uo, nb, k);
  cta_apply_q(w.Vp, nb, nb, Ke, w.tv, Vo, nb, k);
  __syncthreads();
  return k;
}

__device__ __forceinline__ void decode_lower(int64_t t, int* i, int* j) {
  int ii = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while ((int64_t)ii * (ii - 1) / 2 > t) --ii;
  while ((int64_t)(ii + 1) * ii / 2 <= t) ++ii;
  *i = ii;
  *j = (int)(t - (int64_t)ii * (ii - 1) / 2);
}

__global__ void k_aca_compress(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                               const double* __restrict__ y, int64_t n, int nb, int64_t t0, double eps, int kcap,
                               int Kmax, int trunc_cap, double* __restrict__ ws, size_t item_elems,
                               double* __restrict__ Ubase, double* __restrict__ Vbase, int* __restrict__ rank,
                               long long* __restrict__ st) {
  extern __shared__ double dsm[];
  double* row = dsm;
  double* col = dsm + nb;
  int* used = (int*)(dsm + 2 * nb);
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  const int64_t t = t0 + blockIdx.x;
  int ti, tj;
  decode_lower(t, &ti, &tj);
  ItemWs w = item_ws(ws, item_elems, blockIdx.x, nb, Kmax, kcap);
  const int64_t pi0 = (int64_t)ti * nb, pj0 = (int64_t)tj * nb;
  const int mi = (int)min((int64_t)nb, n - pi0), mj = (int)min((int64_t)nb, n - pj0);
  for (int a = threadIdx.x; a < nb; a += blockDim.x) used[a] = (a >= mi);
  const double tol = eps * 0.125;
  int istar = 0, k = 0, nsmall = 0;
  __syncthreads();
  while (k < Kmax) {
    // residual row istar
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      double v = 0.0;
      if (b < mj) {
        v = cov_pts(tab, mp, x, y, n, pi0 + istar, pj0 + b);
        for (int l = 0; l < k; ++l) v = fma(-w.Up[(size_t)l * nb + istar], w.Vp[(size_t)l * nb + b], v);
      }
      row[b] = v;
    }
    if (threadIdx.x == 0) used[istar] = 1;
    double rmax;
    double av = -1.0;
    int ai = 0x7fffffff;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double a = fabs(row[b]);
      if (a > av) { av = a; ai = b; }
    }
    const int jstar = block_argmax(av, ai, sh, shi, &rmax);
    if (!(rmax > 0.0) || rmax <= 1e-3 * tol) {
      // zero residual row: try another unused row
      if (++nsmall >= 3) break;
      int nxt = -1;
      // deterministic choice: first unused row after a stride of 97 from istar
      if (threadIdx.x == 0) {
        for (int s2 = 1; s2 <= nb; ++s2) {
          const int cand = (int)(((int64_t)istar + (int64_t)97 * s2) % nb);
          if (!used[cand]) { nxt = cand; break; }
        }
        shi[0] = nxt;
      }
      __syncthreads();
      nxt = shi[0];
      __syncthreads();
      if (nxt < 0) break;
      istar = nxt;
      continue;
    }
    const double delta = row[jstar];
    // residual column jstar
    double pu = 0.0, pv = 0.0;
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      double v = 0.0;
      if (a < mi) {
        v = cov_pts(tab, mp, x, y, n, pi0 + a, pj0 + jstar);
        for (int l = 0; l < k; ++l) v = fma(-w.Vp[(size_t)l * nb + jstar], w.Up[(size_t)l * nb + a], v);
      }
      col[a] = v;
      w.Up[(size_t)k * nb + a] = v;
      const double rv = row[a] / delta;
      w.Vp[(size_t)k * nb + a] = rv;
      pu = fma(v, v, pu);
      pv = fma(rv, rv, pv);
    }
    const double nu2 = block_sum(pu, sh);
    const double nv2 = block_sum(pv, sh);
    ++k;
    if (sqrt(nu2 * nv2) <= tol) {
      if (++nsmall >= 2) break;
    } else {
      nsmall = 0;
    }
    // next pivot row: largest |col| among unused rows
    av = -1.0;
    ai = 0x7fffffff;
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      if (!used[a]) {
        const double v = fabs(col[a]);
        if (v > av) { av = v; ai = a; }
      }
    }
    double cm;
    const int nxt = block_argmax(av, ai, sh, shi, &cm);
    if (cm < 0.0) break;  // every row used
    istar = nxt;
  }
  if (k >= Kmax && nsmall < 2) {
    if (!trunc_cap) set_status(st, TLR_ERR_RANK_CAP, t);
  }
  __syncthreads();
  const size_t slot = (size_t)nb * kcap;
  const int kr = cta_recompress(w, nb, k, eps, kcap, trunc_cap, Ubase + t * slot, Vbase + t * slot, st, t, sh, shi);
  if (threadIdx.x == 0) rank[t] = kr;
}

// TLR GEMM of panel step k for items q0 .. q0+gridDim.x-1 of the trailing lower triangle
__global__ void k_lr_update(int nb, int nt, int k, int64_t q0, double eps, int kcap, int Kmax, int trunc_cap,
                            double* __restrict__ ws, size_t item_elems, double* __restrict__ Ubase,
                            double* __restrict__ Vbase, int* __restrict__ rank, long long* __restrict__ st) {
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  int ip, jp;
  decode_lower(q0 + blockIdx.x, &ip, &jp);  // ip > jp >= 0 in the trailing (nt-k-1)^2 block
  const int i = k + 1 + ip, j = k + 1 + jp;
  const size_t slot = (size_t)nb * kcap;
  const int64_t tij = dtile_index(i, j), tik = dtile_index(i, k), tjk = dtile_index(j, k);
  const int k0 = rank[tij], k1 = rank[tik], k2 = rank[tjk];
  if (k1 == 0 || k2 == 0) return;
  ItemWs w = item_ws(ws, item_elems, blockIdx.x, nb, Kmax, kcap);
  const double* Uik = Ubase + tik * slot;
  const double* Vik = Vbase + tik * slot;
  const double* Ujk = Ubase + tjk * slot;
  const double* Vjk = Vbase + tjk * slot;
  double* Uij = Ubase + tij * slot;
  double* Vij = Vbase + tij * slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // W = V_ik^T V_jk (k1 x k2)
  for (int e = warp; e < k1 * k2; e += nw) {
    const int a = e % k1, b = e / k1;
    double s = 0.0;
    for (int r = lane; r < nb; r += 32) s = fma(Vik[(size_t)a * nb + r], Vjk[(size_t)b * nb + r], s);
    s = warp_sum(s);
    if (lane == 0) w.W[(size_t)b * k1 + a] = s;
  }
  // copy current factors of (i, j)
  for (size_t e = threadIdx.x; e < (size_t)nb * k0; e += blockDim.x) { w.Up[e] = Uij[e]; w.Vp[e] = Vij[e]; }
  __syncthreads();
  int K;
  if (k2 <= k1) {  // [U_ij, -U_ik W] [V_ij, U_jk]^T
    for (size_t e = threadIdx.x; e < (size_t)nb * k2; e += blockDim.x) {
      const int r = (int)(e % nb), c = (int)(e / nb);
      double s = 0.0;
      for (int l = 0; l < k1; ++l) s = fma(Uik[(size_t)l * nb + r], w.W[(size_t)c * k1 + l], s);
      w.Up[(size_t)(k0 + c) * nb + r] = -s;
      w.Vp[(size_t)(k0 + c) * nb + r] = Ujk[(size_t)c * nb + r];
    }
    K = k0 + k2;
  } else {  // [U_ij, -U_ik] [V_ij, U_jk W^T]^T
    for (size_t e = threadIdx.x; e < (size_t)nb * k1; e += blockDim.x) {
      const int r = (int)(e % nb), c = (int)(e / nb);
      double s = 0.0;
      for (int l = 0; l < k2; ++l) s = fma(Ujk[(size_t)l * nb + r], w.W[(size_t)l * k1 + c], s);
      w.Up[(size_t)(k0 + c) * nb + r] = -Uik[(size_t)c * nb + r];
      w.Vp[(size_t)(k0 + c) * nb + r] = s;
    }
    K = k0 + k1;
  }
  __syncthreads();
  const int kr = cta_recompress(w, nb, K, eps, kcap, trunc_cap, Uij, Vij, st, tij, sh, shi);
  if (threadIdx.x == 0) rank[tij] = kr;
}

}  // namespace

static size_t item_elems_for(int nb, int kcap) {
  const size_t Kmax = 2 * (size_t)kcap;
  return 2 * (size_t)nb * Kmax + (size_t)kcap * kcap + 2 * Kmax * Kmax + 3 * Kmax;
}

size_t tlr_item_elems(int nb, int kcap) { return item_elems_for(nb, kcap); }

int tlr_compress_tiles(tlr_ctx* h, double eps, cudaStream_t s) {
  const int nb = h->nb, kcap = h->kcap, Kmax = 2 * kcap;
  const size_t ie = item_elems_for(nb, kcap);
  int chunk = (int)(h->scratch_elems / ie);
  if (chunk > 65535) chunk = 65535;
  if (chunk < 1) return TLR_ERR_OOM;
  const size_t smem = 2 * (size_t)nb * sizeof(double) + (size_t)nb * sizeof(int);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_aca_compress, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int64_t t0 = 0; t0 < h->ntiles; t0 += chunk) {
    const int cnt = (int)((h->ntiles - t0) < chunk ? (h->ntiles - t0) : chunk);
    k_aca_compress<<<cnt, TLR_THREADS, smem, s>>>(h->tab, h->mp, h->x, h->y, h->n, nb, t0, eps, kcap, Kmax,
                                                   h->opts.truncate_at_cap, h->scratch, ie, h->U, h->V, h->rank,
                                                   h->d_stat);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

int tlr_launch_lr_update(tlr_ctx* h, int k, cudaStream_t s) {
  const int m = h->nt - k - 1;
  const int64_t items = (int64_t)m * (m - 1) / 2;
  if (items <= 0) return TLR_OK;
  const int nb = h->nb, kcap = h->kcap, Kmax = 2 * kcap;
  const size_t ie = item_elems_for(nb, kcap);
  int chunk = (int)(h->scratch_elems / ie);
  if (chunk > 65535) chunk = 65535;
  if (chunk < 1) return TLR_ERR_OOM;
  for (int64_t q0 = 0; q0 < items; q0 += chunk) {
    const int cnt = (int)((items - q0) < chunk ? (items - q0) : chunk);
    k_lr_update<<<cnt, TLR_THREADS, 0, s>>>(nb, h->nt, k, q0, h->opts.eps, kcap, Kmax, h->opts.truncate_at_cap,
                                            h->scratch, ie, h->U, h->V, h->rank, h->d_stat);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}
