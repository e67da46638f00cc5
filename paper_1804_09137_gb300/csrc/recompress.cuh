// Low-rank recompression core shared by the factor and inverse kernels.
//
// cta_recompress(Up, Vp, K) replaces the rank-K product Up Vp^T (nb x K
// factors) by an eps-truncated rank-revealing factorization: Householder QR of
// both factors (double-float), the small core M = R_u R_v^T, column-pivoted QR of
// M stopped when the trailing block's Frobenius norm is <= eps (spectral error
// <= eps), and both orthogonal factors applied back into tile t's block of the
// rank-packed arenas.  One CTA of 256 threads per tile; workspace in global memory (L2).
#pragma once
#include "df.cuh"
#include "tile.cuh"

namespace {

struct ItemWs {  // per-item workspace layout (doubles)
  double* Up;    // nb x Kmax (float64 input; double-float after the QR starts)
  double* Vp;    // nb x Kmax
  dfloat* Uq;    // nb x Kmax double-float output buffers
  dfloat* Vq;
  double* W;     // kcap x kcap
  double* M;     // Kmax x Kmax
  double* Y;     // Kmax x Kmax
  double* tu;    // Kmax
  double* tv;    // Kmax
  double* s;     // Kmax
  int* eu;       // Kmax column scale exponents of Up
  int* ev;       // Kmax column scale exponents of Vp
  dfloat* vs;    // shared memory: two staged reflectors, 2 nb (the kernel's dynamic shared memory)
};

__device__ __forceinline__ ItemWs item_ws(double* base, size_t item_elems, int slot, int nb, int Kmax, int kcap) {
  ItemWs w;
  double* p = base + (size_t)slot * item_elems;
  w.Up = p; p += (size_t)nb * Kmax;
  w.Vp = p; p += (size_t)nb * Kmax;
  w.Uq = (dfloat*)p; p += (size_t)nb * Kmax;
  w.Vq = (dfloat*)p; p += (size_t)nb * Kmax;
  w.W = p; p += (size_t)kcap * kcap;
  w.M = p; p += (size_t)Kmax * Kmax;
  w.Y = p; p += (size_t)Kmax * Kmax;
  w.tu = p; p += Kmax;
  w.tv = p; p += Kmax;
  w.s = p; p += Kmax;
  w.eu = (int*)p;
  w.ev = w.eu + Kmax;
  w.vs = nullptr;
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

// sum_{r = r0 + lane, step 32} a[r] b[r] over r < m as a double-float, four
// independent Dot2 accumulators so that several loads are in flight per lane
__device__ __forceinline__ dfloat df_col_dot(const dfloat* __restrict__ a, const dfloat* __restrict__ b, int r0,
                                             int m, int lane) {
  float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f, s3 = 0.f, e3 = 0.f;
  int r = r0 + lane;
  for (; r + 96 < m; r += 128) {
    const dfloat a0 = a[r], b0 = b[r], a1 = a[r + 32], b1 = b[r + 32];
    const dfloat a2 = a[r + 64], b2 = b[r + 64], a3 = a[r + 96], b3 = b[r + 96];
    df_dot_add(s0, e0, a0, b0);
    df_dot_add(s1, e1, a1, b1);
    df_dot_add(s2, e2, a2, b2);
    df_dot_add(s3, e3, a3, b3);
  }
  for (; r < m; r += 32) df_dot_add(s0, e0, a[r], b[r]);
  return df_add(df_add(df_norm(s0, e0), df_norm(s1, e1)), df_add(df_norm(s2, e2), df_norm(s3, e3)));
}

// b[r] -= d a[r] for r = r0 + lane, step 32, r < m
__device__ __forceinline__ void df_col_axpy(dfloat* __restrict__ b, dfloat d, const dfloat* __restrict__ a, int r0,
                                            int m, int lane) {
  int r = r0 + lane;
  for (; r + 96 < m; r += 128) {
    const dfloat a0 = a[r], b0 = b[r], a1 = a[r + 32], b1 = b[r + 32];
    const dfloat a2 = a[r + 64], b2 = b[r + 64], a3 = a[r + 96], b3 = b[r + 96];
    b[r] = df_sub_prod(b0, d, a0);
    b[r + 32] = df_sub_prod(b1, d, a1);
    b[r + 64] = df_sub_prod(b2, d, a2);
    b[r + 96] = df_sub_prod(b3, d, a3);
  }
  for (; r < m; r += 32) b[r] = df_sub_prod(b[r], d, a[r]);
}

// Householder QR in place in double-float storage A (m x K, ld lda): R on and
// above the diagonal, reflector v below it (v0 = 1), tau[c] in float64.  The
// scalars of each reflector are formed in float64 from double-float sums.
__device__ void cta_geqr2_df(dfloat* __restrict__ A, int lda, int m, int K, double* __restrict__ tau, double* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nref = K < m ? K : m;
  __shared__ dfloat sc_tau, sc_scal;
  __shared__ int sc_on;
  for (int c = 0; c < nref; ++c) {
    dfloat* a = A + (size_t)c * lda;
    float ps = 0.f, pc = 0.f;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) df_dot_add(ps, pc, a[r], a[r]);
    const double sig = block_sum((double)ps + (double)pc, sh);
    if (threadIdx.x == 0) {  // the reflector's scalars, once per column, in float64
      const double alpha = df_to(a[c]);
      double beta = alpha, tc = 0.0, scal = 1.0;
      if (sig > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
        tc = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      sc_on = sig > 0.0;
      sc_tau = df_from(tc);
      sc_scal = df_from(scal);
      tau[c] = tc;
      a[c] = df_from(beta);
    }
    __syncthreads();
    const int on = sc_on;
    const dfloat tcd = sc_tau, scd = sc_scal;
    if (on)
      for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) a[r] = df_mul(a[r], scd);
    __syncthreads();
    if (on) {
      for (int j = c + 1 + warp; j < K; j += nw) {
        dfloat* b = A + (size_t)j * lda;
        const dfloat bc = b[c];
        const dfloat d = df_mul(df_add(df_warp_sum(df_col_dot(a, b, c + 1, m, lane)), bc), tcd);
        if (lane == 0) b[c] = df_add(bc, make_float2(-d.x, -d.y));
        df_col_axpy(b, d, a, c + 1, m, lane);
      }
    }
    __syncthreads();
  }
}

// Householder QR of two m x K double-float matrices in lockstep (A1 -> tau1, A2 -> tau2), same
// arithmetic per column as cta_geqr2_df: the squared norms are reduced in double-float, the two
// reflectors' scalars are formed by two threads at once, and the scaled reflectors are staged in
// shared memory (vs: 2 m double-floats) for the trailing columns of both matrices, which all warps share.
__device__ void cta_geqr2_pair_df(dfloat* __restrict__ A1, double* __restrict__ tau1, dfloat* __restrict__ A2,
                                  double* __restrict__ tau2, int lda, int m, int K, dfloat* __restrict__ vs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nref = K < m ? K : m;
  __shared__ dfloat sc_tau[2], sc_scal[2], red[2][TLR_MAX_WARPS];
  __shared__ int sc_on[2];
  for (int c = 0; c < nref; ++c) {
    dfloat* a1 = A1 + (size_t)c * lda;
    dfloat* a2 = A2 + (size_t)c * lda;
    float ps1 = 0.f, pc1 = 0.f, ps2 = 0.f, pc2 = 0.f;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
      df_dot_add(ps1, pc1, a1[r], a1[r]);
      df_dot_add(ps2, pc2, a2[r], a2[r]);
    }
    const dfloat s1 = df_warp_sum(df_norm(ps1, pc1)), s2 = df_warp_sum(df_norm(ps2, pc2));
    if (lane == 0) { red[0][warp] = s1; red[1][warp] = s2; }
    __syncthreads();
    if (threadIdx.x == 0 || threadIdx.x == 32) {  // the reflectors' scalars, in float64
      const int side = threadIdx.x == 0 ? 0 : 1;
      dfloat t = red[side][0];
      for (int q = 1; q < nw; ++q) t = df_add(t, red[side][q]);
      const double sig = df_to(t);
      dfloat* a = side ? a2 : a1;
      const double alpha = df_to(a[c]);
      double beta = alpha, tc = 0.0, scal = 1.0;
      if (sig > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
        tc = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      sc_on[side] = sig > 0.0;
      sc_tau[side] = df_from(tc);
      sc_scal[side] = df_from(scal);
      (side ? tau2 : tau1)[c] = tc;
      a[c] = df_from(beta);
    }
    __syncthreads();
    const int on1 = sc_on[0], on2 = sc_on[1];
    const dfloat sc1 = sc_scal[0], sc2 = sc_scal[1];
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
      const dfloat v1 = on1 ? df_mul(a1[r], sc1) : a1[r];
      const dfloat v2 = on2 ? df_mul(a2[r], sc2) : a2[r];
      a1[r] = v1;
      a2[r] = v2;
      vs[r] = v1;
      vs[m + r] = v2;
    }
    __syncthreads();
    const int n1 = on1 ? K - c - 1 : 0, n2 = on2 ? K - c - 1 : 0;
    for (int jj = warp; jj < n1 + n2; jj += nw) {
      const int side = jj < n1 ? 0 : 1;
      const int j = c + 1 + (side ? jj - n1 : jj);
      dfloat* b = (side ? A2 : A1) + (size_t)j * lda;
      const dfloat* v = vs + (size_t)side * m;
      const dfloat bc = b[c];
      const dfloat d = df_mul(df_add(df_warp_sum(df_col_dot(v, b, c + 1, m, lane)), bc), sc_tau[side]);
      if (lane == 0) b[c] = df_add(bc, make_float2(-d.x, -d.y));
      df_col_axpy(b, d, v, c + 1, m, lane);
    }
    __syncthreads();
  }
}

// B1 <- Q1 B1 and B2 <- Q2 B2 (double-float), Qi = H_0 ... H_{K-1} from cta_geqr2_df (reflectors Ai,
// taus ti), ncol columns each: reflector by reflector (staged in shared memory, vs: 2 m double-floats),
// every warp taking columns of either side, so both sides share the warps
__device__ void cta_apply_q2_df(const dfloat* __restrict__ A1, const double* __restrict__ t1, dfloat* __restrict__ B1,
                                const dfloat* __restrict__ A2, const double* __restrict__ t2, dfloat* __restrict__ B2,
                                int lda, int m, int K, int ldb, int ncol, dfloat* __restrict__ vs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = K - 1; c >= 0; --c) {
    const double tc1 = t1[c], tc2 = t2[c];
    if (tc1 == 0.0 && tc2 == 0.0) continue;
    __syncthreads();  // the previous reflectors' readers are done
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
      vs[r] = A1[(size_t)c * lda + r];
      vs[m + r] = A2[(size_t)c * lda + r];
    }
    __syncthreads();
    const dfloat td1 = df_from_scaled(tc1, 0), td2 = df_from_scaled(tc2, 0);
    for (int jj = warp; jj < 2 * ncol; jj += nw) {
      const bool first = jj < ncol;
      if ((first ? tc1 : tc2) == 0.0) continue;
      dfloat* b = (first ? B1 : B2) + (size_t)(first ? jj : jj - ncol) * ldb;
      const dfloat* v = vs + (first ? 0 : m);
      const dfloat bc = b[c];
      const dfloat d = df_mul(df_add(df_warp_sum(df_col_dot(v, b, c + 1, m, lane)), bc), first ? td1 : td2);
      if (lane == 0) b[c] = df_add(bc, make_float2(-d.x, -d.y));
      df_col_axpy(b, d, v, c + 1, m, lane);
    }
  }
  __syncthreads();
}

// One matrix of cta_geqr2_pair_df (the same arithmetic): Householder QR in place of an m x K
// double-float matrix, the scaled reflector staged in shared memory vs (m double-floats) for the
// trailing columns.  Used when the two factors of a recompression run on the two CTAs of a cluster.
__device__ void cta_geqr2_one_df(dfloat* __restrict__ A, double* __restrict__ tau, int lda, int m, int K,
                                 dfloat* __restrict__ vs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nref = K < m ? K : m;
  __shared__ dfloat sc_tau, sc_scal, red[TLR_MAX_WARPS];
  __shared__ int sc_on;
  for (int c = 0; c < nref; ++c) {
    dfloat* a = A + (size_t)c * lda;
    float ps = 0.f, pc = 0.f;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) df_dot_add(ps, pc, a[r], a[r]);
    const dfloat s1 = df_warp_sum(df_norm(ps, pc));
    if (lane == 0) red[warp] = s1;
    __syncthreads();
    if (threadIdx.x == 0) {  // the reflector's scalars, in float64
      dfloat t = red[0];
      for (int q = 1; q < nw; ++q) t = df_add(t, red[q]);
      const double sig = df_to(t);
      const double alpha = df_to(a[c]);
      double beta = alpha, tc = 0.0, scal = 1.0;
      if (sig > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
        tc = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      sc_on = sig > 0.0;
      sc_tau = df_from(tc);
      sc_scal = df_from(scal);
      tau[c] = tc;
      a[c] = df_from(beta);
    }
    __syncthreads();
    const int on = sc_on;
    const dfloat sc = sc_scal;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
      const dfloat v1 = on ? df_mul(a[r], sc) : a[r];
      a[r] = v1;
      vs[r] = v1;
    }
    __syncthreads();
    const int n1 = on ? K - c - 1 : 0;
    for (int jj = warp; jj < n1; jj += nw) {
      dfloat* b = A + (size_t)(c + 1 + jj) * lda;
      const dfloat bc = b[c];
      const dfloat d = df_mul(df_add(df_warp_sum(df_col_dot(vs, b, c + 1, m, lane)), bc), sc_tau);
      if (lane == 0) b[c] = df_add(bc, make_float2(-d.x, -d.y));
      df_col_axpy(b, d, vs, c + 1, m, lane);
    }
    __syncthreads();
  }
}

// One matrix of cta_apply_q2_df: B <- Q B (double-float, ncol columns), Q = H_0 ... H_{K-1} from
// cta_geqr2_one_df (reflectors A, taus t), reflector by reflector staged in shared memory vs.
__device__ void cta_apply_q_one_df(const dfloat* __restrict__ A, const double* __restrict__ t, dfloat* __restrict__ B,
                                   int lda, int m, int K, int ldb, int ncol, dfloat* __restrict__ vs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = K - 1; c >= 0; --c) {
    const double tc = t[c];
    if (tc == 0.0) continue;
    __syncthreads();  // the previous reflector's readers are done
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) vs[r] = A[(size_t)c * lda + r];
    __syncthreads();
    const dfloat td = df_from_scaled(tc, 0);
    for (int jj = warp; jj < ncol; jj += nw) {
      dfloat* b = B + (size_t)jj * ldb;
      const dfloat bc = b[c];
      const dfloat d = df_mul(df_add(df_warp_sum(df_col_dot(vs, b, c + 1, m, lane)), bc), td);
      if (lane == 0) b[c] = df_add(bc, make_float2(-d.x, -d.y));
      df_col_axpy(b, d, vs, c + 1, m, lane);
    }
  }
  __syncthreads();
}

// C[0:m, 0:n] = beta C + alpha op(A) op(B) (op(X) = X^T when tX), column-major, in 64 x 64
// blocks blk0, blk0 + nblk_step, ... (lower_only: blocks on or below the diagonal), with the
// products accumulated in double-float (Dot2) on the float32 pipe; inputs are
// split to double-float as they are staged in shared memory.
__device__ __forceinline__ void cta_gemm_df_blocks(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                   int lda, int tA, const double* __restrict__ B, int ldb, int tB,
                                                   double beta, double* __restrict__ C, int ldc, int blk0,
                                                   int nblk_step, int lower_only) {
  __shared__ dfloat As[16][64 + 1];
  __shared__ dfloat Bs[16][64 + 1];
  // 256 threads (16 x 16) compute; in larger blocks the other threads only take part in the barriers
  const bool act = threadIdx.x < 256;
  const int tx = threadIdx.x & 15, ty = (threadIdx.x >> 4) & 15;
  const int mb = (m + 63) / 64, nbk = (n + 63) / 64;
  for (int blk = blk0; blk < mb * nbk; blk += nblk_step) {
    const int bi = blk % mb, bj = blk / mb;
    const int r0 = bi * 64, c0 = bj * 64;
    if (lower_only && r0 + 63 < c0) continue;
    float as[4][4], ae[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { as[i][j] = 0.f; ae[i][j] = 0.f; }
    for (int k0 = 0; k0 < k; k0 += 16) {
      __syncthreads();
      for (int id = threadIdx.x; act && id < 64 * 16; id += 256) {
        int a, kk;
        if (!tA) { a = id & 63; kk = id >> 6; } else { kk = id & 15; a = id >> 4; }
        const int ra = r0 + a, kc = k0 + kk;
        double v = 0.0;
        if (ra < m && kc < k) v = tA ? A[(size_t)ra * lda + kc] : A[(size_t)kc * lda + ra];
        As[kk][a] = df_from_scaled(v, 0);
        if (!tB) { kk = id & 15; a = id >> 4; } else { a = id & 63; kk = id >> 6; }
        const int cb = c0 + a, kc2 = k0 + kk;
        double wv = 0.0;
        if (cb < n && kc2 < k) wv = tB ? B[(size_t)kc2 * ldb + cb] : B[(size_t)cb * ldb + kc2];
        Bs[kk][a] = df_from_scaled(wv, 0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 16 && act; ++kk) {
        dfloat av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_dot_add(as[i][j], ae[i][j], av[i], bv[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
        if (act && r < m && c < n && (!lower_only || r >= c)) {
          double* cp = C + (size_t)c * ldc + r;
          const double v = df_to_scaled(df_norm(as[i][j], ae[i][j]), 0);
          *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * v;
        }
      }
  }
  __syncthreads();
}

// The same in 128 x 32 blocks, for results of at most a few dozen columns (a dense tile or a tall
// factor times a thin one): thread (row ty, column tx) of a 32 x 8 grid takes rows ty + 32 i and
// columns tx + 8 j, so a 64-wide block is not mostly padding.
__device__ __forceinline__ void cta_gemm_df_blocks_n32(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                       int lda, int tA, const double* __restrict__ B, int ldb, int tB,
                                                       double beta, double* __restrict__ C, int ldc, int blk0,
                                                       int nblk_step) {
  __shared__ dfloat As[16][128 + 1];
  __shared__ dfloat Bs[16][32 + 1];
  const bool act = threadIdx.x < 256;
  const int ty = threadIdx.x & 31, tx = (threadIdx.x >> 5) & 7;
  const int mb = (m + 127) / 128, nbk = (n + 31) / 32;
  for (int blk = blk0; blk < mb * nbk; blk += nblk_step) {
    const int r0 = (blk % mb) * 128, c0 = (blk / mb) * 32;
    float as[4][4], ae[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { as[i][j] = 0.f; ae[i][j] = 0.f; }
    for (int k0 = 0; k0 < k; k0 += 16) {
      __syncthreads();
      for (int id = threadIdx.x; act && id < 128 * 16; id += 256) {
        int a, kk;
        if (!tA) { a = id & 127; kk = id >> 7; } else { kk = id & 15; a = id >> 4; }
        const int ra = r0 + a, kc = k0 + kk;
        double v = 0.0;
        if (ra < m && kc < k) v = tA ? A[(size_t)ra * lda + kc] : A[(size_t)kc * lda + ra];
        As[kk][a] = df_from_scaled(v, 0);
      }
      for (int id = threadIdx.x; act && id < 32 * 16; id += 256) {
        int b, kk;
        if (!tB) { kk = id & 15; b = id >> 4; } else { b = id & 31; kk = id >> 5; }
        const int cb = c0 + b, kc = k0 + kk;
        double v = 0.0;
        if (cb < n && kc < k) v = tB ? B[(size_t)kc * ldb + cb] : B[(size_t)cb * ldb + kc];
        Bs[kk][b] = df_from_scaled(v, 0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 16 && act; ++kk) {
        dfloat av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 32 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 8 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_dot_add(as[i][j], ae[i][j], av[i], bv[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + ty + 32 * i, c = c0 + tx + 8 * j;
        if (act && r < m && c < n) {
          double* cp = C + (size_t)c * ldc + r;
          const double v = df_to_scaled(df_norm(as[i][j], ae[i][j]), 0);
          *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * v;
        }
      }
  }
  __syncthreads();
}

__device__ __forceinline__ void cta_gemm_df(int m, int n, int k, double alpha, const double* A, int lda, int tA,
                                            const double* B, int ldb, int tB, double beta, double* C, int ldc) {
  cta_gemm_df_blocks(m, n, k, alpha, A, lda, tA, B, ldb, tB, beta, C, ldc, 0, 1, 0);
}

// Thin products of the low-rank updates (ranks k << nb), double-float accumulation.
//
// W[a + b ldw] = alpha sum_r P[r + a nb] Q[r + b nb] for a < ka, b < kb: every warp takes
// 4 x 4 blocks of W with its lanes striding the nb rows (coalesced column reads), then a
// warp reduction per entry; no CTA barrier inside.
__device__ void cta_gemm_tn_thin(int ka, int kb, int nb, double alpha, const double* __restrict__ P,
                                 const double* __restrict__ Q, double* __restrict__ W, int ldw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ba = (ka + 3) >> 2, bb = (kb + 3) >> 2;
  for (int blk = warp; blk < ba * bb; blk += nw) {
    const int a0 = (blk % ba) * 4, b0 = (blk / ba) * 4;
    float s[4][4], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { s[i][j] = 0.f; c[i][j] = 0.f; }
    for (int r = lane; r < nb; r += 32) {
      dfloat pa[4], qb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) pa[i] = (a0 + i < ka) ? df_from_scaled(P[(size_t)(a0 + i) * nb + r], 0) : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 4; ++j) qb[j] = (b0 + j < kb) ? df_from_scaled(Q[(size_t)(b0 + j) * nb + r], 0) : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_dot_add(s[i][j], c[i][j], pa[i], qb[j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const dfloat v = df_warp_sum(df_norm(s[i][j], c[i][j]));
        if (lane == 0 && a0 + i < ka && b0 + j < kb) W[(size_t)(b0 + j) * ldw + a0 + i] = alpha * df_to_scaled(v, 0);
      }
  }
  __syncthreads();
}

// The same with four rows per lane in flight (every load of a group issued before its products):
// for a kernel that has nothing else to hide the load latency behind.
__device__ void cta_gemm_tn_thin4(int ka, int kb, int nb, double alpha, const double* __restrict__ P,
                                  const double* __restrict__ Q, double* __restrict__ W, int ldw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ba = (ka + 3) >> 2, bb = (kb + 3) >> 2;
  for (int blk = warp; blk < ba * bb; blk += nw) {
    const int a0 = (blk % ba) * 4, b0 = (blk / ba) * 4;
    float s[4][4], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { s[i][j] = 0.f; c[i][j] = 0.f; }
    for (int r0 = lane; r0 < nb; r0 += 128) {
      double pv[4][4], qv[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + 32 * u;
#pragma unroll
        for (int i = 0; i < 4; ++i) pv[u][i] = (r < nb && a0 + i < ka) ? P[(size_t)(a0 + i) * nb + r] : 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) qv[u][j] = (r < nb && b0 + j < kb) ? Q[(size_t)(b0 + j) * nb + r] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dfloat pa[4], qb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) pa[i] = df_from_scaled(pv[u][i], 0);
#pragma unroll
        for (int j = 0; j < 4; ++j) qb[j] = df_from_scaled(qv[u][j], 0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_dot_add(s[i][j], c[i][j], pa[i], qb[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const dfloat v = df_warp_sum(df_norm(s[i][j], c[i][j]));
        if (lane == 0 && a0 + i < ka && b0 + j < kb) W[(size_t)(b0 + j) * ldw + a0 + i] = alpha * df_to_scaled(v, 0);
      }
  }
  __syncthreads();
}

// C[r + b nb] = alpha sum_l A[r + l nb] op(W)[l, b] for r < nb, b < kb, depth ka, with op(W)[l, b] =
// W[l + b ldw] (tw = 0) or W[b + l ldw]: a thread per row (two at a time), 8 output columns at a time, op(W) staged as
// double-float in shared memory 64 x 8 at a time.
__device__ void cta_gemm_nn_thin(int nb, int kb, int ka, double alpha, const double* __restrict__ A,
                                 const double* __restrict__ W, int ldw, int tw, double* __restrict__ C) {
  __shared__ dfloat Ws[64][8];
  for (int rb = 0; rb < nb; rb += 2 * blockDim.x) {  // up to 2 rows per thread at a time
    for (int b0 = 0; b0 < kb; b0 += 8) {
      float s[2][8], c[2][8];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) { s[q][j] = 0.f; c[q][j] = 0.f; }
      for (int l0 = 0; l0 < ka; l0 += 64) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 8; e += blockDim.x) {
          const int l = e >> 3, j = e & 7;
          double v = 0.0;
          if (l0 + l < ka && b0 + j < kb)
            v = tw ? W[(size_t)(l0 + l) * ldw + b0 + j] : W[(size_t)(b0 + j) * ldw + l0 + l];
          Ws[l][j] = df_from_scaled(v, 0);
        }
        __syncthreads();
        const int lmax = min(64, ka - l0);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = rb + threadIdx.x + q * blockDim.x;
          if (r >= nb) continue;
          for (int l = 0; l < lmax; ++l) {
            const dfloat a = df_from_scaled(A[(size_t)(l0 + l) * nb + r], 0);
#pragma unroll
            for (int j = 0; j < 8; ++j) df_dot_add(s[q][j], c[q][j], a, Ws[l][j]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = rb + threadIdx.x + q * blockDim.x;
        if (r >= nb) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (b0 + j < kb) C[(size_t)(b0 + j) * nb + r] = alpha * df_to_scaled(df_norm(s[q][j], c[q][j]), 0);
      }
    }
  }
  __syncthreads();
}

// Recompress Up Vp^T (nb x K each, destroyed) into Uo Vo^T (nb x k, ld nb) with
// singular values > eps.  Returns k (same in all threads).
// ---- stages of the recompression (shared by the one-CTA and the two-CTA cluster versions)
// side 0: the U factor (w.Up, exponents w.eu), side 1: the V factor (w.Vp, w.ev).

// scale every column by a power of two so that its largest entry is in [1, 2) and convert it to
// double-float in place: Q is unchanged, R's columns are scaled back below, and the squares formed in
// double-float stay far inside the float32 exponent range
__device__ void rc_scale_side(const ItemWs& w, int nb, int K, int side) {
  double* P = side ? w.Vp : w.Up;
  int* ex = side ? w.ev : w.eu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < K; j += nw) {
    const double* col = P + (size_t)j * nb;
    double mx = 0.0;
    for (int r = lane; r < nb; r += 32) mx = fmax(mx, fabs(col[r]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) ex[j] = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
  }
  __syncthreads();
  dfloat* D = (dfloat*)P;
  for (size_t e = threadIdx.x; e < (size_t)nb * K; e += blockDim.x) D[e] = df_from_scaled(P[e], -ex[e / nb]);
  __syncthreads();
}

// after the QR of a side: its R factor unscaled to float64 (Ke x K, upper trapezoid) into w.Uq (side 0)
// or w.Vq (side 1)
__device__ void rc_extract_r(const ItemWs& w, int nb, int K, int side) {
  const int Ke = K < nb ? K : nb;
  const dfloat* D = (const dfloat*)(side ? w.Vp : w.Up);
  const int* ex = side ? w.ev : w.eu;
  double* R = (double*)(side ? w.Vq : w.Uq);
  for (int e = threadIdx.x; e < Ke * K; e += blockDim.x) {
    const int a = e % Ke, c = e / Ke;
    R[e] = (a <= c) ? df_to_scaled(D[(size_t)c * nb + a], ex[c]) : 0.0;
  }
  __syncthreads();
}

// one CTA, after both R factors are in w.Uq / w.Vq: the core M = R_u R_v^T, its column-pivoted
// Householder QR stopped at the first step whose trailing block has Frobenius norm <= eps (then
// ||M - Q_k R_k P^T||_2 <= eps), the tile's block in the arena, the U block Q_M[:, :k] (into the
// arena, then as double-float into w.Uq) and the V block P R_k^T (double-float, w.Vq).  Returns k
// (0: nothing is written).
__device__ int rc_core(const ItemWs& w, int nb, int K, double eps, int kcap, int trunc_cap, const TlrView& v,
                       int64_t info, long long* st, double* sh, int* shi, double* flops) {
  const int Ke = K < nb ? K : nb;  // rows of the trapezoidal R factors
  double* Ru = (double*)w.Uq;
  double* Rv = (double*)w.Vq;
  for (int e = threadIdx.x; e < Ke * Ke; e += blockDim.x) {
    const int a = e % Ke, b = e / Ke;
    const int c0 = a > b ? a : b;
    double s = 0.0;
    for (int c = c0; c < K; ++c) s = fma(Ru[(size_t)c * Ke + a], Rv[(size_t)c * Ke + b], s);
    w.M[(size_t)b * Ke + a] = s;
  }
  __syncthreads();
  {  // a non-finite core means the inputs were not finite: report, keep rank 0
    int bad = 0;
    for (int e = threadIdx.x; e < Ke * Ke; e += blockDim.x) bad |= !isfinite(w.M[e]);
    if (block_sum((double)bad, sh) > 0.0) {
      if (threadIdx.x == 0) set_status(st, TLR_ERR_NUMERIC, info);
      return 0;
    }
  }
  // column-pivoted Householder QR of M, stopped at the first step whose trailing
  // block has Frobenius norm <= eps (then ||M - Q_k R_k P^T||_2 <= eps)
  double* nrm = w.s;               // partial column norms^2 (rows >= step)
  double* tm = w.Y;                // reflector taus of M
  int* perm = (int*)(w.Y + Ke);    // column permutation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < Ke; j += nw) {
    double q = 0.0;
    for (int r = lane; r < Ke; r += 32) q = fma(w.M[(size_t)j * Ke + r], w.M[(size_t)j * Ke + r], q);
    q = warp_sum(q);
    if (lane == 0) { nrm[j] = q; perm[j] = j; }
  }
  __syncthreads();
  const double eps2 = eps * eps;
  int k = 0;
  double fl = 2.0 * Ke * Ke * (K - 2.0 * Ke / 3.0) + 2.0 * Ke * Ke;
  for (int c = 0; c < Ke; ++c) {
    double part = 0.0, av = -1.0;
    int ai = 0x7fffffff;
    for (int j = c + threadIdx.x; j < Ke; j += blockDim.x) {
      part += nrm[j];
      if (nrm[j] > av) { av = nrm[j]; ai = j; }
    }
    const double trail = block_sum(part, sh);
    if (trail <= eps2) break;
    const int piv = block_argmax(av, ai, sh, shi, nullptr);
    if (piv < c || piv >= Ke) {  // no valid pivot (non-finite norms): stop here
      if (threadIdx.x == 0) set_status(st, TLR_ERR_NUMERIC, info);
      break;
    }
    if (piv != c) {  // swap columns c and piv
      for (int r = threadIdx.x; r < Ke; r += blockDim.x) {
        const double t = w.M[(size_t)c * Ke + r];
        w.M[(size_t)c * Ke + r] = w.M[(size_t)piv * Ke + r];
        w.M[(size_t)piv * Ke + r] = t;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double tn = nrm[c]; nrm[c] = nrm[piv]; nrm[piv] = tn;
        const int tp = perm[c]; perm[c] = perm[piv]; perm[piv] = tp;
      }
    }
    __syncthreads();
    // reflector of column c (rows c..Ke-1); sigma = sum of squares below the diagonal
    double* a = w.M + (size_t)c * Ke;
    const double alpha = a[c];
    double ps = 0.0;
    for (int r = c + 1 + threadIdx.x; r < Ke; r += blockDim.x) ps = fma(a[r], a[r], ps);
    const double sig = block_sum(ps, sh);
    double beta = alpha, tc = 0.0, scal = 1.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sig), alpha);
      tc = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    __syncthreads();
    if (sig > 0.0)
      for (int r = c + 1 + threadIdx.x; r < Ke; r += blockDim.x) a[r] *= scal;
    __syncthreads();
    if (threadIdx.x == 0) { a[c] = beta; tm[c] = tc; }
    // trailing columns: apply the reflector, recompute the partial norms (rows > c) exactly
    for (int j = c + 1 + warp; j < Ke; j += nw) {
      double* b = w.M + (size_t)j * Ke;
      double d = (lane == 0) ? b[c] : 0.0;
      if (tc != 0.0) {
        for (int r = c + 1 + lane; r < Ke; r += 32) d = fma(a[r], b[r], d);
        d = warp_sum(d) * tc;
        if (lane == 0) b[c] -= d;
      }
      double q = 0.0;
      for (int r = c + 1 + lane; r < Ke; r += 32) {
        const double v = (tc != 0.0) ? fma(-d, a[r], b[r]) : b[r];
        b[r] = v;
        q = fma(v, v, q);
      }
      q = warp_sum(q);
      if (lane == 0) nrm[j] = q;
    }
    fl += 6.0 * (Ke - c) * (Ke - c);
    k = c + 1;
    __syncthreads();
  }
  if (k > kcap) {
    if (!trunc_cap) set_status(st, TLR_ERR_RANK_CAP, info);
    k = kcap;
  }
  // the tile's columns in the arena (a new block when k exceeds its reservation)
  if (!cta_lr_reserve(v, info, k, st)) return 0;
  double* Uo = tileU(v, info);
  // U block = Q_M[:, :k] (Ke x k): apply the k reflectors of M to [I_k; 0]
  for (int j = 0; j < k; ++j)
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      Uo[(size_t)j * nb + r] = (r == j) ? 1.0 : 0.0;
      w.Vq[(size_t)j * nb + r] = make_float2(0.f, 0.f);
    }
  __syncthreads();
  cta_apply_q(w.M, Ke, Ke, k, tm, Uo, nb, k);
  __syncthreads();  // Uo columns were written warp by warp; they are read across warps below
  // V block = P R_k^T (Ke x k): row perm[jj] gets R[:k, jj]
  for (int e = threadIdx.x; e < Ke * k; e += blockDim.x) {
    const int jj = e % Ke, c = e / Ke;
    w.Vq[(size_t)c * nb + perm[jj]] = df_from((jj >= c) ? w.M[(size_t)jj * Ke + c] : 0.0);
  }
  for (size_t e = threadIdx.x; e < (size_t)nb * k; e += blockDim.x) w.Uq[e] = df_from_scaled(Uo[e], 0);
  __syncthreads();
  if (flops && threadIdx.x == 0) atomicAdd(flops, fl + 4.0 * Ke * k * k);
  return k;
}

// flops of the QR of one nb x K factor and of applying its Q to k columns
__device__ __forceinline__ double rc_side_flops(int nb, int K, int k) {
  const double m = nb, KK = K, Kq = K < nb ? K : nb;
  return 2.0 * m * KK * Kq - (KK + m) * Kq * Kq + 2.0 * Kq * Kq * Kq / 3.0 + k * (4.0 * m * Kq - 2.0 * Kq * Kq);
}

// the output of a side: Uo (side 0) or Vo (side 1) from the double-float w.Uq / w.Vq
__device__ void rc_store_side(const ItemWs& w, int nb, int k, const TlrView& v, int64_t t, int side) {
  double* O = side ? tileV(v, t) : tileU(v, t);
  const dfloat* Q = side ? w.Vq : w.Uq;
  for (size_t e = threadIdx.x; e < (size_t)nb * k; e += blockDim.x) O[e] = df_to_scaled(Q[e], 0);
  __syncthreads();
}

// Recompression of the rank-K product Up Vp^T by one CTA (see the file's header); both factors in
// lockstep.  Returns the new rank written to tile `info`.
__device__ int cta_recompress(const ItemWs& w, int nb, int K, double eps, int kcap, int trunc_cap, const TlrView& v,
                              int64_t info, long long* st, double* sh, int* shi, double* flops = nullptr) {
  if (K == 0) return 0;
  rc_scale_side(w, nb, K, 0);
  rc_scale_side(w, nb, K, 1);
  dfloat* Ud = (dfloat*)w.Up;
  dfloat* Vd = (dfloat*)w.Vp;
  cta_geqr2_pair_df(Ud, w.tu, Vd, w.tv, nb, nb, K, w.vs);
  rc_extract_r(w, nb, K, 0);
  rc_extract_r(w, nb, K, 1);
  const int k = rc_core(w, nb, K, eps, kcap, trunc_cap, v, info, st, sh, shi, flops);
  if (k == 0) return 0;
  const int Ke = K < nb ? K : nb;
  cta_apply_q2_df(Ud, w.tu, w.Uq, Vd, w.tv, w.Vq, nb, nb, Ke, nb, k, w.vs);
  __syncthreads();
  rc_store_side(w, nb, k, v, info, 0);
  rc_store_side(w, nb, k, v, info, 1);
  if (flops && threadIdx.x == 0) atomicAdd(flops, 2.0 * rc_side_flops(nb, K, k));
  return k;
}


// ---- two CTAs of a cluster on one recompression
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

// an int in the shared memory of cluster CTA `rank` (distributed shared memory)
__device__ __forceinline__ int dsmem_load_int(const int* p, int rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
  return v;
}

// Both CTAs of a cluster call it with the cluster's workspace: the recompression of cta_recompress with the
// U side (scaling, Householder QR, applying Q, storing U) on cluster rank 0 and the V side on rank 1;
// rank 0 also runs the core (rc_core) between two cluster barriers.  The arithmetic is that of
// cta_recompress.  Returns the new rank on both CTAs (s_k: an int of the caller's shared memory).
__device__ int cluster_recompress(const ItemWs& w, int nb, int K, double tau, int kcap, int trunc_cap,
                                  const TlrView& v, int64_t t, long long* st, double* sh, int* shi, double* flops,
                                  int rank, int* s_k) {
  if (K == 0) return 0;
  const int side = rank;  // 0: U, 1: V
  const int Ke = K < nb ? K : nb;
  rc_scale_side(w, nb, K, side);
  cta_geqr2_one_df((dfloat*)(side ? w.Vp : w.Up), side ? w.tv : w.tu, nb, nb, K, w.vs);
  rc_extract_r(w, nb, K, side);
  cluster_sync_all();  // both R factors are in the workspace
  if (rank == 0) {
    const int kr = rc_core(w, nb, K, tau, kcap, trunc_cap, v, t, st, sh, shi, flops);
    if (threadIdx.x == 0) *s_k = kr;
    __syncthreads();
  }
  cluster_sync_all();  // the core's U and V blocks, the arena block and the rank are out
  const int kr = dsmem_load_int(s_k, 0);
  cluster_sync_all();  // rank 1 has read the rank from rank 0's shared memory
  if (kr > 0) {
    cta_apply_q_one_df((const dfloat*)(side ? w.Vp : w.Up), side ? w.tv : w.tu, side ? w.Vq : w.Uq, nb, nb, Ke, nb,
                       kr, w.vs);
    rc_store_side(w, nb, kr, v, t, side);
    if (flops && threadIdx.x == 0) atomicAdd(flops, rc_side_flops(nb, K, kr));
  }
  return kr;
}

// Adaptive cross approximation with partial pivoting of an mi x mj block (rows
// and columns beyond are zero) whose entries come from E(a, b): each step takes
// the residual row at the pivot row, its largest entry as pivot column, the
// residual column there, and the next pivot row where that column is largest
// among unused rows.  Stops (conv = 1) after two successive rank-one terms with
// ||u|| ||v|| <= tol, when the residual rows are zero, or when every row is used;
// conv = 0 when aca_max terms did not suffice.  Factors go to w.Up / w.Vp (float64, for the
// recompression) and to w.Uq / w.Vq as double-float copies: the residual rows and columns subtract the
// terms so far with double-float dot products (the float64 pipe runs at 1/64 of the float32 rate).
// Shared memory: dsm >= 2 nb doubles + nb ints.
template <class E>
__device__ int cta_aca(const E& entry, int nb, int mi, int mj, double tol, int aca_max, const ItemWs& w,
                       double* dsm, double* sh, int* shi, int* conv_out) {
  double* row = dsm;
  double* col = dsm + nb;
  int* used = (int*)(dsm + 2 * nb);
  for (int a = threadIdx.x; a < nb; a += blockDim.x) used[a] = (a >= mi);
  int istar = 0, k = 0, nsmall = 0, conv = 0;
  __syncthreads();
  while (true) {
    if (k >= aca_max) break;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      double val = 0.0;
      if (b < mj) {  // residual row: the sum over the terms so far in double-float (Dot2)
        float s = 0.f, c = 0.f;
        for (int l = 0; l < k; ++l) df_dot_add(s, c, w.Uq[(size_t)l * nb + istar], w.Vq[(size_t)l * nb + b]);
        val = entry(istar, b) - ((double)s + (double)c);
      }
      row[b] = val;
    }
    if (threadIdx.x == 0) used[istar] = 1;
    double av = -1.0, rmax;
    int ai = 0x7fffffff;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double a = fabs(row[b]);
      if (a > av) { av = a; ai = b; }
    }
    const int jstar = block_argmax(av, ai, sh, shi, &rmax);
    if (jstar < 0 || jstar >= nb) { conv = 0; break; }  // non-finite row
    if (!(rmax > 1e-3 * tol)) {  // residual row (numerically) zero: sample another row
      if (++nsmall >= 3) { conv = 1; break; }
      if (threadIdx.x == 0) {
        int nxt = -1;
        for (int s2 = 1; s2 <= nb; ++s2) {
          const int cand = (int)(((int64_t)istar + (int64_t)97 * s2) % nb);
          if (!used[cand]) { nxt = cand; break; }
        }
        shi[0] = nxt;
      }
      __syncthreads();
      const int nxt = shi[0];
      __syncthreads();
      if (nxt < 0) { conv = 1; break; }
      istar = nxt;
      continue;
    }
    const double delta = row[jstar];
    double pu = 0.0, pv = 0.0;
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      double val = 0.0;
      if (a < mi) {  // residual column, likewise
        float s = 0.f, c = 0.f;
        for (int l = 0; l < k; ++l) df_dot_add(s, c, w.Vq[(size_t)l * nb + jstar], w.Uq[(size_t)l * nb + a]);
        val = entry(a, jstar) - ((double)s + (double)c);
      }
      col[a] = val;
      const double rv = row[a] / delta;
      // the new term in float64 (for the recompression) and in double-float (for the residuals)
      w.Up[(size_t)k * nb + a] = val;
      w.Vp[(size_t)k * nb + a] = rv;
      w.Uq[(size_t)k * nb + a] = df_from_scaled(val, 0);
      w.Vq[(size_t)k * nb + a] = df_from_scaled(rv, 0);
      pu = fma(val, val, pu);
      pv = fma(rv, rv, pv);
    }
    const double nu2 = block_sum(pu, sh);
    const double nv2 = block_sum(pv, sh);
    ++k;
    if (sqrt(nu2 * nv2) <= tol) {
      if (++nsmall >= 2) { conv = 1; break; }
    } else {
      nsmall = 0;
    }
    av = -1.0;
    ai = 0x7fffffff;
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      if (!used[a]) {
        const double val = fabs(col[a]);
        if (val > av) { av = val; ai = a; }
      }
    }
    double cm;
    const int nxt = block_argmax(av, ai, sh, shi, &cm);
    if (cm < 0.0) { conv = 1; break; }  // every row used: the cross approximation is exact
    if (nxt < 0 || nxt >= nb) { conv = 0; break; }  // non-finite column
    istar = nxt;
  }
  *conv_out = conv;
  return k;
}

}  // namespace

