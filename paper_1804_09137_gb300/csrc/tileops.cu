// Generic batched tile operations (see tileops.h).
//
// Update of a target tile by a product of two tiles, alpha op(X) op(Y):
//   low-rank X, Y:  U_x (V_x^T U_y) V_y^T, kept as the thinner of the two groupings;
//   dense X:        (op(X) U_y) V_y^T;   dense Y: U_x (op(Y)^T V_x)^T;
//   dense X and Y:  only into dense targets (the plans close the dense set).
// Low-rank targets append the product's factors and recompress (one CTA per
// tile); dense targets get C += P Q^T by batched 64 x 64-block GEMM.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "recompress.cuh"
#include "tcgemm.h"
#include "tileops.h"

namespace {

struct Opnd {
  bool dense;
  const double* A;
  int tA;
  const double* U;
  const double* V;
  int k;
};

// tile (p, q), p > q, as an operand, optionally transposed
__device__ __forceinline__ Opnd operand(const TlrView& v, int p, int q, bool trans) {
  Opnd o;
  const int64_t t = dtile_index(p, q);
  o.dense = v.dslot[t] >= 0;
  if (o.dense) {
    o.A = tileA(v, t); o.tA = trans; o.U = o.V = nullptr; o.k = v.nb;
  } else {
    o.A = nullptr; o.tA = 0;
    o.U = trans ? tileV(v, t) : tileU(v, t);
    o.V = trans ? tileU(v, t) : tileV(v, t);
    o.k = v.rank[t];
  }
  return o;
}

__device__ __forceinline__ void operands(const TlrView& v, int alg, int a, int b, int k, Opnd* X, Opnd* Y,
                                         double* alpha) {
  if (alg == ALG_CHOL) { *X = operand(v, a, k, false); *Y = operand(v, b, k, true); *alpha = -1.0; }
  else { *X = operand(v, a, k, false); *Y = operand(v, k, b, false); *alpha = 1.0; }
}

// one item: target tile += alpha op(X) op(Y), then recompression; w is this CTA's workspace
__device__ void upd_lr_item(const TlrView& v, int alg, int k, int2 it, double tau, int Kmax, int trunc_cap,
                            ItemWs& w, long long* __restrict__ st, double* __restrict__ flops, double* sh,
                            int* shi, const double* __restrict__ pre) {
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  Opnd X, Y;
  double alpha;
  operands(v, alg, it.x, it.y, k, &X, &Y, &alpha);
  if (X.k == 0 || Y.k == 0) return;
  if (X.dense && Y.dense) {
    if (threadIdx.x == 0) set_status(st, TLR_ERR_STATE, tt);
    return;
  }
  const int k0 = v.rank[tt];
  // the concatenated rank must fit the workspace (else the host widens it and repeats the step)
  const int rin = X.dense ? Y.k : (Y.dense ? X.k : min(X.k, Y.k));
  if (k0 + rin > Kmax) {
    if (threadIdx.x == 0) set_status(st, TLR_ST_WIDEN, tt);
    return;
  }
  double* Ut = tileU(v, tt);
  double* Vt = tileV(v, tt);
  for (size_t e = threadIdx.x; e < (size_t)nb * k0; e += blockDim.x) { w.Up[e] = Ut[e]; w.Vp[e] = Vt[e]; }
  double* Un = w.Up + (size_t)k0 * nb;
  double* Vn = w.Vp + (size_t)k0 * nb;
  int r;
  double pf;  // product flops
  if (!X.dense && !Y.dense) {
    pf = 2.0 * nb * X.k * Y.k * 2.0;
    // thin products for small ranks; 64 x 64-blocked ones once the blocks are mostly filled
    const bool thin = X.k <= 48 && Y.k <= 48;
    if (thin) cta_gemm_tn_thin(X.k, Y.k, nb, 1.0, X.V, Y.U, w.W, X.k);  // W = V_x^T U_y
    else cta_gemm_df(X.k, Y.k, nb, 1.0, X.V, nb, 1, Y.U, nb, 0, 0.0, w.W, X.k);
    if (Y.k <= X.k) {
      if (thin) cta_gemm_nn_thin(nb, Y.k, X.k, alpha, X.U, w.W, X.k, 0, Un);  // U_x W
      else cta_gemm_df(nb, Y.k, X.k, alpha, X.U, nb, 0, w.W, X.k, 0, 0.0, Un, nb);
      for (size_t e = threadIdx.x; e < (size_t)nb * Y.k; e += blockDim.x) Vn[e] = Y.V[e];
      r = Y.k;
    } else {
      if (thin) cta_gemm_nn_thin(nb, X.k, Y.k, 1.0, Y.V, w.W, X.k, 1, Vn);  // V_y W^T
      else cta_gemm_df(nb, X.k, Y.k, 1.0, Y.V, nb, 0, w.W, X.k, 1, 0.0, Vn, nb);
      for (size_t e = threadIdx.x; e < (size_t)nb * X.k; e += blockDim.x) Un[e] = alpha * X.U[e];
      r = X.k;
    }
  } else if (X.dense) {  // U part alpha op(X) U_y: staged by the batched GEMM (pre) or formed here
    pf = pre ? 0.0 : 2.0 * nb * nb * Y.k;
    if (pre) for (size_t e = threadIdx.x; e < (size_t)nb * Y.k; e += blockDim.x) Un[e] = pre[e];
    else cta_gemm_df(nb, Y.k, nb, alpha, X.A, nb, X.tA, Y.U, nb, 0, 0.0, Un, nb);
    for (size_t e = threadIdx.x; e < (size_t)nb * Y.k; e += blockDim.x) Vn[e] = Y.V[e];
    r = Y.k;
  } else {  // V part op(Y)^T V_x, likewise
    pf = pre ? 0.0 : 2.0 * nb * nb * X.k;
    if (pre) for (size_t e = threadIdx.x; e < (size_t)nb * X.k; e += blockDim.x) Vn[e] = pre[e];
    else cta_gemm_df(nb, X.k, nb, 1.0, Y.A, nb, !Y.tA, X.V, nb, 0, 0.0, Vn, nb);
    for (size_t e = threadIdx.x; e < (size_t)nb * X.k; e += blockDim.x) Un[e] = alpha * X.U[e];
    r = X.k;
  }
  __syncthreads();
  if (flops && threadIdx.x == 0) atomicAdd(flops, pf);
  const int kr = cta_recompress(w, nb, k0 + r, tau, v.kcap, trunc_cap, v, tt, st, sh, shi, flops);
  if (threadIdx.x == 0) v.rank[tt] = kr;
}

// Persistent: gridDim.x CTAs (the resident count) take items in list order from
// an atomic counter (*ctr starts at 0), so a launch covers a whole phase and the
// long items, listed first, overlap with the short ones.  Items touch distinct
// target tiles and read only operand tiles that no item of the launch writes.
// Every CTA has the same size, so an item's arithmetic does not depend on which
// CTA takes it: results are bitwise reproducible.
__global__ void __launch_bounds__(256, 3) k_upd_lr_gen(TlrView v, int alg, int k, const int2* __restrict__ items,
                                                       int n_items, int* __restrict__ ctr, double eps,
                                                       const double* __restrict__ d_zeta, double zpow, int Kmax,
                                                       int trunc_cap, double* __restrict__ ws, size_t item_elems,
                                                       long long* __restrict__ st, double* __restrict__ flops,
                                                       const double* __restrict__ pre, int n_pre) {
  extern __shared__ dfloat vs_dyn[];  // 2 nb: staged reflectors of the recompression
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  __shared__ int s_item;
  const double tau = d_zeta ? eps * pow(*d_zeta, zpow) : eps;
  ItemWs w = item_ws(ws, item_elems, blockIdx.x, v.nb, Kmax, v.kcap);
  w.vs = vs_dyn;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
    __syncthreads();
    const int q = s_item;
    __syncthreads();  // every thread holds q before thread 0 takes the next one
    if (q >= n_items) break;
    upd_lr_item(v, alg, k, items[q], tau, Kmax, trunc_cap, w, st, flops, sh, shi,
                q < n_pre ? pre + (size_t)q * v.nb * v.kcap : nullptr);
    __syncthreads();  // the workspace is reused by the next item
  }
}

// items q < cnt with one dense operand: the product that the update kernel would form with the
// dense tile, P_q = alpha op(X) U_y (X dense) or op(Y)^T V_x (Y dense), nb x rank into slot q of P
// (nb x kcap each); other items get an empty descriptor
__global__ void k_dop_desc(TlrView v, int alg, int k, const int2* __restrict__ items, int cnt, double* __restrict__ P,
                           GemmGen* __restrict__ d) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  const int2 it = items[q];
  const int nb = v.nb;
  Opnd X, Y;
  double alpha;
  operands(v, alg, it.x, it.y, k, &X, &Y, &alpha);
  GemmGen g;
  g.A = g.B = nullptr; g.C = P + (size_t)q * nb * v.kcap; g.m = g.n = g.k = 0;
  g.lda = g.ldb = g.ldc = nb; g.tA = g.tB = 0; g.alpha = 1.0; g.beta = 0.0; g.lower = 0;
  if (X.k > 0 && Y.k > 0 && X.dense != Y.dense) {
    g.m = nb; g.k = nb; g.B = X.dense ? Y.U : X.V;
    if (X.dense) { g.n = Y.k; g.A = X.A; g.tA = X.tA; g.alpha = alpha; }
    else { g.n = X.k; g.A = Y.A; g.tA = !Y.tA; }
  }
  d[q] = g;
}

// ---- the same update with each item split over the two CTAs of a cluster: CTA rank 0 forms and
// recompresses the U side (product factor, Householder QR of U, applying Q_U, storing U), rank 1 the
// V side; rank 0 also runs the small core (M = R_u R_v^T, its pivoted QR, the arena block) between
// two cluster barriers.  Halves the latency of an item, which bounds every launch (each launch lasts
// as long as its longest item).
__device__ void upd_lr_item_pair(const TlrView& v, int alg, int k, int2 it, double tau, int Kmax, int trunc_cap,
                                 ItemWs& w, long long* __restrict__ st, double* __restrict__ flops, double* sh,
                                 int* shi, const double* __restrict__ pre, int rank, int* s_k) {
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  Opnd X, Y;
  double alpha;
  operands(v, alg, it.x, it.y, k, &X, &Y, &alpha);
  // both CTAs take the same branches (the same data decide them)
  if (X.k == 0 || Y.k == 0) return;
  if (X.dense && Y.dense) {
    if (rank == 0 && threadIdx.x == 0) set_status(st, TLR_ERR_STATE, tt);
    return;
  }
  const int k0 = v.rank[tt];
  const int r = X.dense ? Y.k : (Y.dense ? X.k : min(X.k, Y.k));
  if (k0 + r > Kmax) {
    if (rank == 0 && threadIdx.x == 0) set_status(st, TLR_ST_WIDEN, tt);
    return;
  }
  const int side = rank;  // 0: U, 1: V
  double* Pold = side ? tileV(v, tt) : tileU(v, tt);
  double* P = side ? w.Vp : w.Up;
  for (size_t e = threadIdx.x; e < (size_t)nb * k0; e += blockDim.x) P[e] = Pold[e];
  double* Pn = P + (size_t)k0 * nb;
  double pf = 0.0;  // product flops
  if (!X.dense && !Y.dense) {
    const bool uside = Y.k <= X.k;  // the product goes to U (else to V)
    if (uside == (side == 0)) {
      pf = 2.0 * nb * X.k * Y.k * 2.0;
      const bool thin = X.k <= 48 && Y.k <= 48;
      if (thin) cta_gemm_tn_thin(X.k, Y.k, nb, 1.0, X.V, Y.U, w.W, X.k);  // W = V_x^T U_y
      else cta_gemm_df(X.k, Y.k, nb, 1.0, X.V, nb, 1, Y.U, nb, 0, 0.0, w.W, X.k);
      if (uside) {
        if (thin) cta_gemm_nn_thin(nb, Y.k, X.k, alpha, X.U, w.W, X.k, 0, Pn);  // U_x W
        else cta_gemm_df(nb, Y.k, X.k, alpha, X.U, nb, 0, w.W, X.k, 0, 0.0, Pn, nb);
      } else {
        if (thin) cta_gemm_nn_thin(nb, X.k, Y.k, 1.0, Y.V, w.W, X.k, 1, Pn);  // V_y W^T
        else cta_gemm_df(nb, X.k, Y.k, 1.0, Y.V, nb, 0, w.W, X.k, 1, 0.0, Pn, nb);
      }
    } else if (side == 1) {
      for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = Y.V[e];
    } else {
      for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = alpha * X.U[e];
    }
  } else if (X.dense) {  // U part alpha op(X) U_y (staged or formed here), V part V_y
    if (side == 0) {
      pf = pre ? 0.0 : 2.0 * nb * nb * Y.k;
      if (pre) for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = pre[e];
      else cta_gemm_df(nb, Y.k, nb, alpha, X.A, nb, X.tA, Y.U, nb, 0, 0.0, Pn, nb);
    } else {
      for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = Y.V[e];
    }
  } else {  // V part op(Y)^T V_x, U part alpha U_x
    if (side == 1) {
      pf = pre ? 0.0 : 2.0 * nb * nb * X.k;
      if (pre) for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = pre[e];
      else cta_gemm_df(nb, X.k, nb, 1.0, Y.A, nb, !Y.tA, X.V, nb, 0, 0.0, Pn, nb);
    } else {
      for (size_t e = threadIdx.x; e < (size_t)nb * r; e += blockDim.x) Pn[e] = alpha * X.U[e];
    }
  }
  __syncthreads();
  if (flops && threadIdx.x == 0 && pf > 0.0) atomicAdd(flops, pf);
  const int kr = cluster_recompress(w, nb, k0 + r, tau, v.kcap, trunc_cap, v, tt, st, sh, shi, flops, rank, s_k);
  if (rank == 0 && threadIdx.x == 0) v.rank[tt] = kr;
}

// Persistent, in clusters of two CTAs: rank 0 takes items in list order from the atomic counter and
// shares the index through distributed shared memory; both CTAs work on the item (upd_lr_item_pair)
// with the cluster's workspace.  Every cluster runs the same arithmetic, so results are reproducible.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 3)
    k_upd_lr_pair(TlrView v, int alg, int k, const int2* __restrict__ items, int n_items, int* __restrict__ ctr,
                  double eps, const double* __restrict__ d_zeta, double zpow, int Kmax, int trunc_cap,
                  double* __restrict__ ws, size_t item_elems, long long* __restrict__ st, double* __restrict__ flops,
                  const double* __restrict__ pre, int n_pre) {
  extern __shared__ dfloat vs_dyn[];  // nb: staged reflectors of this CTA's side
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  __shared__ int s_item, s_k;
  const int rank = cluster_rank();
  const double tau = d_zeta ? eps * pow(*d_zeta, zpow) : eps;
  ItemWs w = item_ws(ws, item_elems, blockIdx.x >> 1, v.nb, Kmax, v.kcap);
  w.vs = vs_dyn;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
    cluster_sync_all();
    const int q = dsmem_load_int(&s_item, 0);
    cluster_sync_all();  // both hold q before rank 0 takes the next one
    if (q >= n_items) break;
    upd_lr_item_pair(v, alg, k, items[q], tau, Kmax, trunc_cap, w, st, flops, sh, shi,
                     q < n_pre ? pre + (size_t)q * v.nb * v.kcap : nullptr, rank, &s_k);
    __syncthreads();
  }
}

// dense target C += alpha op(X) op(Y) as three batched GEMM stages per item:
//   stage 0: W = V_x^T U_y (LR x LR) or T = op(X) U_y (dense X) or T = op(Y)^T V_x (dense Y)
//   stage 1: T = U_x W or T = V_y W^T (LR x LR only)
//   stage 2: C += alpha T V_y^T, alpha U_x T^T or alpha op(X) op(Y)
// an unused stage has k = 0 and beta = 1 (no-op)
__global__ void k_upd_d_desc(TlrView v, int alg, int k, const int2* __restrict__ items, int cnt,
                             GemmGen* __restrict__ d0, GemmGen* __restrict__ d1, GemmGen* __restrict__ d2,
                             double* __restrict__ ws, size_t ws_elems) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  const int2 it = items[q];
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  Opnd X, Y;
  double alpha;
  operands(v, alg, it.x, it.y, k, &X, &Y, &alpha);
  double* W = ws + (size_t)q * ws_elems;
  double* T = W + (size_t)v.kcap * v.kcap;
  GemmGen nop;
  nop.A = nop.B = nullptr; nop.C = T; nop.m = nop.n = 0; nop.k = 0; nop.lda = nop.ldb = nop.ldc = nb;
  nop.tA = nop.tB = 0; nop.alpha = 0.0; nop.beta = 1.0; nop.lower = 0;
  GemmGen g0 = nop, g1 = nop, g2 = nop;
  g2.C = tileA(v, tt); g2.ldc = nb; g2.m = nb; g2.n = nb; g2.alpha = alpha; g2.beta = 1.0;
  g2.lda = nb; g2.ldb = nb;
  auto mk = [&](GemmGen& g, int m, int n, int kk, const double* A, int lda, int tA, const double* B, int ldb, int tB,
                double* C, int ldc) {
    g.m = m; g.n = n; g.k = kk; g.A = A; g.lda = lda; g.tA = tA; g.B = B; g.ldb = ldb; g.tB = tB; g.C = C;
    g.ldc = ldc; g.alpha = 1.0; g.beta = 0.0; g.lower = 0;
  };
  if (X.k == 0 || Y.k == 0) {
    g2.k = 0;
  } else if (X.dense && Y.dense) {
    g2.A = X.A; g2.tA = X.tA; g2.B = Y.A; g2.tB = Y.tA; g2.k = nb;
  } else if (X.dense) {
    mk(g0, nb, Y.k, nb, X.A, nb, X.tA, Y.U, nb, 0, T, nb);
    g2.A = T; g2.tA = 0; g2.B = Y.V; g2.tB = 1; g2.k = Y.k;
  } else if (Y.dense) {
    mk(g0, nb, X.k, nb, Y.A, nb, !Y.tA, X.V, nb, 0, T, nb);
    g2.A = X.U; g2.tA = 0; g2.B = T; g2.tB = 1; g2.k = X.k;
  } else {
    mk(g0, X.k, Y.k, nb, X.V, nb, 1, Y.U, nb, 0, W, X.k);
    if (Y.k <= X.k) {
      mk(g1, nb, Y.k, X.k, X.U, nb, 0, W, X.k, 0, T, nb);
      g2.A = T; g2.tA = 0; g2.B = Y.V; g2.tB = 1; g2.k = Y.k;
    } else {
      mk(g1, nb, X.k, Y.k, Y.V, nb, 0, W, X.k, 1, T, nb);
      g2.A = X.U; g2.tA = 0; g2.B = T; g2.tB = 1; g2.k = X.k;
    }
  }
  d0[q] = g0;
  d1[q] = g1;
  d2[q] = g2;
}

// products A^T B of two thin column blocks (results up to 64 x 64, lda = ldb = depth, beta = 0), a CTA
// per descriptor; any other descriptor takes the 64 x 64 block path
__global__ void __launch_bounds__(256) k_gemm_tn_thin(const GemmGen* __restrict__ desc) {
  const GemmGen g = desc[blockIdx.x];
  if ((g.k <= 0 && g.beta == 1.0) || g.m <= 0 || g.n <= 0) return;
  if (g.tA && !g.tB && g.beta == 0.0 && g.m <= 64 && g.n <= 64 && g.lda == g.k && g.ldb == g.k)
    cta_gemm_tn_thin4(g.m, g.n, g.k, g.alpha, g.A, g.B, g.C, g.ldc);
  else
    cta_gemm_df_blocks(g.m, g.n, g.k, g.alpha, g.A, g.lda, g.tA, g.B, g.ldb, g.tB, g.beta, g.C, g.ldc, 0, 1, g.lower);
}

__global__ void k_gemm_gen(const GemmGen* __restrict__ desc, int k_skip) {
  const GemmGen g = desc[blockIdx.y];
  if ((g.k <= 0 && g.beta == 1.0) || g.m <= 0 || g.n <= 0 || g.k >= k_skip) return;
  if (g.tA && !g.tB && g.beta == 0.0 && g.m <= 64 && g.n <= 64 && g.lda == g.k && g.ldb == g.k) {
    // A^T B of two thin column blocks (ranks x depth): warps on 4 x 4 blocks of the small result, lanes
    // along the depth, instead of a 64 x 64 block mostly outside it
    if (blockIdx.x == 0) cta_gemm_tn_thin(g.m, g.n, g.k, g.alpha, g.A, g.B, g.C, g.ldc);
    return;
  }
  if (g.n <= 32 && !g.lower) {  // a thin result: 128 x 32 blocks
    cta_gemm_df_blocks_n32(g.m, g.n, g.k, g.alpha, g.A, g.lda, g.tA, g.B, g.ldb, g.tB, g.beta, g.C, g.ldc, blockIdx.x,
                           gridDim.x);
    return;
  }
  cta_gemm_df_blocks(g.m, g.n, g.k, g.alpha, g.A, g.lda, g.tA, g.B, g.ldb, g.tB, g.beta, g.C, g.ldc, blockIdx.x,
                     gridDim.x, g.lower);
}

// X = T^{-1} for a lower triangular nb x nb tile T (both column-major, ld nb) by forward
// substitution on the identity, TRINV_COLS columns per CTA.  Column block c0 is zero above
// row c0 and stays so: the sweep starts at the 32-row block holding c0.
#define TRINV_COLS 2
__global__ void k_trinv(const double* __restrict__ T, int nb, double* __restrict__ X) {
  __shared__ double Ls[32][33];
  __shared__ double Xs[32][TRINV_COLS + 1];
  const int c0 = blockIdx.x * TRINV_COLS;
  const int ncol = min(TRINV_COLS, nb - c0);
  for (int e = threadIdx.x; e < nb * TRINV_COLS; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    if (c < ncol) X[(size_t)(c0 + c) * nb + r] = (r == c0 + c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int rb0 = (c0 / 32) * 32; rb0 < nb; rb0 += 32) {
    const int w = min(32, nb - rb0);
    for (int id = threadIdx.x; id < 32 * 32; id += blockDim.x) {
      const int r = id & 31, c = id >> 5;
      Ls[r][c] = (r < w && c < w) ? T[(size_t)(rb0 + c) * nb + rb0 + r] : 0.0;
    }
    for (int id = threadIdx.x; id < 32 * TRINV_COLS; id += blockDim.x) {
      const int r = id % 32, c = id / 32;
      Xs[r][c] = (r < w && c < ncol) ? X[(size_t)(c0 + c) * nb + rb0 + r] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < ncol) {
      const int c = threadIdx.x;
      for (int r = 0; r < w; ++r) {
        double v = Xs[r][c];
        for (int l = 0; l < r; ++l) v -= Ls[r][l] * Xs[l][c];
        Xs[r][c] = v / Ls[r][r];
      }
    }
    __syncthreads();
    for (int id = threadIdx.x; id < 32 * TRINV_COLS; id += blockDim.x) {
      const int r = id % 32, c = id / 32;
      if (r < w && c < ncol) X[(size_t)(c0 + c) * nb + rb0 + r] = Xs[r][c];
    }
    for (int r = rb0 + w + threadIdx.x; r < nb; r += blockDim.x) {
      double acc[TRINV_COLS];
#pragma unroll
      for (int c = 0; c < TRINV_COLS; ++c) acc[c] = 0.0;
      for (int l = 0; l < w; ++l) {
        const double lv = T[(size_t)(rb0 + l) * nb + r];
#pragma unroll
        for (int c = 0; c < TRINV_COLS; ++c) acc[c] = fma(lv, Xs[l][c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < TRINV_COLS; ++c)
        if (c < ncol) X[(size_t)(c0 + c) * nb + r] -= acc[c];
    }
    __syncthreads();
  }
}

struct DenseEntry {
  const double* A;
  int nb;
  __device__ __forceinline__ double operator()(int a, int b) const { return A[(size_t)b * nb + a]; }
};

// low-rank target hit by a dense x dense product: descriptors that materialise
// buf = alpha op(X) op(Y) (d1) and then buf += U_t V_t^T (d2)
__global__ void k_dd_prep(TlrView v, int alg, int k, const int2* __restrict__ items, int cnt, GemmGen* __restrict__ d1,
                          GemmGen* __restrict__ d2, double* __restrict__ bufs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  const int2 it = items[q];
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  Opnd X, Y;
  double alpha;
  operands(v, alg, it.x, it.y, k, &X, &Y, &alpha);
  double* buf = bufs + (size_t)q * nb * nb;
  GemmGen g;
  g.A = X.A; g.tA = X.tA; g.B = Y.A; g.tB = Y.tA; g.C = buf; g.m = nb; g.n = nb; g.k = nb;
  g.lda = nb; g.ldb = nb; g.ldc = nb; g.alpha = alpha; g.beta = 0.0; g.lower = 0;
  d1[q] = g;
  g.A = tileU(v, tt); g.tA = 0; g.B = tileV(v, tt); g.tB = 1; g.k = v.rank[tt]; g.alpha = 1.0; g.beta = 1.0;
  d2[q] = g;
}

// compress the materialised target (ACA on stored entries, then eps-truncated SVD)
__global__ void k_dd_compress(TlrView v, const int2* __restrict__ items, const double* __restrict__ bufs, double eps,
                              const double* __restrict__ d_zeta, double zpow, int aca_max, int Kmax, int trunc_cap,
                              double* __restrict__ ws, size_t item_elems, long long* __restrict__ st) {
  extern __shared__ double dsm[];
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  const int2 it = items[blockIdx.x];
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  const double tau = d_zeta ? eps * pow(*d_zeta, zpow) : eps;
  ItemWs w = item_ws(ws, item_elems, blockIdx.x, nb, Kmax, v.kcap);
  w.vs = reinterpret_cast<dfloat*>(dsm);  // free after the cross approximation
  DenseEntry de{bufs + (size_t)blockIdx.x * nb * nb, nb};
  int conv = 0;
  const int k = cta_aca(de, nb, nb, nb, tau * 0.125, aca_max, w, dsm, sh, shi, &conv);
  if (!conv && threadIdx.x == 0) {
    // below the widest workspace the host widens it and repeats; at it, the rank cap was exceeded
    if (aca_max < 2 * v.kcap) set_status(st, TLR_ST_WIDEN, tt);
    else if (!trunc_cap) set_status(st, TLR_ERR_RANK_CAP, tt);
  }
  if (!conv && aca_max < 2 * v.kcap) return;
  __syncthreads();
  const int kr = cta_recompress(w, nb, k, tau, v.kcap, trunc_cap, v, tt, st, sh, shi);
  if (threadIdx.x == 0) v.rank[tt] = kr;
}

// The same on a cluster of two CTAs per item: rank 0 runs the cross approximation, then both run the
// recompression (cluster_recompress: U side on rank 0, V side on rank 1).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 3)
    k_dd_compress_pair(TlrView v, const int2* __restrict__ items, const double* __restrict__ bufs, double eps,
                       const double* __restrict__ d_zeta, double zpow, int aca_max, int Kmax, int trunc_cap,
                       double* __restrict__ ws, size_t item_elems, long long* __restrict__ st) {
  extern __shared__ double dsm[];
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  __shared__ int s_aca[2], s_k;
  const int rank = cluster_rank();
  const int q = blockIdx.x >> 1;
  const int2 it = items[q];
  const int nb = v.nb;
  const int64_t tt = dtile_index(it.x, it.y);
  const double tau = d_zeta ? eps * pow(*d_zeta, zpow) : eps;
  ItemWs w = item_ws(ws, item_elems, q, nb, Kmax, v.kcap);
  w.vs = reinterpret_cast<dfloat*>(dsm);  // free after the cross approximation
  if (rank == 0) {
    DenseEntry de{bufs + (size_t)q * nb * nb, nb};
    int conv = 0;
    const int k = cta_aca(de, nb, nb, nb, tau * 0.125, aca_max, w, dsm, sh, shi, &conv);
    if (!conv && threadIdx.x == 0) {
      // below the widest workspace the host widens it and repeats; at it, the rank cap was exceeded
      if (aca_max < 2 * v.kcap) set_status(st, TLR_ST_WIDEN, tt);
      else if (!trunc_cap) set_status(st, TLR_ERR_RANK_CAP, tt);
    }
    if (threadIdx.x == 0) { s_aca[0] = k; s_aca[1] = conv; }
    __syncthreads();
  }
  cluster_sync_all();  // the cross factors are in the workspace
  const int k = dsmem_load_int(&s_aca[0], 0), conv = dsmem_load_int(&s_aca[1], 0);
  cluster_sync_all();  // rank 1 has read them
  if (!conv && aca_max < 2 * v.kcap) return;
  const int kr = cluster_recompress(w, nb, k, tau, v.kcap, trunc_cap, v, tt, st, sh, shi, nullptr, rank, &s_k);
  if (rank == 0 && threadIdx.x == 0) v.rank[tt] = kr;
}

// descriptors of X_tmp = alpha op(M) X (or alpha A op(M)) for tile items
// items q < nl: low-rank tiles lr[q] (X = U or V by `which`, op(M) transM); the others dense tiles
// dn[q - nl] (op(M) transM_dense, M on the right when dense_right); products into tmp (low-rank ones
// first, lr_elems each, then dn_elems each)
__global__ void k_trmul_desc(TlrView v, const double* __restrict__ M0, size_t m_stride, int m_by, int transM,
                             int transM_dense, const int2* __restrict__ lr, int nl, const int2* __restrict__ dn,
                             int cnt, int which, int dense_right, double alpha, double* __restrict__ tmp,
                             size_t lr_elems, size_t dn_elems, GemmGen* __restrict__ desc, double** __restrict__ dst) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  const bool dense = q >= nl;
  const int2 it = dense ? dn[q - nl] : lr[q];
  const double* M = M0 + (m_by == 1 ? (size_t)it.x * m_stride : m_by == 2 ? (size_t)it.y * m_stride : 0);
  const int64_t t = dtile_index(it.x, it.y);
  const int nb = v.nb;
  GemmGen g;
  g.C = dense ? tmp + (size_t)nl * lr_elems + (size_t)(q - nl) * dn_elems : tmp + (size_t)q * lr_elems;
  g.ldc = nb; g.lda = nb; g.ldb = nb; g.alpha = alpha; g.beta = 0.0;
  g.lower = 0; g.m = nb; g.k = nb;
  double* X;
  if (dense) {
    X = tileA(v, t);
    g.n = nb;
    if (dense_right) { g.A = X; g.tA = 0; g.B = M; g.tB = transM_dense; }
    else { g.A = M; g.tA = transM_dense; g.B = X; g.tB = 0; }
  } else {
    X = which == 0 ? tileU(v, t) : tileV(v, t);
    g.n = v.rank[t];
    g.A = M; g.tA = transM; g.B = X; g.tB = 0;
  }
  desc[q] = g;
  dst[q] = X;
}

__global__ void k_copy_back(const GemmGen* __restrict__ desc, double* const* __restrict__ dst) {
  const GemmGen g = desc[blockIdx.y];
  double* X = dst[blockIdx.y];
  const int64_t cnt = (int64_t)g.m * g.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = g.C[e];
}

// dynamic shared memory of the persistent low-rank update kernel (two staged reflectors)
size_t upd_smem(int nb) { return 2 * (size_t)nb * sizeof(dfloat); }

// resident CTAs of the persistent low-rank update kernel on the current device for tile size nb
// (remembered per device and tile size; handles on several host threads may use different sizes)
int resident_ctas(int nb) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find({dev, nb});
    if (it != memo.end()) return it->second;
  }
  int per_sm = 0, sms = 0;
  if (tlr_smem_optin((const void*)k_upd_lr_gen, upd_smem(nb)) != TLR_OK) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_upd_lr_gen, TLR_THREADS, upd_smem(nb)) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  const int r = std::max(per_sm, 1) * sms;
  std::lock_guard<std::mutex> lock(mu);
  memo[{dev, nb}] = r;
  return r;
}

int chunk_of(const tlr_ctx* h, size_t per_item, size_t reserve) {
  size_t avail = h->scratch_elems > reserve ? h->scratch_elems - reserve : 0;
  size_t c = per_item ? avail / per_item : 65535;
  if (c > 65535) c = 65535;
  return (int)c;
}

}  // namespace

int tops_resident_ctas(int nb) { return resident_ctas(nb); }

namespace {
// dynamic shared memory of the cluster version (one side's staged reflector)
size_t pair_smem(int nb) { return (size_t)nb * sizeof(dfloat); }

// items on two-CTA clusters (k_upd_lr_pair) unless the environment variable TLR_UPD_PAIR is 0
bool upd_pair_mode() {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("TLR_UPD_PAIR");
    mode = (e && atoi(e) == 0) ? 0 : 1;
  }
  return mode == 1;
}

// resident clusters of k_upd_lr_pair on the current device for tile size nb (0 if unavailable)
int resident_pairs(int nb) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find({dev, nb});
    if (it != memo.end()) return it->second;
  }
  int clusters = 0;
  if (tlr_smem_optin((const void*)k_upd_lr_pair, pair_smem(nb)) == TLR_OK) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 1024);
    cfg.blockDim = dim3(TLR_THREADS);
    cfg.dynamicSmemBytes = pair_smem(nb);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)k_upd_lr_pair, &cfg) != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
  }
  std::lock_guard<std::mutex> lock(mu);
  memo[{dev, nb}] = clusters;
  return clusters;
}
}  // namespace

bool tops_cluster_mode() { return upd_pair_mode(); }

int tops_gemm_thin(const GemmGen* d_desc, int count, cudaStream_t s) {
  for (int c0 = 0; c0 < count; c0 += 1 << 30) {
    const int cnt = count - c0 < (1 << 30) ? count - c0 : (1 << 30);
    k_gemm_tn_thin<<<cnt, 256, 0, s>>>(d_desc + c0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

int tops_gemm(const GemmGen* d_desc, int count, int m, int n, cudaStream_t s, int k_skip) {
  if (count <= 0) return TLR_OK;
  const int blocks = ((m + 63) / 64) * ((n + 63) / 64);
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = count - c0 < 65535 ? count - c0 : 65535;
    k_gemm_gen<<<dim3(blocks, cnt), 256, 0, s>>>(d_desc + c0, k_skip);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

namespace {
// depth from which a batched product runs on the tensor cores (digit slices) instead of the CUDA cores
constexpr int TC_MIN_DEPTH = 256;

// doubles of tensor-core workspace per descriptor of an m x n x k batched product (0: CUDA cores only)
size_t tc_item_doubles(const tlr_ctx* h, int m, int n, int k) {
  const int S = tlr_tc_slices(h);
  if (!S || k < TC_MIN_DEPTH) return 0;
  return (oz_device_item_bytes(m, n, k, S) + 7) / 8;
}

// batched product of device descriptors (m, n, k bounds): depths >= TC_MIN_DEPTH on the tensor cores with
// the workspace tc (tc_doubles), the others on the CUDA cores
// (all_deep: every non-empty descriptor has depth kmax, so no CUDA-core launch is needed after the tensor cores)
int tops_gemm_mixed(tlr_ctx* h, const GemmGen* d_desc, int count, int m, int n, int kmax, double* tc, size_t tc_doubles,
                    cudaStream_t s, bool all_deep = false) {
  const int S = tlr_tc_slices(h);
  if (!S || kmax < TC_MIN_DEPTH || !tc_doubles) return tops_gemm(d_desc, count, m, n, s);
  int rc = oz_run_device(d_desc, count, m, n, kmax, TC_MIN_DEPTH, S, tc, tc_doubles * 8, h->d_stat, s);
  if (rc || all_deep) return rc;
  return tops_gemm(d_desc, count, m, n, s, TC_MIN_DEPTH);
}
}  // namespace

int tlr_smem_optin(const void* f, size_t dyn) {
  // the limit is raised once per device and kernel to all the shared memory a block may have, so that
  // callers on several host threads with different sizes never lower it under one another's launch
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, f) != cudaSuccess) return TLR_ERR_CUDA;
  if (a.sharedSizeBytes + dyn <= 48 * 1024) return TLR_OK;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return TLR_ERR_CUDA;
  const int most = optin - (int)a.sharedSizeBytes;
  if ((int)dyn > most) return TLR_ERR_CUDA;
  if (a.maxDynamicSharedSizeBytes >= most) return TLR_OK;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most) == cudaSuccess ? TLR_OK
                                                                                                   : TLR_ERR_CUDA;
}

// the products of the first n_dop low-rank items with the dense operand, into h->dop (batched GEMM, on the
// tensor cores where the handle's precision allows); false when the buffer cannot be had (the update
// kernel then forms them itself)
static int stage_dense_operand_products(tlr_ctx* h, const TlrView& v, int alg, int k, const int2* d_lr,
                                        int64_t n_dop, cudaStream_t s, bool* staged) {
  *staged = false;
  const size_t slot = (size_t)h->nb * h->kcap;
  const size_t gd = (sizeof(GemmGen) + 7) / 8;
  const size_t tcd = tc_item_doubles(h, h->nb, h->kcap, h->nb);
  const int64_t tc_items = std::min<int64_t>(n_dop, 64);  // the tensor-core workspace is reused in chunks
  const size_t want = (size_t)n_dop * (slot + gd) + (size_t)tc_items * tcd + 64;
  if (want > h->dop_elems) {
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->dop) cudaFree(h->dop);
    h->dop = nullptr;
    h->dop_elems = 0;
    if (cudaMalloc((void**)&h->dop, (want + want / 4) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return TLR_OK;
    }
    h->dop_elems = want + want / 4;
  }
  GemmGen* d = (GemmGen*)(h->dop + (size_t)n_dop * slot);
  double* tc = h->dop + (size_t)n_dop * (slot + gd) + 16;
  tc = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tc) + 127) & ~(uintptr_t)127);
  const size_t tc_avail = tcd ? (size_t)(h->dop + h->dop_elems - tc) : 0;
  k_dop_desc<<<(unsigned)((n_dop + 127) / 128), 128, 0, s>>>(v, alg, k, d_lr, (int)n_dop, h->dop, d);
  TLR_LAUNCH_CHECK();
  int rc = tops_gemm_mixed(h, d, (int)n_dop, h->nb, h->kcap, h->nb, tc, tc_avail, s, true);
  if (rc) return rc;
  *staged = true;
  return TLR_OK;
}

int tops_update(tlr_ctx* h, const TlrView& v, int alg, int k, const int2* d_lr, int64_t n_lr, int64_t n_dop,
                const int2* d_dn, int64_t n_dn, double eps, const double* d_zeta, double zpow, cudaStream_t s,
                int reserve) {
  if (n_dn > 0) {
    PhaseScope ps("update.dense_target", s);
    const size_t per = (size_t)h->kcap * h->kcap + (size_t)h->nb * h->kcap;
    const size_t gd = (sizeof(GemmGen) + 7) / 8;
    const int nc = h->kcap > h->nb ? h->nb : h->kcap;
    const size_t tcd = std::max(tc_item_doubles(h, h->nb, nc, h->nb), tc_item_doubles(h, h->nb, h->nb, h->nb));
    int chunk = chunk_of(h, per + 3 * gd + tcd, 64);
    if (chunk < 1) TLR_RETURN_OOM();
    for (int64_t q0 = 0; q0 < n_dn; q0 += chunk) {
      const int cnt = (int)(n_dn - q0 < chunk ? n_dn - q0 : chunk);
      GemmGen* d0 = (GemmGen*)h->scratch;
      GemmGen* d1 = (GemmGen*)(h->scratch + (size_t)cnt * gd + 1);
      GemmGen* d2 = (GemmGen*)(h->scratch + 2 * ((size_t)cnt * gd + 1));
      double* ws = h->scratch + 3 * ((size_t)cnt * gd + 1);
      // tensor-core workspace after the items' buffers, 128-byte aligned
      double* tc = ws + (size_t)cnt * per + 16;
      tc = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tc) + 127) & ~(uintptr_t)127);
      const size_t tc_avail = (size_t)(h->scratch + h->scratch_elems - tc);
      k_upd_d_desc<<<(cnt + 127) / 128, 128, 0, s>>>(v, alg, k, d_dn + q0, cnt, d0, d1, d2, ws, per);
      TLR_LAUNCH_CHECK();
      // stage 0 (a dense factor times a thin one, depth nb) and stage 2 (dense x dense, depth nb)
      int rc = tops_gemm_mixed(h, d0, cnt, h->nb, nc, h->nb, tc, tcd ? tc_avail : 0, s, true);
      if (rc) return rc;
      rc = tops_gemm(d1, cnt, h->nb, nc, s);
      if (rc) return rc;
      rc = tops_gemm_mixed(h, d2, cnt, h->nb, h->nb, h->nb, tc, tcd ? tc_avail : 0, s);
      if (rc) return rc;
    }
  }
  if (n_lr > 0) {
    PhaseScope ps("update.lowrank_target", s);
    const size_t ie = tlr_item_elems(h->nb, h->kcap, h->kws);
    const int chunk = chunk_of(h, ie, 0);
    if (chunk < 1) TLR_RETURN_OOM();
    const int slots = std::max(resident_ctas(h->nb) - std::max(reserve, 0), 1);
    const int grid = (int)std::min<int64_t>(n_lr, std::min(slots, chunk));
    bool staged = false;
    if (n_dop > 0) {
      PhaseScope ps2("update.dense_operand", s);
      const int rc = stage_dense_operand_products(h, v, alg, k, d_lr, std::min(n_dop, n_lr), s, &staged);
      if (rc) return rc;
    }
    TLR_CUDA_TRY(cudaMemsetAsync(h->d_ctr, 0, sizeof(int), s));
    double* fl = g_tlr_prof.enabled ? g_tlr_prof.d_flops : nullptr;
    const double* pre = staged ? h->dop : nullptr;
    const int n_pre = staged ? (int)std::min(n_dop, n_lr) : 0;
    const int pairs = upd_pair_mode() ? resident_pairs(h->nb) : 0;
    if (g_tlr_prof.enabled) tlr_prof_begin(s);
    if (pairs > 0) {  // each item on a cluster of two CTAs (one workspace a cluster)
      const int cl = (int)std::min<int64_t>(n_lr, std::min(std::max(pairs - std::max(reserve, 0) / 2, 1), chunk));
      k_upd_lr_pair<<<2 * cl, TLR_THREADS, pair_smem(h->nb), s>>>(v, alg, k, d_lr, (int)n_lr, h->d_ctr, eps, d_zeta,
                                                                  zpow, h->kws, h->opts.truncate_at_cap, h->scratch,
                                                                  ie, h->d_stat, fl, pre, n_pre);
    } else {
      k_upd_lr_gen<<<grid, TLR_THREADS, upd_smem(h->nb), s>>>(v, alg, k, d_lr, (int)n_lr, h->d_ctr, eps, d_zeta, zpow,
                                                              h->kws, h->opts.truncate_at_cap, h->scratch, ie,
                                                              h->d_stat, fl, pre, n_pre);
    }
    TLR_LAUNCH_CHECK();
    if (g_tlr_prof.enabled) tlr_prof_end(s);
  }
  return TLR_OK;
}

size_t tops_dd_item_elems(const tlr_ctx* h) {
  // the item's product, recompression buffers and descriptors, its tensor-core slices (if any) and alignment
  const size_t gd = (sizeof(GemmGen) + 7) / 8;
  return (size_t)h->nb * h->nb + tlr_item_elems(h->nb, h->kcap, h->kws) + 2 * gd + tc_item_doubles(h, h->nb, h->nb, h->nb) +
         32;
}

int tops_update_dd(tlr_ctx* h, const TlrView& v, int alg, int k, const int2* d_dd, int64_t n_dd, double eps,
                   const double* d_zeta, double zpow, cudaStream_t s, double* ws_base, size_t ws_elems) {
  if (n_dd <= 0) return TLR_OK;
  if (!ws_base) { ws_base = h->scratch; ws_elems = h->scratch_elems; }
  const size_t nn = (size_t)h->nb * h->nb;
  const size_t ie = tlr_item_elems(h->nb, h->kcap, h->kws);
  const size_t gd = (sizeof(GemmGen) + 7) / 8;
  const size_t tcd = tc_item_doubles(h, h->nb, h->nb, h->nb);
  const size_t per = tops_dd_item_elems(h);
  const int chunk = ws_elems > 64 ? (int)std::min<size_t>((ws_elems - 64) / per, 65535) : 0;
  if (chunk < 1) TLR_RETURN_OOM();
  const size_t smem = 2 * (size_t)h->nb * sizeof(double) + (size_t)h->nb * sizeof(int);
  if (tlr_smem_optin((const void*)k_dd_compress, smem) != TLR_OK ||
      tlr_smem_optin((const void*)k_dd_compress_pair, smem) != TLR_OK)
    return TLR_ERR_CUDA;
  for (int64_t q0 = 0; q0 < n_dd; q0 += chunk) {
    const int cnt = (int)(n_dd - q0 < chunk ? n_dd - q0 : chunk);
    GemmGen* d1 = (GemmGen*)ws_base;
    GemmGen* d2 = (GemmGen*)(ws_base + (size_t)cnt * gd + 1);
    double* bufs = ws_base + 2 * (size_t)cnt * gd + 2;
    double* ws = bufs + (size_t)cnt * nn;
    double* tc = ws + (size_t)cnt * ie + 16;
    tc = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tc) + 127) & ~(uintptr_t)127);
    const size_t tc_avail = tcd ? (size_t)(ws_base + ws_elems - tc) : 0;
    k_dd_prep<<<(cnt + 127) / 128, 128, 0, s>>>(v, alg, k, d_dd + q0, cnt, d1, d2, bufs);
    TLR_LAUNCH_CHECK();
    int rc = tops_gemm_mixed(h, d1, cnt, h->nb, h->nb, h->nb, tc, tc_avail, s, true);
    if (rc) return rc;
    rc = tops_gemm(d2, cnt, h->nb, h->nb, s);
    if (rc) return rc;
    if (upd_pair_mode())
      k_dd_compress_pair<<<2 * cnt, TLR_THREADS, smem, s>>>(v, d_dd + q0, bufs, eps, d_zeta, zpow, h->kws, h->kws,
                                                            h->opts.truncate_at_cap, ws, ie, h->d_stat);
    else
      k_dd_compress<<<cnt, TLR_THREADS, smem, s>>>(v, d_dd + q0, bufs, eps, d_zeta, zpow, h->kws, h->kws,
                                                   h->opts.truncate_at_cap, ws, ie, h->d_stat);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

int tops_trmul(tlr_ctx* h, const TlrView& v, const double* M, int transM, const int2* d_lr, int n_lr, int which,
               int transM_dense, const int2* d_dn, int n_dn, int dense_right, double alpha, cudaStream_t s,
               size_t m_stride, int m_by) {
  // low-rank and dense items in one index space (low-rank first), three launches a chunk
  const size_t nb = h->nb;
  const size_t gd = (sizeof(GemmGen) + 7) / 8 + 1;
  const int total = std::max(n_lr, 0) + std::max(n_dn, 0);
  if (total <= 0) return TLR_OK;
  const size_t lr_elems = nb * (size_t)h->kcap, dn_elems = nb * nb;
  const size_t tcd = tc_item_doubles(h, h->nb, h->nb, h->nb);
  const int chunk = chunk_of(h, dn_elems + gd + tcd, 128);
  if (chunk < 1) TLR_RETURN_OOM();
  for (int q0 = 0; q0 < total; q0 += chunk) {
    const int cnt = total - q0 < chunk ? total - q0 : chunk;
    const int nl = std::max(0, std::min(n_lr - q0, cnt));  // low-rank items of this chunk
    const int2* lr = d_lr + std::min(q0, std::max(n_lr, 0));
    const int2* dn = d_dn + std::max(0, q0 - std::max(n_lr, 0));
    GemmGen* desc = (GemmGen*)h->scratch;
    double** dst = (double**)(h->scratch + (size_t)cnt * (gd - 1) + 8);
    double* tmp = h->scratch + (size_t)cnt * gd + 16;
    double* tc = tmp + (size_t)nl * lr_elems + (size_t)(cnt - nl) * dn_elems + 16;
    tc = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tc) + 127) & ~(uintptr_t)127);
    const size_t tc_avail = tcd ? (size_t)(h->scratch + h->scratch_elems - tc) : 0;
    k_trmul_desc<<<(cnt + 127) / 128, 128, 0, s>>>(v, M, m_stride, m_by, transM, transM_dense, lr, nl, dn, cnt, which,
                                                    dense_right, alpha, tmp, lr_elems, dn_elems, desc, dst);
    TLR_LAUNCH_CHECK();
    const int ncols = cnt > nl ? h->nb : h->kcap;
    int rc = tops_gemm_mixed(h, desc, cnt, h->nb, ncols, h->nb, tc, tc_avail, s, true);
    if (rc) return rc;
    k_copy_back<<<dim3(32, cnt), 256, 0, s>>>(desc, dst);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

int tops_trinv(const double* T, int nb, double* X, cudaStream_t s) {
  k_trinv<<<(nb + TRINV_COLS - 1) / TRINV_COLS, 256, 0, s>>>(T, nb, X);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

