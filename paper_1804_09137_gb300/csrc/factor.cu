// TLR Cholesky of Sigma (Sec. III "Cholesky factorization", Sec. V tile
// low-rank format, Sec. VIII-C TLR GEMM) on hybrid tiles.
//
// Compression (Sec. V): each off-diagonal tile is approximated by adaptive
// cross approximation with partial pivoting, which generates only the rows and
// columns it pivots on, then recompressed to the eps-truncated SVD.  A tile
// whose cross approximation has not converged after dense_rank terms is kept
// dense: near the diagonal the ranks are so high that a dense update (a GEMM)
// is cheaper than low-rank recompression.  The host closes the dense set under
// fill-in (dense (i,k) and (j,k) make (i,j) dense), so a dense x dense product
// never lands in a low-rank tile.
//
// Factorization, right looking, panel step k = 0 .. nt-1:
//   POTRF  D_k = L_kk L_kk^T                              (dense.cu)
//   TRSM   L_ik = A_ik L_kk^{-T}: low rank V_ik <- L_kk^{-1} V_ik; dense A_ik <- A_ik L_kk^{-T}
//   SYRK   D_i -= L_ik L_ik^T                             (batched GEMM, lower blocks)
//   GEMM   A_ij -= L_ik L_jk^T, i > j > k: low-rank targets recompressed to eps
//          (one CTA per tile), dense targets by batched GEMM.
#include "recompress.cuh"
#include "tileops.h"

namespace {

// ------------------------------------------------------------- compression
struct GenEntry {  // entries of Sigma_ij generated from the Matérn table
  const double* tab;
  MaternParams mp;
  const double* x;
  const double* y;
  int64_t n, pi0, pj0;
  __device__ __forceinline__ double operator()(int a, int b) const {
    return cov_pts(tab, mp, x, y, n, pi0 + a, pj0 + b);
  }
};

__global__ void k_aca_compress(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                               const double* __restrict__ y, int64_t n, TlrView v, int64_t t0, double eps,
                               int aca_max, int Kmax, int trunc_cap, double* __restrict__ ws, size_t item_elems,
                               long long* __restrict__ st) {
  extern __shared__ double dsm[];
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  const int nb = v.nb;
  const int64_t t = t0 + blockIdx.x;
  int ti, tj;
  decode_lower(t, &ti, &tj);
  ItemWs w = item_ws(ws, item_elems, blockIdx.x, nb, Kmax, v.kcap);
  w.vs = reinterpret_cast<dfloat*>(dsm);  // free after the cross approximation
  const int64_t pi0 = (int64_t)ti * nb, pj0 = (int64_t)tj * nb;
  const int mi = (int)min((int64_t)nb, n - pi0), mj = (int)min((int64_t)nb, n - pj0);
  GenEntry ge{tab, mp, x, y, n, pi0, pj0};
  int conv = 0;
  const int k = cta_aca(ge, nb, mi, mj, eps * 0.125, aca_max, w, dsm, sh, shi, &conv);
  if (!conv) {  // not compressible within aca_max terms: stored dense
    if (threadIdx.x == 0) v.rank[t] = -1;
    return;
  }
  __syncthreads();
  const int kr = cta_recompress(w, nb, k, eps, v.kcap, trunc_cap, v, t, st, sh, shi);
  if (threadIdx.x == 0) v.rank[t] = kr;
}

// The same on a cluster of two CTAs per tile: rank 0 runs the cross approximation, then both run the
// recompression (cluster_recompress: U side on rank 0, V side on rank 1).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 3)
    k_aca_compress_pair(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                        const double* __restrict__ y, int64_t n, TlrView v, int64_t t0, double eps, int aca_max,
                        int Kmax, int trunc_cap, double* __restrict__ ws, size_t item_elems,
                        long long* __restrict__ st) {
  extern __shared__ double dsm[];
  __shared__ double sh[TLR_THREADS / 32 + 2];
  __shared__ int shi[TLR_THREADS / 32 + 2];
  __shared__ int s_aca[2], s_k;
  const int rank = cluster_rank();
  const int nb = v.nb;
  const int q = blockIdx.x >> 1;
  const int64_t t = t0 + q;
  int ti, tj;
  decode_lower(t, &ti, &tj);
  ItemWs w = item_ws(ws, item_elems, q, nb, Kmax, v.kcap);
  w.vs = reinterpret_cast<dfloat*>(dsm);  // free after the cross approximation
  if (rank == 0) {
    const int64_t pi0 = (int64_t)ti * nb, pj0 = (int64_t)tj * nb;
    const int mi = (int)min((int64_t)nb, n - pi0), mj = (int)min((int64_t)nb, n - pj0);
    GenEntry ge{tab, mp, x, y, n, pi0, pj0};
    int conv = 0;
    const int k = cta_aca(ge, nb, mi, mj, eps * 0.125, aca_max, w, dsm, sh, shi, &conv);
    if (threadIdx.x == 0) { s_aca[0] = k; s_aca[1] = conv; }
    __syncthreads();
  }
  cluster_sync_all();  // the cross factors are in the workspace
  const int k = dsmem_load_int(&s_aca[0], 0), conv = dsmem_load_int(&s_aca[1], 0);
  cluster_sync_all();  // rank 1 has read them
  if (!conv) {  // not compressible within aca_max terms: stored dense
    if (rank == 0 && threadIdx.x == 0) v.rank[t] = -1;
    return;
  }
  const int kr = cluster_recompress(w, nb, k, eps, v.kcap, trunc_cap, v, t, st, sh, shi, nullptr, rank, &s_k);
  if (rank == 0 && threadIdx.x == 0) v.rank[t] = kr;
}

// dense generation of listed tiles (Sigma_ij into the dense pool)
__global__ void k_gen_dense_list(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                                 const double* __restrict__ y, int64_t n, TlrView v, const int2* __restrict__ items) {
  const int2 it = items[blockIdx.y];
  const int64_t t = dtile_index(it.x, it.y);
  double* A = tileA(v, t);
  const int nb = v.nb;
  const int64_t nn = (int64_t)nb * nb;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(id % nb), b = (int)(id / nb);
    A[id] = cov_pts(tab, mp, x, y, n, (int64_t)it.x * nb + a, (int64_t)it.y * nb + b);
  }
}

// ----------------------------------------------------------------- SYRK
// descriptor of D_i -= L_ik L_ik^T for i = i0 + blockIdx.x (one CTA per i)
__global__ void k_syrk_prep(TlrView v, int k, int i0, GemmDesc* __restrict__ desc, double* __restrict__ ws,
                            size_t ws_elems) {
  const int i = i0 + blockIdx.x;
  const int64_t t = dtile_index(i, k);
  const int nb = v.nb;
  GemmDesc d;
  d.C = diagT(v, i);
  d.lower = 1;
  if (v.dslot[t] >= 0) {
    d.P = tileA(v, t); d.Q = d.P; d.r = nb;
  } else {
    const int kr = v.rank[t];
    d.Q = tileU(v, t);
    d.r = kr;
    double* G = ws + (size_t)blockIdx.x * ws_elems;
    double* T = G + (size_t)v.kcap * v.kcap;
    d.P = T;
    if (kr > 0) {
      if (kr <= 48) {
        cta_gemm_tn_thin(kr, kr, nb, 1.0, tileV(v, t), tileV(v, t), G, kr);  // G = V^T V
        cta_gemm_nn_thin(nb, kr, kr, 1.0, tileU(v, t), G, kr, 0, T);         // T = U G
      } else {
        cta_gemm_df(kr, kr, nb, 1.0, tileV(v, t), nb, 1, tileV(v, t), nb, 0, 0.0, G, kr);
        cta_gemm_df(nb, kr, kr, 1.0, tileU(v, t), nb, 0, G, kr, 0, 0.0, T, nb);
      }
    }
  }
  if (threadIdx.x == 0) desc[blockIdx.x] = d;
}

// C -= P Q^T, one 64 x 64 block per CTA (double-float products, like every other tile update)
__global__ void k_gemm_desc(const GemmDesc* __restrict__ desc, int nb) {
  const GemmDesc d = desc[blockIdx.y];
  if (d.r <= 0) return;
  cta_gemm_df_blocks(nb, nb, d.r, -1.0, d.P, nb, 0, d.Q, nb, 1, 1.0, d.C, nb, blockIdx.x, gridDim.x, d.lower);
}

}  // namespace

size_t tlr_item_elems(int nb, int kcap, int kws) {
  const size_t Kmax = (size_t)kws;
  return 4 * (size_t)nb * Kmax + (size_t)kcap * kcap + 2 * Kmax * Kmax + 4 * Kmax;
}

static int chunk_for(const tlr_ctx* h, size_t per_item, size_t reserve = 0) {
  size_t avail = h->scratch_elems > reserve ? h->scratch_elems - reserve : 0;
  size_t c = per_item ? avail / per_item : 65535;
  if (c > 65535) c = 65535;
  return (int)c;
}

int tlr_compress_tiles(tlr_ctx* h, double eps, cudaStream_t s) {
  const int nb = h->nb, kcap = h->kcap, Kmax = h->kws;
  const size_t ie = tlr_item_elems(nb, kcap, h->kws);
  const int chunk = chunk_for(h, ie);
  if (chunk < 1) TLR_RETURN_OOM();
  const size_t smem = 2 * (size_t)nb * sizeof(double) + (size_t)nb * sizeof(int);
  if (tlr_smem_optin((const void*)k_aca_compress, smem) != TLR_OK ||
      tlr_smem_optin((const void*)k_aca_compress_pair, smem) != TLR_OK)
    return TLR_ERR_CUDA;
  int aca_max = h->dense_rank + 8;
  if (aca_max > Kmax) aca_max = Kmax;
  const TlrView v = view_of(h);
  for (int64_t t0 = 0; t0 < h->ntiles; t0 += chunk) {
    const int cnt = (int)((h->ntiles - t0) < chunk ? (h->ntiles - t0) : chunk);
    if (tops_cluster_mode())
      k_aca_compress_pair<<<2 * cnt, TLR_THREADS, smem, s>>>(h->tab, h->mp, h->x, h->y, h->n, v, t0, eps, aca_max,
                                                             Kmax, h->opts.truncate_at_cap, h->scratch, ie,
                                                             h->d_stat);
    else
      k_aca_compress<<<cnt, TLR_THREADS, smem, s>>>(h->tab, h->mp, h->x, h->y, h->n, v, t0, eps, aca_max, Kmax,
                                                     h->opts.truncate_at_cap, h->scratch, ie, h->d_stat);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

int tlr_gen_dense_tiles(tlr_ctx* h, const int2* d_items, int count, cudaStream_t s) {
  const TlrView v = view_of(h);
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = count - c0 < 65535 ? count - c0 : 65535;
    dim3 grid(16, cnt);
    k_gen_dense_list<<<grid, 256, 0, s>>>(h->tab, h->mp, h->x, h->y, h->n, v, d_items + c0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

// L_ik = A_ik L_kk^{-T}: low rank V <- L_kk^{-1} V, dense A <- A L_kk^{-T}, by GEMM with the explicit L_kk^{-1}
static int launch_trsm(tlr_ctx* h, int k, cudaStream_t s) {
  const TlrView v = view_of(h);
  const int64_t* off = h->plan_off + (size_t)k * PLAN_PH;
  const int nlr = (int)(off[PH_TRSM_LR + 1] - off[PH_TRSM_LR]);
  const int nd = (int)(off[PH_TRSM_D + 1] - off[PH_TRSM_D]);
  // L_kk^{-1} is kept for the inverse (tile low-rank TRTRI)
  double* Li = h->linv + (size_t)k * h->nb * h->nb;
  int rc = tops_trinv(h->D + (size_t)k * h->nb * h->nb, h->nb, Li, s);
  if (rc) return rc;
  if (nlr + nd == 0) return TLR_OK;
  return tops_trmul(h, v, Li, 0, h->d_list + off[PH_TRSM_LR], nlr, 1, 1, h->d_list + off[PH_TRSM_D], nd, 1, 1.0, s);
}

static int launch_syrk(tlr_ctx* h, int k, cudaStream_t s) {
  const TlrView v = view_of(h);
  const int items = h->nt - k - 1;
  const size_t per = (size_t)h->kcap * h->kcap + (size_t)h->nb * h->kcap;
  const size_t desc_elems = (sizeof(GemmDesc) * (size_t)items + 7) / 8 + 1;
  const int chunk = chunk_for(h, per, desc_elems);
  if (chunk < 1) TLR_RETURN_OOM();
  GemmDesc* desc = (GemmDesc*)h->scratch;
  double* ws = h->scratch + desc_elems;
  const int mb = (h->nb + 63) / 64;
  for (int i0 = 0; i0 < items; i0 += chunk) {
    const int cnt = items - i0 < chunk ? items - i0 : chunk;
    k_syrk_prep<<<cnt, 256, 0, s>>>(v, k, k + 1 + i0, desc, ws, per);
    TLR_LAUNCH_CHECK();
    k_gemm_desc<<<dim3(mb * mb, cnt), 256, 0, s>>>(desc, h->nb);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

static int launch_updates(tlr_ctx* h, int k, cudaStream_t s) {
  const int64_t* off = h->plan_off + (size_t)k * PLAN_PH;
  const int64_t n_lr = off[PH_UPD_LR + 1] - off[PH_UPD_LR];
  // leading items with a dense operand (partitioned first by the plan)
  int64_t ndop = 0;
  if (h->kind) {
    const int2* hl = h->h_list + off[PH_UPD_LR];
    while (ndop < n_lr && (h->kind[tile_index(hl[ndop].x, k)] || h->kind[tile_index(hl[ndop].y, k)])) ++ndop;
  }
  return tops_update(h, view_of(h), ALG_CHOL, k, h->d_list + off[PH_UPD_LR], n_lr, ndop, h->d_list + off[PH_UPD_D],
                     off[PH_UPD_D + 1] - off[PH_UPD_D], h->opts.eps, nullptr, 0.0, s);
}

int tlr_factor(tlr_ctx* h, cudaStream_t s) {
  const int nt = h->nt, nb = h->nb;
  for (int k = 0; k < nt; ++k) {
    int rc;
    {
      PhaseScope ps("chol.potrf", s);
      rc = tlr_potrf_tile(h, h->D + (size_t)k * nb * nb, nb, nb, (int64_t)k * nb, s);
    }
    if (rc) return rc;
    if (k == nt - 1) break;
    {
      PhaseScope ps("chol.trsm", s);
      if ((rc = launch_trsm(h, k, s))) return rc;
    }
    {
      PhaseScope ps("chol.syrk", s);
      if ((rc = launch_syrk(h, k, s))) return rc;
    }
    {
      PhaseScope ps("chol.update", s);
      if ((rc = launch_updates(h, k, s))) return rc;
    }
  }
  // the last diagonal tile's inverse (the others are formed for the TRSM): the solves apply them all
  return tops_trinv(h->D + (size_t)(nt - 1) * nb * nb, nb, h->linv + (size_t)(nt - 1) * nb * nb, s);
}
