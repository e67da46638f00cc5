// Tile low-rank inverse Z = Sigma^{-1} = L^{-T} L^{-1} of the factored matrix
// (needed by the trace term of the likelihood gradient; not in the paper).
//
// Right-looking tile TRTRI (M = L^{-1}, in place on a copy of the factor), step k:
//   1. A_ik <- -A_ik L_kk^{-1}                 i > k  (low rank: V <- -L_kk^{-T} V)
//   2. A_ij <- A_ij + A_ik A_kj                i > k > j
//   3. A_kj <- L_kk^{-1} A_kj                  j < k  (low rank: U <- L_kk^{-1} U)
//   4. A_kk <- L_kk^{-1}
// then right-looking tile LAUUM (Z = M^T M, lower part), step k:
//   1. A_nn <- A_nn + A_kn^T A_kn              n < k
//   2. A_mn <- A_mn + A_km^T A_kn              n < m < k
//   3. A_kn <- A_kk^T A_kn                     n < k  (low rank: U <- M_kk^T U)
//   4. A_kk <- A_kk^T A_kk
// TRTRI keeps L^{-1} in tile low-rank form (its tiles are sources of later
// products) and recompresses at tau_M = eps sqrt(zeta), zeta = max_a 1 / L_aa^2
// (the scale of L^{-1} squared), so the truncation is relative to the size of
// L^{-1} as eps is to Sigma; a dense x dense product landing on a low-rank tile
// is formed by GEMM and recompressed.  Sigma^{-1}'s tiles are never sources:
// only the gradient pass reads them, so LAUUM accumulates every off-diagonal
// tile densely (no truncation): a row of L^{-1} is expanded to dense right
// after its last use as a source.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "recompress.cuh"
#include "tileops.h"

namespace {

__global__ void k_zeta(const double* __restrict__ D, int nb, int nt, double* __restrict__ out) {
  __shared__ double sh[TLR_THREADS];
  double m = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)nt * nb; e += blockDim.x) {
    const int k = (int)(e / nb), a = (int)(e % nb);
    const double d = D[(size_t)k * nb * nb + (size_t)a * nb + a];
    m = fmax(m, 1.0 / (d * d));
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// copy the factor's tiles into the inverse storage (low rank -> dense where Z is dense)
__global__ void k_copy_to_z(TlrView f, TlrView z, int64_t ntiles) {
  const int64_t t = blockIdx.y;
  const int nb = f.nb;
  const bool fd = f.dslot[t] >= 0, zd = z.dslot[t] >= 0;
  if (zd) {
    double* Az = tileA(z, t);
    if (fd) {
      const double* Af = tileA(f, t);
      for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nb * nb;
           e += (int64_t)gridDim.x * blockDim.x)
        Az[e] = Af[e];
    } else {
      const int kr = f.rank[t];
      const double* U = tileU(f, t);
      const double* V = tileV(f, t);
      for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nb * nb;
           e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % nb), b = (int)(e / nb);
        double s = 0.0;
        for (int l = 0; l < kr; ++l) s = fma(U[(size_t)l * nb + a], V[(size_t)l * nb + b], s);
        Az[e] = s;
      }
    }
  } else {
    const int kr = f.rank[t];
    const size_t cnt = (size_t)nb * kr;
    const double* Uf = tileU(f, t);
    const double* Vf = tileV(f, t);
    double* Uz = tileU(z, t);
    double* Vz = tileV(z, t);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
      Uz[e] = Uf[e];
      Vz[e] = Vf[e];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) z.rank[t] = kr;
  }
}

// tiles (r, n), n < r, still low rank: A = U V^T into their own dense slot (slot = tile index)
__global__ void k_expand_row(TlrView z, int r) {
  const int n = blockIdx.y;
  const int64_t t = dtile_index(r, n);
  if (z.dslot[t] >= 0) return;
  const int nb = z.nb;
  cta_gemm_df_blocks(nb, nb, z.rank[t], 1.0, tileU(z, t), nb, 0, tileV(z, t), nb, 1, 0.0,
                     z.dpool + (size_t)t * nb * nb, nb, blockIdx.x, gridDim.x, 0);
}

__global__ void k_mark_row_dense(TlrView z, int r) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= r) return;
  const int64_t t = dtile_index(r, n);
  z.dslot[t] = (int)t;
}

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = a[e];
}

__global__ void k_eye(double* __restrict__ X, int nb) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nb * nb;
       e += (int64_t)gridDim.x * blockDim.x)
    X[e] = ((e % nb) == (e / nb)) ? 1.0 : 0.0;
}

}  // namespace

static TlrView zview(const tlr_ctx* h) {
  TlrView v;
  v.nb = h->nb; v.nt = h->nt; v.kcap = h->kcap;
  v.D = h->Dz; v.U = h->Uz; v.V = h->Vz; v.rank = h->rankz; v.dslot = h->dslotz; v.dpool = h->dpoolz;
  return v;
}

static int zplan(tlr_ctx* h, cudaStream_t s) {
  const int nt = h->nt;
  const int64_t T = h->ntiles;
  free(h->kindz);
  h->kindz = (char*)calloc(std::max<int64_t>(T, 1), 1);
  if (!h->kindz) return TLR_ERR_OOM;
  char* K = h->kindz;
  // Z keeps the factor's dense tiles; a low-rank factor tile whose rank exceeds
  // 2/5 of dense_rank is also made dense in Z (inverse ranks run about 3.5 times
  // the factor's, and the update of a dense tile is a parallel GEMM)
  std::vector<int> rk(std::max<int64_t>(T, 1), 0);
  if (T > 0) {
    TLR_CUDA_TRY(cudaMemcpyAsync(rk.data(), h->rank, T * sizeof(int), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const int zr = std::max(16, (2 * h->dense_rank) / 5);
  for (int64_t t = 0; t < T; ++t) K[t] = (h->kind ? h->kind[t] : 0) || (zr > 0 && rk[t] > zr);
  auto kd = [&](int p, int q) -> char& { return K[tile_index(p, q)]; };
  // No fill closure: the inverse of a banded triangular matrix is full, so the
  // closure would make every tile dense although the far tiles of L^{-1} and
  // Sigma^{-1} are numerically low rank.  A dense x dense product that lands on
  // a low-rank tile is materialised and recompressed instead (phases *_DD).
  // every tile owns dense slot t: L^{-1}'s dense tiles use it during TRTRI, and
  // every tile of Sigma^{-1} is accumulated densely there during LAUUM
  std::vector<int> slot(std::max<int64_t>(T, 1), -1);
  int nd = 0;
  for (int64_t t = 0; t < T; ++t)
    if (K[t]) { slot[t] = (int)t; ++nd; }
  if (T > h->dcapz) {
    if (h->dpoolz) cudaFree(h->dpoolz);
    h->dpoolz = nullptr;
    h->dcapz = 0;
    const int want = (int)std::max<int64_t>(T, 1);
    if (cudaMalloc((void**)&h->dpoolz, (size_t)want * h->nb * h->nb * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return TLR_ERR_OOM;
    }
    h->dcapz = want;
  }
  h->ndensez = nd;
  std::vector<int2> L;
  std::vector<int64_t> off((size_t)nt * ZPH + 1, 0);
  for (int k = 0; k < nt; ++k) {
    for (int ph = 0; ph < ZPH; ++ph) {
      off[(size_t)k * ZPH + ph] = (int64_t)L.size();
      const char want = ph & 1;  // odd phases: dense tiles
      switch (ph) {
        case ZP_T1_LR: case ZP_T1_D:
          for (int i = k + 1; i < nt; ++i) if (kd(i, k) == want) L.push_back(make_int2(i, k));
          break;
        case ZP_T2_LR: case ZP_T2_D: case ZP_T2_DD:
          for (int i = k + 1; i < nt; ++i)
            for (int j = 0; j < k; ++j) {
              const bool dd = kd(i, k) && kd(k, j);
              if (ph == ZP_T2_D ? kd(i, j) == 1 : (kd(i, j) == 0 && dd == (ph == ZP_T2_DD)))
                L.push_back(make_int2(i, j));
            }
          break;
        case ZP_T3_LR: case ZP_T3_D: case ZP_L3_LR: case ZP_L3_D:
          for (int j = 0; j < k; ++j) if (kd(k, j) == want) L.push_back(make_int2(k, j));
          break;
        case ZP_L2_D:  // LAUUM targets are dense (their rows were expanded before)
          for (int m = 1; m < k; ++m)
            for (int n2 = 0; n2 < m; ++n2) L.push_back(make_int2(m, n2));
          break;
        case ZP_L2_LR: case ZP_L2_DD:
          break;
      }
    }
  }
  off[(size_t)nt * ZPH] = (int64_t)L.size();
  if (getenv("TLR_VERBOSE")) {
    int64_t cnt[ZPH] = {0};
    for (int k = 0; k < nt; ++k)
      for (int ph = 0; ph < ZPH; ++ph) cnt[ph] += off[(size_t)k * ZPH + ph + 1] - off[(size_t)k * ZPH + ph];
    fprintf(stderr, "tlr inverse plan: dense %d; items T1 %lld/%lld T2 %lld/%lld/dd %lld T3 %lld/%lld L2 %lld/%lld/dd %lld L3 %lld/%lld\n",
            nd, (long long)cnt[ZP_T1_LR], (long long)cnt[ZP_T1_D], (long long)cnt[ZP_T2_LR], (long long)cnt[ZP_T2_D],
            (long long)cnt[ZP_T2_DD], (long long)cnt[ZP_T3_LR], (long long)cnt[ZP_T3_D], (long long)cnt[ZP_L2_LR],
            (long long)cnt[ZP_L2_D], (long long)cnt[ZP_L2_DD], (long long)cnt[ZP_L3_LR], (long long)cnt[ZP_L3_D]);
  }
  const int64_t len = std::max<int64_t>((int64_t)L.size(), 1);
  if (len > h->zlist_cap) {
    if (h->d_zlist) cudaFree(h->d_zlist);
    h->d_zlist = nullptr;
    if (cudaMalloc((void**)&h->d_zlist, len * sizeof(int2)) != cudaSuccess) {
      cudaGetLastError();
      h->zlist_cap = 0;
      return TLR_ERR_OOM;
    }
    h->zlist_cap = len;
  }
  free(h->h_zlist);
  free(h->zoff);
  h->h_zlist = (int2*)malloc(len * sizeof(int2));
  h->zoff = (int64_t*)malloc(off.size() * sizeof(int64_t));
  if (!h->h_zlist || !h->zoff) return TLR_ERR_OOM;
  if (!L.empty()) memcpy(h->h_zlist, L.data(), L.size() * sizeof(int2));
  memcpy(h->zoff, off.data(), off.size() * sizeof(int64_t));
  if (!L.empty())
    TLR_CUDA_TRY(cudaMemcpyAsync(h->d_zlist, h->h_zlist, L.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  if (T > 0) TLR_CUDA_TRY(cudaMemcpyAsync(h->dslotz, slot.data(), T * sizeof(int), cudaMemcpyHostToDevice, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  h->zplan_valid = 1;
  return TLR_OK;
}

static int ensure_z(tlr_ctx* h) {
  if (h->Dz) return TLR_OK;
  const size_t nb = h->nb, slot = nb * h->kcap;
  const size_t T = std::max<int64_t>(h->cap_ntiles, 1);
  bool ok = cudaMalloc((void**)&h->Dz, (size_t)h->cap_nt * nb * nb * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->Uz, (h->dense ? 1 : T * slot) * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->Vz, (h->dense ? 1 : T * slot) * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->rankz, T * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->dslotz, T * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return TLR_ERR_OOM;
  }
  return TLR_OK;
}

#define ZTRY(x)                    \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != TLR_OK) return rc_; \
  } while (0)

int tlr_inverse(tlr_ctx* h, cudaStream_t s) {
  ZTRY(ensure_z(h));
  if (!h->zplan_valid) ZTRY(zplan(h, s));
  const int nt = h->nt, nb = h->nb;
  const TlrView f = view_of(h);
  const TlrView z = zview(h);
  const size_t nn = (size_t)nb * nb;
  // zeta lives in the last reduction slot
  double* d_zeta = h->d_red + h->red_len - 1;
  PhaseScope ps_all("inverse", s);
  k_zeta<<<1, TLR_THREADS, 0, s>>>(h->D, nb, nt, d_zeta);
  TLR_LAUNCH_CHECK();
  k_copy<<<1024, 256, 0, s>>>(h->D, h->Dz, (int64_t)nt * nn);
  TLR_LAUNCH_CHECK();
  TLR_CUDA_TRY(cudaMemsetAsync(h->rankz, 0, std::max<int64_t>(h->ntiles, 1) * sizeof(int), s));
  if (h->ntiles > 0) {
    for (int64_t t0 = 0; t0 < h->ntiles; t0 += 65535) {
      // one grid row per tile (gridDim.y), offset via pointer arithmetic is not possible: launch per chunk
      const int64_t cnt = std::min<int64_t>(65535, h->ntiles - t0);
      TlrView fo = f, zo = z;
      fo.rank = f.rank + t0; fo.dslot = f.dslot + t0;
      zo.rank = z.rank + t0; zo.dslot = z.dslot + t0;
      fo.U = f.U ? f.U + (size_t)t0 * nb * h->kcap : f.U; fo.V = f.V ? f.V + (size_t)t0 * nb * h->kcap : f.V;
      zo.U = z.U ? z.U + (size_t)t0 * nb * h->kcap : z.U; zo.V = z.V ? z.V + (size_t)t0 * nb * h->kcap : z.V;
      if (h->dense) { fo.U = f.U; fo.V = f.V; zo.U = z.U; zo.V = z.V; }
      k_copy_to_z<<<dim3(8, (unsigned)cnt), 256, 0, s>>>(fo, zo, cnt);
      TLR_LAUNCH_CHECK();
    }
  }
  const double eps = (h->opts.eps > 0 ? h->opts.eps : 0.0) * (h->opts.inv_scale > 0 ? h->opts.inv_scale : 0.1);
  double* X = h->scratch;  // nb x nb workspace for the diagonal tiles
  // ---- TRTRI
  for (int k = 0; k < nt; ++k) {
    const int64_t* off = h->zoff + (size_t)k * ZPH;
    auto L = [&](int ph) { return h->d_zlist + off[ph]; };
    auto N = [&](int ph) { return (int)(off[ph + 1] - off[ph]); };
    double* Mi = h->dinv;  // L_kk^{-1}, applied by GEMM in steps 1 and 3, stored in step 4
    { PhaseScope ps("trtri.diag", s);
      k_eye<<<256, 256, 0, s>>>(Mi, nb);
      TLR_LAUNCH_CHECK();
      ZTRY(tops_trop_raw(h->Dz + (size_t)k * nn, nb, Mi, nb, TOP_SOLVE, 1.0, s)); }
    { PhaseScope ps("trtri.col", s);  // A_ik <- -A_ik L_kk^{-1}: V <- -L_kk^{-T} V
      ZTRY(tops_trmul(h, z, Mi, 1, L(ZP_T1_LR), N(ZP_T1_LR), 1, 0, L(ZP_T1_D), N(ZP_T1_D), 1, -1.0, s)); }
    { PhaseScope ps("trtri.update", s);
      ZTRY(tops_update(h, z, ALG_TRTRI, k, L(ZP_T2_LR), N(ZP_T2_LR), L(ZP_T2_D), N(ZP_T2_D), eps, d_zeta, 0.5, s)); }
    { PhaseScope ps("trtri.update_dd", s);
      ZTRY(tops_update_dd(h, z, ALG_TRTRI, k, L(ZP_T2_DD), N(ZP_T2_DD), eps, d_zeta, 0.5, s)); }
    { PhaseScope ps("trtri.row", s);  // A_kj <- L_kk^{-1} A_kj: U <- L_kk^{-1} U
      ZTRY(tops_trmul(h, z, Mi, 0, L(ZP_T3_LR), N(ZP_T3_LR), 0, 0, L(ZP_T3_D), N(ZP_T3_D), 0, 1.0, s)); }
    PhaseScope ps_d("trtri.store", s);
    k_copy<<<256, 256, 0, s>>>(Mi, h->Dz + (size_t)k * nn, (int64_t)nn);
    TLR_LAUNCH_CHECK();
  }
  // ---- LAUUM
  GemmGen* desc = (GemmGen*)(h->scratch + nn);
  const int mb = (nb + 63) / 64;
  auto expand_row = [&](int r) -> int {
    if (r < 1) return TLR_OK;
    k_expand_row<<<dim3(mb * mb, r), 256, 0, s>>>(z, r);
    TLR_LAUNCH_CHECK();
    k_mark_row_dense<<<(r + 127) / 128, 128, 0, s>>>(z, r);
    TLR_LAUNCH_CHECK();
    return TLR_OK;
  };
  for (int k = 0; k < nt; ++k) {
    const int64_t* off = h->zoff + (size_t)k * ZPH;
    auto L = [&](int ph) { return h->d_zlist + off[ph]; };
    auto N = [&](int ph) { return (int)(off[ph + 1] - off[ph]); };
    // row k-1 was a source for the last time in step k-1: from now on its tiles are
    // dense targets of Sigma^{-1}
    { PhaseScope ps("lauum.expand", s); ZTRY(expand_row(k - 1)); }
    { PhaseScope ps("lauum.herk", s); ZTRY(tops_herk_row(h, z, k, s)); }
    { PhaseScope ps("lauum.update", s);
      ZTRY(tops_update(h, z, ALG_LAUUM, k, L(ZP_L2_LR), N(ZP_L2_LR), L(ZP_L2_D), N(ZP_L2_D), eps, d_zeta, 1.0, s)); }
    { PhaseScope ps("lauum.update_dd", s);
      ZTRY(tops_update_dd(h, z, ALG_LAUUM, k, L(ZP_L2_DD), N(ZP_L2_DD), eps, d_zeta, 1.0, s)); }
    { PhaseScope ps("lauum.row", s);  // A_kn <- A_kk^T A_kn
      ZTRY(tops_trmul(h, z, h->Dz + (size_t)k * nn, 1, L(ZP_L3_LR), N(ZP_L3_LR), 0, 1, L(ZP_L3_D), N(ZP_L3_D), 0, 1.0,
                      s)); }
    PhaseScope ps_d("lauum.diag", s);
    // D_k <- D_k^T D_k via the workspace
    GemmGen g;
    g.A = h->Dz + (size_t)k * nn; g.B = g.A; g.C = X; g.m = nb; g.n = nb; g.k = nb;
    g.lda = nb; g.ldb = nb; g.ldc = nb; g.tA = 1; g.tB = 0; g.alpha = 1.0; g.beta = 0.0; g.lower = 0;
    TLR_CUDA_TRY(cudaMemcpyAsync(desc, &g, sizeof(g), cudaMemcpyHostToDevice, s));
    ZTRY(tops_gemm(desc, 1, nb, nb, s));
    k_copy<<<256, 256, 0, s>>>(X, h->Dz + (size_t)k * nn, (int64_t)nn);
    TLR_LAUNCH_CHECK();
  }
  { PhaseScope ps("lauum.expand", s); ZTRY(expand_row(nt - 1)); }
  h->zplan_valid = 0;  // the device tile kinds of Z changed: the next inverse re-plans
  return TLR_OK;
}
