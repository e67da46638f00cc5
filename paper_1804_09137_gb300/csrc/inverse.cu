// Tile low-rank inverse Z = Sigma^{-1} = L^{-T} L^{-1} of the factored matrix
// (needed by the trace term of the likelihood gradient; not in the paper).
//
// Right-looking tile TRTRI (M = L^{-1}, in place on a copy of the factor), step k:
//   1. A_ik <- -A_ik L_kk^{-1}                 i > k  (low rank: V <- -L_kk^{-T} V)
//   2. A_ij <- A_ij + A_ik A_kj                i > k > j
//   3. A_kj <- L_kk^{-1} A_kj                  j < k  (low rank: U <- L_kk^{-1} U)
//   4. A_kk <- L_kk^{-1}
// then left-looking tile LAUUM (Z = M^T M, lower part, out of place):
//   Z_mn = sum_{k >= m} M_km^T M_kn           m >= n
// with every tile of Z one GEMM over the stacked thin factors of its products.
// TRTRI keeps L^{-1} in tile low-rank form (its tiles are sources of later
// products) and recompresses at tau_M = eps sqrt(zeta), zeta = max_a 1 / L_aa^2
// (the scale of L^{-1} squared), so the truncation is relative to the size of
// L^{-1} as eps is to Sigma; a dense x dense product landing on a low-rank tile
// is formed by GEMM and recompressed.  Sigma^{-1}'s tiles are never sources:
// only the gradient pass reads them, so LAUUM forms every tile densely (no
// truncation).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "recompress.cuh"
#include "tcgemm.h"
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

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = a[e];
}


}  // namespace

static TlrView zview(const tlr_ctx* h) {
  TlrView v;
  v.nb = h->nb; v.nt = h->nt; v.kcap = h->kcap;
  v.D = h->Dz; v.U = h->Uz; v.V = h->Vz; v.rank = h->rankz; v.dslot = h->dslotz; v.dpool = h->dpoolz;
  v.off = h->offz; v.cap = h->capz; v.top = h->topz; v.arena = h->arenaz;
  return v;
}

#define ZTRY_OOM(x)                \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != TLR_OK) return rc_; \
  } while (0)

static int zplan(tlr_ctx* h, cudaStream_t s) {
  const int nt = h->nt;
  const int64_t T = h->ntiles;
  free(h->kindz);
  h->kindz = (char*)calloc(std::max<int64_t>(T, 1), 1);
  if (!h->kindz) TLR_RETURN_OOM();
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
  // (with the gradient fused into the products Sigma^{-1} is never stored: the dense tiles of L^{-1}
  // get compact slots instead)
  const bool compact = tlr_tc_slices_opt(h) > 0;
  std::vector<int> slot(std::max<int64_t>(T, 1), -1);
  int nd = 0;
  for (int64_t t = 0; t < T; ++t)
    if (K[t]) { slot[t] = compact ? nd : (int)t; ++nd; }
  free(h->hslotz);
  h->hslotz = (int*)malloc(std::max<int64_t>(T, 1) * sizeof(int));
  if (!h->hslotz) TLR_RETURN_OOM();
  memcpy(h->hslotz, slot.data(), std::max<int64_t>(T, 1) * sizeof(int));
  const int64_t pool_want = compact ? std::max(nd, 1) : std::max<int64_t>(T, 1);
  if (pool_want > h->dcapz) {
    if (h->dpoolz) cudaFree(h->dpoolz);
    h->dpoolz = nullptr;
    h->dcapz = 0;
    const int want = (int)pool_want;
    if (cudaMalloc((void**)&h->dpoolz, (size_t)want * h->nb * h->nb * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      TLR_RETURN_OOM();
    }
    h->dcapz = want;
  }
  h->ndensez = nd;
  // Z's arena: the low-rank tiles packed by their factor ranks (with room to grow), plus headroom for
  // the blocks that TRTRI's higher ranks take
  {
    std::vector<int64_t> zo(std::max<int64_t>(T, 1), 0);
    std::vector<int> zc(std::max<int64_t>(T, 1), 0);
    int64_t pos = 0;
    for (int64_t t = 0; t < T; ++t) {
      if (K[t] || rk[t] <= 0) continue;
      int c = rk[t] + rk[t] / 4 + 8;
      c = std::min((c + 7) & ~7, h->kcap);
      zo[t] = pos;
      zc[t] = c;
      pos += (int64_t)c * h->nb;
    }
    const int64_t need = h->dense ? 1 : 2 * pos + std::max<int64_t>(T, 1) * h->nb * 16;
    if (need > h->arenaz) {
      TLR_CUDA_TRY(cudaStreamSynchronize(s));
      ZTRY_OOM(tlr_arena_alloc(&h->Uz, &h->Vz, &h->arenaz, need));
    }
    const unsigned long long top = (unsigned long long)pos;
    if (T > 0) {
      TLR_CUDA_TRY(cudaMemcpyAsync(h->offz, zo.data(), T * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      TLR_CUDA_TRY(cudaMemcpyAsync(h->capz, zc.data(), T * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    TLR_CUDA_TRY(cudaMemcpyAsync(h->topz, &top, sizeof(top), cudaMemcpyHostToDevice, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors die here
  }
  std::vector<int2> L;
  std::vector<int64_t> off((size_t)nt * ZPH + ZG + 1, 0);
  for (int k = 0; k < nt; ++k) {
    for (int ph = 0; ph < ZPH; ++ph) {
      off[(size_t)k * ZPH + ph] = (int64_t)L.size();
      const size_t b = L.size();
      for (int i = k + 1; i < nt; ++i)
        for (int j = 0; j < k; ++j) {
          const bool dd = kd(i, k) && kd(k, j);
          if (ph == ZP_T2_D ? kd(i, j) == 1 : (kd(i, j) == 0 && dd == (ph == ZP_T2_DD)))
            L.push_back(make_int2(i, j));
        }
      if (ph == ZP_T2_LR) {
        // longest recompressions first (cost ~ square of the concatenated rank,
        // estimated from the factor's ranks), so a launch does not end on a tail
        auto r = [&](int p, int q) { return kd(p, q) ? h->nb : std::max(rk[tile_index(p, q)], 1); };
        auto est = [&](int2 t) { const int K = r(t.x, t.y) + std::min(r(t.x, k), r(k, t.y)); return K * K; };
        std::stable_sort(L.begin() + b, L.end(), [&](int2 a, int2 c) { return est(a) > est(c); });
        // items with a dense operand first: their products are formed by a batched GEMM before the launch
        std::stable_partition(L.begin() + b, L.end(), [&](int2 t) { return kd(t.x, k) || kd(k, t.y); });
      }
    }
  }
  // column transforms (tiles (i, k), i > k) and row transforms (tiles (k, j), j < k) of every step
  for (int g = 0; g < ZG; ++g) {
    off[(size_t)nt * ZPH + g] = (int64_t)L.size();
    const char want = g & 1;  // odd lists: dense tiles
    for (int k = 0; k < nt; ++k) {
      if (g <= ZG_T1_D) {
        for (int i = k + 1; i < nt; ++i) if (kd(i, k) == want) L.push_back(make_int2(i, k));
      } else {
        for (int j = 0; j < k; ++j) if (kd(k, j) == want) L.push_back(make_int2(k, j));
      }
    }
  }
  off[(size_t)nt * ZPH + ZG] = (int64_t)L.size();
  if (getenv("TLR_VERBOSE")) {
    int64_t cnt[ZPH] = {0};
    for (int k = 0; k < nt; ++k)
      for (int ph = 0; ph < ZPH; ++ph) cnt[ph] += off[(size_t)k * ZPH + ph + 1] - off[(size_t)k * ZPH + ph];
    const int64_t* g = off.data() + (size_t)nt * ZPH;
    fprintf(stderr, "tlr inverse plan: dense %d; items T1 %lld/%lld T2 %lld/%lld/dd %lld T3 %lld/%lld\n", nd,
            (long long)(g[1] - g[0]), (long long)(g[2] - g[1]), (long long)cnt[ZP_T2_LR], (long long)cnt[ZP_T2_D],
            (long long)cnt[ZP_T2_DD], (long long)(g[3] - g[2]), (long long)(g[4] - g[3]));
  }
  const int64_t len = std::max<int64_t>((int64_t)L.size(), 1);
  if (len > h->zlist_cap) {
    if (h->d_zlist) cudaFree(h->d_zlist);
    h->d_zlist = nullptr;
    if (cudaMalloc((void**)&h->d_zlist, len * sizeof(int2)) != cudaSuccess) {
      cudaGetLastError();
      h->zlist_cap = 0;
      TLR_RETURN_OOM();
    }
    h->zlist_cap = len;
  }
  free(h->h_zlist);
  free(h->zoff);
  h->h_zlist = (int2*)malloc(len * sizeof(int2));
  h->zoff = (int64_t*)malloc(off.size() * sizeof(int64_t));
  if (!h->h_zlist || !h->zoff) TLR_RETURN_OOM();
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
  const size_t nb = h->nb;
  const size_t T = std::max<int64_t>(h->cap_ntiles, 1);
  bool ok = cudaMalloc((void**)&h->Dz, (size_t)h->cap_nt * nb * nb * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->rankz, T * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->dslotz, T * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->offz, T * sizeof(int64_t)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->capz, T * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&h->topz, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    TLR_RETURN_OOM();
  }
  return TLR_OK;
}

#define ZTRY(x)                    \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != TLR_OK) return rc_; \
  } while (0)

struct CopySeg {
  const double* src;
  double* dst;
  int64_t count;
};

__global__ void k_seg_copy(const CopySeg* __restrict__ segs) {
  const CopySeg c = segs[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < c.count; e += (int64_t)gridDim.x * blockDim.x)
    c.dst[e] = c.src[e];
}

__global__ void k_mark_all_dense(int* __restrict__ dslot, int64_t T) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x)
    dslot[t] = (int)t;
}

static int seg_copy(const CopySeg* d_segs, int64_t n, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < n; c0 += 65535) {
    const int cnt = (int)std::min<int64_t>(65535, n - c0);
    k_seg_copy<<<dim3(32, cnt), 256, 0, s>>>(d_segs + c0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

// Left-looking LAUUM: every tile of Z = M^T M (M = L^{-1} after TRTRI, lower) at once,
//   Z_mn = sum_{k >= m} M_km^T M_kn,  m >= n  (M_mm the inverse diagonal tile).
// A product with a low-rank factor is a pair of thin panels, Z_mn += A B^T:
//   both low rank:  G = U_km^T U_kn;  A = V_km, B = V_kn G^T  or  A = V_km G, B = V_kn  (thinner side)
//   M_km dense:     A = M_km^T U_kn,  B = V_kn
//   M_kn dense:     A = V_km,         B = M_kn^T U_km
// The pairs of one tile are stacked along the depth, so each tile of Z is one GEMM
// of depth sum(rank) written once; dense x dense products are added afterwards, one
// GEMM per tile and launch.  Z overwrites the dense sources' slots, so those (and the
// diagonal) are read from a copy.  Workspace: h->scratch (descriptors, G, panels).
static int ensure_aux(tlr_ctx* h, int items);

// LAUUM with the gradient: the tensor-core products of a batch write its tiles of Sigma^{-1} into one of
// two buffers and a CUDA-core kernel on another stream reduces them into the gradient while the next
// batch's products run (the float64 derivative work beside the tensor cores), unless the environment
// variable TLR_LAUUM_OVERLAP is 0 (then the product kernel's epilogue does the reduction itself)
static bool lauum_overlap_mode() {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("TLR_LAUUM_OVERLAP");
    mode = (e && atoi(e) == 0) ? 0 : 1;
  }
  return mode == 1;
}

static int lauum_left(tlr_ctx* h, cudaStream_t s_user, const double* alpha, double* out3) {
  cudaStream_t s = s_user;  // the LAUUM's own stream (the second, higher-priority one when overlapping)
  const int nt = h->nt, nb = h->nb;
  const int64_t T = h->ntiles;
  const size_t nn = (size_t)nb * nb;
  std::vector<int> rk(std::max<int64_t>(T, 1), 0);
  if (T > 0) {
    TLR_CUDA_TRY(cudaMemcpyAsync(rk.data(), h->rankz, T * sizeof(int), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const char* K = h->kindz;
  std::vector<int> dix(std::max<int64_t>(T, 1), -1);
  int nd = 0;
  for (int64_t t = 0; t < T; ++t)
    if (K[t]) dix[t] = nd++;
  // fused: Sigma^{-1} is never stored; the tiles of each target are reduced into the gradient by the
  // tensor-core epilogue, and the dense sources are read where TRTRI left them (Dz, compact dense pool)
  const int S = tlr_tc_slices(h);
  const bool fused = S > 0 && alpha && out3;
  const bool overlap = fused && lauum_overlap_mode();
  const int mb64 = (nb + 63) / 64;  // 64 x 64 blocks a side of a tile (the batch reduction's partials)
  const size_t msave_want = fused ? 0 : (size_t)(nt + nd) * nn;
  if (msave_want > h->msave_elems) {
    if (h->msave) cudaFree(h->msave);
    h->msave = nullptr;
    h->msave_elems = 0;
    if (cudaMalloc((void**)&h->msave, msave_want * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      TLR_RETURN_OOM();
    }
    h->msave_elems = msave_want;
  }
  auto isD = [&](int p, int q) { return p == q || K[tile_index(p, q)]; };
  auto Msrc = [&](int p, int q) -> const double* {
    if (fused) return p == q ? h->Dz + (size_t)p * nn : h->dpoolz + (size_t)h->hslotz[tile_index(p, q)] * nn;
    return p == q ? h->msave + (size_t)p * nn : h->msave + (size_t)(nt + dix[tile_index(p, q)]) * nn;
  };
  std::vector<int64_t> zoff(std::max<int64_t>(T, 1), 0);
  if (T > 0) {
    TLR_CUDA_TRY(cudaMemcpyAsync(zoff.data(), h->offz, T * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  auto Uof = [&](int p, int q) -> const double* { return h->Uz + zoff[tile_index(p, q)]; };
  auto Vof = [&](int p, int q) -> const double* { return h->Vz + zoff[tile_index(p, q)]; };
  auto rnk = [&](int p, int q) { return rk[tile_index(p, q)]; };
  auto Zdst = [&](int m, int n) -> double* {
    return m == n ? h->Dz + (size_t)n * nn : h->dpoolz + (size_t)tile_index(m, n) * nn;
  };
  static_assert(sizeof(GemmGen) % 8 == 0 && sizeof(CopySeg) % 8 == 0, "descriptor regions are 8-byte padded");
  const size_t gd = sizeof(GemmGen) / 8, cd = sizeof(CopySeg) / 8;
  if (!fused) {  // dense sources and diagonal tiles into the copy
    std::vector<CopySeg> cs;
    cs.push_back({h->Dz, h->msave, (int64_t)nt * (int64_t)nn});
    for (int64_t t = 0; t < T; ++t)
      if (K[t]) cs.push_back({h->dpoolz + (size_t)t * nn, h->msave + (size_t)(nt + dix[t]) * nn, (int64_t)nn});
    if (cs.size() * cd > h->scratch_elems) TLR_RETURN_OOM();
    TLR_CUDA_TRY(cudaMemcpyAsync(h->scratch, cs.data(), cs.size() * sizeof(CopySeg), cudaMemcpyHostToDevice, s));
    ZTRY(seg_copy((const CopySeg*)h->scratch, (int64_t)cs.size(), s));
  }
  // targets (m, n), m >= n, and their depth
  std::vector<int2> tg;
  std::vector<int64_t> depth, gel;
  std::vector<int> ndd;  // dense x dense products per target
  for (int m = 0; m < nt; ++m)
    for (int n = 0; n <= m; ++n) {
      int64_t d = 0, g = 0;
      int cdd = 0;
      for (int k = m; k < nt; ++k) {
        const bool dm = isD(k, m), dn = isD(k, n);
        if (dm && dn) { ++cdd; continue; }
        if (!dm && !dn) {
          const int a = rnk(k, m), c = rnk(k, n);
          if (a == 0 || c == 0) continue;
          d += std::min(a, c);
          g += (int64_t)a * c;
        } else {
          d += dm ? rnk(k, n) : rnk(k, m);
        }
      }
      tg.push_back(make_int2(m, n));
      depth.push_back(d);
      gel.push_back(g);
      ndd.push_back(cdd);
    }
  // tensor-core path of the stacked-panel products: bf16 slices of both panels, row exponents,
  // split and GEMM descriptors, per target tile (doubles of workspace)
  const int rows_a = (nb + OZ_BM - 1) / OZ_BM * OZ_BM, rows_b = (nb + OZ_BN - 1) / OZ_BN * OZ_BN;
  const size_t od = (2 * sizeof(OzSrc) + sizeof(OzGemm) + 7) / 8;
  auto slice_dbl = [&](int64_t d) -> size_t {
    if (!S || d == 0) return 0;
    return (oz_slices_elems(nb, (int)d, OZ_BM, S) + oz_slices_elems(nb, (int)d, OZ_BN, S)) / 4 +
           (size_t)(rows_a + rows_b + 1) / 2 + od + 48;
  };
  auto pad = [](int64_t d) { return (d + OZ_BK - 1) / OZ_BK * OZ_BK; };
  // depth of a fused target's operands: its panel and one segment per dense x dense product
  auto fdepth = [&](size_t q) { return pad(depth[q]) + (int64_t)ndd[q] * pad(nb); };
  auto tgt_slices = [&](size_t q) -> size_t {
    return fused ? slice_dbl(fdepth(q)) + (size_t)ndd[q] * (2 * sizeof(OzSrc) + 7) / 8 : slice_dbl(depth[q]);
  };
  // partial sums of the fused gradient: eight per CTA tile of every target (two per 64 x 64 block when
  // overlapping, then the targets' list after them)
  const int tiles_per = ((nb + OZ_BM - 1) / OZ_BM) * ((nb + OZ_BN - 1) / OZ_BN);
  const int64_t part_pairs = overlap ? (int64_t)tg.size() * mb64 * mb64 : (int64_t)tg.size() * tiles_per * 4;
  if (fused) {
    const size_t want = 2 * (size_t)part_pairs + (overlap ? tg.size() : 0);
    if (want > h->gpart_elems) {
      if (h->gpart) cudaFree(h->gpart);
      h->gpart = nullptr;
      h->gpart_elems = 0;
      if (cudaMalloc((void**)&h->gpart, want * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        TLR_RETURN_OOM();
      }
      h->gpart_elems = want;
    }
    TLR_CUDA_TRY(cudaMemsetAsync(h->gpart, 0, 2 * (size_t)part_pairs * sizeof(double), s));
  }
  const int2* d_tg = overlap ? reinterpret_cast<const int2*>(h->gpart + 2 * part_pairs) : nullptr;
  if (overlap) {
    static_assert(sizeof(int2) == sizeof(double), "one target a double");
    TLR_CUDA_TRY(cudaMemcpyAsync((void*)d_tg, tg.data(), tg.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  }
  // one target alone must fit (with the reserve for a full-depth product): grow the workspace if not
  {
    size_t worst = 0;
    for (size_t q = 0; q < tg.size(); ++q) {
      const size_t per = (size_t)(nt - tg[q].x) * (3 * gd + cd + 2) + gd + (size_t)gel[q] +
                         2 * (size_t)nb * depth[q] + 8 + tgt_slices(q);
      worst = std::max(worst, per);
    }
    worst += 64 + slice_dbl(nb) + (overlap ? 2 * nn + 32 : 0);
    if (worst > h->scratch_elems) {
      TLR_CUDA_TRY(cudaStreamSynchronize(s));
      cudaFree(h->scratch);
      h->scratch = nullptr;
      h->scratch_elems = 0;
      const size_t want = worst + worst / 4;
      if (cudaMalloc((void**)&h->scratch, want * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        TLR_RETURN_OOM();
      }
      h->scratch_elems = want;
    }
  }
  size_t budget = h->scratch_elems;
  // overlapping: two buffers of zcap tiles of Sigma^{-1} at the top of the workspace, zcap chosen so that
  // the targets' average preparation needs and their tiles share it
  size_t zcap = 0;
  double* zb2[2] = {nullptr, nullptr};
  if (overlap && !tg.empty()) {
    size_t tot = 0;
    for (size_t q = 0; q < tg.size(); ++q)
      tot += (size_t)(nt - tg[q].x) * (3 * gd + cd + 2) + gd + (size_t)gel[q] + 2 * (size_t)nb * depth[q] + 8 +
             tgt_slices(q);
    const size_t avg = tot / tg.size() + 1;
    const size_t fixed = 64 + slice_dbl(nb) + 32;
    zcap = budget > fixed ? (budget - fixed) / (avg + 2 * nn) : 0;
    zcap = std::max<size_t>(1, std::min<size_t>(zcap, std::min<size_t>(tg.size(), 65535)));
    size_t worst1 = 0;
    for (size_t q = 0; q < tg.size(); ++q)
      worst1 = std::max(worst1, (size_t)(nt - tg[q].x) * (3 * gd + cd + 2) + gd + (size_t)gel[q] +
                                    2 * (size_t)nb * depth[q] + 8 + tgt_slices(q));
    while (zcap > 1 && worst1 + fixed + 2 * zcap * nn > budget) --zcap;
    budget -= 2 * zcap * nn + 32;
    double* zr = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(h->scratch + budget) + 127) & ~(uintptr_t)127);
    zb2[0] = zr;
    zb2[1] = zr + zcap * nn;
    // the batch loop runs on the second stream (after everything so far on the caller's), the reductions
    // on the caller's
    ZTRY(ensure_aux(h, 0));
    for (int i = 0; i < 2; ++i) {
      if (!h->ev_lz[i]) TLR_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_lz[i], cudaEventDisableTiming));
      if (!h->ev_lg[i]) TLR_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_lg[i], cudaEventDisableTiming));
    }
    TLR_CUDA_TRY(cudaEventRecord(h->ev_fork, s_user));
    TLR_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    s = h->aux;
  }
  // on every way out, including an error inside the batch loop, the caller's stream waits for the
  // second one, so that nothing the LAUUM enqueued there outlives the call unordered
  struct Join {
    tlr_ctx* h;
    cudaStream_t from, to;
    ~Join() {
      if (from != to && cudaEventRecord(h->ev_join, from) == cudaSuccess) cudaStreamWaitEvent(to, h->ev_join, 0);
    }
  } join{h, s, s_user};
  int nbatch = 0;
  size_t b0 = 0;
  std::vector<char> host;
  while (b0 < tg.size()) {
    // greedy batch: descriptors, copy segments, G and both panels within the workspace
    // (plus room for one nb x nb x nb product on the tensor cores: the dense sources' products)
    size_t b1 = b0, need = 64 + slice_dbl(nb);
    while (b1 < tg.size()) {
      const int m = tg[b1].x;
      const size_t per = (size_t)(nt - m) * (3 * gd + cd + 2) + gd + (size_t)gel[b1] + 2 * (size_t)nb * depth[b1] + 8 +
                         tgt_slices(b1);
      if (b1 > b0 && (need + per > budget || (overlap && b1 - b0 >= zcap))) break;
      need += per;
      ++b1;
    }
    if (need > budget) TLR_RETURN_OOM();
    std::vector<GemmGen> g1, g1b, g2, gbig;
    std::vector<std::vector<GemmGen>> gdd;
    std::vector<CopySeg> cs;
    // region sizes first (pointers into the workspace below)
    size_t n_g1 = 0, n_g1b = 0, n_g2 = 0, n_cs = 0, g_tot = 0, p_tot = 0;
    for (size_t q = b0; q < b1; ++q) {
      const int m = tg[q].x, n = tg[q].y;
      for (int k = m; k < nt; ++k) {
        const bool dm = isD(k, m), dn = isD(k, n);
        if (dm && dn) continue;
        if (!dm && !dn) {
          if (rnk(k, m) == 0 || rnk(k, n) == 0) continue;
          ++n_g1; ++n_g2; ++n_cs;
        } else {
          if ((dm ? rnk(k, n) : rnk(k, m)) == 0) continue;
          ++n_g1b; ++n_cs;
        }
      }
      g_tot += gel[q];
      p_tot += 2 * (size_t)nb * depth[q];
    }
    const size_t nbig = b1 - b0;
    double* base = h->scratch;
    GemmGen* dg1 = (GemmGen*)base;
    GemmGen* dg1b = dg1 + n_g1;
    GemmGen* dg2 = dg1b + n_g1b;
    GemmGen* dbig = dg2 + n_g2;
    GemmGen* ddd = dbig + nbig;
    size_t n_dd = 0;
    for (size_t q = b0; q < b1 && !fused; ++q)
      for (int k = tg[q].x; k < nt; ++k) n_dd += isD(k, tg[q].x) && isD(k, tg[q].y);
    CopySeg* dcs = (CopySeg*)(ddd + n_dd);
    double* Gw = base + ((size_t)(n_g1 + n_g1b + n_g2 + nbig + n_dd) * gd + n_cs * cd + 8);
    double* Pw = Gw + g_tot + 8;
    if ((size_t)(Pw + p_tot - base) > budget) TLR_RETURN_OOM();
    GemmGen z0;
    memset(&z0, 0, sizeof(z0));
    z0.alpha = 1.0; z0.beta = 0.0;
    auto gemm = [&](int mm, int nn2, int kk, const double* A, int lda, int tA, const double* B, int ldb, int tB,
                    double* C, int ldc, double beta) {
      GemmGen g = z0;
      g.m = mm; g.n = nn2; g.k = kk; g.A = A; g.lda = lda; g.tA = tA; g.B = B; g.ldb = ldb; g.tB = tB;
      g.C = C; g.ldc = ldc; g.beta = beta;
      return g;
    };
    int mx_g = 1, mx_r = 1;
    size_t goff = 0;
    double* P = Pw;
    std::vector<std::vector<int>> ddk(b1 - b0);  // fused: the dense x dense sources of each target
    for (size_t q = b0; q < b1; ++q) {
      const int m = tg[q].x, n = tg[q].y;
      double* Ap = P;
      double* Bp = P + (size_t)nb * depth[q];
      int64_t off = 0;
      int r_dd = 0;
      for (int k = m; k < nt; ++k) {
        const bool dm = isD(k, m), dn = isD(k, n);
        if (dm && dn) {
          if (fused) {
            ddk[q - b0].push_back(k);
            continue;
          }
          if ((int)gdd.size() <= r_dd) gdd.emplace_back();
          gdd[r_dd++].push_back(gemm(nb, nb, nb, Msrc(k, m), nb, 1, Msrc(k, n), nb, 0, Zdst(m, n), nb, 1.0));
          continue;
        }
        if (!dm && !dn) {
          const int a = rnk(k, m), c = rnk(k, n);
          if (a == 0 || c == 0) continue;
          double* G = Gw + goff;
          goff += (size_t)a * c;
          g1.push_back(gemm(a, c, nb, Uof(k, m), nb, 1, Uof(k, n), nb, 0, G, a, 0.0));
          mx_g = std::max(mx_g, std::max(a, c));
          if (a <= c) {  // A = V_km, B = V_kn G^T (depth a)
            cs.push_back({Vof(k, m), Ap + (size_t)off * nb, (int64_t)nb * a});
            g2.push_back(gemm(nb, a, c, Vof(k, n), nb, 0, G, a, 1, Bp + (size_t)off * nb, nb, 0.0));
            off += a;
            mx_r = std::max(mx_r, a);
          } else {  // A = V_km G, B = V_kn (depth c)
            g2.push_back(gemm(nb, c, a, Vof(k, m), nb, 0, G, a, 0, Ap + (size_t)off * nb, nb, 0.0));
            cs.push_back({Vof(k, n), Bp + (size_t)off * nb, (int64_t)nb * c});
            off += c;
            mx_r = std::max(mx_r, c);
          }
        } else if (dm) {  // A = M_km^T U_kn, B = V_kn
          const int c = rnk(k, n);
          if (c == 0) continue;
          g1b.push_back(gemm(nb, c, nb, Msrc(k, m), nb, 1, Uof(k, n), nb, 0, Ap + (size_t)off * nb, nb, 0.0));
          cs.push_back({Vof(k, n), Bp + (size_t)off * nb, (int64_t)nb * c});
          off += c;
          mx_r = std::max(mx_r, c);
        } else {  // A = V_km, B = M_kn^T U_km
          const int a = rnk(k, m);
          if (a == 0) continue;
          cs.push_back({Vof(k, m), Ap + (size_t)off * nb, (int64_t)nb * a});
          g1b.push_back(gemm(nb, a, nb, Msrc(k, n), nb, 1, Uof(k, m), nb, 0, Bp + (size_t)off * nb, nb, 0.0));
          off += a;
          mx_r = std::max(mx_r, a);
        }
      }
      if (off != depth[q]) return TLR_ERR_STATE;
      gbig.push_back(gemm(nb, nb, (int)off, Ap, nb, 0, Bp, nb, 1, fused ? nullptr : Zdst(m, n), nb, 0.0));
      P += 2 * (size_t)nb * depth[q];
    }
    // one upload of descriptors and copy segments, in the order of the device layout
    std::vector<GemmGen> all;
    all.reserve(g1.size() + g1b.size() + g2.size() + gbig.size() + n_dd);
    all.insert(all.end(), g1.begin(), g1.end());
    all.insert(all.end(), g1b.begin(), g1b.end());
    all.insert(all.end(), g2.begin(), g2.end());
    all.insert(all.end(), gbig.begin(), gbig.end());
    std::vector<size_t> dd_off;
    for (auto& r : gdd) { dd_off.push_back(all.size() - (g1.size() + g1b.size() + g2.size() + gbig.size())); all.insert(all.end(), r.begin(), r.end()); }
    if (all.size() != n_g1 + n_g1b + n_g2 + nbig + n_dd || cs.size() != n_cs) return TLR_ERR_STATE;
    host.resize(all.size() * gd * 8 + cs.size() * cd * 8);
    memcpy(host.data(), all.data(), all.size() * sizeof(GemmGen));
    // GemmGen and CopySeg regions are padded to 8-byte multiples (gd, cd doubles per entry)
    memcpy(host.data() + all.size() * sizeof(GemmGen), cs.data(), cs.size() * sizeof(CopySeg));
    TLR_CUDA_TRY(cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    // workspace after the panels: the tensor-core slices of each stage in turn
    char* tcw = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(Pw + p_tot + 8) + 127) & ~(uintptr_t)127);
    const size_t tcw_bytes = reinterpret_cast<char*>(base + budget) > tcw
                                 ? (size_t)(reinterpret_cast<char*>(base + budget) - tcw) : 0;
    {
      PhaseScope ps("lauum.prep", s);
      { PhaseScope p1("lauum.prep.copy", s); ZTRY(seg_copy(dcs, (int64_t)n_cs, s)); }
      { PhaseScope p1("lauum.prep.UtU", s); ZTRY(tops_gemm_thin(dg1, (int)n_g1, s)); }
      {
        PhaseScope p1("lauum.prep.dense", s);
        if (S) ZTRY(oz_run_host(g1b.data(), (int)g1b.size(), S, tcw, tcw_bytes, h->d_stat, s));
        else ZTRY(tops_gemm(dg1b, (int)n_g1b, nb, mx_r, s));
      }
      { PhaseScope p1("lauum.prep.VG", s); ZTRY(tops_gemm(dg2, (int)n_g2, nb, mx_r, s)); }
    }
    if (fused) {
      // each target: operand A = [panel A | M_km^T ...], B = [panel B | M_kn^T ...] as k segments,
      // reduced into the gradient by the epilogue (no tile of Sigma^{-1} is written)
      PhaseScope ps("lauum.gemm_grad", s);
      auto align = [](char* p) { return reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 127) & ~(uintptr_t)127); };
      char* sp = tcw;
      std::vector<OzSrc> src;
      std::vector<OzGemm> gem;
      std::vector<std::pair<int*, size_t>> zero_ex;
      int max_depth = 1;
      for (size_t q = b0; q < b1; ++q) {
        const GemmGen& gb = gbig[q - b0];
        const int m = tg[q].x, n = tg[q].y;
        const int64_t dtot = fdepth(q);
        const int nkb = (int)(dtot / OZ_BK);
        OzGemm og;
        memset(&og, 0, sizeof(og));
        og.m = nb; og.n = nb; og.ldc = nb; og.alpha = 1.0; og.beta = 0.0;
        og.lower = m == n;
        if (overlap) {  // the tile of Sigma^{-1} into this batch's buffer
          og.C = zb2[nbatch & 1] + (q - b0) * nn;
        } else {
          og.mode = 1; og.diag = m == n;
          og.p0a = (int64_t)m * nb; og.p0b = (int64_t)n * nb;
          og.part_off = (int64_t)q * tiles_per;
        }
        if (nkb > 0) {
          sp = align(sp);
          uint16_t* sa = reinterpret_cast<uint16_t*>(sp);
          sp += oz_slices_elems(nb, (int)dtot, OZ_BM, S) * 2;
          uint16_t* sb = reinterpret_cast<uint16_t*>(sp);
          sp += oz_slices_elems(nb, (int)dtot, OZ_BN, S) * 2;
          int* xa = reinterpret_cast<int*>(sp);
          sp += rows_a * sizeof(int);
          int* xb = reinterpret_cast<int*>(sp);
          sp += rows_b * sizeof(int);
          zero_ex.push_back({xa, (size_t)rows_a});
          zero_ex.push_back({xb, (size_t)rows_b});
          int kb = 0;
          if (gb.k > 0) {  // the panels: element (a, c) at Ap[c nb + a], (b, c) at Bp[c nb + b]
            src.push_back({gb.A, nb, 1, nb, gb.k, sa, xa, OZ_BM, kb, nkb, 1});
            src.push_back({gb.B, nb, 1, nb, gb.k, sb, xb, OZ_BN, kb, nkb, 1});
            kb += (int)(pad(gb.k) / OZ_BK);
            max_depth = std::max(max_depth, gb.k);
          }
          for (int k : ddk[q - b0]) {  // M_km^T M_kn: (a, c) at M_km[a nb + c], (b, c) at M_kn[b nb + c]
            src.push_back({Msrc(k, m), nb, 0, nb, nb, sa, xa, OZ_BM, kb, nkb, 1});
            src.push_back({Msrc(k, n), nb, 0, nb, nb, sb, xb, OZ_BN, kb, nkb, 1});
            kb += (int)(pad(nb) / OZ_BK);
            max_depth = std::max(max_depth, nb);
          }
          og.a = {sa, xa, nb, nkb};
          og.b = {sb, xb, nb, nkb};
        }
        gem.push_back(og);
      }
      sp = align(sp);
      OzSrc* dsrc = reinterpret_cast<OzSrc*>(sp);
      sp += src.size() * sizeof(OzSrc);
      sp = align(sp);
      OzGemm* dgem = reinterpret_cast<OzGemm*>(sp);
      sp += gem.size() * sizeof(OzGemm);
      if (sp > reinterpret_cast<char*>(base + budget)) TLR_RETURN_OOM();
      for (auto& z : zero_ex) TLR_CUDA_TRY(cudaMemsetAsync(z.first, 0, z.second * sizeof(int), s));
      if (!src.empty())
        TLR_CUDA_TRY(cudaMemcpyAsync(dsrc, src.data(), src.size() * sizeof(OzSrc), cudaMemcpyHostToDevice, s));
      TLR_CUDA_TRY(cudaMemcpyAsync(dgem, gem.data(), gem.size() * sizeof(OzGemm), cudaMemcpyHostToDevice, s));
      if (!src.empty()) ZTRY(oz_split(dsrc, (int)src.size(), nb, max_depth, S, s, true));
      if (overlap) {
        // the buffer's previous batch has been reduced; this batch's tiles are reduced on the caller's
        // stream while the next batch is prepared and multiplied here
        const int par = nbatch & 1;
        if (nbatch >= 2) TLR_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_lg[par], 0));
        ZTRY(oz_gemm(dgem, (int)gem.size(), nb, nb, S, h->d_stat, s));
        TLR_CUDA_TRY(cudaEventRecord(h->ev_lz[par], s));
        TLR_CUDA_TRY(cudaStreamWaitEvent(s_user, h->ev_lz[par], 0));
        ZTRY(tlr_grad_tiles(h, d_tg + b0, (int)(b1 - b0), zb2[par], (int64_t)b0 * mb64 * mb64, alpha, h->gpart,
                            s_user));
        TLR_CUDA_TRY(cudaEventRecord(h->ev_lg[par], s_user));
        ++nbatch;
      } else {
        OzGradCtx gx;
        memset(&gx, 0, sizeof(gx));
        gx.x = h->x; gx.y = h->y; gx.alpha = alpha; gx.tab = h->tab; gx.mp = h->mp; gx.n = h->n; gx.part = h->gpart;
        ZTRY(oz_gemm(dgem, (int)gem.size(), nb, nb, S, h->d_stat, s, &gx));
      }
    } else {
      PhaseScope ps("lauum.gemm", s);
      if (S) ZTRY(oz_run_host(gbig.data(), (int)gbig.size(), S, tcw, tcw_bytes, h->d_stat, s));
      else ZTRY(tops_gemm(dbig, (int)nbig, nb, nb, s));
    }
    {
      PhaseScope ps("lauum.dense_products", s);
      for (size_t r = 0; r < gdd.size(); ++r) {
        if (S) ZTRY(oz_run_host(gdd[r].data(), (int)gdd[r].size(), S, tcw, tcw_bytes, h->d_stat, s));
        else ZTRY(tops_gemm(ddd + dd_off[r], (int)gdd[r].size(), nb, nb, s));
      }
    }
    b0 = b1;
  }
  if (overlap) {  // the caller's stream continues after the last batch (its reductions are already on it)
    TLR_CUDA_TRY(cudaEventRecord(h->ev_join, s));
    TLR_CUDA_TRY(cudaStreamWaitEvent(s_user, h->ev_join, 0));
    join.from = join.to;  // joined
    s = s_user;
  }
  if (fused) {  // dl/dbeta, dl/dnu from the partial sums, in a fixed order
    ZTRY(tlr_sum_pairs(h->gpart, part_pairs, out3 + 1, h->scratch, s));
  } else if (T > 0) {
    k_mark_all_dense<<<256, 256, 0, s>>>(h->dslotz, T);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

// second stream, fork/join events and the dense x dense workspace for `items` items
static int ensure_aux(tlr_ctx* h, int items) {
  if (!h->aux) {
    int lo = 0, hi = 0;
    TLR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    TLR_CUDA_TRY(cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi));
    TLR_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    TLR_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  }
  const size_t want = (size_t)items * tops_dd_item_elems(h) + 64;  // tops_update_dd keeps 64 back
  if (want > h->scratch_dd_elems) {
    if (h->scratch_dd) cudaFree(h->scratch_dd);
    h->scratch_dd = nullptr;
    h->scratch_dd_elems = 0;
    if (cudaMalloc((void**)&h->scratch_dd, want * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      TLR_RETURN_OOM();
    }
    h->scratch_dd_elems = want;
  }
  return TLR_OK;
}


namespace {
struct InverseScope {  // marks the handle as forming the inverse for the scope's lifetime
  tlr_ctx* h;
  explicit InverseScope(tlr_ctx* hh) : h(hh) { h->in_inverse = 1; }
  ~InverseScope() { h->in_inverse = 0; }
};
}  // namespace

// one attempt; *grow > 0 (the entries Z's arena was asked for) when TRTRI ran out of arena, -1 when an
// update workspace was too narrow, and then the caller enlarges it and starts again
static int inverse_once(tlr_ctx* h, cudaStream_t s, const double* alpha, double* out3, int* fused, int64_t* grow) {
  *grow = 0;
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
  TLR_CUDA_TRY(cudaMemsetAsync(h->rankz, 0, std::max<int64_t>(h->ntiles, 1) * sizeof(int), s));
  if (h->ntiles > 0) {
    for (int64_t t0 = 0; t0 < h->ntiles; t0 += 65535) {
      // one grid row per tile (gridDim.y), offset via pointer arithmetic is not possible: launch per chunk
      const int64_t cnt = std::min<int64_t>(65535, h->ntiles - t0);
      TlrView fo = f, zo = z;
      fo.rank = f.rank + t0; fo.dslot = f.dslot + t0; fo.off = f.off + t0; fo.cap = f.cap + t0;
      zo.rank = z.rank + t0; zo.dslot = z.dslot + t0; zo.off = z.off + t0; zo.cap = z.cap + t0;
      k_copy_to_z<<<dim3(8, (unsigned)cnt), 256, 0, s>>>(fo, zo, cnt);
      TLR_LAUNCH_CHECK();
    }
  }
  const double eps = (h->opts.eps > 0 ? h->opts.eps : 0.0) * (h->opts.inv_scale > 0 ? h->opts.inv_scale : 1.0);
  // dense x dense products run on a second stream next to the other updates of their step
  int max_dd = 0;
  for (int k = 0; k < nt; ++k) {
    const int64_t* off = h->zoff + (size_t)k * ZPH;
    max_dd = std::max(max_dd, (int)(off[ZP_T2_DD + 1] - off[ZP_T2_DD]));
  }
  if (max_dd > 0) ZTRY(ensure_aux(h, std::min(max_dd, 32)));
  // ---- TRTRI (L_kk^{-1} of every diagonal tile comes from the Cholesky)
  const int64_t* gl = h->zoff + (size_t)nt * ZPH;
  auto GL = [&](int g) { return h->d_zlist + gl[g]; };
  auto GN = [&](int g) { return (int)(gl[g + 1] - gl[g]); };
  {  // step 1 of every k at once: no earlier step touches column k
    PhaseScope ps("trtri.col", s);  // A_ik <- -A_ik L_kk^{-1}: V <- -L_kk^{-T} V
    ZTRY(tops_trmul(h, z, h->linv, 1, GL(ZG_T1_LR), GN(ZG_T1_LR), 1, 0, GL(ZG_T1_D), GN(ZG_T1_D), 1, -1.0, s, nn,
                    2));
  }
  for (int k = 0; k < nt; ++k) {
    const int64_t* off = h->zoff + (size_t)k * ZPH;
    auto L = [&](int ph) { return h->d_zlist + off[ph]; };
    auto N = [&](int ph) { return (int)(off[ph + 1] - off[ph]); };
    // the three target sets of step 2 are disjoint and read only column k and row k
    const int ndd = N(ZP_T2_DD);
    if (ndd > 0) {
      TLR_CUDA_TRY(cudaEventRecord(h->ev_fork, s));
      TLR_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
      PhaseScope ps("trtri.update_dd", h->aux);
      ZTRY(tops_update_dd(h, z, ALG_TRTRI, k, L(ZP_T2_DD), ndd, eps, d_zeta, 0.5, h->aux, h->scratch_dd,
                          h->scratch_dd_elems));
    }
    { PhaseScope ps("trtri.update", s);
      // leading items of the low-rank list with a dense operand (partitioned first by the plan)
      int64_t ndop = 0;
      {
        const int2* hl = h->h_zlist + off[ZP_T2_LR];
        const char* K = h->kindz;
        while (ndop < N(ZP_T2_LR) && (K[tile_index(hl[ndop].x, k)] || K[tile_index(k, hl[ndop].y)])) ++ndop;
      }
      ZTRY(tops_update(h, z, ALG_TRTRI, k, L(ZP_T2_LR), N(ZP_T2_LR), ndop, L(ZP_T2_D), N(ZP_T2_D), eps, d_zeta, 0.5, s,
                       std::min(ndd, 32))); }
    if (ndd > 0) {
      TLR_CUDA_TRY(cudaEventRecord(h->ev_join, h->aux));
      TLR_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
  }
  {  // step 3 of every k at once: row k is final after step k - 1 and a source only in step k
    PhaseScope ps("trtri.row", s);  // A_kj <- L_kk^{-1} A_kj: U <- L_kk^{-1} U
    ZTRY(tops_trmul(h, z, h->linv, 0, GL(ZG_T3_LR), GN(ZG_T3_LR), 0, 0, GL(ZG_T3_D), GN(ZG_T3_D), 0, 1.0, s, nn, 1));
  }
  {  // step 4: A_kk <- L_kk^{-1}
    PhaseScope ps("trtri.store", s);
    k_copy<<<1024, 256, 0, s>>>(h->linv, h->Dz, (int64_t)nt * nn);
    TLR_LAUNCH_CHECK();
  }
  // TRTRI's ranks can outgrow Z's arena: checked before LAUUM reads Z
  h->zplan_valid = 0;  // the device tile kinds and layout of Z changed: the next inverse re-plans
  ZTRY(tlr_take_grow(h, s, h->topz, grow));
  if (*grow > 0) return TLR_OK;
  // ---- LAUUM
  if (fused) *fused = tlr_tc_slices(h) > 0 && alpha && out3;
  { PhaseScope ps("lauum", s); ZTRY(lauum_left(h, s, alpha, out3)); }
  return TLR_OK;
}

int tlr_inverse(tlr_ctx* h, cudaStream_t s, const double* alpha, double* out3, int* fused) {
  InverseScope scope(h);
  for (int attempt = 0;; ++attempt) {
    int64_t grow = 0;
    ZTRY(inverse_once(h, s, alpha, out3, fused, &grow));
    if (grow == 0) return TLR_OK;
    if (attempt >= 4) TLR_RETURN_OOM();
    if (grow < 0) ZTRY(tlr_widen(h));
    else ZTRY(tlr_arena_alloc(&h->Uz, &h->Vz, &h->arenaz, std::max(grow + grow / 2, h->arenaz + h->arenaz / 2)));
  }
}
