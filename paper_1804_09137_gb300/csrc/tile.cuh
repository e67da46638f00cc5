// Tile views and CTA-level float64 building blocks shared by the factor,
// inverse and solve kernels.
//
// Off-diagonal tile t = i(i-1)/2 + j (i > j) is either
//   low rank: U_t V_t^T, U_t, V_t in slot t (nb x kcap, column-major, ld nb), rank rank[t];
//   dense:    A_t in dense-pool slot dslot[t] (nb x nb, column-major, ld nb).
// Diagonal tiles are always dense (D + i nb^2).
#pragma once
#include "common.cuh"

struct TlrView {
  int nb, nt, kcap;
  double* D;      // nt diagonal tiles
  double* U;      // low-rank slots
  double* V;
  int* rank;      // per off-diagonal tile
  int* dslot;     // dense-pool slot or -1
  double* dpool;  // dense pool
};

static inline TlrView view_of(const tlr_ctx* h) {
  TlrView v;
  v.nb = h->nb; v.nt = h->nt; v.kcap = h->kcap;
  v.D = h->D; v.U = h->U; v.V = h->V; v.rank = h->rank; v.dslot = h->dslot; v.dpool = h->dpool;
  return v;
}

struct GemmDesc {  // C -= P Q^T (nb x nb), inner dimension r; lower: only the lower triangle
  const double* P;
  const double* Q;
  double* C;
  int r;
  int lower;
};

__device__ __forceinline__ size_t lr_slot(const TlrView& v) { return (size_t)v.nb * v.kcap; }
__device__ __forceinline__ double* tileU(const TlrView& v, int64_t t) { return v.U + t * lr_slot(v); }
__device__ __forceinline__ double* tileV(const TlrView& v, int64_t t) { return v.V + t * lr_slot(v); }
__device__ __forceinline__ double* tileA(const TlrView& v, int64_t t) {
  return v.dpool + (size_t)v.dslot[t] * v.nb * v.nb;
}
__device__ __forceinline__ double* diagT(const TlrView& v, int i) { return v.D + (size_t)i * v.nb * v.nb; }

__device__ __forceinline__ void decode_lower(int64_t t, int* i, int* j) {
  int ii = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while ((int64_t)ii * (ii - 1) / 2 > t) --ii;
  while ((int64_t)(ii + 1) * ii / 2 <= t) ++ii;
  *i = ii;
  *j = (int)(t - (int64_t)ii * (ii - 1) / 2);
}

// Work item of a batched tile operation (built on the host from the tile kinds).
struct TileItem {
  int i, j, k;  // target (i, j); source index k (meaning depends on the operation)
  int kind;     // operation-specific case code
};
