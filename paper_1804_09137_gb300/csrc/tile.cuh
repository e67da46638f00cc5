// Tile views and CTA-level float64 building blocks shared by the factor,
// inverse and solve kernels.
//
// Off-diagonal tile t = i(i-1)/2 + j (i > j) is either
//   low rank: U_t V_t^T with U_t = U + off[t], V_t = V + off[t] (nb x rank[t], column-major, ld nb):
//             a block of cap[t] columns in the rank-packed arenas U and V, handed out by
//             cta_lr_reserve from the counter *top when a tile first needs more columns;
//   dense:    A_t in dense-pool slot dslot[t] (nb x nb, column-major, ld nb).
// Diagonal tiles are always dense (D + i nb^2).
#pragma once
#include "common.cuh"

struct TlrView {
  int nb, nt, kcap;
  double* D;      // nt diagonal tiles
  double* U;      // low-rank arenas (arena entries each)
  double* V;
  int* rank;      // per off-diagonal tile
  int* dslot;     // dense-pool slot or -1
  double* dpool;  // dense pool
  int64_t* off;   // per off-diagonal tile: first arena entry of its columns
  int* cap;       // per off-diagonal tile: columns reserved there
  unsigned long long* top;  // arena entries handed out
  int64_t arena;  // arena size (entries of U, and of V)
};

static inline TlrView view_of(const tlr_ctx* h) {
  TlrView v;
  v.nb = h->nb; v.nt = h->nt; v.kcap = h->kcap;
  v.D = h->D; v.U = h->U; v.V = h->V; v.rank = h->rank; v.dslot = h->dslot; v.dpool = h->dpool;
  v.off = h->off; v.cap = h->cap; v.top = h->top; v.arena = h->arena;
  return v;
}

struct GemmDesc {  // C -= P Q^T (nb x nb), inner dimension r; lower: only the lower triangle
  const double* P;
  const double* Q;
  double* C;
  int r;
  int lower;
};

__device__ __forceinline__ double* tileU(const TlrView& v, int64_t t) { return v.U + v.off[t]; }
__device__ __forceinline__ double* tileV(const TlrView& v, int64_t t) { return v.V + v.off[t]; }

// CTA-wide (every thread calls it): room for k columns of tile t.  A tile keeps its block while k fits;
// otherwise a new block of k + k / 4 + 8 columns (at most kcap) is taken from the arena's counter and
// the old block is left unused.  False, with status TLR_ST_GROW, when the arena is exhausted (the
// host then enlarges it and repeats the operation).
__device__ __forceinline__ bool cta_lr_reserve(const TlrView& v, int64_t t, int k, long long* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (k > v.cap[t]) {
      int c = k + k / 4 + 8;
      c = (c + 7) & ~7;
      if (c > v.kcap) c = v.kcap;
      if (c < k) c = k;
      const unsigned long long need = (unsigned long long)c * v.nb;
      const unsigned long long pos = atomicAdd(v.top, need);
      if (pos + need > (unsigned long long)v.arena) {
        set_status(st, TLR_ST_GROW, t);
        ok = 0;
      } else {
        v.off[t] = (int64_t)pos;
        v.cap[t] = c;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
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

// ---- grid-wide barrier of the cooperative (one-launch) kernels: every CTA is resident (cooperative
// launch); each wait is bounded (about two seconds), after which the CTA records TLR_ERR_TIMEOUT and
// the barrier reports false
constexpr long long BAR_WAIT = 1ll << 32;  // clock cycles before a barrier wait gives up

// grid-wide barrier on a counter zeroed before the launch: the i-th barrier completes when the
// counter reaches i * gridDim.x; false when the wait gave up
__device__ inline bool grid_barrier(unsigned int* bar, unsigned int& target, long long* st) {
  __shared__ int s_ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const long long t0 = clock64();
    while (*(volatile unsigned int*)bar < target) {
      if (clock64() - t0 > BAR_WAIT) {
        set_status(st, TLR_ERR_TIMEOUT, 5);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

