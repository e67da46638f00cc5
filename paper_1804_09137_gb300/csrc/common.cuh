// Internal declarations shared by the CUDA translation units of libtlr.
// Tile layout: n points in Morton order, padded to npad = nt * nb.  Padded
// points (index >= n) are "identity" points: covariance 1 with themselves and
// 0 with every other point, so padded rows/columns factor to the identity and
// add nothing to log|Sigma| or to the solves.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/tlr.h"

#define TLR_THREADS 256
#define TLR_MAX_WARPS 32  // largest block: 1024 threads

// Matérn interpolation table: C(r), dC/dbeta(r), dC/dnu(r) on geometric
// intervals [2^(e_lo + j/4), 2^(e_lo + (j+1)/4)), j = 0..TAB_NINT-1, each a
// degree TAB_DEG polynomial in t in [-1, 1] (monomial coefficients).
#define TAB_SUB 4
#define TAB_OCT 44
#define TAB_NINT (TAB_SUB * TAB_OCT)
#define TAB_DEG 12
#define TAB_NC (TAB_DEG + 1)
#define TAB_NFUN 3
#define TAB_ELEMS (TAB_NFUN * TAB_NINT * TAB_NC)

// status words (device): [0] first error code, [1] info
// plan phases of one panel step
#define PH_TRSM_LR 0
#define PH_TRSM_D 1
#define PH_UPD_LR 2
#define PH_UPD_D 3
#define PLAN_PH 4
// inverse plan phases of one step: TRTRI (1: column k, 2: updates, 3: row k), LAUUM (2: updates, 3: row k)
#define ZP_T2_LR 0
#define ZP_T2_D 1
#define ZP_T2_DD 2
#define ZPH 3
// whole-inverse lists after the per-step ones: column and row transforms of TRTRI
#define ZG_T1_LR 0
#define ZG_T1_D 1
#define ZG_T3_LR 2
#define ZG_T3_D 3
#define ZG 4

#define ST_CODE 0
#define ST_INFO 1
#define ST_BAR 3   // status word 3: grid-barrier counter of the one-launch tile Cholesky
// internal status code (never returned to a caller): a low-rank arena or an update workspace was too
// small; the host enlarges it and repeats the operation
#define TLR_ST_GROW 100
// internal status code: an update item's concatenated rank exceeded the workspaces' bound h->kws; the host
// widens the workspaces to the largest possible (2 kcap) and repeats the operation
#define TLR_ST_WIDEN 101

struct MaternParams {
  double sigma2, beta, nu;
  double cnu;    // 1 / (2^(nu-1) Gamma(nu))
  double psi;    // digamma(nu)
  int e_lo;      // table covers [2^e_lo, 2^(e_lo + TAB_OCT))
  int metric;    // 0 Euclidean, 1 great circle (x = longitude, y = latitude, degrees)
  double radius; // sphere radius of the great-circle distance
  double rad;    // pi / 180
};

struct tlr_ctx {
  int64_t n, npad;
  int nb, nt;
  int64_t ntiles;  // strictly lower tiles nt(nt-1)/2
  int64_t cap_n;   // allocation capacity (points); a handle can be rebound to n <= cap_n
  int cap_nt;
  int64_t cap_ntiles;
  tlr_opts opts;
  int dense;       // eps < 0: every off-diagonal tile dense
  int kcap;        // rank capacity of a low-rank tile
  double* x;       // sorted, padded coordinates (npad)
  double* y;
  int* perm;       // perm[s] = caller index of sorted point s (n entries)
  double* D;       // nt dense diagonal tiles, nb x nb column-major
  double* U;       // rank-packed arenas of the low-rank factors (arena entries each; see tile.cuh)
  double* V;
  int64_t* off;    // ntiles: first arena entry of each tile's columns
  int* cap;        // ntiles: columns reserved there
  unsigned long long* top;  // arena entries handed out (device counter)
  int64_t arena;   // arena size in entries
  int kws;         // concatenated-rank bound of the update workspaces (at most 2 kcap)
  int* rank;       // ntiles ranks (-1 after compression: not compressible below dense_rank)
  int* dslot;      // ntiles dense-pool slot or -1 (low rank)
  double* dpool;   // dense off-diagonal tiles, nb x nb each
  int dcap;        // dense pool capacity (tiles)
  int ndense;      // dense tiles in use
  int dense_rank;  // an off-diagonal tile whose rank exceeds this is stored dense
  char* kind;      // host copy of the tile kinds (1 dense)
  int2* d_list;    // factorization plan: per-step item lists (device)
  int2* h_list;    // host copy
  int64_t list_cap;
  int64_t* plan_off;  // [nt * PLAN_PH + 1] offsets into the lists
  // inverse Z = Sigma^{-1} (TLR, same tile layout), allocated by the first gradient call
  double* Dz;
  double* Uz;
  double* Vz;
  int64_t* offz;   // the inverse's arena layout, as for L
  int* capz;
  unsigned long long* topz;
  int64_t arenaz;
  int* rankz;
  int* dslotz;
  double* dpoolz;
  int dcapz;
  int ndensez;
  char* kindz;
  int2* d_zlist;
  int2* h_zlist;
  int64_t zlist_cap;
  int64_t* zoff;      // [nt * ZPH + ZG + 1]
  int zplan_valid;
  double* tab;     // Matérn table (TAB_ELEMS)
  float2* tabf;    // its coefficients as double-float pairs (TAB_ELEMS; absent in the allocation-free entry point)
  MaternParams mp;
  double* linv;    // nt tiles nb x nb: L_kk^{-1} of every diagonal tile (Cholesky, reused by the inverse)
  double* scratch; // batched-kernel workspace
  size_t scratch_elems;
  size_t item_elems;  // workspace per low-rank update item
  int items_per_launch;
  long long* d_stat;  // status words
  int* d_ctr;         // item counter of the persistent update kernel
  double* d_xk;       // nb: x_k of the current solve step
  double* d_vec;      // 4 vectors of npad
  double* d_red;      // reduction partials
  int red_len;
  int state;          // 0 created, 1 generated, 2 compressed, 3 factored
  int in_inverse;     // 1 while the gradient's inverse is being formed (tensor-core products allowed)
  int tab_valid;
  cudaStream_t last_stream;
  // second stream of the inverse (dense x dense products overlap the other updates of a step)
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join;
  cudaEvent_t ev_lz[2], ev_lg[2];  // LAUUM: a batch's tiles of Sigma^{-1} written / reduced
  double* scratch_dd;
  size_t scratch_dd_elems;
  // copy of the inverse's dense sources (diagonal and dense tiles) read by LAUUM
  double* msave;
  size_t msave_elems;
  int* hslotz;        // host copy of the inverse's dense slots
  double* gpart;      // partial sums of the gradient reduced inside LAUUM
  size_t gpart_elems;
  // products of the low-rank updates with a dense operand, formed by a batched GEMM before the
  // persistent update kernel (nb x kcap per item, with descriptors and tensor-core workspace)
  double* dop;
  size_t dop_elems;
};

// ---------------------------------------------------------------- helpers
#define TLR_CUDA_TRY(call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      fprintf(stderr, "tlr: %s failed: %s (%s:%d)\n", #call,                 \
              cudaGetErrorString(e_), __FILE__, __LINE__);                   \
      return TLR_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

#include <atomic>
extern std::atomic<long long> g_tlr_launches;  // kernel launches issued by the library
#define TLR_LAUNCH_CHECK()                                                   \
  do {                                                                       \
    ++g_tlr_launches;                                                        \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      fprintf(stderr, "tlr: launch failed: %s (%s:%d)\n",                   \
              cudaGetErrorString(e_), __FILE__, __LINE__);                   \
      return TLR_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

static inline int64_t tile_index(int i, int j) { return (int64_t)i * (i - 1) / 2 + j; }
__device__ __forceinline__ int64_t dtile_index(int i, int j) { return (int64_t)i * (i - 1) / 2 + j; }

// record the first device-side failure
__device__ __forceinline__ void set_status(long long* st, long long code, long long info) {
  if (atomicCAS((unsigned long long*)&st[ST_CODE], 0ull, (unsigned long long)code) == 0ull)
    st[ST_INFO] = info;
}

// block-wide sum of one double per thread (any block size up to 1024 threads, a multiple of 32;
// sh holds blockDim.x / 32 + 1 doubles); all threads get the result
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (l < nw) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) sh[nw] = t;
  }
  __syncthreads();
  return sh[nw];
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide argmax of |v| over threads; returns index (ties: smaller index); shv, shi hold
// blockDim.x / 32 + 1 entries
__device__ __forceinline__ int block_argmax(double a, int idx, double* shv, int* shi, double* outv) {
  for (int o = 16; o > 0; o >>= 1) {
    double a2 = __shfl_xor_sync(0xffffffffu, a, o);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (a2 > a || (a2 == a && i2 < idx)) { a = a2; idx = i2; }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) { shv[w] = a; shi[w] = idx; }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = (l < nw) ? shv[l] : -1.0;
    idx = (l < nw) ? shi[l] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      double a2 = __shfl_xor_sync(0xffffffffu, a, o);
      int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (a2 > a || (a2 == a && i2 < idx)) { a = a2; idx = i2; }
    }
    if (l == 0) { shv[nw] = a; shi[nw] = idx; }
  }
  __syncthreads();
  if (outv) *outv = shv[nw];
  return shi[nw];
}

// ------------------------------------------------------- Matérn evaluation
// Interval index and local coordinate t in [-1,1] of r > 0 in the table.
__device__ __forceinline__ int tab_locate(double r, int e_lo, double* t) {
  const int hi = __double2hiint(r);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  const double m = __hiloint2double((hi & 0x800fffff) | 0x3ff00000, __double2loint(r));
  // 2^(q/4) boundaries of the 4 sub-intervals of one octave
  constexpr double b1 = 1.18920711500272106672, b2 = 1.41421356237309504880, b3 = 1.68179283050742908606;
  int q = (m >= b1) + (m >= b2) + (m >= b3);
  const double a = q == 0 ? 1.0 : (q == 1 ? b1 : (q == 2 ? b2 : b3));
  const double b = q == 0 ? b1 : (q == 1 ? b2 : (q == 2 ? b3 : 2.0));
  // 1 / (b - a) of the four sub-intervals (compile-time constants: no float64 division per entry)
  constexpr double i0 = 1.0 / (b1 - 1.0), i1 = 1.0 / (b2 - b1), i2 = 1.0 / (b3 - b2), i3 = 1.0 / (2.0 - b3);
  const double iw = q == 0 ? i0 : (q == 1 ? i1 : (q == 2 ? i2 : i3));
  *t = (2.0 * m - a - b) * iw;
  return TAB_SUB * (e - e_lo) + q;
}

__device__ __forceinline__ double tab_poly(const double* __restrict__ c, double t) {
  double s = c[TAB_DEG];
#pragma unroll
  for (int d = TAB_DEG - 1; d >= 0; --d) s = fma(s, t, c[d]);
  return s;
}

// Evaluate table function f (0: C, 1: dC/dbeta, 2: dC/dnu) at distance r >= 0.
// Distances below the table (r < 2^e_lo, i.e. 2^-44 of the largest distance)
// and r = 0 take the r -> 0 limits (sigma2, 0, 0).
__device__ __forceinline__ double matern_tab(const double* __restrict__ tab, const MaternParams& mp,
                                             int f, double r) {
  if (!(r > 0.0)) return f == 0 ? mp.sigma2 : 0.0;
  double t;
  int j = tab_locate(r, mp.e_lo, &t);
  if (j < 0) return f == 0 ? mp.sigma2 : 0.0;
  if (j >= TAB_NINT) return 0.0;  // beyond the largest distance covered (not reached)
  return tab_poly(tab + ((size_t)f * TAB_NINT + j) * TAB_NC, t);
}

// distance between (xa, ya) and (xb, yb): Euclidean, or the great-circle distance of
// eq. 6 (Sec. IV), hav(d / r) = hav(phi_b - phi_a) + cos(phi_a) cos(phi_b) hav(lam_b - lam_a),
// with hav(t) = sin^2(t / 2), longitude lam = x and latitude phi = y in degrees
__device__ __forceinline__ double pt_dist(const MaternParams& mp, double xa, double ya, double xb, double yb) {
  if (mp.metric == 0) {
    const double dx = xa - xb, dy = ya - yb;
    return sqrt(dx * dx + dy * dy);
  }
  const double pa = ya * mp.rad, pb = yb * mp.rad;
  const double sp = sin(0.5 * (pb - pa)), sl = sin(0.5 * (xb - xa) * mp.rad);
  const double h = fma(cos(pa) * cos(pb), sl * sl, sp * sp);
  return 2.0 * mp.radius * asin(sqrt(fmin(h, 1.0)));
}

// covariance between sorted points p and q (padded points are identity points)
__device__ __forceinline__ double cov_pts(const double* __restrict__ tab, const MaternParams& mp,
                                          const double* __restrict__ x, const double* __restrict__ y,
                                          int64_t n, int64_t p, int64_t q) {
  if (p >= n || q >= n) return (p == q) ? 1.0 : 0.0;
  if (p == q) return mp.sigma2;
  return matern_tab(tab, mp, 0, pt_dist(mp, x[p], y[p], x[q], y[q]));
}

// profiling of the low-rank update kernel (the dominant one): per-launch CUDA
// events and a device-side count of its algorithmic float64 flops
struct TlrProfile {
  int enabled;
  double* d_flops;     // device accumulator
  long long launches;
  double ms;
};
extern thread_local TlrProfile g_tlr_prof;  // per host thread
void tlr_prof_begin(cudaStream_t s);
void tlr_prof_end(cudaStream_t s);
// the same for the tensor-core GEMM (its MMA flops accumulate in d_flops[1])
void tlr_prof_tc_begin(cudaStream_t s);
void tlr_prof_tc_end(cudaStream_t s);
// per-phase device time (events around each phase when profiling is enabled)
void tlr_phase_begin(const char* name, cudaStream_t s);
void tlr_phase_end(cudaStream_t s);
struct PhaseScope {
  cudaStream_t s;
  PhaseScope(const char* name, cudaStream_t st) : s(st) { tlr_phase_begin(name, s); }
  ~PhaseScope() { tlr_phase_end(s); }
};

// ------------------------------------------------------------ host helpers
double tlr_host_digamma(double x);  // psi(x), x > 0 (host)
// records where a call ran out of memory (printed to stderr when TLR_VERBOSE is set)
void tlr_note_oom(const char* file, int line);
#define TLR_RETURN_OOM()               \
  do {                                 \
    tlr_note_oom(__FILE__, __LINE__);  \
    return TLR_ERR_OOM;                \
  } while (0)
// digit slices of the tensor-core contractions for the handle's precision option (0: none).  By
// default (precision 0) only the gradient's inverse uses them: the Cholesky's products with the
// explicit diagonal-tile inverses amplify the rounding of their operands' scale (with tensor-core
// products the l error at eps = 1e-9 exceeded 1e-8 relative).  precision 4..6 (the mixed-precision
// mode) also runs the Cholesky's contractions of depth >= 256 on the tensor cores.  Dense mode, the
// exact full-tile comparator, stays in double-float.
static inline int tlr_tc_slices_opt(const tlr_ctx* h) {  // the option alone (workspace sizing)
  const int p = h->opts.precision;
  if (h->dense) return 0;
  return p == 0 ? 6 : (p == 1 ? 0 : p);
}
static inline int tlr_tc_slices(const tlr_ctx* h) {
  if (h->in_inverse) return tlr_tc_slices_opt(h);
  return (!h->dense && h->opts.precision >= 4) ? h->opts.precision : 0;
}
int tlr_build_table(tlr_ctx* h, cudaStream_t s);
int tlr_gen_diag(tlr_ctx* h, cudaStream_t s);
int tlr_gen_dense_tiles(tlr_ctx* h, const int2* d_items, int count, cudaStream_t s);
int tlr_compress_tiles(tlr_ctx* h, double eps, cudaStream_t s);
int tlr_factor(tlr_ctx* h, cudaStream_t s);
int tlr_plan(tlr_ctx* h, cudaStream_t s);
// low-rank arenas: (re)allocate a pair for at least `need` entries (contents discarded)
int tlr_arena_alloc(double** U, double** V, int64_t* arena, int64_t need);
// CTAs of the persistent low-rank update kernel resident on the current device for tile size nb
int tops_resident_ctas(int nb);
// after a synchronisation: *need = the entries the arena counter d_top asked for when an arena or a
// workspace ran out during the work enqueued so far (status reset), else 0
int tlr_take_grow(tlr_ctx* h, cudaStream_t s, const unsigned long long* d_top, int64_t* need);
// after tlr_take_grow reported a workspace bound exceeded (*need < 0): widen kws to 2 kcap and grow the
// workspace
int tlr_widen(tlr_ctx* h);
int tlr_rebind(tlr_ctx* h, int64_t n, const double* x, const double* y, cudaStream_t s);
int tlr_alloc(int64_t cap_n, const tlr_opts* opts, tlr_ctx** out);
// workspace (doubles) of one low-rank update item for concatenated ranks up to kws
size_t tlr_item_elems(int nb, int kcap, int kws);
// batched-kernel workspace the handle needs for its tile size, rank cap and update bound kws
size_t tlr_scratch_want(const tlr_ctx* h);
int tlr_potrf_tile(tlr_ctx* h, double* A, int lda, int nb, int64_t col0, cudaStream_t s);
int tlr_fwd_solve(tlr_ctx* h, double* r, cudaStream_t s);
int tlr_bwd_solve(tlr_ctx* h, double* r, cudaStream_t s);
int tlr_lmul(tlr_ctx* h, const double* e, double* z, cudaStream_t s);
int tlr_reduce_loglik(tlr_ctx* h, const double* w, double* out3, cudaStream_t s);
// TRTRI + LAUUM; with alpha = Sigma^{-1} z (sorted) and out3 given and tensor-core products enabled,
// the gradient's beta and nu entries are reduced inside LAUUM into out3[1], out3[2] (*fused = 1)
// instead of forming Sigma^{-1}
int tlr_inverse(tlr_ctx* h, cudaStream_t s, const double* alpha = nullptr, double* out3 = nullptr,
                int* fused = nullptr);
// out2[0] = sum part[2 i], out2[1] = sum part[2 i + 1] over i < count, in a fixed order (ws: 512 doubles)
int tlr_sum_pairs(const double* part, int64_t count, double* out2, double* ws, cudaStream_t s);
int tlr_grad_fused(tlr_ctx* h, const double* alpha, double* out3, cudaStream_t s);
// dl/dbeta, dl/dnu partial pairs of `cnt` dense tiles of Sigma^{-1} (Z + t nb^2, targets tg[t] on the
// device), block b of tile t into part[2 (slot0 + t mb^2 + b)], mb = ceil(nb / 64)
int tlr_grad_tiles(const tlr_ctx* h, const int2* tg, int cnt, const double* Z, int64_t slot0, const double* alpha,
                   double* part, cudaStream_t s);
int tlr_predict_var_sorted(tlr_ctx* h, int64_t m, const double* xn, const double* yn, double* var, cudaStream_t s);
int tlr_krige(tlr_ctx* h, const double* a, int64_t m, const double* xn, const double* yn, double* zn,
              cudaStream_t s);
int tlr_permute_in(tlr_ctx* h, const double* src, double* dst, cudaStream_t s);
int tlr_permute_out(tlr_ctx* h, const double* src, double* dst, cudaStream_t s);
