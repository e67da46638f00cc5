// C ABI entry points (include/tlr.h) and the host-side drivers.
//
// The host code owns the ordering of the tile algorithm; each step is a batched
// launch over every tile it touches, enqueued on the caller's stream.  The
// Morton ordering of the points (setup, once per handle) runs on the host.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "tcgemm.h"


std::atomic<long long> g_tlr_launches{0};
thread_local TlrProfile g_tlr_prof = {0, nullptr, 0, 0.0};

namespace {
thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_ev;  // recorded (start, stop) pairs
thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_ev_free;
cudaEvent_t g_ev_open = nullptr;
}  // namespace

void tlr_prof_begin(cudaStream_t s) {
  cudaEvent_t a, b;
  if (!g_ev_free.empty()) {
    a = g_ev_free.back().first;
    b = g_ev_free.back().second;
    g_ev_free.pop_back();
  } else {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  cudaEventRecord(a, s);
  g_ev.push_back({a, b});
}

void tlr_prof_end(cudaStream_t s) {
  if (!g_ev.empty()) cudaEventRecord(g_ev.back().second, s);
}

namespace {
thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_ev_tc;  // tensor-core GEMM launches
}  // namespace

void tlr_prof_tc_begin(cudaStream_t s) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  g_ev_tc.push_back({a, b});
}

void tlr_prof_tc_end(cudaStream_t s) {
  if (!g_ev_tc.empty()) cudaEventRecord(g_ev_tc.back().second, s);
}

namespace {
struct PhaseRec {
  const char* name;
  cudaEvent_t a, b;
  long long l0, l1;  // this library's launch counter at the phase's start and end
};
thread_local std::vector<PhaseRec> g_ph;
thread_local std::vector<int> g_ph_open;
}  // namespace

void tlr_phase_begin(const char* name, cudaStream_t s) {
  if (!g_tlr_prof.enabled) return;
  PhaseRec r{name, nullptr, nullptr, (long long)g_tlr_launches, (long long)g_tlr_launches};
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  cudaEventRecord(r.a, s);
  g_ph.push_back(r);
  g_ph_open.push_back((int)g_ph.size() - 1);
}

void tlr_phase_end(cudaStream_t s) {
  if (!g_tlr_prof.enabled || g_ph_open.empty()) return;
  cudaEventRecord(g_ph[g_ph_open.back()].b, s);
  g_ph[g_ph_open.back()].l1 = (long long)g_tlr_launches;
  g_ph_open.pop_back();
}

void tlr_note_oom(const char* file, int line) {
  if (getenv("TLR_VERBOSE")) fprintf(stderr, "tlr: out of memory at %s:%d\n", file, line);
}

// digamma by upward recurrence to x >= 10 and the asymptotic series
// psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)  (Abramowitz & Stegun 6.3.18)
double tlr_host_digamma(double x) {
  double r = 0.0;
  while (x < 10.0) { r -= 1.0 / x; x += 1.0; }
  const double f = 1.0 / (x * x);
  return r + log(x) - 0.5 / x -
         f * (1.0 / 12 - f * (1.0 / 120 - f * (1.0 / 252 - f * (1.0 / 240 - f * (1.0 / 132)))));
}

namespace {

// Morton (Z-curve) order of the points over their bounding square, 16 bits per axis
std::vector<int> morton_order(const std::vector<double>& x, const std::vector<double>& y) {
  const size_t n = x.size();
  double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
  for (size_t i = 1; i < n; ++i) {
    x0 = std::min(x0, x[i]); x1 = std::max(x1, x[i]);
    y0 = std::min(y0, y[i]); y1 = std::max(y1, y[i]);
  }
  const double ext = std::max(x1 - x0, y1 - y0);
  const double scale = ext > 0 ? 65536.0 / ext : 0.0;
  std::vector<uint32_t> key(n);
  for (size_t i = 0; i < n; ++i) {
    uint32_t qx = (uint32_t)std::min(65535.0, floor((x[i] - x0) * scale));
    uint32_t qy = (uint32_t)std::min(65535.0, floor((y[i] - y0) * scale));
    uint32_t k = 0;
    for (int b = 0; b < 16; ++b) k |= ((qx >> b) & 1u) << (2 * b) | ((qy >> b) & 1u) << (2 * b + 1);
    key[i] = k;
  }
  std::vector<int> p(n);
  std::iota(p.begin(), p.end(), 0);
  std::stable_sort(p.begin(), p.end(), [&](int a, int b) { return key[a] < key[b]; });
  return p;
}

int set_table_range(tlr_ctx* h, double rmax) {
  int E = (int)ceil(log2(rmax > 0 ? rmax : 1.0)) + 1;
  const int e_lo = E - TAB_OCT;
  if (h->tab_valid && e_lo <= h->mp.e_lo) return 0;  // covered already
  h->mp.e_lo = e_lo;
  return 1;
}

double bbox_diag(const double* x, const double* y, size_t n) {
  double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
  for (size_t i = 1; i < n; ++i) {
    x0 = std::min(x0, x[i]); x1 = std::max(x1, x[i]);
    y0 = std::min(y0, y[i]); y1 = std::max(y1, y[i]);
  }
  return hypot(x1 - x0, y1 - y0);
}

// largest distance the table must cover: the bounding-box diagonal, or for the
// great-circle distance half the circumference (no two points are farther apart)
double dist_range(const tlr_ctx* h, const double* x, const double* y, size_t n) {
  if (h->mp.metric == 1) return M_PI * h->mp.radius;
  return bbox_diag(x, y, n);
}

template <class T>
int dmalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    TLR_RETURN_OOM();
  }
  return TLR_OK;
}

void free_ctx(tlr_ctx* h) {
  void* bufs[] = {h->x,     h->y,     h->perm,   h->D,     h->U,     h->V,      h->rank,   h->tab,
                  h->scratch, h->d_stat, h->d_vec, h->d_red, h->dslot, h->dpool, h->d_list, h->Dz,
                  h->Uz,    h->Vz,    h->rankz,  h->dslotz, h->dpoolz, h->d_zlist, h->linv, h->d_ctr, h->scratch_dd, h->msave, h->d_xk, h->dop, h->off, h->cap, h->top, h->offz, h->capz, h->topz,
                  h->gpart, h->tabf};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h->aux) cudaStreamDestroy(h->aux);

  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_lz[i]) cudaEventDestroy(h->ev_lz[i]);
    if (h->ev_lg[i]) cudaEventDestroy(h->ev_lg[i]);
  }
  free(h->kind);
  free(h->h_list);
  free(h->plan_off);
  free(h->kindz);
  free(h->h_zlist);
  free(h->zoff);
  free(h->hslotz);
  delete h;
}

// (Re)bind a handle to n <= cap_n points: Morton order, sorted padded
// coordinates, table range; resets the pipeline state.  Synchronises s.
int bind_points(tlr_ctx* h, int64_t n, const std::vector<double>& hx, const std::vector<double>& hy, cudaStream_t s) {
  if (n > h->cap_n) return -1;
  h->n = n;
  h->nt = (int)((n + h->nb - 1) / h->nb);
  h->npad = (int64_t)h->nt * h->nb;
  h->ntiles = (int64_t)h->nt * (h->nt - 1) / 2;
  std::vector<int> perm(n);
  if (h->opts.order) perm = morton_order(hx, hy);
  else std::iota(perm.begin(), perm.end(), 0);
  std::vector<double> sx(h->npad, 0.0), sy(h->npad, 0.0);
  for (int64_t s2 = 0; s2 < n; ++s2) { sx[s2] = hx[perm[s2]]; sy[s2] = hy[perm[s2]]; }
  h->mp.e_lo = 0;
  h->tab_valid = 0;
  set_table_range(h, dist_range(h, hx.data(), hy.data(), n));
  h->state = 0;
  h->zplan_valid = 0;
  cudaError_t e1 = cudaMemcpyAsync(h->x, sx.data(), h->npad * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaError_t e2 = cudaMemcpyAsync(h->y, sy.data(), h->npad * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaError_t e3 = cudaMemcpyAsync(h->perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaError_t e4 = cudaMemsetAsync(h->d_stat, 0, 4 * sizeof(long long), s);
  cudaError_t e5 = cudaMemsetAsync(h->rank, 0, std::max<int64_t>(h->ntiles, 1) * sizeof(int), s);
  if (e5 == cudaSuccess) e5 = cudaMemsetAsync(h->dslot, 0xff, std::max<int64_t>(h->ntiles, 1) * sizeof(int), s);
  cudaError_t e6 = cudaStreamSynchronize(s);
  if (e1 || e2 || e3 || e4 || e5 || e6) return TLR_ERR_CUDA;
  h->last_stream = s;
  return TLR_OK;
}

#define TRY(x)                 \
  do {                         \
    int rc_ = (x);             \
    if (rc_ != TLR_OK) return rc_; \
  } while (0)

}  // namespace

// Allocate a handle with capacity for cap points (not yet bound to points).
size_t tlr_scratch_want(const tlr_ctx* h) {
  const size_t nb = h->nb;
  const int64_t ct = h->cap_ntiles;
  // workspace: low-rank update items, SYRK items, table nodes, gradient partials
  const size_t ie = h->dense ? 0 : tlr_item_elems(h->nb, h->kcap, h->kws);
  const int64_t max_items = std::max<int64_t>(ct, 1);
  // one item workspace per resident CTA of the persistent update kernel (compression takes as many tiles
  // a launch)
  const int64_t chunk = std::min<int64_t>(max_items, h->dense ? 912 : std::max(tops_resident_ctas(h->nb), 64));
  size_t ws = std::max<size_t>((size_t)chunk * ie, (size_t)TAB_ELEMS);
  ws = std::max(ws, (size_t)chunk * (nb * h->kcap + (size_t)h->kcap * h->kcap + 8));
  ws = std::max(ws, (size_t)(2 * 8 * (int64_t)h->cap_nt * (h->cap_nt + 1) / 2 + 16));
  // gradient partials: 3 per 64 x 64 block of the lower triangle; dense diagonal-tile workspace
  const size_t mb = (nb + 63) / 64;
  ws = std::max(ws, (size_t)(3 * mb * mb * (size_t)h->cap_nt * (h->cap_nt + 1) / 2 + 1024));
  ws = std::max(ws, 2 * nb * nb + 4096);
  // the inverse's stacked-panel products on the tensor cores: slices of one nb x nb x nb product
  // next to two nb x nb panels and their descriptors
  if (tlr_tc_slices_opt(h) > 0) {
    const int S = tlr_tc_slices_opt(h);
    const size_t tc = (oz_slices_elems(h->nb, h->nb, OZ_BM, S) + oz_slices_elems(h->nb, h->nb, OZ_BN, S)) / 4 +
                      2 * nb * nb + 3 * (size_t)h->cap_nt * 64 + 65536;
    ws = std::max(ws, tc);
  }
  return ws;
}

int tlr_widen(tlr_ctx* h) {
  h->kws = 2 * h->kcap;
  const size_t want = tlr_scratch_want(h);
  if (want <= h->scratch_elems) return TLR_OK;
  TLR_CUDA_TRY(cudaDeviceSynchronize());
  cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_elems = 0;
  if (cudaMalloc((void**)&h->scratch, want * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    TLR_RETURN_OOM();
  }
  h->scratch_elems = want;
  return TLR_OK;
}

int tlr_alloc(int64_t n, const tlr_opts* opts, tlr_ctx** out) {
  tlr_ctx* h = new tlr_ctx();
  memset(h, 0, sizeof(*h));
  h->opts = *opts;
  h->nb = opts->nb;
  h->mp.metric = opts->metric == 1 ? 1 : 0;
  h->mp.radius = opts->radius > 0 ? opts->radius : 1.0;
  h->mp.rad = M_PI / 180.0;
  h->cap_n = n;
  h->cap_nt = (int)((n + h->nb - 1) / h->nb);
  h->cap_ntiles = (int64_t)h->cap_nt * (h->cap_nt - 1) / 2;
  h->dense = opts->eps < 0;
  int kc = opts->rank_cap > 0 ? opts->rank_cap : std::max(1, h->nb / 2);
  h->kcap = h->dense ? 1 : std::min(kc, h->nb);
  h->dense_rank = opts->dense_rank > 0 ? opts->dense_rank : std::max(16, h->nb / 9);
  if (h->dense_rank > 2 * h->kcap - 8) h->dense_rank = std::max(1, 2 * h->kcap - 8);

  const size_t nb = h->nb;
  const int64_t cnp = (int64_t)h->cap_nt * h->nb, ct = h->cap_ntiles;
  int rc = TLR_OK;
  rc |= dmalloc(&h->x, cnp);
  rc |= dmalloc(&h->y, cnp);
  rc |= dmalloc(&h->perm, n);
  rc |= dmalloc(&h->D, (size_t)h->cap_nt * nb * nb);
  // rank-packed arenas: room for 32 columns a tile to start with; compression, the factorization and
  // the inverse enlarge them (and repeat) when the ranks need more
  // update workspaces for concatenated ranks up to kws (widened to 2 kcap, and the step repeated, when
  // a larger one occurs); never below what compression's cross approximation may take
  h->kws = std::min(2 * h->kcap, std::max(h->kcap, h->dense_rank + 8));
  h->arena = h->dense ? 1 : std::max<int64_t>(ct, 1) * (int64_t)nb * std::min(h->kcap, 32);
  rc |= dmalloc(&h->U, (size_t)h->arena);
  rc |= dmalloc(&h->V, (size_t)h->arena);
  rc |= dmalloc(&h->off, ct);
  rc |= dmalloc(&h->cap, ct);
  rc |= dmalloc(&h->top, 1);
  rc |= dmalloc(&h->rank, ct);
  rc |= dmalloc(&h->dslot, ct);
  rc |= dmalloc(&h->tab, TAB_ELEMS);
  rc |= dmalloc(&h->tabf, TAB_ELEMS);
  rc |= dmalloc(&h->linv, (size_t)h->cap_nt * nb * nb);
  rc |= dmalloc(&h->d_stat, 4);
  rc |= dmalloc(&h->d_ctr, 4);
  rc |= dmalloc(&h->d_xk, nb);
  rc |= dmalloc(&h->d_vec, 4 * (size_t)cnp);
  h->red_len = 2 * h->cap_nt + 64;
  rc |= dmalloc(&h->d_red, h->red_len);
  h->scratch_elems = tlr_scratch_want(h);
  rc |= dmalloc(&h->scratch, h->scratch_elems);
  if (rc != TLR_OK) {
    free_ctx(h);
    TLR_RETURN_OOM();
  }
  *out = h;
  return TLR_OK;
}


int tlr_arena_alloc(double** U, double** V, int64_t* arena, int64_t need) {
  if (need <= *arena) return TLR_OK;
  if (*U) cudaFree(*U);
  if (*V) cudaFree(*V);
  *U = *V = nullptr;
  *arena = 0;
  const int64_t want = need;
  if (cudaMalloc((void**)U, (size_t)want * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)V, (size_t)want * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (*U) cudaFree(*U);
    *U = nullptr;
    TLR_RETURN_OOM();
  }
  *arena = want;
  return TLR_OK;
}

int tlr_take_grow(tlr_ctx* h, cudaStream_t s, const unsigned long long* d_top, int64_t* need) {
  long long st[2];
  unsigned long long top = 0;
  TLR_CUDA_TRY(cudaMemcpyAsync(st, h->d_stat, sizeof(st), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaMemcpyAsync(&top, d_top, sizeof(top), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  *need = 0;
  if (st[ST_CODE] != TLR_ST_GROW && st[ST_CODE] != TLR_ST_WIDEN) return TLR_OK;
  TLR_CUDA_TRY(cudaMemsetAsync(h->d_stat, 0, 4 * sizeof(long long), s));
  // every block asked for, the failed ones included; -1: the update workspaces were too narrow
  *need = st[ST_CODE] == TLR_ST_WIDEN ? -1 : (int64_t)top;
  return TLR_OK;
}

namespace {
// after an arena ran out (need > 0: the entries asked for) or an update workspace was too narrow
// (need < 0): the arena half as large again as asked for (at least 1.5 times its size), or the widest
// workspaces
int tlr_enlarge(tlr_ctx* h, int64_t need) {
  if (need < 0) return tlr_widen(h);
  return tlr_arena_alloc(&h->U, &h->V, &h->arena, std::max(need + need / 2, h->arena + h->arena / 2));
}

// compression into a fresh arena: every tile starts without columns
int compress_fresh(tlr_ctx* h, double eps, cudaStream_t s) {
  if (h->ntiles <= 0) return TLR_OK;
  TLR_CUDA_TRY(cudaMemsetAsync(h->cap, 0, h->ntiles * sizeof(int), s));
  TLR_CUDA_TRY(cudaMemsetAsync(h->top, 0, sizeof(unsigned long long), s));
  return tlr_compress_tiles(h, eps, s);
}

// compression with the arena enlarged and the compression repeated while it runs out
int compress_grow(tlr_ctx* h, double eps, cudaStream_t s) {
  for (int attempt = 0;; ++attempt) {
    TRY(compress_fresh(h, eps, s));
    int64_t need = 0;
    TRY(tlr_take_grow(h, s, h->top, &need));
    if (need == 0) return TLR_OK;
    if (attempt >= 4) TLR_RETURN_OOM();
    TRY(tlr_enlarge(h, need));
  }
}
}  // namespace

extern "C" {

int tlr_create(int64_t n, const double* x, const double* y, const tlr_opts* opts, tlr_stream_t stream,
               tlr_handle* out) {
  if (n <= 0 || n > (int64_t)INT32_MAX) return -1;
  if (!x) return -2;
  if (!y) return -3;
  if (!opts || opts->nb <= 0 || opts->rank_cap < 0 || !(opts->eps == opts->eps)) return -4;
  if (opts->metric != 0 && opts->metric != 1) return -4;
  if (opts->metric == 1 && !(opts->radius == opts->radius)) return -4;
  if (!(opts->precision == 0 || opts->precision == 1 || (opts->precision >= 4 && opts->precision <= OZ_SMAX)))
    return -4;
  if (!out) return -6;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<double> hx(n), hy(n);
  TLR_CUDA_TRY(cudaMemcpyAsync(hx.data(), x, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaMemcpyAsync(hy.data(), y, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i)
    if (!(hx[i] == hx[i]) || !(hy[i] == hy[i])) return -2;  // NaN location

  tlr_ctx* h = nullptr;
  int rc = tlr_alloc(n, opts, &h);
  if (rc != TLR_OK) return rc;
  rc = bind_points(h, n, hx, hy, s);
  if (rc != TLR_OK) {
    free_ctx(h);
    return rc;
  }
  *out = h;
  return TLR_OK;
}

int tlr_destroy(tlr_handle h) {
  if (!h) return -1;
  cudaDeviceSynchronize();
  free_ctx(h);
  return TLR_OK;
}

int tlr_shape(tlr_handle h, int* nt, int* nb) {
  if (!h) return -1;
  if (nt) *nt = h->nt;
  if (nb) *nb = h->nb;
  return TLR_OK;
}

int tlr_matern_generate(tlr_handle h, tlr_theta th, tlr_stream_t stream) {
  if (!h) return -1;
  if (!(th.sigma2 > 0) || !(th.beta > 0) || !(th.nu > 0) || !isfinite(th.sigma2) || !isfinite(th.beta) ||
      !isfinite(th.nu))
    return -2;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->mp.sigma2 = th.sigma2;
  h->mp.beta = th.beta;
  h->mp.nu = th.nu;
  h->mp.cnu = 1.0 / (pow(2.0, th.nu - 1.0) * tgamma(th.nu));
  h->mp.psi = tlr_host_digamma(th.nu);
  TLR_CUDA_TRY(cudaMemsetAsync(h->d_stat, 0, 4 * sizeof(long long), s));
  {
    PhaseScope ps("generate", s);
    TRY(tlr_build_table(h, s));
    TRY(tlr_gen_diag(h, s));
  }
  if (h->dense) {
    TRY(tlr_plan(h, s));  // every off-diagonal tile dense, generated by the plan
    h->state = 2;
  } else {
    h->state = 1;
  }
  return TLR_OK;
}

int tlr_compress(tlr_handle h, double eps, tlr_stream_t stream) {
  if (!h) return -1;
  if (!(eps >= 0) && !h->dense) return -2;
  if (h->state < 1) return TLR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (h->dense) return TLR_OK;
  h->opts.eps = eps;
  {
    PhaseScope ps("compress", s);
    TRY(compress_grow(h, eps, s));
  }
  {
    PhaseScope ps("plan", s);
    TRY(tlr_plan(h, s));
  }
  h->state = 2;
  return TLR_OK;
}

int tlr_potrf(tlr_handle h, tlr_stream_t stream) {
  if (!h) return -1;
  if (h->state != 2) return TLR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  // the factor's ranks can outgrow the arena: then it is enlarged and the factorization repeated
  // from regenerated tiles (one synchronisation at the end to check)
  for (int attempt = 0;; ++attempt) {
    TRY(tlr_factor(h, s));
    if (h->dense) break;
    int64_t need = 0;
    TRY(tlr_take_grow(h, s, h->top, &need));
    if (need == 0) break;
    if (attempt >= 4) TLR_RETURN_OOM();
    TRY(tlr_enlarge(h, need));
    TRY(tlr_gen_diag(h, s));
    TRY(compress_grow(h, h->opts.eps, s));
    TRY(tlr_plan(h, s));
  }
  h->state = 3;
  return TLR_OK;
}

int tlr_loglik(tlr_handle h, const double* z, double* d_out3, tlr_stream_t stream) {
  if (!h) return -1;
  if (!z) return -2;
  if (!d_out3) return -3;
  if (h->state != 3) return TLR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  double* w = h->d_vec;
  TRY(tlr_permute_in(h, z, w, s));
  TRY(tlr_fwd_solve(h, w, s));
  TRY(tlr_reduce_loglik(h, w, d_out3, s));
  return TLR_OK;
}

int tlr_sample(tlr_handle h, const double* e, double* z, tlr_stream_t stream) {
  if (!h) return -1;
  if (!e) return -2;
  if (!z) return -3;
  if (h->state != 3) return TLR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  double* es = h->d_vec;
  double* zs = h->d_vec + h->npad;
  TRY(tlr_permute_in(h, e, es, s));
  TRY(tlr_lmul(h, es, zs, s));
  TRY(tlr_permute_out(h, zs, z, s));
  return TLR_OK;
}

int tlr_predict(tlr_handle h, const double* z_obs, int64_t m, const double* x_new, const double* y_new,
                double* z_new, tlr_stream_t stream) {
  if (!h) return -1;
  if (!z_obs) return -2;
  if (m < 0) return -3;
  if (!x_new && m > 0) return -4;
  if (!y_new && m > 0) return -5;
  if (!z_new && m > 0) return -6;
  if (h->state != 3) return TLR_ERR_STATE;
  if (m == 0) return TLR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  // the table must cover distances to the new points
  std::vector<double> hx(m + 2), hy(m + 2);
  TLR_CUDA_TRY(cudaMemcpyAsync(hx.data(), x_new, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaMemcpyAsync(hy.data(), y_new, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  // two observed corners (bounding box) join the new points
  double bx[2], by[2];
  {
    std::vector<double> ox(h->n), oy(h->n);
    TLR_CUDA_TRY(cudaMemcpyAsync(ox.data(), h->x, h->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaMemcpyAsync(oy.data(), h->y, h->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    bx[0] = *std::min_element(ox.begin(), ox.end());
    bx[1] = *std::max_element(ox.begin(), ox.end());
    by[0] = *std::min_element(oy.begin(), oy.end());
    by[1] = *std::max_element(oy.begin(), oy.end());
  }
  hx[m] = bx[0]; hy[m] = by[0]; hx[m + 1] = bx[1]; hy[m + 1] = by[1];
  if (set_table_range(h, dist_range(h, hx.data(), hy.data(), m + 2))) TRY(tlr_build_table(h, s));
  double* a = h->d_vec;
  PhaseScope ps("predict", s);
  TRY(tlr_permute_in(h, z_obs, a, s));
  TRY(tlr_fwd_solve(h, a, s));
  TRY(tlr_bwd_solve(h, a, s));
  TRY(tlr_krige(h, a, m, x_new, y_new, z_new, s));
  return TLR_OK;
}

int tlr_predict_var(tlr_handle h, int64_t m, const double* x_new, const double* y_new, double* var_new,
                    tlr_stream_t stream) {
  if (!h) return -1;
  if (m < 0) return -2;
  if (!x_new && m > 0) return -3;
  if (!y_new && m > 0) return -4;
  if (!var_new && m > 0) return -5;
  if (h->state != 3) return TLR_ERR_STATE;
  if (m == 0) return TLR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  // the table must cover distances to the new points (as for tlr_predict)
  std::vector<double> hx(m + 2), hy(m + 2);
  TLR_CUDA_TRY(cudaMemcpyAsync(hx.data(), x_new, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaMemcpyAsync(hy.data(), y_new, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  {
    std::vector<double> ox(h->n), oy(h->n);
    TLR_CUDA_TRY(cudaMemcpyAsync(ox.data(), h->x, h->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaMemcpyAsync(oy.data(), h->y, h->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    hx[m] = *std::min_element(ox.begin(), ox.end());
    hx[m + 1] = *std::max_element(ox.begin(), ox.end());
    hy[m] = *std::min_element(oy.begin(), oy.end());
    hy[m + 1] = *std::max_element(oy.begin(), oy.end());
  }
  if (set_table_range(h, dist_range(h, hx.data(), hy.data(), m + 2))) TRY(tlr_build_table(h, s));
  PhaseScope ps("predict_var", s);
  TRY(tlr_predict_var_sorted(h, m, x_new, y_new, var_new, s));
  return TLR_OK;
}

int tlr_status(tlr_handle h, int64_t* info) {
  if (!h) return -1;
  TLR_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  long long st[2];
  TLR_CUDA_TRY(cudaMemcpy(st, h->d_stat, sizeof(st), cudaMemcpyDeviceToHost));
  if (info) *info = st[ST_INFO];
  return (int)st[ST_CODE];
}

int tlr_rank_stats(tlr_handle h, int* kmin, double* kmean, int* kmax, int64_t* bytes) {
  if (!h) return -1;
  TLR_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  std::vector<int> r(std::max<int64_t>(h->ntiles, 1), 0);
  if (h->ntiles > 0)
    TLR_CUDA_TRY(cudaMemcpy(r.data(), h->rank, h->ntiles * sizeof(int), cudaMemcpyDeviceToHost));
  // low-rank tiles only; dense tiles are counted in bytes and in *ndense of tlr_tile_counts
  int mn = INT32_MAX, mx = 0;
  double sum = 0;
  int64_t nlr = 0;
  for (int64_t t = 0; t < h->ntiles; ++t) {
    if (h->kind && h->kind[t]) continue;
    mn = std::min(mn, r[t]); mx = std::max(mx, r[t]); sum += r[t]; ++nlr;
  }
  if (nlr == 0) mn = 0;
  if (kmin) *kmin = mn;
  if (kmax) *kmax = mx;
  if (kmean) *kmean = nlr > 0 ? sum / nlr : 0.0;
  if (bytes) *bytes = (int64_t)(8.0 * ((double)h->nt * h->nb * h->nb + (double)h->ndense * h->nb * h->nb +
                                       2.0 * h->nb * sum));
  return TLR_OK;
}

int tlr_get_tile(tlr_handle h, int i, int j, double* U, double* V, int* k, int* dense, tlr_stream_t stream) {
  if (!h) return -1;
  if (i < 0 || i >= h->nt) return -2;
  if (j < 0 || j > i) return -3;
  if (!U) return -4;
  if (!V && i != j && !h->dense) return -5;
  if (!k) return -6;
  if (!dense) return -7;
  if (h->state < 1) return TLR_ERR_STATE;
  *dense = 1;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = h->nb;
  if (i == j) {
    TLR_CUDA_TRY(cudaMemcpyAsync(U, h->D + (size_t)i * nb * nb, nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
    *k = h->nb;
  } else {
    const int64_t t = tile_index(i, j);
    int r = 0;
    TLR_CUDA_TRY(cudaMemcpyAsync(&r, h->rank + t, sizeof(int), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    const bool dense_tile = h->kind && h->kind[t] && h->state >= 2;
    if (dense_tile) {
      int sl = -1;
      TLR_CUDA_TRY(cudaMemcpyAsync(&sl, h->dslot + t, sizeof(int), cudaMemcpyDeviceToHost, s));
      TLR_CUDA_TRY(cudaStreamSynchronize(s));
      r = h->nb;
      TLR_CUDA_TRY(cudaMemcpyAsync(U, h->dpool + (size_t)sl * nb * nb, nb * nb * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    } else if (r > 0) {
      *dense = 0;
      int64_t o = 0;
      TLR_CUDA_TRY(cudaMemcpyAsync(&o, h->off + t, sizeof(o), cudaMemcpyDeviceToHost, s));
      TLR_CUDA_TRY(cudaStreamSynchronize(s));
      TLR_CUDA_TRY(cudaMemcpyAsync(U, h->U + o, nb * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
      TLR_CUDA_TRY(cudaMemcpyAsync(V, h->V + o, nb * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (!dense_tile) *dense = 0;
    *k = r;
  }
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  return TLR_OK;
}

int tlr_tile_counts(tlr_handle h, int64_t* n_lowrank, int64_t* n_dense) {
  if (!h) return -1;
  if (n_dense) *n_dense = h->kind ? h->ndense : 0;
  if (n_lowrank) *n_lowrank = h->ntiles - (h->kind ? h->ndense : 0);
  return TLR_OK;
}

int tlr_get_perm(tlr_handle h, int* perm, tlr_stream_t stream) {
  if (!h) return -1;
  if (!perm) return -2;
  cudaStream_t s = (cudaStream_t)stream;
  TLR_CUDA_TRY(cudaMemcpyAsync(perm, h->perm, h->n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  return TLR_OK;
}

int tlr_inverse_stats(tlr_handle h, int* kmin, double* kmean, int* kmax, int64_t* n_dense) {
  if (!h) return -1;
  if (!h->rankz || !h->kindz) return TLR_ERR_STATE;
  TLR_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  std::vector<int> r(std::max<int64_t>(h->ntiles, 1), 0);
  if (h->ntiles > 0)
    TLR_CUDA_TRY(cudaMemcpy(r.data(), h->rankz, h->ntiles * sizeof(int), cudaMemcpyDeviceToHost));
  int mn = INT32_MAX, mx = 0;
  double sum = 0;
  int64_t nlr = 0;
  for (int64_t t = 0; t < h->ntiles; ++t) {
    if (h->kindz[t]) continue;
    mn = std::min(mn, r[t]); mx = std::max(mx, r[t]); sum += r[t]; ++nlr;
  }
  if (nlr == 0) mn = 0;
  if (kmin) *kmin = mn;
  if (kmax) *kmax = mx;
  if (kmean) *kmean = nlr > 0 ? sum / nlr : 0.0;
  if (n_dense) *n_dense = h->ndensez;
  return TLR_OK;
}

int tlr_memory(tlr_handle h, int64_t* total, int64_t* arenas, int64_t* arena_used, int64_t* workspace) {
  if (!h) return -1;
  TLR_CUDA_TRY(cudaStreamSynchronize(h->last_stream));
  unsigned long long top = 0, topz = 0;
  if (h->top) TLR_CUDA_TRY(cudaMemcpy(&top, h->top, sizeof(top), cudaMemcpyDeviceToHost));
  if (h->topz) TLR_CUDA_TRY(cudaMemcpy(&topz, h->topz, sizeof(topz), cudaMemcpyDeviceToHost));
  const double d = sizeof(double);
  const double nn = (double)h->nb * h->nb, ct = (double)std::max<int64_t>(h->cap_ntiles, 1);
  const double cnp = (double)h->cap_nt * h->nb;
  const double ar = 2.0 * d * ((double)h->arena + (double)h->arenaz);
  const double ws = d * ((double)h->scratch_elems + (double)h->scratch_dd_elems + (double)h->dop_elems +
                         (double)h->gpart_elems + (double)h->msave_elems);
  double fixed = d * (2 * cnp + 4 * cnp + (double)h->nb + TAB_ELEMS + h->red_len + 4) + 4.0 * h->cap_n + 16.0;
  fixed += d * 2 * h->cap_nt * nn + ct * (4 + 4 + 8 + 4) + 8;               // D, linv, rank, dslot, off, cap
  fixed += d * (double)h->dcap * nn + 8.0 * (double)h->list_cap;            // dense pool, plan lists
  if (h->Dz) fixed += d * h->cap_nt * nn + ct * (4 + 4 + 8 + 4) + 8 + d * (double)h->dcapz * nn +
                      8.0 * (double)h->zlist_cap;
  if (total) *total = (int64_t)(fixed + ar + ws);
  if (arenas) *arenas = (int64_t)ar;
  if (arena_used) *arena_used = (int64_t)(2.0 * d * ((double)top + (h->Dz ? (double)topz : 0.0)));
  if (workspace) *workspace = (int64_t)ws;
  return TLR_OK;
}

int tlr_profile_phases(char* buf, int64_t len) {
  if (!buf || len <= 0) return -1;
  TLR_CUDA_TRY(cudaDeviceSynchronize());
  struct Acc {
    std::string name;
    double ms;
    int count;
    long long launches;
  };
  std::vector<Acc> acc;
  for (auto& r : g_ph) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    bool found = false;
    for (auto& e : acc)
      if (e.name == r.name) { e.ms += t; e.count += 1; e.launches += r.l1 - r.l0; found = true; }
    if (!found) acc.push_back({r.name, t, 1, r.l1 - r.l0});
  }
  std::string out = "{";
  for (size_t i = 0; i < acc.size(); ++i) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "%s\"%s\": [%.3f, %d, %lld]", i ? ", " : "", acc[i].name.c_str(), acc[i].ms,
             acc[i].count, acc[i].launches);
    out += tmp;
  }
  out += "}";
  snprintf(buf, (size_t)len, "%s", out.c_str());
  return TLR_OK;
}

int tlr_launch_count(int64_t* count) {
  if (!count) return -1;
  *count = g_tlr_launches.load();
  return TLR_OK;
}

int tlr_profile(int enable) {
  if (!g_tlr_prof.d_flops) {
    if (cudaMalloc((void**)&g_tlr_prof.d_flops, 2 * sizeof(double)) != cudaSuccess) TLR_RETURN_OOM();
  }
  TLR_CUDA_TRY(cudaDeviceSynchronize());
  TLR_CUDA_TRY(cudaMemset(g_tlr_prof.d_flops, 0, 2 * sizeof(double)));
  for (auto& e : g_ev) g_ev_free.push_back(e);
  g_ev.clear();
  for (auto& e : g_ev_tc) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  g_ev_tc.clear();
  for (auto& r : g_ph) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  g_ph.clear();
  g_ph_open.clear();
  g_tlr_prof.enabled = enable ? 1 : 0;
  return TLR_OK;
}

int tlr_profile_read_tc(int64_t* launches, double* ms, double* flops) {
  TLR_CUDA_TRY(cudaDeviceSynchronize());
  double tot = 0.0;
  for (auto& e : g_ev_tc) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.first, e.second) == cudaSuccess) tot += t;
  }
  double fl[2] = {0.0, 0.0};
  if (g_tlr_prof.d_flops) TLR_CUDA_TRY(cudaMemcpy(fl, g_tlr_prof.d_flops, sizeof(fl), cudaMemcpyDeviceToHost));
  if (launches) *launches = (int64_t)g_ev_tc.size();
  if (ms) *ms = tot;
  if (flops) *flops = fl[1];
  return TLR_OK;
}

int tlr_profile_read(int64_t* launches, double* ms, double* flops) {
  TLR_CUDA_TRY(cudaDeviceSynchronize());
  double tot = 0.0;
  const bool verbose = getenv("TLR_VERBOSE") != nullptr;
  for (size_t i = 0; i < g_ev.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_ev[i].first, g_ev[i].second) == cudaSuccess) tot += t;
    if (verbose) fprintf(stderr, "tlr launch %zu: %.3f ms\n", i, t);
  }
  double fl = 0.0;
  if (g_tlr_prof.d_flops) TLR_CUDA_TRY(cudaMemcpy(&fl, g_tlr_prof.d_flops, sizeof(double), cudaMemcpyDeviceToHost));
  if (launches) *launches = (int64_t)g_ev.size();
  if (ms) *ms = tot;
  if (flops) *flops = fl;
  return TLR_OK;
}

}  // extern "C"


int tlr_rebind(tlr_ctx* h, int64_t n, const double* x, const double* y, cudaStream_t s) {
  if (n <= 0 || n > h->cap_n) return -1;
  std::vector<double> hx(n), hy(n);
  TLR_CUDA_TRY(cudaMemcpyAsync(hx.data(), x, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaMemcpyAsync(hy.data(), y, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i)
    if (!(hx[i] == hx[i]) || !(hy[i] == hy[i])) return -2;
  return bind_points(h, n, hx, hy, s);
}

// Host plan of one factorization: tile kinds (dense above dense_rank or where
// fill-in from two dense tiles lands), dense-pool slots, per-step item lists.
int tlr_plan(tlr_ctx* h, cudaStream_t s) {
  const int nt = h->nt;
  const int64_t T = h->ntiles;
  std::vector<int> rk(std::max<int64_t>(T, 1), 0);
  if (!h->dense && T > 0) {
    TLR_CUDA_TRY(cudaMemcpyAsync(rk.data(), h->rank, T * sizeof(int), cudaMemcpyDeviceToHost, s));
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  free(h->kind);
  h->kind = (char*)calloc(std::max<int64_t>(T, 1), 1);
  if (!h->kind) TLR_RETURN_OOM();
  for (int64_t t = 0; t < T; ++t) h->kind[t] = h->dense || rk[t] < 0 || rk[t] > h->dense_rank;
  for (int k = 0; k < nt; ++k)  // symbolic right-looking fill closure
    for (int j = k + 1; j < nt; ++j)
      if (h->kind[tile_index(j, k)])
        for (int i = j + 1; i < nt; ++i)
          if (h->kind[tile_index(i, k)]) h->kind[tile_index(i, j)] = 1;
  std::vector<int> slot(std::max<int64_t>(T, 1), -1);
  int nd = 0;
  for (int64_t t = 0; t < T; ++t)
    if (h->kind[t]) slot[t] = nd++;
  if (nd > h->dcap) {
    if (h->dpool) cudaFree(h->dpool);
    h->dpool = nullptr;
    h->dcap = 0;
    const int want = nd + nd / 8 + 1;
    if (cudaMalloc((void**)&h->dpool, (size_t)want * h->nb * h->nb * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      h->dpool = nullptr;
      TLR_RETURN_OOM();
    }
    h->dcap = want;
  }
  h->ndense = nd;
  h->zplan_valid = 0;
  // lists: per step 4 phases, then the dense-generation list
  std::vector<int2> L;
  std::vector<int64_t> off((size_t)nt * PLAN_PH + 1, 0);
  for (int k = 0; k < nt; ++k) {
    for (int ph = 0; ph < PLAN_PH; ++ph) {
      off[(size_t)k * PLAN_PH + ph] = (int64_t)L.size();
      if (ph == PH_TRSM_LR || ph == PH_TRSM_D) {
        const char want = ph == PH_TRSM_D;
        for (int i = k + 1; i < nt; ++i)
          if (h->kind[tile_index(i, k)] == want) L.push_back(make_int2(i, k));
      } else {
        const char want = ph == PH_UPD_D;
        const size_t b = L.size();
        for (int i = k + 2; i < nt; ++i)
          for (int j = k + 1; j < i; ++j)
            if (h->kind[tile_index(i, j)] == want) L.push_back(make_int2(i, j));
        if (ph == PH_UPD_LR) {
          // longest items first (the recompression cost grows with the square of
          // the concatenated rank), so that a launch does not end on a long tail
          auto r = [&](int p, int q) { return h->kind[tile_index(p, q)] ? h->nb : rk[tile_index(p, q)]; };
          auto est = [&](int2 t) { const int K = r(t.x, t.y) + std::min(r(t.x, k), r(t.y, k)); return K * K; };
          std::stable_sort(L.begin() + b, L.end(), [&](int2 a, int2 c) { return est(a) > est(c); });
          // items with a dense operand first: their products are formed by a batched GEMM before the launch
          std::stable_partition(L.begin() + b, L.end(), [&](int2 t) {
            return h->kind[tile_index(t.x, k)] || h->kind[tile_index(t.y, k)];
          });
        }
      }
    }
  }
  off[(size_t)nt * PLAN_PH] = (int64_t)L.size();
  const int64_t gen0 = (int64_t)L.size();
  for (int i = 1; i < nt; ++i)
    for (int j = 0; j < i; ++j)
      if (h->kind[tile_index(i, j)]) L.push_back(make_int2(i, j));
  const int64_t len = std::max<int64_t>((int64_t)L.size(), 1);
  if (len > h->list_cap) {
    if (h->d_list) cudaFree(h->d_list);
    h->d_list = nullptr;
    if (cudaMalloc((void**)&h->d_list, len * sizeof(int2)) != cudaSuccess) {
      cudaGetLastError();
      h->list_cap = 0;
      TLR_RETURN_OOM();
    }
    h->list_cap = len;
  }
  free(h->h_list);
  free(h->plan_off);
  h->h_list = (int2*)malloc(len * sizeof(int2));
  h->plan_off = (int64_t*)malloc(off.size() * sizeof(int64_t));
  if (!h->h_list || !h->plan_off) TLR_RETURN_OOM();
  if (!L.empty()) memcpy(h->h_list, L.data(), L.size() * sizeof(int2));
  memcpy(h->plan_off, off.data(), off.size() * sizeof(int64_t));
  if (!L.empty())
    TLR_CUDA_TRY(cudaMemcpyAsync(h->d_list, h->h_list, L.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  if (T > 0)
    TLR_CUDA_TRY(cudaMemcpyAsync(h->dslot, slot.data(), T * sizeof(int), cudaMemcpyHostToDevice, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors die at return
  if (nd > 0) {
    int rc = tlr_gen_dense_tiles(h, h->d_list + gen0, nd, s);
    if (rc) return rc;
  }
  return TLR_OK;
}

namespace {
// l out; dl/dsigma2 = (q - n) / (2 sigma2) since dSigma/dsigma2 = Sigma / sigma2
__global__ void k_grad_finish(const double* __restrict__ ll3, double* __restrict__ d_ll, double* __restrict__ g3,
                              int64_t n, double sigma2) {
  if (threadIdx.x == 0) {
    d_ll[0] = ll3[0];
    g3[0] = (ll3[2] - (double)n) / (2.0 * sigma2);
  }
}
}  // namespace

extern "C" int tlr_loglik_grad(tlr_handle h, const double* z, double* d_ll, double* d_grad3, tlr_stream_t stream) {
  if (!h) return -1;
  if (!z) return -2;
  if (!d_ll) return -3;
  if (!d_grad3) return -4;
  if (h->state != 3) return TLR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  double* w = h->d_vec;              // L^{-1} z
  double* a = h->d_vec + h->npad;    // Sigma^{-1} z
  double* ll3 = h->d_red + 2 * h->nt;  // (l, log|Sigma|, quad)
  {
    PhaseScope ps("solves", s);
    TRY(tlr_permute_in(h, z, w, s));
    TRY(tlr_fwd_solve(h, w, s));
    TRY(tlr_reduce_loglik(h, w, ll3, s));
    TLR_CUDA_TRY(cudaMemcpyAsync(a, w, h->npad * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(tlr_bwd_solve(h, a, s));
  }
  int fused = 0;
  TRY(tlr_inverse(h, s, a, d_grad3, &fused));
  if (!fused) {
    PhaseScope ps("grad_fused", s);
    TRY(tlr_grad_fused(h, a, d_grad3, s));
  }
  k_grad_finish<<<1, 32, 0, s>>>(ll3, d_ll, d_grad3, h->n, h->mp.sigma2);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}
