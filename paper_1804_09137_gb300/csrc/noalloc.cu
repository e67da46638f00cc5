// Allocation-free dense log-likelihood for small problems.
//
// Some callers cannot call cudaMalloc: code that runs after its process has
// handed all device memory to another allocator (a framework's caching pool,
// a fixed real-time budget), or code for which a device allocation is not
// allowed after start-up because it can synchronise the device or fail under
// memory pressure from other processes.  For them, tlr_loglik_dense_noalloc
// evaluates the Gaussian log-likelihood for n <= TLR_NOALLOC_MAX_N points as
// one dense tile, with all of its workspace in the file-scope device array
// below: the Matérn table, the n x n covariance being factored in place, the
// solve vector, the bounding box of the points and the reduction and status
// words.  The caller passes inputs and the output; the call makes no device
// or host heap allocation of its own.
//
// The array is static device memory of about 8.5 MB.  With CUDA's default lazy
// module loading it is reserved on a device when the library's code for it is
// first used there, i.e. by the first call on that device (which can then fail
// with TLR_ERR_CUDA under memory pressure); with CUDA_MODULE_LOADING=EAGER it is
// reserved when the library is loaded.  Either way the device holds it until
// the process exits.  Host code cannot use the array's name as a device
// address; its address is taken once per device with cudaGetSymbolAddress
// (the first call on each device does this set-up).  Every call shares the
// array and leaves the last call's contents in it, so calls that overlap on the
// GPU (on different streams, or from several host threads) race with each
// other.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

#define TLR_NOALLOC_MAX_N 1024

namespace {

constexpr size_t kD = (size_t)TLR_NOALLOC_MAX_N * TLR_NOALLOC_MAX_N;  // covariance / factor
constexpr size_t kTab = TAB_ELEMS;                                    // Matérn table
constexpr size_t kVals = TAB_ELEMS;                                   // table-node workspace
constexpr size_t kVec = TLR_NOALLOC_MAX_N;                            // solve vector
constexpr size_t kRed = 64;                                           // reduction partials
constexpr size_t kStat = 4;                                           // status words
constexpr size_t kBox = 4;                                            // bounding box of the points
constexpr size_t kTotal = kD + kTab + kVals + kVec + kRed + kStat + kBox;

__device__ __align__(256) double g_noalloc_ws[kTotal];

std::mutex g_mu;
double* g_ws_ptr[128] = {nullptr};  // device address of g_noalloc_ws, per device ordinal

// box[0..3] = min x, max x, min y, max y of the n points (one CTA)
__global__ void k_bbox(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                       double* __restrict__ box) {
  __shared__ double sh[4][TLR_THREADS];
  double v[4] = {x[0], x[0], y[0], y[0]};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    v[0] = fmin(v[0], x[i]); v[1] = fmax(v[1], x[i]);
    v[2] = fmin(v[2], y[i]); v[3] = fmax(v[3], y[i]);
  }
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q)
        sh[q][threadIdx.x] = (q & 1) ? fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + o])
                                     : fmin(sh[q][threadIdx.x], sh[q][threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x < 4) box[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

extern "C" int tlr_loglik_dense_noalloc(int64_t n, const double* x, const double* y, const double* z,
                                        tlr_theta theta, double* d_out3, tlr_stream_t stream) {
  if (n <= 0 || n > TLR_NOALLOC_MAX_N) {
    fprintf(stderr, "tlr_loglik_dense_noalloc: n = %lld outside 1..%d\n", (long long)n, TLR_NOALLOC_MAX_N);
    return -1;
  }
  if (!x) return -2;
  if (!y) return -3;
  if (!z) return -4;
  if (!(theta.sigma2 > 0) || !(theta.beta > 0) || !(theta.nu > 0) || !isfinite(theta.sigma2) ||
      !isfinite(theta.beta) || !isfinite(theta.nu))
    return -5;
  if (!d_out3) return -6;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  TLR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return TLR_ERR_CUDA;
  double* ws;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ws_ptr[dev]) {  // set-up, once per device, with that device current
      void* p = nullptr;
      TLR_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_ws));
      g_ws_ptr[dev] = (double*)p;
    }
    ws = g_ws_ptr[dev];
  }
  // the table must cover the largest distance among the points: bounding box on the device,
  // read back into a stack array
  double* box = ws + kD + kTab + kVals + kVec + kRed + kStat;
  double hb[4];
  k_bbox<<<1, TLR_THREADS, 0, s>>>(x, y, n, box);
  TLR_LAUNCH_CHECK();
  TLR_CUDA_TRY(cudaMemcpyAsync(hb, box, sizeof(hb), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  const double rmax = hypot(hb[1] - hb[0], hb[3] - hb[2]);

  // a one-tile context whose every buffer lives in the static workspace
  tlr_ctx c;
  memset(&c, 0, sizeof(c));
  c.n = n;
  c.npad = n;
  c.nb = (int)n;
  c.nt = 1;
  c.kcap = 1;
  c.x = const_cast<double*>(x);
  c.y = const_cast<double*>(y);
  c.D = ws;
  c.tab = ws + kD;
  c.scratch = ws + kD + kTab;
  c.scratch_elems = kVals;
  double* w = ws + kD + kTab + kVals;
  c.d_red = w + kVec;
  c.red_len = (int)kRed;
  c.d_stat = (long long*)(c.d_red + kRed);
  c.mp.sigma2 = theta.sigma2;
  c.mp.beta = theta.beta;
  c.mp.nu = theta.nu;
  c.mp.cnu = 1.0 / (pow(2.0, theta.nu - 1.0) * tgamma(theta.nu));
  c.mp.psi = tlr_host_digamma(theta.nu);
  c.mp.e_lo = (int)ceil(log2(rmax > 0 ? rmax : 1.0)) + 1 - TAB_OCT;
  c.last_stream = s;

  // the status words must start at zero; everything else is overwritten before it is read
  TLR_CUDA_TRY(cudaMemsetAsync(c.d_stat, 0, kStat * sizeof(double), s));
  int rc = tlr_build_table(&c, s);
  if (!rc) rc = tlr_gen_diag(&c, s);
  if (!rc) rc = tlr_potrf_tile(&c, c.D, c.nb, c.nb, 0, s);
  if (rc) return rc;
  TLR_CUDA_TRY(cudaMemcpyAsync(w, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  rc = tlr_fwd_solve(&c, w, s);
  if (!rc) rc = tlr_reduce_loglik(&c, w, d_out3, s);
  if (rc) return rc;
  long long st[2];
  TLR_CUDA_TRY(cudaMemcpyAsync(st, c.d_stat, sizeof(st), cudaMemcpyDeviceToHost, s));
  TLR_CUDA_TRY(cudaStreamSynchronize(s));
  return (int)st[ST_CODE];
}
