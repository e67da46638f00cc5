// Independent regions (the batched-regions workload; exact MLE per region of a
// large field, Sec. VII-VIII): likelihood and gradient of R unrelated
// problems.  Worker host threads, each with its own stream, take regions in
// turn; a worker keeps one handle per tile size and rebinds it to each
// region's points within its capacity, so regions do not allocate or free
// device memory (cudaFree would synchronise the whole device and serialise the
// workers).
#include <algorithm>
#include <atomic>
#include <map>
#include <thread>
#include <vector>

#include "common.cuh"

extern "C" int tlr_loglik_grad_batched(int R, const int64_t* n, const double* const* x, const double* const* y,
                                       const double* const* z, const tlr_theta* theta, const tlr_opts* opts,
                                       double* d_ll, double* d_grad, int* status, int nworkers,
                                       tlr_stream_t stream) {
  if (R < 0) return -1;
  if (R == 0) return TLR_OK;
  if (!n) return -2;
  if (!x) return -3;
  if (!y) return -4;
  if (!z) return -5;
  if (!theta) return -6;
  if (!opts) return -7;
  if (!d_ll) return -8;
  if (!d_grad) return -9;
  if (!status) return -10;
  for (int r = 0; r < R; ++r)
    if (n[r] <= 0 || !x[r] || !y[r] || !z[r] || opts[r].nb <= 0) return -2;
  int dev = 0;
  TLR_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t start;
  TLR_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  TLR_CUDA_TRY(cudaEventRecord(start, caller));
  const int W = std::max(1, std::min(nworkers > 0 ? nworkers : 8, R));
  // capacity per tile size: the largest region that uses it
  std::map<int, int64_t> cap;
  for (int r = 0; r < R; ++r) cap[opts[r].nb] = std::max(cap[opts[r].nb], n[r]);
  std::atomic<int> next{0};
  std::vector<int> wrc(W, TLR_OK);
  std::vector<cudaStream_t> ws(W, nullptr);
  auto work = [&](int w) {
    cudaSetDevice(dev);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { wrc[w] = TLR_ERR_CUDA; return; }
    ws[w] = s;
    cudaStreamWaitEvent(s, start, 0);
    std::map<int, tlr_handle> hs;  // nb -> handle
    for (int r = next.fetch_add(1); r < R; r = next.fetch_add(1)) {
      tlr_handle h = nullptr;
      auto it = hs.find(opts[r].nb);
      int rc = TLR_OK;
      if (it == hs.end()) {  // allocate once at this tile size's capacity, then bind
        rc = tlr_alloc(cap[opts[r].nb], &opts[r], &h);
        if (rc == TLR_OK) hs[opts[r].nb] = h;
      } else {
        h = it->second;
      }
      if (rc == TLR_OK) rc = tlr_rebind(h, n[r], x[r], y[r], s);
      if (rc == TLR_OK) rc = tlr_matern_generate(h, theta[r], s);
      if (rc == TLR_OK) rc = tlr_compress(h, opts[r].eps, s);
      if (rc == TLR_OK) rc = tlr_potrf(h, s);
      if (rc == TLR_OK) {
        int64_t info = 0;
        rc = tlr_status(h, &info);
      }
      if (rc == TLR_OK) rc = tlr_loglik_grad(h, z[r], d_ll + r, d_grad + 3 * (size_t)r, s);
      if (rc == TLR_OK) {
        int64_t info = 0;
        rc = tlr_status(h, &info);
      }
      status[r] = rc;
    }
    for (auto& kv : hs) tlr_destroy(kv.second);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < W; ++w) th.emplace_back(work, w);
  for (auto& t : th) t.join();
  int rc = TLR_OK;
  for (int w = 0; w < W; ++w) {
    if (ws[w]) {
      cudaEvent_t e;
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      cudaEventRecord(e, ws[w]);
      cudaStreamWaitEvent(caller, e, 0);
      cudaEventDestroy(e);
      cudaStreamDestroy(ws[w]);
    }
    if (wrc[w] != TLR_OK) rc = wrc[w];
  }
  cudaEventDestroy(start);
  return rc;
}
