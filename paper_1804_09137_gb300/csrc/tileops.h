// Generic batched tile operations on a TlrView (hybrid dense / low-rank tiles),
// shared by the Cholesky factorization and the inverse (TRTRI and LAUUM).
#pragma once
#include "tile.cuh"

// update algorithms: target (a, b) at step k
#define ALG_CHOL 0   // A_ab -= L_ak L_bk^T
#define ALG_TRTRI 1  // A_ab += A_ak A_kb


struct GemmGen {
  const double* A;
  const double* B;
  double* C;
  int m, n, k, lda, ldb, ldc, tA, tB;
  double alpha, beta;
  int lower;
};

// low-rank targets (recompressed at tau = eps * zeta^zpow, zeta = *d_zeta or 1) and dense targets;
// the first n_dop low-rank items have a dense operand (their products are formed by a batched GEMM
// first); the persistent low-rank kernel leaves `reserve` CTA slots free for work on another stream
int tops_update(tlr_ctx* h, const TlrView& v, int alg, int k, const int2* d_lr, int64_t n_lr, int64_t n_dop,
                const int2* d_dn, int64_t n_dn, double eps, const double* d_zeta, double zpow, cudaStream_t s,
                int reserve = 0);
// low-rank targets whose two sources are both dense (materialise, ACA, recompress); workspace ws
// (ws_elems doubles), h->scratch when null
int tops_update_dd(tlr_ctx* h, const TlrView& v, int alg, int k, const int2* d_dd, int64_t n_dd, double eps,
                   const double* d_zeta, double zpow, cudaStream_t s, double* ws = nullptr, size_t ws_elems = 0);
// doubles of workspace per item of tops_update_dd
size_t tops_dd_item_elems(const tlr_ctx* h);
// Triangular tile transforms by multiplication with an explicit nb x nb matrix M
// (for instance L_kk^{-1}): low-rank tiles U <- alpha op(M) U (which 0) or V <- alpha op(M) V (which 1);
// dense tiles A <- alpha op(M) A, or A <- alpha A op(M) when dense_right.  op(M) = M^T when transM.
// Batched multi-CTA GEMMs into a workspace, then copied back.  m_by 1 / 2: the item's own matrix
// M + m_stride * (its row / column tile index) instead of M.
int tops_trmul(tlr_ctx* h, const TlrView& v, const double* M, int transM, const int2* d_lr, int n_lr, int which,
               int transM_dense, const int2* d_dn, int n_dn, int dense_right, double alpha, cudaStream_t s,
               size_t m_stride = 0, int m_by = 0);
// X = T^{-1} for a lower triangular nb x nb tile (X fully written)
int tops_trinv(const double* T, int nb, double* X, cudaStream_t s);
// Allows kernel f to start with dyn bytes of dynamic shared memory: above the default 48 KB per block
// (static plus dynamic) the kernel must opt in.  TLR_OK or TLR_ERR_CUDA.
int tlr_smem_optin(const void* f, size_t dyn);
// true when recompressions run on two-CTA clusters (the default; the environment variable TLR_UPD_PAIR=0
// selects one CTA each)
bool tops_cluster_mode();
// batched general GEMM from a device descriptor array
// (descriptors with k >= k_skip are left out: another path computes them)
int tops_gemm(const GemmGen* d_desc, int count, int m, int n, cudaStream_t s, int k_skip = 1 << 30);
// the same for products mostly A^T B of thin column blocks (one CTA a descriptor, four rows a lane in flight)
int tops_gemm_thin(const GemmGen* d_desc, int count, cudaStream_t s);

