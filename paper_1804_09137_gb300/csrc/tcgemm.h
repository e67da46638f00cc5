// Float64-accurate GEMM on the bf16 tensor cores (tcgen05) by splitting each
// operand into bf16 digit slices (Ozaki, Ogita, Oishi, Rump 2012: error-free
// splitting of a product into sums of exactly computable products).
//
//   C = beta C + alpha op(A) op(B),  op(A) m x k,  op(B) k x n,  column-major C.
//
// Every row a of op(A) (column b of op(B)) is scaled by a power of two 2^-s_a so
// that its entries lie in (-1, 1), and the 53-bit fixed-point value is cut into
// S digits of 8 bits, digit j carrying weight 2^-8(j+1): each digit is an exact
// bf16 number.  Products of digits j and l are exact in the tensor core and land
// on the grid 2^-8(j+l+2); for the groups j + l = 0, 1, 2 the float32
// accumulation over a K-chunk of 128 stays below 2^24 grid units, so it is exact,
// and each chunk is added to a double-float running sum; the groups j + l >= 3
// share one float32 accumulator (their rounding lies below 2^-46 of the scale).
// Pairs with j + l >= S are dropped.  The error is at most about
// (S + 1) 2^-8S k max|a_row| max|b_col| (S = 6: ~2^-45 relative to that scale).
//
// The split is a separate pass before the GEMM that writes the slices in the
// tensor core's K-major core-matrix layout, tile by tile, so that the GEMM moves
// each tile into shared memory with one bulk (TMA) copy per operand and stage.
#pragma once
#include "tileops.h"

#define OZ_BM 128     // rows of op(A) per CTA (tcgen05 M)
#define OZ_BN 64      // columns of op(B) per CTA (tcgen05 N)
#define OZ_BK 32      // depth of one pipeline stage
#define OZ_SMAX 6     // largest number of slices (three pipeline stages of shared memory)

// One operand split into slices: rows x depth (padded to the tile grid).
struct OzSplit {
  const uint16_t* sl;  // bf16 slices, [row block][k block][slice][tile in core-matrix layout]
  const int* ex;       // per row: biased float64 exponent E with |x| < 2^(E - 1022) for every x of the row
  int rows;            // logical rows
  int nkb;             // k blocks of OZ_BK
};

// Source description of one operand for the split: element (r, k) of the rows x depth
// matrix is X[k * ld + r] (col = 1) or X[r * ld + k] (col = 0).  An operand may be made of
// several segments along k (multi = 1), each split into its own k blocks kb0 .. of an operand
// with nkb blocks in all; the row exponents are then the maximum over the segments (ex zeroed
// by the caller before the split, all segments of an operand in the same oz_split call).
struct OzSrc {
  const double* X;
  int ld;
  int col;
  int rows;
  int depth;
  uint16_t* out;  // slices destination (oz_slices_elems(rows, depth, block_rows, S) bf16 values)
  int* ex;        // rows exponents
  int block_rows; // OZ_BM for the A operand, OZ_BN for the B operand
  int kb0 = 0;    // first k block of this segment
  int nkb = 0;    // k blocks of the whole operand (0: this segment alone)
  int multi = 0;  // 1: one of several segments (exponents by atomic maximum)
};

// What the epilogue does with op(A) op(B): mode 0 writes C = beta C + alpha op(A) op(B); mode 1
// (the likelihood gradient, tile (ta, tb) of Sigma^{-1} = op(A) op(B)) adds
//   sum over its entries (a, b) [strictly below the diagonal when diag] of
//   (alpha_a alpha_b - Z_ab) dC/dtheta_p(|s_a - s_b|),  p = beta, nu,
// with the derivatives regenerated from the Matern table, into part[2 (part_off + tile)].
struct OzGemm {
  OzSplit a, b;
  double* C;
  int ldc, m, n;
  double alpha, beta;
  int lower;  // only entries with row >= column are written
  int mode = 0;
  int diag = 0;
  int64_t p0a = 0, p0b = 0;  // first sorted point of the row / column tile (mode 1)
  int64_t part_off = 0;      // first partial slot of this item (mode 1)
};

// Shared inputs of the gradient epilogue (mode 1).
struct OzGradCtx {
  const double* x;      // sorted coordinates
  const double* y;
  const double* alpha;  // Sigma^{-1} z in sorted order
  const double* tab;    // Matern table
  MaternParams mp;
  int64_t n;            // points
  double* part;         // partial sums, 2 per CTA tile
};

size_t oz_slices_elems(int rows, int depth, int block_rows, int S);
// Run `count` GEMMs described on the host (GemmGen semantics: column-major, transposes, alpha,
// beta, lower) on the tensor cores with S slices, in chunks that fit the device workspace
// ws (ws_bytes bytes, 128-byte aligned); entries with k = 0 only scale C by beta.  TLR_ERR_OOM when
// one GEMM alone does not fit.  Time-outs are recorded in d_stat.
int oz_run_host(const GemmGen* g, int count, int S, void* ws, size_t ws_bytes, long long* d_stat, cudaStream_t s);
// The same for descriptors in device memory (written by a kernel): every entry has m <= max_m,
// n <= max_n, k <= max_k; slice buffers are sized for those bounds.  Entries with k < k_min are
// skipped (left to the caller's CUDA-core path, which must skip k >= k_min).
int oz_run_device(const GemmGen* d_g, int count, int max_m, int max_n, int max_k, int k_min, int S, void* ws,
                  size_t ws_bytes, long long* d_stat, cudaStream_t s);
// bytes of workspace oz_run_device needs per descriptor for these bounds
size_t oz_device_item_bytes(int max_m, int max_n, int max_k, int S);
// split `count` operands (descriptors on the device); max_rows / max_depth bound the grid.
// segments: some operand is made of several segments (multi = 1), so the exponents are found in a
// pass of their own before the slices; otherwise one pass does both.
int oz_split(const OzSrc* d_src, int count, int max_rows, int max_depth, int S, cudaStream_t s,
             bool segments = false);
// batched GEMMs (descriptors on the device); tiles of the largest m x n; status words for time-outs
int oz_gemm(const OzGemm* d_desc, int count, int max_m, int max_n, int S, long long* d_stat, cudaStream_t s,
            const OzGradCtx* gctx = nullptr);
