// Float64-accurate GEMM on the bf16 tensor cores (see tcgemm.h for the method).
//
// k_oz_slice / k_oz_slice_gen: per-row power-of-two scale and 8-bit digit slices of
// each operand in one pass (a CTA finds the exponents of its 32 rows over the whole
// depth, then slices its share of the depth), written in the K-major core-matrix
// layout of the tensor core (8 rows x 16 bytes per core matrix, the four core
// matrices of a row group along K adjacent), one contiguous block per (row block,
// k block) holding all slices.  An operand made of several segments along k takes
// two passes instead (k_oz_rowexp, exponents by atomic maximum over the segments,
// then k_oz_split).
//
// k_oz_gemm: one CTA per 128 x 64 output tile, three warp roles:
//   warp 0      producer: one bulk (TMA) copy per operand and stage into a
//               three-stage shared-memory ring (mbarrier transaction counts);
//   warp 1      allocates tensor memory (512 columns) and one thread issues the
//               tcgen05.mma of every slice pair j + l < S, 128 x 64 x 16 each;
//   warps 2..5  read the four group accumulators (j + l = 0, 1, 2 and >= 3) of
//               every 64-deep K chunk out of tensor memory (tcgen05.ld; two
//               accumulator sets in turn so the next chunk's products proceed),
//               add them into double-float running sums and write the float64
//               result with its power-of-two scales.
// Every wait is bounded: after about two seconds a role records TLR_ERR_TIMEOUT,
// the others stop, the CTA waits (bounded) for its copies and products in flight,
// frees its tensor memory and returns.
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "df.cuh"
#include "tcgemm.h"

namespace {

constexpr int NSTAGE = 3;
constexpr int CHUNK_KB = 2;               // k blocks per exactly accumulated chunk (64 products)
constexpr int NGROUP = 4;                 // accumulators per chunk: j + l = 0, 1, 2, >= 3
constexpr uint32_t TMEM_COLS = 2 * NGROUP * OZ_BN;  // two accumulator sets: 512 columns
constexpr long long WAIT_CYCLES = 4000000000LL;     // about two seconds
constexpr int OZ_THREADS = 192;

template <int S>
struct OzShape {
  static constexpr int A_SLICE = OZ_BM * OZ_BK * 2;  // bytes of one slice tile
  static constexpr int B_SLICE = OZ_BN * OZ_BK * 2;
  static constexpr int A_BYTES = S * A_SLICE;
  static constexpr int B_BYTES = S * B_SLICE;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = NSTAGE * STAGE + 256;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of the given parity to complete; false after the time limit or when
// another role has given up (abort flag in shared memory)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

// bounded wait that ignores the abort flag (draining in-flight work before exit)
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// instruction descriptor of kind::f16: bf16 A and B (K-major), float32 accumulator, M x N
__host__ __device__ constexpr uint32_t oz_idesc(int M, int N) {
  return (1u << 4)                       // accumulator format: float32
         | (1u << 7)                     // A format: bf16
         | (1u << 10)                    // B format: bf16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// shared-memory matrix descriptor, no swizzle: start address, byte offset between core
// matrices adjacent along K (leading) and along M/N (stride), descriptor version 1
__device__ __forceinline__ uint64_t oz_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on the mbarrier once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// (hi, lo) += x, Knuth's TwoSum with the error term collected in lo
__device__ __forceinline__ void df_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

__device__ __forceinline__ int dexp(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------ split
// E[r] = largest biased exponent over row r (0 for padded rows and zero rows)
__device__ __forceinline__ void rowexp_body(const OzSrc& d) {
  const int rows_pad = round_up(d.rows, d.block_rows);
  if (d.col) {  // element (r, k) at X[k * ld + r]: a thread per row, coalesced across rows
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows_pad) return;
    int E = 0;
    if (r < d.rows)
      for (int k = 0; k < d.depth; ++k) E = max(E, dexp(d.X[(size_t)k * d.ld + r]));
    if (d.multi) atomicMax(&d.ex[r], E);
    else d.ex[r] = E;
  } else {  // element (r, k) at X[r * ld + k]: a warp per row
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= rows_pad) return;
    int E = 0;
    if (r < d.rows)
      for (int k = lane; k < d.depth; k += 32) E = max(E, dexp(d.X[(size_t)r * d.ld + k]));
    for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) {
      if (d.multi) atomicMax(&d.ex[r], E);
      else d.ex[r] = E;
    }
  }
}

__global__ void k_oz_rowexp(const OzSrc* __restrict__ srcs) { rowexp_body(srcs[blockIdx.y]); }

// digits of 8 consecutive k of one row: thread (row r, k octet q)
template <int S>
__global__ void k_oz_split(const OzSrc* __restrict__ srcs) {
  const OzSrc d = srcs[blockIdx.z];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y * blockDim.y + threadIdx.y;
  const int BR = d.block_rows;
  const int rows_pad = round_up(d.rows, BR);
  const int depth_pad = round_up(d.depth, OZ_BK);
  if (r >= rows_pad || q * 8 >= depth_pad) return;
  const int E = d.ex[r];
  uint32_t w[S][4];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int i = 0; i < 4; ++i) w[s][i] = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = q * 8 + j;
    double x = 0.0;
    if (r < d.rows && k < d.depth) x = d.col ? d.X[(size_t)k * d.ld + r] : d.X[(size_t)r * d.ld + k];
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long F = 0ull;  // |x| 2^-(E - 1022) as a fraction with 64 bits
    if (e != 0 && e != 0x7ff) {
      const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = E - e;
      F = sh <= 11 ? (mant << (11 - sh)) : (sh - 11 < 64 ? (mant >> (sh - 11)) : 0ull);
    }
    const uint32_t sgn = (uint32_t)(b >> 63) << 31;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const uint32_t dg = (uint32_t)(F >> (56 - 8 * s)) & 0xffu;
      // dg * 2^-8(s+1): exact in float32, and in bf16 (at most 8 significant bits)
      const float v = (float)dg * __int_as_float((127 - 8 * (s + 1)) << 23);
      const uint32_t h = dg ? ((sgn | (uint32_t)__float_as_int(v)) >> 16) : 0u;
      w[s][j >> 1] |= h << (16 * (j & 1));
    }
  }
  const int nkb = d.nkb > 0 ? d.nkb : depth_pad / OZ_BK;
  const int rb = r / BR, rr = r % BR, kb = d.kb0 + (q * 8) / OZ_BK, kq = ((q * 8) % OZ_BK) / 8;
  const size_t tile = (size_t)BR * OZ_BK;  // bf16 per slice tile
  const size_t in_tile = (size_t)((rr >> 3) * (OZ_BK / 8) + kq) * 64 + (size_t)(rr & 7) * 8;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    uint16_t* dst = d.out + (((size_t)rb * nkb + kb) * S + s) * tile + in_tile;
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// One pass for an operand that is a single segment: a CTA of 32 x 8 threads takes the 32 rows
// r0 .. r0 + 31, finds their exponents over the whole depth, then writes the slices of the k octets
// [q0, q1) (thread (row, y) the octets y, y + 8, ...).  The exponents are stored by the CTAs with
// q0 = 0.  A CTA beyond the operand's padded rows returns at once (uniformly).
template <int S>
__device__ __forceinline__ void slice_rows(const OzSrc& d, int r0, int q0, int q1) {
  __shared__ int part[8][33];
  __shared__ int rowE[32];
  const int BR = d.block_rows;
  const int rows_pad = round_up(d.rows, BR);
  if (r0 >= rows_pad) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (d.col) {  // element (r, k) at X[k ld + r]: a warp reads 32 rows of one k
    const int r = r0 + tx;
    int E = 0;
    if (r < d.rows)
      for (int k = ty; k < d.depth; k += 8) E = max(E, dexp(d.X[(size_t)k * d.ld + r]));
    part[ty][tx] = E;
    __syncthreads();
    if (ty == 0) {
#pragma unroll
      for (int i = 1; i < 8; ++i) E = max(E, part[i][tx]);
      rowE[tx] = E;
    }
  } else {  // element (r, k) at X[r ld + k]: warp y reads the rows y, y + 8, y + 16, y + 24 along k
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = ty + 8 * i, r = r0 + rr;
      int E = 0;
      if (r < d.rows)
        for (int k = tx; k < d.depth; k += 32) E = max(E, dexp(d.X[(size_t)r * d.ld + k]));
      for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
      if (tx == 0) rowE[rr] = E;
    }
  }
  __syncthreads();
  const int r = r0 + tx;
  const int E = rowE[tx];
  if (q0 == 0 && ty == 0) d.ex[r] = E;
  const int depth_pad = round_up(d.depth, OZ_BK);
  const int qend = min(q1, depth_pad / 8);
  const int nkb = d.nkb > 0 ? d.nkb : depth_pad / OZ_BK;
  const int rb = r / BR, rr = r % BR;
  const size_t tile = (size_t)BR * OZ_BK;  // bf16 per slice tile
  for (int q = q0 + ty; q < qend; q += 8) {
    uint32_t w[S][4];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i) w[s][i] = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = q * 8 + j;
      double x = 0.0;
      if (r < d.rows && k < d.depth) x = d.col ? d.X[(size_t)k * d.ld + r] : d.X[(size_t)r * d.ld + k];
      const unsigned long long b = (unsigned long long)__double_as_longlong(x);
      const int e = (int)((b >> 52) & 0x7ff);
      unsigned long long F = 0ull;  // |x| 2^-(E - 1022) as a fraction with 64 bits
      if (e != 0 && e != 0x7ff) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - e;
        F = sh <= 11 ? (mant << (11 - sh)) : (sh - 11 < 64 ? (mant >> (sh - 11)) : 0ull);
      }
      const uint32_t sgn = (uint32_t)(b >> 63) << 31;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const uint32_t dg = (uint32_t)(F >> (56 - 8 * s)) & 0xffu;
        const float v = (float)dg * __int_as_float((127 - 8 * (s + 1)) << 23);
        const uint32_t h = dg ? ((sgn | (uint32_t)__float_as_int(v)) >> 16) : 0u;
        w[s][j >> 1] |= h << (16 * (j & 1));
      }
    }
    const int kb = d.kb0 + (q * 8) / OZ_BK, kq = ((q * 8) % OZ_BK) / 8;
    const size_t in_tile = (size_t)((rr >> 3) * (OZ_BK / 8) + kq) * 64 + (size_t)(rr & 7) * 8;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint16_t* dst = d.out + (((size_t)rb * nkb + kb) * S + s) * tile + in_tile;
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// single-segment operands described on the device: blockIdx.z the operand, blockIdx.y the depth chunk
template <int S>
__global__ void __launch_bounds__(256) k_oz_slice(const OzSrc* __restrict__ srcs, int qpc) {
  const OzSrc d = srcs[blockIdx.z];
  slice_rows<S>(d, blockIdx.x * 32, blockIdx.y * qpc, (blockIdx.y + 1) * qpc);
}

// k octets per depth chunk so that rows32 x count x chunks CTAs fill the GPU about twice
inline int slice_chunk_octets(int rows_pad, int depth_pad, int count) {
  const int Q = depth_pad / 8;
  const long long ctas = (long long)(rows_pad / 32) * count;
  const long long target = 2432;  // 152 SMs x 8 resident CTAs of 256 threads x 2
  int nz = ctas >= target ? 1 : (int)((target + ctas - 1) / ctas);
  nz = std::max(1, std::min(nz, (Q + 7) / 8));
  return round_up((Q + nz - 1) / nz, 8);
}

// ------------------------------------------------------------------ GEMM
template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const OzGemm* __restrict__ descs, int tiles_m,
                                                           long long* __restrict__ st, const OzGradCtx gx,
                                                           double* __restrict__ mma_flops) {
  using Sh = OzShape<S>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const OzGemm g = descs[blockIdx.y];
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int r0 = tm * OZ_BM, c0 = tn * OZ_BN;
  if (r0 >= g.m || c0 >= g.n) return;
  if (g.lower && r0 + OZ_BM - 1 < c0) return;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * Sh::STAGE);
  uint64_t* full = bars;                   // NSTAGE
  uint64_t* empty = bars + NSTAGE;         // NSTAGE
  uint64_t* acc_full = bars + 2 * NSTAGE;  // 2
  uint64_t* acc_empty = acc_full + 2;      // 2
  uint64_t* done = acc_empty + 2;          // 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = g.a.nkb;
  const int nchunk = (nkb + CHUNK_KB - 1) / CHUNK_KB;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0 && nkb > 0) {
      const uint8_t* srcA = reinterpret_cast<const uint8_t*>(g.a.sl) + (size_t)tm * nkb * Sh::A_BYTES;
      const uint8_t* srcB = reinterpret_cast<const uint8_t*>(g.b.sl) + (size_t)tn * nkb * Sh::B_BYTES;
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int stg = kb % NSTAGE, use = kb / NSTAGE;
        if (use > 0 && !mbar_wait(&empty[stg], (use - 1) & 1, abort_flag)) {
          set_status(st, TLR_ERR_TIMEOUT, 1);
          *abort_flag = 1;
          break;
        }
        uint8_t* dst = smem + stg * Sh::STAGE;
        mbar_expect_tx(&full[stg], Sh::STAGE);
        bulk_g2s(dst, srcA + (size_t)kb * Sh::A_BYTES, Sh::A_BYTES, &full[stg]);
        bulk_g2s(dst + Sh::A_BYTES, srcB + (size_t)kb * Sh::B_BYTES, Sh::B_BYTES, &full[stg]);
        issued = kb + 1;
      }
      if (*abort_flag) {  // let the copies in flight land before the CTA exits
        for (int kb = max(0, issued - NSTAGE); kb < issued; ++kb) mbar_drain(&full[kb % NSTAGE], (kb / NSTAGE) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = oz_idesc(OZ_BM, OZ_BN);
      constexpr uint32_t LBO = 128, SBO = (OZ_BK / 8) * 128;
      bool ok = nkb > 0;
      for (int c = 0; c < nchunk && ok; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(&acc_empty[buf], ((c >> 1) - 1) & 1, abort_flag)) {
          set_status(st, TLR_ERR_TIMEOUT, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t gbase = tmem + (uint32_t)(buf * NGROUP * OZ_BN);
        bool started[NGROUP] = {false, false, false, false};
        const int kb1 = min(nkb, (c + 1) * CHUNK_KB);
        for (int kb = c * CHUNK_KB; kb < kb1; ++kb) {
          const int stg = kb % NSTAGE, use = kb / NSTAGE;
          if (!mbar_wait(&full[stg], use & 1, abort_flag)) {
            set_status(st, TLR_ERR_TIMEOUT, 3);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aBase = smem_u32(smem + stg * Sh::STAGE);
          const uint32_t bBase = aBase + Sh::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
            for (int dd = 0; dd < S; ++dd) {
              const int grp = dd < NGROUP - 1 ? dd : NGROUP - 1;
#pragma unroll
              for (int j = 0; j <= dd; ++j) {
                const int l = dd - j;
                const uint64_t ad = oz_sdesc(aBase + j * Sh::A_SLICE + kk * 256, LBO, SBO);
                const uint64_t bd = oz_sdesc(bBase + l * Sh::B_SLICE + kk * 256, LBO, SBO);
                tc_mma(gbase + grp * OZ_BN, ad, bd, idesc, started[grp] ? 1u : 0u);
                started[grp] = true;
              }
            }
          }
          tc_commit(&empty[stg]);  // the stage's shared memory is free once these products finish
        }
        if (!ok) break;
        tc_commit(&acc_full[buf]);  // the chunk's accumulators are complete
      }
      tc_commit(done);  // every product issued has completed
      if (mma_flops && nkb > 0)  // tensor-core work of this tile: S (S + 1) / 2 slice pairs
        atomicAdd(mma_flops, 2.0 * OZ_BM * OZ_BN * OZ_BK * (double)nkb * (S * (S + 1) / 2));
    }
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lane quarter warp % 4
    const int qtr = warp & 3;
    const int row = 32 * qtr + lane;
    float hi[OZ_BN], lo[OZ_BN];
#pragma unroll
    for (int j = 0; j < OZ_BN; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      const int buf = c & 1;
      if (!mbar_wait(&acc_full[buf], (c >> 1) & 1, abort_flag)) {
        set_status(st, TLR_ERR_TIMEOUT, 4);
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(32 * qtr) << 16) + (uint32_t)(buf * NGROUP * OZ_BN);
#pragma unroll
      for (int c16 = 0; c16 < OZ_BN; c16 += 16) {
#pragma unroll
        for (int gq = 0; gq < (S > 3 ? 4 : 3); ++gq) {
          uint32_t v[16];
          tmem_ld16(base + gq * OZ_BN + c16, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) df_acc(hi[c16 + i], lo[c16 + i], __uint_as_float(v[i]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (ok && g.mode == 1) {
      // gradient: (alpha_a alpha_b - Z_ab) dC/dbeta, dC/dnu over this tile's entries, one partial per warp
      const int a = r0 + row;
      const int64_t pa = g.p0a + a;
      double g1 = 0.0, g2 = 0.0;
      if (a < g.m && pa < gx.n) {
        const int ea = nkb > 0 ? g.a.ex[a] : 0;
        const double xa = gx.x[pa], ya = gx.y[pa], wa = gx.alpha[pa];
#pragma unroll
        for (int j = 0; j < OZ_BN; ++j) {
          const int b = c0 + j;
          const int64_t pb = g.p0b + b;
          if (b < g.n && pb < gx.n && (!g.diag || a > b)) {
            const int eb = nkb > 0 ? g.b.ex[b] : 0;
            const double zab =
                (ea == 0 || eb == 0) ? 0.0 : df_to_scaled(df_norm(hi[j], lo[j]), (ea - 1022) + (eb - 1022));
            const double rr = pt_dist(gx.mp, xa, ya, gx.x[pb], gx.y[pb]);
            if (rr > 0.0) {
              double t;
              const int jt = tab_locate(rr, gx.mp.e_lo, &t);
              if (jt >= 0 && jt < TAB_NINT) {  // below the table the derivatives vanish
                const double w = wa * gx.alpha[pb] - zab;
                g1 = fma(w, tab_poly(gx.tab + (size_t)(TAB_NINT + jt) * TAB_NC, t), g1);
                g2 = fma(w, tab_poly(gx.tab + (size_t)(2 * TAB_NINT + jt) * TAB_NC, t), g2);
              }
            }
          }
        }
      }
      g1 = warp_sum(g1);
      g2 = warp_sum(g2);
      if (lane == 0) {
        double* p = gx.part + 8 * (g.part_off + blockIdx.x) + 2 * qtr;
        p[0] = g1;
        p[1] = g2;
      }
    }
    if (ok && g.mode == 0) {
      const int r = r0 + row;
      const int ea = (r < g.m && nkb > 0) ? g.a.ex[r] : 0;
#pragma unroll
      for (int j = 0; j < OZ_BN; ++j) {
        const int cc = c0 + j;
        if (r < g.m && cc < g.n && (!g.lower || r >= cc)) {
          const int eb = nkb > 0 ? g.b.ex[cc] : 0;
          const int sh = (ea - 1022) + (eb - 1022);
          const dfloat v = df_norm(hi[j], lo[j]);
          const double val = (ea == 0 || eb == 0) ? 0.0 : df_to_scaled(v, sh);
          double* cp = g.C + (size_t)cc * g.ldc + r;
          *cp = (g.beta == 0.0 ? 0.0 : g.beta * *cp) + g.alpha * val;
        }
      }
    }
  }
  // every product has completed before the tensor memory is released
  if (threadIdx.x == 32) mbar_drain(done, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int S>
int launch_split(const OzSrc* d_src, int count, int max_rows, int max_depth, bool segments, cudaStream_t s) {
  const int rows_pad = round_up(std::max(max_rows, 1), OZ_BM);
  const int depth_pad = round_up(std::max(max_depth, 1), OZ_BK);
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = std::min(65535, count - c0);
    const dim3 blk(32, 8);
    if (!segments) {  // exponents and slices in one pass
      const int qpc = slice_chunk_octets(rows_pad, depth_pad, cnt);
      k_oz_slice<S><<<dim3(rows_pad / 32, (depth_pad / 8 + qpc - 1) / qpc, cnt), blk, 0, s>>>(d_src + c0, qpc);
      TLR_LAUNCH_CHECK();
      continue;
    }
    // a warp per row covers both source orientations of the exponent pass
    k_oz_rowexp<<<dim3((rows_pad * 32 + 255) / 256, cnt), 256, 0, s>>>(d_src + c0);
    TLR_LAUNCH_CHECK();
    const dim3 grid((rows_pad + 31) / 32, (depth_pad / 8 + 7) / 8, cnt);
    k_oz_split<S><<<grid, blk, 0, s>>>(d_src + c0);
    TLR_LAUNCH_CHECK();
  }
  return TLR_OK;
}

template <int S>
int launch_gemm(const OzGemm* d_desc, int count, int max_m, int max_n, long long* d_stat, cudaStream_t s,
                const OzGradCtx* gctx) {
  OzGradCtx gx;
  if (gctx) gx = *gctx;
  else memset(&gx, 0, sizeof(gx));
  static bool attr_set[64] = {false};
  int dev = 0;
  TLR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 64 && !attr_set[dev]) {
    TLR_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, OzShape<S>::SMEM));
    attr_set[dev] = true;
  }
  const int tm = (max_m + OZ_BM - 1) / OZ_BM, tn = (max_n + OZ_BN - 1) / OZ_BN;
  double* fl = g_tlr_prof.enabled ? g_tlr_prof.d_flops + 1 : nullptr;
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = std::min(65535, count - c0);
    if (fl) tlr_prof_tc_begin(s);
    k_oz_gemm<S><<<dim3(tm * tn, cnt), OZ_THREADS, OzShape<S>::SMEM, s>>>(d_desc + c0, tm, d_stat, gx, fl);
    TLR_LAUNCH_CHECK();
    if (fl) tlr_prof_tc_end(s);
  }
  return TLR_OK;
}

}  // namespace

size_t oz_slices_elems(int rows, int depth, int block_rows, int S) {
  return (size_t)round_up(std::max(rows, 1), block_rows) * round_up(std::max(depth, 1), OZ_BK) * S;
}

int oz_split(const OzSrc* d_src, int count, int max_rows, int max_depth, int S, cudaStream_t s, bool segments) {
  if (count <= 0) return TLR_OK;
  switch (S) {
    case 4: return launch_split<4>(d_src, count, max_rows, max_depth, segments, s);
    case 5: return launch_split<5>(d_src, count, max_rows, max_depth, segments, s);
    case 6: return launch_split<6>(d_src, count, max_rows, max_depth, segments, s);
    default: return -1;
  }
}

int oz_gemm(const OzGemm* d_desc, int count, int max_m, int max_n, int S, long long* d_stat, cudaStream_t s,
            const OzGradCtx* gctx) {
  if (count <= 0) return TLR_OK;
  switch (S) {
    case 4: return launch_gemm<4>(d_desc, count, max_m, max_n, d_stat, s, gctx);
    case 5: return launch_gemm<5>(d_desc, count, max_m, max_n, d_stat, s, gctx);
    case 6: return launch_gemm<6>(d_desc, count, max_m, max_n, d_stat, s, gctx);
    default: return -1;
  }
}

namespace {
size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

size_t oz_item_bytes(const GemmGen& g, int S) {
  if (g.k <= 0 || g.m <= 0 || g.n <= 0) return align128(sizeof(OzGemm));
  return align128(oz_slices_elems(g.m, g.k, OZ_BM, S) * 2) + align128(oz_slices_elems(g.n, g.k, OZ_BN, S) * 2) +
         align128((size_t)round_up(g.m, OZ_BM) * 4) + align128((size_t)round_up(g.n, OZ_BN) * 4) +
         align128(2 * sizeof(OzSrc)) + align128(sizeof(OzGemm));
}
}  // namespace

int oz_run_host(const GemmGen* g, int count, int S, void* ws, size_t ws_bytes, long long* d_stat, cudaStream_t s) {
  // An operand that several products of a chunk share (the same matrix, layout and extent, e.g. one dense
  // tile against many thin factors) is split once and its slices read by all of them.
  struct Key {
    const double* X;
    int ld, col, rows, depth, block_rows;
    bool operator<(const Key& o) const {
      return std::tie(X, ld, col, rows, depth, block_rows) < std::tie(o.X, o.ld, o.col, o.rows, o.depth, o.block_rows);
    }
  };
  char* base = static_cast<char*>(ws);
  int q0 = 0;
  while (q0 < count) {
    std::vector<OzSrc> src;
    std::vector<OzGemm> gem;
    std::map<Key, std::pair<uint16_t*, int*>> seen;
    char* p = base;
    int max_rows = 1, max_depth = 1, max_m = 1, max_n = 1;
    int q1 = q0;
    // greedy chunk within the workspace: slices and exponents first, descriptors at the end
    auto fits = [&](size_t slice_bytes, size_t n_src, size_t n_gem) {
      return (size_t)(p - base) + slice_bytes + align128(n_src * sizeof(OzSrc)) + align128(n_gem * sizeof(OzGemm)) +
                 256 <= ws_bytes;
    };
    for (; q1 < count; ++q1) {
      const GemmGen& x = g[q1];
      OzGemm og;
      memset(&og, 0, sizeof(og));
      og.C = x.C; og.ldc = x.ldc; og.m = x.m; og.n = x.n; og.alpha = x.alpha; og.beta = x.beta; og.lower = x.lower;
      if (x.m <= 0 || x.n <= 0) continue;
      if (x.k <= 0) {
        if (!fits(0, src.size(), gem.size() + 1)) break;
        gem.push_back(og);
        max_m = std::max(max_m, x.m);
        max_n = std::max(max_n, x.n);
        continue;
      }
      // rows of op(A): (r, c) at A[c lda + r] unless transposed; rows of op(B)^T: (j, c) at B[j ldb + c]
      // unless transposed
      const Key ka{x.A, x.lda, x.tA ? 0 : 1, x.m, x.k, OZ_BM}, kb{x.B, x.ldb, x.tB ? 1 : 0, x.n, x.k, OZ_BN};
      const bool new_a = !seen.count(ka), nb_new = !seen.count(kb);  // ka != kb: their block rows differ
      auto bytes_of = [&](const Key& k) {
        return align128(oz_slices_elems(k.rows, k.depth, k.block_rows, S) * 2) +
               align128((size_t)round_up(k.rows, k.block_rows) * 4);
      };
      const size_t add = (new_a ? bytes_of(ka) : 0) + (nb_new ? bytes_of(kb) : 0);
      if (!fits(add, src.size() + (new_a ? 1 : 0) + (nb_new ? 1 : 0), gem.size() + 1)) break;
      auto place = [&](const Key& k) -> std::pair<uint16_t*, int*> {
        auto it = seen.find(k);
        if (it != seen.end()) return it->second;
        uint16_t* sl = reinterpret_cast<uint16_t*>(p);
        p += align128(oz_slices_elems(k.rows, k.depth, k.block_rows, S) * 2);
        int* ex = reinterpret_cast<int*>(p);
        p += align128((size_t)round_up(k.rows, k.block_rows) * 4);
        src.push_back({k.X, k.ld, k.col, k.rows, k.depth, sl, ex, k.block_rows});
        seen[k] = {sl, ex};
        max_rows = std::max(max_rows, k.rows);
        return {sl, ex};
      };
      const auto pa = place(ka);
      const auto pb = place(kb);
      const int nkb = round_up(x.k, OZ_BK) / OZ_BK;
      og.a = {pa.first, pa.second, x.m, nkb};
      og.b = {pb.first, pb.second, x.n, nkb};
      max_depth = std::max(max_depth, x.k);
      max_m = std::max(max_m, x.m);
      max_n = std::max(max_n, x.n);
      gem.push_back(og);
    }
    if (q1 == q0) TLR_RETURN_OOM();
    char* dp = reinterpret_cast<char*>(align128(reinterpret_cast<size_t>(p)));
    OzSrc* dsrc = reinterpret_cast<OzSrc*>(dp);
    dp += align128(src.size() * sizeof(OzSrc));
    OzGemm* dgem = reinterpret_cast<OzGemm*>(dp);
    dp += align128(gem.size() * sizeof(OzGemm));
    if (dp > base + ws_bytes) TLR_RETURN_OOM();
    if (!src.empty())
      TLR_CUDA_TRY(cudaMemcpyAsync(dsrc, src.data(), src.size() * sizeof(OzSrc), cudaMemcpyHostToDevice, s));
    if (!gem.empty())
      TLR_CUDA_TRY(cudaMemcpyAsync(dgem, gem.data(), gem.size() * sizeof(OzGemm), cudaMemcpyHostToDevice, s));
    int rc = oz_split(dsrc, (int)src.size(), max_rows, max_depth, S, s);
    if (rc) return rc;
    rc = oz_gemm(dgem, (int)gem.size(), max_m, max_n, S, d_stat, s);
    if (rc) return rc;
    q0 = q1;
  }
  return TLR_OK;
}

namespace {
// descriptor q -> split descriptors 2q (op(A)), 2q + 1 (op(B)^T) and GEMM descriptor q with fixed-size
// buffers at base + q per
__device__ __forceinline__ void descs_from_gen(const GemmGen& x, int q, int k_min, char* __restrict__ base,
                                               size_t sa_bytes, size_t sb_bytes, size_t xa_bytes, size_t per,
                                               OzSrc* a, OzSrc* b, OzGemm* og) {
  char* p = base + (size_t)q * per;
  uint16_t* sa = reinterpret_cast<uint16_t*>(p);
  uint16_t* sb = reinterpret_cast<uint16_t*>(p + sa_bytes);
  int* xa = reinterpret_cast<int*>(p + sa_bytes + sb_bytes);
  int* xb = reinterpret_cast<int*>(p + sa_bytes + sb_bytes + xa_bytes);
  const bool run = x.m > 0 && x.n > 0 && x.k >= k_min && x.k > 0;
  a->X = x.A; a->ld = x.lda; a->col = x.tA ? 0 : 1; a->rows = run ? x.m : 0; a->depth = x.k; a->out = sa; a->ex = xa;
  a->block_rows = OZ_BM; a->kb0 = 0; a->nkb = 0; a->multi = 0;
  b->X = x.B; b->ld = x.ldb; b->col = x.tB ? 1 : 0; b->rows = run ? x.n : 0; b->depth = x.k; b->out = sb; b->ex = xb;
  b->block_rows = OZ_BN; b->kb0 = 0; b->nkb = 0; b->multi = 0;
  const int nkb = (x.k + OZ_BK - 1) / OZ_BK;
  memset(og, 0, sizeof(*og));
  og->a.sl = sa; og->a.ex = xa; og->a.rows = x.m; og->a.nkb = nkb;
  og->b.sl = sb; og->b.ex = xb; og->b.rows = x.n; og->b.nkb = nkb;
  og->C = x.C; og->ldc = x.ldc; og->m = run ? x.m : 0; og->n = run ? x.n : 0;
  og->alpha = x.alpha; og->beta = x.beta; og->lower = x.lower;
}

// exponents and slices of operand blockIdx.z (descriptor z / 2, side z % 2) straight from the GEMM
// descriptors, depth chunk blockIdx.y; the first CTA of each side-0 operand also stores the GEMM
// descriptor for the product kernel
template <int S>
__global__ void __launch_bounds__(256) k_oz_slice_gen(const GemmGen* __restrict__ g, int k_min, char* __restrict__ base,
                                                      size_t sa_bytes, size_t sb_bytes, size_t xa_bytes, size_t per,
                                                      OzGemm* __restrict__ gem, int qpc) {
  const int z = blockIdx.z, q = z >> 1;
  OzSrc a, b;
  OzGemm og;
  descs_from_gen(g[q], q, k_min, base, sa_bytes, sb_bytes, xa_bytes, per, &a, &b, &og);
  if (!(z & 1) && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) gem[q] = og;
  slice_rows<S>((z & 1) ? b : a, blockIdx.x * 32, blockIdx.y * qpc, (blockIdx.y + 1) * qpc);
}

template <int S>
int launch_split_gen(const GemmGen* d_g, int cnt, int k_min, char* base, size_t sa, size_t sb, size_t xa, size_t per,
                     OzGemm* gem, int max_rows, int max_depth, cudaStream_t s) {
  const int rows_pad = round_up(std::max(max_rows, 1), OZ_BM);
  const int depth_pad = round_up(std::max(max_depth, 1), OZ_BK);
  // 2 cnt operands; callers keep cnt <= 32767
  const int qpc = slice_chunk_octets(rows_pad, depth_pad, 2 * cnt);
  k_oz_slice_gen<S><<<dim3(rows_pad / 32, (depth_pad / 8 + qpc - 1) / qpc, 2 * cnt), dim3(32, 8), 0, s>>>(
      d_g, k_min, base, sa, sb, xa, per, gem, qpc);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}
}  // namespace

size_t oz_device_item_bytes(int max_m, int max_n, int max_k, int S) {
  return align128(oz_slices_elems(max_m, max_k, OZ_BM, S) * 2) + align128(oz_slices_elems(max_n, max_k, OZ_BN, S) * 2) +
         align128((size_t)round_up(max_m, OZ_BM) * 4) + align128((size_t)round_up(max_n, OZ_BN) * 4) +
         2 * sizeof(OzSrc) + sizeof(OzGemm) + 64;
}

int oz_run_device(const GemmGen* d_g, int count, int max_m, int max_n, int max_k, int k_min, int S, void* ws,
                  size_t ws_bytes, long long* d_stat, cudaStream_t s) {
  if (count <= 0) return TLR_OK;
  const size_t sa = align128(oz_slices_elems(max_m, max_k, OZ_BM, S) * 2);
  const size_t sb = align128(oz_slices_elems(max_n, max_k, OZ_BN, S) * 2);
  const size_t xa = align128((size_t)round_up(max_m, OZ_BM) * 4);
  const size_t xb = align128((size_t)round_up(max_n, OZ_BN) * 4);
  const size_t per = sa + sb + xa + xb;
  const size_t per_all = per + 2 * sizeof(OzSrc) + sizeof(OzGemm);
  const int chunk = (int)std::min<size_t>(32767, ws_bytes > 512 ? (ws_bytes - 512) / per_all : 0);
  if (chunk < 1) TLR_RETURN_OOM();
  char* base = static_cast<char*>(ws);
  for (int q0 = 0; q0 < count; q0 += chunk) {
    const int cnt = std::min(chunk, count - q0);
    char* descs = reinterpret_cast<char*>(align128(reinterpret_cast<size_t>(base + (size_t)cnt * per)));
    OzGemm* gem = reinterpret_cast<OzGemm*>(descs + align128((size_t)2 * cnt * sizeof(OzSrc)));
    int rc;
    switch (S) {
      case 4: rc = launch_split_gen<4>(d_g + q0, cnt, k_min, base, sa, sb, xa, per, gem, std::max(max_m, max_n), max_k, s); break;
      case 5: rc = launch_split_gen<5>(d_g + q0, cnt, k_min, base, sa, sb, xa, per, gem, std::max(max_m, max_n), max_k, s); break;
      case 6: rc = launch_split_gen<6>(d_g + q0, cnt, k_min, base, sa, sb, xa, per, gem, std::max(max_m, max_n), max_k, s); break;
      default: rc = -1;
    }
    if (rc) return rc;
    rc = oz_gemm(gem, cnt, max_m, max_n, S, d_stat, s);
    if (rc) return rc;
  }
  return TLR_OK;
}

// Diagnostic entry point: one GEMM through the split and the tensor-core kernel, with
// its own temporary buffers (cudaMalloc, synchronising).
extern "C" int tlr_gemm_tc(int m, int n, int k, const double* A, int lda, int tA, const double* B, int ldb, int tB,
                           double* C, int ldc, double alpha, double beta, int slices, tlr_stream_t stream) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (!A && m > 0 && k > 0) return -4;
  if (!B && n > 0 && k > 0) return -7;
  if (!C && m > 0 && n > 0) return -10;
  if (slices < 4 || slices > OZ_SMAX) return -14;
  if (m == 0 || n == 0) return TLR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ea = oz_slices_elems(m, k, OZ_BM, slices), eb = oz_slices_elems(n, k, OZ_BN, slices);
  const int mp = round_up(m, OZ_BM), np = round_up(n, OZ_BN);
  uint16_t *sa = nullptr, *sb = nullptr;
  int *xa = nullptr, *xb = nullptr;
  OzSrc* dsrc = nullptr;
  OzGemm* dg = nullptr;
  long long* dst = nullptr;
  int rc = TLR_OK;
  if (cudaMalloc((void**)&sa, ea * 2) || cudaMalloc((void**)&sb, eb * 2) || cudaMalloc((void**)&xa, mp * 4) ||
      cudaMalloc((void**)&xb, np * 4) || cudaMalloc((void**)&dsrc, 2 * sizeof(OzSrc)) ||
      cudaMalloc((void**)&dg, sizeof(OzGemm)) || cudaMalloc((void**)&dst, 4 * sizeof(long long))) {
    cudaGetLastError();
    rc = TLR_ERR_OOM;
  }
  if (rc == TLR_OK) {
    // op(A) rows x k: element (r, c) at A[c * lda + r] (tA = 0) or A[r * lda + c];
    // op(B)^T rows x k (the n columns of op(B)): element (j, c) at B[j * ldb + c] (tB = 0) or B[c * ldb + j]
    OzSrc h[2];
    h[0] = {A, lda, tA ? 0 : 1, m, k, sa, xa, OZ_BM};
    h[1] = {B, ldb, tB ? 1 : 0, n, k, sb, xb, OZ_BN};
    OzGemm gg;
    gg.a = {sa, xa, m, round_up(std::max(k, 1), OZ_BK) / OZ_BK};
    gg.b = {sb, xb, n, round_up(std::max(k, 1), OZ_BK) / OZ_BK};
    gg.C = C; gg.ldc = ldc; gg.m = m; gg.n = n; gg.alpha = alpha; gg.beta = beta; gg.lower = 0;
    if (k == 0) { gg.a.nkb = 0; gg.b.nkb = 0; }
    if (cudaMemcpyAsync(dsrc, h, sizeof(h), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(dg, &gg, sizeof(gg), cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(dst, 0, 4 * sizeof(long long), s))
      rc = TLR_ERR_CUDA;
    if (rc == TLR_OK && k > 0) rc = oz_split(dsrc, 2, std::max(m, n), k, slices, s);
    if (rc == TLR_OK) rc = oz_gemm(dg, 1, m, n, slices, dst, s);
    long long hs[2] = {0, 0};
    if (rc == TLR_OK && (cudaMemcpyAsync(hs, dst, sizeof(hs), cudaMemcpyDeviceToHost, s) ||
                         cudaStreamSynchronize(s)))
      rc = TLR_ERR_CUDA;
    if (rc == TLR_OK && hs[0]) rc = (int)hs[0];
  }
  cudaStreamSynchronize(s);
  cudaFree(sa); cudaFree(sb); cudaFree(xa); cudaFree(xb); cudaFree(dsrc); cudaFree(dg); cudaFree(dst);
  return rc;
}
