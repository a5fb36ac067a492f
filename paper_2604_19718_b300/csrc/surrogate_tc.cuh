// surrogate_tc.cuh -- the surrogate's forward pass on the 5th-generation
// tensor cores (tcgen05 MMA, TMEM accumulators, TMA staging), used for
// prediction (screening many candidate windows).
//
// Layout: the batch's windows are concatenated as rows (one row per base, 64
// channels), each window framed by two zero rows on each side:
//   window w occupies rows R_w .. R_w + n_w + 3, R_w = (off[w] - off[0]) + 4w,
//   its bases on rows R_w + 2 .. R_w + n_w + 1.
// The zero rows are the convolution's zero padding, so one tile of 128
// consecutive rows can straddle windows: a 5-tap convolution of the row
// sequence is exactly the per-window convolution on every base row.
//
// A layer (64 -> 64 channels, 5 taps) is the GEMM
//   D[r][co] = sum_{k=0..4} sum_ci X[r + k - 2][ci] W[co][ci][k]
// with M = 128 rows per tile, N = 64 output channels and K = 5 x 64.  The
// input rows r0 - 2 .. r0 + 133 of a tile arrive by one TMA load (128-byte
// swizzle); tap k's A operand is the same tile shifted by k rows.
// Activations are carried as two BF16 parts, x = hi + lo (|x - hi - lo| <=
// 2^-18 |x|), and both parts are multiplied with the BF16 weights, so the
// layer matches FP32 activations to ~1e-5 relative; accumulation is FP32 in
// TMEM.  Warp roles (192 threads, one CTA per SM, persistent over tiles):
//   warp 0  TMA producer: weights once, then the tiles into a 3-stage ring;
//   warp 1  MMA issuer (one thread): 40 MMAs of 128x64x16 per tile into one
//           of two TMEM accumulators, tcgen05.commit to release the stage and
//           to hand the accumulator to the epilogue;
//   warps 2-5  epilogue: one TMEM lane (row) per thread, bias + ReLU, zero on
//           frame rows, write the next layer's hi/lo rows (or, after the last
//           layer, the row's head term wh . h).
// Every wait is bounded; on a timeout the kernel records an error, waits
// (bounded) for its MMAs and copies in flight, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "cf_common.cuh"

namespace sg {

constexpr int TC_M = 128;                        // rows per tile
constexpr int TC_HALO = TC_M + 8;                // staged input rows (2 before, 6 after)
constexpr int TC_ROWB = 64 * 2;                  // bytes per row: 64 BF16 channels
constexpr int TC_TILE_BYTES = TC_HALO * TC_ROWB; // 17408 = 17 KiB
constexpr int TC_W_TAP = 64 * TC_ROWB;           // 8 KiB per tap
constexpr int TC_W_BYTES = 5 * TC_W_TAP;
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 192;
constexpr int TC_TMEM_COLS = 128;                // two 64-column FP32 accumulators
constexpr size_t TC_SMEM = 1024 + TC_W_BYTES + (size_t)TC_STAGES * 2 * TC_TILE_BYTES;
static_assert(TC_TILE_BYTES % 1024 == 0 && TC_W_TAP % 1024 == 0, "128-byte swizzle atoms stay 1024-aligned");

struct TcArgs {
  int nrows;             // rows of the batch (frames included)
  const int *rowwin;     // [nrows] window of a base row, -1 on frame rows
  const float *bias;     // [64]
  const float *wh;       // [64] head weights (last layer)
  __nv_bfloat16 *out_hi, *out_lo;  // [nrows][64] next layer's input (not last)
  float *s_out;          // [nrows] head term per row (last layer)
  int wrow0;             // first weight row of this layer in the weight tensor map
  int last;
  int *err;              // bit 0: a bounded wait gave up
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *tm, int x, int y, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          su32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// bounded parity wait (about a second); false on timeout
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); it++) {
    if (cf::mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// UMMA shared-memory descriptor, K-major operand with 128-byte swizzle:
// start address, leading offset 16 B (unused for swizzled K-major), stride
// 1024 B between 8-row groups, descriptor version 1, base offset 0, swizzle
// mode 2.  The swizzle is a function of the absolute shared-memory address
// (the tiles are 1024-byte aligned), so a start address moved by whole
// 128-byte rows (the tap shift) or by 32 bytes (the next 16 channels) still
// reads the layout TMA wrote -- measured: a base offset of (start >> 7) & 7
// instead gives wrong products.
__device__ __forceinline__ uint64_t tc_desc(const void *p) {
  const uint32_t a = su32(p);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 64
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
              const __grid_constant__ CUtensorMap tm_w, TcArgs a) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sW = base;
  unsigned char *sA = base + TC_W_BYTES;  // [stage][hi, lo][TC_TILE_BYTES]
  __shared__ __align__(8) unsigned long long bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_tf[2], bar_te[2], bar_w,
      bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (a.nrows + TC_M - 1) / TC_M;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; s++) {
      cf::mbar_init(&bar_full[s], 1);
      cf::mbar_init(&bar_empty[s], 1);
    }
    for (int s = 0; s < 2; s++) {
      cf::mbar_init(&bar_tf[s], 1);
      cf::mbar_init(&bar_te[s], 4 * 32);
    }
    cf::mbar_init(&bar_w, 1);
    cf::mbar_init(&bar_drain, 1);
    abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicOr(a.err, 1);
  };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- producer
      cf::mbar_arrive_expect(&bar_w, TC_W_BYTES);
      for (int k = 0; k < 5; k++) tma_2d(sW + k * TC_W_TAP, &tm_w, 0, a.wrow0 + 64 * k, &bar_w);
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
        const int s = it % TC_STAGES;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
        if (!tc_wait(&bar_empty[s], ph ^ 1u) || *(volatile int *)&abort_flag) {
          give_up();
          break;
        }
        cf::mbar_arrive_expect(&bar_full[s], 2 * TC_TILE_BYTES);
        unsigned char *dst = sA + (size_t)s * 2 * TC_TILE_BYTES;
        tma_2d(dst, &tm_hi, 0, tile * TC_M - 2, &bar_full[s]);
        tma_2d(dst + TC_TILE_BYTES, &tm_lo, 0, tile * TC_M - 2, &bar_full[s]);
      }
      // every copy issued has landed before the CTA may exit
      for (int j = max(0, it - TC_STAGES); j < it; j++) tc_wait(&bar_full[j % TC_STAGES], (unsigned)(j / TC_STAGES) & 1u);
      tc_wait(&bar_w, 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      bool ok = tc_wait(&bar_w, 0);
      if (!ok) give_up();
      int it = 0;
      for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, it++) {
        const int s = it % TC_STAGES, acc = it & 1;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u, aph = (unsigned)(it >> 1) & 1u;
        if (!tc_wait(&bar_te[acc], aph ^ 1u) || !tc_wait(&bar_full[s], ph) || *(volatile int *)&abort_flag) {
          give_up();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * 64);
        const unsigned char *tile_a = sA + (size_t)s * 2 * TC_TILE_BYTES;
        uint32_t accum = 0;
#pragma unroll 1
        for (int part = 0; part < 2; part++)
#pragma unroll 1
          for (int k = 0; k < 5; k++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
              const unsigned char *pa = tile_a + part * TC_TILE_BYTES + k * TC_ROWB + j * 32;
              const uint64_t ad = tc_desc(pa);
              const uint64_t bd = tc_desc(sW + k * TC_W_TAP + j * 32);
              tc_mma(d, ad, bd, accum);
              accum = 1;
            }
        tc_commit(&bar_empty[s]);  // the stage is free once these MMAs have read it
        tc_commit(&bar_tf[acc]);   // the accumulator is ready for the epilogue
      }
      tc_commit(&bar_drain);  // all MMAs issued by this thread have completed
      tc_wait(&bar_drain, 0);
    }
  } else {  // ---------------- epilogue: warps 2..5, one TMEM lane (tile row) per thread
    const int q = warp & 3;  // the TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
      const int acc = it & 1;
      const unsigned aph = (unsigned)(it >> 1) & 1u;
      if (!tc_wait(&bar_tf[acc], aph) || *(volatile int *)&abort_flag) {
        give_up();
        break;
      }
      tc_fence_after();
      float v[64];
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 64);
#pragma unroll
      for (int c = 0; c < 4; c++) tc_ld16(taddr + 16 * c, *reinterpret_cast<float(*)[16]>(v + 16 * c));
      tc_wait_ld();
      tc_fence_before();
      cf::mbar_arrive(&bar_te[acc]);  // the accumulator may be overwritten
      const int row = tile * TC_M + r;
      if (row < a.nrows) {
        const bool base_row = a.rowwin[row] >= 0;
        if (a.last) {
          float sacc = 0.f;
#pragma unroll
          for (int c = 0; c < 64; c++) sacc = fmaf(a.wh[c], fmaxf(v[c] + a.bias[c], 0.f), sacc);
          a.s_out[row] = base_row ? sacc : 0.f;
        } else {
          uint4 *ph = reinterpret_cast<uint4 *>(a.out_hi + (size_t)row * 64);
          uint4 *pl = reinterpret_cast<uint4 *>(a.out_lo + (size_t)row * 64);
#pragma unroll
          for (int c8 = 0; c8 < 8; c8++) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
              float h0 = base_row ? fmaxf(v[c8 * 8 + 2 * u] + a.bias[c8 * 8 + 2 * u], 0.f) : 0.f;
              float h1 = base_row ? fmaxf(v[c8 * 8 + 2 * u + 1] + a.bias[c8 * 8 + 2 * u + 1], 0.f) : 0.f;
              const __nv_bfloat16 b0 = __float2bfloat16_rn(h0), b1 = __float2bfloat16_rn(h1);
              const __nv_bfloat16 l0 = __float2bfloat16_rn(h0 - __bfloat162float(b0));
              const __nv_bfloat16 l1 = __float2bfloat16_rn(h1 - __bfloat162float(b1));
              hw[u] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
              lw[u] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            ph[c8] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            pl[c8] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// Row frame of the batch: rowwin[row] = window of a base row, -1 on frame rows.
__global__ void k_tc_rows(const int64_t *off, int nwin, int nrows, int *rowwin) {
  const int w = blockIdx.x;
  if (w >= nwin) return;
  const int64_t o0 = off[0];
  const int n = (int)(off[w + 1] - off[w]);
  const int R = (int)(off[w] - o0) + 4 * w;
  for (int i = threadIdx.x; i < n + 4; i += blockDim.x) {
    const int row = R + i;
    if (row < nrows) rowwin[row] = (i >= 2 && i < n + 2) ? w : -1;
  }
}

// Layer 1 (4 one-hot channels -> 64): h[row][co] = relu(b[co] + sum_k W[co][base(row+k-2)][k]),
// written as BF16 hi/lo parts; frame rows are zero.  One thread per (row, channel).
__global__ void k_tc_layer1(const int64_t *off, const uint8_t *bases, const int *rowwin, int nrows,
                            const __nv_bfloat16 *Wf, const float *bias, __nv_bfloat16 *out_hi, __nv_bfloat16 *out_lo) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(idx / 64), co = (int)(idx % 64);
  if (row >= nrows) return;
  float h = 0.f;
  if (rowwin[row] >= 0) {
    const int64_t o0 = off[0];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 5; k++) {
      const int rr = row + k - 2;
      const int w = (rr >= 0 && rr < nrows) ? rowwin[rr] : -1;
      if (w < 0) continue;
      const int R = (int)(off[w] - o0) + 4 * w;
      const int b = bases[off[w] + (rr - R - 2)];
      acc = fmaf(__bfloat162float(Wf[(b * 5 + k) * 64 + co]), 1.f, acc);
    }
    h = fmaxf(acc + bias[co], 0.f);
  }
  const __nv_bfloat16 hi = __float2bfloat16_rn(h);
  out_hi[(size_t)row * 64 + co] = hi;
  out_lo[(size_t)row * 64 + co] = __float2bfloat16_rn(h - __bfloat162float(hi));
}

// Head: pred[w] = sum over the window's base rows of wh . h4 (in row order,
// one warp per window) + n bh.
__global__ void k_tc_head(const int64_t *off, int nwin, const float *s_rows, const float *P, float *pred) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= nwin) return;
  const int64_t o0 = off[0];
  const int n = (int)(off[w + 1] - off[w]);
  const int R = (int)(off[w] - o0) + 4 * w;
  float s = 0.f;
  for (int i = lane; i < n; i += 32) s += s_rows[R + 2 + i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) pred[w] = n > 0 ? s + (float)n * P[OBH] : 0.f;
}

// Weights of layers 2..4 for the tensor cores: Wtc[l-1][k][co][ci] (BF16,
// ci contiguous: the K-major B operand of tap k), rounded as the FFMA path's.
__global__ void k_prep_tc(const float *P, __nv_bfloat16 *Wtc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * 5 * 64 * 64) return;
  const int ci = i % 64, co = (i / 64) % 64, k = (i / 4096) % 5, l = 1 + i / 20480;
  Wtc[i] = __float2bfloat16_rn(P[OW(l) + (co * 64 + ci) * K + k]);
}

}  // namespace sg
