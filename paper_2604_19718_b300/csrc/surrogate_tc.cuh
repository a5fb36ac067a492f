// surrogate_tc.cuh -- the surrogate's forward pass on the 5th-generation
// tensor cores (tcgen05 MMA, TMEM accumulator, TMA for the weights), used for
// prediction (screening many candidate windows).
//
// Layout: the batch's windows are concatenated as rows (one row per base, 64
// channels), each window framed by two zero rows on each side:
//   window w occupies rows R_w .. R_w + n_w + 3, R_w = (off[w] - off[0]) + 4w,
//   its bases on rows R_w + 2 .. R_w + n_w + 1.
// The zero rows are the convolution's zero padding, so a tile of consecutive
// rows can straddle windows: a 5-tap convolution of the row sequence is
// exactly the per-window convolution on every base row.
//
// One persistent kernel runs all four layers and the head term of a tile of
// TC_OUT = 116 output rows without leaving the SM: layer 1 (one-hot bases,
// 4 -> 64 channels) is evaluated directly into shared memory for the tile's
// 132 input rows (6 rows of halo on each side, recomputed by the neighbouring
// tile); layers 2-4 (64 -> 64 channels, 5 taps) are the GEMMs
//   D[r][co] = sum_{k=0..4} sum_ci X[r + k - 2][ci] W[co][ci][k]
// with M = 128 rows, N = 64 and K = 5 x 64, whose A operand (the previous
// layer's rows, shifted by k rows for tap k) is read from shared memory in
// the 128-byte-swizzled K-major layout the epilogue writes; the last layer's
// epilogue reduces each row to its head term wh . h4.  Only the bases, the
// row frame and the head terms touch global memory.
// Activations are carried as two BF16 parts, x = hi + lo (|x - hi - lo| <=
// 2^-18 |x|), and both parts are multiplied with the BF16 weights, so a layer
// matches FP32 activations to ~1e-5 relative; accumulation is FP32 in TMEM.
// Warp roles (576 threads, one CTA per SM):
//   warp 0   TMA: the three layers' weights once (120 KiB, resident);
//   warp 1   MMA issuer (one thread): 40 MMAs of 128x64x16 per layer into the
//            TMEM accumulator, tcgen05.commit to hand it to the epilogue;
//   warps 2-17 epilogue: layer 1 (one warp per row); then per layer one TMEM lane (row) and 16
//            of the 64 columns per thread: bias + ReLU, zero on frame rows,
//            the next layer's hi/lo rows into shared memory; head terms
//            (all 64 columns of a row, in column order, by the first group).
// Every wait is bounded; on a timeout the kernel records an error, waits
// (bounded) for its MMAs and copies in flight, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "cf_common.cuh"

namespace sg {

constexpr int TC_M = 128;                        // rows per MMA (TMEM lanes)
constexpr int TC_OUT = TC_M - 12;                // output rows per tile (6 rows of halo each side)
constexpr int TC_IN = TC_M + 4;                  // layer-1 rows a tile needs (taps reach 4 rows on)
constexpr int TC_BUF_ROWS = TC_M + 8;            // rows per activation buffer (1024-byte multiple)
constexpr int TC_ROWB = 64 * 2;                  // bytes per row: 64 BF16 channels
constexpr int TC_BUF_BYTES = TC_BUF_ROWS * TC_ROWB;  // 17408 = 17 KiB per part
constexpr int TC_W_TAP = 64 * TC_ROWB;           // 8 KiB per tap
constexpr int TC_W_BYTES = 5 * TC_W_TAP;         // one layer
constexpr int TC_THREADS = 576;
constexpr int TC_EPI = 512;                      // epilogue threads (warps 2-17)
constexpr int TC_CG = 16;                        // columns per epilogue thread (4 groups of warps)
constexpr int TC_TMEM_COLS = 128;                // two 64-column FP32 accumulators
constexpr size_t TC_SMEM = 1024 + 3 * (size_t)TC_W_BYTES + 6 * (size_t)TC_BUF_BYTES;
static_assert(TC_BUF_BYTES % 1024 == 0 && TC_W_TAP % 1024 == 0, "128-byte swizzle atoms stay 1024-aligned");
static_assert(TC_SMEM + 2048 <= 227 * 1024, "shared memory budget (dynamic + static)");

struct TcArgs {
  int nrows;              // rows of the batch (frames included)
  const int8_t *rowbase;  // [nrows] base (0..3) of a base row, -1 on frame rows
  const __nv_bfloat16 *W1;  // layer 1, [base][k][co]
  const float *P;         // parameters: biases of layers 1-4 and the head weights
  float *s_out;           // [nrows] head term per row
  int *err;               // bit 0: a bounded wait gave up
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

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled buffer (the
// layout TMA writes with SWIZZLE_128B and the UMMA descriptor reads)
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * TC_ROWB + ((c ^ (r & 7)) << 4)); }

// 8 activations -> their BF16 hi and lo parts, as two 16-byte chunks
__device__ __forceinline__ void split8(const float *h, uint4 &hi, uint4 &lo) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(h[2 * u]), b1 = __float2bfloat16_rn(h[2 * u + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(h[2 * u] - __bfloat162float(b0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(h[2 * u + 1] - __bfloat162float(b1));
    hw[u] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
    lw[u] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_surr_tc(const __grid_constant__ CUtensorMap tm_w, TcArgs a) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sW = base;  // [layer 2..4][tap][co][ci]
  // activation buffers ([hi, lo] parts of TC_BUF_ROWS rows): X0 / X1 take a
  // tile's layer-1 rows and later its layer-3 rows (alternating by tile), J
  // its layer-2 rows
  unsigned char *X[2] = {base + 3 * TC_W_BYTES, base + 3 * TC_W_BYTES + 2 * TC_BUF_BYTES};
  unsigned char *J = base + 3 * TC_W_BYTES + 4 * TC_BUF_BYTES;
  // bar_l1: a tile's layer-1 rows are in place (all epilogue threads);
  // bar_mid: an epilogue's rows for the next MMA are in place (layer 2 -> J,
  // layer 3 -> X); bar_a1 / bar_a0: the accumulator of layer 2 (columns
  // 64-127) / of layers 3 and 4 (columns 0-63) is ready (tcgen05.commit)
  __shared__ __align__(8) unsigned long long bar_l1, bar_mid, bar_a1, bar_a0, bar_w, bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ __align__(16) float sB[4][64], sWh[64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (a.nrows + TC_OUT - 1) / TC_OUT;
  if (threadIdx.x == 0) {
    cf::mbar_init(&bar_l1, TC_EPI);
    cf::mbar_init(&bar_mid, TC_EPI);
    cf::mbar_init(&bar_a1, 1);
    cf::mbar_init(&bar_a0, 1);
    cf::mbar_init(&bar_w, 1);
    cf::mbar_init(&bar_drain, 1);
    abort_flag = 0;
  }
  for (int i = threadIdx.x; i < 4 * 64; i += TC_THREADS) sB[i / 64][i % 64] = a.P[OB(i / 64) + i % 64];
  if (threadIdx.x < 64) sWh[threadIdx.x] = a.P[OWH + threadIdx.x];
  // rows past the ones a layer writes are read only for discarded outputs; zero them once
  constexpr int ZQ = (TC_BUF_ROWS - TC_M) * TC_ROWB / 16;  // 16-byte words per part
  for (int i = threadIdx.x; i < 6 * ZQ; i += TC_THREADS) {
    const int part = i / ZQ, q = i % ZQ;
    unsigned char *b = part < 2 ? X[0] : (part < 4 ? X[1] : J);
    reinterpret_cast<uint4 *>(b + (part & 1) * TC_BUF_BYTES + TC_M * TC_ROWB)[q] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  cf::fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicOr(a.err, 1);
  };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- weights, once
      cf::mbar_arrive_expect(&bar_w, 3 * TC_W_BYTES);
      for (int q = 0; q < 15; q++) tma_2d(sW + q * TC_W_TAP, &tm_w, 0, 64 * q, &bar_w);
      tc_wait(&bar_w, 0);  // the copies have landed before the CTA may exit
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      bool ok = tc_wait(&bar_w, 0);
      if (!ok) give_up();
      unsigned it = 0, kmid = 0;
      // 40 MMAs of one layer: A = the input rows shifted by tap k, both parts
      auto layer = [&](const unsigned char *src, int l, uint32_t d) {
        const unsigned char *w = sW + (size_t)l * TC_W_BYTES;
        uint32_t accum = 0;
#pragma unroll 1
        for (int part = 0; part < 2; part++)
#pragma unroll 1
          for (int k = 0; k < 5; k++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
              tc_mma(d, tc_desc(src + part * TC_BUF_BYTES + k * TC_ROWB + j * 32), tc_desc(w + k * TC_W_TAP + j * 32),
                     accum);
              accum = 1;
            }
      };
      for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, it++) {
        const unsigned char *x = X[it & 1];
        if (!tc_wait(&bar_l1, it & 1u) || *(volatile int *)&abort_flag) break;
        tc_fence_after();
        layer(x, 0, tmem + 64);  // layer 2 -> columns 64-127
        tc_commit(&bar_a1);
        if (!tc_wait(&bar_mid, kmid++ & 1u) || *(volatile int *)&abort_flag) break;
        tc_fence_after();
        layer(J, 1, tmem);  // layer 3 -> columns 0-63
        tc_commit(&bar_a0);
        if (!tc_wait(&bar_mid, kmid++ & 1u) || *(volatile int *)&abort_flag) break;
        tc_fence_after();
        layer(x, 2, tmem);  // layer 4 -> columns 0-63
        tc_commit(&bar_a0);
      }
      if (ok && *(volatile int *)&abort_flag == 0 && (int)(blockIdx.x + it * gridDim.x) < ntiles) give_up();
      tc_commit(&bar_drain);  // all MMAs issued by this thread have completed
      tc_wait(&bar_drain, 0);
    }
  } else {  // ---------------- epilogue: warps 2..17
    const int q = warp & 3, grp = (warp - 2) >> 2;  // TMEM lane quarter this warp may access; column group
    const int r = q * 32 + lane;                    // the tile row (TMEM lane) of this thread
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    // Layer 1 runs one warp per row (rows ew, ew + 16, ...; TC_L1R at most),
    // lane l on channels 2l, 2l + 1: all lanes read the same weight row of a
    // (base, tap), a broadcast-friendly read through the read-only cache.
    // The row frame a thread reads in a tile -- the five rows around each of
    // its warp's layer-1 rows (two per lane, shuffled to the warp) and its
    // output row of layers 2-4 -- is loaded one tile ahead.
    const int ew = warp - 2;
    constexpr int TC_L1R = (TC_IN + 15) / 16;  // 9 rows per warp at most
    static_assert(TC_L1R * 5 <= 64, "two frame values per lane");
    auto rb = [&](int g) -> int { return (g >= 0 && g < a.nrows) ? (int)__ldg(a.rowbase + g) : -1; };
    auto load_flags = [&](int tile, int (&L)[2], int (&E)[3]) {
      const int g0 = tile * TC_OUT - 6;
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int v = lane + 32 * u, j = v / 5, k = v % 5, i = ew + 16 * j;
        L[u] = (j < TC_L1R && i < TC_IN) ? rb(g0 + i + k - 2) : -1;
      }
#pragma unroll
      for (int l = 0; l < 3; l++) E[l] = rb(g0 + 2 * (l + 1) + r);
    };
    const float2 bias1 = *reinterpret_cast<const float2 *>(&sB[0][2 * lane]);
    const __nv_bfloat162 *W1 = reinterpret_cast<const __nv_bfloat162 *>(a.W1);
    // layer 1 of a tile into x (rows 0 .. TC_IN - 1), then its arrival
    auto layer1 = [&](unsigned char *x, const int (&fl)[2]) {
#pragma unroll
      for (int j = 0; j < TC_L1R; j++) {
        const int i = ew + 16 * j;
        int b5[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
          const int v = 5 * j + k;
          b5[k] = __shfl_sync(0xffffffffu, v < 32 ? fl[0] : fl[1], v & 31);
        }
        if (i >= TC_IN) break;
        float h0 = 0.f, h1 = 0.f;
        if (b5[2] >= 0) {
#pragma unroll
          for (int k = 0; k < 5; k++) {
            if (b5[k] < 0) continue;
            const float2 w = __bfloat1622float2(__ldg(W1 + (b5[k] * 5 + k) * 32 + lane));
            h0 = fmaf(w.x, 1.f, h0);
            h1 = fmaf(w.y, 1.f, h1);
          }
          h0 = fmaxf(h0 + bias1.x, 0.f);
          h1 = fmaxf(h1 + bias1.y, 0.f);
        }
        const __nv_bfloat16 p0 = __float2bfloat16_rn(h0), p1 = __float2bfloat16_rn(h1);
        const __nv_bfloat16 q0 = __float2bfloat16_rn(h0 - __bfloat162float(p0));
        const __nv_bfloat16 q1 = __float2bfloat16_rn(h1 - __bfloat162float(p1));
        const uint32_t off = sw128(i, lane >> 2) + 4 * (lane & 3);
        *reinterpret_cast<uint32_t *>(x + off) =
            (uint32_t)__bfloat16_as_ushort(p0) | ((uint32_t)__bfloat16_as_ushort(p1) << 16);
        *reinterpret_cast<uint32_t *>(x + TC_BUF_BYTES + off) =
            (uint32_t)__bfloat16_as_ushort(q0) | ((uint32_t)__bfloat16_as_ushort(q1) << 16);
      }
      cf::fence_proxy_async();  // generic-proxy writes -> visible to the tensor core
      cf::mbar_arrive(&bar_l1);
    };
    // epilogue of a hidden layer: bias + ReLU of this thread's 16 columns, zero
    // on frame rows, the row's hi/lo parts into dst, then the arrival
    auto hidden = [&](uint32_t col, const float *bias, bool br, unsigned char *dst) {
      float v[TC_CG];
      tc_ld16(tq + col + TC_CG * grp, v);
      tc_wait_ld();
      tc_fence_before();
#pragma unroll
      for (int c = 0; c < TC_CG; c++) v[c] = br ? fmaxf(v[c] + bias[TC_CG * grp + c], 0.f) : 0.f;
#pragma unroll
      for (int c2 = 0; c2 < TC_CG / 8; c2++) {
        uint4 hi, lo;
        split8(v + 8 * c2, hi, lo);
        *reinterpret_cast<uint4 *>(dst + sw128(r, (TC_CG / 8) * grp + c2)) = hi;
        *reinterpret_cast<uint4 *>(dst + TC_BUF_BYTES + sw128(r, (TC_CG / 8) * grp + c2)) = lo;
      }
      cf::fence_proxy_async();
      cf::mbar_arrive(&bar_mid);
    };
    unsigned it = 0, ka1 = 0, ka0 = 0;
    int fl[2], fe[3], nfl[2], nfe[3];
    if ((int)blockIdx.x < ntiles) {
      load_flags(blockIdx.x, fl, fe);
      layer1(X[0], fl);
    }
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
      const int g0 = tile * TC_OUT - 6;  // global row of buffer row 0 (layer 1)
      const bool more = tile + (int)gridDim.x < ntiles;
      if (more) load_flags(tile + gridDim.x, nfl, nfe);
      // layer 2: accumulator columns 64-127 -> J
      if (!tc_wait(&bar_a1, ka1++ & 1u) || *(volatile int *)&abort_flag) {
        give_up();
        break;
      }
      tc_fence_after();
      hidden(64, sB[1], fe[0] >= 0, J);
      // the next tile's layer 1 while the tensor core runs layer 3
      if (more) layer1(X[(it + 1) & 1], nfl);
      // layer 3: columns 0-63 -> this tile's X (its layer-1 rows are consumed)
      if (!tc_wait(&bar_a0, ka0++ & 1u) || *(volatile int *)&abort_flag) {
        give_up();
        break;
      }
      tc_fence_after();
      hidden(0, sB[2], fe[1] >= 0, X[it & 1]);
      // layer 4: head term of output row r (all 64 columns, in column order)
      if (!tc_wait(&bar_a0, ka0++ & 1u) || *(volatile int *)&abort_flag) {
        give_up();
        break;
      }
      tc_fence_after();
      if (grp == 0) {
        const int g = g0 + 6 + r;
        float sacc = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float v[16];
          tc_ld16(tq + c0, v);
          tc_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; c++) sacc = fmaf(sWh[c0 + c], fmaxf(v[c] + sB[3][c0 + c], 0.f), sacc);
        }
        tc_fence_before();
        if (r < TC_OUT && g < a.nrows) a.s_out[g] = fe[2] >= 0 ? sacc : 0.f;
      }
      fl[0] = nfl[0];
      fl[1] = nfl[1];
#pragma unroll
      for (int l = 0; l < 3; l++) fe[l] = nfe[l];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// Row frame of the batch: rowbase[row] = base of a base row, -1 on frame rows.
__global__ void k_tc_rows(const int64_t *off, const uint8_t *bases, int nwin, int nrows, int8_t *rowbase) {
  const int w = blockIdx.x;
  if (w >= nwin) return;
  const int64_t o0 = off[0];
  const int n = (int)(off[w + 1] - off[w]);
  const int R = (int)(off[w] - o0) + 4 * w;
  for (int i = threadIdx.x; i < n + 4; i += blockDim.x) {
    const int row = R + i;
    if (row < nrows) rowbase[row] = (i >= 2 && i < n + 2) ? (int8_t)bases[off[w] + i - 2] : (int8_t)-1;
  }
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
