// cf_common.cuh -- device data layout and warp-level helpers shared by the
// inside, outside and sampling kernels of the codon-constrained partition
// function (arXiv 2604.19718, Section "Dynamic programs over sequences and
// structures": every interval entry is a small rectangular block over the
// codon states at its two ends).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cf_nvtx.h"

namespace cf {

constexpr int NS = 6;        // maximum codon states of one residue
constexpr int BLK = NS * NS; // padded 6x6 block per table entry
constexpr int MAXLOOP = 30;  // maximum bulge / interior loop size
constexpr int NYY = 29;      // interior-loop partial sums, total loop size L = 2..30
constexpr int YRING = 8;     // diagonals of interior-loop adjoints kept in flight

// typed transition variants, index (type at p) * 2 + (type at p+1), U = 0, P = 1
constexpr int XUU = 0, XUP = 1, XPU = 2, XPP = 3;

// energy-factor vector offsets (Boltzmann factors e^{-E/RT})
constexpr int EN_STK = 0;    // [6][6] stack by (outer, inner) pair type
constexpr int EN_BU = 36;    // [31] bulge by loop size
constexpr int EN_IN = 67;    // [31] interior by loop size
constexpr int EN_TM = 98;    // [4][4] terminal mismatch
constexpr int EN_D5 = 114;   // [4][4] 5' dangle [paired][dangling]
constexpr int EN_D3 = 130;   // [4][4] 3' dangle [paired][dangling]
constexpr int EN_EA = 146;   // multiloop closing
constexpr int EN_EB = 147;   // multiloop unpaired base
constexpr int EN_EC = 148;   // multiloop branch
constexpr int EN_N = 149;

// Triangular, diagonal-major cell index: all cells of one anti-diagonal are
// contiguous, so each wavefront step writes one contiguous range.
__host__ __device__ __forceinline__ size_t cidx(int n, int x, int y) {
  size_t d = (size_t)(y - x);
  return d * (size_t)n - d * (d - 1) / 2 + (size_t)x;
}
__host__ __device__ __forceinline__ size_t ncells(int n) { return (size_t)n * (n + 1) / 2; }

// pair type of bases (x 5', y 3'): AU, CG, GC, UA, GU, UG -> 0..5, else -1
__host__ __device__ __forceinline__ int pair_type(int x, int y) {
  int k = x * 4 + y;
  // A=0 C=1 G=2 U=3
  switch (k) {
    case 0 * 4 + 3: return 0;
    case 1 * 4 + 2: return 1;
    case 2 * 4 + 1: return 2;
    case 3 * 4 + 0: return 3;
    case 2 * 4 + 3: return 4;
    case 3 * 4 + 2: return 5;
    default: return -1;
  }
}

template <typename T>
__device__ __forceinline__ T p2(int e) {
  return (T)ldexp(1.0, e);
}
template <>
__device__ __forceinline__ float p2<float>(int e) {
  return ldexpf(1.0f, e);
}

// Everything a wavefront kernel needs; device pointers.
template <typename T>
struct DP {
  int n, m;
  const int *Mp;    // [n] states per position
  const int *base;  // [n*6] base of state a at p
  const int *bnd;   // [n] 1 if T_p crosses a residue boundary
  const T *Tr;      // [n*36] transfer p -> p+1 (scaled)
  const T *X;       // [n*4*36] typed transitions
  const T *en;      // [EN_N] energy factors
  const T *eHL;     // [n+2] hairpin length factor e^{-H(L)/RT}
  const double *u0; // [6] weights of residue 0
  int *E;           // [n] per-diagonal exponents
  unsigned long long *dmax; // [n] bits of the largest mantissa per diagonal
  int *err;         // device error word
  // inside tables [ncell*36]
  T *CH, *QB, *XI, *HB, *QMpp, *QMpu, *G, *QM2pp, *QM2pu, *QM2up, *QM2uu;
  T *YY;            // stored: [ncell][29][36]; checkpointed: ring [2][n][29][36]
  int yyck;         // 1: the interior partial sums are checkpointed (see yy_in)
  T *YYck;          // checkpointed: every 64th diagonal (d % 64 == 63), [n/64 + 1][n][29][36]
  T *YYb;           // checkpointed: the outside pass's recomputed blocks, [2][64][n][29][36]
  T *Q5U, *Q5P, *Gx; // [n*36]
  double *Zm;       // scalar: Z relative to 2^{E[n-1]} and the transfer scaling
  // adjoint tables
  T *hCH, *hQB, *hGc, *hXI, *hHB, *hQMpp, *hQMpu, *hG, *hQM2pp, *hQM2pu, *hQM2up, *hQM2uu;
  T *hYY;           // ring [YRING][n][29*36]
  T *hQ5U, *hQ5P, *hGx; // [n*36]
  T *tgY;           // [ncell*36] sum_L hYY_L[x][y] YY_{L-1}[x+1][y]^T of cells with a boundary at x
  double *hT;       // [n*36]   d log Z / d T_p (boundary positions)
  double *hX;       // [n*4*36] d log Z / d X_p (boundary positions)
  float *P;         // [n*n] pair probabilities (device)
  // Batch of equal-length proteins: every array of protein b lies bstride
  // bytes after protein 0's (one slab per protein); 0 for a single protein.
  // A batched launch takes the protein from blockIdx.y (k_out_tg: z / 2).
  long long bstride;
};

template <typename P>
__host__ __device__ __forceinline__ P *bshift(P *ptr, long long off) {
  return ptr ? (P *)((char *)ptr + off) : ptr;
}
// Protein b's view of a batch: every pointer moved by b slabs.
template <typename T>
__device__ __forceinline__ void dp_shift(DP<T> &p, long long off) {
#define CF_SH(f) p.f = bshift(p.f, off)
  CF_SH(Mp); CF_SH(base); CF_SH(bnd); CF_SH(Tr); CF_SH(X); CF_SH(en); CF_SH(eHL); CF_SH(u0); CF_SH(E);
  CF_SH(dmax); CF_SH(err); CF_SH(CH); CF_SH(QB); CF_SH(XI); CF_SH(HB); CF_SH(QMpp); CF_SH(QMpu); CF_SH(G);
  CF_SH(QM2pp); CF_SH(QM2pu); CF_SH(QM2up); CF_SH(QM2uu); CF_SH(YY); CF_SH(YYck); CF_SH(YYb); CF_SH(Q5U);
  CF_SH(Q5P); CF_SH(Gx); CF_SH(Zm); CF_SH(hCH); CF_SH(hQB); CF_SH(hGc); CF_SH(hXI); CF_SH(hHB); CF_SH(hQMpp);
  CF_SH(hQMpu); CF_SH(hG); CF_SH(hQM2pp); CF_SH(hQM2pu); CF_SH(hQM2up); CF_SH(hQM2uu); CF_SH(hYY); CF_SH(hQ5U);
  CF_SH(hQ5P); CF_SH(hGx); CF_SH(tgY); CF_SH(hT); CF_SH(hX); CF_SH(P);
#undef CF_SH
}

// Where the 29 interior partial sums YY_L of cell (x, x + d) live.  Stored
// form: one table over all cells.  Checkpointed form (the outside pass
// recomputes them in blocks of 64 diagonals): during the inside pass a ring of
// two diagonals, except that every diagonal d with d % 64 == 63 goes to the
// checkpoint store, from which the outside pass restarts the recursion of the
// next block; yy_out gives the block buffers the outside pass reads.
constexpr int YYCK_BLOCK = 64;
template <typename T>
__host__ __device__ __forceinline__ T *yy_in(const DP<T> &p, int x, int d) {
  const size_t cell = (size_t)NYY * BLK;
  if (!p.yyck) return p.YY + cidx(p.n, x, x + d) * cell;
  if (d % YYCK_BLOCK == YYCK_BLOCK - 1) return p.YYck + ((size_t)(d / YYCK_BLOCK) * p.n + x) * cell;
  return p.YY + ((size_t)(d & 1) * p.n + x) * cell;
}
template <typename T>
__host__ __device__ __forceinline__ T *yy_out(const DP<T> &p, int x, int d) {
  const size_t cell = (size_t)NYY * BLK;
  if (!p.yyck) return p.YY + cidx(p.n, x, x + d) * cell;
  if (d % YYCK_BLOCK == YYCK_BLOCK - 1) return p.YYck + ((size_t)(d / YYCK_BLOCK) * p.n + x) * cell;
  return p.YYb + ((size_t)(((d / YYCK_BLOCK) & 1) * YYCK_BLOCK + d % YYCK_BLOCK) * p.n + x) * cell;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Reduce a per-lane accumulator block over the warp (entries a<Ma, b<Mb);
// afterwards every lane holds the totals.
template <typename T>
__device__ __forceinline__ void warp_reduce_block(T (&acc)[BLK], int Ma, int Mb) {
#pragma unroll
  for (int e = 0; e < BLK; e++)
    if ((e / NS) < Ma && (e % NS) < Mb) acc[e] = warp_sum(acc[e]);
}

template <typename T>
__device__ __forceinline__ void zero_block(T (&acc)[BLK]) {
#pragma unroll
  for (int e = 0; e < BLK; e++) acc[e] = (T)0;
}

// acc += f * op(A) op(B); TA/TB select transposed reads of the padded blocks.
// A is Ma x Ms (after op), B is Ms x Mb (after op).
template <bool TA, bool TB, typename T>
__device__ __forceinline__ void acc_mm(T (&acc)[BLK], const T *A, const T *B, int Ma, int Ms, int Mb,
                                       T f) {
#pragma unroll
  for (int a = 0; a < NS; a++) {
    if (a < Ma) {
#pragma unroll
      for (int s = 0; s < NS; s++) {
        if (s < Ms) {
          T av = (TA ? A[s * NS + a] : A[a * NS + s]) * f;
#pragma unroll
          for (int b = 0; b < NS; b++)
            if (b < Mb) acc[a * NS + b] += av * (TB ? B[b * NS + s] : B[s * NS + b]);
        }
      }
    }
  }
}

// acc_mm with both operand blocks first read whole into registers by 16-byte
// loads (blocks are 144/288-byte aligned and padded), so that every load of a
// split point is in flight before its first multiply.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

__device__ __forceinline__ void unpack16(float *r, float4 v) {
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
__device__ __forceinline__ void unpack16(double *r, double2 v) {
  r[0] = v.x;
  r[1] = v.y;
}

template <typename T>
__device__ __forceinline__ void load_block(T (&r)[BLK], const T *src) {
  using V = typename Vec16<T>::type;
  constexpr int W = 16 / sizeof(T);
  const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
  for (int i = 0; i < BLK / W; i++) unpack16(r + W * i, __ldg(s + i));
}

template <bool TA, bool TB, typename T>
__device__ __forceinline__ void acc_mm_v(T (&acc)[BLK], const T *A, const T *B, int Ma, int Ms, int Mb, T f) {
  T ra[BLK], rb[BLK];
  load_block(ra, A);
  load_block(rb, B);
#pragma unroll
  for (int a = 0; a < NS; a++) {
    if (a < Ma) {
#pragma unroll
      for (int s = 0; s < NS; s++) {
        if (s < Ms) {
          T av = (TA ? ra[s * NS + a] : ra[a * NS + s]) * f;
#pragma unroll
          for (int b = 0; b < NS; b++)
            if (b < Mb) acc[a * NS + b] += av * (TB ? rb[b * NS + s] : rb[s * NS + b]);
        }
      }
    }
  }
}

// One entry (a,b) of op(A) op(B) op(C) with inner sizes Mu, Mv.  Loops are
// unrolled to the padded size with predicates so that all loads of one
// contraction issue together instead of one dependent round trip per term.
template <bool TA, bool TB, bool TC, typename T>
__device__ __forceinline__ T e3(const T *A, const T *B, const T *C, int a, int b, int Mu, int Mv) {
  T cv[NS];
#pragma unroll
  for (int v = 0; v < NS; v++) cv[v] = (v < Mv) ? (TC ? C[b * NS + v] : C[v * NS + b]) : (T)0;
  T s = 0;
#pragma unroll
  for (int u = 0; u < NS; u++) {
    if (u < Mu) {
      T av = TA ? A[u * NS + a] : A[a * NS + u];
      T t = 0;
#pragma unroll
      for (int v = 0; v < NS; v++)
        if (v < Mv) t += (TB ? B[v * NS + u] : B[u * NS + v]) * cv[v];
      s += av * t;
    }
  }
  return s;
}

// One entry (a,b) of op(A) op(B).
template <bool TA, bool TB, typename T>
__device__ __forceinline__ T e2(const T *A, const T *B, int a, int b, int Mu) {
  T s = 0;
#pragma unroll
  for (int u = 0; u < NS; u++)
    if (u < Mu) s += (TA ? A[u * NS + a] : A[a * NS + u]) * (TB ? B[b * NS + u] : B[u * NS + b]);
  return s;
}

// Shared-memory versions (operands already on chip): loops unrolled over the
// padded size with the trip count as a predicate, so that the loads of a sum
// issue together.
template <bool TA, bool TB, typename T>
__device__ __forceinline__ T s2(const T *A, const T *B, int a, int b, int Mu) {
  T s = 0;
#pragma unroll
  for (int u = 0; u < NS; u++)
    if (u < Mu) s += (TA ? A[u * NS + a] : A[a * NS + u]) * (TB ? B[b * NS + u] : B[u * NS + b]);
  return s;
}
template <bool TA, bool TB, bool TC, typename T>
__device__ __forceinline__ T s3(const T *A, const T *B, const T *C, int a, int b, int Mu, int Mv) {
  T cv[NS];
#pragma unroll
  for (int v = 0; v < NS; v++) cv[v] = v < Mv ? (TC ? C[b * NS + v] : C[v * NS + b]) : (T)0;
  T s = 0;
#pragma unroll
  for (int u = 0; u < NS; u++) {
    if (u < Mu) {
      const T av = TA ? A[u * NS + a] : A[a * NS + u];
      T t = 0;
#pragma unroll
      for (int v = 0; v < NS; v++)
        if (v < Mv) t += (TB ? B[v * NS + u] : B[u * NS + v]) * cv[v];
      s += av * t;
    }
  }
  return s;
}

// Accessors of the per-cell context staged by the light kernels (sE, sMx,
// sMy, sBx, sBy): exponents of diagonals d-47..d+48 (E[d] itself is passed as
// Ed), codon-state counts of positions within 35 of x or y, bases of
// x-1..x+1 and y-1..y+1.  Other indices fall back to global memory.
#define EA(k) ((k) == d ? Ed : (((k) >= d - 47 && (k) <= d + 48) ? sE[(k) - (d - 47)] : __ldcg(p.E + (k))))
// EA for indices known to lie in d-47..d (no global fallback, so that no load
// of the exponent array is ever issued on the cell's critical path)
#define EAS(k) ((k) == d ? Ed : sE[(k) - (d - 47)])
#define MP(q) (((q) >= x - 35 && (q) <= x + 36) ? sMx[(q) - (x - 35)] : (((q) >= y - 35 && (q) <= y + 36) ? sMy[(q) - (y - 35)] : p.Mp[q]))
#define BASE(q, a) (((q) >= x - 1 && (q) <= x + 1) ? sBx[(q) - (x - 1)][a] : sBy[(q) - (y - 1)][a])

// ---- TMA bulk copies (global -> shared) completing on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// Programmatic dependent launch along a chain of wavefront kernels: a kernel
// launched through a programmatic graph edge may start while its predecessor
// is still running; griddep_wait blocks the calling thread until the
// predecessor grid has completed and its writes are visible (a no-op for a
// kernel launched without such an edge), and griddep_launch_dependents lets
// the successor start once every CTA of this grid has called it or exited.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// raise the transaction count of the current phase by bytes (no arrival)
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// bytes: multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Polls of the first wait of mbar_wait before it gives up (about a second at
// the default).  A test lowers it (cf_debug_set_wait_polls) to make every
// wait give up at once; the drain wait after a timeout keeps its full length,
// so the copies in flight still land before the CTA exits.
// (The test knobs live in constant memory: a kernel reads them from the
// SM's constant cache, not with a round trip to L2 on its critical path.)
static __constant__ unsigned long long g_cf_wait_polls = 1ull << 22;

// Largest departure (log2) of the per-diagonal exponents from the far-band
// chord for which a band is still summed in tiles (48 by default).  A test
// lowers it (cf_debug_set_far_dev_max) to send every band through the
// term-by-term path.
static __constant__ int g_cf_far_dev_max = 48;

// Bits of the device error word besides ERR_STAGE_TIMEOUT: the binary32
// inside pass found the dynamic range of its tables exceeded, or an output of
// the outside pass was not finite.
constexpr int ERR_RANGE_IN = 1 << 6, ERR_OUT_NONFINITE = 1 << 8;

// Bounded wait for a phase of the mbarrier.  On timeout bit 8 of the error
// word is set and false is returned; the copies that were in flight are then
// waited for once more, again bounded.
constexpr int ERR_STAGE_TIMEOUT = 8;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *err) {
  const unsigned long long polls = g_cf_wait_polls;
  for (unsigned long long it = 0; it < polls; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(128);
  }
  atomicOr(err, ERR_STAGE_TIMEOUT);
  for (unsigned long long it = 0; it < (1ull << 22); it++)
    if (mbar_try_wait(bar, parity)) break;
  return false;
}

// Bounded wait for a phase that other threads of the CTA complete by their
// arrivals (no copies to drain): on timeout the error bit is set and false
// is returned at once.
__device__ __forceinline__ bool mbar_wait_peer(unsigned long long *bar, unsigned parity, int *err) {
  const unsigned long long polls = g_cf_wait_polls;
  for (unsigned long long it = 0; it < polls; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(128);
  }
  atomicOr(err, ERR_STAGE_TIMEOUT);
  return false;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  if (v > 0) atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace cf
