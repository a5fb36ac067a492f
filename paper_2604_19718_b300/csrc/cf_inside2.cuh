// cf_inside2.cuh -- inside pass as a CUDA graph over the anti-diagonals d
// (built in codonfold.cu).  Per diagonal d:
//
//   k_in_light<T>(d)    every term that reads diagonals d-1..d-3, one 256-thread
//                       CTA per cell: the ~240 input blocks arrive in shared
//                       memory by TMA bulk copies (sources from a per-diagonal
//                       table), then two phases of row products compute the
//                       chain, XI, the 29 interior partial sums, bulges,
//                       hairpin, QB, the multiloop tables and the exterior
//                       prefix; results go out with 16-byte stores.
//   k_in_bif_grp<T>(d)  the multiloop/exterior bifurcation sums of diagonal d,
//   (binary32)          sum_k G[x][k] QB[k][y] and sum_k Gx[k] QB[k][d], over
//                       the split points not in a far band (every split point
//                       of a short protein or a batch), four cells per CTA;
//                       its inputs lie on diagonals <= d-4, so it runs while
//                       diagonals d-3..d-1 are being filled; sums are relative
//                       to 2^{E[d-4]}.
//   k_in_bif<T>(d)      the same for binary64 proteins over 48 nt, one CTA per
//                       cell.
// Per band of FARD diagonals (binary32): k_in_far sums the far split points
// of the whole band as tiled products, after the light kernel of d0 - 17.
//
// Tables, exponents and recursions are those of cf_inside.cuh.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"

namespace cf {

constexpr int KCH = 32;  // split points per bifurcation chunk
constexpr int BIFRING = 4;

__host__ __device__ __forceinline__ int nchunk_bif(int d) { return d >= 9 ? (d - 8 + KCH - 1) / KCH : 0; }
// exterior split points k = 4..d-4 (those with QB[k][d] on diagonals <= d-4);
// k = 1..3 are added by the light kernel of diagonal d itself
__host__ __device__ __forceinline__ int nchunk_ext(int d) { return d >= 8 ? (d - 7 + KCH - 1) / KCH : 0; }

template <typename T>
struct BifBuf {
  T *main;  // [BIFRING][n][36]  sum_k G[x][k] ec QB[k][y] relative to 2^{E[d-4]}
  T *ext;   // [BIFRING][36]     sum_{k>=4} Gx[k] QB[k][d] relative to 2^{E[d-4]}
  int ncmax;
  float *far;     // [2][n][FARD][farslices][36] far split points of a band, per slice (binary32; nullptr: none)
  int farslices;  // slices per cell in the far buffer
  float *gfac;    // [2][n] far-band rescale factors 2^{E[a] - s a - e0} per band parity (binary32)
  int *gdev;      // [n / FARD + 1] per band: ceil(max over a of |E[a] - s a - e0|), written by k_in_far_factors
  int *spread;    // [1] the spread of interval strengths (bits) found by k_in_range (single problems)
  const T **stab; // [n][SI_N] source of every staged slot of the light cell x = 0 of each diagonal
  T **dtab;       // [n][NCOPY] destination of every result of that cell
};

// Protein b's view of a batch (see DP::bstride); the slot tables hold
// protein 0's addresses, moved by the same offset where they are read.
template <typename T>
__device__ __forceinline__ void bb_shift(BifBuf<T> &b, long long off) {
  b.main = bshift(b.main, off);
  b.ext = bshift(b.ext, off);
  b.far = bshift(b.far, off);
  b.gfac = bshift(b.gfac, off);
  b.gdev = bshift(b.gdev, off);
  b.spread = bshift(b.spread, off);
  b.stab = bshift(b.stab, off);
  b.dtab = bshift(b.dtab, off);
}

// ---------------------------------------------------------------- far bands
// The bifurcation sum of cell (x, y) on diagonal d runs over split points
// a = k - x with halves on diagonals a and d - a.  For the diagonals of a band
// [d0, d0 + FARD), the split points whose halves both lie on diagonals
// <= c = d0 - FARD - 1 are "far": final a whole band earlier, they are summed
// for the band by k_in_far (a tiled product in which every loaded block serves
// up to 16 cells) while the light chain is still FARD - 3 diagonals away; the
// remaining "near" split points (at most 2 (2 FARD - 5) per cell) stay in the
// per-diagonal kernel.  Far blocks are rescaled to a linear exponent with the
// chord s = (E[c] - E[5]) / (c - 5), e0 = E[5] - 5 s: each half is multiplied
// by 2^{E[a] - s a - e0}, so every product of two halves is relative to
// 2^{s d + 2 e0}.  Each CTA of k_in_far sums one slice of split points and
// stores it; the per-diagonal kernel adds the slices in order, so the result
// does not depend on which slice ran first.
// The chord is exact only where E is close to linear.  A protein whose
// composition changes along its length bends E (the best interval of a given
// length moves between regions of different strength), and a factor
// 2^{E[a] - s a - e0} far from one would overflow binary32 or flush the terms
// to zero.  So the factor kernel of each band records the largest deviation
// |E[a] - s a - e0| over the band's split points; past g_cf_far_dev_max
// (log2, 48 unless a test lowers it) the band is not summed in tiles:
// k_in_far returns at once and the per-diagonal kernel takes every split
// point itself, each term with its own power-of-two factor split between its
// two operands (slower; no chord).
constexpr int FARD = 16;   // diagonals per band
// (with the default bound, a product of two tile factors stays within 2^{+-96})
__device__ __forceinline__ int far_dev_max() { return g_cf_far_dev_max; }
constexpr int FARTX = 16;  // rows per far tile
constexpr int FARKC = 8;   // split points staged per step
constexpr int FARKS = 64;   // split points per CTA slice

__host__ __device__ __forceinline__ int far_c(int d0) { return d0 - FARD - 1; }
// does band d0 (a multiple of FARD) have far split points?
__host__ __device__ __forceinline__ bool far_band(int d0) { return d0 >= 3 * FARD; }
__host__ __device__ __forceinline__ int far_kmin(int x0) { return x0 + FARD + 1; }
__host__ __device__ __forceinline__ int far_kmax(int n, int x0, int d0) {
  return x0 + FARTX - 1 + far_c(d0) < n - 1 ? x0 + FARTX - 1 + far_c(d0) : n - 1;
}
// non-empty slices of the tile starting at row x0
__host__ __device__ __forceinline__ int far_nslice(int n, int x0, int d0) {
  return (far_kmax(n, x0, d0) - far_kmin(x0) + FARKS) / FARKS;
}

struct FarChord {
  double s, e0;
};
__device__ __forceinline__ FarChord far_chord(const int *E, int c) {
  const double e5 = (double)__ldcg(E + 5), ec = (double)__ldcg(E + c);
  FarChord r;
  r.s = (ec - e5) / (double)(c - 5);
  r.e0 = e5 - 5.0 * r.s;
  return r;
}

// Range of the binary32 form.  With one exponent per diagonal, the intervals
// of one length are held relative to the strongest of them; binary32 keeps
// about 126 bits below it.  A composition that changes along the protein (a
// block that cannot pair next to an ordinary region) spreads the strengths of
// one diagonal's intervals further, and the weak ones underflow in the inside
// pass (their adjoints overflow in the outside pass).  k_in_range estimates
// that spread after the inside pass from the exterior prefix F(y) = log2 of
// the partition function of [0, y] (its table entries times 2^{E[y]}): the
// strength of an interval [x, x + a] is about F(x + a) - F(x), so
//   spread = max over a <= g_cf_range_maxlen of (max_x - min_x) (F(x + a) - F(x))
// bits.  A prefix that underflowed to zero counts as out of range.  Past
// g_cf_range_limit bits the binary32 inside pass returns CF_ENUMERIC (binary64
// has the range).  The bound on a keeps the slow drift of a long homogeneous
// protein out of the measure (a 4500-nt Dirichlet protein spreads 129 bits
// over all lengths, 99 over lengths up to 400, and its binary32 results are
// within the accuracy bar); the bends that break binary32 are local and show
// at short lengths.  The limit (120 bits over lengths up to 400) was set from
// a calibration over 196 proteins of 200-4500 nt, blocks of 0-30 lysines
// before Dirichlet compositions: every protein whose binary32 results missed
// the bar spread 127 bits or more; the ordinary workloads spread 72-99.  Some
// proteins above the limit would still have been within the bar: the refusal
// is conservative.  The departure of E from a chord is no such measure: it
// also grows with gentle curvature over thousands of diagonals.
static __constant__ int g_cf_range_limit = 120;
static __constant__ int g_cf_range_maxlen = 400;  // lengths a considered (0: all)
__device__ __forceinline__ int range_limit() { return g_cf_range_limit; }

// Everything runs in binary32 (the binary64 pipe of this GPU is a small
// fraction of the binary32 one): a prefix's 72 table entries are binary32
// mantissas, and |F| grows by a few bits per nucleotide (about 2 on the
// 900-nt workload), so below the 51,200-nt bound of this check the rounding
// of F is under 0.01 bits, far below the whole bits the refusal compares.
// Only the binary32 inside pass runs it (binary64 has the range).
template <typename T>
__global__ void __launch_bounds__(1024) k_in_range(DP<T> p, int *spread_out) {
  extern __shared__ float F[];  // [n]
  __shared__ int smax, sflush;
  const int n = p.n, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  if (t == 0) {
    smax = 0;
    sflush = 0;
  }
  __syncthreads();
  for (int y = t; y < n; y += blockDim.x) {
    const T *u = p.Q5U + (size_t)y * BLK, *q = p.Q5P + (size_t)y * BLK;
    float s = 0;
    for (int e = 0; e < BLK; e++) s += (float)u[e] + (float)q[e];
    if (!(s > 0)) atomicOr(&sflush, 1);
    F[y] = s > 0 ? log2f(s) + (float)__ldcg(p.E + y) : 0.0f;
  }
  __syncthreads();
  // one warp per length a, lanes over the start x (x = 0 exists for every a < n)
  int best = 0;
  const int ml = g_cf_range_maxlen;
  const int amax = ml > 0 ? min(n, ml + 1) : n;
  for (int a = 1 + w; a < amax; a += nw) {
    float mx = -3e38f, mn = 3e38f;
    for (int x = lane; x + a < n; x += 32) {
      const float v = F[x + a] - F[x];
      mx = fmaxf(mx, v);
      mn = fminf(mn, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    best = max(best, (int)ceilf(mx - mn));
  }
  if (lane == 0) atomicMax(&smax, best);
  __syncthreads();
  if (t == 0) {
    const int v = sflush ? 100000 : smax;
    *spread_out = v;
    if (sizeof(T) == sizeof(float) && v > range_limit()) atomicOr(p.err, ERR_RANGE_IN);
  }
}

// ---------------------------------------------------------------- K1
// Without far bands (binary64, short proteins): one cell per block (the last
// unit of a diagonal: the exterior sum); warp w of NW takes the chunks w,
// w+NW, ... of 32 split points a = 5..d-4, lanes over the split point;
// per-lane sums are reduced once per warp, then across warps.
template <typename T, int NW>
__device__ __forceinline__ void in_bif_cell(const DP<T> &p, const BifBuf<T> &bb, int d, int cb, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = p.n;
  const int Eref = __ldcg(p.E + d - 4);
  const int slot = d % BIFRING;
  const bool ext = cb == n - d;
  const int x = ext ? 0 : cb, y = x + d;
  const int Ma = p.Mp[x], Mb = p.Mp[y];
  T acc[BLK];
  zero_block(acc);
  const int a1 = d - 4, a2 = d - 3;
  if (w < NW) {
    if (!ext) {
      const int n1 = max(0, a1 - 4), n2 = max(0, d - 3 - a2);
      const int nc = (n1 + n2 + KCH - 1) / KCH;
      const T ec = p.en[EN_EC];
      for (int c = w; c < nc; c += NW) {
        const int q = c * KCH + lane;
        if (q < n1 + n2) {
          const int k = x + (q < n1 ? 5 + q : a2 + q - n1);
          T f = ec * clamp_p2<T>(__ldcg(p.E + k - x) + __ldcg(p.E + y - k) - Eref);
          acc_mm_v<false, false>(acc, p.G + cidx(n, x, k) * BLK, p.QB + cidx(n, k, y) * BLK, Ma, p.Mp[k], Mb, f);
        }
      }
    } else {
      const int nc = nchunk_ext(d);
      for (int c = w; c < nc; c += NW) {
        const int k = 4 + c * KCH + lane;
        if (k <= d - 4) {
          T f = clamp_p2<T>(__ldcg(p.E + k) + __ldcg(p.E + d - k) - Eref);
          acc_mm_v<false, false>(acc, p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, Ma, p.Mp[k], Mb, f);
        }
      }
    }
    warp_reduce_block(acc, Ma, Mb);
    if (lane < 2) {
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e & 1) == lane) red[w][e] = acc[e];
    }
  }
  __syncthreads();
  if (threadIdx.x < BLK) {
    const int e = threadIdx.x;
    T v = 0;
#pragma unroll
    for (int k = 0; k < NW; k++) v += red[k][e];
    T *dst = ext ? bb.ext + (size_t)slot * BLK : bb.main + ((size_t)slot * n + x) * BLK;
    dst[e] = v;
  }
}

// one padded row (6 values) through the read-only path, 8 or 16 bytes at a time
__device__ __forceinline__ void ldg_row6(float (&r)[NS], const float *src) {
  const float2 *s = reinterpret_cast<const float2 *>(src);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    const float2 v = __ldg(s + i);
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void ldg_row6(double (&r)[NS], const double *src) {
  const double2 *s = reinterpret_cast<const double2 *>(src);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    const double2 v = __ldg(s + i);
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}

// acc (rows 3 half .. 3 half + 2 of a 6x6 sum) += f op(A) fb op(B) over the
// live rows (Ma), summation index (Ms) and columns (Mb); TA / TB read A / B
// transposed.  A lane holds three rows of op(A) and one row of B at a time.
// SPLIT applies the term's power-of-two factor in two halves, f to A and fb
// to B, so that neither scaled operand leaves the binary32 range when the
// whole factor is large and one mantissa small (the term itself is in range).
template <bool TA, bool TB, bool SPLIT = false, typename T>
__device__ __forceinline__ void bif_half_acc(T (&acc)[NS / 2 * NS], const T *A, const T *B, T f, int half, int Ma,
                                             int Ms, int Mb, T fb = (T)1) {
  constexpr int HR = NS / 2;
  T av[HR * NS];
#pragma unroll
  for (int r = 0; r < HR; r++) {
    T row[NS];
    if (TA) {
#pragma unroll
      for (int s = 0; s < NS; s++) row[s] = __ldg(A + s * NS + half * HR + r);
    } else {
      ldg_row6(row, A + (half * HR + r) * NS);
    }
#pragma unroll
    for (int s = 0; s < NS; s++) av[r * NS + s] = row[s] * f;
  }
  if (!TB) {
#pragma unroll
    for (int s = 0; s < NS; s++) {
      if (s < Ms) {
        T bv[NS];
        ldg_row6(bv, B + s * NS);
        if (SPLIT) {
#pragma unroll
          for (int b = 0; b < NS; b++) bv[b] *= fb;
        }
#pragma unroll
        for (int r = 0; r < HR; r++)
          if (half * HR + r < Ma) {
#pragma unroll
            for (int b = 0; b < NS; b++)
              if (b < Mb) acc[r * NS + b] = fma(av[r * NS + s], bv[b], acc[r * NS + b]);
          }
      }
    }
  } else {
#pragma unroll
    for (int b = 0; b < NS; b++) {
      if (b < Mb) {
        T bv[NS];
        ldg_row6(bv, B + b * NS);
        if (SPLIT) {
#pragma unroll
          for (int s = 0; s < NS; s++) bv[s] *= fb;
        }
#pragma unroll
        for (int r = 0; r < HR; r++)
          if (half * HR + r < Ma) {
#pragma unroll
            for (int s = 0; s < NS; s++)
              if (s < Ms) acc[r * NS + b] = fma(av[r * NS + s], bv[s], acc[r * NS + b]);
          }
      }
    }
  }
}

// sum acc over the 16 lanes of each half-warp; lanes 0 and 16 store rows
// 0..2 and 3..5 of the result into dst
template <typename T>
__device__ __forceinline__ void bif_half_reduce(T (&acc)[NS / 2 * NS], T *dst, int lane) {
  constexpr int HR = NS / 2;
#pragma unroll
  for (int e = 0; e < HR * NS; e++) {
    T v = acc[e];
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[e] = v;
  }
  if ((lane & 15) == 0) {
#pragma unroll
    for (int e = 0; e < HR * NS; e++) dst[(lane >> 4) * HR * NS + e] = acc[e];
  }
}

// Exterior sum of diagonal d (split points k = 4..d-4 of [0, d]) by all eight
// warps of the CTA, 16 split points per warp and step, in the layout of
// bif_half_acc; the warps' sums are added in order.
template <typename T>
__device__ __forceinline__ void in_bif_ext_group(const DP<T> &p, const BifBuf<T> &bb, int d, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, half = lane >> 4, sl = lane & 15;
  const int n = p.n;
  const int Eref = __ldcg(p.E + d - 4);
  const int Ma = p.Mp[0], Mb = p.Mp[d];
  T acc[NS / 2 * NS];
#pragma unroll
  for (int e = 0; e < NS / 2 * NS; e++) acc[e] = (T)0;
  const int nk = max(0, d - 7), nc = (nk + 15) / 16;
  for (int c = w; c < nc; c += 8) {
    const int k = 4 + c * 16 + sl;
    if (k <= d - 4) {
      const int e = __ldcg(p.E + k) + __ldcg(p.E + d - k) - Eref;
      bif_half_acc<false, false, true>(acc, p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, clamp_p2<T>(e >> 1),
                                       half, Ma, p.Mp[k], Mb, clamp_p2<T>(e - (e >> 1)));
    }
  }
  bif_half_reduce(acc, red[w], lane);
  __syncthreads();
  if (threadIdx.x < BLK) {
    T v = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) v += red[k][threadIdx.x];
    bb.ext[(size_t)(d % BIFRING) * BLK + threadIdx.x] = v;
  }
}

// Near split points of a banded diagonal are few (at most 2 (2 FARD - 5)):
// two warps per cell, four cells per 256-thread CTA.  Within a warp the two
// half-warps take rows 0..2 and 3..5 of the products and their 16 lanes 16
// split points, so that a lane holds three rows of A and of the sum.
template <typename T>
__device__ __forceinline__ void in_bif_group(const DP<T> &p, const BifBuf<T> &bb, int d, int cb0, T (*red)[BLK]) {
  constexpr int NW = 2, NG = 4, HR = NS / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = w / NW, wg = w % NW;
  const int half = lane >> 4, sl = lane & 15;
  const int n = p.n, ncell = n - d;
  const int Eref = __ldcg(p.E + d - 4);
  const int slot = d % BIFRING;
  const int d0 = d / FARD * FARD;
  // a band whose exponent chord bends too far is summed here in full
  const bool banded = bb.far != nullptr && far_band(d0) && __ldcg(bb.gdev + d0 / FARD) <= far_dev_max();
  int a1 = d - 4, a2 = d - 3;
  if (banded) {
    const int c = far_c(d0), alo = max(5, d - c), ahi = min(c, d - 4);
    if (alo <= ahi) {
      a1 = alo - 1;
      a2 = ahi + 1;
    }
  }
  const int cb = cb0 + g;
  if (cb < ncell) {
    const int x = cb, y = x + d;
    const int Ma = p.Mp[x], Mb = p.Mp[y];
    T acc[HR * NS];
#pragma unroll
    for (int e = 0; e < HR * NS; e++) acc[e] = (T)0;
    const int n1 = max(0, a1 - 4), n2 = max(0, d - 3 - a2);
    const int nc = (n1 + n2 + 15) / 16;
    const T ec = p.en[EN_EC];
    for (int c = wg; c < nc; c += NW) {
      const int q = c * 16 + sl;
      if (q < n1 + n2) {
        const int k = x + (q < n1 ? 5 + q : a2 + q - n1);
        const int e = __ldcg(p.E + k - x) + __ldcg(p.E + y - k) - Eref;
        const T *A = p.G + cidx(n, x, k) * BLK, *B = p.QB + cidx(n, k, y) * BLK;
        if (banded)  // near split points of a tiled band: small factors
          bif_half_acc<false, false>(acc, A, B, ec * clamp_p2<T>(e), half, Ma, p.Mp[k], Mb);
        else  // every split point, with factors as large as the exponents' bend
          bif_half_acc<false, false, true>(acc, A, B, ec * clamp_p2<T>(e >> 1), half, Ma, p.Mp[k], Mb,
                                           clamp_p2<T>(e - (e >> 1)));
      }
    }
    bif_half_reduce(acc, red[w], lane);
  }
  // far split points are relative to 2^{s d + 2 e0}: one factor per diagonal
  __shared__ double sfar;
  if (banded && threadIdx.x == 0) {
    const FarChord ch = far_chord(p.E, far_c(d0));
    sfar = (double)p.en[EN_EC] * exp2(ch.s * (double)d + 2.0 * ch.e0 - (double)Eref);
  }
  __syncthreads();
  if (threadIdx.x < NG * BLK) {
    const int g2 = threadIdx.x / BLK, e = threadIdx.x % BLK, cb2 = cb0 + g2;
    if (cb2 < ncell) {
      const int x = cb2;
      T v = red[g2 * NW][e] + red[g2 * NW + 1][e];
      if (banded) {
        // far split points: the slices of the cell's tile in order
        const int nsl = far_nslice(n, x / FARTX * FARTX, d0);
        const float *fp = bb.far + ((((size_t)((d0 / FARD) & 1) * n + x) * FARD + (d - d0)) * bb.farslices) * BLK + e;
        float fv = 0.f;
        for (int sl2 = 0; sl2 < nsl; sl2++) fv += fp[(size_t)sl2 * BLK];
        v += (T)(sfar * (double)fv);
      }
      bb.main[((size_t)slot * n + x) * BLK + e] = v;
    }
  }
}

// binary32 (with or without far bands; a batch, blockIdx.y the protein, has
// none) and short binary64 proteins: CTA b < last takes cells 4b..4b+3, the
// last CTA the exterior sum with all eight warps; 64 registers, so that a CTA
// leaves room for the light kernel's CTAs on its SM (binary64: 128, since 64
// spilled)
template <typename T, bool BT = false>
__global__ void __launch_bounds__(256, 4 / (sizeof(T) / sizeof(float))) k_in_bif_grp(DP<T> p, BifBuf<T> bb, int d) {
  __shared__ T red[8][BLK];
  if (BT) {
    const long long off = (long long)blockIdx.y * p.bstride;
    dp_shift(p, off);
    bb_shift(bb, off);
  }
  if ((int)blockIdx.x == (int)gridDim.x - 1) {
    in_bif_ext_group<T>(p, bb, d, red);
    return;
  }
  in_bif_group<T>(p, bb, d, blockIdx.x * 4, red);
}

// Binary64: grid-stride over the n-d cells and the exterior (one CTA per SM,
// 255 registers): launched with fewer CTAs
// than cells, so that the light kernels of the critical path always find
// room on the SMs.
// (BT: a batch of proteins, blockIdx.y the protein; a compile-time switch so
// that a single protein's kernels read their table pointers straight from the
// parameter bank.)
template <typename T, bool BT = false>
__global__ void __launch_bounds__(256, 1) k_in_bif(DP<T> p, BifBuf<T> bb, int d) {
  __shared__ T red[8][BLK];
  if (BT) {
    const long long off = (long long)blockIdx.y * p.bstride;
    dp_shift(p, off);
    bb_shift(bb, off);
  }
  for (int cb = blockIdx.x; cb <= p.n - d; cb += gridDim.x) {
    in_bif_cell<T, 8>(p, bb, d, cb, red);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- staging

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

// slot layout of the light kernel's staged inputs (blocks of 36 values)
enum : int {
  SI_TX = 0, SI_TY1 = 1, SI_XX = 2, SI_XY1 = 6, SI_CHN = 10, SI_QBI = 11, SI_HBI = 12, SI_Q2I = 13,
  SI_ML = 17, SI_MR = 21, SI_YYP = 25, SI_XIL = 53, SI_CHL = 81, SI_BQ3 = 109, SI_BC3 = 139,
  SI_BC5 = 169, SI_BQ5 = 199, SI_BIF = 229, SI_BIFX = 230, SI_Q5U = 231, SI_Q5P = 232,
  SI_GXK = 233, SI_QBK = 236, SI_N = 239
};

// global source of staged slot s for cell (x, y) of diagonal d, or nullptr
template <typename T>
__device__ __forceinline__ const T *in_slot_src(const DP<T> &p, int s, int x, int y, int d) {
  const int n = p.n;
  if (s == SI_TX) return p.Tr + (size_t)x * BLK;
  if (s == SI_TY1) return d >= 1 ? p.Tr + (size_t)(y - 1) * BLK : nullptr;
  if (s < SI_XY1) return p.X + ((size_t)x * 4 + (s - SI_XX)) * BLK;
  if (s < SI_CHN) return d >= 1 ? p.X + ((size_t)(y - 1) * 4 + (s - SI_XY1)) * BLK : nullptr;
  if (s == SI_CHN) return d >= 1 ? p.CH + cidx(n, x + 1, y) * BLK : nullptr;
  if (s == SI_QBI) return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s == SI_HBI) return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s < SI_ML) {
    if (d < 11) return nullptr;
    const T *t[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
    return t[s - SI_Q2I] + cidx(n, x + 1, y - 1) * BLK;
  }
  if (s < SI_MR) {
    if (d < 5) return nullptr;
    const T *t[4] = {p.QMpp, p.QMpu, p.QM2pp, p.QM2pu};
    return t[s - SI_ML] + cidx(n, x, y - 1) * BLK;
  }
  if (s < SI_YYP) {
    if (d < 10) return nullptr;
    const T *t[4] = {p.QM2up, p.QM2pp, p.QM2uu, p.QM2pu};
    return t[s - SI_MR] + cidx(n, x + 1, y) * BLK;
  }
  const int Lmax = min(MAXLOOP, d - 4);
  if (s < SI_XIL) {  // YY_{L-1}[x+1][y], L = 3..30
    int L = s - SI_YYP + 3;
    return (d >= 6 && L <= Lmax) ? yy_in(p, x + 1, d - 1) + (size_t)(L - 3) * BLK : nullptr;
  }
  if (s < SI_CHL) {  // XI[x][y-L+2]
    int L = s - SI_XIL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.XI + cidx(n, x, yl) * BLK : nullptr;
  }
  if (s < SI_BQ3) {  // CH[y-L+2][y]
    int L = s - SI_CHL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.CH + cidx(n, yl, y) * BLK : nullptr;
  }
  if (s < SI_BIF) {
    const int L = (s - SI_BQ3) % MAXLOOP + 1;
    if (d - L < 4) return nullptr;
    if (s < SI_BC3) return p.QB + cidx(n, x, y - L) * BLK;
    if (s < SI_BC5) return p.CH + cidx(n, y - L, y) * BLK;
    if (s < SI_BQ5) return p.CH + cidx(n, x, x + L) * BLK;
    return p.QB + cidx(n, x + L, y) * BLK;
  }
  return nullptr;  // remaining slots need the bifurcation buffers: in_slot_src2
}

// bifurcation results and exterior-prefix inputs
template <typename T>
__device__ __forceinline__ const T *in_slot_src2(const DP<T> &p, const BifBuf<T> &bb, int s, int x, int d) {
  const int n = p.n, slot = d % BIFRING;
  if (s == SI_BIF) return nchunk_bif(d) > 0 ? bb.main + ((size_t)slot * n + x) * BLK : nullptr;
  if (x != 0 || d == 0) return nullptr;
  if (s == SI_BIFX) return nchunk_ext(d) > 0 ? bb.ext + (size_t)slot * BLK : nullptr;
  if (s == SI_Q5U) return p.Q5U + (size_t)(d - 1) * BLK;
  if (s == SI_Q5P) return p.Q5P + (size_t)(d - 1) * BLK;
  const int k = (s < SI_QBK ? s - SI_GXK : s - SI_QBK) + 1;
  if (k > d - 4) return nullptr;
  return s < SI_QBK ? p.Gx + (size_t)k * BLK : p.QB + cidx(n, k, d) * BLK;
}

// Slots whose source lies on diagonal d-1 (written by the previous light
// kernel): CH[x+1][y], QM*[x][y-1], QM2*[x+1][y], the YY run from (x+1, y),
// XI[x][y-1] (L = 3), the bulges QB[x][y-1] and QB[x+1][y] (L = 1), the
// exterior prefix of d-1 and QB[1][d].  Every other source is on a diagonal
// <= d-2, a fixed table, or the bifurcation sums of d (complete before the
// kernel starts).
__host__ __device__ __forceinline__ bool in_slot_late(int s) {
  return s == SI_CHN || (s >= SI_ML && s <= SI_YYP) || s == SI_XIL || s == SI_BQ3 || s == SI_BQ5 || s == SI_Q5U ||
         s == SI_Q5P || s == SI_QBK;
}

// Along a diagonal every slot's source moves by a fixed stride per cell (the
// tables are diagonal-major), so the light kernel finds it as the source of
// cell x = 0 (a per-diagonal table) plus x times the stride; 0: the slot is
// read by cell x = 0 only (exterior prefix).
__host__ __device__ __forceinline__ int in_slot_stride(int s) {
  if (s >= SI_XX && s < SI_CHN) return 4 * BLK;
  if (s >= SI_YYP && s < SI_XIL) return NYY * BLK;
  if (s > SI_BIF) return 0;
  return BLK;
}

// ---------------------------------------------------------------- K2
constexpr int NT_IN = 256;    // threads per cell of the inside light kernel
constexpr int NT = 512;       // threads per cell on diagonals with few cells
constexpr int NT_WIDE = 256;  // ... and on diagonals with more than WIDE_CELLS cells
constexpr int WIDE_CELLS = 296;

// ---------------------------------------------------------------- row products
// Every table entry is a 6x6 block whose rows and columns beyond the codon-
// state counts are zero, so block products can always run over the full
// padded size: the padding contributes exact zeros.  Fixed trip counts let the
// compiler keep a row of the left operand in registers and stream the rows of
// the right operand with 8/16-byte shared-memory loads.
template <typename T>
struct Row2;
template <>
struct Row2<float> {
  using type = float2;
};
template <>
struct Row2<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ void ld_row(T (&r)[NS], const T *src) {
  using V = typename Row2<T>::type;
  const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    const V v = s[i];
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void st_row(T *dst, const T (&r)[NS]) {
  using V = typename Row2<T>::type;
  V *d = reinterpret_cast<V *>(dst);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    V v;
    v.x = r[2 * i];
    v.y = r[2 * i + 1];
    d[i] = v;
  }
}
// r += (f * av) . B   (av: one row of the left operand)
template <typename T>
__device__ __forceinline__ void row_acc(T (&r)[NS], const T (&av)[NS], const T *B, T f) {
#pragma unroll
  for (int s = 0; s < NS; s++) {
    T bv[NS];
    ld_row(bv, B + s * NS);
    const T x = av[s] * f;
#pragma unroll
    for (int b = 0; b < NS; b++) r[b] = fma(x, bv[b], r[b]);
  }
}
// r += f * (row a of A) . B
template <typename T>
__device__ __forceinline__ void row_mm(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
  ld_row(av, A + a * NS);
  row_acc(r, av, B, f);
}
// r += f * (row a of A) . B . C
template <typename T>
__device__ __forceinline__ void row_mmm(T (&r)[NS], const T *A, const T *B, const T *C, int a, T f) {
  T t[NS];
#pragma unroll
  for (int b = 0; b < NS; b++) t[b] = (T)0;
  row_mm(t, A, B, a, (T)1);
  row_acc(r, t, C, f);
}
// r += f * (row a of A^T) . B  = f * sum_s A[s][a] B[s][.]
template <typename T>
__device__ __forceinline__ void row_tmm(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
#pragma unroll
  for (int s = 0; s < NS; s++) av[s] = A[s * NS + a];
  row_acc(r, av, B, f);
}
// r += f * (row a of A) . B^T  = f * sum_s A[a][s] B[.][s]
template <typename T>
__device__ __forceinline__ void row_mmt(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
  ld_row(av, A + a * NS);
#pragma unroll
  for (int s = 0; s < NS; s++) av[s] *= f;
#pragma unroll
  for (int b = 0; b < NS; b++) {
    T bv[NS];
    ld_row(bv, B + b * NS);
    T acc = r[b];
#pragma unroll
    for (int s = 0; s < NS; s++) acc = fma(av[s], bv[s], acc);
    r[b] = acc;
  }
}
// atomically add a block row to global memory, skipping exact-zero pairs
__device__ __forceinline__ void red_row(float *dst, const float (&r)[NS]) {
#pragma unroll
  for (int i = 0; i < NS / 2; i++)
    if (r[2 * i] != 0.f || r[2 * i + 1] != 0.f)
      asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst + 2 * i), "f"(r[2 * i]), "f"(r[2 * i + 1])
                   : "memory");
}
__device__ __forceinline__ void red_row(double *dst, const double (&r)[NS]) {
#pragma unroll
  for (int i = 0; i < NS; i++)
    if (r[i] != 0.0) atomicAdd(dst + i, r[i]);
}

template <typename T>
__device__ __forceinline__ void row_zero(T (&r)[NS]) {
#pragma unroll
  for (int b = 0; b < NS; b++) r[b] = (T)0;
}
template <typename T>
__device__ __forceinline__ T row_absmax(const T (&r)[NS]) {
  T m = 0;
#pragma unroll
  for (int b = 0; b < NS; b++) m = fmax(m, fabs(r[b]));
  return m;
}

// ---------------------------------------------------------------- K0: far band
// Grid (tiles, slices), 256 threads: the CTA takes a tile of FARTX rows x and
// the FARD diagonals of band d0 (thread (tx, tj) owns cell (x0 + tx,
// x0 + tx + d0 + tj)) and a slice of FARKS split points k.  Split points are
// staged FARKC at a time into two alternating stages: G[x][k] for the tile's
// rows and QB[k][y] for its FARTX + FARD - 1 columns, one TMA bulk copy per
// block; the linear-exponent factors of both halves are applied as the
// blocks are used.  The slice's sums go to their own place in the band buffer.
// the rescale factors of band d0, once per band (binary64 exp2: the
// exponents reach the thousands), and the band's largest deviation from the
// chord over its split points a = 5..c; one CTA
__global__ void k_in_far_factors(DP<float> p, BifBuf<float> bb, int d0) {
  __shared__ int sdev;
  const int c = far_c(d0);
  const FarChord ch = far_chord(p.E, c);
  float *dst = bb.gfac + (size_t)((d0 / FARD) & 1) * p.n;
  if (threadIdx.x == 0) sdev = 0;
  __syncthreads();
  int dev = 0;
  for (int a = threadIdx.x; a <= c; a += blockDim.x) {
    const double z = (double)__ldcg(p.E + a) - ch.s * a - ch.e0;
    dst[a] = (float)exp2(z);
    if (a >= 5) dev = max(dev, (int)ceil(fabs(z)));
  }
  atomicMax(&sdev, dev);
  __syncthreads();
  if (threadIdx.x == 0) bb.gdev[d0 / FARD] = sdev;
}

__global__ void __launch_bounds__(256) k_in_far(DP<float> p, BifBuf<float> bb, int d0) {
  constexpr int TY = FARTX + FARD - 1, STAGE = FARKC * (FARTX + TY) * BLK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *buf = (float *)smem_raw;  // [2][STAGE]: G [FARKC][FARTX][36], QB [FARKC][TY][36]
  float *gf = buf + 2 * STAGE;     // [c + 1] factors 2^{E[a] - s a - e0}
  __shared__ __align__(8) unsigned long long sbar[2];
  const int n = p.n, t = threadIdx.x, tx = t % FARTX, tj = t / FARTX;
  const int x0 = blockIdx.x * FARTX, x = x0 + tx, d = d0 + tj, y = x + d;
  const int c = far_c(d0);
  const int kbeg = far_kmin(x0) + blockIdx.y * FARKS;
  const int kend = min(far_kmax(n, x0, d0), kbeg + FARKS - 1);
  if (kbeg > kend) return;
  if (__ldcg(bb.gdev + d0 / FARD) > far_dev_max()) return;  // summed by the per-diagonal kernel
  const float *gsrc = bb.gfac + (size_t)((d0 / FARD) & 1) * n;
  for (int a = t; a <= c; a += 256) gf[a] = __ldcg(gsrc + a);
  if (t == 0) {
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
  }
  __syncthreads();
  auto stage = [&](int k0, int bsel) {
    float *Gs = buf + (size_t)bsel * STAGE, *Qs = Gs + FARKC * FARTX * BLK;
    for (int q = t; q < FARKC * (FARTX + TY); q += 256) {
      const float *src = nullptr;
      float *dst;
      if (q < FARKC * FARTX) {
        const int kk = q / FARTX, r = q % FARTX, xx = x0 + r, k = k0 + kk;
        dst = Gs + (size_t)q * BLK;
        if (k <= kend && xx < n && k - xx >= 5) src = p.G + cidx(n, xx, k) * BLK;
      } else {
        const int q2 = q - FARKC * FARTX, kk = q2 / TY, cy = q2 % TY, k = k0 + kk, yy = x0 + d0 + cy;
        dst = Qs + (size_t)q2 * BLK;
        if (k <= kend && yy < n && yy - k >= 4) src = p.QB + cidx(n, k, yy) * BLK;
      }
      if (src) {
        mbar_expect(&sbar[bsel], BLK * 4);
        bulk_g2s(dst, src, BLK * 4, &sbar[bsel]);
      } else {
#pragma unroll
        for (int e = 0; e < BLK; e++) dst[e] = 0.f;
      }
    }
    __syncthreads();
    if (t == 0) mbar_arrive(&sbar[bsel]);
  };
  const bool live = y < n;
  const int alo = max(5, d - c), ahi = min(c, d - 4);
  float acc[BLK];
  zero_block(acc);
  unsigned ph[2] = {0u, 0u};
  stage(kbeg, 0);
  int bsel = 0;
  for (int k0 = kbeg; k0 <= kend; k0 += FARKC, bsel ^= 1) {
    if (k0 + FARKC <= kend) stage(k0 + FARKC, bsel ^ 1);  // released at the end of the previous step
    if (!__syncthreads_and(mbar_wait(&sbar[bsel], ph[bsel], p.err))) return;
    ph[bsel] ^= 1u;
    const float *Gs = buf + (size_t)bsel * STAGE, *Qs = Gs + FARKC * FARTX * BLK;
    if (live) {
#pragma unroll 1
      for (int kk = 0; kk < FARKC; kk++) {
        const int k = k0 + kk, a = k - x;
        if (a < alo || a > ahi || k > kend) continue;
        const float f = gf[a] * gf[d - a];
        const float *A = Gs + ((size_t)kk * FARTX + tx) * BLK;
        const float *B = Qs + ((size_t)kk * TY + (tx + tj)) * BLK;
#pragma unroll
        for (int r = 0; r < NS; r++) {
          float av[NS];
          ld_row(av, A + r * NS);
#pragma unroll
          for (int s2 = 0; s2 < NS; s2++) {
            float bv[NS];
            ld_row(bv, B + s2 * NS);
            const float xa = av[s2] * f;
#pragma unroll
            for (int b = 0; b < NS; b++) acc[r * NS + b] = fmaf(xa, bv[b], acc[r * NS + b]);
          }
        }
      }
    }
    fence_proxy_async();
    __syncthreads();  // the next step's copies reuse this stage
  }
  if (live) {
    float *dst = bb.far + ((((size_t)((d0 / FARD) & 1) * n + x) * FARD + tj) * bb.farslices + blockIdx.y) * BLK;
#pragma unroll
    for (int e = 0; e < BLK; e++) dst[e] = acc[e];
  }
}

// ---------------------------------------------------------------- checkpointed YY
// One diagonal D of the interior partial sums, recomputed for the outside pass
// from diagonal D - 1 (the block buffer, or the checkpoint at the start of a
// block) with the light kernel's own recursion and operation order:
//   YY_2 = XI,  YY_L[x][y] = T_x YY_{L-1}[x+1][y] + XI[x][y-L+2] CH[y-L+2][y],
// so the values equal those the inside pass computed, bit for bit.  One
// thread per output row (cell, L, state a): 29 x 6 rows per cell.
template <typename T>
__global__ void __launch_bounds__(192) k_yy_step(DP<T> p, int D) {
  const int n = p.n, x = blockIdx.x, y = x + D;
  const int t = threadIdx.x;
  if (t >= NYY * NS) return;
  const int L = 2 + t / NS, a = t % NS;
  const int Lmax = min(MAXLOOP, D - 4);
  T r[NS];
  row_zero(r);
  if (D >= 6 && L <= Lmax) {
    if (L == 2) {
      ld_row(r, p.XI + cidx(n, x, y) * BLK + a * NS);
    } else {
      row_mm(r, p.Tr + (size_t)x * BLK, yy_out(p, x + 1, D - 1) + (size_t)(L - 3) * BLK, a, (T)1);
      const int yl = y - L + 2;
      if (yl - x >= 6) row_mm(r, p.XI + cidx(n, x, yl) * BLK, p.CH + cidx(n, yl, y) * BLK, a, (T)1);
    }
  }
  st_row(yy_out(p, x, D) + (size_t)(L - 2) * BLK + a * NS, r);
}

__host__ __device__ constexpr size_t in_far_smem(int c) {
  return ((size_t)2 * FARKC * (FARTX + FARTX + FARD - 1) * BLK + (size_t)(c + 1)) * sizeof(float);
}

// ---------------------------------------------------------------- K2
// Light work of one cell (x, y) of diagonal d in two phases of independent
// work, split by task and block row (6 threads per task, one output row
// each):
//   phase A  chain, XI, the 28 interior partial sums YY_3..YY_30, the bulge
//            sums (12 partial blocks), the QB terms (hairpin-interior,
//            stack in 3 parts, multiloop in 2), QMpu, G, QM2pu/up/uu and the
//            exterior row;
//   phase B  HB (sum over interior sizes, bulges and hairpin), QB, QMpp,
//            QM2pp and the exterior Q5P, entry by entry.
// Staged input slots that a diagonal does not use are zero-filled, so every
// task runs unconditionally; loop weights that do not apply are zero.
// Phase A runs 16 groups of 5 tasks, one warp per group (lanes 0..29: task
// i = lane / 6, block row lane % 6), so that every warp follows one code path:
//   groups 0..5   interior partial sums YY_L, L = 3 + 5g + i (L <= 30)
//   groups 6..11  bulge pairs: task j = 5(g-6) + i, side j & 1 (0: 3', 1: 5'),
//                 sizes L = 2(j >> 1) + 1 and the next one
//   group 12      chain, XI, QB hairpin-interior term, QB multiloop (2 parts)
//   group 13      QB stack for outer pair types P = 0..4 (P = 5 in group 15)
//   group 14      QMpu, G, QM2pu, QM2up, QM2uu
//   group 15      exterior Gx, Q5U, Q5P split points 1..3 (cell x = 0), stack P = 5
constexpr int NGROUP = 16;
// shared result slots (blocks); every final result is copied to its table at
// the end of the cell
enum : int {
  LO_CH = 0, LO_XI = 1, LO_YY = 2,            // YY_L at LO_YY + L - 3
  LO_BU = 30, NLO_BU = 30, LO_QBH = 60, LO_QBS = 61, LO_QBM = 67, LO_Q5K = 69,
  LO_QMPU = 70, LO_G = 71, LO_M2PU = 72, LO_M2UP = 73, LO_M2UU = 74, LO_GX = 75, LO_Q5U = 76,
  LO_HB = 77, LO_QB = 78, LO_QMPP = 79, LO_QM2PP = 80, LO_Q5P = 81, LO_N = 82
};

// pair type of bases (x, y) from a packed table: 3 bits per entry, 7 = no pair
__device__ __forceinline__ int pair_type_lut(int bx, int by) {
  constexpr unsigned long long PT = 0xf7b9d7e7f1ffull;
  const int v = (int)((PT >> (3 * (bx * 4 + by))) & 7ull);
  return v;
}

// Threads per entry in the HB sum of phase B, and the first thread of the
// QB/QMpp entries (a warp boundary after the HB threads).
template <int NTT>
struct LightMap {
  static constexpr int GHB = NTT >= 512 ? 8 : 4;
  static constexpr int QB0 = (GHB * BLK + 31) / 32 * 32;
  static_assert(QB0 + BLK <= NTT, "phase B needs one thread per QB entry");
};

// Results written by the light cell: entry k of the copy-out list reads
// shared slot light_slot(k) and goes to light_dst(k) (nullptr: not written on
// this diagonal).
constexpr int NCOPY = 43;
__device__ __forceinline__ int light_slot(int k) {
  static_assert(LO_QB == LO_HB + 1 && LO_QMPP == LO_HB + 2 && LO_QM2PP == LO_HB + 3 && LO_G == LO_QMPU + 1 &&
                    LO_M2PU == LO_QMPU + 2 && LO_M2UP == LO_QMPU + 3 && LO_M2UU == LO_QMPU + 4 &&
                    LO_GX == LO_QMPU + 5 && LO_Q5U == LO_QMPU + 6,
                "result slots in copy-out order");
  if (k <= 2) return k == 0 ? LO_CH : LO_XI;  // CH, XI, YY_2 (= XI)
  if (k < 31) return LO_YY + k - 3;           // YY_L, L = 3..30
  if (k < 35) return LO_HB + k - 31;          // HB, QB, QMpp, QM2pp
  if (k < 42) return LO_QMPU + k - 35;        // QMpu, G, QM2pu, QM2up, QM2uu, Gx, Q5U
  return LO_Q5P;
}
template <typename T>
__device__ __forceinline__ T *light_dst(const DP<T> &p, int k, int x, int d, size_t c) {
  const int Lmax = min(MAXLOOP, d - 4);
  if (k == 0) return p.CH + c * BLK;
  if (k == 1) return d >= 6 ? p.XI + c * BLK : nullptr;
  if (k < 31) return (d >= 6 && k <= Lmax) ? yy_in(p, x, d) + (size_t)(k - 2) * BLK : nullptr;  // YY_k
  switch (k) {
    case 31: return d >= 2 ? p.HB + c * BLK : nullptr;
    case 32: return d >= 4 ? p.QB + c * BLK : nullptr;
    case 33: return d >= 4 ? p.QMpp + c * BLK : nullptr;
    case 34: return d >= 4 ? p.QM2pp + c * BLK : nullptr;
    case 35: return d >= 5 ? p.QMpu + c * BLK : nullptr;
    case 36: return d >= 5 ? p.G + c * BLK : nullptr;
    case 37: return d >= 10 ? p.QM2pu + c * BLK : nullptr;
    case 38: return d >= 10 ? p.QM2up + c * BLK : nullptr;
    case 39: return d >= 10 ? p.QM2uu + c * BLK : nullptr;
    case 40: return (x == 0 && d >= 1) ? p.Gx + (size_t)d * BLK : nullptr;
    case 41: return x == 0 ? p.Q5U + (size_t)d * BLK : nullptr;
    case 42: return x == 0 ? p.Q5P + (size_t)d * BLK : nullptr;
  }
  return nullptr;
}

// stride of result k along a diagonal, as in_slot_stride
__host__ __device__ __forceinline__ int light_dst_stride(int k) {
  if (k >= 2 && k < 31) return NYY * BLK;
  if (k >= 40) return 0;
  return BLK;
}

// the per-diagonal tables of slot sources and result destinations of cell
// x = 0 (once per problem: they hold only table addresses)
template <typename T>
__global__ void k_in_slot_tab(DP<T> p, BifBuf<T> bb) {
  const int d = blockIdx.x;
  for (int s = threadIdx.x; s < SI_N; s += blockDim.x)
    bb.stab[(size_t)d * SI_N + s] = s < SI_BIF ? in_slot_src(p, s, 0, d, d) : in_slot_src2(p, bb, s, 0, d);
  for (int k = threadIdx.x; k < NCOPY; k += blockDim.x)
    bb.dtab[(size_t)d * NCOPY + k] = light_dst(p, k, 0, d, cidx(p.n, 0, d));
}

template <typename T, int NTT, bool BT>
__device__ __forceinline__ void in_light_cell(const DP<T> &p, const BifBuf<T> &bb, int d, int x,
                                              unsigned char *smem_raw) {
  using LM = LightMap<NTT>;
  T *S = (T *)smem_raw;                // [SI_N][36] staged inputs
  T *O = S + (size_t)SI_N * BLK;       // [LO_N][36] phase A results
  __shared__ int sEd;
  __shared__ T smax[NTT / 32];  // largest magnitude per warp (table precision suffices for ilogb)
  __shared__ int sE[96], sE0[4], sBx[3][NS], sBy[3][NS];
  __shared__ T sEn[EN_N], sHL, wIn[MAXLOOP + 1];
  __shared__ __align__(8) unsigned long long sbar;
  __shared__ T *sDst[NCOPY];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int y = x + d;
  const size_t c = cidx(n, x, y);
  // per-cell context, each value loaded by its own thread before any copy is
  // issued so that all loads are in flight together: exponents of diagonals
  // d-47..d-1, bases of x-1..x+1 and y-1..y+1, energy factors, and the
  // largest mantissa and exponent of diagonal d-1 (last thread)
  static_assert(NTT > EN_N && NTT > 100 + 6 * NS && NTT >= SI_N, "one context value and slot per thread");
  // the barrier (one arrival per thread) is initialised first: its release
  // fence would otherwise wait for the context loads below
  if (t == 0) mbar_init(&sbar, NTT);
  int cE = 0, cB = 0;
  T cEn = 0;
  unsigned long long cMax = 0;
  // Values of diagonal d-1 come from the previous light kernel, which may
  // still be running (programmatic launch): they are read after griddep_wait
  // ("late"); every other input is final and is read before it.
  bool lateE = false;
  if (t < EN_N) cEn = p.en[t];
  if (t < 96) {
    const int k = d - 47 + t;
    if (k >= 0 && k < d) {
      if (k == d - 1) lateE = true;
      else cE = __ldcg(p.E + k);
    }
  } else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    const int q = (side == 0 ? x : y) - 1 + r;
    if (q >= 0 && q < n) cB = p.base[q * NS + a];
  } else if (t >= 96 + 6 * NS && t < 100 + 6 * NS) {
    const int k = t - 96 - 6 * NS;  // exponents of diagonals 0..3 (exterior split points)
    if (k < d) {
      if (k == d - 1) lateE = true;
      else cE = __ldcg(p.E + k);
    }
  } else if (t == NTT - 1 && d > 0) {
    lateE = true;  // largest mantissa and exponent of diagonal d-1
  }
  T cHL = 0;
  if (t == NTT - 2) cHL = p.eHL[d + 1];  // hairpin length factor of the cell
  const long long boff = BT ? (long long)blockIdx.y * p.bstride : 0;  // batch: protein 0's addresses + boff
  const T *src0 = t < SI_N ? bshift(bb.stab[(size_t)d * SI_N + t], boff) : nullptr;
  T *dst0 = t < NCOPY ? bshift(bb.dtab[(size_t)d * NCOPY + t], boff) : nullptr;
  __syncthreads();
  // Staging: one TMA bulk copy per input block (the interior partial sums
  // YY_{L-1}[x+1][y], L = 3..Lmax, are contiguous and go as one copy); slots
  // this cell does not use are zero-filled.  Every thread arrives once at the
  // barrier with the bytes of its copy (copies that complete earlier leave
  // the transaction count transiently negative, which the barrier allows).
  // Slots whose source lies on diagonal d-1 are issued after griddep_wait,
  // the rest before it.
  unsigned nbytes = 0;
  const int LmaxS = min(MAXLOOP, d - 4);
  const bool stage = t < SI_N && !(t > SI_YYP && t < SI_XIL && d >= 6 && t - SI_YYP + 3 <= LmaxS);  // not in the YY run
  const bool late = stage && in_slot_late(t);
  auto issue = [&]() {
    const int s = t;
    T *dst = S + (size_t)s * BLK;
    const int st = in_slot_stride(s);
    const T *src = src0 == nullptr ? nullptr : (st ? src0 + (size_t)x * st : (x == 0 ? src0 : nullptr));
    if (src) {
      const unsigned bytes = (s == SI_YYP ? (unsigned)(LmaxS - 2) : 1u) * BLK * (unsigned)sizeof(T);
      bulk_g2s(dst, src, bytes, &sbar);
      nbytes = bytes;
    } else {
#pragma unroll
      for (int q = 0; q < BLK; q++) dst[q] = (T)0;
    }
  };
  if (stage && !late) issue();
  griddep_wait();
  if (lateE) {
    cE = __ldcg(p.E + d - 1);
    if (t == NTT - 1) cMax = __ldcg(p.dmax + d - 1);
  }
  if (late) issue();
  griddep_launch_dependents();  // the next diagonal's kernel may start its own early part
  mbar_arrive_expect(&sbar, nbytes);
  // destinations of the results (copied out at the end of the cell)
  if (t < NCOPY) {
    const int st = light_dst_stride(t);
    sDst[t] = dst0 == nullptr ? nullptr : (st ? dst0 + (size_t)x * st : (x == 0 ? dst0 : nullptr));
  }
  // the context reaches shared memory while the copies are in flight
  if (t < EN_N) sEn[t] = cEn;
  if (t < 96) {
    sE[t] = cE;
  } else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    if (side == 0) sBx[r][a] = cB;
    else sBy[r][a] = cB;
  } else if (t < 100 + 6 * NS) {
    sE0[t - 96 - 6 * NS] = cE;
  } else if (t == NTT - 1) {
    int e = 0;
    if (d > 0) {
      const double mx = __longlong_as_double((long long)cMax);
      e = cE;
      if (mx > 0) {
        if (isfinite(mx)) e += ilogb(mx);
        else atomicOr(p.err, 1);
      }
    }
    sEd = e;
    if (x == 0) p.E[d] = e;
  } else if (t == NTT - 2) {
    sHL = cHL;
  }
  if (!__syncthreads_and(mbar_wait(&sbar, 0, p.err))) return;
  const int Ed = sEd;
  const T *en = sEn;
  const T *Tx = S + SI_TX * BLK, *Ty1 = S + SI_TY1 * BLK;
  const T *Xl = S + SI_XX * BLK, *Xr = S + SI_XY1 * BLK;
  const int Lmax = min(MAXLOOP, d - 4);
  T lmax = 0;
  // interior-loop weights e^{-I(L)} 2^{E[d-L+2]-E[d]} for the HB sum of phase B
  if (t >= 2 && t <= MAXLOOP) wIn[t] = en[EN_IN + t] * clamp_p2<T>(EAS(d - t + 2) - Ed);

  // ---------------- phase A: one warp per group of tasks
  // Every task but the stack is a sum of at most three terms
  //   f * (row a of A) . B [. C]
  // described by pointers, so that the product code exists once.
  for (int vw = w; vw < NGROUP; vw += NTT / 32) {
    const int i = lane / NS, a = lane - i * NS;
    if (i >= 5) continue;
    const T *A0 = nullptr, *B0 = nullptr, *C0 = nullptr, *A1 = nullptr, *B1 = nullptr, *C1 = nullptr;
    const T *A2 = nullptr, *B2 = nullptr;
    T f0 = 1, f1 = 1, f2 = 1;
    int oslot = -1, post = 0;  // post: 1 identity (d = 0), 2 XI mismatch factor, 3 stack
    bool scaled = false;       // counts toward the diagonal maximum
    if (vw < 6) {
      const int L = 3 + 5 * vw + i;
      if (L > MAXLOOP) continue;
      if (d >= 6 && L <= Lmax) {
        A0 = Tx, B0 = S + (SI_YYP + L - 3) * BLK;
        A1 = S + (SI_XIL + L - 3) * BLK, B1 = S + (SI_CHL + L - 3) * BLK;
      }
      oslot = LO_YY + L - 3;  // relative to 2^{E[d-L+2]}
    } else if (vw < 12) {
      const int j = 5 * (vw - 6) + i, side = j & 1, L = 2 * (j >> 1) + 1;
      if (d - L >= 4) {
        A0 = S + ((side ? SI_BC5 : SI_BQ3) + L - 1) * BLK, B0 = S + ((side ? SI_BQ5 : SI_BC3) + L - 1) * BLK;
        f0 = en[EN_BU + L] * clamp_p2<T>(EAS(d - L) - Ed);
      }
      if (d - L - 1 >= 4) {
        A1 = S + ((side ? SI_BC5 : SI_BQ3) + L) * BLK, B1 = S + ((side ? SI_BQ5 : SI_BC3) + L) * BLK;
        f1 = en[EN_BU + L + 1] * clamp_p2<T>(EAS(d - L - 1) - Ed);
      }
      oslot = LO_BU + j;
    } else if (vw == 12) {
      if (i == 0) {  // chain
        if (d == 0) post = 1;
        else A0 = Tx, B0 = S + SI_CHN * BLK;
        oslot = LO_CH;
      } else if (i == 1) {  // XI
        if (d >= 6) A0 = Tx, B0 = S + SI_QBI * BLK, C0 = Ty1, f0 = clamp_p2<T>(EAS(d - 2) - Ed), post = 2;
        oslot = LO_XI;
        scaled = true;
      } else if (i == 2) {  // QB: hairpin-interior term
        if (d >= 4) A0 = Tx, B0 = S + SI_HBI * BLK, C0 = Ty1;
        oslot = LO_QBH;
      } else {  // QB: multiloop
        if (d >= 11) {
          const T *q2 = S + SI_Q2I * BLK, *xl = Xl + (i == 3 ? XPU : XPP) * BLK;
          A0 = xl, B0 = q2 + (i == 3 ? 0 : 2) * BLK, C0 = Xr + XUP * BLK;
          A1 = xl, B1 = q2 + (i == 3 ? 1 : 3) * BLK, C1 = Xr + XPP * BLK;
        }
        oslot = LO_QBM + i - 3;
      }
    } else if (vw == 13 || (vw == 15 && i == 3)) {
      oslot = LO_QBS + (vw == 13 ? i : 5);
      if (d >= 6) post = 3;
    } else if (vw == 14) {
      // QMpu, G (inner state y-1), QM2pu, QM2up, QM2uu
      const T F1 = clamp_p2<T>(EAS(d - 1) - Ed), eb = en[EN_EB];
      if (i < 2) {
        if (d >= 5) {
          f0 = f1 = i == 0 ? eb * F1 : F1;
          A0 = S + SI_ML * BLK, B0 = Xr + (i == 0 ? XPU : XPP) * BLK;
          A1 = S + (SI_ML + 1) * BLK, B1 = Xr + (i == 0 ? XUU : XUP) * BLK;
        }
      } else if (d >= 10) {
        f0 = f1 = eb * F1;
        if (i == 2) {
          A0 = S + (SI_ML + 2) * BLK, B0 = Xr + XPU * BLK;
          A1 = S + (SI_ML + 3) * BLK, B1 = Xr + XUU * BLK;
        } else {
          A0 = Xl + XUU * BLK, B0 = S + (SI_MR + (i == 3 ? 0 : 2)) * BLK;
          A1 = Xl + XUP * BLK, B1 = S + (SI_MR + (i == 3 ? 1 : 3)) * BLK;
        }
      }
      oslot = LO_QMPU + i;
      scaled = true;
    } else {
      // exterior prefix [0, d] (cell x = 0): rows are the states of position 0
      if (x != 0 || i > 2) continue;
      const T *pu = S + SI_Q5U * BLK, *pp = S + SI_Q5P * BLK;
      const T F1 = clamp_p2<T>(EAS(d - 1) - Ed);
      if (i < 2) {
        if (d == 0 && i == 1) post = 1;
        if (d >= 1) {
          f0 = f1 = F1;
          A0 = pu, B0 = Xr + (i == 0 ? XUP : XUU) * BLK;
          A1 = pp, B1 = Xr + (i == 0 ? XPP : XPU) * BLK;
        }
        oslot = i == 0 ? LO_GX : LO_Q5U;
        scaled = true;
      } else {
        // split points k = 1..3 use QB[k][d] of diagonals d-1..d-3
        if (d >= 5) A0 = S + SI_GXK * BLK, B0 = S + SI_QBK * BLK, f0 = clamp_p2<T>(sE0[1] + EAS(d - 1) - Ed);
        if (d >= 6) A1 = S + (SI_GXK + 1) * BLK, B1 = S + (SI_QBK + 1) * BLK, f1 = clamp_p2<T>(sE0[2] + EAS(d - 2) - Ed);
        if (d >= 7) A2 = S + (SI_GXK + 2) * BLK, B2 = S + (SI_QBK + 2) * BLK, f2 = clamp_p2<T>(sE0[3] + EAS(d - 3) - Ed);
        oslot = LO_Q5K;
      }
    }
    T r[NS];
    row_zero(r);
    if (post == 3) {
      // QB stack for outer pair type P: sum over inner states (a2, b2) of
      // Tx[a][a2] QBI[a2][b2] stk[P][pt(a2, b2)] Ty1[b2][b], kept where the
      // outer pair (a, b) has type P
      const int P = oslot - LO_QBS;
      const int bxa = BASE(x, a);
      bool any = false;
#pragma unroll
      for (int b = 0; b < NS; b++) any |= pair_type_lut(bxa, BASE(y, b)) == P;
      if (any) {
        const T *qin = S + SI_QBI * BLK;
        T tx[NS], t1[NS];
        ld_row(tx, Tx + a * NS);
        row_zero(t1);
#pragma unroll
        for (int a2 = 0; a2 < NS; a2++) {
          const int ba = BASE((x + 1), a2);
          T qv[NS];
          ld_row(qv, qin + a2 * NS);
#pragma unroll
          for (int b2 = 0; b2 < NS; b2++) {
            const int pti = pair_type_lut(ba, BASE((y - 1), b2));
            const T st = pti < 6 ? en[EN_STK + P * 6 + pti] : (T)0;
            t1[b2] = fma(tx[a2] * qv[b2], st, t1[b2]);
          }
        }
        row_acc(r, t1, Ty1, (T)1);
#pragma unroll
        for (int b = 0; b < NS; b++)
          if (pair_type_lut(bxa, BASE(y, b)) != P) r[b] = (T)0;
      }
    } else if (post == 1) {
      const int M = p.Mp[x];
#pragma unroll
      for (int b = 0; b < NS; b++) r[b] = (a == b && a < M) ? (T)1 : (T)0;
    } else {
#pragma unroll
      for (int q = 0; q < 3; q++) {
        const T *A = q == 0 ? A0 : (q == 1 ? A1 : A2), *B = q == 0 ? B0 : (q == 1 ? B1 : B2);
        const T *C = q == 0 ? C0 : (q == 1 ? C1 : nullptr);
        const T f = q == 0 ? f0 : (q == 1 ? f1 : f2);
        if (!A) continue;
        if (C) {
          T t[NS];
          row_zero(t);
          row_mm(t, A, B, a, f);
          row_acc(r, t, C, (T)1);
        } else {
          row_mm(r, A, B, a, f);
        }
      }
      if (post == 2) {
        const int bxa = BASE(x, a);
#pragma unroll
        for (int b = 0; b < NS; b++) r[b] *= en[EN_TM + BASE(y, b) * 4 + bxa];
      }
    }
    st_row(O + (size_t)oslot * BLK + a * NS, r);
    if (scaled) lmax = fmax(lmax, row_absmax(r));
  }
  __syncthreads();

  // ---------------- phase B: HB, QB, QMpp, QM2pp, exterior Q5P per entry
  // HB: GHB consecutive threads per entry split the interior sizes and bulge parts
  {
    constexpr int GHB = LM::GHB;
    const int e = t / GHB, g = t % GHB, a = e / NS, b = e % NS;
    T v = 0;
    if (e < BLK && d >= 2) {
      const T tmo = en[EN_TM + BASE(x, a) * 4 + BASE(y, b)];
      // unrolled with the trip count as a predicate: the loads issue together
#pragma unroll
      for (int i = 0; i < (MAXLOOP - 1 + GHB - 1) / GHB; i++) {
        const int L = 2 + g + i * GHB;
        if (L <= Lmax) {
          const T yv = (L == 2) ? O[LO_XI * BLK + e] : O[(LO_YY + L - 3) * BLK + e];
          v = fma(wIn[L] * tmo, yv, v);
        }
      }
#pragma unroll
      for (int i = 0; i < (NLO_BU + GHB - 1) / GHB; i++) {
        const int j = g + i * GHB;
        if (j < NLO_BU) v += O[(LO_BU + j) * BLK + e];
      }
      if (g == 0) v = fma(sHL * clamp_p2<T>(-Ed) * tmo, O[LO_CH * BLK + e], v);
    }
#pragma unroll
    for (int o = 1; o < GHB; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (e < BLK && g == 0) {
      O[LO_HB * BLK + e] = v;
      lmax = fmax(lmax, fabs(v));
    }
  }
  if (t >= LM::QB0 && t < LM::QB0 + BLK) {
    const int e = t - LM::QB0, a = e / NS, b = e % NS;
    T qb = 0;
    if (d >= 4) {
      const int pto = pair_type(BASE(x, a), BASE(y, b));
      if (pto >= 0) {
        T v = O[LO_QBH * BLK + e];
#pragma unroll
        for (int j = 0; j < 6; j++) v += O[(LO_QBS + j) * BLK + e];
        v += en[EN_EA] * en[EN_EC] * (O[LO_QBM * BLK + e] + O[(LO_QBM + 1) * BLK + e]);
        qb = v * clamp_p2<T>(EAS(d - 2) - Ed);
      }
      O[LO_QB * BLK + e] = qb;
      const T s2v = S[SI_BIF * BLK + e] * clamp_p2<T>(EAS(d - 4) - Ed);
      const T mpp = en[EN_EC] * qb + s2v;
      O[LO_QM2PP * BLK + e] = s2v;
      O[LO_QMPP * BLK + e] = mpp;
      lmax = fmax(lmax, fmax(fabs(qb), fmax(fabs(mpp), fabs(s2v))));
    }
    if (x == 0) {
      T v;
      if (d == 0) {
        v = 0;
        lmax = fmax(lmax, (T)1);
      } else {
        v = qb + S[SI_BIFX * BLK + e] * clamp_p2<T>(EAS(d - 4) - Ed) + O[LO_Q5K * BLK + e];
        lmax = fmax(lmax, fabs(v));
      }
      O[LO_Q5P * BLK + e] = v;
    }
  }

  lmax = warp_max(lmax);
  if (lane == 0) smax[w] = lmax;
  __syncthreads();

  // ---------------- results to their tables, 16 bytes per thread and step
  {
    constexpr int CH16 = BLK * (int)sizeof(T) / 16;
    using V = typename Vec16<T>::type;
    for (int it = t; it < NCOPY * CH16; it += NTT) {
      const int k = it / CH16, q = it - k * CH16;
      T *dst = sDst[k];
      if (dst) reinterpret_cast<V *>(dst)[q] = reinterpret_cast<const V *>(O + (size_t)light_slot(k) * BLK)[q];
    }
  }
  // ---- diagonal maximum for the next exponent
  if (t == 0) {
    double m = 0;
    for (int k = 0; k < NTT / 32; k++) m = fmax(m, (double)smax[k]);
    atomic_max_pos(&p.dmax[d], m);
  }
}

template <typename T, int NTT, bool BT = false>
__global__ void __launch_bounds__(NTT, 1024 / NTT) k_in_light(DP<T> p, BifBuf<T> bb, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (BT) {
    const long long off = (long long)blockIdx.y * p.bstride;
    dp_shift(p, off);
    bb_shift(bb, off);
  }
  in_light_cell<T, NTT, BT>(p, bb, d, blockIdx.x, smem_raw);
}

template <typename T, int NTT = NT_IN>
constexpr size_t in_light_smem() {
  return (size_t)(SI_N + LO_N) * BLK * sizeof(T);
}

}  // namespace cf
