// cf_outside2.cuh -- outside pass (hand-written adjoint of the inside pass)
// as a CUDA graph from d = n-1 down to 0.  Per diagonal d:
//   k_out_light<T>(d)  every reverse statement that diagonals d-1..d-3 read,
//                      one CTA per cell, inputs staged into shared memory;
//   k_out_off<T>(d)    after the light kernel of d+4: the near bifurcation
//                      gathers of d
//                        hG[x][y]  += sum_{y'} hQM2pp[x][y'] (ec QB[y][y'])^T   (row gather)
//                        hQB[x][y] += sum_{x'} (ec G[x'][x])^T hQM2pp[x'][y]    (column gather)
//                        hGx[d]     = sum_{y'} hQ5P[y'] QB[d][y']^T             (exterior)
//                      and the side work (scatters) of diagonal d+4.
// Per band of OFD target diagonals (binary32): k_out_far<ROW> sums the far
// gather terms.  After the chain: k_out_tg (transfer gradients), then the
// marginals of cf_outside.cuh.
//
// Adjoint scaling and the statements themselves are those described in
// cf_outside.cuh: hA = (dZ/dA_true) 2^{E[d]} / Z, every reverse statement
// reuses its forward statement's power-of-two factor, gradients of the
// transfers accumulate in binary64 at residue-boundary positions.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"
#include "cf_inside2.cuh"

namespace cf {

// source of a staged slot for the cells x = xlo..xhi of a diagonal (src is
// the source of cell xlo; nullptr: no cell reads the slot)
template <typename T>
struct OSlot {
  const T *src;
  int xlo, xhi;
};

template <typename T>
struct OutBuf {
  T *hg;   // [BIFRING][n][36] row gathers (contribution to hG)
  T *hq;   // [BIFRING][n][36] column gathers (contribution to hQB)
  T *hgx;  // [BIFRING][36]    exterior gather hGx[d]
  float *far;  // [2 gathers][3 slots][n][OFD][36] far terms of a band (binary32; nullptr: none)
  float *fwh;      // [2][n] far-band rescale factors 2^{E[D] - s D - e0} and their inverses (binary32)
  int *fdev;       // [1] ceil(max over D of |E[D] - s D - e0|), written by k_out_far_factors
  OSlot<T> *otab;  // [n][SO_N] sources of the light kernel's staged slots per diagonal
  const T **stab;  // [n][SS_N] sources of the side work's staged slots for cell x = 0 (nullptr: not staged)
};

// Protein b's view of a batch (see DP::bstride).
template <typename T>
__device__ __forceinline__ void ob_shift(OutBuf<T> &o, long long off) {
  o.hg = bshift(o.hg, off);
  o.hq = bshift(o.hq, off);
  o.hgx = bshift(o.hgx, off);
  o.far = bshift(o.far, off);
  o.fwh = bshift(o.fwh, off);
  o.fdev = bshift(o.fdev, off);
  o.otab = bshift(o.otab, off);
  o.stab = bshift(o.stab, off);
}

// ---------------------------------------------------------------- far bands
// The gathers of a target cell on diagonal a read adjoints hQM2pp on
// diagonals a+4 .. n-1.  For the targets of a band [alo, alo + OFD), the terms
// whose adjoint lies on a diagonal >= c = alo + 2 OFD + 3 are "far": final a
// whole band earlier, they are summed for the band at once by k_out_far (a
// tiled product in which every loaded block serves up to 16 targets) while the
// reverse light chain is still OFD diagonals away; the near terms (adjoint
// diagonals a+4 .. c-1, at most 2 OFD + 1 per gather) stay in k_out_off.
// Far blocks are rescaled to a linear exponent with the chord s, e0 of E over
// diagonals 5 .. n-1: forward blocks by 2^{E[D] - s D - e0}, adjoint blocks by
// 2^{s D + e0 - E[D]}; every far term of a target on diagonal a is then
// relative to the common factor ec 2^{E[a] - s a}.  As for the inside far
// bands, the factor kernel records the largest deviation of E from the chord;
// past g_cf_far_dev_max no band of the pass is tiled (k_out_far returns at once)
// and the per-diagonal gathers take every term with its exact factor.
constexpr int OFD = 16;   // target diagonals per band
constexpr int OFTX = 16;  // target rows per tile
constexpr int OFKC = 4;   // summation indices staged per step
constexpr int OFKS = 64;  // summation indices per CTA slice
__host__ __device__ __forceinline__ int of_c(int alo) { return alo + 2 * OFD + 3; }
__host__ __device__ __forceinline__ bool of_band(int n, int alo) { return of_c(alo) <= n - 1; }

struct OChord {
  double s, e0;
};
__device__ __forceinline__ OChord of_chord(const int *E, int n) {
  const double e5 = (double)E[5], el = (double)E[n - 1];
  OChord r;
  r.s = (el - e5) / (double)(n - 6);
  r.e0 = e5 - 5.0 * r.s;
  return r;
}

__host__ __device__ __forceinline__ int out_nrow(int n, int x, int d) {  // hG terms y' = y+4..n-1
  int cnt = n - (x + d) - 4;
  return (d >= 5 && cnt > 0) ? (cnt + KCH - 1) / KCH : 0;
}
__host__ __device__ __forceinline__ int out_ncol(int x, int d) {  // hQB terms x' = 0..x-5
  int cnt = x - 4;
  return (d >= 4 && cnt > 0) ? (cnt + KCH - 1) / KCH : 0;
}
__host__ __device__ __forceinline__ int out_next(int n, int d) {  // hGx terms y' = d+4..n-1
  int cnt = n - d - 4;
  return (d >= 1 && cnt > 0) ? (cnt + KCH - 1) / KCH : 0;
}

// ---------------------------------------------------------------- K1'
// Binary64 over 48 nt: one 256-thread block per cell
// (last block: the exterior gather); the row- and column-gather chunks are
// dealt to the eight warps; lanes over the summation index.
template <typename T>
__device__ __forceinline__ void out_bif_cell(const DP<T> &p, const OutBuf<T> &ob, int d, int cb, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = p.n;
  const int *E = p.E;
  const int Ed = E[d];
  const int slot = d % BIFRING;
  const T ec = p.en[EN_EC];
  const bool ext = cb == n - d;
  T acc[BLK];
  zero_block(acc);
  int Ma, Mb;
  if (ext) {
    Ma = p.Mp[0];
    Mb = p.Mp[d];
    const int nq = out_next(n, d);
    for (int q = w; q < nq; q += 8) {
      const int yy = d + 4 + q * KCH + lane;
      if (yy <= n - 1) {
        T f = clamp_p2<T>(Ed + E[yy - d] - E[yy]);
        acc_mm_v<false, true>(acc, p.hQ5P + (size_t)yy * BLK, p.QB + cidx(n, d, yy) * BLK, Ma, p.Mp[yy], Mb, f);
      }
    }
  } else {
    // row chunks 0..nr-1 and column chunks nr..nr+nq-1 dealt round-robin to
    // all eight warps (a cell near either end has almost only one kind)
    const int x = cb, y = x + d;
    Ma = p.Mp[x];
    Mb = p.Mp[y];
    const int ylim = n - 1, xlo = 0;  // no far bands here: every term
    const int nr = ylim >= y + 4 ? (ylim - y - 4 + KCH) / KCH : 0;
    const int nq = x - 5 >= xlo ? (x - 5 - xlo + KCH) / KCH : 0;
    for (int q = w; q < nr; q += 8) {
      const int yy = y + 4 + q * KCH + lane;
      if (yy <= ylim) {
        T f = ec * clamp_p2<T>(Ed + E[yy - y] - E[yy - x]);
        acc_mm_v<false, true>(acc, p.hQM2pp + cidx(n, x, yy) * BLK, p.QB + cidx(n, y, yy) * BLK, Ma, p.Mp[yy], Mb, f);
      }
    }
    warp_reduce_block(acc, Ma, Mb);
    if (lane < 2) {
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e & 1) == lane) red[w][e] = acc[e];
    }
    zero_block(acc);
    const int q0 = ((w - nr) % 8 + 8) % 8;  // this warp owns the chunks nr + q with nr + q = w (mod 8)
    for (int q = q0; q < nq; q += 8) {
      const int xx = x - 5 - q * KCH - lane;
      if (xx >= xlo) {
        T f = ec * clamp_p2<T>(E[x - xx] + Ed - E[y - xx]);
        acc_mm_v<true, false>(acc, p.G + cidx(n, xx, x) * BLK, p.hQM2pp + cidx(n, xx, y) * BLK, Ma, p.Mp[xx], Mb, f);
      }
    }
    warp_reduce_block(acc, Ma, Mb);
    if (lane < 2) {
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e & 1) == lane) red[8 + w][e] = acc[e];
    }
  }
  if (ext) {
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
    T v = 0, u = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) v += red[k][e];
    if (ext) {
      ob.hgx[(size_t)slot * BLK + e] = v;
    } else {
#pragma unroll
      for (int k = 0; k < 8; k++) u += red[8 + k][e];
      const int x = cb;
      ob.hg[((size_t)slot * n + x) * BLK + e] = v;
      ob.hq[((size_t)slot * n + x) * BLK + e] = u;
    }
  }
}

// binary32: at most 2 OFD - 1 near terms per gather and cell (a banded
// diagonal keeps the adjoint diagonals below c; an unbanded one lies within
// 2 OFD + 3 of the last diagonal), so a pair of warps per cell (row gather,
// column gather) and four cells per 256-thread CTA; within a warp the two
// half-warps take rows 0..2 and 3..5 of the sum (bif_half_acc) and their 16
// lanes 16 terms.  Without far bands (a short protein, a batch) a warp takes
// every term of its gather, 16 per step.
// Exterior gather hGx[d] = sum_{yy >= d+4} hQ5P[yy] QB[d][yy]^T by all eight
// warps of the CTA, 16 terms per warp and step; the warps' sums are added in
// order.
template <typename T>
__device__ __forceinline__ void out_bif_ext_group(const DP<T> &p, const OutBuf<T> &ob, int d, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, half = lane >> 4, sl = lane & 15;
  const int n = p.n, Ed = p.E[d];
  const int Ma = p.Mp[0], Mb = p.Mp[d];
  T acc[NS / 2 * NS];
#pragma unroll
  for (int e = 0; e < NS / 2 * NS; e++) acc[e] = (T)0;
  const int nk = d >= 1 ? max(0, n - d - 4) : 0, nc = (nk + 15) / 16;
  for (int c = w; c < nc; c += 8) {
    const int yy = d + 4 + c * 16 + sl;
    if (yy <= n - 1) {
      const int e = Ed + p.E[yy - d] - p.E[yy];
      bif_half_acc<false, true, true>(acc, p.hQ5P + (size_t)yy * BLK, p.QB + cidx(n, d, yy) * BLK, clamp_p2<T>(e >> 1),
                                      half, Ma, p.Mp[yy], Mb, clamp_p2<T>(e - (e >> 1)));
    }
  }
  bif_half_reduce(acc, red[w], lane);
  __syncthreads();
  if (threadIdx.x < BLK) {
    T v = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) v += red[k][threadIdx.x];
    ob.hgx[(size_t)(d % BIFRING) * BLK + threadIdx.x] = v;
  }
}

template <typename T>
__device__ __forceinline__ void out_bif_group(const DP<T> &p, const OutBuf<T> &ob, int d, int cb0, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = w >> 1, half = lane >> 4, sl = lane & 15;
  const int n = p.n, ncell = n - d;
  const int *E = p.E;
  const int Ed = E[d];
  const int slot = d % BIFRING;
  const T ec = p.en[EN_EC];
  const int alo = d / OFD * OFD;
  const bool banded = ob.far != nullptr && of_band(n, alo) && __ldcg(ob.fdev) <= far_dev_max();
  if (cb0 + g < ncell) {
    const int x = cb0 + g, y = x + d;
    const int Ma = p.Mp[x], Mb = p.Mp[y];
    T acc[NS / 2 * NS];
#pragma unroll
    for (int e = 0; e < NS / 2 * NS; e++) acc[e] = (T)0;
    if ((w & 1) == 0) {
      const int ylim = banded ? min(n - 1, x + of_c(alo) - 1) : n - 1;
      const int nr = ylim >= y + 4 ? (ylim - y - 4 + 16) / 16 : 0;
      for (int q = 0; q < nr; q++) {
        const int yy = y + 4 + q * 16 + sl;
        if (yy <= ylim) {
          const int e = Ed + E[yy - y] - E[yy - x];
          const T *A = p.hQM2pp + cidx(n, x, yy) * BLK, *B = p.QB + cidx(n, y, yy) * BLK;
          if (banded)
            bif_half_acc<false, true>(acc, A, B, ec * clamp_p2<T>(e), half, Ma, p.Mp[yy], Mb);
          else  // every term, with factors as large as the exponents' bend: split between the operands
            bif_half_acc<false, true, true>(acc, A, B, ec * clamp_p2<T>(e >> 1), half, Ma, p.Mp[yy], Mb,
                                            clamp_p2<T>(e - (e >> 1)));
        }
      }
    } else {
      const int xlo = banded ? max(0, y - of_c(alo) + 1) : 0;
      const int nq = x - 5 >= xlo ? (x - 5 - xlo + 16) / 16 : 0;
      for (int q = 0; q < nq; q++) {
        const int xx = x - 5 - q * 16 - sl;
        if (xx >= xlo) {
          const int e = E[x - xx] + Ed - E[y - xx];
          const T *A = p.G + cidx(n, xx, x) * BLK, *B = p.hQM2pp + cidx(n, xx, y) * BLK;
          if (banded)
            bif_half_acc<true, false>(acc, A, B, ec * clamp_p2<T>(e), half, Ma, p.Mp[xx], Mb);
          else
            bif_half_acc<true, false, true>(acc, A, B, ec * clamp_p2<T>(e >> 1), half, Ma, p.Mp[xx], Mb,
                                            clamp_p2<T>(e - (e >> 1)));
        }
      }
    }
    bif_half_reduce(acc, red[w], lane);
  }
  // far terms are relative to ec 2^{E[d] - s d}: one factor per diagonal
  __shared__ double sfar;
  if (banded && threadIdx.x == 0) {
    const OChord ch = of_chord(E, n);
    sfar = (double)ec * exp2((double)Ed - ch.s * (double)d);
  }
  __syncthreads();
  if (threadIdx.x < 4 * BLK) {
    const int g2 = threadIdx.x / BLK, e = threadIdx.x % BLK, x = cb0 + g2;
    if (x < ncell) {
      T v = red[2 * g2][e], u = red[2 * g2 + 1][e];
      if (banded) {
        const double fac = sfar;
        const size_t fo = (((size_t)((alo / OFD) % 3) * n + x) * OFD + (d - alo)) * BLK + e;
        v += (T)(fac * (double)ob.far[fo]);
        u += (T)(fac * (double)ob.far[(size_t)3 * n * OFD * BLK + fo]);
      }
      ob.hg[((size_t)slot * n + x) * BLK + e] = v;
      ob.hq[((size_t)slot * n + x) * BLK + e] = u;
    }
  }
}


// ---------------------------------------------------------------- K0': far band
// Grid (tiles, slices), 256 threads: thread (tx, tj) owns the target
// (x, y) = (x0 + tx, x0 + tx + alo + tj).  ROW: the row gather
//   sum_{yy >= x + c} hQM2pp[x][yy] QB[y][yy]^T
// staged per summation index yy as the tile's 16 adjoint rows and its
// 31 QB rows; COL: the column gather
//   sum_{xx <= y - c} G[xx][x]^T hQM2pp[xx][y]
// staged per xx as 16 G columns and 31 adjoint columns.  Blocks arrive by TMA
// bulk copies into two alternating stages; each CTA takes a slice of OFKS
// summation indices and adds its sums into the band buffer (zeroed first).
// the rescale factors of every far band of the pass (one chord over diagonals
// 5..n-1), once per pass (binary64 exp2: the exponents reach the thousands),
// and the largest deviation from the chord; one CTA
__global__ void k_out_far_factors(DP<float> p, OutBuf<float> ob) {
  __shared__ int sdev;
  const OChord ch = of_chord(p.E, p.n);
  if (threadIdx.x == 0) sdev = 0;
  __syncthreads();
  int dev = 0;
  for (int D = threadIdx.x; D < p.n; D += blockDim.x) {
    const double z = (double)p.E[D] - ch.s * D - ch.e0;
    ob.fwh[D] = (float)exp2(z);
    ob.fwh[p.n + D] = (float)exp2(-z);
    if (D >= 5) dev = max(dev, (int)ceil(fabs(z)));
  }
  atomicMax(&sdev, dev);
  __syncthreads();
  if (threadIdx.x == 0) *ob.fdev = sdev;
}

template <bool ROW>
__global__ void __launch_bounds__(256) k_out_far(DP<float> p, OutBuf<float> ob, int alo) {
  constexpr int TY = OFTX + OFD - 1, STAGE = OFKC * (OFTX + TY) * BLK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *buf = (float *)smem_raw;          // [2][STAGE]: A [OFKC][OFTX][36], B [OFKC][TY][36]
  float *fw = buf + 2 * STAGE;             // [n] 2^{E[D] - s D - e0} (forward blocks)
  float *fh = fw + p.n;                    // [n] 2^{s D + e0 - E[D]} (adjoint blocks)
  __shared__ __align__(8) unsigned long long sbar[2];
  const int n = p.n, t = threadIdx.x, tx = t % OFTX, tj = t / OFTX;
  const int x0 = blockIdx.x * OFTX, x = x0 + tx, y = x + alo + tj, c = of_c(alo);
  // summation range of the tile and of this slice
  const int lo = ROW ? x0 + c : 0, hi = ROW ? n - 1 : x0 + OFTX - 1 + alo + OFD - 1 - c;
  const int kbeg = lo + blockIdx.y * OFKS, kend = min(hi, kbeg + OFKS - 1);
  if (kbeg > kend) return;
  if (__ldcg(ob.fdev) > far_dev_max()) return;  // every term is gathered per diagonal
  for (int D = t; D < n; D += 256) {
    fw[D] = __ldcg(ob.fwh + D);
    fh[D] = __ldcg(ob.fwh + n + D);
  }
  if (t == 0) {
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
  }
  __syncthreads();
  auto stage = [&](int k0, int bsel) {
    float *As = buf + (size_t)bsel * STAGE, *Bs = As + OFKC * OFTX * BLK;
    for (int q = t; q < OFKC * (OFTX + TY); q += 256) {
      const float *src = nullptr;
      float *dst;
      if (q < OFKC * OFTX) {
        const int kk = q / OFTX, r = q % OFTX, k = k0 + kk, xr = x0 + r;
        dst = As + (size_t)q * BLK;
        if (k <= kend && xr < n) {
          if (ROW) {
            if (k < n && k - xr >= 4) src = p.hQM2pp + cidx(n, xr, k) * BLK;
          } else if (xr - k >= 5) {
            src = p.G + cidx(n, k, xr) * BLK;
          }
        }
      } else {
        const int q2 = q - OFKC * OFTX, kk = q2 / TY, cq = q2 % TY, k = k0 + kk, yr = x0 + alo + cq;
        dst = Bs + (size_t)q2 * BLK;
        if (k <= kend && yr < n) {
          if (ROW) {
            if (k < n && k - yr >= 4) src = p.QB + cidx(n, yr, k) * BLK;
          } else if (yr - k >= 0) {
            src = p.hQM2pp + cidx(n, k, yr) * BLK;
          }
        }
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
  float acc[BLK];
  zero_block(acc);
  unsigned ph[2] = {0u, 0u};
  stage(kbeg, 0);
  int bsel = 0;
  for (int k0 = kbeg; k0 <= kend; k0 += OFKC, bsel ^= 1) {
    if (k0 + OFKC <= kend) stage(k0 + OFKC, bsel ^ 1);
    if (!__syncthreads_and(mbar_wait(&sbar[bsel], ph[bsel], p.err))) return;
    ph[bsel] ^= 1u;
    const float *As = buf + (size_t)bsel * STAGE, *Bs = As + OFKC * OFTX * BLK;
    if (live) {
#pragma unroll 1
      for (int kk = 0; kk < OFKC; kk++) {
        const int k = k0 + kk;
        if (k > kend) break;
        if (ROW ? (k < x + c) : (k > y - c)) continue;
        const float f = ROW ? fh[k - x] * fw[k - y] : fw[x - k] * fh[y - k];
        const float *A = As + ((size_t)kk * OFTX + tx) * BLK;
        const float *B = Bs + ((size_t)kk * TY + (tx + tj)) * BLK;
#pragma unroll
        for (int r = 0; r < NS; r++) {
          float av[NS];
          if (ROW) {
            ld_row(av, A + r * NS);  // row r of the adjoint block
          } else {
#pragma unroll
            for (int s2 = 0; s2 < NS; s2++) av[s2] = A[s2 * NS + r];  // column r of G
          }
#pragma unroll
          for (int s2 = 0; s2 < NS; s2++) av[s2] *= f;
          if (ROW) {
            // acc[r][b] += sum_s h[r][s] QB[b][s]
#pragma unroll
            for (int b = 0; b < NS; b++) {
              float bv[NS];
              ld_row(bv, B + b * NS);
              float v = acc[r * NS + b];
#pragma unroll
              for (int s2 = 0; s2 < NS; s2++) v = fmaf(av[s2], bv[s2], v);
              acc[r * NS + b] = v;
            }
          } else {
            // acc[r][b] += sum_s G[s][r] h[s][b]
#pragma unroll
            for (int s2 = 0; s2 < NS; s2++) {
              float bv[NS];
              ld_row(bv, B + s2 * NS);
#pragma unroll
              for (int b = 0; b < NS; b++) acc[r * NS + b] = fmaf(av[s2], bv[b], acc[r * NS + b]);
            }
          }
        }
      }
    }
    fence_proxy_async();
    __syncthreads();  // the next step's copies reuse this stage
  }
  if (live) {
    float *dst = ob.far + (((size_t)(ROW ? 0 : 3) + (alo / OFD) % 3) * n + x) * OFD * BLK + (size_t)tj * BLK;
#pragma unroll
    for (int r = 0; r < NS; r++) {
      float rr[NS];
#pragma unroll
      for (int b = 0; b < NS; b++) rr[b] = acc[r * NS + b];
      red_row(dst + r * NS, rr);
    }
  }
}

__host__ __device__ constexpr size_t out_far_smem(int n) {
  return ((size_t)2 * OFKC * (OFTX + OFTX + OFD - 1) * BLK + 2 * (size_t)n) * sizeof(float);
}
__host__ __device__ __forceinline__ int out_far_tiles(int n, int alo) { return (n - alo + OFTX - 1) / OFTX; }
__host__ __device__ __forceinline__ int out_far_slices(int n, int alo, bool row) {
  const int c = of_c(alo);
  const int span = row ? n - c : (n - alo + OFTX) + alo + OFD - c;  // widest tile's range
  return span > 0 ? (span + OFKS - 1) / OFKS : 0;
}

// ---------------------------------------------------------------- K2' staging
// Blocks the light kernel reads for cell (x, y): transfers around the cell,
// its own QB, adjoints of the cells that enclose it, the interior-loop adjoint
// ring of diagonal d+1, the chains of its three shortest interior scatters
// and the chains/adjoints of the longer intervals that use it as a bulge.
enum : int {
  SO_TXL = 0, SO_TY = 1, SO_XXL = 2, SO_XY = 6,
  SO_QB = 10, SO_GC = 11, SO_HXIE = 12, SO_H2UU = 13, SO_H2UP = 14, SO_H2PU = 15, SO_HMPU = 16, SO_HG1 = 17,
  SO_HCHL = 18, SO_HCH = 19, SO_GX = 20, SO_HQ5P = 21,
  SO_HYR = 22, SO_CHL = 50, SO_BC3U = 53, SO_BC5U = 83, SO_BH3U = 113, SO_BH5U = 143,
  SO_HGC = 173, SO_HQC = 174, SO_HGXC = 175, SO_HQ5U1 = 176, SO_HGX1 = 177,
  SO_N = 178
};
constexpr int NCHL_LIGHT = 3;  // interior scatters into hXI kept on the critical path: L = 3..5

template <typename T>
__device__ __forceinline__ const T *out_slot_src(const DP<T> &p, int s, int x, int y, int d) {
  const int n = p.n;
  const bool hasL = x >= 1, hasR = y <= n - 2, encl = hasL && hasR;
  if (s == SO_TXL) return hasL ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
  if (s == SO_TY) return hasR ? p.Tr + (size_t)y * BLK : nullptr;
  if (s < SO_XY) return hasL ? p.X + ((size_t)(x - 1) * 4 + (s - SO_XXL)) * BLK : nullptr;
  if (s < SO_QB) return hasR ? p.X + ((size_t)y * 4 + (s - SO_XY)) * BLK : nullptr;
  switch (s) {
    case SO_QB: return d >= 4 ? p.QB + cidx(n, x, y) * BLK : nullptr;
    case SO_GC: return encl ? p.hGc + cidx(n, x - 1, y + 1) * BLK : nullptr;
    case SO_HXIE: return encl ? p.hXI + cidx(n, x - 1, y + 1) * BLK : nullptr;
    case SO_H2UU: return hasL ? p.hQM2uu + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_H2UP: return hasL ? p.hQM2up + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_H2PU: return hasR ? p.hQM2pu + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HMPU: return hasR ? p.hQMpu + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HG1: return hasR ? p.hG + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HCHL: return hasL ? p.hCH + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_HCH: return d >= 1 ? p.hCH + cidx(n, x, y) * BLK : nullptr;
    case SO_GX: return (x >= 1 && d >= 4) ? p.Gx + (size_t)x * BLK : nullptr;
    case SO_HQ5P: return (x >= 1 && d >= 4) ? p.hQ5P + (size_t)y * BLK : nullptr;
    default: break;
  }
  const int Lmax = min(MAXLOOP, d - 4);
  if (s < SO_CHL) {  // ring hYY_{L+1}[x-1][y], L = 2..29 (block L-1)
    int L = s - SO_HYR + 2;
    bool ok = hasL && d >= 6 && L <= Lmax && L + 1 <= min(MAXLOOP, d + 1 - 4);
    return ok ? p.hYY + (((size_t)((d + 1) % YRING) * n + (x - 1)) * NYY + (L - 1)) * BLK : nullptr;
  }
  if (s < SO_BC3U) {  // CH[yl][y], yl = y - L + 2, L = 3..5
    int L = s - SO_CHL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.CH + cidx(n, yl, y) * BLK : nullptr;
  }
  // users of QB[x][y] as the inner pair of a bulge of a longer interval
  const int L = (s - SO_BC3U) % MAXLOOP + 1;
  const bool up3 = d >= 4 && y + L <= n - 1, up5 = d >= 4 && x - L >= 0;
  if (s < SO_BC5U) return up3 ? p.CH + cidx(n, y, y + L) * BLK : nullptr;
  if (s < SO_BH3U) return up5 ? p.CH + cidx(n, x - L, x) * BLK : nullptr;
  if (s < SO_BH5U) return up3 ? p.hHB + cidx(n, x, y + L) * BLK : nullptr;
  return up5 ? p.hHB + cidx(n, x - L, y) * BLK : nullptr;
}

// gather results of k_out_off and the exterior inputs of the cell (0, d)
template <typename T>
__device__ __forceinline__ const T *out_slot_src2(const DP<T> &p, const OutBuf<T> &ob, int s, int x, int d) {
  const int n = p.n, slot = d % BIFRING;
  if (s == SO_HGC) return out_nrow(n, x, d) > 0 ? ob.hg + ((size_t)slot * n + x) * BLK : nullptr;
  if (s == SO_HQC) return out_ncol(x, d) > 0 ? ob.hq + ((size_t)slot * n + x) * BLK : nullptr;
  if (x != 0) return nullptr;
  if (s == SO_HGXC) return out_next(n, d) > 0 ? ob.hgx + (size_t)slot * BLK : nullptr;
  if (s == SO_HQ5U1) return d + 1 < n ? p.hQ5U + (size_t)(d + 1) * BLK : nullptr;
  if (s == SO_HGX1) return d + 1 < n ? p.hGx + (size_t)(d + 1) * BLK : nullptr;
  return nullptr;
}

// The cells of diagonal d that read slot s form one range x = xlo..xhi (a
// neighbour on the left or right, a bulge that fits, the exterior cell), and
// the slot's source moves by a fixed stride per cell along the diagonal.
__host__ __device__ __forceinline__ void out_slot_range(int n, int s, int d, int &xlo, int &xhi) {
  xlo = 0;
  xhi = n - 1 - d;
  if (s == SO_TXL || (s >= SO_XXL && s < SO_XY) || s == SO_H2UU || s == SO_H2UP || s == SO_HCHL ||
      (s >= SO_HYR && s < SO_CHL) || s == SO_GX || s == SO_HQ5P)
    xlo = 1;  // a left neighbour
  if (s == SO_TY || (s >= SO_XY && s < SO_QB) || s == SO_H2PU || s == SO_HMPU || s == SO_HG1)
    xhi = n - 2 - d;  // a right neighbour
  if (s == SO_GC || s == SO_HXIE) {  // an enclosing pair
    xlo = 1;
    xhi = n - 2 - d;
  }
  if (s >= SO_BC3U && s < SO_HGC) {  // bulges of length L around the cell
    const int L = (s - SO_BC3U) % MAXLOOP + 1;
    if (s < SO_BC5U || (s >= SO_BH3U && s < SO_BH5U)) xhi = n - 1 - L - d;
    else xlo = L;
  }
  if (s == SO_HGC) xhi = n - d - 5;  // row gather terms
  if (s == SO_HQC) xlo = 5;          // column gather terms
  if (s >= SO_HGXC) xhi = 0;         // exterior
}
// Slots written by the light kernel of diagonal d+1: the adjoints of the
// neighbours (x-1, y) and (x, y+1), hQ5P[y] (for x = 1, y = d+1), the
// interior-loop adjoint ring of d+1, the L = 1 bulge adjoints hHB of
// (x, y+1) and (x-1, y), and the exterior adjoints of d+1.  Every other
// source is a forward table, an adjoint of a diagonal >= d+2, or a gather
// result of the off-chain launch of d (complete before the kernel starts);
// the light kernel of d+1 scatters into hXI of diagonals d+1..d-2 only, none
// of which this kernel reads.
__host__ __device__ __forceinline__ bool out_slot_late(int s) {
  return (s >= SO_H2UU && s <= SO_HCHL) || s == SO_HQ5P || (s >= SO_HYR && s < SO_CHL) || s == SO_BH3U ||
         s == SO_BH5U || s == SO_HQ5U1 || s == SO_HGX1;
}
__host__ __device__ __forceinline__ int out_slot_stride(int s) {
  if (s >= SO_XXL && s < SO_QB) return 4 * BLK;
  if (s >= SO_HYR && s < SO_CHL) return NYY * BLK;
  return BLK;
}

// per-diagonal table of slot sources (once per problem: table addresses only)
template <typename T>
__global__ void k_out_slot_tab(DP<T> p, OutBuf<T> ob) {
  const int d = blockIdx.x;
  for (int s = threadIdx.x; s < SO_N; s += blockDim.x) {
    OSlot<T> e;
    out_slot_range(p.n, s, d, e.xlo, e.xhi);
    e.src = nullptr;
    if (e.xlo <= e.xhi)
      e.src = s < SO_HGC ? out_slot_src(p, s, e.xlo, e.xlo + d, d) : out_slot_src2(p, ob, s, e.xlo, d);
    ob.otab[(size_t)d * SO_N + s] = e;
  }
}

// ---------------------------------------------------------------- K2'
// Thread mapping as in k_in_light: compact entries e = a*M_b + b, work lists
// split into NT/(M_x*M_y) groups.  Registers bounded so that six 256-thread
// CTAs fit an SM (their shared memory allows six as well).
// (BT: a batch of proteins, blockIdx.y the protein; compile-time, so that a
// single protein's kernels read their table pointers from the parameter bank.)
template <typename T, int NTT, bool BT = false>
__global__ void __launch_bounds__(NTT, 1536 / NTT) k_out_light(DP<T> p, OutBuf<T> ob, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long boff = BT ? (long long)blockIdx.y * p.bstride : 0;  // batch: protein b's slab
  if (BT) {
    dp_shift(p, boff);
    ob_shift(ob, boff);
  }
  T *S = (T *)smem_raw;            // [SO_N][36]
  T *HY = S + (size_t)SO_N * BLK;  // [29][36] interior partial-sum adjoints
  T *W = HY + NYY * BLK;           // work blocks
  T *hMPP = W, *hHB = W + BLK, *hQB = W + 2 * BLK;
  T *hM2 = W + 5 * BLK;            // uu, up, pu, pp
  T *hMPU = W + 9 * BLK, *hGG = W + 10 * BLK;
  T *hQ5Uo = W + 11 * BLK, *hQ5Po = W + 12 * BLK, *hGxo = W + 13 * BLK;  // exterior (cell (0, d))
  T *RED = W + 14 * BLK;           // [NTT]
  __shared__ double sps[NTT / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int x = blockIdx.x, y = x + d;
  // small per-cell context on chip: exponents around d, codon-state counts
  // around x and y, bases of x-1..x+1 and y-1..y+1, energy factors, the
  // exponents of the prefixes [0, x] and [0, y]; every value is loaded into a
  // register by its own thread, together with the thread's staged-slot entry,
  // so that all loads are in flight at once
  __shared__ int sE[96], sMx[72], sMy[72], sBx[3][NS], sBy[3][NS];
  __shared__ T sEn[EN_N];
  __shared__ int sExy[2];
  static_assert(NTT >= SO_N && NTT >= EN_N && NTT >= 96 + 6 * NS + 2, "one context value per thread and kind");
  int cE = 0, cMx = 0, cMy = 0, cB = 0;
  T cEn = 0;
  if (t < 96) {
    const int k = d - 47 + t;
    if (k >= 0 && k < n) cE = p.E[k];
  } else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    const int q = (side == 0 ? x : y) - 1 + r;
    if (q >= 0 && q < n) cB = p.base[q * NS + a];
  } else if (t < 98 + 6 * NS) {
    cE = p.E[t == 96 + 6 * NS ? x : y];
  }
  if (t < 72) {
    const int qx = x - 35 + t, qy = y - 35 + t;
    if (qx >= 0 && qx < n) cMx = p.Mp[qx];
    if (qy >= 0 && qy < n) cMy = p.Mp[qy];
  }
  if (t < EN_N) cEn = p.en[t];
  // loop-length weights: bulge users eBu(L) 2^{E[d]-E[d+L]}, interior
  // eIn(L) 2^{E[d-L+2]-E[d]}, from the thread's own loads (no extra phase)
  __shared__ T wBuU[MAXLOOP + 1], wIn[MAXLOOP + 1];
  T cwU = 0, cwI = 0;
  if (t <= MAXLOOP) {
    const int L = t, E0 = p.E[d];
    const T bu = p.en[EN_BU + L], in = p.en[EN_IN + L];
    if (L >= 1 && d + L < n) cwU = bu * clamp_p2<T>(E0 - p.E[d + L]);
    if (L >= 2 && d - L + 2 >= 0) cwI = in * clamp_p2<T>(p.E[d - L + 2] - E0);
  }
  OSlot<T> e{nullptr, 0, -1};
  if (t < SO_N) {
    e = ob.otab[(size_t)d * SO_N + t];
    e.src = bshift(e.src, boff);  // the table holds protein 0's addresses
  }
  // staging: one TMA bulk copy per input block, completing on a barrier at
  // which every thread arrives once with its copy's bytes
  __shared__ __align__(8) unsigned long long obar;
  if (t == 0) mbar_init(&obar, NTT);
  __syncthreads();
  {
    // slots written by the light kernel of d+1 (which may still be running:
    // programmatic launch) are issued after griddep_wait, the rest before it
    unsigned bytes = 0;
    const bool late = out_slot_late(t);
    auto issue = [&]() {
      if (e.src && x >= e.xlo && x <= e.xhi) {
        bytes = BLK * (unsigned)sizeof(T);
        bulk_g2s(S + (size_t)t * BLK, e.src + (size_t)(x - e.xlo) * out_slot_stride(t), bytes, &obar);
      }
    };
    if (!late) issue();
    griddep_wait();
    if (late) issue();
    griddep_launch_dependents();  // the next diagonal's kernel may start its own early part
    mbar_arrive_expect(&obar, bytes);
  }
  if (t < 96) sE[t] = cE;
  else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    if (side == 0) sBx[r][a] = cB;
    else sBy[r][a] = cB;
  } else if (t < 98 + 6 * NS) {
    sExy[t - 96 - 6 * NS] = cE;
  }
  if (t < 72) {
    sMx[t] = cMx;
    sMy[t] = cMy;
  }
  if (t < EN_N) sEn[t] = cEn;
  if (t <= MAXLOOP) {
    wBuU[t] = cwU;
    wIn[t] = cwI;
  }
  if (!__syncthreads_and(mbar_wait(&obar, 0, p.err))) return;
  const T *en = sEn;
  const int Ed = sE[47];  // E[d], staged with its neighbours
  const int Mx = MP(x), My = MP(y), MM = Mx * My;
  const int M1 = (d >= 1) ? MP(x + 1) : 0, Mv = (d >= 1) ? MP(y - 1) : 0;
  const size_t c = cidx(n, x, y);
  const T eb = en[EN_EB], ec = en[EN_EC], sml = en[EN_EA] * en[EN_EC];
  const bool hasL = x >= 1, hasR = y <= n - 2, encl = hasL && hasR;
  const int Mxl = hasL ? MP(x - 1) : 0, Myr = hasR ? MP(y + 1) : 0;
  const int M0 = MP(0);
  const T F1u = (d + 1 < n) ? clamp_p2<T>(Ed - EAS(d + 1)) : (T)0;
  const T F2u = (d + 2 < n) ? clamp_p2<T>(Ed - EAS(d + 2)) : (T)0;
  const T *gc = S + SO_GC * BLK;
  const T *Xxl = S + SO_XXL * BLK, *Xy = S + SO_XY * BLK;

  // ---------------- A: QM2 adjoints with unpaired ends; exterior prefix adjoint
  if (d >= 10 && (t < MM || (t >= 64 && t < 64 + MM) || (t >= 128 && t < 128 + MM))) {
    const int g = t / 64, e = t - 64 * g, a = e / My, b = e % My, pe = a * NS + b;
    const bool mlu = encl && d + 2 >= 11;
    T v = 0;
    if (g == 0) {  // QM2uu
      if (mlu) v = sml * F2u * s3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
      if (hasL) v += eb * F1u * s2<true, false>(Xxl + XUU * BLK, S + SO_H2UU * BLK, a, b, Mxl);
    } else if (g == 1) {  // QM2up
      if (mlu) v = sml * F2u * s3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
      if (hasL) v += eb * F1u * s2<true, false>(Xxl + XUU * BLK, S + SO_H2UP * BLK, a, b, Mxl);
    } else {  // QM2pu
      if (mlu) v = sml * F2u * s3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
      if (hasL) v += eb * F1u * s2<true, false>(Xxl + XUP * BLK, S + SO_H2UU * BLK, a, b, Mxl);
      if (hasR) v += eb * F1u * s2<false, true>(S + SO_H2PU * BLK, Xy + XUU * BLK, a, b, Myr);
    }
    hM2[g * BLK + pe] = v;
    T *dst = g == 0 ? p.hQM2uu : (g == 1 ? p.hQM2up : p.hQM2pu);
    dst[c * BLK + pe] = v;
  }
  if (x == 0 && t >= 192 && t < 192 + M0 * My) {
    const int e = t - 192, a = e / My, b = e % My, pe = a * NS + b;
    T hu, hp;
    if (d == n - 1) {
      hu = hp = (T)(p.u0[a] / *p.Zm);
    } else {
      const T *hu1 = S + SO_HQ5U1 * BLK, *hg1 = S + SO_HGX1 * BLK;
      const int Mn = MP(d + 1);
      hu = F1u * (s2<false, true>(hu1, Xy + XUU * BLK, a, b, Mn) + s2<false, true>(hg1, Xy + XUP * BLK, a, b, Mn));
      hp = F1u * (s2<false, true>(hu1, Xy + XPU * BLK, a, b, Mn) + s2<false, true>(hg1, Xy + XPP * BLK, a, b, Mn));
    }
    p.hQ5U[(size_t)d * BLK + pe] = hu;
    p.hQ5P[(size_t)d * BLK + pe] = hp;
    hQ5Uo[pe] = hu;
    hQ5Po[pe] = hp;
  }
  __syncthreads();

  // ---------------- B: hGx (exterior), hG, hQMpu, hQMpp
  if (x == 0 && d >= 1 && t < M0 * My) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    const T v = out_next(n, d) > 0 ? S[SO_HGXC * BLK + pe] : (T)0;
    p.hGx[(size_t)d * BLK + pe] = v;
    hGxo[pe] = v;
  } else if (t >= 64 && t < 64 + MM && d >= 5) {
    const int e = t - 64, pe = (e / My) * NS + (e % My);
    const T v = out_nrow(n, x, d) > 0 ? S[SO_HGC * BLK + pe] : (T)0;
    hGG[pe] = v;
    p.hG[c * BLK + pe] = v;
  } else if (t >= 128 && t < 128 + MM && d >= 5) {
    const int e = t - 128, a = e / My, b = e % My, pe = a * NS + b;
    T v = 0;
    if (hasR)
      v = F1u * (eb * s2<false, true>(S + SO_HMPU * BLK, Xy + XUU * BLK, a, b, Myr) +
                 s2<false, true>(S + SO_HG1 * BLK, Xy + XUP * BLK, a, b, Myr));
    hMPU[pe] = v;
    p.hQMpu[c * BLK + pe] = v;
  } else if (t >= 192 && t < 192 + MM && d >= 4) {
    const int e = t - 192, a = e / My, b = e % My, pe = a * NS + b;
    T v = 0;
    if (hasR)
      v = F1u * (eb * s2<false, true>(S + SO_HMPU * BLK, Xy + XPU * BLK, a, b, Myr) +
                 s2<false, true>(S + SO_HG1 * BLK, Xy + XPP * BLK, a, b, Myr));
    hMPP[pe] = v;
    p.hQMpp[c * BLK + pe] = v;
  }
  __syncthreads();

  // ---------------- C: hQM2pp (0..), hHB (64..)
  if (t < MM && d >= 4) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    T v = 0;
    if (d >= 9) {
      v = hMPP[pe];
      if (encl && d + 2 >= 11) v += sml * F2u * s3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
      if (hasR && d + 1 >= 10) v += eb * F1u * s2<false, true>(S + SO_H2PU * BLK, Xy + XPU * BLK, a, b, Myr);
      if (hasL && d + 1 >= 10) v += eb * F1u * s2<true, false>(Xxl + XUP * BLK, S + SO_H2UP * BLK, a, b, Mxl);
    }
    hM2[3 * BLK + pe] = v;
    p.hQM2pp[c * BLK + pe] = v;
  } else if (t >= 64 && t < 64 + MM && d >= 2) {
    const int e = t - 64, a = e / My, b = e % My, pe = a * NS + b;
    T v = 0;
    if (encl) v = F2u * s3<true, false, true>(S + SO_TXL * BLK, gc, S + SO_TY * BLK, a, b, Mxl, Myr);
    hHB[pe] = v;
    p.hHB[c * BLK + pe] = v;
  }
  __syncthreads();

  // ---------------- D: hQB as a sum over its users (groups of threads)
  const int GR = min(NTT / MM, 32);  // groups for the reductions below
  if (d >= 4) {
    const int G = GR, g = t / MM, e = t % MM;
    if (g < G) {
      const int a = e / My, b = e % My, pe = a * NS + b;
      T v = 0;
      // terms: bulge users (2 per length), the own-cell terms, then the
      // enclosing pair's interior (XI) and stack terms split by the outer
      // state of x-1 so that the groups stay balanced
      constexpr int KXI = 2 * MAXLOOP + 1, KST = KXI + NS, KEND = KST + NS;
      for (int k = g; k < KEND; k += G) {
        if (k < 2 * MAXLOOP) {
          const int L = k / 2 + 1;
          if ((k & 1) == 0) {
            if (y + L > n - 1) continue;
            const T f = wBuU[L];
            v += f * s2<false, true>(S + (SO_BH3U + L - 1) * BLK, S + (SO_BC3U + L - 1) * BLK, a, b, MP(y + L));
          } else {
            if (x - L < 0) continue;
            const T f = wBuU[L];
            v += f * s2<true, false>(S + (SO_BC5U + L - 1) * BLK, S + (SO_BH5U + L - 1) * BLK, a, b, MP(x - L));
          }
        } else if (k == 2 * MAXLOOP) {
          v += ec * hMPP[pe];
          if (out_ncol(x, d) > 0) v += S[SO_HQC * BLK + pe];
          if (x == 0) v += hQ5Po[pe];  // computed above in this kernel
          else v += clamp_p2<T>(sExy[0] + Ed - sExy[1]) * s2<true, false>(S + SO_GX * BLK, S + SO_HQ5P * BLK, a, b, M0);
        } else if (k < KST) {
          // XI[x-1][y+1] = F (T_{x-1} QB T_y) o tm, outer state wv of x-1
          const int wv = k - KXI;
          if (!encl || wv >= Mxl) continue;
          const T *Txl = S + SO_TXL * BLK, *Ty = S + SO_TY * BLK, *hxi1 = S + SO_HXIE * BLK;
          const T tl = Txl[wv * NS + a];
          if (tl == (T)0) continue;
          const int bw = BASE((x - 1), wv);
          T s2v = 0;
#pragma unroll
          for (int z = 0; z < NS; z++)
            if (z < Myr) s2v += hxi1[wv * NS + z] * en[EN_TM + BASE((y + 1), z) * 4 + bw] * Ty[b * NS + z];
          v += F2u * tl * s2v;
        } else {
          // stack of the enclosing pair (x-1, y+1), outer state a1 of x-1
          const int a1 = k - KST;
          if (!encl || a1 >= Mxl) continue;
          const int pti = pair_type(BASE(x, a), BASE(y, b));
          if (pti < 0) continue;
          const T *Txl = S + SO_TXL * BLK, *Ty = S + SO_TY * BLK;
          const T tl = Txl[a1 * NS + a];
          if (tl == (T)0) continue;
          const int ba = BASE((x - 1), a1);
          T s2v = 0;
#pragma unroll
          for (int b1 = 0; b1 < NS; b1++) {
            const int pto = b1 < Myr ? pair_type(ba, BASE((y + 1), b1)) : -1;
            if (pto >= 0) s2v += gc[a1 * NS + b1] * en[EN_STK + pto * 6 + pti] * Ty[b * NS + b1];
          }
          v += F2u * tl * s2v;
        }
      }
      RED[t] = v;
    }
  }
  __syncthreads();
  double psum = 0;
  if (d >= 4 && t < MM) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    T v = 0;
    for (int g = 0; g < GR; g++) v += RED[g * MM + t];
    p.hQB[c * BLK + pe] = v;
    const T gq = pair_type(BASE(x, a), BASE(y, b)) >= 0 ? v : (T)0;
    hQB[pe] = gq;
    p.hGc[c * BLK + pe] = gq;
    psum = (double)S[SO_QB * BLK + pe] * (double)v;
  }
  // ---------------- E: interior partial-sum adjoints over (L, entry)
  if (d >= 6) {
    const int Lmax = min(MAXLOOP, d - 4);
    const int nitem = (Lmax - 1) * MM;
    const T *Txl = S + SO_TXL * BLK;
    for (int it = t; it < nitem; it += NTT) {
      const int L = it / MM + 2, e = it % MM, a = e / My, b = e % My, pe = a * NS + b;
      T v = wIn[L] * en[EN_TM + BASE(x, a) * 4 + BASE(y, b)] * hHB[pe];
      if (hasL && L + 1 <= min(MAXLOOP, d + 1 - 4)) v += s2<true, false>(Txl, S + (SO_HYR + L - 2) * BLK, a, b, Mxl);
      HY[(L - 2) * BLK + pe] = v;
      p.hYY[(((size_t)(d % YRING) * n + x) * NYY + (L - 2)) * BLK + pe] = v;
    }
  }
  psum = warp_sum(psum);
  if (lane == 0) sps[w] = psum;
  __syncthreads();

  // ---------------- F: interior scatters into hXI that this and the next three
  // diagonals read (L = 2: the cell's own XI; L = 3..5); every other scatter
  // runs in the side work of k_out_off and the transfer gradients in k_out_tg,
  // off the critical path
  if (d >= 6) {
    const int Lmax = min(MAXLOOP, d - 4);
    for (int it = t; it < (1 + NCHL_LIGHT) * BLK; it += NTT) {
      const int L = it / BLK + 2, e = it % BLK, yl = y - L + 2;
      if (L > Lmax || yl - x < 6) continue;
      const int Ml = MP(yl);
      if (e >= Mx * Ml) continue;
      const int r = e / Ml, s2i = e % Ml;
      const T *hy = HY + (L - 2) * BLK;
      const T v = (L == 2) ? hy[r * NS + s2i] : s2<false, true>(hy, S + (SO_CHL + L - 3) * BLK, r, s2i, My);
      if (v != (T)0) atomicAdd(p.hXI + cidx(n, x, yl) * BLK + r * NS + s2i, v);
    }
  }
  // final chain adjoint of this cell (its scatters all came from longer intervals)
  if (d >= 1 && t >= 192 && t < 192 + MM) {
    const int e = t - 192, a = e / My, b = e % My, pe = a * NS + b;
    T v = S[SO_HCH * BLK + pe];
    if (d >= 2) v += p.eHL[d + 1] * clamp_p2<T>(-Ed) * en[EN_TM + BASE(x, a) * 4 + BASE(y, b)] * hHB[pe];
    if (hasL) v += s2<true, false>(S + SO_TXL * BLK, S + SO_HCHL * BLK, a, b, Mxl);
    p.hCH[c * BLK + pe] = v;
  }
  __syncthreads();
  if (t == 0 && d >= 4) {
    double ps = 0;
    for (int k = 0; k < NTT / 32; k++) ps += sps[k];
    p.P[(size_t)x * n + y] = (float)ps;
    p.P[(size_t)y * n + x] = (float)ps;
  }
}

// ---------------------------------------------------------------- K3'
// Side work of diagonal d (side_cell, in the k_out_off launch of d-4): the
// parts of the adjoint of diagonal d that no diagonal d-1..d-3 reads, run
// beside the light chain: the bulge scatters into the chain adjoints of
// diagonals L <= d-4, the interior scatters into hXI of diagonals <= d-4 and
// into the chain adjoints of diagonals <= 28, and the ring term of the
// transfer gradients.  It starts after the light kernel of d and must end
// before the light kernel of d-4, the first reader of what it writes; the
// interior-loop adjoint ring keeps YRING >= 5 diagonals so that its slot of d
// is intact.
enum : int {
  SS_TX = 0, SS_TY1 = 1, SS_XX = 2, SS_XY1 = 6, SS_QBI = 10, SS_HBI = 11, SS_CHN = 12, SS_Q2I = 13,
  SS_ML = 17, SS_MR = 21, SS_Q5UM = 25, SS_Q5PM = 26,
  SS_HGC = 27, SS_HHB = 28, SS_HCH = 29, SS_HXI = 30, SS_HM2 = 31, SS_HMPU = 35, SS_HG = 36,
  SS_HQ5U = 37, SS_HGX = 38,
  SS_HY = 39, SS_YYP = 68, SS_XIL = 96, SS_CHL = 124, SS_BQ3 = 152, SS_BQ5 = 182,
  SS_N = 212
};
static_assert(YRING >= 5, "the side work reads the ring slot of its diagonal until the light kernel of d-4");
constexpr int NT3 = 256;

template <typename T>
__device__ __forceinline__ const T *side_slot_src(const DP<T> &p, int s, int x, int y, int d) {
  const int n = p.n;
  const size_t c = cidx(n, x, y);
  if (s == SS_TX) return p.Tr + (size_t)x * BLK;
  if (s == SS_TY1) return d >= 1 ? p.Tr + (size_t)(y - 1) * BLK : nullptr;
  if (s < SS_XY1) return p.X + ((size_t)x * 4 + (s - SS_XX)) * BLK;
  if (s < SS_QBI) return d >= 1 ? p.X + ((size_t)(y - 1) * 4 + (s - SS_XY1)) * BLK : nullptr;
  if (s == SS_QBI) return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s == SS_HBI) return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s == SS_CHN) return d >= 1 ? p.CH + cidx(n, x + 1, y) * BLK : nullptr;
  if (s < SS_ML) {
    if (d < 11) return nullptr;
    const T *t[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
    return t[s - SS_Q2I] + cidx(n, x + 1, y - 1) * BLK;
  }
  if (s < SS_MR) {
    if (d < 5) return nullptr;
    const T *t[4] = {p.QMpp, p.QMpu, p.QM2pp, p.QM2pu};
    return t[s - SS_ML] + cidx(n, x, y - 1) * BLK;
  }
  if (s < SS_Q5UM) {
    if (d < 10) return nullptr;
    const T *t[4] = {p.QM2up, p.QM2pp, p.QM2uu, p.QM2pu};
    return t[s - SS_MR] + cidx(n, x + 1, y) * BLK;
  }
  switch (s) {
    case SS_Q5UM: return (x == 0 && d >= 1) ? p.Q5U + (size_t)(d - 1) * BLK : nullptr;
    case SS_Q5PM: return (x == 0 && d >= 1) ? p.Q5P + (size_t)(d - 1) * BLK : nullptr;
    case SS_HGC: return d >= 4 ? p.hGc + c * BLK : nullptr;
    case SS_HHB: return d >= 2 ? p.hHB + c * BLK : nullptr;
    case SS_HCH: return d >= 1 ? p.hCH + c * BLK : nullptr;
    case SS_HXI: return d >= 6 ? p.hXI + c * BLK : nullptr;
    case SS_HM2: return d >= 10 ? p.hQM2uu + c * BLK : nullptr;
    case SS_HM2 + 1: return d >= 10 ? p.hQM2up + c * BLK : nullptr;
    case SS_HM2 + 2: return d >= 10 ? p.hQM2pu + c * BLK : nullptr;
    case SS_HM2 + 3: return d >= 4 ? p.hQM2pp + c * BLK : nullptr;
    case SS_HMPU: return d >= 5 ? p.hQMpu + c * BLK : nullptr;
    case SS_HG: return d >= 5 ? p.hG + c * BLK : nullptr;
    case SS_HQ5U: return x == 0 ? p.hQ5U + (size_t)d * BLK : nullptr;
    case SS_HGX: return (x == 0 && d >= 1) ? p.hGx + (size_t)d * BLK : nullptr;
    default: break;
  }
  const int Lmax = min(MAXLOOP, d - 4);
  if (s < SS_YYP) {  // this diagonal's interior-loop adjoints hYY_L, L = 2..30
    const int L = s - SS_HY + 2;
    return (d >= 6 && L <= Lmax) ? p.hYY + (((size_t)(d % YRING) * n + x) * NYY + (L - 2)) * BLK : nullptr;
  }
  if (s < SS_XIL) {  // YY_{L-1}[x+1][y], L = 3..30
    const int L = s - SS_YYP + 3;
    return (d >= 6 && L <= Lmax) ? yy_out(p, x + 1, d - 1) + (size_t)(L - 3) * BLK : nullptr;
  }
  if (s < SS_BQ3) {  // XI[x][yl] and CH[yl][y], yl = y - L + 2, L = 3..30
    const int L = (s - SS_XIL) % 28 + 3, yl = y - L + 2;
    if (!(d >= 6 && L <= Lmax && yl - x >= 6)) return nullptr;
    return s < SS_CHL ? p.XI + cidx(n, x, yl) * BLK : p.CH + cidx(n, yl, y) * BLK;
  }
  const int L = (s - SS_BQ3) % MAXLOOP + 1;
  if (d - L < 4) return nullptr;
  return s < SS_BQ5 ? p.QB + cidx(n, x, y - L) * BLK : p.QB + cidx(n, x + L, y) * BLK;
}

struct SideCtx {
  int sE[96], sMx[72], sMy[72], sBx[3][NS], sBy[3][NS];
};

// slots read only by the transfer gradients (cells at a residue boundary)
__device__ __forceinline__ bool side_slot_tg(int s) {
  return s < SS_HHB || s == SS_HCH || (s >= SS_HXI && s < SS_HY) || (s >= SS_YYP && s < SS_XIL);
}

// stride of a side slot's source per cell along a diagonal
__host__ __device__ __forceinline__ int side_slot_stride(int s) {
  if (s >= SS_XX && s < SS_QBI) return 4 * BLK;
  if (s >= SS_HY && s < SS_XIL) return NYY * BLK;
  return BLK;
}

// per-diagonal table of the side work's slot sources for cell x = 0; the
// slots of the exterior cell and those read only by the transfer gradients
// (summed after the pass) are not staged, except the partial sums
// YY_{L-1}[x+1][y] of the ring term
template <typename T>
__global__ void k_side_slot_tab(DP<T> p, OutBuf<T> ob) {
  const int d = blockIdx.x;
  for (int s = threadIdx.x; s < SS_N; s += blockDim.x) {
    const bool staged = !side_slot_tg(s) || (s >= SS_YYP && s < SS_XIL);
    ob.stab[(size_t)d * SS_N + s] = staged && d >= 5 ? side_slot_src(p, s, 0, d, d) : nullptr;
  }
}

template <typename T>
__device__ __forceinline__ bool side_cell(const DP<T> &p, const OutBuf<T> &ob, int d, int x, T *S, SideCtx &cx, T *sEn, T *wBu,
                                          unsigned long long *sbar, unsigned phase, long long boff) {
  int *sE = cx.sE, *sMx = cx.sMx, *sMy = cx.sMy;
  int (*sBx)[NS] = cx.sBx, (*sBy)[NS] = cx.sBy;
  const int t = threadIdx.x;
  const int n = p.n;
  const int y = x + d;
  const bool bx = p.bnd[x] != 0;
  if (d < 5) return true;  // no scatter below d = 5
  // context values, one load per thread, in flight while the copies are issued
  int cE = 0, cMx = 0, cMy = 0, cB = 0;
  T cEn = 0;
  if (t < 96) {
    const int k = d - 47 + t;
    if (k >= 0 && k < n) cE = p.E[k];
  }
  if (t < 72) {
    const int qx = x - 35 + t, qy = y - 35 + t;
    if (qx >= 0 && qx < n) cMx = p.Mp[qx];
    if (qy >= 0 && qy < n) cMy = p.Mp[qy];
  }
  if (t >= 96 && t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    const int q = (side == 0 ? x : y) - 1 + r;
    if (q >= 0 && q < n) cB = p.base[q * NS + a];
  }
  if (t < EN_N) cEn = p.en[t];
  static_assert(NT3 >= SS_N, "one staged slot per thread");
  const T *src0 = t < SS_N ? bshift(ob.stab[(size_t)d * SS_N + t], boff) : nullptr;
  // staging: one TMA bulk copy per input block, the interior-loop adjoints
  // hYY_L (L = 2..Lmax) and partial sums YY_{L-1}[x+1][y] (L = 3..Lmax) as one
  // copy each; the partial sums only for a boundary at x (the ring term of the
  // transfer gradient T_x)
  const bool ytg = bx && d >= 6;
  const int Lmax = min(MAXLOOP, d - 4);
  // every thread arrives once at the barrier with the bytes of its copy
  unsigned nbytes = 0;
  {
    const int s = t;
    const bool skip = src0 == nullptr || (!ytg && s >= SS_YYP && s < SS_XIL) ||
                      (d >= 6 && s > SS_HY && s < SS_YYP && s - SS_HY + 2 <= Lmax) ||  // part of the hYY run
                      (d >= 6 && s > SS_YYP && s < SS_XIL && s - SS_YYP + 3 <= Lmax);   // part of the YY run
    if (!skip) {
      const T *src = src0 + (size_t)x * side_slot_stride(s);
      unsigned nb = 1;
      if (s == SS_HY) nb = (unsigned)(Lmax - 1);
      else if (s == SS_YYP) nb = (unsigned)(Lmax - 2);
      nbytes = nb * BLK * (unsigned)sizeof(T);
      bulk_g2s(S + (size_t)s * BLK, src, nbytes, sbar);
    }
  }
  mbar_arrive_expect(sbar, nbytes);
  if (t < 96) sE[t] = cE;
  if (t < 72) {
    sMx[t] = cMx;
    sMy[t] = cMy;
  }
  if (t >= 96 && t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    if (side == 0) sBx[r][a] = cB;
    else sBy[r][a] = cB;
  }
  if (t < EN_N) sEn[t] = cEn;
  if (!__syncthreads_and(mbar_wait(sbar, phase, p.err))) return false;
  const T *en = sEn;
  const int Ed = sE[47];  // E[d], staged with its neighbours
  const int Mx = MP(x), My = MP(y), M1 = MP(x + 1);
  if (t <= MAXLOOP) {
    const int L = t;
    wBu[L] = (L >= 1 && d - L >= 4) ? en[EN_BU + L] * clamp_p2<T>(EAS(d - L) - Ed) : (T)0;
  }
  __syncthreads();
  const T *hHB = S + SS_HHB * BLK, *HY = S + SS_HY * BLK;

  T *YtP = S + (size_t)SS_N * BLK;  // [6][36] partial sums of the ring term of T_x
  if (ytg && t >= NT3 - 6 * BLK) {
    const int i = t - (NT3 - 6 * BLK), j = i / BLK, e = i % BLK, a = e / NS, u = e % NS;
    T v = 0;
    if (a < Mx && u < M1)
      for (int L = 3 + j; L <= Lmax; L += 6) v += s2<false, true>(HY + (L - 2) * BLK, S + (SS_YYP + L - 3) * BLK, a, u, My);
    YtP[i] = v;
  }

  // ---------------- bulge and interior scatters, one block row per thread and step
  //   bulge 3' (L = 1..30):  hCH[y-L][y] += wBu(L) QB[x][y-L]^T hHB
  //   bulge 5' (L = 1..30):  hCH[x][x+L] += wBu(L) hHB QB[x+L][y]^T
  //   interior (L = 3..Lmax, yl = y-L+2, yl-x >= 6):
  //     hCH[yl][y] += XI[x][yl]^T hYY_L,  hXI[x][yl] += hYY_L CH[yl][y]^T (L >= 6:
  //     the light kernel takes L = 3..5)
  // Blocks are zero-padded, so each row runs over the full padded size.
  {
    const int Lmax = min(MAXLOOP, d - 4);
    constexpr int NPROD = 4 * MAXLOOP;
    for (int rt = t; rt < NS * NPROD; rt += NT3) {
      const int q = rt / NS, a = rt - q * NS;
      const int kind = q / MAXLOOP, L = q % MAXLOOP + 1;
      T r[NS];
      row_zero(r);
      T *dst = nullptr;
      if (kind == 0) {
        if (d >= 5 && d - L >= 4) {
          row_tmm(r, S + (SS_BQ3 + L - 1) * BLK, hHB, a, wBu[L]);
          dst = p.hCH + cidx(n, y - L, y) * BLK;
        }
      } else if (kind == 1) {
        if (d >= 5 && d - L >= 4) {
          row_mmt(r, hHB, S + (SS_BQ5 + L - 1) * BLK, a, wBu[L]);
          dst = p.hCH + cidx(n, x, x + L) * BLK;
        }
      } else if (d >= 6 && L >= 3 && L <= Lmax && y - L + 2 - x >= 6) {
        const int yl = y - L + 2;
        const T *hy = HY + (L - 2) * BLK;
        if (kind == 2) {
          row_tmm(r, S + (SS_XIL + L - 3) * BLK, hy, a, (T)1);
          dst = p.hCH + cidx(n, yl, y) * BLK;
        } else if (L >= 3 + NCHL_LIGHT) {
          row_mmt(r, hy, S + (SS_CHL + L - 3) * BLK, a, (T)1);
          dst = p.hXI + cidx(n, x, yl) * BLK;
        }
      }
      if (dst) red_row(dst + a * NS, r);
    }
  }

  // ---------------- the one transfer-gradient term that reads the ring of
  // interior-loop adjoints: sum_L hYY_L YY_{L-1}[x+1][y]^T for T_x (the rest
  // of the transfer gradients is summed after the pass by k_out_tg); six
  // partial sums over L = 3+j, 9+j, ... added in order
  if (ytg) {
    __syncthreads();
    if (t < BLK) {
      const int a = t / NS, u = t % NS;
      if (a < Mx && u < M1) {
        T v = 0;
#pragma unroll
        for (int j = 0; j < 6; j++) v += YtP[j * BLK + t];
        p.tgY[cidx(n, x, y) * BLK + t] = v;
      }
    }
  }
  return true;
}


// The off-chain work that the light kernel of diagonal d waits for, as one
// launch: CTAs 0..nbif-1 take the bifurcation gathers of diagonal d (GRP, with
// far bands: four cells per CTA, then the exterior, at 64 registers so that
// the CTAs leave room for the light kernels; else one cell per CTA), the
// others the side work of the cells of diagonal d+4.  Both parts start after
// the light kernel of d+4.  GRP is the form of binary32 and of short binary64
// proteins (binary64: two CTAs per SM, at four it spilled 1.8 KB a thread);
// the other binary64 form takes one CTA per SM (254 registers, no spills).
template <typename T, bool GRP, bool BT = false>
__global__ void __launch_bounds__(NT3, GRP ? 4 / (sizeof(T) / sizeof(float)) : 1) k_out_off(DP<T> p, OutBuf<T> ob, int d, int nbif) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long boff = BT ? (long long)blockIdx.y * p.bstride : 0;
  if (BT) {
    dp_shift(p, boff);
    ob_shift(ob, boff);
  }
  __shared__ T red[16][BLK];
  __shared__ SideCtx cx;
  __shared__ T sEn[EN_N], wBu[MAXLOOP + 1];
  __shared__ __align__(8) unsigned long long sbar;
  if ((int)blockIdx.x < nbif) {
    if constexpr (!GRP)
      out_bif_cell(p, ob, d, blockIdx.x, red);
    else if ((int)blockIdx.x == nbif - 1)
      out_bif_ext_group(p, ob, d, red);
    else
      out_bif_group(p, ob, d, blockIdx.x * 4, red);
    return;
  }
  if (threadIdx.x == 0) mbar_init(&sbar, NT3);  // one arrival per thread (side work)
  __syncthreads();
  side_cell(p, ob, d + 4, blockIdx.x - nbif, (T *)smem_raw, cx, sEn, wBu, &sbar, 0u, boff);
}

template <typename T>
constexpr size_t out_side_smem() {
  return (size_t)(SS_N + 6) * BLK * sizeof(T);
}

// ---------------------------------------------------------------- K4': transfer gradients
// After the reverse chain, d log Z / d T_q and d log Z / d X_q of every
// boundary position q, summed over the cells that read them:
//   role 0  cells (q, y), y > q, where T_q, X_q join the outer pair's left
//           base to the next position (T_x, X_x of the cell);
//   role 1  cells (x, q+1), x <= q, where they join the position before the
//           right base to it (T_{y-1}, X_{y-1}).
// Terms per cell (fq = 2^{E[d-2]-E[d]}, F = 2^{E[d-1]-E[d]}, Hxi = hXI with
// the inner mismatch factor):
//   T_x     fq hQB (HB[x+1][y-1] T_{y-1} + stack(QB[x+1][y-1]) T_{y-1})^T
//           + fq Hxi (QB[x+1][y-1] T_{y-1})^T + hCH CH[x+1][y]^T + tgY
//   T_{y-1} the same terms seen from the right;
//   X       the multiloop-closing and unpaired-start terms, and the exterior
//           prefix for x = 0.
// Grid (chunks of TG_CELLS partner cells, q, role); one warp per cell at a
// time stages the cell's blocks into its shared-memory slice, lanes over the
// M_q x M_{q+1} entries; the CTA adds its warps' sums and issues one binary64
// atomic per entry.
constexpr int TG_CELLS = 64;
constexpr int TG_NB = 22;  // staged blocks per cell
template <typename T>
constexpr size_t out_tg_smem() {  // two buffers per warp
  return (size_t)16 * TG_NB * BLK * sizeof(T) > (size_t)8 * BLK * 5 * sizeof(double)
             ? (size_t)16 * TG_NB * BLK * sizeof(T)
             : (size_t)8 * BLK * 5 * sizeof(double);
}

template <typename T>
__device__ __forceinline__ const T *tg_src(const DP<T> &p, int role, int k, int x, int y) {
  const int n = p.n, d = y - x;
  if (role == 0) {
    switch (k) {
      case 0: return d >= 4 ? p.hGc + cidx(n, x, y) * BLK : nullptr;
      case 1: return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
      case 2: return p.Tr + (size_t)(y - 1) * BLK;
      case 3: return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
      case 4: return d >= 6 ? p.hXI + cidx(n, x, y) * BLK : nullptr;
      case 5: return p.hCH + cidx(n, x, y) * BLK;
      case 6: return p.CH + cidx(n, x + 1, y) * BLK;
      case 7: return d >= 6 ? p.tgY + cidx(n, x, y) * BLK : nullptr;
      case 8: case 9: case 10: case 11: {
        if (d < 11) return nullptr;
        const T *t4[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
        return t4[k - 8] + cidx(n, x + 1, y - 1) * BLK;
      }
      case 12: return p.X + ((size_t)(y - 1) * 4 + XUP) * BLK;
      case 13: return p.X + ((size_t)(y - 1) * 4 + XPP) * BLK;
      case 14: return d >= 10 ? p.hQM2uu + cidx(n, x, y) * BLK : nullptr;
      case 15: return d >= 10 ? p.hQM2up + cidx(n, x, y) * BLK : nullptr;
      case 16: case 17: case 18: case 19: {
        if (d < 10) return nullptr;
        const T *t4[4] = {p.QM2up, p.QM2pp, p.QM2uu, p.QM2pu};
        return t4[k - 16] + cidx(n, x + 1, y) * BLK;
      }
      default: return nullptr;
    }
  }
  switch (k) {
    case 0: return d >= 4 ? p.hGc + cidx(n, x, y) * BLK : nullptr;
    case 1: return p.Tr + (size_t)x * BLK;
    case 2: return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
    case 3: return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
    case 4: return d >= 6 ? p.hXI + cidx(n, x, y) * BLK : nullptr;
    case 5: return p.X + ((size_t)x * 4 + XPU) * BLK;
    case 6: return p.X + ((size_t)x * 4 + XPP) * BLK;
    case 7: case 8: case 9: case 10: {
      if (d < 11) return nullptr;
      const T *t4[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
      return t4[k - 7] + cidx(n, x + 1, y - 1) * BLK;
    }
    case 11: case 12: case 13: case 14: {
      if (d < 5) return nullptr;
      const T *t4[4] = {p.QMpp, p.QMpu, p.QM2pp, p.QM2pu};
      return t4[k - 11] + cidx(n, x, y - 1) * BLK;
    }
    case 15: return d >= 5 ? p.hQMpu + cidx(n, x, y) * BLK : nullptr;
    case 16: return d >= 5 ? p.hG + cidx(n, x, y) * BLK : nullptr;
    case 17: return d >= 10 ? p.hQM2pu + cidx(n, x, y) * BLK : nullptr;
    case 18: return x == 0 ? p.Q5U + (size_t)(d - 1) * BLK : nullptr;
    case 19: return x == 0 ? p.Q5P + (size_t)(d - 1) * BLK : nullptr;
    case 20: return x == 0 ? p.hQ5U + (size_t)d * BLK : nullptr;
    case 21: return x == 0 ? p.hGx + (size_t)d * BLK : nullptr;
    default: return nullptr;
  }
}

// one warp stages the TG_NB blocks of cell (x, y) into dst with 16-byte
// asynchronous copies (absent blocks zero-filled), as one commit group
template <typename T>
__device__ __forceinline__ void tg_issue(const DP<T> &p, int role, int x, int y, T *dst, int lane) {
  constexpr int CH = BLK * sizeof(T) / 16;
  const T *mine = lane < TG_NB ? tg_src(p, role, lane, x, y) : nullptr;
#pragma unroll
  for (int j0 = 0; j0 < TG_NB * CH; j0 += 32) {
    const int j = j0 + lane;
    const T *src = (const T *)__shfl_sync(0xffffffffu, (unsigned long long)mine, (j / CH) & 31);
    if (j < TG_NB * CH) {
      const char *g = src ? (const char *)src + 16 * (j % CH) : (const char *)p.Tr;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32((char *)dst + 16 * j)), "l"(g),
                   "r"(src ? 16 : 0)
                   : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <typename T, bool BT = false>
__global__ void __launch_bounds__(256) k_out_tg(DP<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (BT) dp_shift(p, (long long)(blockIdx.z >> 1) * p.bstride);  // batch: z = 2 protein + role
  // a batch (codon-state layout) has its boundaries at q = 3r + 2 only: one
  // grid row per boundary instead of one per position
  const int n = p.n, q = BT ? 3 * (int)blockIdx.y + 2 : (int)blockIdx.y, role = blockIdx.z & 1;
  if (q >= n - 1 || p.bnd[q] == 0) return;
  const int ncell = role == 0 ? n - 1 - q : q + 1;  // role 0: y = q+1..n-1; role 1: x = 0..q
  const int c0 = blockIdx.x * TG_CELLS;
  if (c0 >= ncell) return;
  const int c1 = min(ncell, c0 + TG_CELLS);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T *buf = (T *)smem_raw + (size_t)w * 2 * TG_NB * BLK;
  const int Mr = p.Mp[q], Mc = p.Mp[q + 1], NE = Mr * Mc;
  const T *en = p.en;
  const T eb = en[EN_EB], sml = en[EN_EA] * en[EN_EC];
  T acc[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};  // T, X_UU, X_UP, X_PU, X_PP (a lane's cells)
  // cells c0+w, c0+w+8, ...: the next cell's blocks are in flight while the
  // current one is summed
  if (c0 + w < c1) tg_issue(p, role, role == 0 ? q : c0 + w, role == 0 ? q + 1 + c0 + w : q + 1, buf, lane);
  for (int i = c0 + w, it = 0; i < c1; i += 8, it++) {
    const int x = role == 0 ? q : i, y = role == 0 ? q + 1 + i : q + 1, d = y - x;
    const T *B = buf + (size_t)(it & 1) * TG_NB * BLK;
    if (i + 8 < c1) {
      const int i2 = i + 8;
      tg_issue(p, role, role == 0 ? q : i2, role == 0 ? q + 1 + i2 : q + 1, buf + (size_t)((it + 1) & 1) * TG_NB * BLK, lane);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncwarp();
    const int Ed = p.E[d];
    const T fq = clamp_p2<T>((d >= 2 ? p.E[d - 2] : 0) - Ed), F = clamp_p2<T>(p.E[d - 1] - Ed);
    const int Mx = p.Mp[x], My = p.Mp[y], M1 = p.Mp[x + 1], Mv = p.Mp[y - 1];
    const int *bx0 = p.base + (size_t)x * NS, *bx1 = p.base + (size_t)(x + 1) * NS;
    const int *by0 = p.base + (size_t)y * NS, *bv = p.base + (size_t)(y - 1) * NS;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int e = lane + 32 * k;
      if (e >= NE) continue;
      T tv = 0, xuu = 0, xup = 0, xpu = 0, xpp = 0;
      if (role == 0) {
        const int a = e / Mc, u = e % Mc;  // T_x[a][u]
        const T *hQB = B, *hbi = B + BLK, *Ty1 = B + 2 * BLK, *qin = B + 3 * BLK, *hXI = B + 4 * BLK;
        const T *hCH = B + 5 * BLK, *CHN = B + 6 * BLK, *Yt = B + 7 * BLK, *q2 = B + 8 * BLK;
        const T *XrUP = B + 12 * BLK, *XrPP = B + 13 * BLK, *hM2uu = B + 14 * BLK, *hM2up = B + 15 * BLK;
        const T *MR = B + 16 * BLK;  // QM2 up, pp, uu, pu of (x+1, y)
        if (d >= 4) {
          const int pa = bx0[a], bu = bx1[u];
          for (int b = 0; b < My; b++) {
            const T gq = hQB[a * NS + b];
            if (gq == (T)0) continue;
            T tt = s2<false, false>(hbi, Ty1, u, b, Mv);
            if (d >= 6) {
              const int pto = pair_type(pa, by0[b]);
#pragma unroll
              for (int b2 = 0; b2 < NS; b2++) {
                const int pti = b2 < Mv ? pair_type(bu, bv[b2]) : -1;
                if (pti < 0 || pto < 0) continue;
                tt += qin[u * NS + b2] * Ty1[b2 * NS + b] * en[EN_STK + pto * 6 + pti];
              }
            }
            tv += fq * gq * tt;
          }
        }
        if (d >= 6)
          for (int z = 0; z < My; z++)
            tv += fq * (hXI[a * NS + z] * en[EN_TM + by0[z] * 4 + bx0[a]]) * s2<false, false>(qin, Ty1, u, z, Mv);
        tv += s2<false, true>(hCH, CHN, a, u, My);
        if (d >= 6) tv += Yt[a * NS + u];
        if (d >= 10) {
          if (d >= 11) {
            T su = 0, sp2 = 0;
            for (int b = 0; b < My; b++) {
              const T gq = hQB[a * NS + b];
              if (gq == (T)0) continue;
              su += gq * (s2<false, false>(q2, XrUP, u, b, Mv) + s2<false, false>(q2 + BLK, XrPP, u, b, Mv));
              sp2 += gq * (s2<false, false>(q2 + 2 * BLK, XrUP, u, b, Mv) + s2<false, false>(q2 + 3 * BLK, XrPP, u, b, Mv));
            }
            xpu = fq * sml * su;
            xpp = fq * sml * sp2;
          }
          xuu = F * (eb * (s2<false, true>(hM2up, MR, a, u, My) + s2<false, true>(hM2uu, MR + 2 * BLK, a, u, My)));
          xup = F * (eb * (s2<false, true>(hM2up, MR + BLK, a, u, My) + s2<false, true>(hM2uu, MR + 3 * BLK, a, u, My)));
        }
      } else {
        const int v2 = e / Mc, b = e % Mc;  // T_{y-1}[v2][b]
        const T *hQB = B, *Tx = B + BLK, *hbi = B + 2 * BLK, *qin = B + 3 * BLK, *hXI = B + 4 * BLK;
        const T *XlPU = B + 5 * BLK, *XlPP = B + 6 * BLK, *q2 = B + 7 * BLK, *ML = B + 11 * BLK;
        const T *hMPU = B + 15 * BLK, *hGG = B + 16 * BLK, *hM2pu = B + 17 * BLK;
        const int pb = by0[b], pv = bv[v2];
        for (int a = 0; a < Mx; a++) {
          if (d >= 4) {
            const T gg = hQB[a * NS + b];
            if (gg != (T)0) {
              T tt = s2<false, false>(Tx, hbi, a, v2, M1);
              if (d >= 6) {
                const int pto = pair_type(bx0[a], pb);
#pragma unroll
                for (int a2 = 0; a2 < NS; a2++) {
                  const int pti = a2 < M1 ? pair_type(bx1[a2], pv) : -1;
                  if (pti < 0 || pto < 0) continue;
                  tt += Tx[a * NS + a2] * qin[a2 * NS + v2] * en[EN_STK + pto * 6 + pti];
                }
              }
              tv += fq * gg * tt;
            }
          }
          if (d >= 6) tv += fq * s2<false, false>(Tx, qin, a, v2, M1) * (hXI[a * NS + b] * en[EN_TM + pb * 4 + bx0[a]]);
        }
        if (d >= 11) {
          T su = 0, sp2 = 0;
          for (int a = 0; a < Mx; a++) {
            const T gq = hQB[a * NS + b];
            if (gq == (T)0) continue;
            su += gq * (s2<false, false>(XlPU, q2, a, v2, M1) + s2<false, false>(XlPP, q2 + 2 * BLK, a, v2, M1));
            sp2 += gq * (s2<false, false>(XlPU, q2 + BLK, a, v2, M1) + s2<false, false>(XlPP, q2 + 3 * BLK, a, v2, M1));
          }
          xup = fq * sml * su;
          xpp = fq * sml * sp2;
        }
        T xpu2 = 0, xuu2 = 0, xpp2 = 0, xup2 = 0;
        if (d >= 5) {
          // ML: QMpp, QMpu, QM2pp, QM2pu of (x, y-1)
          T a1 = eb * s2<true, false>(ML, hMPU, v2, b, Mx), a2 = eb * s2<true, false>(ML + BLK, hMPU, v2, b, Mx);
          const T a3 = s2<true, false>(ML, hGG, v2, b, Mx), a4 = s2<true, false>(ML + BLK, hGG, v2, b, Mx);
          if (d >= 10) {
            a1 += eb * s2<true, false>(ML + 2 * BLK, hM2pu, v2, b, Mx);
            a2 += eb * s2<true, false>(ML + 3 * BLK, hM2pu, v2, b, Mx);
          }
          xpu2 = F * a1;
          xuu2 = F * a2;
          xpp2 = F * a3;
          xup2 = F * a4;
        }
        if (x == 0) {
          // exterior prefix: Q5U[d] and Gx[d] from Q5*[d-1] X_{d-1}
          const T *q5u = B + 18 * BLK, *q5p = B + 19 * BLK, *hu = B + 20 * BLK, *hg = B + 21 * BLK;
          xuu2 += F * s2<true, false>(q5u, hu, v2, b, Mx);
          xpu2 += F * s2<true, false>(q5p, hu, v2, b, Mx);
          xup2 += F * s2<true, false>(q5u, hg, v2, b, Mx);
          xpp2 += F * s2<true, false>(q5p, hg, v2, b, Mx);
        }
        acc[k][1] += xuu2;
        acc[k][2] += xup2;
        acc[k][3] += xpu2;
        acc[k][4] += xpp2;
      }
      acc[k][0] += tv;
      acc[k][1] += xuu;
      acc[k][2] += xup;
      acc[k][3] += xpu;
      acc[k][4] += xpp;
    }
    __syncwarp();  // the buffer is refilled two cells later
  }
  // the CTA's sum per entry, one binary64 atomic each
  __syncthreads();
  double *R = (double *)smem_raw;  // [8][36][5]
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int e = lane + 32 * k;
    if (e < BLK)
      for (int v = 0; v < 5; v++) R[((size_t)w * BLK + e) * 5 + v] = e < NE ? (double)acc[k][v] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NE * 5; t += blockDim.x) {
    const int e = t / 5, v = t % 5;
    double s = 0;
    for (int ww = 0; ww < 8; ww++) s += R[((size_t)ww * BLK + e) * 5 + v];
    if (s == 0.0) continue;
    const int pe = (e / Mc) * NS + e % Mc;
    const int xk[4] = {XUU, XUP, XPU, XPP};
    if (v == 0) atomicAdd(p.hT + (size_t)q * BLK + pe, s);
    else atomicAdd(p.hX + ((size_t)q * 4 + xk[v - 1]) * BLK + pe, s);
  }
}

template <typename T, int NTT = NT>
constexpr size_t out_light_smem() {
  return ((size_t)(SO_N + NYY + 14) * BLK + NTT) * sizeof(T);
}

}  // namespace cf
