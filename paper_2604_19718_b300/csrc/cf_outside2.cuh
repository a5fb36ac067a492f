// cf_outside2.cuh -- outside pass (hand-written adjoint of the inside pass) as
// two kernels per anti-diagonal d, run as a CUDA graph from d = n-1 down to 0:
//
//   k_out_bif<T>(d)   the transposed bifurcation gathers of diagonal d, in chunks
//                     of 32 terms (one warp per chunk):
//                       hG[x][y]  += sum_{y'} hQM2pp[x][y'] (ec QB[y][y'])^T    (row gather)
//                       hQB[x][y] += sum_{x'} (ec G[x'][x])^T hQM2pp[x'][y]     (column gather)
//                       hGx[d]     = sum_{y'} hQ5P[y'] QB[d][y']^T              (exterior)
//                     Its inputs lie on diagonals >= d+4, so it runs while
//                     d+3..d+1 are being finished.
//   k_out_light<T>(d) every other reverse statement of diagonal d, one 128-thread
//                     block per cell, inputs staged into shared memory.
//
// Adjoint scaling and the statements themselves are those of cf_outside.cuh:
// hA = (dZ/dA_true) 2^{E[d]} / Z, every reverse statement reuses its forward
// statement's power-of-two factor, gradients of the transfers accumulate in
// binary64 at residue-boundary positions.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"
#include "cf_inside2.cuh"

namespace cf {

template <typename T>
struct OutBuf {
  T *hg;   // [BIFRING][n][ncmax][36] row-gather chunks
  T *hq;   // [BIFRING][n][ncmax][36] column-gather chunks
  T *hgx;  // [BIFRING][ncmax][36]    exterior chunks
  int ncmax;
};

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
// chunks per cell used for the launch shape (upper bound over x)
__host__ __device__ __forceinline__ int out_cell_chunks(int n, int d) {
  int cnt = n - d - 8;
  return (cnt > 0 ? (cnt + KCH - 1) / KCH : 0) + 2;
}

// ---------------------------------------------------------------- K1'
// grid (chunks_per_cell / 4 rounded up, n - d [+1 for the exterior row]), 128 threads
template <typename T>
__global__ void __launch_bounds__(128) k_out_bif(DP<T> p, OutBuf<T> ob, int d) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int n = p.n;
  const int *E = p.E;
  const int Ed = E[d];
  const int slot = d % BIFRING;
  const T ec = p.en[EN_EC];
  T acc[BLK];
  zero_block(acc);
  T dummy = 0;
  if (blockIdx.y == (unsigned)(n - d)) {
    // exterior: hGx[d]
    if (q >= out_next(n, d)) return;
    const int M0 = p.Mp[0], Md = p.Mp[d];
    const int yy = d + 4 + q * KCH + lane;
    if (yy <= n - 1) {
      T f = clamp_p2<T>(Ed + E[yy - d] - E[yy]);
      acc_mm<false, true>(acc, p.hQ5P + (size_t)yy * BLK, p.QB + cidx(n, d, yy) * BLK, M0, p.Mp[yy], Md, f);
    }
    warp_reduce_block(acc, M0, Md);
    store_block(ob.hgx + ((size_t)slot * ob.ncmax + q) * BLK, acc, M0, Md, lane, dummy);
    return;
  }
  const int x = blockIdx.y, y = x + d;
  const int nr = out_nrow(n, x, d), nq = out_ncol(x, d);
  if (q >= nr + nq) return;
  const int Mx = p.Mp[x], My = p.Mp[y];
  if (q < nr) {
    const int yy = y + 4 + q * KCH + lane;
    if (yy <= n - 1) {
      T f = ec * clamp_p2<T>(Ed + E[yy - y] - E[yy - x]);
      acc_mm<false, true>(acc, p.hQM2pp + cidx(n, x, yy) * BLK, p.QB + cidx(n, y, yy) * BLK, Mx, p.Mp[yy], My, f);
    }
    warp_reduce_block(acc, Mx, My);
    store_block(ob.hg + (((size_t)slot * n + x) * ob.ncmax + q) * BLK, acc, Mx, My, lane, dummy);
  } else {
    const int c = q - nr;
    const int xx = x - 5 - c * KCH - lane;
    if (xx >= 0) {
      T f = ec * clamp_p2<T>(E[x - xx] + Ed - E[y - xx]);
      acc_mm<true, false>(acc, p.G + cidx(n, xx, x) * BLK, p.hQM2pp + cidx(n, xx, y) * BLK, Mx, p.Mp[xx], My, f);
    }
    warp_reduce_block(acc, Mx, My);
    store_block(ob.hq + (((size_t)slot * n + x) * ob.ncmax + c) * BLK, acc, Mx, My, lane, dummy);
  }
}

// ---------------------------------------------------------------- K2' staging
enum : int {
  SO_TXL = 0, SO_TX = 1, SO_TY1 = 2, SO_TY = 3,
  SO_XXL = 4, SO_XX = 8, SO_XY1 = 12, SO_XY = 16,
  SO_QB = 20, SO_QBI = 21, SO_HBI = 22, SO_Q2I = 23, SO_CHN = 27, SO_ML = 28, SO_MR = 32,
  SO_GC = 36, SO_HXIE = 37, SO_H2UU = 38, SO_H2UP = 39, SO_H2PU = 40, SO_HMPU = 41, SO_HG1 = 42,
  SO_HCHL = 43, SO_HCH = 44, SO_HXI = 45, SO_GX = 46, SO_HQ5P = 47,
  SO_HYR = 48, SO_YYP = 76, SO_XIL = 104, SO_CHL = 132,
  SO_BQ3 = 160, SO_BQ5 = 190, SO_BC3U = 220, SO_BC5U = 250, SO_BH3U = 280, SO_BH5U = 310,
  SO_N = 340
};

template <typename T>
__device__ __forceinline__ const T *out_slot_src(const DP<T> &p, int s, int x, int y, int d) {
  const int n = p.n;
  const bool hasL = x >= 1, hasR = y <= n - 2, encl = hasL && hasR;
  if (s < SO_XXL) {
    if (s == SO_TXL) return hasL ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
    if (s == SO_TX) return p.Tr + (size_t)x * BLK;
    if (s == SO_TY1) return d >= 1 ? p.Tr + (size_t)(y - 1) * BLK : nullptr;
    return hasR ? p.Tr + (size_t)y * BLK : nullptr;
  }
  if (s < SO_QB) {
    const int g = (s - SO_XXL) / 4, k = (s - SO_XXL) % 4;
    const int pos[4] = {x - 1, x, y - 1, y};
    const bool ok[4] = {hasL, true, d >= 1, hasR};
    return ok[g] ? p.X + ((size_t)pos[g] * 4 + k) * BLK : nullptr;
  }
  if (s == SO_QB) return d >= 4 ? p.QB + cidx(n, x, y) * BLK : nullptr;
  if (s == SO_QBI) return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s == SO_HBI) return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s < SO_CHN) {
    if (d < 11) return nullptr;
    const T *t[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
    return t[s - SO_Q2I] + cidx(n, x + 1, y - 1) * BLK;
  }
  if (s == SO_CHN) return d >= 1 ? p.CH + cidx(n, x + 1, y) * BLK : nullptr;
  if (s < SO_MR) {
    if (d < 5) return nullptr;
    const T *t[4] = {p.QMpp, p.QMpu, p.QM2pp, p.QM2pu};
    return t[s - SO_ML] + cidx(n, x, y - 1) * BLK;
  }
  if (s < SO_GC) {
    if (d < 10) return nullptr;
    const T *t[4] = {p.QM2up, p.QM2pp, p.QM2uu, p.QM2pu};
    return t[s - SO_MR] + cidx(n, x + 1, y) * BLK;
  }
  switch (s) {
    case SO_GC: return encl ? p.hGc + cidx(n, x - 1, y + 1) * BLK : nullptr;
    case SO_HXIE: return encl ? p.hXI + cidx(n, x - 1, y + 1) * BLK : nullptr;
    case SO_H2UU: return hasL ? p.hQM2uu + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_H2UP: return hasL ? p.hQM2up + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_H2PU: return hasR ? p.hQM2pu + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HMPU: return hasR ? p.hQMpu + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HG1: return hasR ? p.hG + cidx(n, x, y + 1) * BLK : nullptr;
    case SO_HCHL: return hasL ? p.hCH + cidx(n, x - 1, y) * BLK : nullptr;
    case SO_HCH: return d >= 1 ? p.hCH + cidx(n, x, y) * BLK : nullptr;
    case SO_HXI: return d >= 6 ? p.hXI + cidx(n, x, y) * BLK : nullptr;
    case SO_GX: return (x >= 1 && d >= 4) ? p.Gx + (size_t)x * BLK : nullptr;
    case SO_HQ5P: return (x >= 1 && d >= 4) ? p.hQ5P + (size_t)y * BLK : nullptr;
    default: break;
  }
  const int Lmax = min(MAXLOOP, d - 4);
  if (s < SO_YYP) {  // ring hYY_{L+1}[x-1][y], L = 2..29 (block L-1)
    int L = s - SO_HYR + 2;
    bool ok = hasL && d >= 6 && L <= Lmax && L + 1 <= min(MAXLOOP, d + 1 - 4);
    return ok ? p.hYY + (((size_t)((d + 1) % YRING) * n + (x - 1)) * NYY + (L - 1)) * BLK : nullptr;
  }
  if (s < SO_XIL) {  // YY_{L-1}[x+1][y], L = 3..30 (only needed for the gradient of T_x)
    int L = s - SO_YYP + 3;
    return (d >= 6 && L <= Lmax) ? p.YY + (cidx(n, x + 1, y) * NYY + (L - 3)) * BLK : nullptr;
  }
  if (s < SO_CHL) {
    int L = s - SO_XIL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.XI + cidx(n, x, yl) * BLK : nullptr;
  }
  if (s < SO_BQ3) {
    int L = s - SO_CHL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.CH + cidx(n, yl, y) * BLK : nullptr;
  }
  const int L = (s - SO_BQ3) % MAXLOOP + 1;
  if (s < SO_BQ5) return (d - L >= 4) ? p.QB + cidx(n, x, y - L) * BLK : nullptr;
  if (s < SO_BC3U) return (d - L >= 4) ? p.QB + cidx(n, x + L, y) * BLK : nullptr;
  // users of QB[x][y] as the inner pair of a bulge of a longer interval
  const bool up3 = d >= 4 && y + L <= n - 1, up5 = d >= 4 && x - L >= 0;
  if (s < SO_BC5U) return up3 ? p.CH + cidx(n, y, y + L) * BLK : nullptr;
  if (s < SO_BH3U) return up5 ? p.CH + cidx(n, x - L, x) * BLK : nullptr;
  if (s < SO_BH5U) return up3 ? p.hHB + cidx(n, x, y + L) * BLK : nullptr;
  return up5 ? p.hHB + cidx(n, x - L, y) * BLK : nullptr;
}

// ---------------------------------------------------------------- K2'
template <typename T>
__global__ void __launch_bounds__(128) k_out_light(DP<T> p, OutBuf<T> ob, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = (T *)smem_raw;            // [SO_N][36]
  T *HY = S + (size_t)SO_N * BLK;  // [29][36] interior partial-sum adjoints
  T *W = HY + NYY * BLK;           // work blocks
  T *hMPP = W, *hHB = W + BLK, *hQB = W + 2 * BLK, *G = W + 3 * BLK, *hCHf = W + 4 * BLK, *Hxi = W + 5 * BLK;
  T *ACC = W + 6 * BLK;            // [3][36]
  T *hM2 = W + 9 * BLK;            // uu, up, pu, pp
  T *hMPU = W + 13 * BLK, *hGG = W + 14 * BLK;
  __shared__ double sps[4];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int x = blockIdx.x, y = x + d;
  for (int s = t; s < SO_N; s += blockDim.x) {
    const T *src = out_slot_src(p, s, x, y, d);
    if (src) stage_block(S + (size_t)s * BLK, src);
  }
  cp_async_wait_all();
  __syncthreads();
  const int *E = p.E;
  const int *base = p.base;
  const T *en = p.en;
  const int Ed = E[d];
  const int Mx = p.Mp[x], My = p.Mp[y];
  const size_t c = cidx(n, x, y);
  const T eb = en[EN_EB], ec = en[EN_EC], sml = en[EN_EA] * en[EN_EC];
  const bool hasL = x >= 1, hasR = y <= n - 2, encl = hasL && hasR;
  const int Mxl = hasL ? p.Mp[x - 1] : 0, Myr = hasR ? p.Mp[y + 1] : 0;
  const T F1u = (d + 1 < n) ? clamp_p2<T>(Ed - E[d + 1]) : (T)0;
  const T F2u = (d + 2 < n) ? clamp_p2<T>(Ed - E[d + 2]) : (T)0;
  const T *gc = S + SO_GC * BLK;
  const T *Xxl = S + SO_XXL * BLK, *Xy = S + SO_XY * BLK;
  const int slot = d % BIFRING;
  const bool bx = p.bnd[x] != 0, by1 = d >= 1 && p.bnd[y - 1] != 0;

  // ---------------- A: exterior adjoint (cell (0, d)), multiloop tables with unpaired ends
  if (x == 0 && t >= 3 * BLK) {
    // threads 108..127: hQ5U, hQ5P of prefix [0, d] (entries strided by 20)
    const int M0 = p.Mp[0];
    for (int e = t - 3 * BLK; e < BLK; e += 128 - 3 * BLK) {
      const int a = e / NS, b = e % NS;
      if (a >= M0 || b >= My) continue;
      T hu, hp;
      if (d == n - 1) {
        hu = hp = (T)(p.u0[a] / *p.Zm);
      } else {
        const T *hu1 = p.hQ5U + (size_t)(d + 1) * BLK, *hg1 = p.hGx + (size_t)(d + 1) * BLK;
        const int M1 = p.Mp[d + 1];
        hu = F1u * (e2<false, true>(hu1, Xy + XUU * BLK, a, b, M1) + e2<false, true>(hg1, Xy + XUP * BLK, a, b, M1));
        hp = F1u * (e2<false, true>(hu1, Xy + XPU * BLK, a, b, M1) + e2<false, true>(hg1, Xy + XPP * BLK, a, b, M1));
      }
      p.hQ5U[(size_t)d * BLK + e] = hu;
      p.hQ5P[(size_t)d * BLK + e] = hp;
    }
  }
  if (d >= 10 && t < 3 * BLK) {
    const int g = t / BLK, e = t % BLK, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      const bool mlu = encl && d + 2 >= 11;
      T v = 0;
      if (g == 0) {  // QM2uu
        if (mlu) v = sml * F2u * e3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
        if (hasL) v += eb * F1u * e2<true, false>(Xxl + XUU * BLK, S + SO_H2UU * BLK, a, b, Mxl);
      } else if (g == 1) {  // QM2up
        if (mlu) v = sml * F2u * e3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
        if (hasL) v += eb * F1u * e2<true, false>(Xxl + XUU * BLK, S + SO_H2UP * BLK, a, b, Mxl);
      } else {  // QM2pu
        if (mlu) v = sml * F2u * e3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
        if (hasL) v += eb * F1u * e2<true, false>(Xxl + XUP * BLK, S + SO_H2UU * BLK, a, b, Mxl);
        if (hasR) v += eb * F1u * e2<false, true>(S + SO_H2PU * BLK, Xy + XUU * BLK, a, b, Myr);
      }
      hM2[g * BLK + e] = v;
      T *dst = g == 0 ? p.hQM2uu : (g == 1 ? p.hQM2up : p.hQM2pu);
      dst[c * BLK + e] = v;
    }
  }
  __syncthreads();
  if (x == 0 && d >= 1 && t < BLK) {
    // hGx[d] from its chunks
    const int M0 = p.Mp[0], a = t / NS, b = t % NS;
    if (a < M0 && b < My) {
      T v = 0;
      const int nq = out_next(n, d);
      for (int q = 0; q < nq; q++) v += ob.hgx[((size_t)slot * ob.ncmax + q) * BLK + t];
      p.hGx[(size_t)d * BLK + t] = v;
    }
  }

  // ---------------- B: hG, hQMpu, hQMpp (from the users one diagonal up)
  if (t < 3 * BLK) {
    const int g = t / BLK, e = t % BLK, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      if (g == 0 && d >= 5) {
        T v = 0;
        const int nr = out_nrow(n, x, d);
        const T *bp = ob.hg + (((size_t)slot * n + x) * ob.ncmax) * BLK + e;
        for (int q = 0; q < nr; q++) v += bp[(size_t)q * BLK];
        hGG[e] = v;
        p.hG[c * BLK + e] = v;
      } else if (g == 1 && d >= 5) {
        T v = 0;
        if (hasR)
          v = F1u * (eb * e2<false, true>(S + SO_HMPU * BLK, Xy + XUU * BLK, a, b, Myr) +
                     e2<false, true>(S + SO_HG1 * BLK, Xy + XUP * BLK, a, b, Myr));
        hMPU[e] = v;
        p.hQMpu[c * BLK + e] = v;
      } else if (g == 2 && d >= 4) {
        T v = 0;
        if (hasR)
          v = F1u * (eb * e2<false, true>(S + SO_HMPU * BLK, Xy + XPU * BLK, a, b, Myr) +
                     e2<false, true>(S + SO_HG1 * BLK, Xy + XPP * BLK, a, b, Myr));
        hMPP[e] = v;
        p.hQMpp[c * BLK + e] = v;
      }
    }
  }
  __syncthreads();

  // ---------------- C: hQM2pp (0..35), hHB (36..71)
  if (t < BLK) {
    const int a = t / NS, b = t % NS;
    if (d >= 4 && a < Mx && b < My) {
      T v = hMPP[t];
      if (d >= 9) {
        if (encl && d + 2 >= 11) v += sml * F2u * e3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
        if (hasR && d + 1 >= 10) v += eb * F1u * e2<false, true>(S + SO_H2PU * BLK, Xy + XPU * BLK, a, b, Myr);
        if (hasL && d + 1 >= 10) v += eb * F1u * e2<true, false>(Xxl + XUP * BLK, S + SO_H2UP * BLK, a, b, Mxl);
      } else {
        v = 0;
      }
      hM2[3 * BLK + t] = v;
      p.hQM2pp[c * BLK + t] = v;
    }
  } else if (t < 2 * BLK) {
    const int e = t - BLK, a = e / NS, b = e % NS;
    if (d >= 2 && a < Mx && b < My) {
      T v = 0;
      if (encl) v = F2u * e3<true, false, true>(S + SO_TXL * BLK, gc, S + SO_TY * BLK, a, b, Mxl, Myr);
      hHB[e] = v;
      p.hHB[c * BLK + e] = v;
    }
  }
  __syncthreads();

  // ---------------- D: hQB = sum of its users (three groups of threads)
  if (d >= 4 && t < 3 * BLK) {
    const int g = t / BLK, e = t % BLK, a = e / NS, b = e % NS;
    T v = 0;
    if (a < Mx && b < My) {
      for (int q = g; q < 2 * MAXLOOP; q += 3) {
        const int L = q / 2 + 1;
        if ((q & 1) == 0) {
          if (y + L > n - 1) continue;
          T f = en[EN_BU + L] * clamp_p2<T>(Ed - E[d + L]);
          v += f * e2<false, true>(S + (SO_BH3U + L - 1) * BLK, S + (SO_BC3U + L - 1) * BLK, a, b, p.Mp[y + L]);
        } else {
          if (x - L < 0) continue;
          T f = en[EN_BU + L] * clamp_p2<T>(Ed - E[d + L]);
          v += f * e2<true, false>(S + (SO_BC5U + L - 1) * BLK, S + (SO_BH5U + L - 1) * BLK, a, b, p.Mp[x - L]);
        }
      }
      if (g == 0) {
        v += ec * hMPP[e];
        const int nq = out_ncol(x, d);
        const int nr = out_nrow(n, x, d);
        (void)nr;
        const T *bp = ob.hq + (((size_t)slot * n + x) * ob.ncmax) * BLK + e;
        for (int q = 0; q < nq; q++) v += bp[(size_t)q * BLK];
        if (x == 0) v += p.hQ5P[(size_t)y * BLK + e];  // computed above in this kernel
        else v += clamp_p2<T>(E[x] + Ed - E[y]) * e2<true, false>(S + SO_GX * BLK, S + SO_HQ5P * BLK, a, b, p.Mp[0]);
      } else if (g == 1 && encl) {
        // XI[x-1][y+1] = F (T_{x-1} QB T_y) o tm
        const T *Txl = S + SO_TXL * BLK, *Ty = S + SO_TY * BLK, *hxi1 = S + SO_HXIE * BLK;
        T s2 = 0;
        for (int wv = 0; wv < Mxl; wv++) {
          const T tl = Txl[wv * NS + a];
          const int bw = base[(x - 1) * NS + wv];
          for (int z = 0; z < Myr; z++)
            s2 += tl * hxi1[wv * NS + z] * en[EN_TM + base[(y + 1) * NS + z] * 4 + bw] * Ty[b * NS + z];
        }
        v += F2u * s2;
      } else if (g == 2 && encl) {
        // stack of the enclosing pair (x-1, y+1)
        const int pti = pair_type(base[x * NS + a], base[y * NS + b]);
        if (pti >= 0) {
          const T *Txl = S + SO_TXL * BLK, *Ty = S + SO_TY * BLK;
          T s2 = 0;
          for (int a1 = 0; a1 < Mxl; a1++) {
            const T tl = Txl[a1 * NS + a];
            const int ba = base[(x - 1) * NS + a1];
            for (int b1 = 0; b1 < Myr; b1++) {
              const int pto = pair_type(ba, base[(y + 1) * NS + b1]);
              if (pto < 0) continue;
              s2 += tl * gc[a1 * NS + b1] * en[EN_STK + pto * 6 + pti] * Ty[b * NS + b1];
            }
          }
          v += F2u * s2;
        }
      }
    }
    ACC[g * BLK + e] = v;
  }
  __syncthreads();
  double psum = 0;
  if (d >= 4 && t < BLK) {
    const int a = t / NS, b = t % NS;
    if (a < Mx && b < My) {
      const T v = ACC[t] + ACC[BLK + t] + ACC[2 * BLK + t];
      p.hQB[c * BLK + t] = v;
      const T gq = pair_type(base[x * NS + a], base[y * NS + b]) >= 0 ? v : (T)0;
      hQB[t] = gq;
      p.hGc[c * BLK + t] = gq;
      psum = (double)S[SO_QB * BLK + t] * (double)v;
    }
  }
  // ---------------- E: interior partial-sum adjoints (all threads over (L, entry))
  if (d >= 6) {
    const int Lmax = min(MAXLOOP, d - 4);
    const int nitem = (Lmax - 1) * BLK;
    const T *Txl = S + SO_TXL * BLK;
    for (int it = t; it < nitem; it += blockDim.x) {
      const int L = it / BLK + 2, e = it % BLK, a = e / NS, b = e % NS;
      if (a >= Mx || b >= My) continue;
      const int ey = (L == 2) ? Ed : E[d - L + 2];
      T v = en[EN_IN + L] * clamp_p2<T>(ey - Ed) * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * hHB[e];
      if (hasL && L + 1 <= min(MAXLOOP, d + 1 - 4)) v += e2<true, false>(Txl, S + (SO_HYR + L - 2) * BLK, a, b, Mxl);
      HY[(L - 2) * BLK + e] = v;
      p.hYY[(((size_t)(d % YRING) * n + x) * NYY + (L - 2)) * BLK + e] = v;
    }
  }
  __syncthreads();
  // block sum of the pair probability
  psum = warp_sum(psum);
  if (lane == 0) sps[w] = psum;

  // ---------------- F: scatters into shorter chains and XI (atomic)
  if (d >= 5) {
    // bulges of HB[x][y]: hCH[y-L][y] += f QB[x][y-L]^T hHB ; hCH[x][x+L] += f hHB QB[x+L][y]^T
    for (int it = t; it < 2 * MAXLOOP * BLK; it += blockDim.x) {
      const int q = it / BLK, e = it % BLK, L = q / 2 + 1;
      if (d - L < 4) continue;
      const T f = en[EN_BU + L] * clamp_p2<T>(E[d - L] - Ed);
      const int r = e / NS, s2 = e % NS;
      if ((q & 1) == 0) {
        const int Ml = p.Mp[y - L];
        if (r >= Ml || s2 >= My) continue;
        const T v = f * e2<true, false>(S + (SO_BQ3 + L - 1) * BLK, hHB, r, s2, Mx);
        if (v != (T)0) atomicAdd(p.hCH + cidx(n, y - L, y) * BLK + e, v);
      } else {
        const int Ml = p.Mp[x + L];
        if (r >= Mx || s2 >= Ml) continue;
        const T v = f * e2<false, true>(hHB, S + (SO_BQ5 + L - 1) * BLK, r, s2, My);
        if (v != (T)0) atomicAdd(p.hCH + cidx(n, x, x + L) * BLK + e, v);
      }
    }
  }
  if (d >= 6) {
    // YY_L += XI[x][yl] CH[yl][y]: hXI[x][yl] += hYY CH^T ; hCH[yl][y] += XI^T hYY
    const int Lmax = min(MAXLOOP, d - 4);
    for (int it = t; it < 2 * (Lmax - 1) * BLK; it += blockDim.x) {
      const int q = it / BLK, e = it % BLK, L = q / 2 + 2, r = e / NS, s2 = e % NS;
      const int yl = y - L + 2;
      if (yl - x < 6) continue;
      const int Ml = p.Mp[yl];
      const T *hy = HY + (L - 2) * BLK;
      if ((q & 1) == 0) {
        if (r >= Mx || s2 >= Ml) continue;
        const T *ch = (L == 2) ? nullptr : S + (SO_CHL + L - 3) * BLK;
        const T v = (L == 2) ? hy[e] : e2<false, true>(hy, ch, r, s2, My);
        if (v != (T)0) atomicAdd(p.hXI + cidx(n, x, yl) * BLK + e, v);
      } else {
        if (L == 2) continue;
        if (r >= Ml || s2 >= My) continue;
        const T v = e2<true, false>(S + (SO_XIL + L - 3) * BLK, hy, r, s2, Mx);
        if (v != (T)0) atomicAdd(p.hCH + cidx(n, yl, y) * BLK + e, v);
      }
    }
  }
  // final chain adjoint of this cell (its scatters all came from longer intervals)
  if (d >= 1 && t < BLK) {
    const int a = t / NS, b = t % NS;
    if (a < Mx && b < My) {
      T v = S[SO_HCH * BLK + t];
      if (d >= 2) v += p.eHL[d + 1] * clamp_p2<T>(-Ed) * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * hHB[t];
      if (hasL) v += e2<true, false>(S + SO_TXL * BLK, S + SO_HCHL * BLK, a, b, Mxl);
      hCHf[t] = v;
      p.hCH[c * BLK + t] = v;
    }
  }
  // adjoint of XI[x][y] with its own L = 2 contribution, times the inner mismatch
  if (d >= 6 && t >= BLK && t < 2 * BLK) {
    const int e = t - BLK, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      const T h = S[SO_HXI * BLK + e] + HY[e];
      Hxi[e] = h * en[EN_TM + base[y * NS + b] * 4 + base[x * NS + a]];
    }
  }
  __syncthreads();
  if (t == 0 && d >= 4) {
    const double ps = sps[0] + sps[1] + sps[2] + sps[3];
    p.P[(size_t)x * n + y] = (float)ps;
    p.P[(size_t)y * n + x] = (float)ps;
  }

  // ---------------- G: gradients of the boundary transfers T_x, T_{y-1}, X_x, X_{y-1}
  if (!(bx || by1)) return;
  const T *Tx = S + SO_TX * BLK, *Ty1 = S + SO_TY1 * BLK;
  const T *hbi = S + SO_HBI * BLK, *qin = S + SO_QBI * BLK;
  const T *Xl = S + SO_XX * BLK, *Xr = S + SO_XY1 * BLK;
  const T fq = clamp_p2<T>((d >= 2 ? E[d - 2] : 0) - Ed);
  const int Mu = (d >= 1) ? p.Mp[x + 1] : 0, Mv = (d >= 1) ? p.Mp[y - 1] : 0;
  if (bx && t < BLK) {
    const int a = t / NS, u = t % NS;
    if (a < Mx && u < Mu) {
      T s = 0;
      // QB[x][y] = f (T_x HB T_{y-1} + stack)
      if (d >= 4) {
        for (int b = 0; b < My; b++) {
          const T g = hQB[a * NS + b];
          if (g == (T)0) continue;
          T tt = e2<false, false>(hbi, Ty1, u, b, Mv);
          if (d >= 6) {
            const int pto = pair_type(base[x * NS + a], base[y * NS + b]);
            const int bu = base[(x + 1) * NS + u];
            for (int b2 = 0; b2 < Mv; b2++) {
              const int pti = pair_type(bu, base[(y - 1) * NS + b2]);
              if (pti < 0 || pto < 0) continue;
              tt += qin[u * NS + b2] * Ty1[b2 * NS + b] * en[EN_STK + pto * 6 + pti];
            }
          }
          s += fq * g * tt;
        }
      }
      // XI[x][y] = f (T_x QB' T_{y-1}) o tm
      if (d >= 6)
        for (int z = 0; z < My; z++) s += fq * Hxi[a * NS + z] * e2<false, false>(qin, Ty1, u, z, Mv);
      // YY_L[x][y] = T_x YY_{L-1}[x+1][y] + ...
      if (d >= 6) {
        const int Lmax = min(MAXLOOP, d - 4);
        for (int L = 3; L <= Lmax; L++) s += e2<false, true>(HY + (L - 2) * BLK, S + (SO_YYP + L - 3) * BLK, a, u, My);
      }
      // CH[x][y] = T_x CH[x+1][y]
      if (d >= 1) s += e2<false, true>(hCHf, S + SO_CHN * BLK, a, u, My);
      atomicAdd(p.hT + (size_t)x * BLK + t, (double)s);
    }
  }
  if (by1 && t >= BLK && t < 2 * BLK) {
    const int e = t - BLK, v2 = e / NS, b = e % NS;
    if (v2 < Mv && b < My) {
      T s = 0;
      if (d >= 4) {
        for (int a = 0; a < Mx; a++) {
          const T g = hQB[a * NS + b];
          if (g == (T)0) continue;
          T tt = e2<false, false>(Tx, hbi, a, v2, Mu);
          if (d >= 6) {
            const int pto = pair_type(base[x * NS + a], base[y * NS + b]);
            const int bv = base[(y - 1) * NS + v2];
            for (int a2 = 0; a2 < Mu; a2++) {
              const int pti = pair_type(base[(x + 1) * NS + a2], bv);
              if (pti < 0 || pto < 0) continue;
              tt += Tx[a * NS + a2] * qin[a2 * NS + v2] * en[EN_STK + pto * 6 + pti];
            }
          }
          s += fq * g * tt;
        }
      }
      if (d >= 6)
        for (int wv = 0; wv < Mx; wv++) s += fq * e2<false, false>(Tx, qin, wv, v2, Mu) * Hxi[wv * NS + b];
      atomicAdd(p.hT + (size_t)(y - 1) * BLK + e, (double)s);
    }
  }
  if (bx && t >= 2 * BLK && t < 3 * BLK) {
    const int e = t - 2 * BLK, a = e / NS, u = e % NS;
    if (a < Mx && u < Mu) {
      double* hx = p.hX + (size_t)x * 4 * BLK;
      if (d >= 11) {
        const T *q2 = S + SO_Q2I * BLK;
        T su = 0, sp = 0;
        for (int b = 0; b < My; b++) {
          const T g = hQB[a * NS + b];
          if (g == (T)0) continue;
          su += g * (e2<false, false>(q2, Xr + XUP * BLK, u, b, Mv) + e2<false, false>(q2 + BLK, Xr + XPP * BLK, u, b, Mv));
          sp += g * (e2<false, false>(q2 + 2 * BLK, Xr + XUP * BLK, u, b, Mv) + e2<false, false>(q2 + 3 * BLK, Xr + XPP * BLK, u, b, Mv));
        }
        atomicAdd(hx + XPU * BLK + e, (double)(fq * sml * su));
        atomicAdd(hx + XPP * BLK + e, (double)(fq * sml * sp));
      }
      if (d >= 10) {
        const T F = clamp_p2<T>(E[d - 1] - Ed);
        const T *r_up = S + SO_MR * BLK, *r_pp = S + (SO_MR + 1) * BLK, *r_uu = S + (SO_MR + 2) * BLK,
                *r_pu = S + (SO_MR + 3) * BLK;
        const T xuu = eb * (e2<false, true>(hM2 + BLK, r_up, a, u, My) + e2<false, true>(hM2, r_uu, a, u, My));
        const T xup = eb * (e2<false, true>(hM2 + BLK, r_pp, a, u, My) + e2<false, true>(hM2, r_pu, a, u, My));
        atomicAdd(hx + XUU * BLK + e, (double)(F * xuu));
        atomicAdd(hx + XUP * BLK + e, (double)(F * xup));
      }
    }
  }
  if (by1 && t >= 3 * BLK) {
    // threads 108..127 cover the entries of X_{y-1} with stride 20
    double *hx = p.hX + (size_t)(y - 1) * 4 * BLK;
    for (int e = t - 3 * BLK; e < BLK; e += 128 - 3 * BLK) {
      const int v2 = e / NS, b = e % NS;
      if (v2 >= Mv || b >= My) continue;
      double xpu = 0, xuu = 0, xpp = 0, xup = 0;
      if (d >= 11) {
        const T *q2 = S + SO_Q2I * BLK;
        T su = 0, sp = 0;
        for (int a = 0; a < Mx; a++) {
          const T g = hQB[a * NS + b];
          if (g == (T)0) continue;
          su += g * (e2<false, false>(Xl + XPU * BLK, q2, a, v2, Mu) + e2<false, false>(Xl + XPP * BLK, q2 + 2 * BLK, a, v2, Mu));
          sp += g * (e2<false, false>(Xl + XPU * BLK, q2 + BLK, a, v2, Mu) + e2<false, false>(Xl + XPP * BLK, q2 + 3 * BLK, a, v2, Mu));
        }
        xup += (double)(fq * sml * su);
        xpp += (double)(fq * sml * sp);
      }
      if (d >= 5) {
        const T F = clamp_p2<T>(E[d - 1] - Ed);
        const T *mpp = S + SO_ML * BLK, *mpu = S + (SO_ML + 1) * BLK, *q2pp = S + (SO_ML + 2) * BLK,
                *q2pu = S + (SO_ML + 3) * BLK;
        T a1 = eb * e2<true, false>(mpp, hMPU, v2, b, Mx), a2 = eb * e2<true, false>(mpu, hMPU, v2, b, Mx);
        T a3 = e2<true, false>(mpp, hGG, v2, b, Mx), a4 = e2<true, false>(mpu, hGG, v2, b, Mx);
        if (d >= 10) {
          a1 += eb * e2<true, false>(q2pp, hM2 + 2 * BLK, v2, b, Mx);
          a2 += eb * e2<true, false>(q2pu, hM2 + 2 * BLK, v2, b, Mx);
        }
        xpu += (double)(F * a1);
        xuu += (double)(F * a2);
        xpp += (double)(F * a3);
        xup += (double)(F * a4);
      }
      if (x == 0) {
        // exterior: Q5U[d] and Gx[d] from Q5*[d-1] X_{d-1}
        const T F = clamp_p2<T>(E[d - 1] - Ed);
        const int M0 = p.Mp[0];
        const T *q5u = p.Q5U + (size_t)(d - 1) * BLK, *q5p = p.Q5P + (size_t)(d - 1) * BLK;
        const T *hu = p.hQ5U + (size_t)d * BLK, *hg = p.hGx + (size_t)d * BLK;
        xuu += (double)(F * e2<true, false>(q5u, hu, v2, b, M0));
        xpu += (double)(F * e2<true, false>(q5p, hu, v2, b, M0));
        xup += (double)(F * e2<true, false>(q5u, hg, v2, b, M0));
        xpp += (double)(F * e2<true, false>(q5p, hg, v2, b, M0));
      }
      atomicAdd(hx + XPU * BLK + e, xpu);
      atomicAdd(hx + XUU * BLK + e, xuu);
      atomicAdd(hx + XPP * BLK + e, xpp);
      atomicAdd(hx + XUP * BLK + e, xup);
    }
  }
}

template <typename T>
constexpr size_t out_light_smem() {
  return (size_t)(SO_N + NYY + 15) * BLK * sizeof(T);
}

}  // namespace cf
