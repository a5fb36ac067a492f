// cf_window.cuh -- batched partition functions of many short, fixed
// sequences (one codon per residue, so every position has a single state).
//
// This is the structure-only dynamic program of the paper's Section "Dynamic
// programs over structures for a given sequence" with the nearest-neighbour
// loop energies of the codon-constrained path (hairpin, stack, bulge,
// interior up to 30, multiloop a + c(B+1) + bU with d2 dangles, exterior
// dangles).  With one state per position the dangle of a branch is a number,
// so the typed U/P ports of the codon tables are not needed and each interval
// keeps three scalars:
//   QB[i][j]  i and j pair,
//   QM1[i][j] exactly one multiloop branch that starts at i and ends at or
//             before j, the rest unpaired,
//   QM[i][j]  at least one multiloop branch in [i, j].
// One CTA owns one window at a time (persistent over the batch) and fills its
// diagonals in order; a warp computes one cell, its lanes splitting the loop
// and split-point sums.  Values on diagonal d are stored relative to 2^{E[d]}
// with E[d] = E[d-1] + ilogb(largest stored value on d-1), as in the long
// protein path; the exterior prefix is accumulated in double.
#pragma once
#include "cf_common.cuh"

namespace cf {

constexpr int WT = 256;           // threads per window CTA
constexpr int WMAXN = 1024;       // longest window
constexpr int NLOOPPAIR = 496;    // (l1, l2) with l1 + l2 <= 30

struct WinArgs {
  const uint8_t *bases;   // concatenated windows, codes 0..3
  const int64_t *off;     // [nwin + 1]
  int nwin;
  const float *en;        // [EN_N] Boltzmann factors
  const float *eHL;       // [WMAXN + 2] hairpin length factors
  float log2eb;           // log2 of the multiloop unpaired factor
  float *scratch;         // per CTA: QB, QM1, QM of ncells(nmax) each
  size_t stride;          // floats per CTA
  double *logz;           // [nwin]
  int *err;               // bit 0: base code out of range
};

__device__ __forceinline__ float wp2(int e) {
  return e < -126 ? 0.f : __int_as_float((min(e, 127) + 127) << 23);
}

// 2^e * eb^k: exact power of two when the unpaired factor eb is one
__device__ __forceinline__ float wpow(int e, int k, float log2eb) {
  return log2eb == 0.f ? wp2(e) : exp2f((float)e + (float)k * log2eb);
}

__global__ void __launch_bounds__(WT) k_window(WinArgs a) {
  __shared__ uint8_t sb[WMAXN];
  __shared__ int sE[WMAXN];
  __shared__ double sq[WMAXN];
  __shared__ float sEn[EN_N];
  __shared__ uint8_t sl1[NLOOPPAIR], sl2[NLOOPPAIR];
  __shared__ float smax[WT / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < EN_N; i += WT) sEn[i] = a.en[i];
  for (int i = t; i < NLOOPPAIR; i += WT) {
    // enumerate (l1, l2) by total L, then l1
    int L = 0, r = i;
    while (r >= L + 1) { r -= L + 1; L++; }
    sl1[i] = (uint8_t)r;
    sl2[i] = (uint8_t)(L - r);
  }
  float *QB = a.scratch + (size_t)blockIdx.x * a.stride;
  const float ea = sEn[EN_EA], ec = sEn[EN_EC];
  for (int win = blockIdx.x; win < a.nwin; win += gridDim.x) {
    const int64_t o = a.off[win];
    const int n = (int)(a.off[win + 1] - o);
    const size_t nc = ncells(n);
    float *QM1 = QB + nc, *QM = QM1 + nc;
    __syncthreads();  // previous window fully consumed
    if (n == 0) {
      if (t == 0) a.logz[win] = 0.0;
      continue;
    }
    for (int i = t; i < n; i += WT) {
      int b = a.bases[o + i];
      if (b > 3) { atomicOr(a.err, 1); b = 0; }
      sb[i] = (uint8_t)b;
      sE[i] = 0;
    }
    __syncthreads();
    float lmax = 0.f;
    for (int d = 4; d < n; d++) {
      const int Ed = sE[d];
      for (int x = w; x + d < n; x += WT / 32) {
        const int y = x + d;
        const int pt = pair_type(sb[x], sb[y]);
        // ---- QB: hairpin, stack / bulge / interior, multiloop closing
        float acc = 0.f;
        if (pt >= 0) {
          const int bx1 = sb[x + 1], by1 = sb[y - 1];
          const float tmo = sEn[EN_TM + bx1 * 4 + by1];
          if (lane == 0) acc = a.eHL[d - 1] * tmo * wp2(-Ed);
          for (int q = lane; q < NLOOPPAIR; q += 32) {
            const int l1 = sl1[q], l2 = sl2[q];
            const int k = x + 1 + l1, l = y - 1 - l2;
            if (l - k < 4) continue;
            const float v = QB[cidx(n, k, l)];
            if (v == 0.f) continue;
            const int L = l1 + l2;
            float f;
            if (L == 0) f = sEn[EN_STK + pt * 6 + pair_type(sb[k], sb[l])];
            else if (l1 == 0 || l2 == 0) f = sEn[EN_BU + L];
            else f = sEn[EN_IN + L] * tmo * sEn[EN_TM + sb[l + 1] * 4 + sb[k - 1]];
            acc += f * v * wp2(sE[l - k] - Ed);
          }
          if (d >= 11) {
            float s = 0.f;
            for (int u = x + 6 + lane; u <= y - 5; u += 32)
              s += QM[cidx(n, x + 1, u - 1)] * QM1[cidx(n, u, y - 1)] * wp2(sE[u - x - 2] + sE[y - 1 - u] - Ed);
            acc += ea * ec * sEn[EN_D5 + sb[y] * 4 + by1] * sEn[EN_D3 + sb[x] * 4 + bx1] * s;
          }
        }
        acc = warp_sum(acc);
        const size_t c = cidx(n, x, y);
        if (lane == 0) QB[c] = acc;
        lmax = fmaxf(lmax, acc);
        __syncwarp();
        // ---- QM1: one branch (x, l), l <= y, then y - l unpaired
        const float dx = x > 0 ? sEn[EN_D5 + sb[x] * 4 + sb[x - 1]] : 1.f;
        float m1 = 0.f;
        for (int l = x + 4 + lane; l <= y; l += 32) {
          const float v = QB[cidx(n, x, l)];
          if (v == 0.f) continue;
          const float dl = l + 1 < n ? sEn[EN_D3 + sb[l] * 4 + sb[l + 1]] : 1.f;
          m1 += v * dl * wpow(sE[l - x] - Ed, y - l, a.log2eb);
        }
        m1 = warp_sum(m1) * ec * dx;
        if (lane == 0) QM1[c] = m1;
        lmax = fmaxf(lmax, m1);
        __syncwarp();
        // ---- QM: first branch starts at u, preceded by unpaired bases or by QM
        float mm = 0.f;
        for (int u = x + lane; u <= y - 4; u += 32) {
          const float v = QM1[cidx(n, u, y)];
          if (v == 0.f) continue;
          float pre = wpow(sE[y - u] - Ed, u - x, a.log2eb);
          if (u >= x + 5) pre += QM[cidx(n, x, u - 1)] * wp2(sE[u - 1 - x] + sE[y - u] - Ed);
          mm += v * pre;
        }
        mm = warp_sum(mm);
        if (lane == 0) QM[c] = mm;
        lmax = fmaxf(lmax, mm);
      }
      // ---- exponent of the next diagonal
      lmax = warp_max(lmax);
      if (lane == 0) smax[w] = lmax;
      __syncthreads();
      if (t == 0) {
        float m = 0.f;
        for (int k = 0; k < WT / 32; k++) m = fmaxf(m, smax[k]);
        if (!(m <= 3.0e38f)) atomicOr(a.err, 2);  // inf or nan
        if (d + 1 < n) sE[d + 1] = Ed + (m > 0.f ? ilogbf(m) : 0);
      }
      lmax = 0.f;
      __syncthreads();
    }
    // ---- exterior prefix q[j] = Q5[0..j] / 2^{E[j]} in double (warp 0)
    if (w == 0) {
      for (int j = 0; j < n; j++) {
        double s = 0.0;
        const double dj = j + 1 < n ? (double)sEn[EN_D3 + sb[j] * 4 + sb[j + 1]] : 1.0;
        for (int k = lane; k + 4 <= j; k += 32) {
          const float v = QB[cidx(n, k, j)];
          if (v == 0.f) continue;
          const double pre = k > 0 ? sq[k - 1] * ldexp(1.0, sE[k - 1] + sE[j - k] - sE[j]) : 1.0;
          const double dk = k > 0 ? (double)sEn[EN_D5 + sb[k] * 4 + sb[k - 1]] : 1.0;
          s += pre * (double)v * dk;
        }
        s = warp_sum(s) * dj;
        if (lane == 0) sq[j] = s + (j > 0 ? sq[j - 1] * ldexp(1.0, sE[j - 1] - sE[j]) : 1.0);
        __syncwarp();
      }
      if (lane == 0) {
        const double z = sq[n - 1];
        a.logz[win] = (z > 0 && isfinite(z)) ? log(z) + sE[n - 1] * 0.6931471805599453 : nan("");
      }
    }
  }
}

}  // namespace cf
