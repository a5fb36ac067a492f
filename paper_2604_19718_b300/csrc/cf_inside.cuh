// cf_inside.cuh -- inside pass (partition function) over the codon-constrained
// nearest-neighbour model, one anti-diagonal d = y - x per launch, one warp per
// cell (x, y).
//
// The sequence side is the codon-pair tensor train of the paper (Eq. pair-tt)
// laid along each loop's backbone (Section "Dynamic programs over sequences and
// structures"); every table entry is a block over the codon states at its two
// ends.  Tables of anti-diagonal d hold mantissas relative to 2^{E[d]}; E[d] is
// set from the largest mantissa of diagonal d-1 (the power-of-two analogue of
// the row renormalisation of Algorithm "EfficientFreeEnergy").  The chain CH
// carries exponent 0, the interior partial sums YY_L carry E[d-L+2].
//
// Tables, for the interval [x, y] (ports = codon states at x and at y):
//   CH[x][y]    chain T_x ... T_{y-1}
//   XI[x][y]    inner pair (x+1, y-1) extended by one base on each side with its
//               terminal mismatch, as seen from an enclosing interior loop
//   YY_L[x][y]  sum over inner pairs whose loop has L unpaired bases in total,
//               chains from x and to y included (L = 2..30)
//   HB[x][y]    everything inside a closing pair (x-1, y+1) except the stack and
//               the multiloop: hairpin + interior (with the closing mismatch) + bulges
//   QB[x][y]    x pairs with y
//   QMpp/QMpu   multiloop segment with >= 1 branch, branch starting at x, the
//               last base y paired (pp) or unpaired (pu)
//   G[x][y]     QM*[x][y-1] followed by the transition into a branch at y
//   QM2**       >= 2 branches; first/last base unpaired (u) or paired (p)
//   Q5U/Q5P[y]  exterior prefix [0, y], y unpaired / paired; Gx[y] as G
#pragma once
#include "cf_common.cuh"

namespace cf {

// 2^e from its IEEE-754 bit pattern (exponent field e + bias, zero mantissa);
// exponents below the normal range give 0, above 120 are clamped to 2^120.
template <typename T>
__device__ __forceinline__ T clamp_p2(int e);
template <>
__device__ __forceinline__ float clamp_p2<float>(int e) {
  e = e > 120 ? 120 : e;
  return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}
template <>
__device__ __forceinline__ double clamp_p2<double>(int e) {
  e = e > 120 ? 120 : e;
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

// store the warp-reduced block: entry e owned by lane e % 32
template <typename T>
__device__ __forceinline__ void store_block(T *dst, const T (&acc)[BLK], int Ma, int Mb, int lane,
                                            T &lmax) {
#pragma unroll
  for (int e = 0; e < BLK; e++)
    if ((e / NS) < Ma && (e % NS) < Mb && (e & 31) == lane) {
      dst[e] = acc[e];
      lmax = fmax(lmax, fabs(acc[e]));
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * WPB) k_inside(DP<T> p, int d) {
  __shared__ int sE;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  if (threadIdx.x == 0) {
    int e = 0;
    if (d > 0) {
      double mx = __longlong_as_double((long long)p.dmax[d - 1]);
      e = p.E[d - 1];
      if (mx > 0) {
        if (isfinite(mx)) e += ilogb(mx);
        else atomicOr(p.err, 1);
      }
    }
    sE = e;
    if (blockIdx.x == 0) p.E[d] = e;
  }
  __syncthreads();
  const int Ed = sE;
  const int x = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (x >= n - d) return;
  const int y = x + d;
  const int Mx = p.Mp[x], My = p.Mp[y];
  const size_t c = cidx(n, x, y);
  const T *en = p.en;
  const int *base = p.base;
  T lmax = 0;

  // ---- chain CH[x][y] = T_x CH[x+1][y]
  {
    T *ch = p.CH + c * BLK;
    if (d == 0) {
      for (int e = lane; e < Mx * My; e += 32) {
        int a = e / My, b = e % My;
        ch[a * NS + b] = (a == b) ? (T)1 : (T)0;
      }
    } else {
      const T *chn = p.CH + cidx(n, x + 1, y) * BLK;
      const T *tx = p.Tr + (size_t)x * BLK;
      int M1 = p.Mp[x + 1];
      for (int e = lane; e < Mx * My; e += 32) {
        int a = e / My, b = e % My;
        ch[a * NS + b] = e2<false, false>(tx, chn, a, b, M1);
      }
    }
  }
  // ---- XI[x][y] = (T_x QB[x+1][y-1] T_{y-1}) o tm[x_y][x_x]
  if (d >= 6) {
    T f = clamp_p2<T>(p.E[d - 2] - Ed);
    const T *qb = p.QB + cidx(n, x + 1, y - 1) * BLK;
    const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
    int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
    T *xi = p.XI + c * BLK;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T v = e3<false, false, false>(tx, qb, ty, a, b, Mu, Mv);
      v *= f * en[EN_TM + base[y * NS + b] * 4 + base[x * NS + a]];
      xi[a * NS + b] = v;
      lmax = fmax(lmax, fabs(v));
    }
  }
  __syncwarp();

  // ---- YY_L and HB
  T acc[BLK];
  zero_block(acc);
  if (d >= 6) {
    const int Lmax = min(MAXLOOP, d - 4);
    const int L = lane + 2;
    if (L <= Lmax) {
      const T *tx = p.Tr + (size_t)x * BLK;
      const int M1 = p.Mp[x + 1];
      const T *yp = (L >= 3) ? p.YY + (cidx(n, x + 1, y) * NYY + (L - 3)) * BLK : nullptr;
      const int yl = y - L + 2;
      const bool hasxi = (yl - x) >= 6;
      const T *xi = hasxi ? p.XI + cidx(n, x, yl) * BLK : nullptr;
      const T *ch = hasxi ? p.CH + cidx(n, yl, y) * BLK : nullptr;
      const int Ml = p.Mp[yl];
      T *yo = p.YY + (c * NYY + (L - 2)) * BLK;
      // E[d] itself is still being published by this launch: use the block's copy
      const int Eyy = (L == 2) ? Ed : p.E[d - L + 2];
      T wgt = en[EN_IN + L] * clamp_p2<T>(Eyy - Ed);
#pragma unroll
      for (int a = 0; a < NS; a++) {
        if (a < Mx) {
#pragma unroll
          for (int b = 0; b < NS; b++) {
            if (b < My) {
              T v = 0;
              if (yp) {
#pragma unroll
                for (int s = 0; s < NS; s++)
                  if (s < M1) v += tx[a * NS + s] * yp[s * NS + b];
              }
              if (hasxi) {
#pragma unroll
                for (int s = 0; s < NS; s++)
                  if (s < Ml) v += xi[a * NS + s] * ch[s * NS + b];
              }
              yo[a * NS + b] = v;
              acc[a * NS + b] += wgt * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * v;
            }
          }
        }
      }
    }
  }
  if (d >= 2) {
    // bulges: inner pair (x, y-L) or (x+L, y)
    for (int t = lane; t < 2 * MAXLOOP; t += 32) {
      int L = t / 2 + 1;
      if (d - L < 4) continue;
      T f = en[EN_BU + L] * clamp_p2<T>(p.E[d - L] - Ed);
      if ((t & 1) == 0)
        acc_mm<false, false>(acc, p.QB + cidx(n, x, y - L) * BLK, p.CH + cidx(n, y - L, y) * BLK, Mx,
                             p.Mp[y - L], My, f);
      else
        acc_mm<false, false>(acc, p.CH + cidx(n, x, x + L) * BLK, p.QB + cidx(n, x + L, y) * BLK, Mx,
                             p.Mp[x + L], My, f);
    }
    if (lane == 0) {
      // hairpin closed by (x-1, y+1): d+1 unpaired bases
      T h = p.eHL[d + 1] * clamp_p2<T>(-Ed);
      const T *ch = p.CH + c * BLK;
#pragma unroll
      for (int a = 0; a < NS; a++)
        if (a < Mx)
#pragma unroll
          for (int b = 0; b < NS; b++)
            if (b < My)
              acc[a * NS + b] += h * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * ch[a * NS + b];
    }
    warp_reduce_block(acc, Mx, My);
    store_block(p.HB + c * BLK, acc, Mx, My, lane, lmax);
  }

  // ---- QB[x][y]: closing pair (x, y)
  if (d >= 4) {
    T f = clamp_p2<T>(p.E[d - 2] - Ed);
    const size_t ci = cidx(n, x + 1, y - 1);
    const T *hb = p.HB + ci * BLK;
    const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
    const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
    const T *qin = (d >= 6) ? p.QB + ci * BLK : nullptr;
    const bool ml = d >= 11;
    const T *Xl = p.X + (size_t)x * 4 * BLK, *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
    T *qb = p.QB + c * BLK;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      int pto = pair_type(base[x * NS + a], base[y * NS + b]);
      T v = 0;
      if (pto >= 0) {
        v = e3<false, false, false>(tx, hb, ty, a, b, Mu, Mv);
        if (qin) {
#pragma unroll
          for (int a2 = 0; a2 < NS; a2++) {
            if (a2 < Mu) {
              T t = tx[a * NS + a2];
              const int ba = base[(x + 1) * NS + a2];
#pragma unroll
              for (int b2 = 0; b2 < NS; b2++) {
                if (b2 < Mv) {
                  int pti = pair_type(ba, base[(y - 1) * NS + b2]);
                  T e = pti >= 0 ? en[EN_STK + pto * 6 + pti] : (T)0;
                  v += t * qin[a2 * NS + b2] * ty[b2 * NS + b] * e;
                }
              }
            }
          }
        }
        if (ml) {
          T s = e3<false, false, false>(Xl + XPU * BLK, p.QM2uu + ci * BLK, Xr + XUP * BLK, a, b, Mu, Mv) +
                e3<false, false, false>(Xl + XPU * BLK, p.QM2up + ci * BLK, Xr + XPP * BLK, a, b, Mu, Mv) +
                e3<false, false, false>(Xl + XPP * BLK, p.QM2pu + ci * BLK, Xr + XUP * BLK, a, b, Mu, Mv) +
                e3<false, false, false>(Xl + XPP * BLK, p.QM2pp + ci * BLK, Xr + XPP * BLK, a, b, Mu, Mv);
          v += en[EN_EA] * en[EN_EC] * s;
        }
        v *= f;
      }
      qb[a * NS + b] = v;
      lmax = fmax(lmax, fabs(v));
    }
  }
  __syncwarp();

  // ---- QMpp = ec QB + QM2pp, QM2pp = sum_k G[x][k] ec QB[k][y]
  if (d >= 4) {
    zero_block(acc);
    const T ec = en[EN_EC];
    for (int k = x + 5 + lane; k <= y - 4; k += 32) {
      T f = ec * clamp_p2<T>(p.E[k - x] + p.E[y - k] - Ed);
      acc_mm<false, false>(acc, p.G + cidx(n, x, k) * BLK, p.QB + cidx(n, k, y) * BLK, Mx, p.Mp[k], My, f);
    }
    if (d >= 9) warp_reduce_block(acc, Mx, My);
    const T *qb = p.QB + c * BLK;
    T *q2 = p.QM2pp + c * BLK, *qm = p.QMpp + c * BLK;
#pragma unroll
    for (int e = 0; e < BLK; e++)
      if ((e / NS) < Mx && (e % NS) < My && (e & 31) == lane) {
        q2[e] = acc[e];
        T v = ec * qb[e] + acc[e];
        qm[e] = v;
        lmax = fmax(lmax, fmax(fabs(v), fabs(acc[e])));
      }
  }

  // ---- derived multiloop tables from diagonal d-1
  if (d >= 5) {
    const T F1 = clamp_p2<T>(p.E[d - 1] - Ed), eb = en[EN_EB];
    const T *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
    const int Mv = p.Mp[y - 1];
    const size_t cl = cidx(n, x, y - 1);
    const T *mpp = p.QMpp + cl * BLK, *mpu = p.QMpu + cl * BLK;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T u = eb * F1 * (e2<false, false>(mpp, Xr + XPU * BLK, a, b, Mv) + e2<false, false>(mpu, Xr + XUU * BLK, a, b, Mv));
      T g = F1 * (e2<false, false>(mpp, Xr + XPP * BLK, a, b, Mv) + e2<false, false>(mpu, Xr + XUP * BLK, a, b, Mv));
      p.QMpu[c * BLK + a * NS + b] = u;
      p.G[c * BLK + a * NS + b] = g;
      lmax = fmax(lmax, fmax(fabs(u), fabs(g)));
    }
    if (d >= 10) {
      const T *q2pp = p.QM2pp + cl * BLK, *q2pu = p.QM2pu + cl * BLK;
      const size_t cr = cidx(n, x + 1, y);
      const T *Xl = p.X + (size_t)x * 4 * BLK;
      const int Mu = p.Mp[x + 1];
      for (int e = lane; e < Mx * My; e += 32) {
        int a = e / My, b = e % My;
        T pu = eb * F1 * (e2<false, false>(q2pp, Xr + XPU * BLK, a, b, Mv) + e2<false, false>(q2pu, Xr + XUU * BLK, a, b, Mv));
        T up = eb * F1 * (e2<false, false>(Xl + XUU * BLK, p.QM2up + cr * BLK, a, b, Mu) +
                          e2<false, false>(Xl + XUP * BLK, p.QM2pp + cr * BLK, a, b, Mu));
        T uu = eb * F1 * (e2<false, false>(Xl + XUU * BLK, p.QM2uu + cr * BLK, a, b, Mu) +
                          e2<false, false>(Xl + XUP * BLK, p.QM2pu + cr * BLK, a, b, Mu));
        p.QM2pu[c * BLK + a * NS + b] = pu;
        p.QM2up[c * BLK + a * NS + b] = up;
        p.QM2uu[c * BLK + a * NS + b] = uu;
        lmax = fmax(lmax, fmax(fabs(pu), fmax(fabs(up), fabs(uu))));
      }
    }
  }

  // ---- exterior prefix [0, y] (the warp of cell (0, y))
  if (x == 0) {
    const int M0 = p.Mp[0];
    T *q5u = p.Q5U + (size_t)d * BLK, *q5p = p.Q5P + (size_t)d * BLK;
    if (d == 0) {
      for (int e = lane; e < M0 * M0; e += 32) {
        int a = e / M0, b = e % M0;
        q5u[a * NS + b] = (a == b) ? (T)1 : (T)0;
        q5p[a * NS + b] = 0;
      }
      lmax = fmax(lmax, (T)1);
    } else {
      const T F1 = clamp_p2<T>(p.E[d - 1] - Ed);
      const T *Xr = p.X + (size_t)(d - 1) * 4 * BLK;
      const int Mv = p.Mp[d - 1];
      const T *pu = p.Q5U + (size_t)(d - 1) * BLK, *pp = p.Q5P + (size_t)(d - 1) * BLK;
      T *gx = p.Gx + (size_t)d * BLK;
      for (int e = lane; e < M0 * My; e += 32) {
        int a = e / My, b = e % My;
        T g = F1 * (e2<false, false>(pu, Xr + XUP * BLK, a, b, Mv) + e2<false, false>(pp, Xr + XPP * BLK, a, b, Mv));
        T u = F1 * (e2<false, false>(pu, Xr + XUU * BLK, a, b, Mv) + e2<false, false>(pp, Xr + XPU * BLK, a, b, Mv));
        gx[a * NS + b] = g;
        q5u[a * NS + b] = u;
        lmax = fmax(lmax, fmax(fabs(g), fabs(u)));
      }
      zero_block(acc);
      for (int k = 1 + lane; k <= d - 4; k += 32) {
        T f = clamp_p2<T>(p.E[k] + p.E[d - k] - Ed);
        acc_mm<false, false>(acc, p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, M0, p.Mp[k], My, f);
      }
      warp_reduce_block(acc, M0, My);
      const T *qb0 = p.QB + c * BLK;
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e / NS) < M0 && (e % NS) < My && (e & 31) == lane) {
          T v = (d >= 4 ? qb0[e] : (T)0) + acc[e];
          q5p[e] = v;
          lmax = fmax(lmax, fabs(v));
        }
    }
  }

  lmax = warp_max(lmax);
  if (lane == 0) atomic_max_pos(&p.dmax[d], (double)lmax);
}

// Z relative to 2^{E[n-1]}: sum_a u0[a] sum_b (Q5U + Q5P)[n-1][a][b]
template <typename T>
__global__ void k_inside_finish(DP<T> p) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = p.n, M0 = p.Mp[0], Ml = p.Mp[n - 1];
  const T *u = p.Q5U + (size_t)(n - 1) * BLK, *q = p.Q5P + (size_t)(n - 1) * BLK;
  double z = 0;
  for (int a = 0; a < M0; a++) {
    double s = 0;
    for (int b = 0; b < Ml; b++) s += (double)u[a * NS + b] + (double)q[a * NS + b];
    z += p.u0[a] * s;
  }
  *p.Zm = z;
}

}  // namespace cf
