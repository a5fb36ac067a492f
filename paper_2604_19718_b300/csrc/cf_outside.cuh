// cf_outside.cuh -- outside pass written as the hand-written adjoint of the
// inside pass (cf_inside.cuh), one anti-diagonal per launch from d = n-1 down
// to 0, one warp per cell.
//
// Adjoint mantissas: for a table A of diagonal d (exponent E[d]),
//   hA = (dZ/dA_true) * 2^{E[d]} / Z,
// so every reverse statement reuses the forward statement's power-of-two
// factor, and A * hA summed over a block is directly a probability (pair
// probabilities, Eq. pair-probability).  The transfers T_p and typed
// transitions X_p have exponent 0; hT, hX accumulate dlogZ/dT, dlogZ/dX in
// binary64 at residue-boundary positions only, from which the codon
// marginals follow (T o hT is the joint codon marginal of the two residues,
// the derivative form of Eq. marginal-codon).
//
// Gathers read finished adjoints of longer intervals; only the short chains
// (bulges, interior-loop chains), XI and the per-position gradients receive
// atomic adds, always from longer intervals than their own.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"

namespace cf {

template <typename T>
__device__ __forceinline__ void atomic_add_T(T *a, T v) {
  atomicAdd(a, v);
}

// atomically add a per-lane full block (entries a<Ma, b<Mb) to dst (T or double)
template <typename D, typename T>
__device__ __forceinline__ void atomic_add_block(D *dst, const T (&acc)[BLK], int Ma, int Mb) {
#pragma unroll
  for (int e = 0; e < BLK; e++)
    if ((e / NS) < Ma && (e % NS) < Mb && acc[e] != (T)0) atomicAdd(dst + e, (D)acc[e]);
}

template <typename T>
__global__ void __launch_bounds__(32 * WPB) k_outside(DP<T> p, int d) {
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  const int x = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (x >= n - d) return;
  const int y = x + d;
  const int Mx = p.Mp[x], My = p.Mp[y];
  const size_t c = cidx(n, x, y);
  const T *en = p.en;
  const int *base = p.base;
  const int *E = p.E;
  const int Ed = E[d];
  const T eb = en[EN_EB], ec = en[EN_EC], sml = en[EN_EA] * en[EN_EC];
  // factors of the users one and two diagonals up
  const T F1u = (d + 1 < n) ? clamp_p2<T>(Ed - E[d + 1]) : (T)0;
  const T F2u = (d + 2 < n) ? clamp_p2<T>(Ed - E[d + 2]) : (T)0;
  const bool encl = (x >= 1) && (y <= n - 2);  // enclosing pair (x-1, y+1) exists
  const T *gc = encl ? p.hGc + cidx(n, x - 1, y + 1) * BLK : nullptr;
  const int Mxl = encl ? p.Mp[x - 1] : 0, Myr = encl ? p.Mp[y + 1] : 0;
  const T *Xxl = (x >= 1) ? p.X + (size_t)(x - 1) * 4 * BLK : nullptr;  // X_{x-1}
  const T *Xy = (y <= n - 2) ? p.X + (size_t)y * 4 * BLK : nullptr;     // X_y
  T acc[BLK];

  // ---------------- exterior (cell (0, y)) ----------------
  if (x == 0) {
    const int M0 = p.Mp[0];
    T *hu = p.hQ5U + (size_t)d * BLK, *hp = p.hQ5P + (size_t)d * BLK;
    if (d == n - 1) {
      double zi = 1.0 / *p.Zm;
      for (int e = lane; e < M0 * My; e += 32) {
        int a = e / My, b = e % My;
        T v = (T)(p.u0[a] * zi);
        hu[a * NS + b] = v;
        hp[a * NS + b] = v;
      }
    } else {
      const T *hu1 = p.hQ5U + (size_t)(d + 1) * BLK, *hg1 = p.hGx + (size_t)(d + 1) * BLK;
      const int M1 = p.Mp[d + 1];
      for (int e = lane; e < M0 * My; e += 32) {
        int a = e / My, b = e % My;
        hu[a * NS + b] = F1u * (e2<false, true>(hu1, Xy + XUU * BLK, a, b, M1) + e2<false, true>(hg1, Xy + XUP * BLK, a, b, M1));
        hp[a * NS + b] = F1u * (e2<false, true>(hu1, Xy + XPU * BLK, a, b, M1) + e2<false, true>(hg1, Xy + XPP * BLK, a, b, M1));
      }
    }
    if (d >= 1) {
      // hGx[d] = sum_{y' >= d+4} hQ5P[y'] QB[d][y']^T 2^{E[d] + E[y'-d] - E[y']}
      zero_block(acc);
      for (int yy = d + 4 + lane; yy <= n - 1; yy += 32) {
        T f = clamp_p2<T>(Ed + E[yy - d] - E[yy]);
        acc_mm<false, true>(acc, p.hQ5P + (size_t)yy * BLK, p.QB + cidx(n, d, yy) * BLK, M0, p.Mp[yy], My, f);
      }
      warp_reduce_block(acc, M0, My);
      T dummy = 0;
      store_block(p.hGx + (size_t)d * BLK, acc, M0, My, lane, dummy);
    }
    __syncwarp();
    // gradients of the transition X_{d-1} used by Q5U[d] and Gx[d]
    if (d >= 1 && p.bnd[d - 1]) {
      const T F = clamp_p2<T>(E[d - 1] - Ed);
      const int Mv = p.Mp[d - 1];
      const T *q5u = p.Q5U + (size_t)(d - 1) * BLK, *q5p = p.Q5P + (size_t)(d - 1) * BLK;
      const T *hg = p.hGx + (size_t)d * BLK;
      double *hx = p.hX + (size_t)(d - 1) * 4 * BLK;
      for (int e = lane; e < Mv * My; e += 32) {
        int a = e / My, b = e % My;  // a: state at d-1, b: state at d
        atomicAdd(hx + XUU * BLK + a * NS + b, (double)(F * e2<true, false>(q5u, hu, a, b, M0)));
        atomicAdd(hx + XPU * BLK + a * NS + b, (double)(F * e2<true, false>(q5p, hu, a, b, M0)));
        atomicAdd(hx + XUP * BLK + a * NS + b, (double)(F * e2<true, false>(q5u, hg, a, b, M0)));
        atomicAdd(hx + XPP * BLK + a * NS + b, (double)(F * e2<true, false>(q5p, hg, a, b, M0)));
      }
    }
    __syncwarp();
  }

  // ---------------- derived multiloop tables ----------------
  T *hm2uu = p.hQM2uu + c * BLK, *hm2up = p.hQM2up + c * BLK, *hm2pu = p.hQM2pu + c * BLK;
  T *hmpu = p.hQMpu + c * BLK, *hg = p.hG + c * BLK, *hmpp = p.hQMpp + c * BLK, *hm2pp = p.hQM2pp + c * BLK;
  const bool mlu = encl && (d + 2 >= 11);  // enclosing pair uses these QM2 as its multiloop
  if (d >= 10) {
    const T *uu1 = (x >= 1) ? p.hQM2uu + cidx(n, x - 1, y) * BLK : nullptr;
    const T *up1 = (x >= 1) ? p.hQM2up + cidx(n, x - 1, y) * BLK : nullptr;
    const T *pu1 = (y <= n - 2) ? p.hQM2pu + cidx(n, x, y + 1) * BLK : nullptr;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T vuu = 0, vup = 0, vpu = 0;
      if (mlu) {
        vuu = sml * F2u * e3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
        vup = sml * F2u * e3<true, false, true>(Xxl + XPU * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
        vpu = sml * F2u * e3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XUP * BLK, a, b, Mxl, Myr);
      }
      if (uu1) {
        vuu += eb * F1u * e2<true, false>(Xxl + XUU * BLK, uu1, a, b, p.Mp[x - 1]);
        vup += eb * F1u * e2<true, false>(Xxl + XUU * BLK, up1, a, b, p.Mp[x - 1]);
        vpu += eb * F1u * e2<true, false>(Xxl + XUP * BLK, uu1, a, b, p.Mp[x - 1]);
      }
      if (pu1) vpu += eb * F1u * e2<false, true>(pu1, Xy + XUU * BLK, a, b, p.Mp[y + 1]);
      hm2uu[a * NS + b] = vuu;
      hm2up[a * NS + b] = vup;
      hm2pu[a * NS + b] = vpu;
    }
  }
  if (d >= 5) {
    // hG[x][y]: G[x][y] feeds QM2pp[x][y'] as the left factor of split point y
    zero_block(acc);
    for (int yy = y + 4 + lane; yy <= n - 1; yy += 32) {
      T f = ec * clamp_p2<T>(Ed + E[yy - y] - E[yy - x]);
      acc_mm<false, true>(acc, p.hQM2pp + cidx(n, x, yy) * BLK, p.QB + cidx(n, y, yy) * BLK, Mx, p.Mp[yy], My, f);
    }
    warp_reduce_block(acc, Mx, My);
    T dummy = 0;
    store_block(hg, acc, Mx, My, lane, dummy);
    if (y <= n - 2) {
      const T *mpu1 = p.hQMpu + cidx(n, x, y + 1) * BLK, *g1 = p.hG + cidx(n, x, y + 1) * BLK;
      const int M1 = p.Mp[y + 1];
      for (int e = lane; e < Mx * My; e += 32) {
        int a = e / My, b = e % My;
        hmpu[a * NS + b] = F1u * (eb * e2<false, true>(mpu1, Xy + XUU * BLK, a, b, M1) + e2<false, true>(g1, Xy + XUP * BLK, a, b, M1));
      }
    }
  }
  if (d >= 4) {
    const bool r = y <= n - 2;
    const T *mpu1 = r ? p.hQMpu + cidx(n, x, y + 1) * BLK : nullptr;
    const T *g1 = r ? p.hG + cidx(n, x, y + 1) * BLK : nullptr;
    const T *pu1 = r ? p.hQM2pu + cidx(n, x, y + 1) * BLK : nullptr;
    const T *up1 = (x >= 1) ? p.hQM2up + cidx(n, x - 1, y) * BLK : nullptr;
    const int M1 = r ? p.Mp[y + 1] : 0;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T vpp = 0;
      if (r) vpp = F1u * (eb * e2<false, true>(mpu1, Xy + XPU * BLK, a, b, M1) + e2<false, true>(g1, Xy + XPP * BLK, a, b, M1));
      hmpp[a * NS + b] = vpp;
      T v2 = vpp;
      if (d >= 9) {
        if (mlu) v2 += sml * F2u * e3<true, false, true>(Xxl + XPP * BLK, gc, Xy + XPP * BLK, a, b, Mxl, Myr);
        if (r && d + 1 >= 10) v2 += eb * F1u * e2<false, true>(pu1, Xy + XPU * BLK, a, b, M1);
        if (up1 && d + 1 >= 10) v2 += eb * F1u * e2<true, false>(Xxl + XUP * BLK, up1, a, b, p.Mp[x - 1]);
      }
      hm2pp[a * NS + b] = (d >= 9) ? v2 : (T)0;
    }
  }
  __syncwarp();

  // ---------------- hQB ----------------
  T *hqb = p.hQB + c * BLK;
  if (d >= 4) {
    zero_block(acc);
    // split point k = x of QM2pp[x'][y] = sum_k G[x'][k] ec QB[k][y]
    for (int xx = x - 5 - lane; xx >= 0; xx -= 32) {
      T f = ec * clamp_p2<T>(E[x - xx] + Ed - E[y - xx]);
      acc_mm<true, false>(acc, p.G + cidx(n, xx, x) * BLK, p.hQM2pp + cidx(n, xx, y) * BLK, Mx, p.Mp[xx], My, f);
    }
    // bulges of longer intervals containing (x, y) as the inner pair
    for (int t = lane; t < 2 * MAXLOOP; t += 32) {
      int L = t / 2 + 1;
      if ((t & 1) == 0) {
        if (y + L > n - 1) continue;  // HB[x][y+L] 3' bulge
        T f = en[EN_BU + L] * clamp_p2<T>(Ed - E[d + L]);
        acc_mm<false, true>(acc, p.hHB + cidx(n, x, y + L) * BLK, p.CH + cidx(n, y, y + L) * BLK, Mx, p.Mp[y + L], My, f);
      } else {
        if (x - L < 0) continue;  // HB[x-L][y] 5' bulge
        T f = en[EN_BU + L] * clamp_p2<T>(Ed - E[d + L]);
        acc_mm<true, false>(acc, p.CH + cidx(n, x - L, x) * BLK, p.hHB + cidx(n, x - L, y) * BLK, Mx, p.Mp[x - L], My, f);
      }
    }
    warp_reduce_block(acc, Mx, My);
    const T *qb = p.QB + c * BLK;
    const T *hxi1 = encl ? p.hXI + cidx(n, x - 1, y + 1) * BLK : nullptr;
    const T *Txl = (x >= 1) ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
    const T *Ty = (y <= n - 2) ? p.Tr + (size_t)y * BLK : nullptr;
    double psum = 0;
#pragma unroll
    for (int e = 0; e < BLK; e++) {
      int a = e / NS, b = e % NS;
      if (a < Mx && b < My && (e & 31) == lane) {
        T v = acc[e] + ec * hmpp[e];
        if (x == 0) v += p.hQ5P[(size_t)y * BLK + e];
        else v += clamp_p2<T>(E[x] + Ed - E[y]) * e2<true, false>(p.Gx + (size_t)x * BLK, p.hQ5P + (size_t)y * BLK, a, b, p.Mp[0]);
        if (encl) {
          // XI[x-1][y+1] = F (T_{x-1} QB T_y) o tm
          T s = 0;
          for (int w = 0; w < Mxl; w++) {
            T tl = Txl[w * NS + a];
            if (tl == (T)0) continue;
            for (int z = 0; z < Myr; z++)
              s += tl * hxi1[w * NS + z] * en[EN_TM + base[(y + 1) * NS + z] * 4 + base[(x - 1) * NS + w]] * Ty[b * NS + z];
          }
          // stack: QB[x-1][y+1] uses QB[x][y] as its inner pair
          int pti = pair_type(base[x * NS + a], base[y * NS + b]);
          if (pti >= 0) {
            for (int a1 = 0; a1 < Mxl; a1++) {
              T tl = Txl[a1 * NS + a];
              if (tl == (T)0) continue;
              for (int b1 = 0; b1 < Myr; b1++) {
                int pto = pair_type(base[(x - 1) * NS + a1], base[(y + 1) * NS + b1]);
                if (pto < 0) continue;
                s += tl * gc[a1 * NS + b1] * en[EN_STK + pto * 6 + pti] * Ty[b * NS + b1];
              }
            }
          }
          v += F2u * s;
        }
        hqb[e] = v;
        T g = (pair_type(base[x * NS + a], base[y * NS + b]) >= 0) ? v : (T)0;
        p.hGc[c * BLK + e] = g;
        psum += (double)qb[e] * (double)v;
      }
    }
    psum = warp_sum(psum);
    if (lane == 0) {
      float pv = (float)psum;
      p.P[(size_t)x * n + y] = pv;
      p.P[(size_t)y * n + x] = pv;
    }
  }
  __syncwarp();

  // gradients of T_x, T_{y-1}, X_x, X_{y-1} used by QB[x][y] itself
  if (d >= 4 && (p.bnd[x] || p.bnd[y - 1])) {
    const T f = clamp_p2<T>(E[d - 2] - Ed);
    const size_t ci = cidx(n, x + 1, y - 1);
    const T *G = p.hGc + c * BLK;
    const T *hb = p.HB + ci * BLK, *qin = p.QB + ci * BLK;
    const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
    const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
    const T *Xl = p.X + (size_t)x * 4 * BLK, *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
    const T *q2[4] = {p.QM2uu + ci * BLK, p.QM2up + ci * BLK, p.QM2pu + ci * BLK, p.QM2pp + ci * BLK};
    const bool ml = d >= 11, stk = d >= 6;
    if (p.bnd[x]) {
      double *ht = p.hT + (size_t)x * BLK;
      double *hx = p.hX + (size_t)x * 4 * BLK;
      for (int e = lane; e < Mx * Mu; e += 32) {
        int a = e / Mu, u = e % Mu;
        // hT_x[a][u] = f sum_b G[a][b] (HB T_{y-1})[u][b] + stack
        T s = 0;
        for (int b = 0; b < My; b++) {
          T g = G[a * NS + b];
          if (g == (T)0) continue;
          T t = e2<false, false>(hb, ty, u, b, Mv);
          if (stk) {
            int pto = pair_type(base[x * NS + a], base[y * NS + b]);
            for (int b2 = 0; b2 < Mv; b2++) {
              int pti = pair_type(base[(x + 1) * NS + u], base[(y - 1) * NS + b2]);
              if (pti < 0 || pto < 0) continue;
              t += qin[u * NS + b2] * ty[b2 * NS + b] * en[EN_STK + pto * 6 + pti];
            }
          }
          s += g * t;
        }
        atomicAdd(ht + a * NS + u, (double)(f * s));
        if (ml) {
          // X_x^{P,t1}: t1 = U uses QM2uu, QM2up; t1 = P uses QM2pu, QM2pp
          T su = 0, sp = 0;
          for (int b = 0; b < My; b++) {
            T g = G[a * NS + b];
            if (g == (T)0) continue;
            su += g * (e2<false, false>(q2[0], Xr + XUP * BLK, u, b, Mv) + e2<false, false>(q2[1], Xr + XPP * BLK, u, b, Mv));
            sp += g * (e2<false, false>(q2[2], Xr + XUP * BLK, u, b, Mv) + e2<false, false>(q2[3], Xr + XPP * BLK, u, b, Mv));
          }
          atomicAdd(hx + XPU * BLK + a * NS + u, (double)(f * sml * su));
          atomicAdd(hx + XPP * BLK + a * NS + u, (double)(f * sml * sp));
        }
      }
    }
    if (p.bnd[y - 1]) {
      double *ht = p.hT + (size_t)(y - 1) * BLK;
      double *hx = p.hX + (size_t)(y - 1) * 4 * BLK;
      for (int e = lane; e < Mv * My; e += 32) {
        int v = e / My, b = e % My;
        T s = 0;
        for (int a = 0; a < Mx; a++) {
          T g = G[a * NS + b];
          if (g == (T)0) continue;
          T t = e2<false, false>(tx, hb, a, v, Mu);
          if (stk) {
            int pto = pair_type(base[x * NS + a], base[y * NS + b]);
            for (int a2 = 0; a2 < Mu; a2++) {
              int pti = pair_type(base[(x + 1) * NS + a2], base[(y - 1) * NS + v]);
              if (pti < 0 || pto < 0) continue;
              t += tx[a * NS + a2] * qin[a2 * NS + v] * en[EN_STK + pto * 6 + pti];
            }
          }
          s += g * t;
        }
        atomicAdd(ht + v * NS + b, (double)(f * s));
        if (ml) {
          // X_{y-1}^{t2,P}: t2 = U uses QM2uu (t1=U), QM2pu (t1=P); t2 = P uses QM2up, QM2pp
          T su = 0, sp = 0;
          for (int a = 0; a < Mx; a++) {
            T g = G[a * NS + b];
            if (g == (T)0) continue;
            su += g * (e2<false, false>(Xl + XPU * BLK, q2[0], a, v, Mu) + e2<false, false>(Xl + XPP * BLK, q2[2], a, v, Mu));
            sp += g * (e2<false, false>(Xl + XPU * BLK, q2[1], a, v, Mu) + e2<false, false>(Xl + XPP * BLK, q2[3], a, v, Mu));
          }
          atomicAdd(hx + XUP * BLK + v * NS + b, (double)(f * sml * su));
          atomicAdd(hx + XPP * BLK + v * NS + b, (double)(f * sml * sp));
        }
      }
    }
  }

  // ---------------- hHB and its bulge chains ----------------
  T *hhb = p.hHB + c * BLK;
  if (d >= 2) {
    const T *Txl = (x >= 1) ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
    const T *Ty = (y <= n - 2) ? p.Tr + (size_t)y * BLK : nullptr;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T v = 0;
      if (encl && d + 2 >= 4) v = F2u * e3<true, false, true>(Txl, gc, Ty, a, b, Mxl, Myr);
      hhb[a * NS + b] = v;
    }
    __syncwarp();
    for (int t = lane; t < 2 * MAXLOOP; t += 32) {
      int L = t / 2 + 1;
      if (d - L < 4) continue;
      T f = en[EN_BU + L] * clamp_p2<T>(E[d - L] - Ed);
      zero_block(acc);
      if ((t & 1) == 0) {
        // HB += QB[x][y-L] CH[y-L][y]  ->  hCH[y-L][y] += QB^T hHB
        acc_mm<true, false>(acc, p.QB + cidx(n, x, y - L) * BLK, hhb, p.Mp[y - L], Mx, My, f);
        atomic_add_block(p.hCH + cidx(n, y - L, y) * BLK, acc, p.Mp[y - L], My);
      } else {
        // HB += CH[x][x+L] QB[x+L][y]  ->  hCH[x][x+L] += hHB QB^T
        acc_mm<false, true>(acc, hhb, p.QB + cidx(n, x + L, y) * BLK, Mx, My, p.Mp[x + L], f);
        atomic_add_block(p.hCH + cidx(n, x, x + L) * BLK, acc, Mx, p.Mp[x + L]);
      }
    }
  }

  // ---------------- interior partial sums YY_L ----------------
  if (d >= 6) {
    const int Lmax = min(MAXLOOP, d - 4);
    const int L = lane + 2;
    const int slot = d % YRING, slot1 = (d + 1) % YRING;
    if (L <= Lmax) {
      T w = en[EN_IN + L] * clamp_p2<T>(E[d - L + 2] - Ed);
      const bool rec = (x >= 1) && (L + 1 <= min(MAXLOOP, d + 1 - 4));
      const T *Txl = (x >= 1) ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
      const T *h1 = rec ? p.hYY + (((size_t)slot1 * n + (x - 1)) * NYY + (L + 1 - 2)) * BLK : nullptr;
      const int M1 = (x >= 1) ? p.Mp[x - 1] : 0;
      T hy[BLK];
      zero_block(hy);
#pragma unroll
      for (int a = 0; a < NS; a++)
        if (a < Mx)
#pragma unroll
          for (int b = 0; b < NS; b++)
            if (b < My) {
              T v = w * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * hhb[a * NS + b];
              if (rec)
                for (int s = 0; s < M1; s++) v += Txl[s * NS + a] * h1[s * NS + b];
              hy[a * NS + b] = v;
            }
      T *ho = p.hYY + (((size_t)slot * n + x) * NYY + (L - 2)) * BLK;
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e / NS) < Mx && (e % NS) < My) ho[e] = hy[e];
      const int yl = y - L + 2;
      if (yl - x >= 6) {
        // YY_L += XI[x][yl] CH[yl][y]
        zero_block(acc);
        acc_mm<false, true>(acc, hy, p.CH + cidx(n, yl, y) * BLK, Mx, My, p.Mp[yl], (T)1);
        atomic_add_block(p.hXI + cidx(n, x, yl) * BLK, acc, Mx, p.Mp[yl]);
        if (L >= 3) {
          zero_block(acc);
          acc_mm<true, false>(acc, p.XI + cidx(n, x, yl) * BLK, hy, p.Mp[yl], Mx, My, (T)1);
          atomic_add_block(p.hCH + cidx(n, yl, y) * BLK, acc, p.Mp[yl], My);
        }
      }
      if (L >= 3 && p.bnd[x]) {
        // YY_L += T_x YY_{L-1}[x+1][y]  ->  hT_x += hYY YY_{L-1}^T
        zero_block(acc);
        acc_mm<false, true>(acc, hy, p.YY + (cidx(n, x + 1, y) * NYY + (L - 3)) * BLK, Mx, My, p.Mp[x + 1], (T)1);
        atomic_add_block(p.hT + (size_t)x * BLK, acc, Mx, p.Mp[x + 1]);
      }
    }
  }
  __syncwarp();

  // ---------------- XI gradients into T_x, T_{y-1} ----------------
  if (d >= 6 && (p.bnd[x] || p.bnd[y - 1])) {
    const T f = clamp_p2<T>(E[d - 2] - Ed);
    const T *hxi = p.hXI + c * BLK;
    const T *qb = p.QB + cidx(n, x + 1, y - 1) * BLK;
    const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
    const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
    if (p.bnd[x]) {
      for (int e = lane; e < Mx * Mu; e += 32) {
        int w = e / Mu, a = e % Mu;
        T s = 0;
        for (int z = 0; z < My; z++)
          s += hxi[w * NS + z] * en[EN_TM + base[y * NS + z] * 4 + base[x * NS + w]] * e2<false, false>(qb, ty, a, z, Mv);
        atomicAdd(p.hT + (size_t)x * BLK + w * NS + a, (double)(f * s));
      }
    }
    if (p.bnd[y - 1]) {
      for (int e = lane; e < Mv * My; e += 32) {
        int b = e / My, z = e % My;
        T s = 0;
        for (int w = 0; w < Mx; w++)
          s += e2<false, false>(tx, qb, w, b, Mu) * hxi[w * NS + z] * en[EN_TM + base[y * NS + z] * 4 + base[x * NS + w]];
        atomicAdd(p.hT + (size_t)(y - 1) * BLK + b * NS + z, (double)(f * s));
      }
    }
  }

  // ---------------- chains ----------------
  if (d >= 1) {
    T *hch = p.hCH + c * BLK;
    const T *Txl = (x >= 1) ? p.Tr + (size_t)(x - 1) * BLK : nullptr;
    const T *h1 = (x >= 1) ? p.hCH + cidx(n, x - 1, y) * BLK : nullptr;
    const T hp = (d >= 2) ? p.eHL[d + 1] * clamp_p2<T>(-Ed) : (T)0;
    for (int e = lane; e < Mx * My; e += 32) {
      int a = e / My, b = e % My;
      T v = hch[a * NS + b];
      if (d >= 2) v += hp * en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]] * hhb[a * NS + b];
      if (h1) v += e2<true, false>(Txl, h1, a, b, p.Mp[x - 1]);
      hch[a * NS + b] = v;
    }
    __syncwarp();
    if (p.bnd[x]) {
      const T *chn = p.CH + cidx(n, x + 1, y) * BLK;
      const int M1 = p.Mp[x + 1];
      for (int e = lane; e < Mx * M1; e += 32) {
        int a = e / M1, s = e % M1;
        atomicAdd(p.hT + (size_t)x * BLK + a * NS + s, (double)e2<false, true>(hch, chn, a, s, My));
      }
    }
  }

  // ---------------- transitions used by the derived tables ----------------
  if (d >= 5 && p.bnd[y - 1]) {
    const T F = clamp_p2<T>(E[d - 1] - Ed);
    const size_t cl = cidx(n, x, y - 1);
    const int Mv = p.Mp[y - 1];
    const T *mpp = p.QMpp + cl * BLK, *mpu = p.QMpu + cl * BLK;
    const T *q2pp = p.QM2pp + cl * BLK, *q2pu = p.QM2pu + cl * BLK;
    double *hx = p.hX + (size_t)(y - 1) * 4 * BLK;
    for (int e = lane; e < Mv * My; e += 32) {
      int v = e / My, b = e % My;
      T xpu = eb * e2<true, false>(mpp, hmpu, v, b, Mx);
      T xuu = eb * e2<true, false>(mpu, hmpu, v, b, Mx);
      T xpp = e2<true, false>(mpp, hg, v, b, Mx);
      T xup = e2<true, false>(mpu, hg, v, b, Mx);
      if (d >= 10) {
        xpu += eb * e2<true, false>(q2pp, hm2pu, v, b, Mx);
        xuu += eb * e2<true, false>(q2pu, hm2pu, v, b, Mx);
      }
      atomicAdd(hx + XPU * BLK + v * NS + b, (double)(F * xpu));
      atomicAdd(hx + XUU * BLK + v * NS + b, (double)(F * xuu));
      atomicAdd(hx + XPP * BLK + v * NS + b, (double)(F * xpp));
      atomicAdd(hx + XUP * BLK + v * NS + b, (double)(F * xup));
    }
  }
  if (d >= 10 && p.bnd[x]) {
    const T F = clamp_p2<T>(E[d - 1] - Ed);
    const size_t cr = cidx(n, x + 1, y);
    const int Mu = p.Mp[x + 1];
    const T *u2up = p.QM2up + cr * BLK, *u2pp = p.QM2pp + cr * BLK, *u2uu = p.QM2uu + cr * BLK, *u2pu = p.QM2pu + cr * BLK;
    double *hx = p.hX + (size_t)x * 4 * BLK;
    for (int e = lane; e < Mx * Mu; e += 32) {
      int a = e / Mu, u = e % Mu;
      T xuu = eb * (e2<false, true>(hm2up, u2up, a, u, My) + e2<false, true>(hm2uu, u2uu, a, u, My));
      T xup = eb * (e2<false, true>(hm2up, u2pp, a, u, My) + e2<false, true>(hm2uu, u2pu, a, u, My));
      atomicAdd(hx + XUU * BLK + a * NS + u, (double)(F * xuu));
      atomicAdd(hx + XUP * BLK + a * NS + u, (double)(F * xup));
    }
  }
}

// Joint codon marginals of adjacent residues at each boundary transfer,
// trans[r][a][b] = T o (hT + sum_k hX_k o dangle_k), and residue 0's
// marginal from the top-level weights.
template <typename T>
__global__ void k_marginals(DP<T> p, double *trans, double *p0) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = p.n;
  if (r == 0) {
    int M0 = p.Mp[0], Ml = p.Mp[n - 1];
    const T *u = p.Q5U + (size_t)(n - 1) * BLK, *q = p.Q5P + (size_t)(n - 1) * BLK;
    for (int a = 0; a < M0; a++) {
      double s = 0;
      for (int b = 0; b < Ml; b++) s += (double)u[a * NS + b] + (double)q[a * NS + b];
      p0[a] = p.u0[a] * s / *p.Zm;
    }
  }
  if (r >= p.m - 1) return;
  const int q = 3 * r + 2;
  const int Ma = p.Mp[q], Mb = p.Mp[q + 1];
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) {
      double v = 0;
      if (a < Ma && b < Mb) {
        int x0 = p.base[q * NS + a], y0 = p.base[(q + 1) * NS + b];
        double d3 = (double)p.en[EN_D3 + x0 * 4 + y0], d5 = (double)p.en[EN_D5 + y0 * 4 + x0];
        double g = p.hT[(size_t)q * BLK + a * NS + b];
        const double *hx = p.hX + (size_t)q * 4 * BLK + a * NS + b;
        g += hx[XUU * BLK] + hx[XUP * BLK] * d5 + hx[XPU * BLK] * d3 + hx[XPP * BLK] * d3 * d5;
        v = (double)p.Tr[(size_t)q * BLK + a * NS + b] * g;
      }
      trans[(size_t)r * BLK + a * NS + b] = v;
    }
}

// Unpaired probability of every base: 1 - sum of its pair probabilities.
__global__ void k_unpaired(float *P, int n) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0;
  for (int j = lane; j < n; j += 32)
    if (j != i) s += (double)P[(size_t)i * n + j];
  s = warp_sum(s);
  if (lane == 0) P[(size_t)i * n + i] = (float)(1.0 - s);
}

}  // namespace cf
