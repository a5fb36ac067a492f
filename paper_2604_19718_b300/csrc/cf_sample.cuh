// cf_sample.cuh -- exact sampling of (codon sequence, structure) by stochastic
// traceback of the inside tables (paper Section "Sequence sampling": the
// partition function is backtracked, drawing every summed-over degree of
// freedom, here the codon states as well as the structure).
//
// One warp per sample at a time; lanes evaluate the alternatives of one
// recursion element in parallel and a warp scan picks the first alternative
// whose running sum exceeds u * total.  Weights are evaluated in binary64 from
// the stored mantissas and their power-of-two factors.  Random numbers: Philox
// 4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011), key = seed, counter =
// (sample, draw), so a sample depends only on (seed, sample index).
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"

namespace cf {

struct Philox {
  uint32_t k0, k1, c0, c1;
  uint32_t draw;
  __device__ void round(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t a, uint32_t b) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(M0, x0), lo0 = M0 * x0;
    uint32_t hi1 = __umulhi(M1, x2), lo1 = M1 * x2;
    uint32_t y0 = hi1 ^ x1 ^ a, y1 = lo1, y2 = hi0 ^ x3 ^ b, y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  // uniform double in [0, 1) from the next counter value
  __device__ double uniform() {
    uint32_t x0 = c0, x1 = c1, x2 = draw++, x3 = 0x5eed5eedu;
    uint32_t a = k0, b = k1;
    for (int r = 0; r < 10; r++) {
      round(x0, x1, x2, x3, a, b);
      a += 0x9E3779B9u;
      b += 0xBB67AE85u;
    }
    uint64_t bits = ((uint64_t)x0 << 21) ^ (uint64_t)x1;
    return (double)(bits & ((1ull << 53) - 1)) * (1.0 / 9007199254740992.0);
  }
};

// Warp-cooperative choice among K alternatives with weights w(k) >= 0.
// Returns the chosen index, or -1 if all weights are zero.
template <typename F>
__device__ int warp_select(int K, const F &w, double u, int lane) {
  double tot = 0;
  for (int k = lane; k < K; k += 32) tot += w(k);
  tot = warp_sum(tot);
  if (!(tot > 0)) return -1;
  const double target = u * tot;
  double run = 0;
  int last = -1;
  for (int b0 = 0; b0 < K; b0 += 32) {
    int k = b0 + lane;
    double v = (k < K) ? w(k) : 0.0;
    double s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    unsigned hit = __ballot_sync(0xffffffffu, v > 0 && run + s > target);
    unsigned nz = __ballot_sync(0xffffffffu, v > 0);
    if (hit) return b0 + __ffs(hit) - 1;
    if (nz) last = b0 + 31 - __clz(nz);
    run += __shfl_sync(0xffffffffu, s, 31);
  }
  return last;
}

// element kinds of the traceback stack
enum : int { EL_EXT = 0, EL_B, EL_HB, EL_YY, EL_XI, EL_M2, EL_G, EL_M, EL_CH };

__host__ __device__ __forceinline__ int2 el_pack(int kind, int x, int y, int p1, int p2, int L) {
  // p1, p2: port = state + 6 * type (0..11); L: 0..31
  return make_int2(x | (y << 16), kind | (p1 << 4) | (p2 << 8) | (L << 12));
}

template <typename T>
struct SampleArgs {
  DP<T> p;
  const int *cid;   // [n*6] sense codon id of state a at position p
  const int *sctab; // single-codon layout: [m][36] codon of the states at 3r+1, 3r+2 (see below); else null
  int nsamples;
  uint64_t seed;
  int2 *stack;      // [warps][n + 64]
  int *state;       // [warps][n]
  int32_t *codons;  // [nsamples * m]
  int32_t *partner; // [nsamples * n]
  int *err;
};

template <typename T>
__device__ __forceinline__ double dv(const T *blk, int a, int b) {
  return (double)blk[a * NS + b];
}

// Entry (a, b) of the interior partial sum YY_L of cell (x, y) from its
// definition, for the checkpointed form (where YY is not kept for every
// cell): the sum over the L - 1 placements j of the inner pair of
//   CH[x][x+j] XI[x+j][y-L+2+j] CH[y-L+2+j][y]
// (every term on XI's diagonal d - L + 2, the exponent of YY_L).
template <typename T>
__device__ __forceinline__ double yy_entry(const DP<T> &p, int x, int y, int L, int a, int b) {
  const int n = p.n, d = y - x;
  double s = 0;
  for (int j = 0; j <= L - 2; j++) {
    const int xi = x + j, yi = y - L + 2 + j;
    if (yi - xi < 6) continue;
    const T *c1 = p.CH + cidx(n, x, xi) * BLK, *xb = p.XI + cidx(n, xi, yi) * BLK, *c2 = p.CH + cidx(n, yi, y) * BLK;
    const int Mu = p.Mp[xi], Mv = p.Mp[yi];
    for (int u = 0; u < Mu; u++) {
      const double cu = dv(c1, a, u);
      if (cu == 0) continue;
      double t = 0;
      for (int v = 0; v < Mv; v++) t += dv(xb, u, v) * dv(c2, v, b);
      s += cu * t;
    }
  }
  (void)d;
  return s;
}

__device__ __forceinline__ double dp2(int e) { return ldexp(1.0, e); }

template <typename T>
__global__ void __launch_bounds__(128) k_sample(SampleArgs<T> s) {
  const DP<T> &p = s.p;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int n = p.n, m = p.m;
  const T *en = p.en;
  const int *base = p.base;
  const int *E = p.E;
  int2 *stk = s.stack + (size_t)warp * (n + 64);
  int *st = s.state + (size_t)warp * n;
  const int cap = n + 64;
  for (int smp = warp; smp < s.nsamples; smp += nw) {
    Philox rng;
    rng.k0 = (uint32_t)s.seed;
    rng.k1 = (uint32_t)(s.seed >> 32);
    rng.c0 = (uint32_t)smp;
    rng.c1 = 0x51A3E5u;
    rng.draw = 0;
    int32_t *par = s.partner + (size_t)smp * n;
    for (int q = lane; q < n; q += 32) {
      st[q] = -1;
      par[q] = -1;
    }
    __syncwarp();
    int bad = 0;
    // top level: state a0 at 0 and the port of position n-1
    const int M0 = p.Mp[0], Ml = p.Mp[n - 1];
    {
      const T *u5 = p.Q5U + (size_t)(n - 1) * BLK, *p5 = p.Q5P + (size_t)(n - 1) * BLK;
      double u = rng.uniform();
      int k = warp_select(M0 * 2 * Ml, [&](int k) {
        int a = k / (2 * Ml), r = k % (2 * Ml), t = r / Ml, b = r % Ml;
        return p.u0[a] * (t ? dv(p5, a, b) : dv(u5, a, b));
      }, u, lane);
      if (k < 0) bad = 1;
      else {
        int a = k / (2 * Ml), r = k % (2 * Ml);
        stk[0] = el_pack(EL_EXT, a, n - 1, (r % Ml) + 6 * (r / Ml), 0, 0);
      }
    }
    int sp = bad ? 0 : 1;
    while (sp > 0 && !bad) {
      int2 el = stk[--sp];
      const int x = el.x & 0xffff, y = el.x >> 16;
      const int kind = el.y & 15, p1 = (el.y >> 4) & 15, p2 = (el.y >> 8) & 15, L = (el.y >> 12) & 31;
      const int d = y - x;
      auto push = [&](int2 e) {
        if (sp >= cap) bad = 2;
        else stk[sp++] = e;
      };
      // per-position states: written by lane 0 only, checked per residue at the end
      auto setst = [&](int q, int a) {
        if (lane == 0) st[q] = a;
      };
      double u = rng.uniform();
      if (kind == EL_EXT) {
        // x holds a0 (state at 0); prefix [0, y] with port p1 at y
        const int a0 = x, b = p1 % 6, t = p1 / 6;
        if (y == 0) {
          if (b != a0) bad = 4;
          setst(0, a0);
          continue;
        }
        setst(y, b);
        const int Mq = p.Mp[y - 1];
        const T *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
        const T *pu = p.Q5U + (size_t)(y - 1) * BLK, *pp = p.Q5P + (size_t)(y - 1) * BLK;
        if (t == 0) {
          int k = warp_select(2 * Mq, [&](int k) {
            int tq = k / Mq, q = k % Mq;
            return tq ? dv(pp, a0, q) * dv(Xr + XPU * BLK, q, b) : dv(pu, a0, q) * dv(Xr + XUU * BLK, q, b);
          }, u, lane);
          if (k < 0) bad = 5;
          else push(el_pack(EL_EXT, a0, y - 1, (k % Mq) + 6 * (k / Mq), 0, 0));
          continue;
        }
        // y paired with k: k = 0, or k in [1, y-4] through Gx[k] with state s at k
        const int K = 1 + 6 * max(0, y - 4);
        int k = warp_select(K, [&](int k) {
          if (k == 0) return dv(p.QB + cidx(n, 0, y) * BLK, a0, b);
          int kk = (k - 1) / 6 + 1, sst = (k - 1) % 6;
          if (sst >= p.Mp[kk]) return 0.0;
          return dv(p.Gx + (size_t)kk * BLK, a0, sst) * dv(p.QB + cidx(n, kk, y) * BLK, sst, b) *
                 dp2(E[kk] + E[y - kk] - E[y]);
        }, u, lane);
        if (k < 0) { bad = 6; continue; }
        if (k == 0) {
          push(el_pack(EL_B, 0, y, a0, b, 0));
          continue;
        }
        const int kk = (k - 1) / 6 + 1, sst = (k - 1) % 6;
        push(el_pack(EL_B, kk, y, sst, b, 0));
        // Gx[kk] = Q5*[kk-1] X_{kk-1}^{*P}: choose the port at kk-1
        const int Mk1 = p.Mp[kk - 1];
        const T *X1 = p.X + (size_t)(kk - 1) * 4 * BLK;
        const T *qu = p.Q5U + (size_t)(kk - 1) * BLK, *qp = p.Q5P + (size_t)(kk - 1) * BLK;
        double u2 = rng.uniform();
        int k2 = warp_select(2 * Mk1, [&](int k) {
          int tq = k / Mk1, q = k % Mk1;
          return tq ? dv(qp, a0, q) * dv(X1 + XPP * BLK, q, sst) : dv(qu, a0, q) * dv(X1 + XUP * BLK, q, sst);
        }, u2, lane);
        if (k2 < 0) bad = 7;
        else push(el_pack(EL_EXT, a0, kk - 1, (k2 % Mk1) + 6 * (k2 / Mk1), 0, 0));
        continue;
      }
      if (kind == EL_B) {
        const int a = p1, b = p2;
        setst(x, a);
        setst(y, b);
        if (lane == 0) {
          s.partner[(size_t)smp * n + x] = y;
          s.partner[(size_t)smp * n + y] = x;
        }
        const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
        const size_t ci = cidx(n, x + 1, y - 1);
        const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
        const T *hb = p.HB + ci * BLK, *qin = p.QB + ci * BLK;
        const T *Xl = p.X + (size_t)x * 4 * BLK, *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
        const T *q2[4] = {p.QM2uu + ci * BLK, p.QM2up + ci * BLK, p.QM2pu + ci * BLK, p.QM2pp + ci * BLK};
        const int pto = pair_type(base[x * NS + a], base[y * NS + b]);
        const int MM = Mu * Mv;
        const double sml = (double)en[EN_EA] * (double)en[EN_EC];
        // [0, MM): HB (u,v); [MM, 2MM): stack (u,v); [2MM, 6MM): multiloop (t1,t2,u,v)
        int k = warp_select(6 * MM, [&](int k) {
          int g = k / MM, r = k % MM, uu = r / Mv, vv = r % Mv;
          if (g == 0) return (double)tx[a * NS + uu] * dv(hb, uu, vv) * (double)ty[vv * NS + b];
          if (g == 1) {
            if (d < 6) return 0.0;
            int pti = pair_type(base[(x + 1) * NS + uu], base[(y - 1) * NS + vv]);
            if (pti < 0 || pto < 0) return 0.0;
            return (double)tx[a * NS + uu] * dv(qin, uu, vv) * (double)ty[vv * NS + b] * (double)en[EN_STK + pto * 6 + pti];
          }
          if (d < 11) return 0.0;
          int tt = g - 2, t1 = tt >> 1, t2 = tt & 1;
          return sml * (double)Xl[(2 + t1) * BLK + a * NS + uu] * dv(q2[tt], uu, vv) *
                 (double)Xr[(t2 * 2 + 1) * BLK + vv * NS + b];
        }, u, lane);
        if (k < 0) { bad = 8; continue; }
        int g = k / MM, r = k % MM, uu = r / Mv, vv = r % Mv;
        if (g == 0) push(el_pack(EL_HB, x + 1, y - 1, uu, vv, 0));
        else if (g == 1) push(el_pack(EL_B, x + 1, y - 1, uu, vv, 0));
        else {
          int tt = g - 2;
          push(el_pack(EL_M2, x + 1, y - 1, uu + 6 * (tt >> 1), vv + 6 * (tt & 1), 0));
        }
        continue;
      }
      if (kind == EL_HB) {
        // closing pair (x-1, y+1): hairpin, interior (L), bulges (L, side, state)
        const int a = p1, b = p2;
        setst(x, a);
        setst(y, b);
        const size_t c = cidx(n, x, y);
        const double tmo = (double)en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]];
        const int Ed = E[d];
        int k = warp_select(1 + NYY + 2 * MAXLOOP * NS, [&](int k) {
          if (k == 0) return (double)p.eHL[d + 1] * dp2(-Ed) * tmo * dv(p.CH + c * BLK, a, b);
          if (k <= NYY) {
            int LL = k + 1;
            if (d < 6 || LL > min(MAXLOOP, d - 4)) return 0.0;
            int ey = (LL == 2) ? Ed : E[d - LL + 2];
            const double yy = p.yyck ? yy_entry(p, x, y, LL, a, b) : dv(p.YY + (c * NYY + (LL - 2)) * BLK, a, b);
            return (double)en[EN_IN + LL] * dp2(ey - Ed) * tmo * yy;
          }
          int r = k - 1 - NYY, LL = r / (2 * NS) + 1, side = (r / NS) & 1, sst = r % NS;
          if (d - LL < 4) return 0.0;
          double f = (double)en[EN_BU + LL] * dp2(E[d - LL] - Ed);
          if (side == 0) {
            if (sst >= p.Mp[y - LL]) return 0.0;
            return f * dv(p.QB + cidx(n, x, y - LL) * BLK, a, sst) * dv(p.CH + cidx(n, y - LL, y) * BLK, sst, b);
          }
          if (sst >= p.Mp[x + LL]) return 0.0;
          return f * dv(p.CH + cidx(n, x, x + LL) * BLK, a, sst) * dv(p.QB + cidx(n, x + LL, y) * BLK, sst, b);
        }, u, lane);
        if (k < 0) { bad = 9; continue; }
        if (k == 0) push(el_pack(EL_CH, x, y, a, b, 0));
        else if (k <= NYY) push(el_pack(EL_YY, x, y, a, b, k + 1));
        else {
          int r = k - 1 - NYY, LL = r / (2 * NS) + 1, side = (r / NS) & 1, sst = r % NS;
          if (side == 0) {
            push(el_pack(EL_B, x, y - LL, a, sst, 0));
            push(el_pack(EL_CH, y - LL, y, sst, b, 0));
          } else {
            push(el_pack(EL_CH, x, x + LL, a, sst, 0));
            push(el_pack(EL_B, x + LL, y, sst, b, 0));
          }
        }
        continue;
      }
      if (kind == EL_YY && p.yyck) {
        // checkpointed form: the placement j of the inner pair and the states
        // (u at x+j, v at y-L+2+j) in one draw, from the definition of YY_L
        const int a = p1, b = p2;
        setst(x, a);
        setst(y, b);
        int k = warp_select((L - 1) * BLK, [&](int k) {
          const int j = k / BLK, u = (k % BLK) / NS, v = k % NS;
          const int xi = x + j, yi = y - L + 2 + j;
          if (yi - xi < 6 || u >= p.Mp[xi] || v >= p.Mp[yi]) return 0.0;
          return dv(p.CH + cidx(n, x, xi) * BLK, a, u) * dv(p.XI + cidx(n, xi, yi) * BLK, u, v) *
                 dv(p.CH + cidx(n, yi, y) * BLK, v, b);
        }, u, lane);
        if (k < 0) { bad = 10; continue; }
        const int j = k / BLK, uu = (k % BLK) / NS, vv = k % NS, xi = x + j, yi = y - L + 2 + j;
        push(el_pack(EL_CH, x, xi, a, uu, 0));
        push(el_pack(EL_XI, xi, yi, uu, vv, 0));
        push(el_pack(EL_CH, yi, y, vv, b, 0));
        continue;
      }
      if (kind == EL_YY) {
        // YY_L[x][y] = T_x YY_{L-1}[x+1][y] + XI[x][y-L+2] CH[y-L+2][y]
        const int a = p1, b = p2;
        setst(x, a);
        setst(y, b);
        const int M1 = p.Mp[x + 1], yl = y - L + 2, Ml = p.Mp[yl];
        const T *tx = p.Tr + (size_t)x * BLK;
        const T *yp = (L >= 3) ? p.YY + (cidx(n, x + 1, y) * NYY + (L - 3)) * BLK : nullptr;
        const bool hasxi = (yl - x) >= 6;
        int k = warp_select(M1 + Ml, [&](int k) {
          if (k < M1) return yp ? (double)tx[a * NS + k] * dv(yp, k, b) : 0.0;
          int sst = k - M1;
          if (!hasxi) return 0.0;
          return dv(p.XI + cidx(n, x, yl) * BLK, a, sst) * dv(p.CH + cidx(n, yl, y) * BLK, sst, b);
        }, u, lane);
        if (k < 0) { bad = 10; continue; }
        if (k < M1) push(el_pack(EL_YY, x + 1, y, k, b, L - 1));
        else {
          push(el_pack(EL_XI, x, yl, a, k - M1, 0));
          push(el_pack(EL_CH, yl, y, k - M1, b, 0));
        }
        continue;
      }
      if (kind == EL_XI) {
        // inner pair (x+1, y-1) with unpaired x, y of the enclosing interior loop
        const int w = p1, z = p2;
        setst(x, w);
        setst(y, z);
        const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
        const T *tx = p.Tr + (size_t)x * BLK, *ty = p.Tr + (size_t)(y - 1) * BLK;
        const T *qb = p.QB + cidx(n, x + 1, y - 1) * BLK;
        int k = warp_select(Mu * Mv, [&](int k) {
          int uu = k / Mv, vv = k % Mv;
          return (double)tx[w * NS + uu] * dv(qb, uu, vv) * (double)ty[vv * NS + z];
        }, u, lane);
        if (k < 0) { bad = 11; continue; }
        push(el_pack(EL_B, x + 1, y - 1, k / Mv, k % Mv, 0));
        continue;
      }
      if (kind == EL_M2) {
        const int a = p1 % 6, t1 = p1 / 6, b = p2 % 6, t2 = p2 / 6;
        setst(x, a);
        setst(y, b);
        if (t1 == 0) {
          // x unpaired: port at x+1
          const int M1 = p.Mp[x + 1];
          const T *Xl = p.X + (size_t)x * 4 * BLK;
          const size_t cr = cidx(n, x + 1, y);
          const T *q2[4] = {p.QM2uu + cr * BLK, p.QM2up + cr * BLK, p.QM2pu + cr * BLK, p.QM2pp + cr * BLK};
          int k = warp_select(2 * M1, [&](int k) {
            int t = k / M1, sst = k % M1;
            return (double)Xl[t * BLK + a * NS + sst] * dv(q2[t * 2 + t2], sst, b);
          }, u, lane);
          if (k < 0) { bad = 12; continue; }
          push(el_pack(EL_M2, x + 1, y, (k % M1) + 6 * (k / M1), p2, 0));
          continue;
        }
        if (t2 == 0) {
          // y unpaired: port at y-1 (QM2pp or QM2pu of [x, y-1])
          const int Mq = p.Mp[y - 1];
          const T *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
          const size_t cl = cidx(n, x, y - 1);
          int k = warp_select(2 * Mq, [&](int k) {
            int t = k / Mq, q = k % Mq;
            return t ? dv(p.QM2pp + cl * BLK, a, q) * (double)Xr[XPU * BLK + q * NS + b]
                     : dv(p.QM2pu + cl * BLK, a, q) * (double)Xr[XUU * BLK + q * NS + b];
          }, u, lane);
          if (k < 0) { bad = 13; continue; }
          push(el_pack(EL_M2, x, y - 1, p1, (k % Mq) + 6 * (k / Mq), 0));
          continue;
        }
        // both ends paired: split point k with state s at k
        const int Ed = E[d];
        const int K = NS * max(0, d - 8);
        int k = warp_select(K, [&](int k) {
          int kk = x + 5 + k / NS, sst = k % NS;
          if (sst >= p.Mp[kk]) return 0.0;
          return dv(p.G + cidx(n, x, kk) * BLK, a, sst) * dv(p.QB + cidx(n, kk, y) * BLK, sst, b) *
                 dp2(E[kk - x] + E[y - kk] - Ed);
        }, u, lane);
        if (k < 0) { bad = 14; continue; }
        const int kk = x + 5 + k / NS, sst = k % NS;
        push(el_pack(EL_B, kk, y, sst, b, 0));
        push(el_pack(EL_G, x, kk, a, sst, 0));
        continue;
      }
      if (kind == EL_G) {
        // G[x][y] = QM*[x][y-1] X_{y-1}^{*P}: port at y-1
        const int a = p1, b = p2;
        const int Mq = p.Mp[y - 1];
        const T *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
        const size_t cl = cidx(n, x, y - 1);
        int k = warp_select(2 * Mq, [&](int k) {
          int t = k / Mq, q = k % Mq;
          return t ? dv(p.QMpp + cl * BLK, a, q) * (double)Xr[XPP * BLK + q * NS + b]
                   : dv(p.QMpu + cl * BLK, a, q) * (double)Xr[XUP * BLK + q * NS + b];
        }, u, lane);
        if (k < 0) { bad = 15; continue; }
        push(el_pack(EL_M, x, y - 1, a, (k % Mq) + 6 * (k / Mq), 0));
        continue;
      }
      if (kind == EL_M) {
        // QM with a branch starting at x; port p2 at y
        const int a = p1, b = p2 % 6, t = p2 / 6;
        setst(x, a);
        setst(y, b);
        const size_t c = cidx(n, x, y);
        if (t == 1) {
          int k = warp_select(2, [&](int k) {
            return k == 0 ? (double)en[EN_EC] * dv(p.QB + c * BLK, a, b) : dv(p.QM2pp + c * BLK, a, b);
          }, u, lane);
          if (k < 0) { bad = 16; continue; }
          if (k == 0) push(el_pack(EL_B, x, y, a, b, 0));
          else push(el_pack(EL_M2, x, y, a + 6, b + 6, 0));
          continue;
        }
        const int Mq = p.Mp[y - 1];
        const T *Xr = p.X + (size_t)(y - 1) * 4 * BLK;
        const size_t cl = cidx(n, x, y - 1);
        int k = warp_select(2 * Mq, [&](int k) {
          int tq = k / Mq, q = k % Mq;
          return tq ? dv(p.QMpp + cl * BLK, a, q) * (double)Xr[XPU * BLK + q * NS + b]
                    : dv(p.QMpu + cl * BLK, a, q) * (double)Xr[XUU * BLK + q * NS + b];
        }, u, lane);
        if (k < 0) { bad = 17; continue; }
        push(el_pack(EL_M, x, y - 1, a, (k % Mq) + 6 * (k / Mq), 0));
        continue;
      }
      if (kind == EL_CH) {
        // unpaired stretch x..y with end states fixed: bridge over the transfers
        const int a = p1, b = p2;
        setst(x, a);
        int cur = a;
        for (int q = x; q < y; q++) {
          const int Mn = p.Mp[q + 1];
          const T *tq = p.Tr + (size_t)q * BLK, *cn = p.CH + cidx(n, q + 1, y) * BLK;
          double uq = (q == x) ? u : rng.uniform();
          int k = warp_select(Mn, [&](int k) { return (double)tq[cur * NS + k] * dv(cn, k, b); }, uq, lane);
          if (k < 0) { bad = 18; break; }
          cur = k;
          setst(q + 1, cur);
        }
        if (cur != b) bad = 19;
        continue;
      }
      bad = 20;
    }
    __syncwarp();
    __threadfence_block();
    for (int r = lane; r < m; r += 32) {
      int q = 3 * r;
      int cod = -1;
      if (s.sctab) {
        // single-codon layout: the states at 3r+1 (first and second base)
        // and 3r+2 (third base) fix the codon, which fixes the state at 3r
        const int a1 = st[q + 1], a2 = st[q + 2];
        const int e = (a1 >= 0 && a2 >= 0) ? s.sctab[(size_t)r * BLK + a1 * NS + a2] : -1;
        if (e < 0 || st[q] != (e >> 8)) bad = bad ? bad : 21;
        cod = e >= 0 ? (e & 255) : -1;
      } else {
        const int a = st[q];
        if (a < 0 || st[q + 1] != a || st[q + 2] != a) bad = bad ? bad : 21;
        cod = (a >= 0) ? s.cid[q * NS + a] : -1;
      }
      s.codons[(size_t)smp * m + r] = cod;
    }
    bad = __reduce_max_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicCAS(s.err, 0, bad);
    __syncwarp();
  }
}

}  // namespace cf
