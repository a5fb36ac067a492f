// cf_subopt.cuh -- every (codon sequence, structure) whose cost is within a
// gap of the minimum free energy (paper SI "Suboptimal sequence generation",
// Alg. subopt, here over the min-sum tables of the nearest-neighbour model in
// cf_mfe.cuh).
//
// Depth-first over partial configurations: a partial configuration is a
// list of recursion elements still to be decomposed, the codon states and
// pairs fixed so far, and the slack left of the gap.  Expanding its last
// element E (table value v) runs through E's alternatives in a fixed order
// (the traceback's order, k_mfe_trace); an alternative of cost c with
// c <= v + slack gives a child whose slack is slack - (c - v) and whose list
// holds E's list with the alternative's sub-elements pushed.  A child with an
// empty list is a complete configuration of cost MFE + gap - slack.  The
// recursions are unambiguous (each configuration has one derivation), so
// every configuration within the gap is found exactly once.  One CTA: the
// alternatives come in groups with a lower bound each (k_sub_mins), the
// threads test 256 groups at a time, evaluate the alternatives of the groups
// within the limit 256 at a time, and the smallest feasible index at or after
// the element's cursor is taken; thread 0 keeps the frames (one per depth,
// each with its own copy of the list, states and pairs) in global memory.
// Chains and the inner pair of an interior loop are elements of their own, so
// that their state choices branch as well.
#pragma once
#include "cf_mfe.cuh"

namespace cf {

enum : int { MT_TOP = 16, MT_XIN = 17 };  // the root; the inner pair of an interior loop inside XI

__device__ __forceinline__ int4 el_make(int kind, int x, int y, int a, int b) {
  return make_int4(kind | (a << 8) | (b << 16), x, y, 0);
}

// The element's own table value.
__device__ __forceinline__ mq el_want(const MfeDP &p, int4 E, mq best) {
  const int n = p.n, kind = E.x & 255, a = (E.x >> 8) & 255, b = (E.x >> 16) & 255, x = E.y, y = E.z;
  switch (kind) {
    case MT_TOP: return best;
    case MT_EXT: return (a < NS ? p.Q5U : p.Q5P)[(size_t)x * BLK + y * NS + a % NS];  // x = j, y = a0, a = port
    case MT_QB: return p.QB[cidx(n, x, y) * BLK + a * NS + b];
    case MT_CH: return p.CH[cidx(n, x, y) * BLK + a * NS + b];
    case MT_QMP: return p.QMP[cidx(n, x, y) * BLK + a * NS + b];
    case MT_QMU: return p.QMU[cidx(n, x, y) * BLK + a * NS + b];
    case MT_GP: return p.GP[cidx(n, x, y) * BLK + a * NS + b];
    case MT_BP: return p.BP[cidx(n, x, y) * BLK + a * NS + b];
    case MT_M2PU: return p.M2PU[cidx(n, x, y) * BLK + a * NS + b];
    case MT_M2UP: return p.M2UP[cidx(n, x, y) * BLK + a * NS + b];
    case MT_M2UU: return p.M2UU[cidx(n, x, y) * BLK + a * NS + b];
    case MT_XIN: return p.XI[cidx(n, x, y) * BLK + a * NS + b];
  }
  return MQINF;
}

// QB alternatives: stack, bulges, multiloop, hairpin and interior loops
constexpr int SB_STACK = BLK, SB_BULGE = MAXLOOP * 2 * BLK, SB_ML = 4 * BLK, SB_HI = BLK * (1 + NINTERIOR * BLK);
constexpr int SB_QB = SB_STACK + SB_BULGE + SB_ML + SB_HI;

__device__ __forceinline__ int el_count(const MfeDP &p, int4 E) {
  const int kind = E.x & 255, a = (E.x >> 8) & 255, x = E.y, y = E.z;
  switch (kind) {
    case MT_TOP: return NS * 2 * p.Mp[p.n - 1];
    case MT_EXT:
      if (x == 0) return 1;
      if (a < NS) return 2 * p.Mp[x - 1];
      return 1 + max(0, x - 4) * 2 * NS * NS;
    case MT_CH: return x == y ? 1 : NS;
    case MT_QB: return SB_QB;
    case MT_QMP: return 2;
    case MT_QMU: case MT_M2PU: case MT_GP: case MT_M2UP: case MT_M2UU: return 2 * NS;
    case MT_BP: return max(0, y - x - 8) * NS;
    case MT_XIN: return BLK;
  }
  return 0;
}

// Cost of alternative k of E, and (kids != nullptr) its sub-elements in push
// order (the last one is decomposed first) with their own table values
// (kw, the terms of the cost that they stand for); returns the number of kids.
__device__ mq el_alt(const MfeDP &p, int4 E, int k, int4 *kids, int *nk, mq *kw = nullptr) {
  const int n = p.n, kind = E.x & 255, a = (E.x >> 8) & 255, b = (E.x >> 16) & 255, x = E.y, y = E.z;
  const mq *en = p.en;
  int c = 0;
  mq v = MQINF;
  auto kid = [&](int4 e, mq w) {
    if (kids) {
      kids[c] = e;
      if (kw) kw[c] = w;
      c++;
    }
  };
  switch (kind) {
    case MT_TOP: {  // residue 0's state and the port of position n-1, (a, type, b) ascending
      const int Ml = p.Mp[n - 1], a0 = k / (2 * Ml), r = k % (2 * Ml), tp = r / Ml, bb = r % Ml;
      const mq q5 = (tp ? p.Q5P : p.Q5U)[(size_t)(n - 1) * BLK + a0 * NS + bb];
      v = p.u0[a0] + q5;
      kid(el_make(MT_EXT, n - 1, a0, bb + NS * tp, 0), q5);
      break;
    }
    case MT_EXT: {
      const int j = x, a0 = y, port = a;
      if (j == 0) {
        v = port == a0 ? el_want(p, E, 0) : MQINF;
      } else if (port < NS) {  // j unpaired: (type, state) at j-1
        const int Mp = p.Mp[j - 1], tp = k / Mp, s = k % Mp;
        const mq q5 = (tp ? p.Q5P : p.Q5U)[(size_t)(j - 1) * BLK + a0 * NS + s];
        v = q5 + p.chi[(size_t)(j - 1) * 4 * BLK + (tp ? XPU : XUU) * BLK + s * NS + port];
        kid(el_make(MT_EXT, j - 1, a0, s + NS * tp, 0), q5);
      } else {  // j paired: the branch (0, j), then the last branch (kk, j)
        const int bb = port - NS;
        if (k == 0) {
          v = p.QB[cidx(n, 0, j) * BLK + a0 * NS + bb];
          kid(el_make(MT_QB, 0, j, a0, bb), v);
        } else {
          const int q = k - 1, kk = 1 + q / (2 * NS * NS), r = q % (2 * NS * NS), tp = r / (NS * NS),
                    s1 = (r / NS) % NS, s = r % NS;
          const mq *ch = p.chi + (size_t)(kk - 1) * 4 * BLK;
          const mq q5 = (tp ? p.Q5P : p.Q5U)[(size_t)(kk - 1) * BLK + a0 * NS + s1];
          const mq qb = p.QB[cidx(n, kk, j) * BLK + s * NS + bb];
          v = q5 + ch[(tp ? XPP : XUP) * BLK + s1 * NS + s] + qb;
          kid(el_make(MT_QB, kk, j, s, bb), qb);
          kid(el_make(MT_EXT, kk - 1, a0, s1 + NS * tp, 0), q5);
        }
      }
      break;
    }
    case MT_CH: {  // chain x..y with end states a, b: the next state
      if (x == y) {
        v = a == b ? 0 : MQINF;
      } else {
        const mq cw = p.CH[cidx(n, x + 1, y) * BLK + k * NS + b];
        v = p.tau[(size_t)x * BLK + a * NS + k] + cw;
        kid(el_make(MT_CH, x + 1, y, k, b), cw);
      }
      break;
    }
    case MT_QB: {
      const int i = x, j = y, d = j - i;
      const mq *ti = p.tau + (size_t)i * BLK, *tj1 = p.tau + (size_t)(j - 1) * BLK;
      int q = k;
      if (q < SB_STACK) {  // stack: (a2, b2)
        const int a2 = q / NS, b2 = q % NS;
        mq qb = MQINF;
        if (d >= 6) {
          const int po = pair_type(p.base[i * NS + a], p.base[j * NS + b]);
          const int pi = pair_type(p.base[(i + 1) * NS + a2], p.base[(j - 1) * NS + b2]);
          if (po >= 0 && pi >= 0) {
            qb = p.QB[cidx(n, i + 1, j - 1) * BLK + a2 * NS + b2];
            v = ti[a * NS + a2] + qb + tj1[b2 * NS + b] + en[EN_STK + po * 6 + pi];
          }
        }
        kid(el_make(MT_QB, i + 1, j - 1, a2, b2), qb);
        break;
      }
      q -= SB_STACK;
      if (q < SB_BULGE) {  // bulges: size L, 3' before 5', then the two free states
        const int L = 1 + q / (2 * BLK), side = (q / BLK) & 1, s1 = (q % BLK) / NS, s2 = q % NS;
        mq qb = MQINF, cw = MQINF;
        if (side == 0) {
          const int l = j - 1 - L;
          if (l - (i + 1) >= 4) {
            qb = p.QB[cidx(n, i + 1, l) * BLK + s1 * NS + s2];
            cw = p.CH[cidx(n, l, j) * BLK + s2 * NS + b];
            v = en[EN_BU + L] + ti[a * NS + s1] + qb + cw;
          }
          kid(el_make(MT_CH, l, j, s2, b), cw);
          kid(el_make(MT_QB, i + 1, l, s1, s2), qb);
        } else {
          const int kk = i + 1 + L;
          if ((j - 1) - kk >= 4) {
            cw = p.CH[cidx(n, i, kk) * BLK + a * NS + s1];
            qb = p.QB[cidx(n, kk, j - 1) * BLK + s1 * NS + s2];
            v = en[EN_BU + L] + cw + qb + tj1[s2 * NS + b];
          }
          kid(el_make(MT_CH, i, kk, a, s1), cw);
          kid(el_make(MT_QB, kk, j - 1, s1, s2), qb);
        }
        break;
      }
      q -= SB_BULGE;
      if (q < SB_ML) {  // multiloop: (type at i+1, type at j-1, state at i+1, state at j-1)
        const int t1 = q / (2 * BLK), t2 = (q / BLK) & 1, s = (q % BLK) / NS, s2 = q % NS;
        mq q2 = MQINF;
        if (d >= 11) {
          const mq *cx = p.chi + (size_t)i * 4 * BLK, *cy = p.chi + (size_t)(j - 1) * 4 * BLK;
          const mq *Q2 = t1 ? (t2 ? p.BP : p.M2PU) : (t2 ? p.M2UP : p.M2UU);
          q2 = Q2[cidx(n, i + 1, j - 1) * BLK + s * NS + s2];
          v = en[EN_EA] + en[EN_EC] + cx[(t1 ? XPP : XPU) * BLK + a * NS + s] + q2 +
              cy[(t2 ? XPP : XUP) * BLK + s2 * NS + b];
        }
        kid(el_make(t1 ? (t2 ? MT_BP : MT_M2PU) : (t2 ? MT_M2UP : MT_M2UU), i + 1, j - 1, s, s2), q2);
        break;
      }
      q -= SB_ML;
      {  // hairpin, then interior loops (l1 then l2), over (u at i+1, v at j-1), then (w at k-1, z at l+1)
        const int xi = i + 1, yi = j - 1;
        const int u = (q % BLK) / NS, vv = q % NS, sh = q / BLK;
        const mq outer = ti[a * NS + u] + tj1[vv * NS + b] + en[EN_TM + p.base[xi * NS + u] * 4 + p.base[yi * NS + vv]];
        if (sh == 0) {
          mq cw = MQINF;
          if (outer < MQHALF) {
            cw = p.CH[cidx(n, xi, yi) * BLK + u * NS + vv];
            v = outer + p.hq[d - 1] + cw;
          }
          kid(el_make(MT_CH, xi, yi, u, vv), cw);
        } else {
          const int qq = (sh - 1) / BLK, w = ((sh - 1) % BLK) / NS, z = (sh - 1) % NS;
          int l1, l2;
          interior_shape(qq, l1, l2);
          const int kk = i + 1 + l1, l = j - 1 - l2;
          mq c1 = MQINF, xw = MQINF, c2 = MQINF;
          if (outer < MQHALF && l - kk >= 4) {
            c1 = p.CH[cidx(n, xi, kk - 1) * BLK + u * NS + w];
            xw = p.XI[cidx(n, kk - 1, l + 1) * BLK + w * NS + z];
            c2 = p.CH[cidx(n, l + 1, yi) * BLK + z * NS + vv];
            v = outer + en[EN_IN + l1 + l2] + c1 + xw + c2;
          }
          kid(el_make(MT_CH, xi, kk - 1, u, w), c1);
          kid(el_make(MT_CH, l + 1, yi, z, vv), c2);
          kid(el_make(MT_XIN, kk - 1, l + 1, w, z), xw);
        }
      }
      break;
    }
    case MT_XIN: {  // the inner pair (x+1, y-1) inside XI[x][y]: states (a2, b2)
      const int a2 = k / NS, b2 = k % NS;
      const mq tmi = en[EN_TM + p.base[y * NS + b] * 4 + p.base[x * NS + a]];
      const mq qb = p.QB[cidx(n, x + 1, y - 1) * BLK + a2 * NS + b2];
      v = p.tau[(size_t)x * BLK + a * NS + a2] + qb + p.tau[(size_t)(y - 1) * BLK + b2 * NS + b] + tmi;
      kid(el_make(MT_QB, x + 1, y - 1, a2, b2), qb);
      break;
    }
    case MT_QMP: {  // a branch (x, y), then >= 2 branches
      if (k == 0) {
        const mq qb = p.QB[cidx(n, x, y) * BLK + a * NS + b];
        v = en[EN_EC] + qb;
        kid(el_make(MT_QB, x, y, a, b), qb);
      } else {
        v = p.BP[cidx(n, x, y) * BLK + a * NS + b];
        kid(el_make(MT_BP, x, y, a, b), v);
      }
      break;
    }
    case MT_QMU: case MT_M2PU: {  // y unpaired: (type at y-1, state at y-1)
      const bool one = kind == MT_QMU;
      const int tp = k / NS, s = k % NS;
      const mq *Pt = tp ? (one ? p.QMP : p.BP) : (one ? p.QMU : p.M2PU);
      const mq pw = Pt[cidx(n, x, y - 1) * BLK + a * NS + s];
      v = en[EN_EB] + pw + p.chi[(size_t)(y - 1) * 4 * BLK + (tp ? XPU : XUU) * BLK + s * NS + b];
      kid(el_make(tp ? (one ? MT_QMP : MT_BP) : kind, x, y - 1, a, s), pw);
      break;
    }
    case MT_GP: {  // the branch start at y: (type at y-1, state at y-1)
      const int tp = k / NS, s = k % NS;
      const mq pw = (tp ? p.QMP : p.QMU)[cidx(n, x, y - 1) * BLK + a * NS + s];
      v = pw + p.chi[(size_t)(y - 1) * 4 * BLK + (tp ? XPP : XUP) * BLK + s * NS + b];
      kid(el_make(tp ? MT_QMP : MT_QMU, x, y - 1, a, s), pw);
      break;
    }
    case MT_BP: {  // last branch (kk, y): kk ascending, state at kk
      const int kk = x + 5 + k / NS, s = k % NS;
      const mq gw = p.GP[cidx(n, x, kk) * BLK + a * NS + s], qb = p.QB[cidx(n, kk, y) * BLK + s * NS + b];
      v = en[EN_EC] + gw + qb;
      kid(el_make(MT_QB, kk, y, s, b), qb);
      kid(el_make(MT_GP, x, kk, a, s), gw);
      break;
    }
    default: {  // MT_M2UP / MT_M2UU: x unpaired: (type at x+1, state at x+1)
      const bool lastp = kind == MT_M2UP;
      const int tp = k / NS, s = k % NS;
      const mq *Pt = tp ? (lastp ? p.BP : p.M2PU) : (lastp ? p.M2UP : p.M2UU);
      const mq pw = Pt[cidx(n, x + 1, y) * BLK + s * NS + b];
      v = en[EN_EB] + p.chi[(size_t)x * 4 * BLK + (tp ? XUP : XUU) * BLK + a * NS + s] + pw;
      kid(el_make(tp ? (lastp ? MT_BP : MT_M2PU) : kind, x + 1, y, s, b), pw);
      break;
    }
  }
  if (nk) *nk = c;
  return mclamp(v);
}

// Lower bounds for groups of alternatives.  An element's index space splits
// into contiguous groups (a QB element: the stack, each bulge (L, side), the
// multiloop, the hairpin, each interior shape (l1, l2); a paired exterior
// element: each start kk of the last branch; a last multiloop branch: each
// kk), and each group has a lower bound on its alternatives' costs from
// per-cell minima of the tables, so that a group above the limit is skipped
// without evaluating its alternatives.  The minima are exact minima over a
// cell's 36 entries (or a position's), so a bound is never above a cost.
struct SubMins {
  mq *QB, *CH, *XI, *GP;  // [ncells]
  mq *tau, *chie;         // [n]: min of tau_p; min of chi_p over the XPP and XUP transitions
  mq *q5;                 // [n][6]: min over s and both tables of Q5U/Q5P[p][a0][s]
};

// one thread per cell, the first n threads also per position
__global__ void k_sub_mins(MfeDP p, SubMins mn) {
  const int n = p.n;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncells(n)) {
    const mq *qb = p.QB + c * BLK, *ch = p.CH + c * BLK, *xi = p.XI + c * BLK, *gp = p.GP + c * BLK;
    mq a = MQINF, b = MQINF, x = MQINF, g = MQINF;
    for (int e = 0; e < BLK; e++) {
      a = mmin(a, qb[e]);
      b = mmin(b, ch[e]);
      x = mmin(x, xi[e]);
      g = mmin(g, gp[e]);
    }
    mn.QB[c] = mclamp(a);
    mn.CH[c] = mclamp(b);
    mn.XI[c] = mclamp(x);
    mn.GP[c] = mclamp(g);
  }
  if (c < (size_t)n) {
    const mq *t = p.tau + c * BLK, *ch = p.chi + c * 4 * BLK;
    mq a = MQINF, e2 = MQINF;
    for (int e = 0; e < BLK; e++) {
      a = mmin(a, t[e]);
      e2 = mmin(e2, mmin(ch[XPP * BLK + e], ch[XUP * BLK + e]));
    }
    mn.tau[c] = mclamp(a);
    mn.chie[c] = mclamp(e2);
    for (int a0 = 0; a0 < NS; a0++) {
      mq v = MQINF;
      for (int s = 0; s < NS; s++)
        v = mmin(v, mmin(p.Q5U[c * BLK + a0 * NS + s], p.Q5P[c * BLK + a0 * NS + s]));
      mn.q5[c * NS + a0] = mclamp(v);
    }
  }
}

constexpr int SG_BULGE0 = 1, SG_ML = 1 + MAXLOOP * 2, SG_HP = SG_ML + 1, SG_IN0 = SG_HP + 1;
constexpr int SB_IN0 = SB_STACK + SB_BULGE + SB_ML + BLK;  // first interior-loop index of a QB element
constexpr mq MQ_NOBOUND = -MQINF;

__device__ __forceinline__ bool ext_paired(int4 E) { return (E.x & 255) == MT_EXT && E.y > 0 && ((E.x >> 8) & 255) >= NS; }

__device__ __forceinline__ int el_ngroups(const MfeDP &p, int4 E) {
  const int kind = E.x & 255;
  if (kind == MT_QB) return SG_IN0 + NINTERIOR;
  if (ext_paired(E)) return 1 + max(0, E.y - 4);
  if (kind == MT_BP) return max(0, E.z - E.y - 8);
  return 1;
}

// the group holding index k
__device__ __forceinline__ int el_group_of(const MfeDP &p, int4 E, int k) {
  const int kind = E.x & 255;
  if (kind == MT_QB) {
    if (k < SB_STACK) return 0;
    if (k < SB_STACK + SB_BULGE) return SG_BULGE0 + (k - SB_STACK) / BLK;
    if (k < SB_STACK + SB_BULGE + SB_ML) return SG_ML;
    if (k < SB_IN0) return SG_HP;
    return SG_IN0 + (k - SB_IN0) / (BLK * BLK);
  }
  if (ext_paired(E)) return k == 0 ? 0 : 1 + (k - 1) / (2 * BLK);
  if (kind == MT_BP) return k / NS;
  return 0;
}

// index range [k0, k1) of group g
__device__ __forceinline__ void el_group(const MfeDP &p, int4 E, int g, int &k0, int &k1) {
  const int kind = E.x & 255;
  if (kind == MT_QB) {
    if (g == 0) k0 = 0, k1 = SB_STACK;
    else if (g < SG_ML) k0 = SB_STACK + (g - SG_BULGE0) * BLK, k1 = k0 + BLK;
    else if (g == SG_ML) k0 = SB_STACK + SB_BULGE, k1 = k0 + SB_ML;
    else if (g == SG_HP) k0 = SB_STACK + SB_BULGE + SB_ML, k1 = SB_IN0;
    else k0 = SB_IN0 + (g - SG_IN0) * BLK * BLK, k1 = k0 + BLK * BLK;
  } else if (ext_paired(E)) {
    if (g == 0) k0 = 0, k1 = 1;
    else k0 = 1 + (g - 1) * 2 * BLK, k1 = k0 + 2 * BLK;
  } else if (kind == MT_BP) {
    k0 = g * NS, k1 = k0 + NS;
  } else {
    k0 = 0, k1 = el_count(p, E);
  }
}

// a lower bound on the cost of every alternative of group g (MQ_NOBOUND: none
// known); `outer` is the QB element's minimum over (u, v) of the closing
// pair's terms of a hairpin or interior loop
__device__ __forceinline__ mq el_group_lb(const MfeDP &p, const SubMins &mn, int4 E, int g, mq outer) {
  const int n = p.n, kind = E.x & 255, a = (E.x >> 8) & 255, x = E.y, y = E.z;
  const mq *en = p.en;
  if (kind == MT_QB) {
    const int i = x, j = y;
    if (g >= SG_BULGE0 && g < SG_ML) {
      const int L = 1 + (g - SG_BULGE0) / 2, side = (g - SG_BULGE0) & 1;
      if (side == 0) {
        const int l = j - 1 - L;
        if (l - (i + 1) < 4) return MQINF;
        return en[EN_BU + L] + mn.tau[i] + mn.QB[cidx(n, i + 1, l)] + mn.CH[cidx(n, l, j)];
      }
      const int kk = i + 1 + L;
      if ((j - 1) - kk < 4) return MQINF;
      return en[EN_BU + L] + mn.CH[cidx(n, i, kk)] + mn.QB[cidx(n, kk, j - 1)] + mn.tau[j - 1];
    }
    if (g >= SG_IN0) {
      if (outer >= MQHALF) return MQINF;
      int l1, l2;
      interior_shape(g - SG_IN0, l1, l2);
      const int kk = i + 1 + l1, l = j - 1 - l2;
      if (l - kk < 4) return MQINF;
      return outer + en[EN_IN + l1 + l2] + mn.CH[cidx(n, i + 1, kk - 1)] + mn.XI[cidx(n, kk - 1, l + 1)] +
             mn.CH[cidx(n, l + 1, j - 1)];
    }
    return MQ_NOBOUND;
  }
  if (ext_paired(E)) {
    if (g == 0) return MQ_NOBOUND;
    const int kk = g;
    return mn.q5[(size_t)(kk - 1) * NS + E.z] + mn.chie[kk - 1] + mn.QB[cidx(n, kk, x)];
  }
  if (kind == MT_BP) {
    const int kk = x + 5 + g;
    return en[EN_EC] + mn.GP[cidx(n, x, kk)] + mn.QB[cidx(n, kk, y)];
  }
  (void)a;
  return MQ_NOBOUND;
}

// One level of the depth-first search.  The pending list lives in one array
// kept in place: the frame's element was taken from position npend, and its
// children push their sub-elements from there on; leaving the frame puts the
// element back at npend, so that the list below a frame is its parent's
// again (each descendant restores the entry it took in turn).  The element's
// own decisions (codon states and the pair it fixes) do not depend on the
// alternative taken, so they are made when the frame is entered and undone
// (the positions it set, at most four) when it is left.
struct SubFrame {
  int4 elem;
  long long slack;    // what is left of the gap
  long long want;     // the element's table value
  int npend, cursor;  // pending elements below it; its next alternative
  int nch, ch[4];     // positions its decisions set
};

constexpr int SUB_RING = 512;  // frames kept in shared memory (the deepest ones), the rest in global memory
constexpr int SUB_NT = 256;    // threads of the search CTA (512 was slower: 4.23 against 4.13 s at 900 nt)
constexpr int SUB_NW = SUB_NT / 32;

struct SubArgs {
  MfeDP p;
  SubMins mn;
  mq gap;
  int max_out, pcap;
  int4 *pend;          // [pcap] pending elements
  mq *pendw;           // [pcap] their table values
  SubFrame *frames;    // [depth cap] frames pushed out of the ring
  int depth_cap;
  long long max_steps;
  unsigned long long max_ns;  // the enumeration stops (with an error) past this device time
  int32_t *codons, *partner;  // [max_out][m], [max_out][n]
  const int *sctab;           // single-codon layout: the codon table of traced_codon; else null
  long long *cost;            // [max_out]
  long long *count;           // [2]: configurations found (capped at max_out + 1), steps taken
};

// dynamic shared memory of k_mfe_subopt: the states and partners (2n ints),
// then the frame ring and its depth tags
__host__ __device__ constexpr size_t sub_smem(int n) {
  return ((size_t)2 * n * sizeof(int) + 15) / 16 * 16 + (size_t)SUB_RING * (sizeof(SubFrame) + sizeof(int));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

// The smallest k over the block for which ok holds (INT_MAX if none), k
// increasing with the thread index; one block barrier, the per-warp minima
// double-buffered by round parity.
__device__ __forceinline__ int block_first(bool ok, int k, int (*swmin)[SUB_NW], int &par) {
  const unsigned b = __ballot_sync(0xffffffffu, ok);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int kw = b ? __shfl_sync(0xffffffffu, k, __ffs(b) - 1) : INT_MAX;
  if (lane == 0) swmin[par][w] = kw;
  __syncthreads();
  int m = INT_MAX;
#pragma unroll
  for (int i = 0; i < SUB_NW; i++) m = min(m, swmin[par][i]);
  par ^= 1;
  return m;
}

// The element's own decisions into the states and partners (scs), the
// positions set recorded in the frame; a position already decided otherwise
// is an inconsistency (bit 4 of the error).
__device__ __forceinline__ void el_decide(int n, int4 E, int *scs, SubFrame &f, int &bad) {
  const int kind = E.x & 255, a = (E.x >> 8) & 255, b = (E.x >> 16) & 255, x = E.y, y = E.z;
  f.nch = 0;
  auto set = [&](int q, int v) {
    if (scs[q] >= 0) {
      if (scs[q] != v) bad = 4;
    } else {
      scs[q] = v;
      f.ch[f.nch++] = q;
    }
  };
  switch (kind) {
    case MT_EXT:
      if (x == 0) set(0, y);
      else if (a < NS) set(x, a);
      break;
    case MT_CH: set(x, a); break;
    case MT_QB:
      set(x, a);
      set(y, b);
      set(n + x, y);
      set(n + y, x);
      break;
    case MT_QMU: case MT_M2PU: set(y, b); break;
    case MT_M2UP: case MT_M2UU: set(x, a); break;
    default: break;
  }
}

__global__ void __launch_bounds__(SUB_NT) k_mfe_subopt(SubArgs s) {
  const MfeDP &p = s.p;
  const unsigned long long t0 = global_ns();
  const int n = p.n, t = threadIdx.x;
  extern __shared__ __align__(16) unsigned char sub_smem_raw[];
  int *scs = reinterpret_cast<int *>(sub_smem_raw);  // [n] state of each position, then [n] partner (-1: not yet)
  SubFrame *ring = reinterpret_cast<SubFrame *>(sub_smem_raw + ((size_t)2 * n * sizeof(int) + 15) / 16 * 16);
  int *rtag = reinterpret_cast<int *>(ring + SUB_RING);  // the frame index each ring slot holds
  __shared__ int sdepth, sbad, sdone, scur, swmin[2][SUB_NW];
  __shared__ int4 sE;
  __shared__ long long sfound, sslack, swant;
  __shared__ mq souter;
  __shared__ int swsum[SUB_NW], spref[SUB_NT + 1], sk0[SUB_NT];  // blockDim.x = SUB_NT
  const mq best = *p.best;
  for (int q = t; q < 2 * n; q += blockDim.x) scs[q] = -1;
  for (int q = t; q < SUB_RING; q += blockDim.x) rtag[q] = -1;
  __syncthreads();
  if (t == 0) {
    SubFrame f0;
    f0.elem = el_make(MT_TOP, 0, 0, 0, 0);
    f0.slack = s.gap;
    f0.want = best;
    f0.npend = 0;
    f0.cursor = 0;
    f0.nch = 0;
    ring[0] = f0;
    rtag[0] = 0;
    sE = f0.elem;
    sslack = f0.slack;
    swant = best;
    scur = 0;
    sdepth = 1;
    sbad = 0;
    sdone = 0;
    sfound = 0;
  }
  long long steps = 0;
  int par = 0;
  while (true) {
    __syncthreads();
    const int depth = sdepth;
    if (depth == 0 || sbad || sdone || best >= MQHALF) break;
    if (++steps > s.max_steps || (t == 0 && (steps & 255) == 0 && global_ns() - t0 > s.max_ns)) {
      if (t == 0) sbad = 2;  // bounded: the other threads see it at the next step
      if (steps > s.max_steps) break;
    }
    const int4 E = sE;
    const long long slack = sslack;
    const int cur = scur;
    const mq want = swant;
    const mq limit = want + slack;
    const int K = el_count(p, E), G = el_ngroups(p, E), kind = E.x & 255;
    // this thread's last evaluated alternative
    int mk = INT_MAX, mnk = 0;
    mq mc = MQINF;
    int4 mkids[3];
    mq mkw[3];
    int kf = -1;
    if (G == 1 && K - cur <= 32) {
      // at most 32 alternatives left: warp 0 alone scans and decides (warp
      // ballot, no block barrier); the other warps go on to the next step
      if ((t >> 5) != 0) continue;
      const int k = cur + (t & 31);
      bool ok = false;
      if (k < K) {
        mk = k;
        mc = el_alt(p, E, k, mkids, &mnk, mkw);
        ok = mc <= limit;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      kf = bal ? cur + __ffs(bal) - 1 : -1;
    } else if (G == 1) {  // one group: its alternatives one per thread
      for (int b0 = cur; b0 < K && kf < 0; b0 += blockDim.x) {
        const int k = b0 + t;
        bool ok = false;
        mk = INT_MAX;
        if (k < K) {
          mk = k;
          mc = el_alt(p, E, k, mkids, &mnk, mkw);
          ok = mc <= limit;
        }
        const int fk = block_first(ok, k, swmin, par);
        if (fk != INT_MAX) kf = fk;
      }
    } else {
      // a QB element's closing-pair minimum for the hairpin and interior bounds
      if (kind == MT_QB) {
        if (t == 0) souter = MQINF;
        __syncthreads();
        if (t < BLK) {
          const int i = E.y, j = E.z, a = (E.x >> 8) & 255, b = (E.x >> 16) & 255, u = t / NS, vv = t % NS;
          const mq o = p.tau[(size_t)i * BLK + a * NS + u] + p.tau[(size_t)(j - 1) * BLK + vv * NS + b] +
                       p.en[EN_TM + p.base[(i + 1) * NS + u] * 4 + p.base[(j - 1) * NS + vv]];
          atomicMin(&souter, mclamp(o));
        }
        __syncthreads();
      }
      const mq outer = kind == MT_QB ? souter : MQINF;
      // groups in chunks of one per thread; the live ones (bound within the
      // limit) are packed in ascending order and their indices scanned one
      // per thread
      const int gcur = cur < K ? el_group_of(p, E, cur) : G;
      for (int gb = gcur; gb < G && kf < 0; gb += blockDim.x) {
        const int g = gb + t;
        int k0 = 0, k1 = 0;
        if (g < G) {
          el_group(p, E, g, k0, k1);
          k0 = max(k0, cur);
          if (k0 < k1 && el_group_lb(p, s.mn, E, g, outer) > limit) k1 = k0;
        }
        const int len = max(0, k1 - k0);
        int incl = len;  // inclusive prefix of len: warp scans, then the warp totals
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if ((t & 31) >= o) incl += v;
        }
        if ((t & 31) == 31) swsum[t >> 5] = incl;
        __syncthreads();
        int wbase = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
          if (w < (t >> 5)) wbase += swsum[w];
          total += swsum[w];
        }
        spref[t] = wbase + incl - len;
        sk0[t] = k0;
        if (t == 0) spref[blockDim.x] = total;
        __syncthreads();
        for (int v0 = 0; v0 < total && kf < 0; v0 += blockDim.x) {
          const int v = v0 + t;
          int k = INT_MAX;
          bool ok = false;
          mk = INT_MAX;
          if (v < total) {
            int lo = 0, hi = blockDim.x;  // the last slot with spref <= v
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (spref[mid] <= v) lo = mid;
              else hi = mid;
            }
            k = sk0[lo] + (v - spref[lo]);
            mk = k;
            mc = el_alt(p, E, k, mkids, &mnk, mkw);
            ok = mc <= limit;
          }
          const int fk = block_first(ok, k, swmin, par);
          if (fk != INT_MAX) kf = fk;
        }
        __syncthreads();  // spref / sk0 / swsum reused by the next chunk
      }
    }
    // the search's bookkeeping, by one thread: the one that evaluated the
    // alternative taken, or thread 0 when none is left (the others wait at
    // the next step's barrier)
    const int fi = depth - 1;  // the current frame's index (always in the ring)
    SubFrame &h = ring[fi % SUB_RING];
    if (kf < 0) {
      if (t != 0) continue;
      for (int c = 0; c < h.nch; c++) scs[h.ch[c]] = -1;
      if (fi > 0) {
        s.pend[h.npend] = E;  // the parent's list again
        s.pendw[h.npend] = want;
        const int pi = fi - 1, ps = pi % SUB_RING;
        if (rtag[ps] != pi) {
          ring[ps] = s.frames[pi];
          rtag[ps] = pi;
        }
        sE = ring[ps].elem;
        sslack = ring[ps].slack;
        swant = ring[ps].want;
        scur = ring[ps].cursor;
      }
      sdepth = depth - 1;
      continue;
    }
    if (mk != kf) continue;
    h.cursor = kf + 1;
    const long long nslack = slack - (mc - want);
    const int np = h.npend;
    int m2 = np;
    for (int q = 0; q < mnk; q++) {
      if (m2 < s.pcap) {
        s.pend[m2] = mkids[q];
        s.pendw[m2] = mkw[q];
        m2++;
      } else {
        sbad = 5;
      }
    }
    if (m2 == 0) {  // complete: MFE + gap - slack
      const long long idx = sfound;
      if (idx < s.max_out) {
        for (int r = 0; r < p.m; r++) {
          const int c = traced_codon(p.cid, s.sctab, scs, r);
          if (c < 0) sbad = 6;
          s.codons[(size_t)idx * p.m + r] = c;
        }
        for (int q = 0; q < n; q++) s.partner[(size_t)idx * n + q] = scs[n + q];
        s.cost[idx] = best + (s.gap - nslack);
      }
      sfound = idx + 1;
      if (sfound > s.max_out) sdone = 1;
      scur = kf + 1;
      continue;
    }
    if (depth >= s.depth_cap) {
      sbad = 3;
      continue;
    }
    SubFrame g;
    g.elem = mnk > 0 ? mkids[mnk - 1] : s.pend[np - 1];
    g.want = mnk > 0 ? mkw[mnk - 1] : s.pendw[np - 1];
    g.npend = m2 - 1;
    g.slack = nslack;
    g.cursor = 0;
    int bad = 0;
    el_decide(n, g.elem, scs, g, bad);
    if (bad) sbad = bad;
    const int ci = fi + 1, cs = ci % SUB_RING;
    if (rtag[cs] >= 0 && rtag[cs] == ci - SUB_RING) s.frames[ci - SUB_RING] = ring[cs];  // a live ancestor
    ring[cs] = g;
    rtag[cs] = ci;
    sE = g.elem;
    sslack = nslack;
    swant = g.want;
    scur = 0;
    sdepth = depth + 1;
  }
  __syncthreads();
  if (t == 0) {
    s.count[0] = sfound;
    s.count[1] = steps;
    if (sbad) atomicOr(p.err, 1 << (8 + sbad));
  }
}

}  // namespace cf
