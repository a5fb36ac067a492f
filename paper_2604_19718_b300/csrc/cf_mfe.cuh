// cf_mfe.cuh -- minimum free energy over (codon sequence, structure): paper
// Section "Minimization" (Eq. min-problem), the zero-temperature limit of the
// partition function obtained by evaluating the same recursions in the
// min-sum (tropical) semiring instead of the sum-product one (SI
// "Generalization via evaluation algebras").
//
// Costs are exact integers in units of 2^-32 kcal/mol (int64): every
// elementary energy term, and every codon log-weight and codon-pair bonus
// converted to kcal/mol as -kT w, is rounded once to that grid; all
// recursions add these integers and take minima, so the result does not
// depend on the order of evaluation and equals, bit for bit, any other exact
// evaluation of the same model.  "Infinite" cost (no configuration) is
// MQINF; sums of up to three infinite terms stay below 2^62, and every stored
// value at or above MQINF / 2 is stored as MQINF.
//
// Tables (6x6 blocks over the codon states at the two ends, diagonal-major as
// the partition-function tables; rows and columns beyond the state counts are
// MQINF), for the interval [x, y]:
//   CH        chain of transfer costs x -> y
//   QB        x pairs with y
//   XI        the pair (x+1, y-1) extended by one base on each side with its
//             inner mismatch, as seen from an enclosing interior loop
//   QMP, QMU  multiloop segment with >= 1 branch, the first starting at x,
//             last base y paired (QMP) or unpaired (QMU)
//   GP[x][k]  QMP/QMU[x][k-1] followed by the transition into a branch at k
//   BP        >= 2 branches, first at x, last ending at y (= QM2 with both
//             ends paired); M2PU, M2UP, M2UU the other end types
//   Q5U/Q5P   exterior prefix [0, y], y unpaired / paired; GX[k] as GP
// Partial minima kept for three diagonals only (a ring):
//   W_L[x][y] L = 2..30  min over inner pairs whose interior loop has L
//                        unpaired bases in total: CH . XI . CH
//   R_L[x][y] L = 1..31  QB[x][y-L] . CH[y-L][y]   (3' bulges)
//   F_L[x][y] L = 1..31  CH[x][x+L] . QB[x+L][y]   (5' bulges)
// Each is a one-step recursion along a row or column, so a cell needs O(30)
// block products instead of enumerating its loops.  The only O(n) sums are
// BP[x][y] = c + min_k GP[x][k] . QB[k][y] and the exterior split points,
// summed by k_mfe_bif from diagonals <= d - 4.
#pragma once
#include <climits>

#include "cf_common.cuh"

namespace cf {

typedef long long mq;
constexpr mq MQINF = 0x1010101010101010LL;  // the byte pattern cudaMemset(0x10) writes
constexpr mq MQHALF = MQINF / 2;
constexpr int MW = 29;   // W_L, L = 2..30
constexpr int MRF = 31;  // R_L and F_L, L = 1..31
// threads per cell of the light kernel: each thread's one-step tasks run
// one after the other, each waiting on its table reads, so more threads per
// cell shorten the cell (measured, MFE pass at 900 / 3000 nt: 128 threads
// 58.4 / 1310 ms, 256 52.5 / 968 ms, 512 61.2 / 1098 ms)
constexpr int MFE_NT = 256;

__device__ __forceinline__ mq mclamp(mq v) { return v >= MQHALF ? MQINF : v; }
__device__ __forceinline__ mq mmin(mq a, mq b) { return a < b ? a : b; }

struct MfeDP {
  int n, m;
  const int *Mp, *base, *cid;  // [n], [n*6], [n*6]
  const mq *tau;               // [n][36] transfer costs p -> p+1
  const mq *chi;               // [n][4][36] typed transition costs, index (type at p) * 2 + (type at p+1)
  const mq *en;                // [EN_N] costs, layout of the energy-factor vector
  const mq *hq;                // [n + 2] hairpin cost by loop length
  const mq *u0;                // [6] cost of residue 0's codon weights
  mq *CH, *QB, *XI, *QMP, *QMU, *GP, *BP, *M2PU, *M2UP, *M2UU;  // [ncells][36]
  mq *W, *R, *F;               // rings [3][n][MW or MRF][36]
  mq *Q5U, *Q5P, *GX, *X5;     // [n][36]
  mq *best;                    // [1]
  int *err;
};

__device__ __forceinline__ const mq *mblk(const mq *t, int n, int x, int y) { return t + cidx(n, x, y) * BLK; }
__device__ __forceinline__ mq *mblkw(mq *t, int n, int x, int y) { return t + cidx(n, x, y) * BLK; }
__device__ __forceinline__ mq *mring(mq *t, int nb, int n, int d, int x, int l) {
  return t + (((size_t)(d % 3) * n + x) * nb + l) * BLK;
}

// min over s of A[a][s] + B[s][b] (padded blocks: padding is MQINF)
__device__ __forceinline__ mq mm2(const mq *A, const mq *B, int a, int b) {
  mq v = MQINF;
#pragma unroll
  for (int s = 0; s < NS; s++) v = mmin(v, A[a * NS + s] + B[s * NS + b]);
  return v;
}

// ---------------------------------------------------------------- costs of the transfers
// tau_q[a][b] = 0 on the diagonal inside a residue; across the boundary from
// residue r to r+1 (q = 3r + 2): cost(lw[r+1][b]) + cost(pb[c_a][c_b]); the
// typed transitions add the dangle costs of a paired end (3' dangle of a
// paired base at q, 5' dangle of a paired base at q+1).  One thread per q.
// Single-codon layout (smap, sc1 non-null): tau_3r joins a first base to the
// (first, second) pairs that start with it at cost 0, tau_3r+1 joins a pair
// to a third base at the cost of the codon's weight (smap[r][slot] packs the
// codon's two states), tau_3r+2 joins any two states at cost 0 (the layout
// has no pair bonuses), and residue 0's states cost nothing.
__device__ __forceinline__ mq mq_weight(double kT, double w) { return llround(__dmul_rn(-__dmul_rn(kT, w), 4294967296.0)); }

__global__ void k_mfe_transfers(int n, const int *Mp, const int *base, const int *cid, const mq *en, double kT,
                                const double *lw, const double *pb, mq *tau, mq *chi, mq *u0,
                                const int *smap = nullptr, const int *sc1 = nullptr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0)
    for (int a = 0; a < NS; a++) u0[a] = a < Mp[0] ? (smap ? 0 : mq_weight(kT, lw[a])) : MQINF;
  if (q >= n) return;
  const int Ma = Mp[q], Mb = q + 1 < n ? Mp[q + 1] : 0;
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) {
      const int e = a * NS + b;
      mq t = MQINF, d3 = 0, d5 = 0;
      if (a < Ma && b < Mb) {
        if (smap) {
          const int r = q / 3;
          if (q % 3 == 0) {
            t = base[(size_t)q * NS + a] == sc1[(size_t)(q + 1) * NS + b] ? 0 : MQINF;
          } else if (q % 3 == 1) {
            for (int s2 = 0; s2 < 6; s2++) {
              const int sm = smap[(size_t)r * 6 + s2];
              if (sm >= 0 && (sm & 15) == a && ((sm >> 4) & 15) == b) t = mq_weight(kT, lw[(size_t)r * 6 + s2]);
            }
          } else {
            t = 0;
          }
        } else if (q % 3 != 2) {
          t = a == b ? 0 : MQINF;
        } else {
          const int r1 = (q + 1) / 3;
          t = mq_weight(kT, lw[(size_t)r1 * 6 + b]) +
              mq_weight(kT, pb[61 * cid[(size_t)q * NS + a] + cid[(size_t)(q + 1) * NS + b]]);
        }
        const int x0 = base[(size_t)q * NS + a], y0 = base[(size_t)(q + 1) * NS + b];
        d3 = en[EN_D3 + x0 * 4 + y0];
        d5 = en[EN_D5 + y0 * 4 + x0];
      }
      tau[(size_t)q * BLK + e] = t;
      mq *c = chi + (size_t)q * 4 * BLK;
      c[XUU * BLK + e] = t;
      c[XUP * BLK + e] = t >= MQHALF ? MQINF : t + d5;
      c[XPU * BLK + e] = t >= MQHALF ? MQINF : t + d3;
      c[XPP * BLK + e] = t >= MQHALF ? MQINF : t + d3 + d5;
    }
}

// ---------------------------------------------------------------- light kernel
// One 128-thread CTA per cell (x, y) of diagonal d.  Phase A: every block that
// reads earlier diagonals only (one task per block entry, tasks dealt to the
// threads); phase B: QB and XI; phase C: QMP (needs QB and BP) and the
// exterior Q5P; then every result is written out.
enum : int {
  MO_CH = 0, MO_R = 1, MO_F = MO_R + MRF, MO_W = MO_F + MRF,  // W_L, L = 3..30 at MO_W + L - 3
  MO_S = MO_W + 28, MO_STK, MO_B3, MO_B5, MO_MLU, MO_MLP, MO_XIP, MO_QMU, MO_GP, MO_M2PU, MO_M2UP, MO_M2UU,
  MO_Q5U, MO_GX, MO_Q5P3, MO_N
};

__device__ __forceinline__ mq mfe_task(const MfeDP &p, int op, int x, int y, int d, int a, int b) {
  const int n = p.n;
  const mq *en = p.en;
  const mq *tx = p.tau + (size_t)x * BLK, *ty1 = d >= 1 ? p.tau + (size_t)(y - 1) * BLK : nullptr;
  if (op == MO_CH) {
    if (d == 0) return (a == b && a < p.Mp[x]) ? 0 : MQINF;
    return mm2(tx, mblk(p.CH, n, x + 1, y), a, b);
  }
  if (op < MO_F) {  // R_L[x][y] = R_{L-1}[x][y-1] . tau_{y-1}, R_1 = QB[x][y-1] . tau_{y-1}
    const int L = op - MO_R + 1;
    if (d - L < 4) return MQINF;
    const mq *A = L == 1 ? mblk(p.QB, n, x, y - 1) : mring(p.R, MRF, n, d - 1, x, L - 2);
    return mm2(A, ty1, a, b);
  }
  if (op < MO_W) {  // F_L[x][y] = tau_x . F_{L-1}[x+1][y], F_1 = tau_x . QB[x+1][y]
    const int L = op - MO_F + 1;
    if (d - L < 4) return MQINF;
    const mq *B = L == 1 ? mblk(p.QB, n, x + 1, y) : mring(p.F, MRF, n, d - 1, x + 1, L - 2);
    return mm2(tx, B, a, b);
  }
  if (op < MO_S) {  // W_L[x][y] = min(tau_x . W_{L-1}[x+1][y], XI[x][y-L+2] . CH[y-L+2][y])
    const int L = op - MO_W + 3;
    if (L > d - 4) return MQINF;
    const int yl = y - L + 2;
    return mmin(mm2(tx, mring(p.W, MW, n, d - 1, x + 1, L - 3), a, b),
                mm2(mblk(p.XI, n, x, yl), mblk(p.CH, n, yl, y), a, b));
  }
  const int xb = p.base[x * NS + a], yb = p.base[y * NS + b];
  switch (op) {
    case MO_S: {  // (a, b) = states at x+1, y-1: hairpin and interior loops closed by (x, y)
      if (d < 4) return MQINF;
      mq v = p.hq[d - 1] + mblk(p.CH, n, x + 1, y - 1)[a * NS + b];
      const int Lm = min(MAXLOOP, d - 6);
      for (int L = 2; L <= Lm; L++) v = mmin(v, en[EN_IN + L] + mring(p.W, MW, n, d - 2, x + 1, L - 2)[a * NS + b]);
      return v + en[EN_TM + p.base[(x + 1) * NS + a] * 4 + p.base[(y - 1) * NS + b]];
    }
    case MO_STK: {  // stacked pair (x+1, y-1)
      if (d < 6) return MQINF;
      const int po = pair_type(xb, yb);
      if (po < 0) return MQINF;
      const mq *Qi = mblk(p.QB, n, x + 1, y - 1);
      mq v = MQINF;
      for (int a2 = 0; a2 < NS; a2++)
        for (int b2 = 0; b2 < NS; b2++) {
          const mq q = Qi[a2 * NS + b2];
          if (q >= MQHALF) continue;
          const int pi = pair_type(p.base[(x + 1) * NS + a2], p.base[(y - 1) * NS + b2]);
          if (pi < 0) continue;
          v = mmin(v, tx[a * NS + a2] + q + ty1[b2 * NS + b] + en[EN_STK + po * 6 + pi]);
        }
      return v;
    }
    case MO_B3: {  // (a, b) = states at x+1, y: min over 3' bulge sizes of Bu(L) + R_{L+1}[x+1][y]
      mq v = MQINF;
      const int Lm = min(MAXLOOP, d - 6);
      for (int L = 1; L <= Lm; L++) v = mmin(v, en[EN_BU + L] + mring(p.R, MRF, n, d - 1, x + 1, L)[a * NS + b]);
      return v;
    }
    case MO_B5: {  // (a, b) = states at x, y-1: min over 5' bulge sizes of Bu(L) + F_{L+1}[x][y-1]
      mq v = MQINF;
      const int Lm = min(MAXLOOP, d - 6);
      for (int L = 1; L <= Lm; L++) v = mmin(v, en[EN_BU + L] + mring(p.F, MRF, n, d - 1, x, L)[a * NS + b]);
      return v;
    }
    case MO_MLU:
    case MO_MLP: {  // (a, b) = states at x, y-1: chi_x[(a,P) -> t] . QM2_{t t'}[x+1][y-1], t' = U / P
      if (d < 11) return MQINF;
      const int tp = op == MO_MLP;
      const mq *cx = p.chi + (size_t)x * 4 * BLK;
      const mq *QU = mblk(tp ? p.M2UP : p.M2UU, n, x + 1, y - 1), *QP = mblk(tp ? p.BP : p.M2PU, n, x + 1, y - 1);
      return mmin(mm2(cx + XPU * BLK, QU, a, b), mm2(cx + XPP * BLK, QP, a, b));
    }
    case MO_XIP:  // (a, b) = states at x, y-1: tau_x . QB[x+1][y-1]
      if (d < 6) return MQINF;
      return mm2(tx, mblk(p.QB, n, x + 1, y - 1), a, b);
    case MO_QMU: {  // last base y unpaired after >= 1 branch
      if (d < 5) return MQINF;
      const mq *c = p.chi + (size_t)(y - 1) * 4 * BLK;
      return en[EN_EB] + mmin(mm2(mblk(p.QMU, n, x, y - 1), ty1, a, b), mm2(mblk(p.QMP, n, x, y - 1), c + XPU * BLK, a, b));
    }
    case MO_GP: {  // transition into a branch starting at y
      if (d < 5) return MQINF;
      const mq *c = p.chi + (size_t)(y - 1) * 4 * BLK;
      return mmin(mm2(mblk(p.QMU, n, x, y - 1), c + XUP * BLK, a, b), mm2(mblk(p.QMP, n, x, y - 1), c + XPP * BLK, a, b));
    }
    case MO_M2PU: {
      if (d < 10) return MQINF;
      const mq *c = p.chi + (size_t)(y - 1) * 4 * BLK;
      return en[EN_EB] + mmin(mm2(mblk(p.M2PU, n, x, y - 1), ty1, a, b), mm2(mblk(p.BP, n, x, y - 1), c + XPU * BLK, a, b));
    }
    case MO_M2UP: {
      if (d < 10) return MQINF;
      const mq *c = p.chi + (size_t)x * 4 * BLK;
      return en[EN_EB] + mmin(mm2(tx, mblk(p.M2UP, n, x + 1, y), a, b), mm2(c + XUP * BLK, mblk(p.BP, n, x + 1, y), a, b));
    }
    case MO_M2UU: {
      if (d < 10) return MQINF;
      const mq *c = p.chi + (size_t)x * 4 * BLK;
      return en[EN_EB] + mmin(mm2(tx, mblk(p.M2UU, n, x + 1, y), a, b), mm2(c + XUP * BLK, mblk(p.M2PU, n, x + 1, y), a, b));
    }
    case MO_Q5U: {  // exterior prefix [0, d], d unpaired (cell x = 0 only)
      if (x != 0) return MQINF;
      if (d == 0) return (a == b && a < p.Mp[0]) ? 0 : MQINF;
      const mq *c = p.chi + (size_t)(d - 1) * 4 * BLK;
      return mmin(mm2(p.Q5U + (size_t)(d - 1) * BLK, ty1, a, b), mm2(p.Q5P + (size_t)(d - 1) * BLK, c + XPU * BLK, a, b));
    }
    case MO_GX: {
      if (x != 0 || d == 0) return MQINF;
      const mq *c = p.chi + (size_t)(d - 1) * 4 * BLK;
      return mmin(mm2(p.Q5U + (size_t)(d - 1) * BLK, c + XUP * BLK, a, b),
                  mm2(p.Q5P + (size_t)(d - 1) * BLK, c + XPP * BLK, a, b));
    }
    case MO_Q5P3: {  // exterior split points k = 1..3 (QB[k][d] on diagonals d-1..d-3)
      if (x != 0) return MQINF;
      mq v = MQINF;
      for (int k = 1; k <= 3 && k <= d - 4; k++) v = mmin(v, mm2(p.GX + (size_t)k * BLK, mblk(p.QB, n, k, d), a, b));
      return v;
    }
  }
  return MQINF;
}

// Launched by a programmatic edge from the light kernel of d - 1: every task
// reads diagonals up to d - 1, so the kernel waits for its predecessor first
// (the launch itself overlaps the predecessor's end).
// MINB CTAs per SM: five (48 registers) up to MFE_BIF2_MAXN nt, four (64
// registers) beyond, where the bifurcation kernel needs the room (measured,
// against no bound, 62 registers: 900 nt 52.5 -> 50.2 ms with five, 3000 nt
// 970 -> 1009 ms with five, 935 ms with four)
template <int MINB>
__global__ void __launch_bounds__(MFE_NT, MINB) k_mfe_light(MfeDP p, int d) {
  __shared__ mq O[MO_N][BLK];
  __shared__ mq QBs[BLK], XIs[BLK];
  const int t = threadIdx.x, n = p.n;
  const int x = blockIdx.x, y = x + d;
  griddep_wait();
  griddep_launch_dependents();
  for (int task = t; task < MO_N * BLK; task += MFE_NT) {
    const int op = task / BLK, e = task % BLK;
    O[op][e] = mclamp(mfe_task(p, op, x, y, d, e / NS, e % NS));
  }
  __syncthreads();
  const mq *en = p.en;
  if (t < 2 * BLK) {
    const int e = t % BLK, a = e / NS, b = e % NS;
    const mq *tx = p.tau + (size_t)x * BLK;
    mq v = MQINF;
    if (t < BLK) {  // QB
      if (d >= 4 && a < p.Mp[x] && b < p.Mp[y] && pair_type(p.base[x * NS + a], p.base[y * NS + b]) >= 0) {
        const mq *ty1 = p.tau + (size_t)(y - 1) * BLK, *cy = p.chi + (size_t)(y - 1) * 4 * BLK;
        for (int u = 0; u < NS; u++) {
          const mq l = tx[a * NS + u];
          if (l >= MQHALF) continue;
          for (int w = 0; w < NS; w++) v = mmin(v, l + O[MO_S][u * NS + w] + ty1[w * NS + b]);
        }
        v = mmin(v, O[MO_STK][e]);
        for (int s = 0; s < NS; s++) {
          v = mmin(v, tx[a * NS + s] + O[MO_B3][s * NS + b]);
          v = mmin(v, O[MO_B5][a * NS + s] + ty1[s * NS + b]);
          v = mmin(v, en[EN_EA] + en[EN_EC] + O[MO_MLU][a * NS + s] + cy[XUP * BLK + s * NS + b]);
          v = mmin(v, en[EN_EA] + en[EN_EC] + O[MO_MLP][a * NS + s] + cy[XPP * BLK + s * NS + b]);
        }
      }
      QBs[e] = mclamp(v);
    } else {  // XI: inner mismatch tm[base at y][base at x]
      if (d >= 6 && a < p.Mp[x] && b < p.Mp[y]) {
        const mq *ty1 = p.tau + (size_t)(y - 1) * BLK;
        v = mm2(O[MO_XIP], ty1, a, b) + en[EN_TM + p.base[y * NS + b] * 4 + p.base[x * NS + a]];
      }
      XIs[e] = mclamp(v);
    }
  }
  __syncthreads();
  // write-out: one thread per entry and block
  const size_t c = cidx(n, x, y) * BLK;
  for (int task = t; task < 10 * BLK; task += MFE_NT) {
    const int k = task / BLK, e = task % BLK;
    switch (k) {
      case 0: p.CH[c + e] = O[MO_CH][e]; break;
      case 1: p.QB[c + e] = QBs[e]; break;
      case 2: p.XI[c + e] = XIs[e]; break;
      case 3: p.QMP[c + e] = d >= 4 ? mclamp(mmin(en[EN_EC] + QBs[e], p.BP[c + e])) : MQINF; break;
      case 4: p.QMU[c + e] = O[MO_QMU][e]; break;
      case 5: p.GP[c + e] = O[MO_GP][e]; break;
      case 6: p.M2PU[c + e] = O[MO_M2PU][e]; break;
      case 7: p.M2UP[c + e] = O[MO_M2UP][e]; break;
      case 8: p.M2UU[c + e] = O[MO_M2UU][e]; break;
      case 9:
        if (x == 0) {
          p.Q5U[(size_t)d * BLK + e] = O[MO_Q5U][e];
          p.GX[(size_t)d * BLK + e] = O[MO_GX][e];
          p.Q5P[(size_t)d * BLK + e] = mclamp(mmin(mmin(QBs[e], O[MO_Q5P3][e]), d >= 8 ? p.X5[(size_t)d * BLK + e] : MQINF));
        }
        break;
    }
  }
  for (int task = t; task < (MW + 2 * MRF) * BLK; task += MFE_NT) {
    const int k = task / BLK, e = task % BLK;
    if (k < MW) mring(p.W, MW, n, d, x, k)[e] = k == 0 ? XIs[e] : O[MO_W + k - 1][e];
    else if (k < MW + MRF) mring(p.R, MRF, n, d, x, k - MW)[e] = O[MO_R + k - MW][e];
    else mring(p.F, MRF, n, d, x, k - MW - MRF)[e] = O[MO_F + k - MW - MRF][e];
  }
}

// ---------------------------------------------------------------- bifurcation
// BP[x][y] = c + min_{k = x+5..y-4} GP[x][k] . QB[k][y] and, for the last
// cell of the launch, the exterior X5[d] = min_{k = 4..d-4} GX[k] . QB[k][d].
// Inputs lie on diagonals <= d - 4.  wpc warps per cell (1, 2, 4 or 8, chosen
// per diagonal so that a long diagonal's few cells still fill the SMs), lanes
// and warps over the split points, then a warp minimum per entry and, for
// wpc > 1, the minimum of the cell's warps in shared memory (integer minima:
// the same result in any order).
// MINB CTAs per SM: two (128 registers) up to MFE_BIF2_MAXN nt, one beyond
// (measured with one warp per cell: 900 nt 95.9 -> 79.8 ms with two, 3000 nt
// 1339 -> 1443 ms)
constexpr int MFE_BIF2_MAXN = 2000;
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_mfe_bif(MfeDP p, int d, int wpc) {
  __shared__ mq red[8][BLK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, n = p.n;
  const int sub = w % wpc;
  const int x = blockIdx.x * (8 / wpc) + w / wpc;
  const bool valid = x <= n - d;
  const bool ext = x == n - d;
  const int y = ext ? d : x + d;
  mq acc[BLK];
#pragma unroll
  for (int e = 0; e < BLK; e++) acc[e] = MQINF;
  if (valid) {
    const int k0 = ext ? 4 : x + 5, k1 = y - 4;
    for (int k = k0 + sub * 32 + lane; k <= k1; k += 32 * wpc) {
      const mq *A = ext ? p.GX + (size_t)k * BLK : mblk(p.GP, n, x, k);
      const mq *B = mblk(p.QB, n, k, y);
#pragma unroll
      for (int s = 0; s < NS; s++) {
        mq bv[NS], av[NS];
#pragma unroll
        for (int j = 0; j < NS; j++) {
          bv[j] = __ldg(B + s * NS + j);
          av[j] = __ldg(A + j * NS + s);
        }
#pragma unroll
        for (int a = 0; a < NS; a++)
#pragma unroll
          for (int b = 0; b < NS; b++) acc[a * NS + b] = mmin(acc[a * NS + b], av[a] + bv[b]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < BLK; e++) {
    mq v = acc[e];
#pragma unroll
    for (int o = 16; o; o >>= 1) v = mmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    acc[e] = v;
  }
  const mq c = ext ? 0 : p.en[EN_EC];
  mq *dst = !valid ? nullptr : ext ? p.X5 + (size_t)d * BLK : mblkw(p.BP, n, x, y);
  if (wpc == 1) {  // uniform over the launch
    if (valid) {
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if (lane == (e & 31)) dst[e] = mclamp(acc[e] + c);
    }
    return;
  }
#pragma unroll
  for (int e = 0; e < BLK; e++)
    if (lane == (e & 31)) red[w][e] = acc[e];
  __syncthreads();
  if (valid && sub == 0)
    for (int e = lane; e < BLK; e += 32) {
      mq v = red[w][e];
      for (int j = 1; j < wpc; j++) v = mmin(v, red[w + j][e]);
      dst[e] = mclamp(v + c);
    }
}

__global__ void k_mfe_final(MfeDP p) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = p.n;
  mq best = MQINF;
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) {
      const mq u = p.Q5U[(size_t)(n - 1) * BLK + a * NS + b], q = p.Q5P[(size_t)(n - 1) * BLK + a * NS + b];
      best = mmin(best, p.u0[a] + mmin(u, q));
    }
  *p.best = mclamp(best);
}

// ---------------------------------------------------------------- traceback
// One CTA follows the minimum back through the tables.  At every element the
// alternatives are enumerated in a fixed order (stated below per element) and
// the first whose cost equals the element's value is taken: the threads test
// 256 alternatives at a time and the smallest matching index wins.  Interior
// loops are enumerated directly (their partial minima W were kept for three
// diagonals only); every other alternative is a stored table entry.
enum : int { MT_EXT = 0, MT_QB, MT_CH, MT_QMP, MT_QMU, MT_GP, MT_BP, MT_M2PU, MT_M2UP, MT_M2UU };

struct MfeTrace {
  MfeDP p;
  int4 *stack;   // [cap] (kind | a << 8 | b << 16, x, y, unused)
  int cap;
  int *state;    // [n] codon state per position
  int32_t *codons, *partner;
  const int *sctab;  // single-codon layout: [m][36] codon | (state at 3r) << 8 of the states at 3r+1, 3r+2; else null
};

// the codon of residue r from the traced states: the state at 3r (codon
// states), or, in the single-codon layout, the states at 3r+1 and 3r+2
// (checked against the state at 3r); -1 if they do not form one
__device__ __forceinline__ int traced_codon(const int *cid, const int *sctab, const int *state, int r) {
  const int q = 3 * r;
  if (!sctab) return state[q] >= 0 ? cid[q * NS + state[q]] : -1;
  const int a1 = state[q + 1], a2 = state[q + 2];
  const int e = (a1 >= 0 && a2 >= 0) ? sctab[(size_t)r * BLK + a1 * NS + a2] : -1;
  return (e >= 0 && state[q] == (e >> 8)) ? (e & 255) : -1;
}

template <typename F>
__device__ int cta_first(int K, mq target, const F &cost, int *sfirst) {
  for (int b0 = 0; b0 < K; b0 += blockDim.x) {
    if (threadIdx.x == 0) *sfirst = INT_MAX;
    __syncthreads();
    const int k = b0 + (int)threadIdx.x;
    if (k < K && cost(k) == target) atomicMin(sfirst, k);
    __syncthreads();
    const int f = *sfirst;
    __syncthreads();
    if (f != INT_MAX) return f;
  }
  return -1;
}

// the 435 interior loop shapes (l1, l2 >= 1, l1 + l2 <= 30), by l1 then l2:
// the shapes with l1 = a + 1 start at index a (59 - a) / 2, so a is the
// smaller root of a^2 - 59 a + 2 q = 0 rounded down (corrected by one
// where the binary32 square root lands on the other side)
__device__ __forceinline__ void interior_shape(int q, int &l1, int &l2) {
  static_assert(MAXLOOP == 30, "closed form for loops of at most 30 bases");
  int a = (int)((59.0f - sqrtf((float)(3481 - 8 * q))) * 0.5f);
  if (a * (59 - a) / 2 > q) a--;
  else if ((a + 1) * (58 - a) / 2 <= q) a++;
  l1 = a + 1;
  l2 = 1 + q - a * (59 - a) / 2;
}
constexpr int NINTERIOR = 435;

__global__ void __launch_bounds__(256) k_mfe_trace(MfeTrace T) {
  __shared__ int sfirst, sp, sbad;
  const MfeDP &p = T.p;
  const int n = p.n, t = threadIdx.x;
  const mq *en = p.en;
  for (int q = t; q < n; q += blockDim.x) {
    T.state[q] = -1;
    T.partner[q] = -1;
  }
  if (t == 0) {
    sp = 0;
    sbad = 0;
  }
  __syncthreads();
  auto fail = [&](int code) {
    if (t == 0) {
      sbad = code;
      atomicOr(p.err, 1 << 4);
    }
  };
  auto push = [&](int kind, int x, int y, int a, int b) {
    if (t == 0) {
      if (sp < T.cap) T.stack[sp++] = make_int4(kind | (a << 8) | (b << 16), x, y, 0);
      else sbad = 99;
    }
  };
  auto setst = [&](int q, int a) {
    if (t == 0) {
      if (T.state[q] >= 0 && T.state[q] != a) sbad = 98;
      T.state[q] = a;
    }
  };
  const mq best = *p.best;
  {  // top: residue 0's state a and the port of position n-1, (a, type, b) ascending
    const int Ml = p.Mp[n - 1];
    const int k = cta_first(NS * 2 * Ml, best, [&](int k) {
      const int a = k / (2 * Ml), r = k % (2 * Ml), tp = r / Ml, b = r % Ml;
      return p.u0[a] + (tp ? p.Q5P : p.Q5U)[(size_t)(n - 1) * BLK + a * NS + b];
    }, &sfirst);
    if (best >= MQHALF || k < 0) fail(1);
    else {
      const int a = k / (2 * Ml), r = k % (2 * Ml);
      push(MT_EXT, n - 1, a, r % Ml + NS * (r / Ml), 0);
    }
  }
  __syncthreads();
  for (int guard = 0; guard < 64 * n + 64; guard++) {
    if (sp == 0 || sbad) break;
    const int4 it = T.stack[sp - 1];
    __syncthreads();
    if (t == 0) sp--;
    const int kind = it.x & 255, a = (it.x >> 8) & 255, b = (it.x >> 16) & 255, x = it.y, y = it.z;
    if (kind == MT_EXT) {  // x = j, y = a0, a = port at j
      const int j = x, a0 = y, port = a;
      const mq want = (port < NS ? p.Q5U : p.Q5P)[(size_t)j * BLK + a0 * NS + port % NS];
      if (j == 0) {
        if (port != a0) fail(2);
        setst(0, a0);
      } else if (port < NS) {  // j unpaired: (type, state) at j-1
        const int bb = port, Mp = p.Mp[j - 1];
        const mq *c = p.chi + (size_t)(j - 1) * 4 * BLK;
        const int k = cta_first(2 * Mp, want, [&](int k) {
          const int tp = k / Mp, s = k % Mp;
          return (tp ? p.Q5P : p.Q5U)[(size_t)(j - 1) * BLK + a0 * NS + s] + c[(tp ? XPU : XUU) * BLK + s * NS + bb];
        }, &sfirst);
        if (k < 0) fail(3);
        else {
          setst(j, bb);
          push(MT_EXT, j - 1, a0, k % Mp + NS * (k / Mp), 0);
        }
      } else {  // j paired: the branch (0, j), else the last branch (k, j), k ascending, (type at k-1, state at k-1, state at k)
        const int bb = port - NS;
        if (p.QB[cidx(n, 0, j) * BLK + a0 * NS + bb] == want) {
          push(MT_QB, 0, j, a0, bb);
        } else {
          const int k = cta_first(max(0, j - 4) * 2 * NS * NS, want, [&](int q) {
            const int kk = 1 + q / (2 * NS * NS), r = q % (2 * NS * NS), tp = r / (NS * NS), s1 = (r / NS) % NS,
                      s = r % NS;
            const mq *c = p.chi + (size_t)(kk - 1) * 4 * BLK;
            return (tp ? p.Q5P : p.Q5U)[(size_t)(kk - 1) * BLK + a0 * NS + s1] + c[(tp ? XPP : XUP) * BLK + s1 * NS + s] +
                   p.QB[cidx(n, kk, j) * BLK + s * NS + bb];
          }, &sfirst);
          if (k < 0) fail(4);
          else {
            const int kk = 1 + k / (2 * NS * NS), r = k % (2 * NS * NS), tp = r / (NS * NS), s1 = (r / NS) % NS, s = r % NS;
            push(MT_QB, kk, j, s, bb);
            push(MT_EXT, kk - 1, a0, s1 + NS * tp, 0);
          }
        }
      }
    } else if (kind == MT_CH) {  // chain x..y with end states a, b: next states in order
      if (t == 0) {
        int cur = a;
        T.state[x] = (T.state[x] >= 0 && T.state[x] != a) ? (sbad = 97, a) : a;
        for (int q = x; q < y && !sbad; q++) {
          const mq want = p.CH[cidx(n, q, y) * BLK + cur * NS + b];
          int nx = -1;
          for (int s = 0; s < NS && nx < 0; s++)
            if (p.tau[(size_t)q * BLK + cur * NS + s] + p.CH[cidx(n, q + 1, y) * BLK + s * NS + b] == want) nx = s;
          if (nx < 0) sbad = 5;
          else {
            cur = nx;
            if (T.state[q + 1] >= 0 && T.state[q + 1] != cur) sbad = 96;
            T.state[q + 1] = cur;
          }
        }
      }
    } else if (kind == MT_QB) {
      const int i = x, j = y;
      const mq want = p.QB[cidx(n, i, j) * BLK + a * NS + b];
      if (t == 0) {
        T.partner[i] = j;
        T.partner[j] = i;
      }
      setst(i, a);
      setst(j, b);
      const mq *ti = p.tau + (size_t)i * BLK, *tj1 = p.tau + (size_t)(j - 1) * BLK;
      const int d = j - i;
      bool done = false;
      // 1. stack: (a2, b2) ascending
      if (d >= 6) {
        const int po = pair_type(p.base[i * NS + a], p.base[j * NS + b]);
        const int k = cta_first(BLK, want, [&](int k) {
          const int a2 = k / NS, b2 = k % NS;
          const int pi = pair_type(p.base[(i + 1) * NS + a2], p.base[(j - 1) * NS + b2]);
          if (po < 0 || pi < 0) return MQINF;
          return ti[a * NS + a2] + p.QB[cidx(n, i + 1, j - 1) * BLK + a2 * NS + b2] + tj1[b2 * NS + b] +
                 en[EN_STK + po * 6 + pi];
        }, &sfirst);
        if (k >= 0) {
          push(MT_QB, i + 1, j - 1, k / NS, k % NS);
          done = true;
        }
      }
      // 2. bulges: size L ascending, 3' before 5', then the two free states
      if (!done) {
        const int k = cta_first(MAXLOOP * 2 * BLK, want, [&](int k) {
          const int L = 1 + k / (2 * BLK), side = (k / BLK) & 1, s1 = (k % BLK) / NS, s2 = k % NS;
          if (side == 0) {  // inner pair (i+1, l), l = j-1-L; states a2 = s1 at i+1, s = s2 at l
            const int l = j - 1 - L;
            if (l - (i + 1) < 4) return MQINF;
            return en[EN_BU + L] + ti[a * NS + s1] + p.QB[cidx(n, i + 1, l) * BLK + s1 * NS + s2] +
                   p.CH[cidx(n, l, j) * BLK + s2 * NS + b];
          }
          const int kk = i + 1 + L;  // inner pair (kk, j-1); states s = s1 at kk, b2 = s2 at j-1
          if ((j - 1) - kk < 4) return MQINF;
          return en[EN_BU + L] + p.CH[cidx(n, i, kk) * BLK + a * NS + s1] + p.QB[cidx(n, kk, j - 1) * BLK + s1 * NS + s2] +
                 tj1[s2 * NS + b];
        }, &sfirst);
        if (k >= 0) {
          const int L = 1 + k / (2 * BLK), side = (k / BLK) & 1, s1 = (k % BLK) / NS, s2 = k % NS;
          if (side == 0) {
            const int l = j - 1 - L;
            push(MT_CH, l, j, s2, b);
            push(MT_QB, i + 1, l, s1, s2);
          } else {
            const int kk = i + 1 + L;
            push(MT_CH, i, kk, a, s1);
            push(MT_QB, kk, j - 1, s1, s2);
          }
          done = true;
        }
      }
      // 3. multiloop: (type at i+1, type at j-1, state at i+1, state at j-1)
      if (!done && d >= 11) {
        const mq *cx = p.chi + (size_t)i * 4 * BLK, *cy = p.chi + (size_t)(j - 1) * 4 * BLK;
        const int k = cta_first(4 * BLK, want, [&](int k) {
          const int t1 = k / (2 * BLK), t2 = (k / BLK) & 1, s = (k % BLK) / NS, s2 = k % NS;
          const mq *Q2 = t1 ? (t2 ? p.BP : p.M2PU) : (t2 ? p.M2UP : p.M2UU);
          return en[EN_EA] + en[EN_EC] + cx[(t1 ? XPP : XPU) * BLK + a * NS + s] +
                 Q2[cidx(n, i + 1, j - 1) * BLK + s * NS + s2] + cy[(t2 ? XPP : XUP) * BLK + s2 * NS + b];
        }, &sfirst);
        if (k >= 0) {
          const int t1 = k / (2 * BLK), t2 = (k / BLK) & 1, s = (k % BLK) / NS, s2 = k % NS;
          push(t1 ? (t2 ? MT_BP : MT_M2PU) : (t2 ? MT_M2UP : MT_M2UU), i + 1, j - 1, s, s2);
          done = true;
        }
      }
      // 4. hairpin, then interior loops (l1 then l2), over (u at i+1, v at j-1), then (w at k-1, z at l+1)
      if (!done) {
        const int xi = i + 1, yi = j - 1;
        const int k = cta_first(BLK * (1 + NINTERIOR * BLK), want, [&](int k) {
          const int u = (k % BLK) / NS, v = k % NS, sh = k / BLK;
          const mq outer = ti[a * NS + u] + tj1[v * NS + b] +
                           en[EN_TM + p.base[xi * NS + u] * 4 + p.base[yi * NS + v]];
          if (outer >= MQHALF) return MQINF;
          if (sh == 0) return outer + p.hq[d - 1] + p.CH[cidx(n, xi, yi) * BLK + u * NS + v];
          const int q = (sh - 1) / BLK, w = ((sh - 1) % BLK) / NS, z = (sh - 1) % NS;
          int l1, l2;
          interior_shape(q, l1, l2);
          const int kk = i + 1 + l1, l = j - 1 - l2;
          if (l - kk < 4) return MQINF;
          return outer + en[EN_IN + l1 + l2] + p.CH[cidx(n, xi, kk - 1) * BLK + u * NS + w] +
                 p.XI[cidx(n, kk - 1, l + 1) * BLK + w * NS + z] + p.CH[cidx(n, l + 1, yi) * BLK + z * NS + v];
        }, &sfirst);
        if (k < 0) {
          fail(6);
        } else {
          const int u = (k % BLK) / NS, v = k % NS, sh = k / BLK;
          if (sh == 0) {
            push(MT_CH, xi, yi, u, v);
          } else {
            const int q = (sh - 1) / BLK, w = ((sh - 1) % BLK) / NS, z = (sh - 1) % NS;
            int l1, l2;
            interior_shape(q, l1, l2);
            const int kk = i + 1 + l1, l = j - 1 - l2;
            // the inner pair (kk, l) inside XI[kk-1][l+1]: states (a2, b2) ascending
            const mq xv = p.XI[cidx(n, kk - 1, l + 1) * BLK + w * NS + z];
            const mq tmi = en[EN_TM + p.base[(l + 1) * NS + z] * 4 + p.base[(kk - 1) * NS + w]];
            const int k2 = cta_first(BLK, xv, [&](int k2) {
              const int a2 = k2 / NS, b2 = k2 % NS;
              return p.tau[(size_t)(kk - 1) * BLK + w * NS + a2] + p.QB[cidx(n, kk, l) * BLK + a2 * NS + b2] +
                     p.tau[(size_t)l * BLK + b2 * NS + z] + tmi;
            }, &sfirst);
            if (k2 < 0) fail(7);
            else {
              push(MT_CH, xi, kk - 1, u, w);
              push(MT_CH, l + 1, yi, z, v);
              push(MT_QB, kk, l, k2 / NS, k2 % NS);
            }
          }
        }
      }
    } else if (kind == MT_QMP) {  // a branch (x, y), else >= 2 branches
      const mq want = p.QMP[cidx(n, x, y) * BLK + a * NS + b];
      if (en[EN_EC] + p.QB[cidx(n, x, y) * BLK + a * NS + b] == want) push(MT_QB, x, y, a, b);
      else if (p.BP[cidx(n, x, y) * BLK + a * NS + b] == want) push(MT_BP, x, y, a, b);
      else fail(8);
    } else if (kind == MT_QMU || kind == MT_M2PU) {  // y unpaired: (type at y-1, state at y-1)
      const bool one = kind == MT_QMU;
      const mq want = (one ? p.QMU : p.M2PU)[cidx(n, x, y) * BLK + a * NS + b];
      const mq *c = p.chi + (size_t)(y - 1) * 4 * BLK;
      const int k = cta_first(2 * NS, want, [&](int k) {
        const int tp = k / NS, s = k % NS;
        const mq *Pt = tp ? (one ? p.QMP : p.BP) : (one ? p.QMU : p.M2PU);
        return en[EN_EB] + Pt[cidx(n, x, y - 1) * BLK + a * NS + s] + c[(tp ? XPU : XUU) * BLK + s * NS + b];
      }, &sfirst);
      if (k < 0) fail(9);
      else {
        setst(y, b);
        const int tp = k / NS, s = k % NS;
        push(tp ? (one ? MT_QMP : MT_BP) : kind, x, y - 1, a, s);
      }
    } else if (kind == MT_GP) {  // y = k, the branch start: (type at k-1, state at k-1)
      const mq want = p.GP[cidx(n, x, y) * BLK + a * NS + b];
      const mq *c = p.chi + (size_t)(y - 1) * 4 * BLK;
      const int k = cta_first(2 * NS, want, [&](int k) {
        const int tp = k / NS, s = k % NS;
        return (tp ? p.QMP : p.QMU)[cidx(n, x, y - 1) * BLK + a * NS + s] + c[(tp ? XPP : XUP) * BLK + s * NS + b];
      }, &sfirst);
      if (k < 0) fail(10);
      else push(k / NS ? MT_QMP : MT_QMU, x, y - 1, a, k % NS);
    } else if (kind == MT_BP) {  // last branch (k, y): k ascending, state at k
      const mq want = p.BP[cidx(n, x, y) * BLK + a * NS + b];
      const int K = max(0, y - x - 8) * NS;
      const int k = cta_first(K, want, [&](int q) {
        const int kk = x + 5 + q / NS, s = q % NS;
        return en[EN_EC] + p.GP[cidx(n, x, kk) * BLK + a * NS + s] + p.QB[cidx(n, kk, y) * BLK + s * NS + b];
      }, &sfirst);
      if (k < 0) fail(11);
      else {
        const int kk = x + 5 + k / NS, s = k % NS;
        push(MT_QB, kk, y, s, b);
        push(MT_GP, x, kk, a, s);
      }
    } else {  // MT_M2UP / MT_M2UU: x unpaired: (type at x+1, state at x+1)
      const bool lastp = kind == MT_M2UP;
      const mq want = (lastp ? p.M2UP : p.M2UU)[cidx(n, x, y) * BLK + a * NS + b];
      const mq *c = p.chi + (size_t)x * 4 * BLK;
      const int k = cta_first(2 * NS, want, [&](int k) {
        const int tp = k / NS, s = k % NS;
        const mq *Pt = tp ? (lastp ? p.BP : p.M2PU) : (lastp ? p.M2UP : p.M2UU);
        return en[EN_EB] + c[(tp ? XUP : XUU) * BLK + a * NS + s] + Pt[cidx(n, x + 1, y) * BLK + s * NS + b];
      }, &sfirst);
      if (k < 0) fail(12);
      else {
        setst(x, a);
        const int tp = k / NS, s = k % NS;
        push(tp ? (lastp ? MT_BP : MT_M2PU) : kind, x + 1, y, s, b);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (sp != 0 && !sbad) fail(13);  // the guard ran out
  __syncthreads();
  for (int q = t; q < n; q += blockDim.x)
    if (T.state[q] < 0 && !sbad) atomicOr(p.err, 1 << 5);
  __syncthreads();
  for (int r = t; r < p.m; r += blockDim.x) {
    const int c = traced_codon(p.cid, T.sctab, T.state, r);
    if (c < 0 && !sbad) atomicOr(p.err, 1 << 5);
    T.codons[r] = sbad ? -1 : c;
  }
  if (t == 0 && sbad) atomicOr(p.err, 1 << 4);
}

}  // namespace cf
