// cf_inside.cuh -- definitions shared by the inside pass (partition function)
// over the codon-constrained nearest-neighbour model: the tables, the
// power-of-two factors and the final sum; the wavefront kernels are in
// cf_inside2.cuh.
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
// exponents below the normal range give 0; above, binary32 clamps at 2^120
// and binary64 at 2^1000 (a factor that large multiplies mantissas that are
// correspondingly small, so the clamp is never reached by a term that counts).
template <typename T>
__device__ __forceinline__ T clamp_p2(int e);
template <>
__device__ __forceinline__ float clamp_p2<float>(int e) {
  e = e > 120 ? 120 : e;
  return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}
template <>
__device__ __forceinline__ double clamp_p2<double>(int e) {
  e = e > 1000 ? 1000 : e;
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

// Z relative to 2^{E[n-1]}: sum_a u0[a] sum_b (Q5U + Q5P)[n-1][a][b]
template <typename T>
__global__ void k_inside_finish(DP<T> p) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (p.bstride) dp_shift(p, (long long)blockIdx.y * p.bstride);
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

// Position transfers of the sequence tensor train (Eq. pair-tt), one thread
// per position q, in binary64:
//   T_q[a][b] = delta_ab                      inside a residue (q % 3 != 2),
//   T_q[a][b] = s_r e^{lw[r+1][b] + pb[c_a][c_b]}  across the boundary from
//               residue r to r+1 (q = 3r + 2), c_a, c_b the sense codon ids;
// s_r = M_q / sum_ab e^{...} makes the average row sum one (an exact rescale,
// log s_r is stored in ls[r] and undone in log Z).  The typed transitions add
// the dangles of a paired end: X_UU = T, X_UP = T d5[b][a], X_PU = T d3[a][b],
// X_PP = T d3 d5, with the bases of states a at q and b at q+1.  Entries beyond
// the state counts, and the row of the last position, are zero.  Thread 0 also
// writes u0[a] = e^{lw[0][a]} (residue 0's weights enter at the top).
// (Batch: blockIdx.y is the protein, every array bstride bytes per protein.)
__global__ void k_transfers(int n, const int *Mp, const int *base, const int *cid, const double *en,
                            const double *lw, const double *pb, double *Tr, double *X, double *u0, double *ls,
                            long long bstride = 0) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (bstride) {
    const long long o = (long long)blockIdx.y * bstride;
    Mp = bshift(Mp, o), base = bshift(base, o), cid = bshift(cid, o), en = bshift(en, o), lw = bshift(lw, o);
    pb = bshift(pb, o), Tr = bshift(Tr, o), X = bshift(X, o), u0 = bshift(u0, o), ls = bshift(ls, o);
  }
  if (q == 0)
    for (int a = 0; a < NS; a++) u0[a] = a < Mp[0] ? exp(lw[a]) : 0.0;
  if (q >= n) return;
  double t[BLK];
  for (int e = 0; e < BLK; e++) t[e] = 0.0;
  const int Ma = Mp[q], Mb = q + 1 < n ? Mp[q + 1] : 0;
  if (q + 1 < n) {
    if (q % 3 != 2) {
      for (int a = 0; a < Ma; a++) t[a * NS + a] = 1.0;
    } else {
      const int r1 = (q + 1) / 3;
      double sum = 0;
      for (int a = 0; a < Ma; a++)
        for (int b = 0; b < Mb; b++) {
          const double w = lw[(size_t)r1 * 6 + b] + pb[61 * cid[(size_t)q * NS + a] + cid[(size_t)(q + 1) * NS + b]];
          t[a * NS + b] = exp(w);
          sum += t[a * NS + b];
        }
      const double s = Ma / sum;
      for (int a = 0; a < Ma; a++)
        for (int b = 0; b < Mb; b++) t[a * NS + b] *= s;
      ls[r1 - 1] = log(s);
    }
  }
  double *tq = Tr + (size_t)q * BLK, *xq = X + (size_t)q * 4 * BLK;
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) {
      const int e = a * NS + b;
      double d3 = 0, d5 = 0;
      if (a < Ma && b < Mb) {
        const int x0 = base[(size_t)q * NS + a], y0 = base[(size_t)(q + 1) * NS + b];
        d3 = en[EN_D3 + x0 * 4 + y0];
        d5 = en[EN_D5 + y0 * 4 + x0];
      }
      tq[e] = t[e];
      xq[XUU * BLK + e] = t[e];
      xq[XUP * BLK + e] = t[e] * d5;
      xq[XPU * BLK + e] = t[e] * d3;
      xq[XPP * BLK + e] = t[e] * d3 * d5;
    }
}

// Typed transitions of given position transfers T (binary64, [n][36]), as in
// k_transfers: X_UU = T, X_UP = T d5[b][a], X_PU = T d3[a][b], X_PP = T d3 d5
// with the bases of states a at q and b at q+1; one thread per position
// (the single-codon layout, whose transfers the host builds).
__global__ void k_typed_x(int n, const int *Mp, const int *base, const double *en, const double *Tr, double *X) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int Ma = Mp[q], Mb = q + 1 < n ? Mp[q + 1] : 0;
  const double *tq = Tr + (size_t)q * BLK;
  double *xq = X + (size_t)q * 4 * BLK;
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) {
      const int e = a * NS + b;
      double d3 = 0, d5 = 0;
      if (a < Ma && b < Mb) {
        const int x0 = base[(size_t)q * NS + a], y0 = base[(size_t)(q + 1) * NS + b];
        d3 = en[EN_D3 + x0 * 4 + y0];
        d5 = en[EN_D5 + y0 * 4 + x0];
      }
      xq[XUU * BLK + e] = tq[e];
      xq[XUP * BLK + e] = tq[e] * d5;
      xq[XPU * BLK + e] = tq[e] * d3;
      xq[XPP * BLK + e] = tq[e] * d3 * d5;
    }
}

// Copy of a binary64 table in the precision of a pass (batch: blockIdx.y).
template <typename T>
__global__ void k_cast(const double *src, T *dst, size_t cnt, long long bstride = 0) {
  if (bstride) {
    src = bshift(src, (long long)blockIdx.y * bstride);
    dst = bshift(dst, (long long)blockIdx.y * bstride);
  }
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < cnt; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (T)src[k];
}

// log Z (natural log) in binary64: log of the scaled sum, plus the exponent
// of the last diagonal, minus the transfer rescales, summed in residue order.
// (Batch: blockIdx.y is the protein.)
__global__ void k_logz(const double *Zm, const int *E_last, const double *ls, int nls, double *logz,
                       long long bstride = 0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (bstride) {
    const long long o = (long long)blockIdx.y * bstride;
    Zm = bshift(Zm, o), E_last = bshift(E_last, o), ls = bshift(ls, o), logz = bshift(logz, o);
  }
  double sc = 0;
  for (int r = 0; r < nls; r++) sc += ls[r];
  *logz = log(*Zm) + (double)*E_last * 0.69314718055994530942 - sc;
}

}  // namespace cf
