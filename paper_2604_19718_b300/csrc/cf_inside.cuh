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
