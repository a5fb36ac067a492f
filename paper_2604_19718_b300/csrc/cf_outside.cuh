// cf_outside.cuh -- conventions of the outside pass (the hand-written adjoint
// of the inside pass) and its final kernels (marginals, unpaired
// probabilities); the wavefront kernels are in cf_outside2.cuh.
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

// Joint codon marginals of adjacent residues at each boundary transfer,
// trans[r][a][b] = T o (hT + sum_k hX_k o dangle_k), and residue 0's
// marginal from the top-level weights.
template <typename T>
__global__ void k_marginals(DP<T> p, double *trans, double *p0) {
  if (p.bstride) {  // batch: blockIdx.y is the protein
    const long long o = (long long)blockIdx.y * p.bstride;
    dp_shift(p, o);
    trans = bshift(trans, o);
    p0 = bshift(p0, o);
  }
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

// Codon marginal of state a at residue r (Eq. marginal-codon): residue 0 from
// p0, every later residue as the summed gradient of the transfers entering it
// (each transfer T_q, q = 3r - 1, carries the residue's weight exactly once).
__device__ __forceinline__ double codon_marg_of(const double *trans, const double *p0, int r, int a, int Mprev) {
  if (r == 0) return p0[a];
  const double *t = trans + (size_t)(r - 1) * BLK + a;
  double s = 0;
  for (int b = 0; b < Mprev; b++) s += t[b * NS];
  return s;
}

// Outputs of the outside pass from the transfer gradients, each summed in a
// fixed order (results independent of scheduling).  The first
// ceil((6m + n) / blockDim) blocks take one thread per entry of
//   cm[r][a]   codon marginals (m x 6, unused slots 0) and
//   bm[i][b]   base marginals (n x 4), Eq. marginal-base: the state of
//              position i is its residue's codon, so p_i(b) sums the codon
//              marginals of the residue's codons with base b at i;
// the remaining blocks one warp per entry of
//   pg[x][y]   d log Z / d pb[x][y] over sense codon ids (61 x 61): the
//              transfer gradients of every residue boundary whose two states
//              are codons x and y, lanes striding over the boundaries.
template <typename T>
__global__ void k_codon_out(DP<T> p, const double *trans, const double *p0, const int *cid, double *cm,
                            double *bm, double *pg) {
  if (p.bstride) {  // batch: blockIdx.y is the protein
    const long long o = (long long)blockIdx.y * p.bstride;
    dp_shift(p, o);
    trans = bshift(trans, o), p0 = bshift(p0, o), cid = bshift(cid, o);
    cm = bshift(cm, o), bm = bshift(bm, o), pg = bshift(pg, o);
  }
  const int n = p.n, m = p.m;
  const int nb1 = (6 * m + n + blockDim.x - 1) / blockDim.x;
  if ((int)blockIdx.x < nb1) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m * 6) {
      const int r = t / 6, a = t % 6;
      const int q = 3 * r;  // first position of residue r
      cm[t] = (a < p.Mp[q]) ? codon_marg_of(trans, p0, r, a, r ? p.Mp[q - 1] : 0) : 0.0;
      if (!isfinite(cm[t])) atomicOr(p.err, ERR_OUT_NONFINITE);
      return;
    }
    const int u = t - m * 6;
    if (u >= n) return;
    const int r = u / 3, q = 3 * r;
    double acc[4] = {0, 0, 0, 0};
    for (int a = 0; a < p.Mp[u]; a++)
      acc[p.base[(size_t)u * NS + a]] += codon_marg_of(trans, p0, r, a, r ? p.Mp[q - 1] : 0);
    for (int b = 0; b < 4; b++) bm[(size_t)u * 4 + b] = acc[b];
    return;
  }
  const int lane = threadIdx.x & 31;
  const int u = (blockIdx.x - nb1) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (u >= 61 * 61) return;  // whole warps leave together
  const int x = u / 61, y = u % 61;
  double s = 0;
  for (int r = lane; r + 1 < m; r += 32) {
    const int q = 3 * r + 2;
    for (int a = 0; a < p.Mp[q]; a++) {
      if (cid[(size_t)q * NS + a] != x) continue;
      for (int b = 0; b < p.Mp[q + 1]; b++)
        if (cid[(size_t)(q + 1) * NS + b] == y) s += trans[(size_t)r * BLK + a * NS + b];
    }
  }
  s = warp_sum(s);
  if (lane == 0) pg[u] = s;
}

// Codon and base marginals in the single-codon layout (Eq. single-tt): the
// codon of residue r is fixed by the transfer from its second position
// (state = first and second base) to its third (state = third base), which
// also carries the codon's weight, so its marginal is T o (hT + sum_k hX_k o
// dangle_k) at q = 3r+1 for the codon's state pair.  smap[r][s] packs, for
// codon slot s, the two states (bits 0-3, 4-7) and the three bases (bits
// 8-9, 10-11, 12-13); -1 past the residue's codons.  One thread per codon
// slot, then one per (position, base).
template <typename T>
__device__ __forceinline__ double sc_codon_marg(const DP<T> &p, int r, int sm) {
  const int q = 3 * r + 1, a = sm & 15, b = (sm >> 4) & 15;
  const int x0 = p.base[q * NS + a], y0 = p.base[(q + 1) * NS + b];
  const double d3 = (double)p.en[EN_D3 + x0 * 4 + y0], d5 = (double)p.en[EN_D5 + y0 * 4 + x0];
  double g = p.hT[(size_t)q * BLK + a * NS + b];
  const double *hx = p.hX + (size_t)q * 4 * BLK + a * NS + b;
  g += hx[XUU * BLK] + hx[XUP * BLK] * d5 + hx[XPU * BLK] * d3 + hx[XPP * BLK] * d3 * d5;
  return (double)p.Tr[(size_t)q * BLK + a * NS + b] * g;
}
template <typename T>
__global__ void k_codon_out_sc(DP<T> p, const int *smap, double *cm, double *bm) {
  const int n = p.n, m = p.m, t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 6 * m) {
    const int sm = smap[t];
    const double v = sm >= 0 ? sc_codon_marg(p, t / 6, sm) : 0.0;
    if (!isfinite(v)) atomicOr(p.err, ERR_OUT_NONFINITE);
    cm[t] = v;
    return;
  }
  const int u = t - 6 * m;
  if (u >= n) return;
  const int r = u / 3, off = u % 3;
  double acc[4] = {0, 0, 0, 0};
  for (int s = 0; s < 6; s++) {
    const int sm = smap[r * 6 + s];
    if (sm >= 0) acc[(sm >> (8 + 2 * off)) & 3] += sc_codon_marg(p, r, sm);
  }
  for (int b = 0; b < 4; b++) bm[(size_t)u * 4 + b] = acc[b];
}

// Unpaired probability of every base: 1 - sum of its pair probabilities; a
// row with a non-finite entry raises ERR_OUT_NONFINITE.
__global__ void k_unpaired(float *P, int n, int *err, long long bstride = 0) {
  if (bstride) {  // batch: blockIdx.y is the protein
    P = bshift(P, (long long)blockIdx.y * bstride);
    err = bshift(err, (long long)blockIdx.y * bstride);
  }
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0;
  for (int j = lane; j < n; j += 32)
    if (j != i) s += (double)P[(size_t)i * n + j];
  s = warp_sum(s);
  if (lane == 0) {
    if (!isfinite(s)) atomicOr(err, ERR_OUT_NONFINITE);
    P[(size_t)i * n + i] = (float)(1.0 - s);
  }
}

}  // namespace cf
