// cf_inside2.cuh -- inside pass as two kernels per anti-diagonal d, run as a
// CUDA graph (see codonfold.cu):
//
//   k_in_bif<T>(d)   the multiloop/exterior bifurcation sums of diagonal d,
//                    sum_k G[x][k] QB[k][y] and sum_k Gx[k] QB[k][d], split in
//                    chunks of 32 split points (one warp per chunk, lanes over k).
//                    Its inputs lie on diagonals <= d-4, so the graph lets it run
//                    while diagonals d-3..d-1 are still being filled.  Chunk
//                    partials are relative to 2^{E[d-4]}.
//   k_in_light<T>(d) everything else of diagonal d, one 128-thread block per
//                    cell: the ~230 input blocks are staged into shared memory
//                    with asynchronous 16-byte copies (one memory round trip),
//                    then the chain, XI, the 29 interior partial sums, bulges,
//                    hairpin, QB, multiloop tables and the exterior prefix are
//                    computed from shared memory.
//
// Tables, exponents and recursions are those of cf_inside.cuh.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"

namespace cf {

constexpr int KCH = 32;  // split points per bifurcation chunk
constexpr int BIFRING = 4;

__host__ __device__ __forceinline__ int nchunk_bif(int d) { return d >= 9 ? (d - 8 + KCH - 1) / KCH : 0; }
// exterior split points k = 4..d-4 (those with QB[k][d] on diagonals <= d-4);
// k = 1..3 are added by the light kernel of diagonal d itself
__host__ __device__ __forceinline__ int nchunk_ext(int d) { return d >= 8 ? (d - 7 + KCH - 1) / KCH : 0; }

template <typename T>
struct BifBuf {
  T *main;  // [BIFRING][n][ncmax][36]
  T *ext;   // [BIFRING][ncmax][36]
  int ncmax;
};

// ---------------------------------------------------------------- K1
template <typename T>
__global__ void __launch_bounds__(128) k_in_bif(DP<T> p, BifBuf<T> bb, int d) {
  const int lane = threadIdx.x & 31;
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n = p.n;
  const int nc = nchunk_bif(d), ncx = nchunk_ext(d);
  const int nmain = (n - d) * nc;
  if (item >= nmain + ncx) return;
  const int Eref = p.E[d - 4];
  const int slot = d % BIFRING;
  T acc[BLK];
  zero_block(acc);
  if (item < nmain) {
    const int x = item / nc, c = item % nc, y = x + d;
    const int Mx = p.Mp[x], My = p.Mp[y];
    const int k = x + 5 + c * KCH + lane;
    if (k <= y - 4) {
      T f = p.en[EN_EC] * clamp_p2<T>(p.E[k - x] + p.E[y - k] - Eref);
      acc_mm<false, false>(acc, p.G + cidx(n, x, k) * BLK, p.QB + cidx(n, k, y) * BLK, Mx, p.Mp[k], My, f);
    }
    warp_reduce_block(acc, Mx, My);
    T dummy = 0;
    store_block(bb.main + (((size_t)slot * n + x) * bb.ncmax + c) * BLK, acc, Mx, My, lane, dummy);
  } else {
    const int c = item - nmain;
    const int M0 = p.Mp[0], Md = p.Mp[d];
    const int k = 4 + c * KCH + lane;
    if (k <= d - 4) {
      T f = clamp_p2<T>(p.E[k] + p.E[d - k] - Eref);
      acc_mm<false, false>(acc, p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, M0, p.Mp[k], Md, f);
    }
    warp_reduce_block(acc, M0, Md);
    T dummy = 0;
    store_block(bb.ext + ((size_t)slot * bb.ncmax + c) * BLK, acc, M0, Md, lane, dummy);
  }
}

// ---------------------------------------------------------------- staging

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// copy one padded block (36 values) global -> shared with 16-byte async copies
template <typename T>
__device__ __forceinline__ void stage_block(T *dst, const T *src) {
  constexpr int CH = BLK * sizeof(T) / 16;
#pragma unroll
  for (int q = 0; q < CH; q++) cp_async16((char *)dst + 16 * q, (const char *)src + 16 * q);
}

// slot layout of the light kernel's staged inputs (blocks of 36 values)
enum : int {
  SI_TX = 0, SI_TY1 = 1, SI_XX = 2, SI_XY1 = 6, SI_CHN = 10, SI_QBI = 11, SI_HBI = 12, SI_Q2I = 13,
  SI_ML = 17, SI_MR = 21, SI_YYP = 25, SI_XIL = 53, SI_CHL = 81, SI_BQ3 = 109, SI_BC3 = 139,
  SI_BC5 = 169, SI_BQ5 = 199, SI_N = 229
};

// global source of staged slot s for cell (x, y) of diagonal d, or nullptr
template <typename T>
__device__ __forceinline__ const T *in_slot_src(const DP<T> &p, int s, int x, int y, int d) {
  const int n = p.n;
  if (s == SI_TX) return p.Tr + (size_t)x * BLK;
  if (s == SI_TY1) return d >= 1 ? p.Tr + (size_t)(y - 1) * BLK : nullptr;
  if (s < SI_XY1) return p.X + ((size_t)x * 4 + (s - SI_XX)) * BLK;
  if (s < SI_CHN) return d >= 1 ? p.X + ((size_t)(y - 1) * 4 + (s - SI_XY1)) * BLK : nullptr;
  if (s == SI_CHN) return d >= 1 ? p.CH + cidx(n, x + 1, y) * BLK : nullptr;
  if (s == SI_QBI) return d >= 6 ? p.QB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s == SI_HBI) return d >= 4 ? p.HB + cidx(n, x + 1, y - 1) * BLK : nullptr;
  if (s < SI_ML) {
    if (d < 11) return nullptr;
    const T *t[4] = {p.QM2uu, p.QM2up, p.QM2pu, p.QM2pp};
    return t[s - SI_Q2I] + cidx(n, x + 1, y - 1) * BLK;
  }
  if (s < SI_MR) {
    if (d < 5) return nullptr;
    const T *t[4] = {p.QMpp, p.QMpu, p.QM2pp, p.QM2pu};
    return t[s - SI_ML] + cidx(n, x, y - 1) * BLK;
  }
  if (s < SI_YYP) {
    if (d < 10) return nullptr;
    const T *t[4] = {p.QM2up, p.QM2pp, p.QM2uu, p.QM2pu};
    return t[s - SI_MR] + cidx(n, x + 1, y) * BLK;
  }
  const int Lmax = min(MAXLOOP, d - 4);
  if (s < SI_XIL) {  // YY_{L-1}[x+1][y], L = 3..30
    int L = s - SI_YYP + 3;
    return (d >= 6 && L <= Lmax) ? p.YY + (cidx(n, x + 1, y) * NYY + (L - 3)) * BLK : nullptr;
  }
  if (s < SI_CHL) {  // XI[x][y-L+2]
    int L = s - SI_XIL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.XI + cidx(n, x, yl) * BLK : nullptr;
  }
  if (s < SI_BQ3) {  // CH[y-L+2][y]
    int L = s - SI_CHL + 3, yl = y - L + 2;
    return (d >= 6 && L <= Lmax && yl - x >= 6) ? p.CH + cidx(n, yl, y) * BLK : nullptr;
  }
  const int L = (s - SI_BQ3) % MAXLOOP + 1;
  if (d - L < 4) return nullptr;
  if (s < SI_BC3) return p.QB + cidx(n, x, y - L) * BLK;
  if (s < SI_BC5) return p.CH + cidx(n, y - L, y) * BLK;
  if (s < SI_BQ5) return p.CH + cidx(n, x, x + L) * BLK;
  return p.QB + cidx(n, x + L, y) * BLK;
}

// ---------------------------------------------------------------- K2
template <typename T>
__global__ void __launch_bounds__(128) k_in_light(DP<T> p, BifBuf<T> bb, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = (T *)smem_raw;                // [SI_N][36] staged inputs
  T *O = S + (size_t)SI_N * BLK;       // outputs: CH, XI, QB, HB
  T *YO = O + 4 * BLK;                 // [29][36] interior partial sums
  T *ACC = YO + NYY * BLK;             // [3][36] group partials
  __shared__ int sE;
  __shared__ double smax[4];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int x = blockIdx.x, y = x + d;
  // issue the staging copies first: they overlap the exponent bookkeeping
  for (int s = t; s < SI_N; s += blockDim.x) {
    const T *src = in_slot_src(p, s, x, y, d);
    if (src) stage_block(S + (size_t)s * BLK, src);
  }
  if (t == 0) {
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
    if (x == 0) p.E[d] = e;
  }
  cp_async_wait_all();
  __syncthreads();
  const int Ed = sE;
  const int Mx = p.Mp[x], My = p.Mp[y];
  const int *base = p.base;
  const T *en = p.en;
  const size_t c = cidx(n, x, y);
  const T *Tx = S + SI_TX * BLK, *Ty1 = S + SI_TY1 * BLK;
  T *CHo = O, *XIo = O + BLK, *QBo = O + 2 * BLK, *HBo = O + 3 * BLK;
  double lmax = 0.0;

  // ---- P1: chain and XI
  if (t < BLK) {
    const int a = t / NS, b = t % NS;
    if (a < Mx && b < My) {
      T v;
      if (d == 0) v = (a == b) ? (T)1 : (T)0;
      else v = e2<false, false>(Tx, S + SI_CHN * BLK, a, b, p.Mp[x + 1]);
      CHo[t] = v;
      p.CH[c * BLK + t] = v;
    }
  } else if (t >= 64 && t < 64 + BLK && d >= 6) {
    const int e = t - 64, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      T f = clamp_p2<T>(p.E[d - 2] - Ed);
      T v = e3<false, false, false>(Tx, S + SI_QBI * BLK, Ty1, a, b, p.Mp[x + 1], p.Mp[y - 1]);
      v *= f * en[EN_TM + base[y * NS + b] * 4 + base[x * NS + a]];
      XIo[e] = v;
      p.XI[c * BLK + e] = v;
      lmax = fmax(lmax, (double)fabs(v));
    }
  }
  __syncthreads();

  // ---- P2: interior partial sums, bulges, hairpin -> HB (three groups)
  if (d >= 2 && t < 3 * BLK) {
    const int g = t / BLK, e = t % BLK, a = e / NS, b = e % NS;
    T acc = 0;
    if (a < Mx && b < My) {
      const T tmo = en[EN_TM + base[x * NS + a] * 4 + base[y * NS + b]];
      const int Lmax = min(MAXLOOP, d - 4);
      const int M1 = p.Mp[x + 1];
      for (int L = 2 + g; L <= Lmax; L += 3) {
        T v;
        if (L == 2) {
          v = XIo[e];
        } else {
          v = e2<false, false>(Tx, S + (SI_YYP + L - 3) * BLK, a, b, M1);
          const int yl = y - L + 2;
          if (yl - x >= 6) v += e2<false, false>(S + (SI_XIL + L - 3) * BLK, S + (SI_CHL + L - 3) * BLK, a, b, p.Mp[yl]);
        }
        YO[(L - 2) * BLK + e] = v;
        p.YY[(c * NYY + (L - 2)) * BLK + e] = v;
        const int ey = (L == 2) ? Ed : p.E[d - L + 2];
        acc += en[EN_IN + L] * clamp_p2<T>(ey - Ed) * tmo * v;
      }
      for (int q = g; q < 2 * MAXLOOP; q += 3) {
        const int L = q / 2 + 1;
        if (d - L < 4) continue;
        const T f = en[EN_BU + L] * clamp_p2<T>(p.E[d - L] - Ed);
        if ((q & 1) == 0)
          acc += f * e2<false, false>(S + (SI_BQ3 + L - 1) * BLK, S + (SI_BC3 + L - 1) * BLK, a, b, p.Mp[y - L]);
        else
          acc += f * e2<false, false>(S + (SI_BC5 + L - 1) * BLK, S + (SI_BQ5 + L - 1) * BLK, a, b, p.Mp[x + L]);
      }
      if (g == 0) acc += p.eHL[d + 1] * clamp_p2<T>(-Ed) * tmo * CHo[e];
    }
    ACC[g * BLK + e] = acc;
  }
  __syncthreads();
  if (d >= 2 && t < BLK) {
    const int a = t / NS, b = t % NS;
    if (a < Mx && b < My) {
      T v = ACC[t] + ACC[BLK + t] + ACC[2 * BLK + t];
      HBo[t] = v;
      p.HB[c * BLK + t] = v;
      lmax = fmax(lmax, (double)fabs(v));
    }
  }

  // ---- P3: QB (closing pair (x, y)), in threads 64..99
  if (d >= 4 && t >= 64 && t < 64 + BLK) {
    const int e = t - 64, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      const int pto = pair_type(base[x * NS + a], base[y * NS + b]);
      T v = 0;
      if (pto >= 0) {
        const int Mu = p.Mp[x + 1], Mv = p.Mp[y - 1];
        v = e3<false, false, false>(Tx, S + SI_HBI * BLK, Ty1, a, b, Mu, Mv);
        if (d >= 6) {
          const T *qin = S + SI_QBI * BLK;
#pragma unroll
          for (int a2 = 0; a2 < NS; a2++) {
            if (a2 < Mu) {
              const T tv = Tx[a * NS + a2];
              const int ba = base[(x + 1) * NS + a2];
#pragma unroll
              for (int b2 = 0; b2 < NS; b2++) {
                if (b2 < Mv) {
                  const int pti = pair_type(ba, base[(y - 1) * NS + b2]);
                  const T es = pti >= 0 ? en[EN_STK + pto * 6 + pti] : (T)0;
                  v += tv * qin[a2 * NS + b2] * Ty1[b2 * NS + b] * es;
                }
              }
            }
          }
        }
        if (d >= 11) {
          const T *Xl = S + SI_XX * BLK, *Xr = S + SI_XY1 * BLK, *q2 = S + SI_Q2I * BLK;
          T s2 = e3<false, false, false>(Xl + XPU * BLK, q2 + 0 * BLK, Xr + XUP * BLK, a, b, Mu, Mv) +
                 e3<false, false, false>(Xl + XPU * BLK, q2 + 1 * BLK, Xr + XPP * BLK, a, b, Mu, Mv) +
                 e3<false, false, false>(Xl + XPP * BLK, q2 + 2 * BLK, Xr + XUP * BLK, a, b, Mu, Mv) +
                 e3<false, false, false>(Xl + XPP * BLK, q2 + 3 * BLK, Xr + XPP * BLK, a, b, Mu, Mv);
          v += en[EN_EA] * en[EN_EC] * s2;
        }
        v *= clamp_p2<T>(p.E[d - 2] - Ed);
      }
      QBo[e] = v;
      p.QB[c * BLK + e] = v;
      lmax = fmax(lmax, (double)fabs(v));
    }
  }
  __syncthreads();

  // ---- P4: QMpp / QM2pp (threads 0..35), QMpu and G (36..71), QM2pu/up/uu (72..107)
  const int slot = d % BIFRING;
  if (d >= 4 && t < BLK) {
    const int a = t / NS, b = t % NS;
    if (a < Mx && b < My) {
      T s2 = 0;
      const int nc = nchunk_bif(d);
      if (nc > 0) {
        const T *bp = bb.main + (((size_t)slot * n + x) * bb.ncmax) * BLK + t;
        T s0 = 0, s1 = 0;
        int q = 0;
        for (; q + 1 < nc; q += 2) {
          s0 += bp[(size_t)q * BLK];
          s1 += bp[(size_t)(q + 1) * BLK];
        }
        if (q < nc) s0 += bp[(size_t)q * BLK];
        s2 = (s0 + s1) * clamp_p2<T>(p.E[d - 4] - Ed);
      }
      const T v = en[EN_EC] * QBo[t] + s2;
      p.QM2pp[c * BLK + t] = s2;
      p.QMpp[c * BLK + t] = v;
      lmax = fmax(lmax, fmax((double)fabs(v), (double)fabs(s2)));
    }
  } else if (d >= 5 && t >= BLK && t < 2 * BLK) {
    const int e = t - BLK, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      const T F1 = clamp_p2<T>(p.E[d - 1] - Ed), eb = en[EN_EB];
      const T *Xr = S + SI_XY1 * BLK, *mpp = S + SI_ML * BLK, *mpu = S + (SI_ML + 1) * BLK;
      const int Mv = p.Mp[y - 1];
      const T u = eb * F1 * (e2<false, false>(mpp, Xr + XPU * BLK, a, b, Mv) + e2<false, false>(mpu, Xr + XUU * BLK, a, b, Mv));
      const T g = F1 * (e2<false, false>(mpp, Xr + XPP * BLK, a, b, Mv) + e2<false, false>(mpu, Xr + XUP * BLK, a, b, Mv));
      p.QMpu[c * BLK + e] = u;
      p.G[c * BLK + e] = g;
      lmax = fmax(lmax, fmax((double)fabs(u), (double)fabs(g)));
    }
  } else if (d >= 10 && t >= 2 * BLK && t < 3 * BLK) {
    const int e = t - 2 * BLK, a = e / NS, b = e % NS;
    if (a < Mx && b < My) {
      const T F1 = clamp_p2<T>(p.E[d - 1] - Ed), eb = en[EN_EB];
      const T *Xr = S + SI_XY1 * BLK, *Xl = S + SI_XX * BLK;
      const int Mv = p.Mp[y - 1], Mu = p.Mp[x + 1];
      const T *q2pp = S + (SI_ML + 2) * BLK, *q2pu = S + (SI_ML + 3) * BLK;
      const T *r_up = S + SI_MR * BLK, *r_pp = S + (SI_MR + 1) * BLK, *r_uu = S + (SI_MR + 2) * BLK,
              *r_pu = S + (SI_MR + 3) * BLK;
      const T pu = eb * F1 * (e2<false, false>(q2pp, Xr + XPU * BLK, a, b, Mv) + e2<false, false>(q2pu, Xr + XUU * BLK, a, b, Mv));
      const T up = eb * F1 * (e2<false, false>(Xl + XUU * BLK, r_up, a, b, Mu) + e2<false, false>(Xl + XUP * BLK, r_pp, a, b, Mu));
      const T uu = eb * F1 * (e2<false, false>(Xl + XUU * BLK, r_uu, a, b, Mu) + e2<false, false>(Xl + XUP * BLK, r_pu, a, b, Mu));
      p.QM2pu[c * BLK + e] = pu;
      p.QM2up[c * BLK + e] = up;
      p.QM2uu[c * BLK + e] = uu;
      lmax = fmax(lmax, fmax((double)fabs(pu), fmax((double)fabs(up), (double)fabs(uu))));
    }
  }

  // ---- P5: exterior prefix [0, d] (cell (0, d)), threads 0..35
  if (x == 0 && t < BLK) {
    const int M0 = p.Mp[0];
    const int a = t / NS, b = t % NS;
    T *q5u = p.Q5U + (size_t)d * BLK, *q5p = p.Q5P + (size_t)d * BLK;
    if (d == 0) {
      if (a < M0 && b < M0) {
        q5u[t] = (a == b) ? (T)1 : (T)0;
        q5p[t] = 0;
      }
      lmax = fmax(lmax, 1.0);
    } else if (a < M0 && b < My) {
      const T F1 = clamp_p2<T>(p.E[d - 1] - Ed);
      const T *Xr = S + SI_XY1 * BLK;
      const int Mv = p.Mp[d - 1];
      const T *pu = p.Q5U + (size_t)(d - 1) * BLK, *pp = p.Q5P + (size_t)(d - 1) * BLK;
      const T g = F1 * (e2<false, false>(pu, Xr + XUP * BLK, a, b, Mv) + e2<false, false>(pp, Xr + XPP * BLK, a, b, Mv));
      const T u = F1 * (e2<false, false>(pu, Xr + XUU * BLK, a, b, Mv) + e2<false, false>(pp, Xr + XPU * BLK, a, b, Mv));
      p.Gx[(size_t)d * BLK + t] = g;
      q5u[t] = u;
      T s2 = 0;
      const int ncx = nchunk_ext(d);
      const T *bp = bb.ext + ((size_t)slot * bb.ncmax) * BLK + t;
      for (int q = 0; q < ncx; q++) s2 += bp[(size_t)q * BLK];
      T v = (d >= 4 ? QBo[t] : (T)0) + s2 * clamp_p2<T>(p.E[d - 4 >= 0 ? d - 4 : 0] - Ed);
      // split points k = 1..3 use QB[k][d] of diagonals d-1..d-3
      for (int k = 1; k <= 3 && k <= d - 4; k++)
        v += clamp_p2<T>(p.E[k] + p.E[d - k] - Ed) *
             e2<false, false>(p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, a, b, p.Mp[k]);
      q5p[t] = v;
      lmax = fmax(lmax, fmax((double)fabs(g), fmax((double)fabs(u), (double)fabs(v))));
    }
  }

  // ---- diagonal maximum for the next exponent
  lmax = warp_max(lmax);
  if (lane == 0) smax[w] = lmax;
  __syncthreads();
  if (t == 0) {
    double m = fmax(fmax(smax[0], smax[1]), fmax(smax[2], smax[3]));
    atomic_max_pos(&p.dmax[d], m);
  }
}

template <typename T>
constexpr size_t in_light_smem() {
  return (size_t)(SI_N + 4 + NYY + 3) * BLK * sizeof(T);
}

}  // namespace cf
