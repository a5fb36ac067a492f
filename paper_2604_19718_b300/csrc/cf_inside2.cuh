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
  T *main;  // [BIFRING][n][36]  sum_k G[x][k] ec QB[k][y] relative to 2^{E[d-4]}
  T *ext;   // [BIFRING][36]     sum_{k>=4} Gx[k] QB[k][d] relative to 2^{E[d-4]}
  int ncmax;
};

// ---------------------------------------------------------------- K1
// One cell per block (the last unit of a diagonal: the exterior sum); warp w
// of NW takes the chunks w, w+NW, ... of 32 split points, lanes over the split
// point; per-lane sums are reduced once per warp, then across warps.
template <typename T, int NW>
__device__ __forceinline__ void in_bif_cell(const DP<T> &p, const BifBuf<T> &bb, int d, int cb, T (*red)[BLK]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = p.n;
  const int Eref = __ldcg(p.E + d - 4);
  const int slot = d % BIFRING;
  const bool ext = cb == n - d;
  const int x = ext ? 0 : cb, y = x + d;
  const int Ma = p.Mp[x], Mb = p.Mp[y];
  T acc[BLK];
  zero_block(acc);
  if (w < NW) {
    if (!ext) {
      const int nc = nchunk_bif(d);
      const T ec = p.en[EN_EC];
      for (int c = w; c < nc; c += NW) {
        const int k = x + 5 + c * KCH + lane;
        if (k <= y - 4) {
          T f = ec * clamp_p2<T>(__ldcg(p.E + k - x) + __ldcg(p.E + y - k) - Eref);
          acc_mm_v<false, false>(acc, p.G + cidx(n, x, k) * BLK, p.QB + cidx(n, k, y) * BLK, Ma, p.Mp[k], Mb, f);
        }
      }
    } else {
      const int nc = nchunk_ext(d);
      for (int c = w; c < nc; c += NW) {
        const int k = 4 + c * KCH + lane;
        if (k <= d - 4) {
          T f = clamp_p2<T>(__ldcg(p.E + k) + __ldcg(p.E + d - k) - Eref);
          acc_mm_v<false, false>(acc, p.Gx + (size_t)k * BLK, p.QB + cidx(n, k, d) * BLK, Ma, p.Mp[k], Mb, f);
        }
      }
    }
    warp_reduce_block(acc, Ma, Mb);
    if (lane < 2) {
#pragma unroll
      for (int e = 0; e < BLK; e++)
        if ((e & 1) == lane) red[w][e] = acc[e];
    }
  }
  __syncthreads();
  if (threadIdx.x < BLK) {
    const int e = threadIdx.x;
    T v = 0;
#pragma unroll
    for (int k = 0; k < NW; k++) v += red[k][e];
    T *dst = ext ? bb.ext + (size_t)slot * BLK : bb.main + ((size_t)slot * n + x) * BLK;
    dst[e] = v;
  }
}

// Grid-stride over the n-d cells and the exterior: launched with fewer CTAs
// than cells, so that the light kernels of the critical path always find
// room on the SMs.
template <typename T>
__global__ void __launch_bounds__(256) k_in_bif(DP<T> p, BifBuf<T> bb, int d) {
  __shared__ T red[8][BLK];
  for (int cb = blockIdx.x; cb <= p.n - d; cb += gridDim.x) {
    in_bif_cell<T, 8>(p, bb, d, cb, red);
    __syncthreads();
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
  SI_BC5 = 169, SI_BQ5 = 199, SI_BIF = 229, SI_BIFX = 230, SI_Q5U = 231, SI_Q5P = 232,
  SI_GXK = 233, SI_QBK = 236, SI_N = 239
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
  if (s < SI_BIF) {
    const int L = (s - SI_BQ3) % MAXLOOP + 1;
    if (d - L < 4) return nullptr;
    if (s < SI_BC3) return p.QB + cidx(n, x, y - L) * BLK;
    if (s < SI_BC5) return p.CH + cidx(n, y - L, y) * BLK;
    if (s < SI_BQ5) return p.CH + cidx(n, x, x + L) * BLK;
    return p.QB + cidx(n, x + L, y) * BLK;
  }
  return nullptr;  // remaining slots need the bifurcation buffers: in_slot_src2
}

// bifurcation results and exterior-prefix inputs
template <typename T>
__device__ __forceinline__ const T *in_slot_src2(const DP<T> &p, const BifBuf<T> &bb, int s, int x, int d) {
  const int n = p.n, slot = d % BIFRING;
  if (s == SI_BIF) return nchunk_bif(d) > 0 ? bb.main + ((size_t)slot * n + x) * BLK : nullptr;
  if (x != 0 || d == 0) return nullptr;
  if (s == SI_BIFX) return nchunk_ext(d) > 0 ? bb.ext + (size_t)slot * BLK : nullptr;
  if (s == SI_Q5U) return p.Q5U + (size_t)(d - 1) * BLK;
  if (s == SI_Q5P) return p.Q5P + (size_t)(d - 1) * BLK;
  const int k = (s < SI_QBK ? s - SI_GXK : s - SI_QBK) + 1;
  if (k > d - 4) return nullptr;
  return s < SI_QBK ? p.Gx + (size_t)k * BLK : p.QB + cidx(n, k, d) * BLK;
}

// ---------------------------------------------------------------- K2
// Thread mapping: the M_x*M_y live entries of a block are numbered compactly
// (e = a*M_y + b); work lists over (task, entry) are split into NT/(M_x*M_y)
// groups so that small codon-state counts keep all threads busy.
constexpr int NT = 512;       // threads per cell on diagonals with few cells
constexpr int NT_WIDE = 256;  // ... and on diagonals with more than WIDE_CELLS cells
constexpr int WIDE_CELLS = 296;

template <typename T, int NTT>
__device__ __forceinline__ void in_light_cell(const DP<T> &p, const BifBuf<T> &bb, int d, int x,
                                              unsigned char *smem_raw) {
  T *S = (T *)smem_raw;                // [SI_N][36] staged inputs
  T *O = S + (size_t)SI_N * BLK;       // outputs: CH, XI, QB, HB
  T *YO = O + 4 * BLK;                 // [29][36] interior partial sums
  T *RED = YO + NYY * BLK;             // [NTT] group partials of HB
  T *RED2 = RED + NTT;                  // [4][36] partial terms of QB
  __shared__ int sEd;
  __shared__ double smax[NTT / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int y = x + d;
  for (int s = t; s < SI_N; s += NTT) {
    const T *src = s < SI_BIF ? in_slot_src(p, s, x, y, d) : in_slot_src2(p, bb, s, x, d);
    if (src) stage_block(S + (size_t)s * BLK, src);
  }
  // small per-cell context on chip: exponents around d, codon-state counts
  // around x and y, bases of x-1..x+1 and y-1..y+1, energy factors
  __shared__ int sE[96], sMx[72], sMy[72], sBx[3][NS], sBy[3][NS];
  __shared__ T sEn[EN_N];
  for (int i = t; i < 96; i += NTT) {
    const int k = d - 47 + i;
    sE[i] = (k >= 0 && k < d) ? __ldcg(p.E + k) : 0;
  }
  for (int i = t; i < 72; i += NTT) {
    const int qx = x - 35 + i, qy = y - 35 + i;
    sMx[i] = (qx >= 0 && qx < n) ? p.Mp[qx] : 0;
    sMy[i] = (qy >= 0 && qy < n) ? p.Mp[qy] : 0;
  }
  for (int i = t; i < 3 * NS; i += NTT) {
    const int r = i / NS, a = i % NS, qx = x - 1 + r, qy = y - 1 + r;
    sBx[r][a] = (qx >= 0 && qx < n) ? p.base[qx * NS + a] : 0;
    sBy[r][a] = (qy >= 0 && qy < n) ? p.base[qy * NS + a] : 0;
  }
  for (int i = t; i < EN_N; i += NTT) sEn[i] = p.en[i];
  if (t == 0) {
    int e = 0;
    if (d > 0) {
      double mx = __longlong_as_double((long long)__ldcg(p.dmax + d - 1));
      e = __ldcg(p.E + d - 1);
      if (mx > 0) {
        if (isfinite(mx)) e += ilogb(mx);
        else atomicOr(p.err, 1);
      }
    }
    sEd = e;
    if (x == 0) p.E[d] = e;
  }
  cp_async_wait_all();
  __syncthreads();
  const int Ed = sEd;
  const int Mx = MP(x), My = MP(y), MM = Mx * My;
  const int M1 = (d >= 1) ? MP(x + 1) : 0, Mv = (d >= 1) ? MP(y - 1) : 0;
  const T *en = sEn;
  const size_t c = cidx(n, x, y);
  const T *Tx = S + SI_TX * BLK, *Ty1 = S + SI_TY1 * BLK;
  T *CHo = O, *XIo = O + BLK, *QBo = O + 2 * BLK, *HBo = O + 3 * BLK;
  double lmax = 0.0;
  // loop-length weights of this cell: interior eIn(L) 2^{E[d-L+2]-E[d]},
  // bulge eBu(L) 2^{E[d-L]-E[d]}, hairpin eH(d+1) 2^{-E[d]}
  __shared__ T wIn[MAXLOOP + 1], wBu[MAXLOOP + 1], wHp;
  if (t <= MAXLOOP) {
    const int L = t;
    wIn[L] = (L >= 2 && d - L + 2 >= 0) ? en[EN_IN + L] * clamp_p2<T>(EA(d - L + 2) - Ed) : (T)0;
    wBu[L] = (L >= 1 && d - L >= 4) ? en[EN_BU + L] * clamp_p2<T>(EA(d - L) - Ed) : (T)0;
  } else if (t == 64 && d >= 2) {
    wHp = p.eHL[d + 1] * clamp_p2<T>(-Ed);
  }
  __syncthreads();

  // ---- P1: chain (threads 0..MM-1) and XI (128..128+MM-1)
  if (t < MM) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    T v;
    if (d == 0) v = (a == b) ? (T)1 : (T)0;
    else v = s2<false, false>(Tx, S + SI_CHN * BLK, a, b, M1);
    CHo[pe] = v;
    p.CH[c * BLK + pe] = v;
  } else if (d >= 6 && t >= 128 && t < 128 + MM) {
    const int e = t - 128, a = e / My, b = e % My, pe = a * NS + b;
    const T f = clamp_p2<T>(EA(d - 2) - Ed);
    T v = s3<false, false, false>(Tx, S + SI_QBI * BLK, Ty1, a, b, M1, Mv);
    v *= f * en[EN_TM + BASE(y, b) * 4 + BASE(x, a)];
    XIo[pe] = v;
    p.XI[c * BLK + pe] = v;
    lmax = fmax(lmax, (double)fabs(v));
  }
  __syncthreads();

  // ---- P2: interior partial sums and bulges, split over groups -> HB
  const int GR = min(NTT / MM, 32);  // groups for the reductions below
  if (d >= 2) {
    const int G = GR, g = t / MM, e = t % MM;
    if (g < G) {
      const int a = e / My, b = e % My, pe = a * NS + b;
      const T tmo = en[EN_TM + BASE(x, a) * 4 + BASE(y, b)];
      const int Lmax = min(MAXLOOP, d - 4);
      const int nyy = (d >= 6) ? Lmax - 1 : 0;
      const int ntask = nyy + 2 * MAXLOOP;
      T acc = 0;
      for (int k = g; k < ntask; k += G) {
        if (k < nyy) {
          const int L = k + 2;
          T v;
          if (L == 2) {
            v = XIo[pe];
          } else {
            v = s2<false, false>(Tx, S + (SI_YYP + L - 3) * BLK, a, b, M1);
            const int yl = y - L + 2;
            if (yl - x >= 6) v += s2<false, false>(S + (SI_XIL + L - 3) * BLK, S + (SI_CHL + L - 3) * BLK, a, b, MP(yl));
          }
          YO[(L - 2) * BLK + pe] = v;
          p.YY[(c * NYY + (L - 2)) * BLK + pe] = v;
          acc += wIn[L] * tmo * v;
        } else {
          const int q = k - nyy, L = q / 2 + 1;
          if (d - L < 4) continue;
          const T f = wBu[L];
          if ((q & 1) == 0)
            acc += f * s2<false, false>(S + (SI_BQ3 + L - 1) * BLK, S + (SI_BC3 + L - 1) * BLK, a, b, MP(y - L));
          else
            acc += f * s2<false, false>(S + (SI_BC5 + L - 1) * BLK, S + (SI_BQ5 + L - 1) * BLK, a, b, MP(x + L));
        }
      }
      if (g == 0) acc += wHp * tmo * CHo[pe];
      RED[t] = acc;
    }
  }
  __syncthreads();
  if (d >= 2 && t < MM) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    T v = 0;
    for (int g = 0; g < GR; g++) v += RED[g * MM + t];
    HBo[pe] = v;
    p.HB[c * BLK + pe] = v;
    lmax = fmax(lmax, (double)fabs(v));
  }
  // ---- P3: QB of the closing pair (x, y): four partial terms per entry
  if (d >= 4 && t >= 64 && t < 64 + 4 * MM) {
    const int sub = (t - 64) / MM, e = (t - 64) % MM, a = e / My, b = e % My;
    const int pto = pair_type(BASE(x, a), BASE(y, b));
    T v = 0;
    if (pto >= 0) {
      if (sub == 0) {
        v = s3<false, false, false>(Tx, S + SI_HBI * BLK, Ty1, a, b, M1, Mv);
      } else if (sub == 1) {
        if (d >= 6) {
          const T *qin = S + SI_QBI * BLK;
          for (int a2 = 0; a2 < M1; a2++) {
            const T tv = Tx[a * NS + a2];
            if (tv == (T)0) continue;
            const int ba = BASE((x + 1), a2);
            for (int b2 = 0; b2 < Mv; b2++) {
              const int pti = pair_type(ba, BASE((y - 1), b2));
              if (pti >= 0) v += tv * qin[a2 * NS + b2] * Ty1[b2 * NS + b] * en[EN_STK + pto * 6 + pti];
            }
          }
        }
      } else if (d >= 11) {
        const T *Xl = S + SI_XX * BLK, *Xr = S + SI_XY1 * BLK, *q2 = S + SI_Q2I * BLK;
        if (sub == 2)
          v = s3<false, false, false>(Xl + XPU * BLK, q2 + 0 * BLK, Xr + XUP * BLK, a, b, M1, Mv) +
              s3<false, false, false>(Xl + XPU * BLK, q2 + 1 * BLK, Xr + XPP * BLK, a, b, M1, Mv);
        else
          v = s3<false, false, false>(Xl + XPP * BLK, q2 + 2 * BLK, Xr + XUP * BLK, a, b, M1, Mv) +
              s3<false, false, false>(Xl + XPP * BLK, q2 + 3 * BLK, Xr + XPP * BLK, a, b, M1, Mv);
        v *= en[EN_EA] * en[EN_EC];
      }
    }
    RED2[t - 64] = v;
  }
  __syncthreads();
  if (d >= 4 && t < MM) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    const T v = (RED2[t] + RED2[MM + t] + RED2[2 * MM + t] + RED2[3 * MM + t]) * clamp_p2<T>(EA(d - 2) - Ed);
    QBo[pe] = v;
    p.QB[c * BLK + pe] = v;
    lmax = fmax(lmax, (double)fabs(v));
  }
  __syncthreads();

  // ---- P4: QMpp/QM2pp (0..MM), QMpu+G (64..), QM2pu/up/uu (128..), exterior (192..)
  if (d >= 4 && t < MM) {
    const int a = t / My, b = t % My, pe = a * NS + b;
    (void)a;
    (void)b;
    const T s2v = nchunk_bif(d) > 0 ? S[SI_BIF * BLK + pe] * clamp_p2<T>(EA(d - 4) - Ed) : (T)0;
    const T v = en[EN_EC] * QBo[pe] + s2v;
    p.QM2pp[c * BLK + pe] = s2v;
    p.QMpp[c * BLK + pe] = v;
    lmax = fmax(lmax, fmax((double)fabs(v), (double)fabs(s2v)));
  } else if (d >= 5 && t >= 64 && t < 64 + MM) {
    const int e = t - 64, a = e / My, b = e % My, pe = a * NS + b;
    const T F1 = clamp_p2<T>(EA(d - 1) - Ed), eb = en[EN_EB];
    const T *Xr = S + SI_XY1 * BLK, *mpp = S + SI_ML * BLK, *mpu = S + (SI_ML + 1) * BLK;
    const T u = eb * F1 * (s2<false, false>(mpp, Xr + XPU * BLK, a, b, Mv) + s2<false, false>(mpu, Xr + XUU * BLK, a, b, Mv));
    const T gg = F1 * (s2<false, false>(mpp, Xr + XPP * BLK, a, b, Mv) + s2<false, false>(mpu, Xr + XUP * BLK, a, b, Mv));
    p.QMpu[c * BLK + pe] = u;
    p.G[c * BLK + pe] = gg;
    lmax = fmax(lmax, fmax((double)fabs(u), (double)fabs(gg)));
  } else if (d >= 10 && t >= 128 && t < 128 + MM) {
    const int e = t - 128, a = e / My, b = e % My, pe = a * NS + b;
    const T F1 = clamp_p2<T>(EA(d - 1) - Ed), eb = en[EN_EB];
    const T *Xr = S + SI_XY1 * BLK, *Xl = S + SI_XX * BLK;
    const T *q2pp = S + (SI_ML + 2) * BLK, *q2pu = S + (SI_ML + 3) * BLK;
    const T *r_up = S + SI_MR * BLK, *r_pp = S + (SI_MR + 1) * BLK, *r_uu = S + (SI_MR + 2) * BLK,
            *r_pu = S + (SI_MR + 3) * BLK;
    const T pu = eb * F1 * (s2<false, false>(q2pp, Xr + XPU * BLK, a, b, Mv) + s2<false, false>(q2pu, Xr + XUU * BLK, a, b, Mv));
    const T up = eb * F1 * (s2<false, false>(Xl + XUU * BLK, r_up, a, b, M1) + s2<false, false>(Xl + XUP * BLK, r_pp, a, b, M1));
    const T uu = eb * F1 * (s2<false, false>(Xl + XUU * BLK, r_uu, a, b, M1) + s2<false, false>(Xl + XUP * BLK, r_pu, a, b, M1));
    p.QM2pu[c * BLK + pe] = pu;
    p.QM2up[c * BLK + pe] = up;
    p.QM2uu[c * BLK + pe] = uu;
    lmax = fmax(lmax, fmax((double)fabs(pu), fmax((double)fabs(up), (double)fabs(uu))));
  } else if (x == 0 && t >= 192 && t < 192 + MP(0) * My) {
    // ---- exterior prefix [0, d]
    const int M0 = MP(0), e = t - 192, a = e / My, b = e % My, pe = a * NS + b;
    T *q5u = p.Q5U + (size_t)d * BLK, *q5p = p.Q5P + (size_t)d * BLK;
    if (d == 0) {
      q5u[pe] = (a == b) ? (T)1 : (T)0;
      q5p[pe] = 0;
      lmax = fmax(lmax, 1.0);
    } else {
      const T F1 = clamp_p2<T>(EA(d - 1) - Ed);
      const T *Xr = S + SI_XY1 * BLK;
      const T *pu = S + SI_Q5U * BLK, *pp = S + SI_Q5P * BLK;
      const T gg = F1 * (s2<false, false>(pu, Xr + XUP * BLK, a, b, Mv) + s2<false, false>(pp, Xr + XPP * BLK, a, b, Mv));
      const T u = F1 * (s2<false, false>(pu, Xr + XUU * BLK, a, b, Mv) + s2<false, false>(pp, Xr + XPU * BLK, a, b, Mv));
      p.Gx[(size_t)d * BLK + pe] = gg;
      q5u[pe] = u;
      T v = (d >= 4 ? QBo[pe] : (T)0);
      if (nchunk_ext(d) > 0) v += S[SI_BIFX * BLK + pe] * clamp_p2<T>(EA(d - 4) - Ed);
      // split points k = 1..3 use QB[k][d] of diagonals d-1..d-3
      for (int k = 1; k <= 3 && k <= d - 4; k++)
        v += clamp_p2<T>(EA(k) + EA(d - k) - Ed) *
             s2<false, false>(S + (SI_GXK + k - 1) * BLK, S + (SI_QBK + k - 1) * BLK, a, b, MP(k));
      q5p[pe] = v;
      lmax = fmax(lmax, fmax((double)fabs(gg), fmax((double)fabs(u), (double)fabs(v))));
    }
  }

  // ---- diagonal maximum for the next exponent
  lmax = warp_max(lmax);
  if (lane == 0) smax[w] = lmax;
  __syncthreads();
  if (t == 0) {
    double m = 0;
    for (int k = 0; k < NTT / 32; k++) m = fmax(m, smax[k]);
    atomic_max_pos(&p.dmax[d], m);
  }
}

template <typename T, int NTT>
__global__ void __launch_bounds__(NTT) k_in_light(DP<T> p, BifBuf<T> bb, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  in_light_cell<T, NTT>(p, bb, d, blockIdx.x, smem_raw);
}

template <typename T, int NTT = NT>
constexpr size_t in_light_smem() {
  return ((size_t)(SI_N + 4 + NYY + 4) * BLK + NTT) * sizeof(T);
}

}  // namespace cf
