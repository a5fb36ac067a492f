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
constexpr int NT_IN = 256;    // threads per cell of the inside light kernel
constexpr int NT = 512;       // threads per cell on diagonals with few cells
constexpr int NT_WIDE = 256;  // ... and on diagonals with more than WIDE_CELLS cells
constexpr int WIDE_CELLS = 296;

// ---------------------------------------------------------------- row products
// Every table entry is a 6x6 block whose rows and columns beyond the codon-
// state counts are zero, so block products can always run over the full
// padded size: the padding contributes exact zeros.  Fixed trip counts let the
// compiler keep a row of the left operand in registers and stream the rows of
// the right operand with 8/16-byte shared-memory loads.
template <typename T>
struct Row2;
template <>
struct Row2<float> {
  using type = float2;
};
template <>
struct Row2<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ void ld_row(T (&r)[NS], const T *src) {
  using V = typename Row2<T>::type;
  const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    const V v = s[i];
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void st_row(T *dst, const T (&r)[NS]) {
  using V = typename Row2<T>::type;
  V *d = reinterpret_cast<V *>(dst);
#pragma unroll
  for (int i = 0; i < NS / 2; i++) {
    V v;
    v.x = r[2 * i];
    v.y = r[2 * i + 1];
    d[i] = v;
  }
}
// r += (f * av) . B   (av: one row of the left operand)
template <typename T>
__device__ __forceinline__ void row_acc(T (&r)[NS], const T (&av)[NS], const T *B, T f) {
#pragma unroll
  for (int s = 0; s < NS; s++) {
    T bv[NS];
    ld_row(bv, B + s * NS);
    const T x = av[s] * f;
#pragma unroll
    for (int b = 0; b < NS; b++) r[b] = fma(x, bv[b], r[b]);
  }
}
// r += f * (row a of A) . B
template <typename T>
__device__ __forceinline__ void row_mm(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
  ld_row(av, A + a * NS);
  row_acc(r, av, B, f);
}
// r += f * (row a of A) . B . C
template <typename T>
__device__ __forceinline__ void row_mmm(T (&r)[NS], const T *A, const T *B, const T *C, int a, T f) {
  T t[NS];
#pragma unroll
  for (int b = 0; b < NS; b++) t[b] = (T)0;
  row_mm(t, A, B, a, (T)1);
  row_acc(r, t, C, f);
}
// r += f * (row a of A^T) . B  = f * sum_s A[s][a] B[s][.]
template <typename T>
__device__ __forceinline__ void row_tmm(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
#pragma unroll
  for (int s = 0; s < NS; s++) av[s] = A[s * NS + a];
  row_acc(r, av, B, f);
}
// r += f * (row a of A) . B^T  = f * sum_s A[a][s] B[.][s]
template <typename T>
__device__ __forceinline__ void row_mmt(T (&r)[NS], const T *A, const T *B, int a, T f) {
  T av[NS];
  ld_row(av, A + a * NS);
#pragma unroll
  for (int s = 0; s < NS; s++) av[s] *= f;
#pragma unroll
  for (int b = 0; b < NS; b++) {
    T bv[NS];
    ld_row(bv, B + b * NS);
    T acc = r[b];
#pragma unroll
    for (int s = 0; s < NS; s++) acc = fma(av[s], bv[s], acc);
    r[b] = acc;
  }
}
// atomically add a block row to global memory, skipping exact-zero pairs
__device__ __forceinline__ void red_row(float *dst, const float (&r)[NS]) {
#pragma unroll
  for (int i = 0; i < NS / 2; i++)
    if (r[2 * i] != 0.f || r[2 * i + 1] != 0.f)
      asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst + 2 * i), "f"(r[2 * i]), "f"(r[2 * i + 1])
                   : "memory");
}
__device__ __forceinline__ void red_row(double *dst, const double (&r)[NS]) {
#pragma unroll
  for (int i = 0; i < NS; i++)
    if (r[i] != 0.0) atomicAdd(dst + i, r[i]);
}

template <typename T>
__device__ __forceinline__ void row_zero(T (&r)[NS]) {
#pragma unroll
  for (int b = 0; b < NS; b++) r[b] = (T)0;
}
template <typename T>
__device__ __forceinline__ T row_absmax(const T (&r)[NS]) {
  T m = 0;
#pragma unroll
  for (int b = 0; b < NS; b++) m = fmax(m, fabs(r[b]));
  return m;
}

// ---------------------------------------------------------------- K2
// Light work of one cell (x, y) of diagonal d in two phases of independent
// work, split by task and block row (6 threads per task, one output row
// each):
//   phase A  chain, XI, the 28 interior partial sums YY_3..YY_30, the bulge
//            sums (12 partial blocks), the QB terms (hairpin-interior,
//            stack in 3 parts, multiloop in 2), QMpu, G, QM2pu/up/uu and the
//            exterior row;
//   phase B  HB (sum over interior sizes, bulges and hairpin), QB, QMpp,
//            QM2pp and the exterior Q5P, entry by entry.
// Staged input slots that a diagonal does not use are zero-filled, so every
// task runs unconditionally; loop weights that do not apply are zero.
enum : int {
  LT_CH = 0, LT_XI = 1, LT_YY = 2,            // YY_L, L = 3..30: tasks 2..29
  LT_BU = 30, NLT_BU = 12,                    // bulges: tasks 30..41
  LT_QBH = 42, LT_QBS = 43, NLT_QBS = 3,      // QB: hairpin-interior term, stack in 3 parts
  LT_QBM = 46,                                // QB: multiloop, 2 parts (46, 47)
  LT_QMPU = 48, LT_G = 49, LT_M2PU = 50, LT_M2UP = 51, LT_M2UU = 52,
  LT_GX = 53, LT_Q5U = 54, LT_Q5K = 55,       // exterior (x == 0)
  NLT = 56
};
// shared result slots (blocks): phase A writes 0..LO_Q5U, phase B the rest;
// every final result is copied to its table at the end of the cell
enum : int {
  LO_CH = 0, LO_XI = 1, LO_YY = 2,            // YY_L at LO_YY + L - 3
  LO_BU = 30, LO_QBH = 42, LO_QBS = 43, LO_QBM = 46, LO_Q5K = 48,
  LO_QMPU = 49, LO_G = 50, LO_M2PU = 51, LO_M2UP = 52, LO_M2UU = 53, LO_GX = 54, LO_Q5U = 55,
  LO_HB = 56, LO_QB = 57, LO_QMPP = 58, LO_QM2PP = 59, LO_Q5P = 60, LO_N = 61
};

// Threads per entry in the HB sum of phase B, and the first thread of the
// QB/QMpp entries (a warp boundary after the HB threads).
template <int NTT>
struct LightMap {
  static constexpr int GHB = NTT >= 512 ? 8 : 4;
  static constexpr int QB0 = (GHB * BLK + 31) / 32 * 32;
  static_assert(QB0 + BLK <= NTT, "phase B needs one thread per QB entry");
};

template <typename T, int NTT>
__device__ __forceinline__ void in_light_cell(const DP<T> &p, const BifBuf<T> &bb, int d, int x,
                                              unsigned char *smem_raw) {
  using LM = LightMap<NTT>;
  T *S = (T *)smem_raw;                // [SI_N][36] staged inputs
  T *O = S + (size_t)SI_N * BLK;       // [LO_N][36] phase A results
  __shared__ int sEd;
  __shared__ double smax[NTT / 32];
  __shared__ int sE[96], sBx[3][NS], sBy[3][NS];
  __shared__ T sEn[EN_N];
  __shared__ __align__(8) unsigned long long sbar;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = p.n;
  const int y = x + d;
  // per-cell context, each value loaded by its own thread before any copy is
  // issued so that all loads are in flight together: exponents of diagonals
  // d-47..d-1, bases of x-1..x+1 and y-1..y+1, energy factors, and the
  // largest mantissa and exponent of diagonal d-1 (last thread)
  static_assert(NTT > EN_N && NTT > 96 + 6 * NS, "one context value per thread");
  int cE = 0, cB = 0;
  T cEn = 0;
  unsigned long long cMax = 0;
  if (t < EN_N) cEn = p.en[t];
  if (t < 96) {
    const int k = d - 47 + t;
    if (k >= 0 && k < d) cE = __ldcg(p.E + k);
  } else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    const int q = (side == 0 ? x : y) - 1 + r;
    if (q >= 0 && q < n) cB = p.base[q * NS + a];
  } else if (t == NTT - 1 && d > 0) {
    cMax = __ldcg(p.dmax + d - 1);
    cE = __ldcg(p.E + d - 1);
  }
  if (t == 0) mbar_init(&sbar, 1);
  __syncthreads();
  // Staging: one TMA bulk copy per input block (the interior partial sums
  // YY_{L-1}[x+1][y], L = 3..Lmax, are contiguous and go as one copy); slots
  // this cell does not use are zero-filled.  Each issuing thread adds its
  // bytes to the barrier's transaction count before its copy; thread 0 arrives
  // once every thread has done so.
  {
    const int LmaxS = min(MAXLOOP, d - 4);
    for (int s = t; s < SI_N; s += NTT) {
      T *dst = S + (size_t)s * BLK;
      if (s > SI_YYP && s < SI_XIL && d >= 6 && s - SI_YYP + 3 <= LmaxS) continue;  // part of the YY run
      const T *src = s < SI_BIF ? in_slot_src(p, s, x, y, d) : in_slot_src2(p, bb, s, x, d);
      if (src) {
        const unsigned bytes = (s == SI_YYP ? (unsigned)(LmaxS - 2) : 1u) * BLK * (unsigned)sizeof(T);
        mbar_expect(&sbar, bytes);
        bulk_g2s(dst, src, bytes, &sbar);
      } else {
#pragma unroll
        for (int q = 0; q < BLK; q++) dst[q] = (T)0;
      }
    }
  }
  if (t < EN_N) sEn[t] = cEn;
  if (t < 96) {
    sE[t] = cE;
  } else if (t < 96 + 6 * NS) {
    const int i = t - 96, side = i / (3 * NS), r = (i / NS) % 3, a = i % NS;
    if (side == 0) sBx[r][a] = cB;
    else sBy[r][a] = cB;
  } else if (t == NTT - 1) {
    int e = 0;
    if (d > 0) {
      const double mx = __longlong_as_double((long long)cMax);
      e = cE;
      if (mx > 0) {
        if (isfinite(mx)) e += ilogb(mx);
        else atomicOr(p.err, 1);
      }
    }
    sEd = e;
    if (x == 0) p.E[d] = e;
  }
  __syncthreads();
  if (t == 0) mbar_arrive(&sbar);
  if (!mbar_wait(&sbar, 0, p.err)) return;
  const int Ed = sEd;
  const T *en = sEn;
  const size_t c = cidx(n, x, y);
  const T *Tx = S + SI_TX * BLK, *Ty1 = S + SI_TY1 * BLK;
  const T *Xl = S + SI_XX * BLK, *Xr = S + SI_XY1 * BLK;
  const int Lmax = min(MAXLOOP, d - 4);
  double lmax = 0.0;

  // ---------------- phase A: one block row per thread and step
  for (int rt = t; rt < NS * NLT; rt += NTT) {
    const int task = rt / NS, a = rt - task * NS;
    T r[NS];
    row_zero(r);
    int oslot = -1;      // shared result slot
    bool scaled = true;  // counts toward the diagonal maximum
    if (task == LT_CH) {
      if (d == 0) {
        const int Mx = p.Mp[x];
#pragma unroll
        for (int b = 0; b < NS; b++) r[b] = (a == b && a < Mx) ? (T)1 : (T)0;
      } else {
        row_mm(r, Tx, S + SI_CHN * BLK, a, (T)1);
      }
      oslot = LO_CH;
      scaled = false;
    } else if (task == LT_XI) {
      if (d >= 6) {
        row_mmm(r, Tx, S + SI_QBI * BLK, Ty1, a, clamp_p2<T>(EA(d - 2) - Ed));
        const int bxa = BASE(x, a);
#pragma unroll
        for (int b = 0; b < NS; b++) r[b] *= en[EN_TM + BASE(y, b) * 4 + bxa];
      }
      oslot = LO_XI;
    } else if (task < LT_BU) {
      const int L = task - LT_YY + 3;
      if (d >= 6 && L <= Lmax) {
        row_mm(r, Tx, S + (SI_YYP + L - 3) * BLK, a, (T)1);
        row_mm(r, S + (SI_XIL + L - 3) * BLK, S + (SI_CHL + L - 3) * BLK, a, (T)1);
      }
      oslot = LO_YY + L - 3;
      scaled = false;  // relative to 2^{E[d-L+2]}
    } else if (task < LT_QBH) {
      // bulges: side 3' (QB[x][y-L] CH[y-L][y]) for even j, 5' (CH[x][x+L] QB[x+L][y]) for odd
      const int j = task - LT_BU, side = j & 1, L0 = (j >> 1) * 5 + 1;
#pragma unroll
      for (int L = L0; L < L0 + 5; L++) {
        if (d - L < 4) break;
        const T f = en[EN_BU + L] * clamp_p2<T>(EA(d - L) - Ed);
        if (side == 0)
          row_mm(r, S + (SI_BQ3 + L - 1) * BLK, S + (SI_BC3 + L - 1) * BLK, a, f);
        else
          row_mm(r, S + (SI_BC5 + L - 1) * BLK, S + (SI_BQ5 + L - 1) * BLK, a, f);
      }
      oslot = LO_BU + j;
      scaled = false;
    } else if (task == LT_QBH) {
      if (d >= 4) row_mmm(r, Tx, S + SI_HBI * BLK, Ty1, a, (T)1);
      oslot = LO_QBH;
      scaled = false;
    } else if (task < LT_QBM) {
      // stack: sum over inner states (a2, b2) with the factor of the
      // (outer, inner) pair types; this part takes a2 in {2j, 2j+1}
      if (d >= 6) {
        const T *qin = S + SI_QBI * BLK;
        int pto[NS];
        const int bxa = BASE(x, a);
#pragma unroll
        for (int b = 0; b < NS; b++) pto[b] = pair_type(bxa, BASE(y, b));
        const int j = task - LT_QBS;
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int a2 = 2 * j + q;
          const T tv = Tx[a * NS + a2];
          if (tv != (T)0) {
            const int ba = BASE((x + 1), a2);
#pragma unroll
            for (int b2 = 0; b2 < NS; b2++) {
              const int pti = pair_type(ba, BASE((y - 1), b2));
              const T u = tv * qin[a2 * NS + b2];
              if (pti >= 0 && u != (T)0) {
                T tyr[NS];
                ld_row(tyr, Ty1 + b2 * NS);
#pragma unroll
                for (int b = 0; b < NS; b++)
                  if (pto[b] >= 0) r[b] = fma(u * en[EN_STK + pto[b] * 6 + pti], tyr[b], r[b]);
              }
            }
          }
        }
      }
      oslot = LO_QBS + task - LT_QBS;
      scaled = false;
    } else if (task < LT_QMPU) {
      if (d >= 11) {
        const T *q2 = S + SI_Q2I * BLK;
        if (task == LT_QBM) {
          row_mmm(r, Xl + XPU * BLK, q2 + 0 * BLK, Xr + XUP * BLK, a, (T)1);
          row_mmm(r, Xl + XPU * BLK, q2 + 1 * BLK, Xr + XPP * BLK, a, (T)1);
        } else {
          row_mmm(r, Xl + XPP * BLK, q2 + 2 * BLK, Xr + XUP * BLK, a, (T)1);
          row_mmm(r, Xl + XPP * BLK, q2 + 3 * BLK, Xr + XPP * BLK, a, (T)1);
        }
      }
      oslot = LO_QBM + task - LT_QBM;
      scaled = false;
    } else if (task == LT_QMPU || task == LT_G) {
      if (d >= 5) {
        const T F1 = clamp_p2<T>(EA(d - 1) - Ed);
        const T *mpp = S + SI_ML * BLK, *mpu = S + (SI_ML + 1) * BLK;
        if (task == LT_QMPU) {
          const T f = en[EN_EB] * F1;
          row_mm(r, mpp, Xr + XPU * BLK, a, f);
          row_mm(r, mpu, Xr + XUU * BLK, a, f);
        } else {
          row_mm(r, mpp, Xr + XPP * BLK, a, F1);
          row_mm(r, mpu, Xr + XUP * BLK, a, F1);
        }
      }
      oslot = task == LT_QMPU ? LO_QMPU : LO_G;
    } else if (task <= LT_M2UU) {
      if (d >= 10) {
        const T f = en[EN_EB] * clamp_p2<T>(EA(d - 1) - Ed);
        if (task == LT_M2PU) {
          row_mm(r, S + (SI_ML + 2) * BLK, Xr + XPU * BLK, a, f);
          row_mm(r, S + (SI_ML + 3) * BLK, Xr + XUU * BLK, a, f);
        } else if (task == LT_M2UP) {
          row_mm(r, Xl + XUU * BLK, S + SI_MR * BLK, a, f);
          row_mm(r, Xl + XUP * BLK, S + (SI_MR + 1) * BLK, a, f);
        } else {
          row_mm(r, Xl + XUU * BLK, S + (SI_MR + 2) * BLK, a, f);
          row_mm(r, Xl + XUP * BLK, S + (SI_MR + 3) * BLK, a, f);
        }
      }
      oslot = LO_M2PU + task - LT_M2PU;
    } else if (task < NLT && x == 0) {
      // exterior prefix [0, d]: rows are the states of position 0
      const T *pu = S + SI_Q5U * BLK, *pp = S + SI_Q5P * BLK;
      if (task == LT_GX) {
        if (d >= 1) {
          const T F1 = clamp_p2<T>(EA(d - 1) - Ed);
          row_mm(r, pu, Xr + XUP * BLK, a, F1);
          row_mm(r, pp, Xr + XPP * BLK, a, F1);
        }
        oslot = LO_GX;
      } else if (task == LT_Q5U) {
        if (d == 0) {
          const int M0 = p.Mp[0];
#pragma unroll
          for (int b = 0; b < NS; b++) r[b] = (a == b && a < M0) ? (T)1 : (T)0;
        } else {
          const T F1 = clamp_p2<T>(EA(d - 1) - Ed);
          row_mm(r, pu, Xr + XUU * BLK, a, F1);
          row_mm(r, pp, Xr + XPU * BLK, a, F1);
        }
        oslot = LO_Q5U;
      } else {
        // split points k = 1..3 use QB[k][d] of diagonals d-1..d-3
        for (int k = 1; k <= 3 && k <= d - 4; k++)
          row_mm(r, S + (SI_GXK + k - 1) * BLK, S + (SI_QBK + k - 1) * BLK, a, clamp_p2<T>(EA(k) + EA(d - k) - Ed));
        oslot = LO_Q5K;
        scaled = false;
      }
    }
    if (oslot >= 0) {
      st_row(O + (size_t)oslot * BLK + a * NS, r);
      if (scaled) lmax = fmax(lmax, (double)row_absmax(r));
    }
  }
  __syncthreads();

  // ---------------- phase B: HB, QB, QMpp, QM2pp, exterior Q5P per entry
  // HB: GHB consecutive threads per entry split the interior sizes and bulge parts
  {
    constexpr int GHB = LM::GHB;
    const int e = t / GHB, g = t % GHB, a = e / NS, b = e % NS;
    T v = 0;
    if (e < BLK && d >= 2) {
      const T tmo = en[EN_TM + BASE(x, a) * 4 + BASE(y, b)];
      for (int L = 2 + g; L <= Lmax; L += GHB) {
        const T wl = en[EN_IN + L] * clamp_p2<T>(EA(d - L + 2) - Ed);
        const T yv = (L == 2) ? O[LO_XI * BLK + e] : O[(LO_YY + L - 3) * BLK + e];
        v = fma(wl * tmo, yv, v);
      }
      for (int j = g; j < NLT_BU; j += GHB) v += O[(LO_BU + j) * BLK + e];
      if (g == 0) v = fma(p.eHL[d + 1] * clamp_p2<T>(-Ed) * tmo, O[LO_CH * BLK + e], v);
    }
#pragma unroll
    for (int o = 1; o < GHB; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (e < BLK && g == 0) {
      O[LO_HB * BLK + e] = v;
      lmax = fmax(lmax, (double)fabs(v));
    }
  }
  if (t >= LM::QB0 && t < LM::QB0 + BLK) {
    const int e = t - LM::QB0, a = e / NS, b = e % NS;
    T qb = 0;
    if (d >= 4) {
      const int pto = pair_type(BASE(x, a), BASE(y, b));
      if (pto >= 0) {
        T v = O[LO_QBH * BLK + e];
#pragma unroll
        for (int j = 0; j < NLT_QBS; j++) v += O[(LO_QBS + j) * BLK + e];
        v += en[EN_EA] * en[EN_EC] * (O[LO_QBM * BLK + e] + O[(LO_QBM + 1) * BLK + e]);
        qb = v * clamp_p2<T>(EA(d - 2) - Ed);
      }
      O[LO_QB * BLK + e] = qb;
      const T s2v = S[SI_BIF * BLK + e] * clamp_p2<T>(EA(d - 4) - Ed);
      const T mpp = en[EN_EC] * qb + s2v;
      O[LO_QM2PP * BLK + e] = s2v;
      O[LO_QMPP * BLK + e] = mpp;
      lmax = fmax(lmax, fmax((double)fabs(qb), fmax((double)fabs(mpp), (double)fabs(s2v))));
    }
    if (x == 0) {
      T v;
      if (d == 0) {
        v = 0;
        lmax = fmax(lmax, 1.0);
      } else {
        v = qb + S[SI_BIFX * BLK + e] * clamp_p2<T>(EA(d - 4) - Ed) + O[LO_Q5K * BLK + e];
        lmax = fmax(lmax, (double)fabs(v));
      }
      O[LO_Q5P * BLK + e] = v;
    }
  }

  lmax = warp_max(lmax);
  if (lane == 0) smax[w] = lmax;
  __syncthreads();

  // ---------------- results to their tables, 16 bytes per thread and step
  {
    constexpr int CH16 = BLK * (int)sizeof(T) / 16;
    using V = typename Vec16<T>::type;
    for (int it = t; it < 45 * CH16; it += NTT) {
      const int k = it / CH16, q = it - k * CH16;
      int slot;
      T *dst = nullptr;
      if (k == 0) {
        slot = LO_CH;
        dst = p.CH + c * BLK;
      } else if (k == 1) {
        slot = LO_XI;
        if (d >= 6) dst = p.XI + c * BLK;
      } else if (k == 2) {  // YY_2 is XI itself
        slot = LO_XI;
        if (d >= 6) dst = p.YY + (c * NYY) * BLK;
      } else if (k < 31) {  // YY_L, L = 3..30
        const int L = k;
        slot = LO_YY + L - 3;
        if (d >= 6 && L <= Lmax) dst = p.YY + (c * NYY + (L - 2)) * BLK;
      } else if (k == 31) {
        slot = LO_HB;
        if (d >= 2) dst = p.HB + c * BLK;
      } else if (k == 32) {
        slot = LO_QB;
        if (d >= 4) dst = p.QB + c * BLK;
      } else if (k == 33) {
        slot = LO_QMPP;
        if (d >= 4) dst = p.QMpp + c * BLK;
      } else if (k == 34) {
        slot = LO_QM2PP;
        if (d >= 4) dst = p.QM2pp + c * BLK;
      } else if (k == 35) {
        slot = LO_QMPU;
        if (d >= 5) dst = p.QMpu + c * BLK;
      } else if (k == 36) {
        slot = LO_G;
        if (d >= 5) dst = p.G + c * BLK;
      } else if (k < 40) {
        slot = LO_M2PU + k - 37;
        T *tab[3] = {p.QM2pu, p.QM2up, p.QM2uu};
        if (d >= 10) dst = tab[k - 37] + c * BLK;
      } else if (k == 40) {
        slot = LO_GX;
        if (x == 0 && d >= 1) dst = p.Gx + (size_t)d * BLK;
      } else if (k == 41) {
        slot = LO_Q5U;
        if (x == 0) dst = p.Q5U + (size_t)d * BLK;
      } else if (k == 42) {
        slot = LO_Q5P;
        if (x == 0) dst = p.Q5P + (size_t)d * BLK;
      } else {
        slot = 0;
      }
      if (dst) reinterpret_cast<V *>(dst)[q] = reinterpret_cast<const V *>(O + (size_t)slot * BLK)[q];
    }
  }
  // ---- diagonal maximum for the next exponent
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

template <typename T, int NTT = NT_IN>
constexpr size_t in_light_smem() {
  return (size_t)(SI_N + LO_N) * BLK * sizeof(T);
}

}  // namespace cf
