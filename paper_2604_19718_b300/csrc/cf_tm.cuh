// cf_tm.cuh -- log Z of a protein under the paper's own tensor-based free
// energy model (SI "Tensor-based free energy models", Eq. general-model):
// gamma x gamma matrices V_x (unpaired base x), B^rho_{x,y} (the two sides of
// a base pair, rho = 0..nrho-1) and S (weighted trace Tr_S[X] = tr(S X)),
// summed over every codon sequence of the protein with the codon-pair tensor
// train of Eq. pair-tt (the same position transfers T_p as the
// nearest-neighbour path).
//
// The recursion is Eq. complicated-pf with the fold of Eq. fold generalised
// to codon states as in Eq. design-fold.  For an interval [i, j) the block
// Q[i, j] is a matrix over (codon state at i, zeta) x (codon state at j-1,
// zeta'), flattened state-major and padded to TM_D = 6 states x TM_G = 4:
//   Q[i, i+1]  = delta_ab V_{x_i(a)}
//   Q[i, j+1]  = Q[i, j] X_j + sum_{k=i}^{j-4} L[i, k] F[k, j]
//   X_j        = T_{j-1} (x) V_j                 (base j unpaired)
//   L[i, i]    = identity, L[i, k] = Q[i, k] (T_{k-1} (x) I)
//   F[k, j]    = sum_rho B^rho_{k,j} Tr_S[B^rho_{j,k} Y],
//   Y          = (T_k (x) I) Q[k+1, j] (T_{j-1} (x) I)   (k paired to j)
//   Z          = sum_{a,c} u0[a] Tr_S[Q[0, n]_{a c}].
// The paper evaluates the same sum column by column with a triangular
// matrix product per column (Alg. fast-pf); here it runs by interval length
// (anti-diagonals), like the nearest-neighbour path: per length L, the folds
// of the pairs at distance L-1 (k_tm_fold) and then the cells of length L
// (k_tm_cell, one CTA per cell, or a cluster of CTAs per cell when a length
// has few cells), so that a per-length power-of-two exponent
// E[L] keeps binary32 mantissas in range: Q and L of length L carry E[L], F
// of distance D carries E[D-1], and every product term takes the exact
// factor 2^{E[.] + E[.] - E[L]}.  E[L] is set from the largest mantissa of
// length L-1.
#pragma once
#include "cf_common.cuh"
#include "cf_inside.cuh"

namespace cf {

constexpr int TM_G = 4;             // largest structural dimension gamma
constexpr int TM_R = 4;             // largest number of pair conformations rho
constexpr int TM_D = NS * TM_G;     // padded block side (state, zeta)
constexpr int TM_BLK = TM_D * TM_D;  // 576 entries per block
constexpr int TM_NT = TM_BLK;       // threads of the cell and fold kernels: one per block entry

// model on the device (binary64): V[x][g][g], B[rho][x][y][g][g], SB = S B, S[g][g]
struct TmModelDev {
  double V[4][TM_G][TM_G];
  double B[TM_R][4][4][TM_G][TM_G];
  double SB[TM_R][4][4][TM_G][TM_G];
  double S[TM_G][TM_G];
};

template <typename T>
struct TmArgs {
  int n, nrho;
  const int *Mp, *base;       // codon-state counts, base of state a at p [n*6]
  const double *Tr;           // position transfers [n*36] (binary64 masters)
  const double *u0, *ls;      // residue-0 weights, per-boundary log rescales
  int nls;
  const TmModelDev *mod;
  T *Q, *L, *F;               // [ncell][TM_BLK], diagonal-major (cidx of [i, j-1])
  int *E;                     // [n + 1] per-length exponents
  unsigned long long *dmax;   // [n + 1] largest |mantissa| per length (binary64 bits)
  double *Zm, *logz;
  int *err;
};

__device__ __forceinline__ size_t tm_cell(int n, int i, int len) { return cidx(n, i, i + len - 1) * TM_BLK; }

// Q[i, i+1] (block-diagonal V) and L[i, i+1] for every position; one CTA per position
template <typename T>
__global__ void __launch_bounds__(TM_NT) k_tm_init(TmArgs<T> a) {
  const int i = blockIdx.x, t = threadIdx.x, n = a.n;
  const int r = t / TM_D, c = t % TM_D, ar = r / TM_G, zr = r % TM_G, ac = c / TM_G, zc = c % TM_G;
  const int M = a.Mp[i];
  __shared__ T q[TM_BLK];
  T v = 0;
  if (ar == ac && ar < M) v = (T)a.mod->V[a.base[i * NS + ar]][zr][zc];
  q[t] = v;
  a.Q[tm_cell(n, i, 1) + t] = v;
  __syncthreads();
  if (i + 1 < n) {  // L[i, i+1] = Q[i, i+1] (T_i (x) I)
    T s = 0;
    const double *tr = a.Tr + (size_t)i * BLK;
#pragma unroll
    for (int b = 0; b < NS; b++) s += q[r * TM_D + b * TM_G + zc] * (T)tr[b * NS + ac];
    a.L[tm_cell(n, i, 1) + t] = s;
  }
  // the largest |entry| of length 1
  T m = fabs(v);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((t & 31) == 0) atomic_max_pos(a.dmax + 1, (double)m);
}

// F of the pairs (k, k + D), D = len - 1 >= 4, from Q[k+1, k+D] (length D-1);
// one CTA per k
template <typename T>
__global__ void __launch_bounds__(TM_NT) k_tm_fold(TmArgs<T> a, int len) {
  const int n = a.n, D = len - 1, k = blockIdx.x, j = k + D, t = threadIdx.x;
  const int r = t / TM_D, c = t % TM_D, ar = r / TM_G, zr = r % TM_G, ac = c / TM_G, zc = c % TM_G;
  __shared__ T q[TM_BLK], y1[TM_BLK], tk[BLK], tj[BLK], tr[TM_R][BLK];
  __shared__ int xk[NS], xj[NS];
  q[t] = a.Q[tm_cell(n, k + 1, D - 1) + t];
  if (t < BLK) {
    tk[t] = (T)a.Tr[(size_t)k * BLK + t];
    tj[t] = (T)a.Tr[(size_t)(j - 1) * BLK + t];
  }
  if (t < NS) {
    xk[t] = t < a.Mp[k] ? a.base[k * NS + t] : 0;
    xj[t] = t < a.Mp[j] ? a.base[j * NS + t] : 0;
  }
  __syncthreads();
  // y1 = (T_k (x) I) Q
  {
    T s = 0;
#pragma unroll
    for (int b = 0; b < NS; b++) s += tk[ar * NS + b] * q[(b * TM_G + zr) * TM_D + c];
    y1[t] = s;
  }
  __syncthreads();
  // Y = y1 (T_{j-1} (x) I), into q
  {
    T s = 0;
#pragma unroll
    for (int e = 0; e < NS; e++) s += y1[r * TM_D + e * TM_G + zc] * tj[e * NS + ac];
    q[t] = s;
  }
  __syncthreads();
  // the closed loop's trace per (state at k, state at j, rho): Tr_S[B^rho_{j,k} Y_{ac}]
  if (t < BLK * a.nrho) {
    const int rho = t / BLK, ak = (t % BLK) / NS, cj = t % NS;
    const double(*sb)[TM_G] = a.mod->SB[rho][xj[cj]][xk[ak]];
    T s = 0;
#pragma unroll
    for (int e1 = 0; e1 < TM_G; e1++)
#pragma unroll
      for (int e2 = 0; e2 < TM_G; e2++) s += (T)sb[e2][e1] * q[(ak * TM_G + e1) * TM_D + cj * TM_G + e2];
    tr[rho][ak * NS + cj] = s;
  }
  __syncthreads();
  T f = 0;
  if (ar < a.Mp[k] && ac < a.Mp[j])
    for (int rho = 0; rho < a.nrho; rho++) f += (T)a.mod->B[rho][xk[ar]][xj[ac]][zr][zc] * tr[rho][ar * NS + ac];
  a.F[cidx(n, k, j) * TM_BLK + t] = f;
}

// four consecutive values (16-byte aligned) to and from registers
template <typename T>
__device__ __forceinline__ void ld4(T (&v)[4], const T *p);
template <>
__device__ __forceinline__ void ld4<float>(float (&v)[4], const float *p) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<double>(double (&v)[4], const double *p) {
  const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
  v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}
template <typename T>
__device__ __forceinline__ void ldcg4(T (&v)[4], const T *p);
template <>
__device__ __forceinline__ void ldcg4<float>(float (&v)[4], const float *p) {
  const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
  v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
template <>
__device__ __forceinline__ void ldcg4<double>(double (&v)[4], const double *p) {
  const double2 q0 = __ldcg(reinterpret_cast<const double2 *>(p)), q1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
  v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st4<float>(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, const double (&v)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// The cells of length len >= 2; one CTA per cell i, warp-specialised.
// Warp 0 is the producer: its lane 0 streams the split points, tm_kc at a
// time (a group), through a ring of up to TM_NST stages of dynamic shared
// memory, one bulk copy per block of its real rows only (4 M_i rows of
// L[i, k], 4 M_k rows of F[k, j]), each stage completing on its "full"
// mbarrier.  Warps 1-5 are the consumers: consumer c = t - 32 < 144 owns
// output row r = c / 6 (state at i, zeta) and the four columns of the codon
// state qs = c % 6 at j (its four zeta'), so that a block product reads
// 16-byte rows: per state b of the summation index, one 4-vector of the left
// block and four of the right block give 16 FMAs, over the real states of
// the split point only; rows past the real states of i stay zero.  Each
// consumer warp arrives on the stage's "empty" mbarrier when it is done
// with it, and the producer waits for all five before refilling it, so no
// block barrier runs per group.  A wait that runs out sets the error and a
// shared stop flag; the producer then drains its copies in flight.  Launches
// with few long cells split each cell's groups over a cluster of 2, 4 or 8
// CTAs, whose partial sums rank 0 adds over distributed shared memory.
constexpr int TM_NC = TM_D * NS;       // 144 consumer threads
constexpr int TM_NCW = 5;              // consumer warps (the last has 16 idle lanes)
constexpr int TM_NTH = 32 * (1 + TM_NCW);  // 192 threads
constexpr int TM_NST = 8;              // most pipeline stages of a CTA
template <typename T>
__host__ __device__ constexpr int tm_kc() {
  return sizeof(T) == sizeof(float) ? 4 : 2;  // 18 KB per stage in both precisions
}
template <typename T>
__host__ __device__ constexpr size_t tm_stage_bytes() {
  return (size_t)2 * tm_kc<T>() * TM_BLK * sizeof(T);
}
// Stages of the launch for the cells of length len (n - len + 1 CTAs): as
// many as keep all its CTAs resident at once within about 200 KB of shared
// memory per SM (148 SMs), at least one, at most TM_NST and its number of
// groups.  Few long cells get a deep pipeline each, many short ones more CTAs.
template <typename T>
inline int tm_cell_stages(int n, int len, int split = 1) {
  const int ns = len - 5;  // split points k = i+1 .. i+len-5
  if (ns <= 0) return 0;
  const int ng = ((ns + tm_kc<T>() - 1) / tm_kc<T>() + split - 1) / split;  // groups of one CTA
  const int per_sm = ((n - len + 1) * split + 147) / 148;
  const long long budget = 200 * 1024 / per_sm - 1024 - (long long)(2 * TM_BLK + BLK) * sizeof(T);
  const int fit = (int)std::max(1ll, budget / (long long)tm_stage_bytes<T>());
  return std::min(std::min(fit, TM_NST), ng);
}
// the most dynamic shared memory a launch takes (at most 200 KB of stages)
template <typename T>
__host__ __device__ constexpr size_t tm_cell_smem() {
  return (size_t)(TM_NST < 200 * 1024 / tm_stage_bytes<T>() ? TM_NST : 200 * 1024 / tm_stage_bytes<T>()) *
         tm_stage_bytes<T>();
}
// barrier 1 among the consumer warps only
__device__ __forceinline__ void tm_consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * TM_NCW) : "memory"); }
// Launches with few cells split each cell's groups over a cluster of two
// CTAs (TM_SPLIT_CELLS cells or fewer, TM_SPLIT_GROUPS groups or more), of
// four (TM_SPLIT4_*) or of eight (TM_SPLIT8_*).
constexpr int TM_SPLIT_CELLS = 444, TM_SPLIT_GROUPS = 8, TM_SPLIT4_CELLS = 148, TM_SPLIT4_GROUPS = 16;
constexpr int TM_SPLIT8_CELLS = 74, TM_SPLIT8_GROUPS = 32;
// every thread of every CTA of the cluster
__device__ __forceinline__ void tm_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// four consecutive values from the shared memory of CTA `rank` of the cluster
template <typename T>
__device__ __forceinline__ void ld4_peer(T (&v)[4], const T *local, unsigned rank);
template <>
__device__ __forceinline__ void ld4_peer<float>(float (&v)[4], const float *local, unsigned rank) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "r"(ra)
               : "memory");
}
template <>
__device__ __forceinline__ void ld4_peer<double>(double (&v)[4], const double *local, unsigned rank) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];\n" : "=d"(v[0]), "=d"(v[1]) : "r"(ra) : "memory");
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];\n" : "=d"(v[2]), "=d"(v[3]) : "r"(ra + 16u) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(TM_NTH) k_tm_cell(TmArgs<T> a, int len, int nst, int split) {
  // split s > 1: blockIdx.x = s cell + rank, the s CTAs of a cell one cluster
  const int rank = split > 1 ? (int)(blockIdx.x % split) : 0;
  const int n = a.n, i = blockIdx.x / split, t = threadIdx.x, w = t >> 5, c = t - 32;
  const int j = i + len - 1;  // the new last base
  const bool cons = c >= 0 && c < TM_NC;
  const int r = cons ? c / NS : 0, qs = cons ? c % NS : 0;
  constexpr int KC = tm_kc<T>();
  extern __shared__ __align__(128) unsigned char tm_smem[];  // [nst] stages: KC blocks of L, then KC of F
  __shared__ __align__(16) T q[TM_BLK];
  __shared__ __align__(16) T x[TM_BLK];
  __shared__ T tq[BLK], sFac[TM_NST][KC];
  __shared__ int sEL, sMk[TM_NST][KC], sstop;
  __shared__ T smx[TM_NCW];
  __shared__ __align__(16) T part[TM_BLK];  // split > 1: a rank's partial sums, read by rank 0
  __shared__ __align__(8) unsigned long long sfull[TM_NST], sempty[TM_NST];
  const int Mi = a.Mp[i];
  const bool live = cons && r < TM_G * Mi;  // a real row of the output
  const int k0 = i + 1, k1 = j - 4, ngt = k1 >= k0 ? (k1 - k0 + KC) / KC : 0;
  // this CTA's groups [gb, gb + ng): all, or rank r its r-th share of ceil(ngt / split)
  const int gq = (ngt + split - 1) / split, gb = min(ngt, rank * gq), ng = min(ngt, gb + gq) - gb;
  // this length's exponent from the largest mantissa of length len - 1
  if (t == 0) {
    const double mx = __longlong_as_double((long long)__ldcg(a.dmax + len - 1));
    int e = __ldcg(a.E + len - 1);
    if (mx > 0) {
      if (isfinite(mx)) e += ilogb(mx);
      else atomicOr(a.err, 1);
    }
    sEL = e;
    if (i == 0 && rank == 0) a.E[len] = e;
    sstop = 0;
    for (int s = 0; s < nst; s++) {
      mbar_init(&sfull[s], 1);
      mbar_init(&sempty[s], TM_NCW);
    }
  }
  __syncthreads();
  const int EL = sEL;
  T acc[4] = {0, 0, 0, 0};
  int issued = 0;  // producer: groups issued
  if (w == 0) {
    if (t == 0) {
      // group g into stage g % nst once the consumers have released it
      for (int g = 0; g < ng; g++) {
        const int s = g % nst;
        int pm[KC], pe[KC];
#pragma unroll
        for (int u = 0; u < KC; u++) {  // in flight while the stage is awaited
          const int k = k0 + (gb + g) * KC + u;
          pm[u] = k <= k1 ? __ldg(a.Mp + k) : 0;
          pe[u] = k <= k1 ? __ldcg(a.E + (k - i)) + __ldcg(a.E + (j - k - 1)) : 0;
        }
        if (g >= nst && !mbar_wait_peer(&sempty[s], (unsigned)(g / nst - 1) & 1u, a.err)) {
          sstop = 1;
          break;
        }
        if (*(volatile int *)&sstop) break;
        T *sL = reinterpret_cast<T *>(tm_smem + (size_t)s * tm_stage_bytes<T>());
        T *sF = sL + (size_t)KC * TM_BLK;
        unsigned bytes = 0;
#pragma unroll
        for (int u = 0; u < KC; u++) {
          sMk[s][u] = pm[u];
          sFac[s][u] = pm[u] ? clamp_p2<T>(pe[u] - EL) : (T)0;
          if (pm[u]) bytes += (unsigned)((Mi + pm[u]) * TM_G * TM_D * sizeof(T));
        }
        fence_proxy_async();
        mbar_arrive_expect(&sfull[s], bytes);
#pragma unroll
        for (int u = 0; u < KC; u++) {
          const int k = k0 + (gb + g) * KC + u;
          if (!pm[u]) continue;
          bulk_g2s(sL + (size_t)u * TM_BLK, a.L + tm_cell(n, i, k - i), (unsigned)(Mi * TM_G * TM_D * sizeof(T)),
                   &sfull[s]);
          bulk_g2s(sF + (size_t)u * TM_BLK, a.F + cidx(n, k, j) * TM_BLK, (unsigned)(pm[u] * TM_G * TM_D * sizeof(T)),
                   &sfull[s]);
        }
        issued = g + 1;
      }
    }
  } else {
    // X_j = T_{j-1} (x) V_j and Q[i, j] (length len - 1), four entries per consumer
    const int Mj1 = a.Mp[j - 1], Mj = a.Mp[j];
    if (cons) {
      T v4[4];
#pragma unroll
      for (int z = 0; z < 4; z++) {
        const int e = 4 * c + z, u = e / TM_D, cc = e % TM_D, br = u / TM_G, zr = u % TM_G, ac = cc / TM_G,
                  zc = cc % TM_G;
        v4[z] = ac < Mj ? (T)a.Tr[(size_t)(j - 1) * BLK + br * NS + ac] * (T)a.mod->V[a.base[j * NS + ac]][zr][zc]
                        : (T)0;
      }
      st4(x + 4 * c, v4);
      ldcg4(v4, a.Q + tm_cell(n, i, len - 1) + 4 * c);
      st4(q + 4 * c, v4);
    }
    tm_consumer_sync();
    if (live && rank == 0) {
      for (int b = 0; b < Mj1; b++) {  // states at j - 1
        T l4[4];
        ld4(l4, q + r * TM_D + 4 * b);
#pragma unroll
        for (int z1 = 0; z1 < 4; z1++) {
          T f4[4];
          ld4(f4, x + (4 * b + z1) * TM_D + 4 * qs);
#pragma unroll
          for (int z = 0; z < 4; z++) acc[z] = fma(l4[z1], f4[z], acc[z]);
        }
      }
      const T f = clamp_p2<T>(__ldcg(a.E + len - 1) - EL);
#pragma unroll
      for (int z = 0; z < 4; z++) acc[z] *= f;
      // k = i: the pair (i, j) closes the interval's first base (L[i, i] = identity)
      if (j - i >= 4) {
        T f4[4];
        ldcg4(f4, a.F + cidx(n, i, j) * TM_BLK + r * TM_D + 4 * qs);
        const T fe = clamp_p2<T>(__ldcg(a.E + len - 2) - EL);
#pragma unroll
        for (int z = 0; z < 4; z++) acc[z] = fma(f4[z], fe, acc[z]);
      }
    }
    // k = i+1 .. j-4: L[i, k] F[k, j], one group of KC split points per stage
    for (int g = 0; g < ng; g++) {
      const int s = g % nst;
      const bool ok = mbar_wait(&sfull[s], (unsigned)(g / nst) & 1u, a.err);
      // the whole warp leaves together (its __syncwarp below needs every lane)
      if (__any_sync(0xffffffffu, !ok || *(volatile int *)&sstop)) {
        sstop = 1;
        break;
      }
      if (live) {
        const T *sL = reinterpret_cast<const T *>(tm_smem + (size_t)s * tm_stage_bytes<T>());
        const T *sF = sL + (size_t)KC * TM_BLK;
#pragma unroll
        for (int u = 0; u < KC; u++) {
          const T *Lb = sL + (size_t)u * TM_BLK, *Fb = sF + (size_t)u * TM_BLK;
          const int Mk = sMk[s][u];
          T sm[4] = {0, 0, 0, 0};
          for (int b = 0; b < Mk; b++) {
            T l4[4];
            ld4(l4, Lb + r * TM_D + 4 * b);
#pragma unroll
            for (int z1 = 0; z1 < 4; z1++) {
              T f4[4];
              ld4(f4, Fb + (4 * b + z1) * TM_D + 4 * qs);
#pragma unroll
              for (int z = 0; z < 4; z++) sm[z] = fma(l4[z1], f4[z], sm[z]);
            }
          }
          const T f = sFac[s][u];
#pragma unroll
          for (int z = 0; z < 4; z++) acc[z] = fma(sm[z], f, acc[z]);
        }
      }
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&sempty[s]);  // this warp is done with the stage
    }
  }
  __syncthreads();  // every consumer is past its reads of q and of the stages
  const bool stop = sstop;
  // a wait ran out: the copies still in flight land before the CTA exits
  if (stop && t == 0)
    for (int h = issued - 1; h >= 0 && h >= issued - nst; h--) mbar_wait(&sfull[h % nst], (unsigned)(h / nst) & 1u, a.err);
  if (split > 1) {
    // rank 0 adds the other ranks' partial sums in rank order; every CTA of
    // the cluster passes both cluster barriers on every path (a rank's
    // shared memory lives until rank 0 has read it)
    if (rank > 0 && cons) st4(part + 4 * c, acc);
    tm_cluster_sync();
    if (rank == 0 && cons)
      for (int q = 1; q < split; q++) {
        T o4[4];
        ld4_peer(o4, part + 4 * c, (unsigned)q);
#pragma unroll
        for (int z = 0; z < 4; z++) acc[z] += o4[z];
      }
    tm_cluster_sync();
    if (rank > 0) return;
  }
  if (stop) return;
  if (cons) {
    st4(a.Q + tm_cell(n, i, len) + r * TM_D + 4 * qs, acc);
    st4(q + r * TM_D + 4 * qs, acc);
  }
  // the largest |mantissa| of this length (idle lanes hold zeros)
  if (w > 0) {
    T m = fmax(fmax(fabs(acc[0]), fabs(acc[1])), fmax(fabs(acc[2]), fabs(acc[3])));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) smx[w - 1] = m;
  }
  if (cons && c < BLK) tq[c] = i + len < n ? (T)a.Tr[(size_t)(i + len - 1) * BLK + c] : (T)0;
  __syncthreads();
  if (t == 0) {
    double mm = 0;
    for (int v = 0; v < TM_NCW; v++) mm = fmax(mm, (double)smx[v]);
    atomic_max_pos(a.dmax + len, mm);
  }
  if (cons && i + len < n) {  // L[i, i+len] = Q[i, i+len] (T_{i+len-1} (x) I): column state qs at i + len
    const int Mj = a.Mp[j];
    T l4[4] = {0, 0, 0, 0};
    for (int b = 0; b < Mj; b++) {
      const T tb = tq[b * NS + qs];
      T q4[4];
      ld4(q4, q + r * TM_D + 4 * b);
#pragma unroll
      for (int z = 0; z < 4; z++) l4[z] = fma(q4[z], tb, l4[z]);
    }
    st4(a.L + tm_cell(n, i, len) + r * TM_D + 4 * qs, l4);
  }
}

// Z relative to 2^{E[n]}: sum_{a,c} u0[a] Tr_S[Q[0, n]_{a c}], then log Z
template <typename T>
__global__ void k_tm_finish(TmArgs<T> a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = a.n;
  const T *q = a.Q + tm_cell(n, 0, n);
  double z = 0;
  for (int ar = 0; ar < a.Mp[0]; ar++)
    for (int ac = 0; ac < a.Mp[n - 1]; ac++) {
      double s = 0;
      for (int e1 = 0; e1 < TM_G; e1++)
        for (int e2 = 0; e2 < TM_G; e2++) s += a.mod->S[e2][e1] * (double)q[(ar * TM_G + e1) * TM_D + ac * TM_G + e2];
      z += a.u0[ar] * s;
    }
  *a.Zm = z;
  double sc = 0;
  for (int k = 0; k < a.nls; k++) sc += a.ls[k];
  *a.logz = log(z) + (double)a.E[n] * 0.69314718055994530942 - sc;
  if (!(z > 0) || !isfinite(*a.logz)) atomicOr(a.err, 2);
}

}  // namespace cf
