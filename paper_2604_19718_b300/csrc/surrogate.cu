// surrogate.cu -- learned window free-energy surrogate, trained and run by
// this library's own kernels.
//
// The exact DP labels windows of designed sequences with their ensemble free
// energy G = -RT ln Z; this network predicts G from the bases alone, so that
// many candidate codon choices can be screened before the exact DP re-scores
// the best few.  (The paper has no learned component: it scores every
// candidate exactly.)
//
// Network, per window of n <= 256 bases:
//   h0 = one-hot bases (4 channels);  h_l = relu(b_l + W_l * h_{l-1}),
//   l = 1..4, 64 channels, 5 taps, zero padding;  g = mean_t(wh . h4) + bh,
//   predicted G = n g.  Training loss (1/B) sum_w (g_w - G_w/n_w)^2, Adam.
// Conv weights are held as FP32 masters and used as BF16 (rounded once per
// update); all products accumulate in FP32.
//
// Layout: activations [window][64][256] FP32, positions >= n zero.  Forward
// and input-gradient convolutions run one CTA per window with the input tile
// and the BF16 weights in shared memory; each warp owns 8 output channels and
// each lane 8 positions 32 apart (conflict-free tile reads, one 16-byte weight
// read per tap).  Weight gradients run persistent CTAs that accumulate in
// registers over their windows and write per-CTA partials, summed in a fixed
// order (deterministic gradients).
#include "cf_nvtx.h"
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/codonfold.h"

namespace cf {
void set_last_error(const std::string &msg);
}

namespace sg {

constexpr int C = 64, K = 5, LP = 256;
constexpr int LPH = LP + 4;      // halo row of the forward tile
constexpr int LPW = LP + 5;      // odd row stride of the weight-gradient tiles
constexpr int LPD = LP + 1;
constexpr int NT = 256;
constexpr int NPARAM = 63041;
// flat parameter offsets: W1 b1 W2 b2 W3 b3 W4 b4 wh bh
__host__ __device__ constexpr int OW(int l) { return l == 0 ? 0 : 1344 + (l - 1) * 20544; }
__host__ __device__ constexpr int CIN(int l) { return l == 0 ? 4 : 64; }
__host__ __device__ constexpr int OB(int l) { return OW(l) + C * CIN(l) * K; }
constexpr int OWH = 62976, OBH = 63040;
// BF16 weight buffers: forward [ci][k][co] per layer, input-gradient [o][k'][c] for layers 2..4
__host__ __device__ constexpr int WF_OFF(int l) { return l == 0 ? 0 : 1280 + (l - 1) * 20480; }
constexpr int WF_N = 62720;
__host__ __device__ constexpr int WB_OFF(int l) { return (l - 1) * 20480; }  // layers 1..3
constexpr int WB_N = 61440;
static_assert(OB(3) == 62912 && OB(0) == 1280 && OW(3) + C * 64 * K + C == OWH, "parameter layout");

__global__ void k_prep(const float *P, __nv_bfloat16 *Wf, __nv_bfloat16 *Wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= WF_N) return;
  int l = 3;
  while (i < WF_OFF(l)) l--;
  const int r = i - WF_OFF(l), cin = CIN(l);
  // forward layout r = (ci*K + k)*C + co
  const int co = r % C, k = (r / C) % K, ci = r / (C * K);
  Wf[i] = __float2bfloat16_rn(P[OW(l) + (co * cin + ci) * K + k]);
  if (l >= 1) {
    // input-gradient layout r = (o*K + kp)*C + c holds W[o][c][K-1-kp]
    const int c = r % C, kp = (r / C) % K, o = r / (C * K);
    Wb[WB_OFF(l) + r] = __float2bfloat16_rn(P[OW(l) + (o * C + c) * K + (K - 1 - kp)]);
  }
}

__device__ __forceinline__ void bf8(const __nv_bfloat16 *p, float (&w)[8]) {
  const uint4 v = *reinterpret_cast<const uint4 *>(p);
  const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    w[2 * q] = __uint_as_float(u[q] << 16);
    w[2 * q + 1] = __uint_as_float(u[q] & 0xffff0000u);
  }
}

// MODE 0: out = relu(bias + W * in) on [0, n), zero beyond.
// MODE 1: out = (W^T-flipped * in) * (gate > 0): the gradient with respect to
//         the pre-activation of the previous layer, gate = that layer's output.
// Layer input: `in` ([window][CI][LP]) or, when CI == 4, the window's bases.
template <int CI, int MODE>
__global__ void __launch_bounds__(NT) k_conv(const uint8_t *bases, const int64_t *off, const float *in,
                                             const __nv_bfloat16 *W, const float *bias, const float *gate,
                                             float *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(smem);
  float *sIn = reinterpret_cast<float *>(smem + CI * K * C * sizeof(__nv_bfloat16));
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = (int)(off[b + 1] - off[b]);
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(W);
    uint4 *dst = reinterpret_cast<uint4 *>(sW);
    for (int i = tid; i < CI * K * C / 8; i += NT) dst[i] = src[i];
  }
  for (int i = tid; i < CI * LPH; i += NT) {
    const int c = i / LPH, h = i % LPH, t = h - 2;
    float v = 0.f;
    if (t >= 0 && t < n) {
      if (CI == 4) v = (bases[off[b] + t] == c) ? 1.f : 0.f;
      else v = in[((size_t)b * CI + c) * LP + t];
    }
    sIn[i] = v;
  }
  __syncthreads();
  float acc[8][8];
#pragma unroll
  for (int o = 0; o < 8; o++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[o][j] = 0.f;
  const int co0 = w * 8;
  for (int ci = 0; ci < CI; ci++) {
    const float *row = sIn + ci * LPH + lane;
#pragma unroll
    for (int k = 0; k < K; k++) {
      float wv[8];
      bf8(sW + (ci * K + k) * C + co0, wv);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const float x = row[32 * j + k];
#pragma unroll
        for (int o = 0; o < 8; o++) acc[o][j] = fmaf(wv[o], x, acc[o][j]);
      }
    }
  }
#pragma unroll
  for (int o = 0; o < 8; o++) {
    const int co = co0 + o;
    const float bo = MODE == 0 ? bias[co] : 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int t = lane + 32 * j;
      const size_t idx = ((size_t)b * C + co) * LP + t;
      float v = 0.f;
      if (t < n) {
        if (MODE == 0) v = fmaxf(acc[o][j] + bo, 0.f);
        else v = gate[idx] > 0.f ? acc[o][j] : 0.f;
      }
      out[idx] = v;
    }
  }
}

// Head: S[w][c] = sum_t h4[c][t], pred G = sum_c wh[c] S[c] + n bh.  With
// targets: dg[w] = 2 (g - G/n) / B and loss += (g - G/n)^2 / B.
__global__ void __launch_bounds__(NT) k_head(const int64_t *off, const float *h4, const float *P, float *S,
                                             float *pred, const float *target, float *dg, float *loss, int B) {
  __shared__ float red[NT / 32];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = (int)(off[b + 1] - off[b]);
  float part = 0.f;
  for (int c = w; c < C; c += NT / 32) {
    const float *row = h4 + ((size_t)b * C + c) * LP;
    float s = 0.f;
    for (int t = lane; t < LP; t += 32) s += row[t];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) S[(size_t)b * C + c] = s;
    part += s * P[OWH + c];
  }
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int k = 0; k < NT / 32; k++) s += red[k];
    const float g = (n > 0 ? s / (float)n : 0.f) + P[OBH];
    pred[b] = (float)n * g;
    if (target) {
      const float r = n > 0 ? g - target[b] / (float)n : 0.f;
      dg[b] = 2.f * r / (float)B;
      atomicAdd(loss, r * r / (float)B);
    }
  }
}

// Gradient at the last layer's pre-activation: dg wh[c] / n where h4 > 0.
__global__ void __launch_bounds__(NT) k_dpre4(const int64_t *off, const float *h4, const float *P, const float *dg,
                                              float *dpre) {
  const int b = blockIdx.x;
  const int n = (int)(off[b + 1] - off[b]);
  const float s = n > 0 ? dg[b] / (float)n : 0.f;
  for (int i = threadIdx.x; i < C * LP; i += NT) {
    const size_t idx = (size_t)b * C * LP + i;
    dpre[idx] = h4[idx] > 0.f ? s * P[OWH + i / LP] : 0.f;
  }
}

// Weight and bias gradients of one layer: dW[o][c][k] = sum_w sum_t
// dpre[o][t] h[c][t+k-2], db[o] = sum dpre[o][t].  Persistent CTAs; each
// writes its partial sums to part[blockIdx.x][...].
template <int CI>
__global__ void __launch_bounds__(NT) k_dw(const uint8_t *bases, const int64_t *off, const float *hin,
                                           const float *dpre, int nwin, float *part) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *sD = reinterpret_cast<float *>(smem);   // [C][LPD]
  float *sH = sD + C * LPD;                      // [CI][LPW], halo 2
  constexpr int OB_ = CI == 64 ? 4 : 1;          // output channels per thread
  constexpr int CB_ = CI == 64 ? 4 : 1;          // input channels per thread
  const int tid = threadIdx.x;
  const int o0 = CI == 64 ? (tid / 16) * 4 : tid / 4;
  const int c0 = CI == 64 ? (tid % 16) * 4 : tid % 4;
  float acc[OB_][CB_][K], accb[OB_];
#pragma unroll
  for (int a = 0; a < OB_; a++) {
    accb[a] = 0.f;
#pragma unroll
    for (int c = 0; c < CB_; c++)
#pragma unroll
      for (int k = 0; k < K; k++) acc[a][c][k] = 0.f;
  }
  for (int b = blockIdx.x; b < nwin; b += gridDim.x) {
    const int n = (int)(off[b + 1] - off[b]);
    __syncthreads();
    for (int i = tid; i < C * LP; i += NT) {
      const int o = i / LP, t = i % LP;
      sD[o * LPD + t] = dpre[(size_t)b * C * LP + i];
    }
    for (int i = tid; i < CI * LPW; i += NT) {
      const int c = i / LPW, h = i % LPW, t = h - 2;
      float v = 0.f;
      if (t >= 0 && t < n) {
        if (CI == 4) v = (bases[off[b] + t] == c) ? 1.f : 0.f;
        else v = hin[((size_t)b * CI + c) * LP + t];
      }
      sH[i] = v;
    }
    __syncthreads();
    float hw[CB_][K];
#pragma unroll
    for (int c = 0; c < CB_; c++)
#pragma unroll
      for (int k = 0; k < K - 1; k++) hw[c][k + 1] = sH[(c0 + c) * LPW + k];
    for (int t = 0; t < n; t++) {
#pragma unroll
      for (int c = 0; c < CB_; c++) {
#pragma unroll
        for (int k = 0; k < K - 1; k++) hw[c][k] = hw[c][k + 1];
        hw[c][K - 1] = sH[(c0 + c) * LPW + t + K - 1];
      }
#pragma unroll
      for (int a = 0; a < OB_; a++) {
        const float dv = sD[(o0 + a) * LPD + t];
        accb[a] += dv;
#pragma unroll
        for (int c = 0; c < CB_; c++)
#pragma unroll
          for (int k = 0; k < K; k++) acc[a][c][k] = fmaf(dv, hw[c][k], acc[a][c][k]);
      }
    }
  }
  // partial layout: dW [C][CI][K] then db [C]
  float *dst = part + (size_t)blockIdx.x * (C * CI * K + C);
#pragma unroll
  for (int a = 0; a < OB_; a++) {
#pragma unroll
    for (int c = 0; c < CB_; c++)
#pragma unroll
      for (int k = 0; k < K; k++) dst[((o0 + a) * CI + c0 + c) * K + k] = acc[a][c][k];
    if (c0 == 0) dst[C * CI * K + o0 + a] = accb[a];
  }
}

// grad[dst + i] = sum_g part[g][i], fixed order.
__global__ void k_reduce(const float *part, int nparts, int len, float *grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.f;
  for (int g = 0; g < nparts; g++) s += part[(size_t)g * len + i];
  grad[i] = s;
}

// Head gradients: dwh[c] = sum_w dg[w] S[w][c] / n_w, dbh = sum_w dg[w].
__global__ void k_head_grad(const int64_t *off, const float *S, const float *dg, int nwin, float *grad) {
  const int c = threadIdx.x;
  float s = 0.f;
  for (int b = 0; b < nwin; b++) {
    const int n = (int)(off[b + 1] - off[b]);
    if (n == 0) continue;
    s += c < C ? dg[b] * S[(size_t)b * C + c] / (float)n : dg[b];
  }
  if (c < C) grad[OWH + c] = s;
  else if (c == C) grad[OBH] = s;
}

__global__ void k_adam(float *P, const float *G, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float g = G[i];
  const float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace sg

#include "surrogate_tc.cuh"

// ------------------------------------------------------------------ host

struct cf_surrogate {
  int device = 0;
  cudaStream_t stream = nullptr;
  int max_batch = 0, dw_grid = 0;
  long step = 0;
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  __nv_bfloat16 *Wf = nullptr, *Wb = nullptr;
  float *h[4] = {}, *dp[2] = {}, *S = nullptr, *pred = nullptr, *dg = nullptr, *loss = nullptr, *tgt = nullptr;
  float *part = nullptr;
  // tensor-core prediction path (surrogate_tc.cuh): weights of layers 2-4 and
  // the error word; the row frame (base per row), per-row head terms,
  // predictions and offsets of a chunk, grown on demand (the path keeps no
  // per-window activations, so its chunks are not bounded by max_batch)
  __nv_bfloat16 *Wtc = nullptr;
  int *tcerr = nullptr;
  int8_t *rowbase = nullptr;
  float *srow = nullptr, *tpred = nullptr;
  int64_t *toff = nullptr;
  size_t rows_cap = 0, twin_cap = 0;
  std::vector<void *> tc_allocs;
  int path = 1;  // prediction: 0 CUDA cores (FP32 activations), 1 tensor cores
  int sms = 148;
  uint8_t *bases = nullptr;
  size_t bases_cap = 0;
  int64_t *off = nullptr;
  std::vector<void *> allocs, base_allocs;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  float last_ms = 0;
};

namespace {

using namespace sg;

cf_status sfail(cf_status s, const std::string &m) {
  cf::set_last_error(m);
  return s;
}

#define SG_CUDA(call)                                                                             \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return sfail(e_ == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA,                        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

template <typename V>
cudaError_t salloc(std::vector<void *> &list, V **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max(count, (size_t)1) * sizeof(V));
  if (e != cudaSuccess) return e;
  list.push_back(q);
  *p = (V *)q;
  return cudaSuccess;
}

bool on_device(const void *ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device memory of a device other than `device` (the kernels read the
// window inputs in place, so such buffers are rejected)
bool on_other_device(const void *ptr, int device) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device != device;
}

size_t conv_smem(int ci) { return (size_t)ci * K * C * 2 + (size_t)ci * LPH * 4; }
size_t dw_smem(int ci) { return ((size_t)C * LPD + (size_t)ci * LPW) * 4; }

cf_status refresh_bf16(cf_surrogate *s) {
  k_prep<<<(WF_N + 255) / 256, 256, 0, s->stream>>>(s->P, s->Wf, s->Wb);
  k_prep_tc<<<(3 * 5 * 64 * 64 + 255) / 256, 256, 0, s->stream>>>(s->P, s->Wtc);
  SG_CUDA(cudaGetLastError());
  return CF_OK;
}

// cuTensorMapEncodeTiled from the driver (looked up once through the runtime)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D BF16 row tensor [rows][64] (128-byte rows), box 64 x box_rows, 128-byte swizzle
bool row_map(CUtensorMap *m, const void *base, size_t rows, unsigned box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {64, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Windows per chunk of the tensor-core path.
constexpr int TC_CHUNK = 1 << 16;

// The tensor-core path's chunk buffers for up to nwin windows (grown, never shrunk).
cf_status tc_reserve(cf_surrogate *s, int nwin) {
  if ((size_t)nwin <= s->twin_cap) return CF_OK;
  SG_CUDA(cudaStreamSynchronize(s->stream));
  for (void *q : s->tc_allocs) cudaFree(q);
  s->tc_allocs.clear();
  s->twin_cap = s->rows_cap = 0;
  const size_t rows = (size_t)nwin * (CF_SURROGATE_MAX_LEN + 4);
  SG_CUDA(salloc(s->tc_allocs, &s->rowbase, rows));
  SG_CUDA(salloc(s->tc_allocs, &s->srow, rows));
  SG_CUDA(salloc(s->tc_allocs, &s->tpred, (size_t)nwin));
  SG_CUDA(salloc(s->tc_allocs, &s->toff, (size_t)nwin + 1));
  s->rows_cap = rows;
  s->twin_cap = (size_t)nwin;
  return CF_OK;
}

// The forward pass on the tensor cores for a staged batch of nb windows.
cf_status forward_tc(cf_surrogate *s, const uint8_t *db, const int64_t *doff, int nb, const std::vector<int64_t> &hoff) {
  cudaStream_t st = s->stream;
  const int nrows = (int)(hoff[nb] - hoff[0]) + 4 * nb;
  if ((size_t)nrows > s->rows_cap) return sfail(CF_EINVAL, "surrogate: batch exceeds the row buffers");
  k_tc_rows<<<nb, 128, 0, st>>>(doff, db, nb, nrows, s->rowbase);
  SG_CUDA(cudaGetLastError());
  CUtensorMap tw;
  if (!row_map(&tw, s->Wtc, 3 * 5 * 64, 64)) return sfail(CF_ECUDA, "surrogate: weight tensor map");
  const int ntiles = (nrows + TC_OUT - 1) / TC_OUT;
  const int grid = std::max(1, std::min(ntiles, s->sms));
  TcArgs a;
  a.nrows = nrows;
  a.rowbase = s->rowbase;
  a.W1 = s->Wf + WF_OFF(0);
  a.P = s->P;
  a.s_out = s->srow;
  a.err = s->tcerr;
  k_surr_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(tw, a);
  SG_CUDA(cudaGetLastError());
  k_tc_head<<<(nb + 3) / 4, 128, 0, st>>>(doff, nb, s->srow, s->P, s->tpred);
  SG_CUDA(cudaGetLastError());
  return CF_OK;
}

// Stage a batch: copy host inputs to the device, validate window lengths.
cf_status stage(cf_surrogate *s, const uint8_t *bases, const int64_t *offsets, int nwin, const uint8_t **db,
                const int64_t **doff, std::vector<int64_t> &hoff, bool tc = false) {
  hoff.assign((size_t)nwin + 1, 0);
  cudaStream_t st = s->stream;
  if (on_other_device(offsets, s->device) || on_other_device(bases, s->device))
    return sfail(CF_EINVAL, "surrogate: window inputs are device memory of another device");
  const bool odev = on_device(offsets), bdev = on_device(bases);
  if (odev) {
    SG_CUDA(cudaMemcpyAsync(hoff.data(), offsets, sizeof(int64_t) * (nwin + 1), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
  } else {
    std::copy(offsets, offsets + nwin + 1, hoff.begin());
  }
  if (hoff[0] < 0) return sfail(CF_EINVAL, "surrogate: offsets[0] < 0");
  for (int w = 0; w < nwin; w++) {
    const int64_t len = hoff[w + 1] - hoff[w];
    if (len < 0 || len > CF_SURROGATE_MAX_LEN)
      return sfail(CF_EINVAL, "surrogate: window length outside 0..CF_SURROGATE_MAX_LEN");
  }
  if (bdev) {
    *db = bases;
  } else {
    const size_t total = (size_t)hoff[nwin];
    if (s->bases_cap < total) {
      SG_CUDA(cudaStreamSynchronize(st));
      for (void *q : s->base_allocs) cudaFree(q);
      s->base_allocs.clear();
      s->bases_cap = std::max(total, (size_t)1 << 20);
      SG_CUDA(salloc(s->base_allocs, &s->bases, s->bases_cap));
    }
    SG_CUDA(cudaMemcpyAsync(s->bases, bases, total, cudaMemcpyHostToDevice, st));
    *db = s->bases;
  }
  if (odev) {
    *doff = offsets;
  } else {
    int64_t *dst = tc ? s->toff : s->off;  // the tensor-core path's chunks exceed max_batch
    SG_CUDA(cudaMemcpyAsync(dst, hoff.data(), sizeof(int64_t) * (nwin + 1), cudaMemcpyHostToDevice, st));
    *doff = dst;
  }
  return CF_OK;
}

cf_status forward(cf_surrogate *s, const uint8_t *db, const int64_t *doff, int nb, const float *tgt) {
  cudaStream_t st = s->stream;
  k_conv<4, 0><<<nb, NT, conv_smem(4), st>>>(db, doff, nullptr, s->Wf + WF_OFF(0), s->P + OB(0), nullptr, s->h[0]);
  for (int l = 1; l < 4; l++)
    k_conv<64, 0><<<nb, NT, conv_smem(64), st>>>(db, doff, s->h[l - 1], s->Wf + WF_OFF(l), s->P + OB(l), nullptr,
                                                 s->h[l]);
  k_head<<<nb, NT, 0, st>>>(doff, s->h[3], s->P, s->S, s->pred, tgt, s->dg, s->loss, nb);
  SG_CUDA(cudaGetLastError());
  return CF_OK;
}

cf_status backward(cf_surrogate *s, const uint8_t *db, const int64_t *doff, int nb) {
  cudaStream_t st = s->stream;
  k_dpre4<<<nb, NT, 0, st>>>(doff, s->h[3], s->P, s->dg, s->dp[0]);
  int cur = 0;
  for (int l = 3; l >= 0; l--) {
    const int ci = CIN(l), len = C * ci * K + C;
    if (l > 0)
      k_dw<64><<<s->dw_grid, NT, dw_smem(64), st>>>(db, doff, s->h[l - 1], s->dp[cur], nb, s->part);
    else
      k_dw<4><<<s->dw_grid, NT, dw_smem(4), st>>>(db, doff, nullptr, s->dp[cur], nb, s->part);
    k_reduce<<<(len + 255) / 256, 256, 0, st>>>(s->part, s->dw_grid, len, s->G + OW(l));
    if (l > 0) {
      k_conv<64, 1><<<nb, NT, conv_smem(64), st>>>(db, doff, s->dp[cur], s->Wb + WB_OFF(l), nullptr, s->h[l - 1],
                                                   s->dp[cur ^ 1]);
      cur ^= 1;
    }
  }
  k_head_grad<<<1, 96, 0, st>>>(doff, s->S, s->dg, nb, s->G);
  SG_CUDA(cudaGetLastError());
  return CF_OK;
}

cf_status copy_out(cf_surrogate *s, void *dst, const void *src, size_t bytes) {
  SG_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s->stream));
  return CF_OK;
}

#define SG_TRY(x)                 \
  do {                            \
    cf_status r_ = (x);           \
    if (r_ != CF_OK) return r_;   \
  } while (0)

}  // namespace

extern "C" {

cf_status cf_surrogate_create(int device, void *stream, int max_batch, cf_surrogate **out) {
  if (!out || max_batch < 1) return sfail(CF_EINVAL, "cf_surrogate_create: bad argument");
  *out = nullptr;
  SG_CUDA(cudaSetDevice(device));
  cf_surrogate *s = new (std::nothrow) cf_surrogate;
  if (!s) return sfail(CF_ENOMEM, "cf_surrogate_create: host memory");
  s->device = device;
  s->stream = (cudaStream_t)stream;
  s->max_batch = max_batch;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  s->dw_grid = std::min(sms, max_batch);
  auto &L = s->allocs;
  const size_t act = (size_t)max_batch * C * LP;
  cudaError_t e = cudaSuccess;
  float **bufs4[] = {&s->P, &s->G, &s->M, &s->V};
  for (float **q : bufs4)
    if (e == cudaSuccess) e = salloc(L, q, (size_t)NPARAM);
  if (e == cudaSuccess) e = salloc(L, &s->Wf, (size_t)WF_N);
  if (e == cudaSuccess) e = salloc(L, &s->Wb, (size_t)WB_N);
  for (int l = 0; l < 4 && e == cudaSuccess; l++) e = salloc(L, &s->h[l], act);
  for (int l = 0; l < 2 && e == cudaSuccess; l++) e = salloc(L, &s->dp[l], act);
  if (e == cudaSuccess) e = salloc(L, &s->S, (size_t)max_batch * C);
  if (e == cudaSuccess) e = salloc(L, &s->pred, (size_t)max_batch);
  if (e == cudaSuccess) e = salloc(L, &s->dg, (size_t)max_batch);
  if (e == cudaSuccess) e = salloc(L, &s->tgt, (size_t)max_batch);
  if (e == cudaSuccess) e = salloc(L, &s->loss, (size_t)1);
  if (e == cudaSuccess) e = salloc(L, &s->part, (size_t)s->dw_grid * (C * 64 * K + C));
  if (e == cudaSuccess) e = salloc(L, &s->off, (size_t)max_batch + 1);
  s->sms = sms;
  if (e == cudaSuccess) e = salloc(L, &s->Wtc, (size_t)3 * 5 * 64 * 64);
  if (e == cudaSuccess) e = salloc(L, &s->tcerr, (size_t)1);
  if (e == cudaSuccess) e = cudaMemset(s->tcerr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->P, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMemset(s->M, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMemset(s->V, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev[1]);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_conv<64, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem(64));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_conv<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem(64));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_dw<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw_smem(64));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_dw<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw_smem(4));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_surr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e != cudaSuccess) {
    cf_surrogate_free(s);
    return sfail(e == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA,
                 std::string("cf_surrogate_create: ") + cudaGetErrorString(e));
  }
  *out = s;
  return CF_OK;
}

cf_status cf_surrogate_free(cf_surrogate *s) {
  if (!s) return CF_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  for (void *q : s->allocs) cudaFree(q);
  for (void *q : s->base_allocs) cudaFree(q);
  for (void *q : s->tc_allocs) cudaFree(q);
  for (auto &e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
  return CF_OK;
}

cf_status cf_surrogate_set_params(cf_surrogate *s, const float *params) {
  if (!s || !params) return sfail(CF_EINVAL, "cf_surrogate_set_params: NULL argument");
  SG_CUDA(cudaSetDevice(s->device));
  SG_CUDA(cudaMemcpyAsync(s->P, params, sizeof(float) * NPARAM,
                          on_device(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  SG_CUDA(cudaMemsetAsync(s->M, 0, sizeof(float) * NPARAM, s->stream));
  SG_CUDA(cudaMemsetAsync(s->V, 0, sizeof(float) * NPARAM, s->stream));
  s->step = 0;
  SG_TRY(refresh_bf16(s));
  SG_CUDA(cudaStreamSynchronize(s->stream));
  return CF_OK;
}

cf_status cf_surrogate_get_params(const cf_surrogate *s, float *params) {
  if (!s || !params) return sfail(CF_EINVAL, "cf_surrogate_get_params: NULL argument");
  SG_CUDA(cudaSetDevice(s->device));
  SG_CUDA(cudaMemcpyAsync(params, s->P, sizeof(float) * NPARAM,
                          on_device(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  SG_CUDA(cudaStreamSynchronize(s->stream));
  return CF_OK;
}

cf_status cf_surrogate_predict(cf_surrogate *s, const uint8_t *bases, const int64_t *offsets, int nwin,
                               float *G_out) {
  cf::CfRange nvtx_range("cf_surrogate_predict");
  if (!s || nwin < 0) return sfail(CF_EINVAL, "cf_surrogate_predict: bad argument");
  if (nwin == 0) return CF_OK;
  if (!bases || !offsets || !G_out) return sfail(CF_EINVAL, "cf_surrogate_predict: NULL argument");
  SG_CUDA(cudaSetDevice(s->device));
  const bool odev = on_device(offsets), bdev = on_device(bases);
  std::vector<int64_t> all((size_t)nwin + 1);
  if (odev) {
    SG_CUDA(cudaMemcpyAsync(all.data(), offsets, sizeof(int64_t) * (nwin + 1), cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(cudaStreamSynchronize(s->stream));
  } else {
    std::copy(offsets, offsets + nwin + 1, all.begin());
  }
  const int chunk = s->path ? std::max(s->max_batch, TC_CHUNK) : s->max_batch;
  if (s->path) SG_TRY(tc_reserve(s, std::min(chunk, nwin)));
  SG_CUDA(cudaEventRecord(s->ev[0], s->stream));
  float total_ms = 0;
  for (int w0 = 0; w0 < nwin; w0 += chunk) {
    const int nb = std::min(chunk, nwin - w0);
    // re-base this chunk's offsets so that its bases start at the chunk's first window
    std::vector<int64_t> o(all.begin() + w0, all.begin() + w0 + nb + 1);
    // device bases keep absolute offsets; host bases are staged from the chunk's first window
    const uint8_t *src = bdev ? bases : bases + o[0];
    if (!bdev) {
      const int64_t o0 = o[0];
      for (auto &v : o) v -= o0;
    }
    const uint8_t *db;
    const int64_t *doff;
    std::vector<int64_t> hoff;
    SG_TRY(stage(s, src, o.data(), nb, &db, &doff, hoff, s->path != 0));
    if (s->path) SG_TRY(forward_tc(s, db, doff, nb, hoff));
    else SG_TRY(forward(s, db, doff, nb, nullptr));
    SG_TRY(copy_out(s, G_out + w0, s->path ? s->tpred : s->pred, sizeof(float) * nb));
    SG_CUDA(cudaStreamSynchronize(s->stream));  // host offsets / staging buffers reused by the next chunk
  }
  SG_CUDA(cudaEventRecord(s->ev[1], s->stream));
  SG_CUDA(cudaEventSynchronize(s->ev[1]));
  SG_CUDA(cudaEventElapsedTime(&total_ms, s->ev[0], s->ev[1]));
  s->last_ms = total_ms;
  if (s->path) {
    int err = 0;
    SG_CUDA(cudaMemcpy(&err, s->tcerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      SG_CUDA(cudaMemset(s->tcerr, 0, sizeof(int)));
      return sfail(CF_ETIMEOUT, "cf_surrogate_predict: a bounded wait of the tensor-core pipeline gave up");
    }
  }
  return CF_OK;
}

cf_status cf_surrogate_set_path(cf_surrogate *s, int path) {
  if (!s || path < 0 || path > 1) return sfail(CF_EINVAL, "cf_surrogate_set_path: bad argument");
  s->path = path;
  return CF_OK;
}

static cf_status grad_common(cf_surrogate *s, const uint8_t *bases, const int64_t *offsets, int nwin,
                             const float *G_target) {
  if (nwin < 1 || nwin > s->max_batch) return sfail(CF_EINVAL, "surrogate: batch must hold 1..max_batch windows");
  if (!bases || !offsets || !G_target) return sfail(CF_EINVAL, "surrogate: NULL argument");
  SG_CUDA(cudaSetDevice(s->device));
  const uint8_t *db;
  const int64_t *doff;
  std::vector<int64_t> hoff;
  SG_TRY(stage(s, bases, offsets, nwin, &db, &doff, hoff));
  SG_CUDA(cudaMemcpyAsync(s->tgt, G_target, sizeof(float) * nwin,
                          on_device(G_target) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  SG_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(float), s->stream));
  SG_TRY(forward(s, db, doff, nwin, s->tgt));
  SG_TRY(backward(s, db, doff, nwin));
  return CF_OK;
}

cf_status cf_surrogate_grad(cf_surrogate *s, const uint8_t *bases, const int64_t *offsets, int nwin,
                            const float *G_target, float *loss_out, float *grad_out) {
  cf::CfRange nvtx_range("cf_surrogate_grad");
  if (!s) return sfail(CF_EINVAL, "cf_surrogate_grad: NULL surrogate");
  SG_TRY(grad_common(s, bases, offsets, nwin, G_target));
  if (loss_out) SG_TRY(copy_out(s, loss_out, s->loss, sizeof(float)));
  if (grad_out) SG_TRY(copy_out(s, grad_out, s->G, sizeof(float) * NPARAM));
  SG_CUDA(cudaStreamSynchronize(s->stream));
  return CF_OK;
}

cf_status cf_surrogate_train_step(cf_surrogate *s, const uint8_t *bases, const int64_t *offsets, int nwin,
                                  const float *G_target, float lr, float *loss_out) {
  cf::CfRange nvtx_range("cf_surrogate_train_step");
  if (!s) return sfail(CF_EINVAL, "cf_surrogate_train_step: NULL surrogate");
  if (!(lr > 0.f) || !std::isfinite(lr)) return sfail(CF_EINVAL, "cf_surrogate_train_step: lr must be > 0");
  SG_CUDA(cudaSetDevice(s->device));
  SG_CUDA(cudaEventRecord(s->ev[0], s->stream));
  SG_TRY(grad_common(s, bases, offsets, nwin, G_target));
  s->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s->stream>>>(s->P, s->G, s->M, s->V, lr, b1, b2, 1e-8f, c1, c2);
  SG_CUDA(cudaGetLastError());
  SG_TRY(refresh_bf16(s));
  SG_CUDA(cudaEventRecord(s->ev[1], s->stream));
  if (loss_out) SG_TRY(copy_out(s, loss_out, s->loss, sizeof(float)));
  SG_CUDA(cudaStreamSynchronize(s->stream));
  SG_CUDA(cudaEventElapsedTime(&s->last_ms, s->ev[0], s->ev[1]));
  return CF_OK;
}

float cf_surrogate_last_ms(const cf_surrogate *s) { return s ? s->last_ms : 0.f; }

}  // extern "C"
