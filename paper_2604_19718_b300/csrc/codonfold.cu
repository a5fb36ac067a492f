// codonfold.cu -- C ABI (include/codonfold.h) and host orchestration of the
// codon-constrained partition-function kernels for sm_103a.
//
// Host work is limited to validating inputs, listing the codon states of each
// position (amino acid -> codons, bases, sense ids), the model's loop-length
// factor tables, choosing launch shapes and moving inputs and outputs.  Every
// step of the computation runs in kernels: the position transfers (Eq.
// pair-tt with soft weights) and log Z in cf_inside.cuh, the inside wavefront
// in cf_inside2.cuh, the outside pass and the marginals in cf_outside2.cuh and
// cf_outside.cuh, the sampler in cf_sample.cuh and the fixed-sequence windows
// in cf_window.cuh, the minimum free energy pass and its traceback in
// cf_mfe.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/codonfold.h"
#include "cf_common.cuh"
#include "cf_inside.cuh"
#include "cf_inside2.cuh"
#include "cf_mfe.cuh"
#include "cf_outside.cuh"
#include "cf_outside2.cuh"
#include "cf_sample.cuh"
#include "cf_window.cuh"
#include "cf_tm.cuh"
#include "cf_subopt.cuh"

using namespace cf;

namespace {

const char kAminoAcids[] = "ARNDCQEGHILKMFPSTWYV";
// Codons of each amino acid (standard genetic code), written per amino acid.
const char *kCodonsOf[20] = {
    "GCU GCC GCA GCG",          // A
    "CGU CGC CGA CGG AGA AGG",  // R
    "AAU AAC",                  // N
    "GAU GAC",                  // D
    "UGU UGC",                  // C
    "CAA CAG",                  // Q
    "GAA GAG",                  // E
    "GGU GGC GGA GGG",          // G
    "CAU CAC",                  // H
    "AUU AUC AUA",              // I
    "UUA UUG CUU CUC CUA CUG",  // L
    "AAA AAG",                  // K
    "AUG",                      // M
    "UUU UUC",                  // F
    "CCU CCC CCA CCG",          // P
    "UCU UCC UCA UCG AGU AGC",  // S
    "ACU ACC ACA ACG",          // T
    "UGG",                      // W
    "UAU UAC",                  // Y
    "GUU GUC GUA GUG",          // V
};

int base_index(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'U': return 3;
  }
  return -1;
}

struct GeneticCode {
  std::vector<int> codons[20];  // 6-bit codon numbers (A,C,G,U = 0..3), ascending
  int sense_id[64];
  GeneticCode() {
    std::vector<int> all;
    for (int a = 0; a < 20; a++) {
      const char *s = kCodonsOf[a];
      const size_t len = std::strlen(s);
      for (size_t k = 0; k + 2 < len; k += 4) {
        int c = 16 * base_index(s[k]) + 4 * base_index(s[k + 1]) + base_index(s[k + 2]);
        codons[a].push_back(c);
        all.push_back(c);
      }
      std::sort(codons[a].begin(), codons[a].end());
    }
    std::sort(all.begin(), all.end());
    for (int i = 0; i < 64; i++) sense_id[i] = -1;
    for (size_t i = 0; i < all.size(); i++) sense_id[all[i]] = (int)i;
  }
};

const GeneticCode &gcode() {
  static GeneticCode g;
  return g;
}

thread_local std::string g_last_error;

}  // namespace

struct cf_model {
  double params[CF_NPARAMS];
  double kT;
  double en[EN_N];
};

template <typename T>
struct PrecTables {
  bool inside_alloc = false, outside_alloc = false;
  bool stale = false;  // hold a previous protein's values: cleared before the next inside pass
  DP<T> dp{};
  BifBuf<T> bb{};
  cudaGraphExec_t gin = nullptr;  // inside pass as one graph
  int gin_nodes = 0;
  OutBuf<T> ob{};
  cudaGraphExec_t gout = nullptr;  // outside pass as one graph
  int gout_nodes = 0;
  std::vector<void *> allocs;
};

// Minimum free energy form: integer-cost tables, the pass as one graph, and
// the traceback's scratch (per protein length).
struct MfeTables {
  bool alloc = false;
  MfeDP dp{};
  cudaGraphExec_t g = nullptr;
  int nodes = 0;
  int4 *stack = nullptr;
  int *state = nullptr;
  int32_t *codons = nullptr, *partner = nullptr;
  std::vector<void *> allocs;
};

// Tensor-model tables of one precision (cf_tm.cuh), allocated on the first
// cf_tm_inside of a protein, with the pass captured as a CUDA graph for the
// model it was built for.
template <typename T>
struct TmTables {
  T *Q = nullptr, *L = nullptr, *F = nullptr;
  int *E = nullptr, *err = nullptr;
  unsigned long long *dmax = nullptr;
  double *Zm = nullptr, *logz = nullptr;
  bool alloc = false;
  cudaGraphExec_t g = nullptr;
  const void *gmodel = nullptr;  // the model's device copy and rho count the graph was built for
  int gnrho = 0;
};

struct cf_problem {
  const cf_model *model = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int n = 0, m = 0;
  std::vector<int> M, base, bnd, cid;
  std::vector<double> eHL;
  // device, shared by both precisions
  int *dM = nullptr, *dbase = nullptr, *dbnd = nullptr, *dE = nullptr, *derr = nullptr;
  unsigned long long *ddmax = nullptr;
  double *du0 = nullptr, *dZm = nullptr, *dtrans = nullptr, *dp0 = nullptr;
  double *dcm = nullptr, *dbm = nullptr, *dpg = nullptr;  // codon, base marginals; pair-bonus gradient
  int *dcid = nullptr;                                    // [n*6] sense codon id of state a at p
  // binary64 masters of the position transfers (k_transfers), the weights
  // they are made from, the per-boundary log rescales and log Z
  double *dlw = nullptr, *dpb = nullptr, *dTr64 = nullptr, *dX64 = nullptr, *den64 = nullptr;
  double *dls = nullptr, *dlogz = nullptr;
  float *dP = nullptr;
  std::vector<void *> shared_allocs;
  PrecTables<float> f32;
  PrecTables<double> f64;
  int last_prec = -1;
  bool have_inside = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float t_in = 0, t_out = 0;
  int l_in = 0, l_out = 0;
  // sampler scratch, grown on demand
  std::vector<void *> smp_allocs;
  size_t smp_cap = 0;
  int2 *smp_stack = nullptr;
  int *smp_state = nullptr, *smp_err = nullptr;
  // batched window DP: energy tables (once) and buffers grown on demand
  std::vector<void *> win_allocs, win_buf_allocs;
  float *win_en = nullptr, *win_ehl = nullptr;
  int *win_err = nullptr;
  float *win_scratch = nullptr;
  size_t win_scratch_cap = 0;
  uint8_t *win_bases = nullptr;
  int64_t *win_off = nullptr;
  double *win_logz = nullptr;
  size_t win_bases_cap = 0, win_nwin_cap = 0;
  // pinned host staging of host-side window inputs and outputs
  uint8_t *win_hbases = nullptr;
  int64_t *win_hoff = nullptr;
  double *win_hlogz = nullptr;
  size_t win_hbases_cap = 0, win_hnwin_cap = 0;
  float t_win = 0;
  MfeTables mfe;
  float t_mfe = 0;
  long long sub_steps = 0;  // element expansions of the last cf_subopt
  // position-state layout: 0 codon states (codon-pair tensor train), 1 the
  // single-codon layout (first base; first and second base; third base)
  int layout_req = 0, layout = 0;
  std::vector<int> smap;   // single-codon layout: [m][6] packed states and bases of each codon slot
  std::vector<int> sc1;    // single-codon layout: first base of each state at a residue's second position
  int *dsmap = nullptr;
  // single-codon layout: per residue and (state at 3r+1, state at 3r+2) the
  // sense codon id | (the state it needs at 3r) << 8, -1 for no codon
  std::vector<int> sctab;
  int *dsctab = nullptr;
  int *dsc1 = nullptr;  // sc1 on the device (the MFE's transfer costs)
  int nls = 0;             // per-transfer log rescales undone in log Z
  // tensor-based model (cf_tm_inside)
  std::vector<void *> tm_allocs;
  TmTables<float> tm32;
  TmTables<double> tm64;
  float t_tm = 0;
  int ck_request = -1;  // -1: checkpoint the interior partial sums from CF_CHECKPOINT_MIN_N on; 0 never; 1 always
  int batch = 1;        // proteins of a batch (cf_batch_*), one slab each
  long long bstride = 0;  // bytes between the slabs of a batch
};

namespace {

cf_status fail(cf_problem *p, cf_status s, const std::string &msg) {
  if (p) p->err = msg;
  g_last_error = msg;
  return s;
}

cf_status cuda_fail(cf_problem *p, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(p, e == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA, m);
}

#define CF_CUDA(p, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, #call); \
  } while (0)

// Test hook (cf_debug_fail_alloc): the number of further device allocations
// that succeed before one is made to fail; negative = off.
std::atomic<long long> g_fail_alloc_after{-1};

// A batch of equal-length proteins places every array of its first protein in
// one slab (bump allocation from this thread's arena while it is set); the
// other proteins' slabs follow at a fixed stride.
struct Arena {
  char *base = nullptr;
  size_t cap = 0, used = 0;
};
thread_local Arena *g_arena = nullptr;

template <typename V>
cudaError_t dalloc(std::vector<void *> &list, V **ptr, size_t count) {
  long long k = g_fail_alloc_after.load();
  while (k >= 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 0) return cudaErrorMemoryAllocation;  // forced failure, nothing allocated
  if (g_arena) {
    const size_t bytes = (count * sizeof(V) + 255) / 256 * 256;
    if (g_arena->used + bytes > g_arena->cap) return cudaErrorMemoryAllocation;
    *ptr = (V *)(g_arena->base + g_arena->used);
    g_arena->used += bytes;
    return cudaSuccess;  // owned by the batch buffer, not by the list
  }
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(V));
  if (e != cudaSuccess) return e;
  list.push_back(q);
  *ptr = (V *)q;
  return cudaSuccess;
}

void free_list(std::vector<void *> &list) {
  for (void *q : list) cudaFree(q);
  list.clear();
}

void free_mfe(MfeTables &t) {
  if (t.g) cudaGraphExecDestroy(t.g);
  t.g = nullptr;
  free_list(t.allocs);
  t = MfeTables{};
}

template <typename T>
void free_prec(PrecTables<T> &t) {
  if (t.gin) cudaGraphExecDestroy(t.gin);
  if (t.gout) cudaGraphExecDestroy(t.gout);
  t.gin = nullptr;
  t.gout = nullptr;
  free_list(t.allocs);
  t.inside_alloc = t.outside_alloc = false;
  t.dp = DP<T>{};
}

// Where a caller's buffer lives, seen from a problem on `device`: 0 host
// memory (pageable or pinned), 1 device memory the problem's kernels may read
// and write (memory of that device, or managed memory), -1 device memory of
// another device (rejected: a kernel of this problem must not touch it).
int classify_ptr(int type, int ptr_device, int device) {
  if (type == cudaMemoryTypeManaged) return 1;
  if (type == cudaMemoryTypeDevice) return ptr_device == device ? 1 : -1;
  return 0;
}

int ptr_kind(const void *ptr, int device) {
  if (!ptr) return 0;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return classify_ptr((int)a.type, a.device, device);
}

bool is_device_ptr(const void *ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Checkpointing of the interior partial sums (the outside pass recomputes
// them in blocks of 64 diagonals instead of reading a table of 29 blocks per
// cell): from this length on unless the problem asks otherwise.
bool yy_checkpointed(const cf_problem *p) {
  return p->ck_request == 1 || (p->ck_request < 0 && p->n >= CF_CHECKPOINT_MIN_N);
}
size_t yy_inside_elems(int n, int ck) {
  return ck ? (size_t)2 * n * NYY * BLK : ncells(n) * NYY * BLK;
}
size_t yy_ck_elems(int n) { return ((size_t)n / YYCK_BLOCK + 1) * n * NYY * BLK; }
size_t yy_block_elems(int n) { return (size_t)2 * YYCK_BLOCK * n * NYY * BLK; }

template <typename T>
cf_status alloc_inside(cf_problem *p, PrecTables<T> &t) {
  if (t.inside_alloc) return CF_OK;
  const int n = p->n;
  const size_t nc = ncells(n) * BLK;
  DP<T> &d = t.dp;
  d.n = n;
  d.m = p->m;
  d.Mp = p->dM;
  d.base = p->dbase;
  d.bnd = p->dbnd;
  d.u0 = p->du0;
  d.E = p->dE;
  d.dmax = p->ddmax;
  d.err = p->derr;
  d.Zm = p->dZm;
  d.P = p->dP;
  T *tr, *x, *en, *eh;
  auto &L = t.allocs;
  CF_CUDA(p, dalloc(L, &tr, (size_t)n * BLK));
  CF_CUDA(p, dalloc(L, &x, (size_t)n * 4 * BLK));
  CF_CUDA(p, dalloc(L, &en, (size_t)EN_N));
  CF_CUDA(p, dalloc(L, &eh, (size_t)n + 2));
  k_cast<T><<<148, 256, 0, p->stream>>>(p->dTr64, tr, (size_t)n * BLK);
  k_cast<T><<<148, 256, 0, p->stream>>>(p->dX64, x, (size_t)n * 4 * BLK);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaStreamSynchronize(p->stream));
  std::vector<T> h;
  h.assign(p->model->en, p->model->en + EN_N);
  CF_CUDA(p, cudaMemcpy(en, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  h.assign(p->eHL.begin(), p->eHL.end());
  CF_CUDA(p, cudaMemcpy(eh, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  d.Tr = tr;
  d.X = x;
  d.en = en;
  d.eHL = eh;
  T **tabs[] = {&d.CH, &d.QB, &d.XI, &d.HB, &d.QMpp, &d.QMpu, &d.G, &d.QM2pp, &d.QM2pu, &d.QM2up, &d.QM2uu};
  for (T **q : tabs) {
    CF_CUDA(p, dalloc(L, q, nc));
    CF_CUDA(p, cudaMemset(*q, 0, nc * sizeof(T)));
  }
  // interior partial sums: stored whole, or checkpointed (a ring of two
  // diagonals and every 64th diagonal; the outside pass recomputes blocks)
  d.yyck = yy_checkpointed(p) ? 1 : 0;
  const size_t yy_elems = yy_inside_elems(n, d.yyck);
  d.YYck = nullptr;
  d.YYb = nullptr;
  CF_CUDA(p, dalloc(L, &d.YY, yy_elems));
  CF_CUDA(p, cudaMemset(d.YY, 0, yy_elems * sizeof(T)));
  if (d.yyck) {
    const size_t ck = yy_ck_elems(n);
    CF_CUDA(p, dalloc(L, &d.YYck, ck));
    CF_CUDA(p, cudaMemset(d.YYck, 0, ck * sizeof(T)));
  }
  T **ext[] = {&d.Q5U, &d.Q5P, &d.Gx};
  for (T **q : ext) {
    CF_CUDA(p, dalloc(L, q, (size_t)n * BLK));
    CF_CUDA(p, cudaMemset(*q, 0, (size_t)n * BLK * sizeof(T)));
  }
  t.bb.ncmax = 1;
  CF_CUDA(p, dalloc(L, &t.bb.main, (size_t)BIFRING * n * BLK));
  CF_CUDA(p, dalloc(L, &t.bb.ext, (size_t)BIFRING * BLK));
  t.bb.far = nullptr;
  t.bb.farslices = far_nslice(n, 0, std::max(0, (n - 1) / FARD * FARD));  // the widest band's slices
  t.bb.gfac = nullptr;
  t.bb.gdev = nullptr;
  t.bb.spread = nullptr;
  if (n * sizeof(float) <= 200 * 1024 && p->batch == 1) {
    CF_CUDA(p, dalloc(L, &t.bb.spread, (size_t)1));
    CF_CUDA(p, cudaMemset(t.bb.spread, 0, sizeof(int)));
    CF_CUDA(p, cudaFuncSetAttribute((const void *)k_in_range<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(n * sizeof(float))));
  }
  if (sizeof(T) == sizeof(float) && n > 3 * FARD) {
    CF_CUDA(p, dalloc(L, &t.bb.far, (size_t)2 * n * FARD * t.bb.farslices * BLK));
    CF_CUDA(p, dalloc(L, &t.bb.gfac, (size_t)2 * n));
    CF_CUDA(p, dalloc(L, &t.bb.gdev, (size_t)n / FARD + 1));
    CF_CUDA(p, cudaMemset(t.bb.gdev, 0, ((size_t)n / FARD + 1) * sizeof(int)));
  }
  const T **stab = nullptr;
  CF_CUDA(p, dalloc(L, &stab, (size_t)n * SI_N));
  t.bb.stab = stab;
  CF_CUDA(p, dalloc(L, &t.bb.dtab, (size_t)n * NCOPY));
  k_in_slot_tab<T><<<n, 256, 0, p->stream>>>(t.dp, t.bb);
  CF_CUDA(p, cudaGetLastError());
  t.inside_alloc = true;
  return CF_OK;
}

// Binary64 proteins up to this length (every batch) take the grouped
// bifurcation gathers: a gather has at most n - 4 terms, a few steps of
// 16 for two warps.
constexpr int GRP64_MAXN = 48;

// Grid size cap of the per-cell bifurcation kernels without far bands, which
// loop over their cells grid-stride.  A cap of one or two CTAs per SM leaves
// room for the light CTAs but starves the off-chain kernels (measured: slower
// at 900 nt), so the graphs use a cap above every diagonal's cell count: one
// CTA per cell.
int offchain_ctas(const cf_problem *p, int per_sm) {
  int sms = 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) cudaGetLastError();
  return std::max(1, sms * per_sm);
}

// Scheduling priority of a kernel node: the light-kernel chain is the
// critical path, the bifurcation kernels fill in behind it.
cudaError_t set_priority(cudaGraphNode_t node, bool high) {
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e != cudaSuccess) return e;
  cudaKernelNodeAttrValue v = {};
  v.priority = high ? hi : lo;
  return cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributePriority, &v);
}

// A programmatic edge between consecutive kernels of a chain: the successor
// may start once every CTA of the predecessor has called
// griddep_launch_dependents, so that the launch and the successor's early
// part (loads of inputs the predecessor does not write) overlap the
// predecessor's end; the successor's griddep_wait then waits for it to finish.
cudaError_t add_programmatic_edge(cudaGraph_t g, cudaGraphNode_t from, cudaGraphNode_t to) {
  cudaGraphEdgeData ed = {};
  ed.from_port = cudaGraphKernelNodePortProgrammatic;
  ed.to_port = cudaGraphKernelNodePortDefault;
  ed.type = cudaGraphDependencyTypeProgrammatic;
  return cudaGraphAddDependencies(g, &from, &to, &ed, 1);
}

// The inside pass as a CUDA graph: a chain of light kernels, one per
// anti-diagonal (consecutive ones joined by programmatic edges), and the
// bifurcation kernel of diagonal d hanging off the light
// kernel of diagonal d-4, so that it runs while d-3..d-1 are being filled;
// with far bands (binary32) the far kernel of band d0 (after its factor table)
// hangs off the light kernel of d0 - 17 and precedes the band's bifurcation
// kernels.
template <typename T>
cf_status build_inside_graph(cf_problem *p, PrecTables<T> &t) {
  if (t.gin) return CF_OK;
  const int n = p->n;
  const int cap_bif = offchain_ctas(p, 64);
  const size_t smem = in_light_smem<T, NT_IN>();
  const bool BT = p->batch > 1;  // batched kernels move their pointers per protein
  const void *klight = BT ? (const void *)k_in_light<T, NT_IN, true> : (const void *)k_in_light<T, NT_IN, false>;
  CF_CUDA(p, cudaFuncSetAttribute(klight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaGraph_t g;
  CF_CUDA(p, cudaGraphCreate(&g, 0));
  cudaGraphNode_t mset;
  cudaMemsetParams ms = {};
  ms.dst = p->ddmax;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = (size_t)n * 2;
  ms.height = p->batch;
  ms.pitch = p->batch > 1 ? (size_t)p->bstride : 0;
  cudaError_t e = cudaGraphAddMemsetNode(&mset, g, nullptr, 0, &ms);
  std::vector<cudaGraphNode_t> k2(n);
  std::vector<cudaGraphNode_t> k1(n);
  int nodes = 0;
  DP<T> dp = t.dp;
  BifBuf<T> bb = t.bb;
  // far bands (binary32): band d0 hangs off the light kernel of d0 - FARD - 1
  // and precedes the bifurcation kernels of its FARD diagonals
  const bool banded = bb.far != nullptr;
  std::vector<cudaGraphNode_t> kf((size_t)n / FARD + 1, nullptr);
  if (banded)
    CF_CUDA(p, cudaFuncSetAttribute((const void *)k_in_far, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)in_far_smem(n)));
  for (int d = 0; d < n && e == cudaSuccess; d++) {
    int dd = d;
    void *args[] = {&dp, &bb, &dd};
    const int d0 = d / FARD * FARD;
    if (banded && d == d0 && far_band(d0)) {
      DP<float> dpf;
      BifBuf<float> bbf;
      std::memcpy(&dpf, &dp, sizeof(dpf));
      std::memcpy(&bbf, &bb, sizeof(bbf));
      int b0 = d0;
      void *fargs[] = {&dpf, &bbf, &b0};
      // the band's rescale factors, after the light kernel of c and after the
      // far kernel two bands back (same factor buffer)
      cudaKernelNodeParams kq = {};
      kq.func = (void *)k_in_far_factors;
      kq.gridDim = dim3(1);
      kq.blockDim = dim3(512);
      kq.kernelParams = fargs;
      cudaGraphNode_t qdeps[2] = {k2[far_c(d0)], nullptr}, kfq;
      int nq = 1;
      if (d0 / FARD >= 2 && kf[d0 / FARD - 2]) qdeps[nq++] = kf[d0 / FARD - 2];
      e = cudaGraphAddKernelNode(&kfq, g, qdeps, nq, &kq);
      if (e == cudaSuccess) e = set_priority(kfq, false);
      nodes++;
      cudaKernelNodeParams kp = {};
      kp.func = (void *)k_in_far;
      kp.gridDim = dim3((n - d0 + FARTX - 1) / FARTX, far_nslice(n, 0, d0));
      kp.blockDim = dim3(256);
      kp.sharedMemBytes = (unsigned)in_far_smem(far_c(d0));
      kp.kernelParams = fargs;
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(&kf[d0 / FARD], g, &kfq, 1, &kp);
      if (e == cudaSuccess) e = set_priority(kf[d0 / FARD], false);
      nodes++;
      if (e != cudaSuccess) break;
    }
    if (d >= 8) {
      cudaKernelNodeParams kp = {};
      // few near split points, or a short protein: two warps per cell
      kp.func = BT ? (void *)k_in_bif_grp<T, true> : (void *)k_in_bif_grp<T, false>;
      kp.gridDim = dim3((n - d + 3) / 4 + 1, p->batch);
      if constexpr (sizeof(T) != sizeof(float)) {
        if (n > GRP64_MAXN) {  // binary64 (no far bands): one CTA per cell
          kp.func = BT ? (void *)k_in_bif<T, true> : (void *)k_in_bif<T, false>;
          kp.gridDim = dim3(std::min(n - d + 1, cap_bif), p->batch);
        }
      }
      kp.blockDim = dim3(256);
      kp.kernelParams = args;
      cudaGraphNode_t bdeps[2] = {k2[d - 4], nullptr};
      int nb = 1;
      if (banded && far_band(d0)) bdeps[nb++] = kf[d0 / FARD];
      e = cudaGraphAddKernelNode(&k1[d], g, bdeps, nb, &kp);
      if (e == cudaSuccess) e = set_priority(k1[d], false);
      nodes++;
    }
    if (e != cudaSuccess) break;
    cudaGraphNode_t deps[2];
    int nd = 0;
    if (d == 0) deps[nd++] = mset;
    if (d >= 8) deps[nd++] = k1[d];
    cudaKernelNodeParams kp = {};
    kp.func = (void *)klight;
    kp.gridDim = dim3(n - d, p->batch);
    kp.blockDim = dim3(NT_IN);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&k2[d], g, deps, nd, &kp);
    if (e == cudaSuccess && d > 0) e = add_programmatic_edge(g, k2[d - 1], k2[d]);
    if (e == cudaSuccess) e = set_priority(k2[d], true);
    nodes++;
  }
  if (e == cudaSuccess) {
    void *args[] = {&dp};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_inside_finish<T>;
    kp.gridDim = dim3(1, p->batch);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    cudaGraphNode_t fin;
    e = cudaGraphAddKernelNode(&fin, g, &k2[n - 1], 1, &kp);
    nodes++;
    if (e == cudaSuccess && t.bb.spread && sizeof(T) == sizeof(float)) {  // the range of the binary32 tables
      int *sp = t.bb.spread;
      void *rargs[] = {&dp, &sp};
      cudaKernelNodeParams kr = {};
      kr.func = (void *)k_in_range<T>;
      kr.gridDim = dim3(1, p->batch);
      kr.blockDim = dim3(1024);
      kr.sharedMemBytes = (unsigned)(sizeof(float) * n);
      kr.kernelParams = rargs;
      cudaGraphNode_t rn;
      e = cudaGraphAddKernelNode(&rn, g, &fin, 1, &kr);
      nodes++;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&t.gin, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(p, e, "inside graph");
  t.gin_nodes = nodes;
  return CF_OK;
}

template <typename T>
cf_status alloc_outside(cf_problem *p, PrecTables<T> &t) {
  if (t.outside_alloc) return CF_OK;
  const int n = p->n;
  const size_t nc = ncells(n) * BLK;
  DP<T> &d = t.dp;
  auto &L = t.allocs;
  T **tabs[] = {&d.hCH, &d.hQB, &d.hGc, &d.hXI, &d.hHB, &d.hQMpp, &d.hQMpu, &d.hG, &d.hQM2pp, &d.hQM2pu, &d.hQM2up, &d.hQM2uu};
  for (T **q : tabs) {
    CF_CUDA(p, dalloc(L, q, nc));
    CF_CUDA(p, cudaMemset(*q, 0, nc * sizeof(T)));
  }
  CF_CUDA(p, dalloc(L, &d.hYY, (size_t)YRING * n * NYY * BLK));
  CF_CUDA(p, cudaMemset(d.hYY, 0, (size_t)YRING * n * NYY * BLK * sizeof(T)));
  if (d.yyck) {
    CF_CUDA(p, dalloc(L, &d.YYb, yy_block_elems(n)));
    CF_CUDA(p, cudaMemset(d.YYb, 0, yy_block_elems(n) * sizeof(T)));
  }
  T **ext[] = {&d.hQ5U, &d.hQ5P, &d.hGx};
  for (T **q : ext) {
    CF_CUDA(p, dalloc(L, q, (size_t)n * BLK));
    CF_CUDA(p, cudaMemset(*q, 0, (size_t)n * BLK * sizeof(T)));
  }
  CF_CUDA(p, dalloc(L, &d.tgY, nc));
  CF_CUDA(p, dalloc(L, &d.hT, (size_t)n * BLK));
  CF_CUDA(p, dalloc(L, &d.hX, (size_t)n * 4 * BLK));
  CF_CUDA(p, dalloc(L, &t.ob.hg, (size_t)BIFRING * n * BLK));
  CF_CUDA(p, dalloc(L, &t.ob.hq, (size_t)BIFRING * n * BLK));
  CF_CUDA(p, dalloc(L, &t.ob.hgx, (size_t)BIFRING * BLK));
  t.ob.far = nullptr;
  t.ob.fwh = nullptr;
  t.ob.fdev = nullptr;
  if (sizeof(T) == sizeof(float) && of_band(n, 0) && p->batch == 1) {  // a batch gathers every term per diagonal
    CF_CUDA(p, dalloc(L, &t.ob.far, (size_t)6 * n * OFD * BLK));
    CF_CUDA(p, dalloc(L, &t.ob.fwh, (size_t)2 * n));
    CF_CUDA(p, dalloc(L, &t.ob.fdev, (size_t)1));
    CF_CUDA(p, cudaMemset(t.ob.fdev, 0, sizeof(int)));
  }
  CF_CUDA(p, dalloc(L, &t.ob.otab, (size_t)n * SO_N));
  const T **sstab = nullptr;
  CF_CUDA(p, dalloc(L, &sstab, (size_t)n * SS_N));
  t.ob.stab = sstab;
  k_out_slot_tab<T><<<n, 256, 0, p->stream>>>(t.dp, t.ob);
  k_side_slot_tab<T><<<n, 256, 0, p->stream>>>(t.dp, t.ob);
  CF_CUDA(p, cudaGetLastError());
  t.outside_alloc = true;
  return CF_OK;
}

// zero `bytes` at ptr, and at the same place of every slab of a batch
cudaError_t add_memset(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep, int ndep, void *ptr,
                       size_t bytes, int batch = 1, long long bstride = 0) {
  cudaMemsetParams ms = {};
  ms.dst = ptr;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = bytes / 4;
  ms.height = batch;
  ms.pitch = batch > 1 ? (size_t)bstride : 0;
  return cudaGraphAddMemsetNode(node, g, dep, ndep, &ms);
}

// The outside pass as a CUDA graph: a chain of light kernels from d = n-1 down
// to 0; the off-chain launch of diagonal d (its transposed bifurcation gathers
// and the side work of diagonal d+4) hangs off the light kernel of d+4 and
// precedes the light kernel of d; the far gathers of a band hang off the light
// kernel of a_lo + 35; the transfer gradients and the marginals follow the
// chain.
template <typename T>
cf_status build_outside_graph(cf_problem *p, PrecTables<T> &t) {
  if (t.gout) return CF_OK;
  const int n = p->n;
  const int cap_bif = offchain_ctas(p, 64);
  const size_t nc = ncells(n) * BLK;
  const size_t smem = out_light_smem<T, NT>(), smemw = out_light_smem<T, NT_WIDE>(), smem3 = out_side_smem<T>();
  // batched kernels move their pointers per protein; a single protein's keep
  // them in the parameter bank
  const bool BT = p->batch > 1;
  const void *klight = BT ? (const void *)k_out_light<T, NT, true> : (const void *)k_out_light<T, NT, false>;
  const void *klightw = BT ? (const void *)k_out_light<T, NT_WIDE, true> : (const void *)k_out_light<T, NT_WIDE, false>;
  const void *ktgf = BT ? (const void *)k_out_tg<T, true> : (const void *)k_out_tg<T, false>;
  // binary32 (far bands, or a short protein or a batch without them) and
  // short binary64 proteins: grouped gathers, two warps per cell; longer
  // binary64 proteins: one CTA per cell
  const bool GRP = sizeof(T) == sizeof(float) || n <= GRP64_MAXN;
  const void *koff = BT ? (const void *)k_out_off<T, true, true> : (const void *)k_out_off<T, true, false>;
  if constexpr (sizeof(T) != sizeof(float))
    if (!GRP) koff = BT ? (const void *)k_out_off<T, false, true> : (const void *)k_out_off<T, false, false>;
  CF_CUDA(p, cudaFuncSetAttribute(klight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CF_CUDA(p, cudaFuncSetAttribute(klightw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemw));
  CF_CUDA(p, cudaFuncSetAttribute(ktgf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out_tg_smem<T>()));
  CF_CUDA(p, cudaFuncSetAttribute(koff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3));
  cudaGraph_t g;
  CF_CUDA(p, cudaGraphCreate(&g, 0));
  DP<T> dp = t.dp;
  OutBuf<T> ob = t.ob;
  cudaGraphNode_t m[5];
  const int B = p->batch;
  const long long bs = p->bstride;
  cudaError_t e = add_memset(g, &m[0], nullptr, 0, dp.hCH, nc * sizeof(T), B, bs);
  if (e == cudaSuccess) e = add_memset(g, &m[1], &m[0], 1, dp.hXI, nc * sizeof(T), B, bs);
  if (e == cudaSuccess) e = add_memset(g, &m[2], &m[1], 1, dp.hT, (size_t)n * BLK * sizeof(double), B, bs);
  if (e == cudaSuccess) e = add_memset(g, &m[3], &m[2], 1, dp.hX, (size_t)n * 4 * BLK * sizeof(double), B, bs);
  if (e == cudaSuccess) e = add_memset(g, &m[4], &m[3], 1, dp.P, (size_t)n * n * sizeof(float), B, bs);
  std::vector<cudaGraphNode_t> k2(n), k1(n);
  // far bands (binary32): both gathers of band alo hang off the light kernel
  // of diagonal of_c(alo) and precede the bifurcation kernels of the band
  const bool banded = ob.far != nullptr;
  std::vector<cudaGraphNode_t> kfr((size_t)n / OFD + 1, nullptr), kfc((size_t)n / OFD + 1, nullptr);
  if (banded) {
    CF_CUDA(p, cudaFuncSetAttribute((const void *)k_out_far<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)out_far_smem(n)));
    CF_CUDA(p, cudaFuncSetAttribute((const void *)k_out_far<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)out_far_smem(n)));
  }
  int nodes = 0;
  // far-band rescale factors of the pass, before the first light kernel
  cudaGraphNode_t first = m[4];
  if (banded && e == cudaSuccess) {
    DP<float> dpf;
    OutBuf<float> obf;
    std::memcpy(&dpf, &dp, sizeof(dpf));
    std::memcpy(&obf, &ob, sizeof(obf));
    void *qargs[] = {&dpf, &obf};
    cudaKernelNodeParams kq = {};
    kq.func = (void *)k_out_far_factors;
    kq.gridDim = dim3(1);
    kq.blockDim = dim3(512);
    kq.kernelParams = qargs;
    e = cudaGraphAddKernelNode(&first, g, &m[4], 1, &kq);
    nodes++;
  }
  for (int d = n - 1; d >= 0 && e == cudaSuccess; d--) {
    int dd = d;
    void *args[] = {&dp, &ob, &dd};
    const int alo = d / OFD * OFD;
    const bool fb = banded && of_band(n, alo);
    if (fb && d == alo + OFD - 1) {
      DP<float> dpf;
      OutBuf<float> obf;
      std::memcpy(&dpf, &dp, sizeof(dpf));
      std::memcpy(&obf, &ob, sizeof(obf));
      int a0 = alo;
      void *fargs[] = {&dpf, &obf, &a0};
      const size_t slot = (size_t)((alo / OFD) % 3) * n * OFD * BLK, len = (size_t)n * OFD * BLK * sizeof(float);
      cudaGraphNode_t z[2];
      e = add_memset(g, &z[0], &k2[of_c(alo)], 1, obf.far + slot, len);
      if (e == cudaSuccess) e = add_memset(g, &z[1], &k2[of_c(alo)], 1, obf.far + (size_t)3 * n * OFD * BLK + slot, len);
      for (int kind = 0; kind < 2 && e == cudaSuccess; kind++) {
        cudaKernelNodeParams kp = {};
        kp.func = kind == 0 ? (void *)k_out_far<true> : (void *)k_out_far<false>;
        kp.gridDim = dim3(out_far_tiles(n, alo), std::max(1, out_far_slices(n, alo, kind == 0)));
        kp.blockDim = dim3(256);
        kp.sharedMemBytes = (unsigned)out_far_smem(n);
        kp.kernelParams = fargs;
        cudaGraphNode_t &kn = kind == 0 ? kfr[alo / OFD] : kfc[alo / OFD];
        e = cudaGraphAddKernelNode(&kn, g, &z[kind], 1, &kp);
        if (e == cudaSuccess) e = set_priority(kn, false);
        nodes++;
      }
      if (e != cudaSuccess) break;
    }
    // one off-chain launch per diagonal d: the bifurcation gathers of d and the
    // side work of d+4 (its scatters land on diagonals <= d), both after the
    // light kernel of d+4
    const bool hasb = d <= n - 5 && d >= 1, hass = d + 4 <= n - 1 && d >= 1;  // no side work below d = 5
    if (hasb || hass) {
      int nbif = hasb ? (GRP ? (n - d + 3) / 4 + 1 : n - d + 1) : 0;
      void *oargs[] = {&dp, &ob, &dd, &nbif};
      cudaKernelNodeParams kp = {};
      kp.func = (void *)koff;
      kp.gridDim = dim3(nbif + (hass ? n - d - 4 : 0), B);
      kp.blockDim = dim3(NT3);
      kp.sharedMemBytes = (unsigned)smem3;
      kp.kernelParams = oargs;
      cudaGraphNode_t bdeps[3] = {k2[d + 4], nullptr, nullptr};
      int nb = 1;
      if (hasb && fb) {
        bdeps[nb++] = kfr[alo / OFD];
        bdeps[nb++] = kfc[alo / OFD];
      }
      e = cudaGraphAddKernelNode(&k1[d], g, bdeps, nb, &kp);
      if (e == cudaSuccess) e = set_priority(k1[d], false);
      nodes++;
      if (e != cudaSuccess) break;
    }
    cudaGraphNode_t deps[3];
    int nd = 0;
    if (d == n - 1) deps[nd++] = first;
    if (hasb || hass) deps[nd++] = k1[d];
    cudaKernelNodeParams kp = {};
    const bool wide = (long long)(n - d) * B > WIDE_CELLS;  // the launch's cells, over every protein of a batch
    kp.func = (void *)(wide ? klightw : klight);
    kp.gridDim = dim3(n - d, B);
    kp.blockDim = dim3(wide ? NT_WIDE : NT);
    kp.sharedMemBytes = (unsigned)(wide ? smemw : smem);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&k2[d], g, deps, nd, &kp);
    if (e == cudaSuccess && d < n - 1) e = add_programmatic_edge(g, k2[d + 1], k2[d]);  // the chain
    if (e == cudaSuccess) e = set_priority(k2[d], true);
    nodes++;
  }
  // checkpointed interior partial sums: block b (diagonals 64b .. 64b + 62;
  // 64b + 63 is a checkpoint) is recomputed by a chain of one launch per
  // diagonal, after the last reader of the previous block that used its
  // buffer (block b + 2: the off-chain launch of 64b + 125) and before the
  // light kernel of 64b + 64, after which the off-chain launches read it
  if (e == cudaSuccess && dp.yyck) {
    const int nblk = (n + YYCK_BLOCK - 1) / YYCK_BLOCK;
    for (int b = nblk - 1; b >= 0 && e == cudaSuccess; b--) {
      const int D0 = b * YYCK_BLOCK, D1 = std::min(n - 1, D0 + YYCK_BLOCK - 2);
      cudaGraphNode_t prev = nullptr;
      for (int D = D0; D <= D1 && e == cudaSuccess; D++) {
        int DD = D;
        void *args[] = {&dp, &DD};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)k_yy_step<T>;
        kp.gridDim = dim3(n - D);
        kp.blockDim = dim3(192);
        kp.kernelParams = args;
        cudaGraphNode_t deps[1];
        int nd = 0;
        if (prev) deps[nd++] = prev;
        else if (D0 + 125 <= n - 1 && k1[D0 + 125]) deps[nd++] = k1[D0 + 125];
        else deps[nd++] = first;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, g, deps, nd, &kp);
        if (e == cudaSuccess) e = set_priority(node, false);
        nodes++;
        prev = node;
      }
      if (e == cudaSuccess && prev)
        e = cudaGraphAddDependencies(g, &prev, &k2[std::min(n - 1, D0 + YYCK_BLOCK)], nullptr, 1);
    }
  }
  // transfer gradients of every boundary position, after the whole chain
  cudaGraphNode_t ktg = nullptr;
  if (e == cudaSuccess) {
    void *args[] = {&dp};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)ktgf;
    kp.gridDim = dim3((n + TG_CELLS - 1) / TG_CELLS, BT ? std::max(1, n / 3 - 1) : n, 2 * B);
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = (unsigned)out_tg_smem<T>();
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&ktg, g, &k2[0], 1, &kp);
    nodes++;
  }
  cudaGraphNode_t fin = nullptr;
  if (e == cudaSuccess && p->layout == 1) {  // single-codon layout: codon and base marginals at q = 3r+1
    const int *smap = p->dsmap;
    double *cm = p->dcm, *bm = p->dbm;
    void *args[] = {&dp, &smap, &cm, &bm};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_codon_out_sc<T>;
    kp.gridDim = dim3((p->m * 6 + n + 127) / 128);
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&fin, g, &ktg, 1, &kp);
    nodes++;
  } else if (e == cudaSuccess) {
    double *trans = p->dtrans, *p0 = p->dp0;
    void *args[] = {&dp, &trans, &p0};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_marginals<T>;
    kp.gridDim = dim3((std::max(p->m - 1, 1) + 127) / 128, B);
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&fin, g, &ktg, 1, &kp);
    nodes++;
  }
  if (e == cudaSuccess) {
    float *P = dp.P;
    int nn = n;
    int *er = dp.err;
    long long bsl = bs;
    void *args[] = {&P, &nn, &er, &bsl};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_unpaired;
    kp.gridDim = dim3((n + 7) / 8, B);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    cudaGraphNode_t un;
    e = cudaGraphAddKernelNode(&un, g, &fin, 1, &kp);
    nodes++;
  }
  if (e == cudaSuccess && p->layout == 0) {
    const double *trans = p->dtrans, *p0 = p->dp0;
    const int *cid = p->dcid;
    double *cm = p->dcm, *bm = p->dbm, *pg = p->dpg;
    void *args[] = {&dp, &trans, &p0, &cid, &cm, &bm, &pg};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_codon_out<T>;
    // threads, then 4 warps a block for the codon-pair gradient (a batch
    // returns none, so its graph launches the marginal blocks only)
    kp.gridDim = dim3((p->m * 6 + n + 127) / 128 + (B > 1 ? 0 : (61 * 61 + 3) / 4), B);
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    cudaGraphNode_t co;
    e = cudaGraphAddKernelNode(&co, g, &fin, 1, &kp);
    nodes++;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&t.gout, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(p, e, "outside graph");
  t.gout_nodes = nodes;
  return CF_OK;
}

template <typename T>
cf_status clear_tables(cf_problem *p, PrecTables<T> &t);

template <typename T>
cf_status run_inside(cf_problem *p, PrecTables<T> &t, double *logZ) {
  cf_status s = alloc_inside(p, t);
  if (s != CF_OK) {
    free_prec(t);  // a failed allocation leaves no partial tables: the next call starts over
    return s;
  }
  const int n = p->n;
  cudaStream_t st = p->stream;
  s = build_inside_graph(p, t);
  if (s != CF_OK) return s;
  if (t.stale) {  // a new protein of the same length: its padding must be zero
    s = clear_tables(p, t);
    if (s != CF_OK) return s;
    t.stale = false;
  }
  CF_CUDA(p, cudaMemsetAsync(p->derr, 0, sizeof(int), st));
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  CF_CUDA(p, cudaGraphLaunch(t.gin, st));
  int launches = t.gin_nodes;
  k_logz<<<dim3(1, p->batch), 32, 0, st>>>(p->dZm, p->dE + (n - 1), p->dls, p->nls, p->dlogz,
                                           p->batch > 1 ? p->bstride : 0);
  launches++;
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaEventRecord(p->ev[1], st));
  double zm = 0, lz = 0;
  int err = 0;
  CF_CUDA(p, cudaMemcpyAsync(&zm, p->dZm, sizeof(double), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaMemcpyAsync(&lz, p->dlogz, sizeof(double), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaMemcpyAsync(&err, p->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  CF_CUDA(p, cudaEventElapsedTime(&p->t_in, p->ev[0], p->ev[1]));
  p->l_in = launches;
  if (err & ERR_STAGE_TIMEOUT) return fail(p, CF_ETIMEOUT, "inside: a bounded wait for staged inputs gave up");
  if (err & ERR_RANGE_IN)
    return fail(p, CF_ENUMERIC,
                "inside: binary32 range exceeded (the strengths of the intervals of one length spread over more "
                "bits than binary32 holds: a composition that changes strongly along the protein); use CF_FP64");
  if (err || !(zm > 0) || !std::isfinite(zm))
    return fail(p, CF_ENUMERIC, "inside: non-finite or zero partition function after scaling");
  *logZ = lz;
  return CF_OK;
}

template <typename T>
cf_status run_outside(cf_problem *p, PrecTables<T> &t) {
  cf_status s = alloc_outside(p, t);
  if (s != CF_OK) {
    // the outside tables share the precision's allocation list: release it
    // whole, and the inside results with it
    free_prec(t);
    p->have_inside = false;
    return s;
  }
  const int n = p->n;
  const size_t nc = ncells(n) * BLK;
  DP<T> &d = t.dp;
  cudaStream_t st = p->stream;
  s = build_outside_graph(p, t);
  if (s != CF_OK) return s;
  CF_CUDA(p, cudaMemsetAsync(p->derr, 0, sizeof(int), st));  // the inside pass has read its flags
  CF_CUDA(p, cudaEventRecord(p->ev[2], st));
  CF_CUDA(p, cudaGraphLaunch(t.gout, st));
  int launches = t.gout_nodes;
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaEventRecord(p->ev[3], st));
  p->l_out = launches;
  return CF_OK;
}

cf_status copy_out(cf_problem *p, void *dst, const void *src, size_t bytes, bool src_on_device) {
  cudaMemcpyKind k;
  bool ddev = is_device_ptr(dst);
  if (src_on_device) k = ddev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  else k = ddev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  CF_CUDA(p, cudaMemcpyAsync(dst, src, bytes, k, p->stream));
  return CF_OK;
}

template <typename T>
cf_status run_sample(cf_problem *p, PrecTables<T> &t, int ns, uint64_t seed, int32_t *codons, int32_t *partner) {
  const int n = p->n, m = p->m;
  cudaStream_t st = p->stream;
  const int warps = std::min(ns, 148 * 16);
  const size_t need_stack = (size_t)warps * (n + 64), need_state = (size_t)warps * n;
  if (p->smp_cap < (size_t)warps) {
    free_list(p->smp_allocs);
    p->smp_cap = 0;  // stays 0 if an allocation below fails
    CF_CUDA(p, dalloc(p->smp_allocs, &p->smp_stack, need_stack));
    CF_CUDA(p, dalloc(p->smp_allocs, &p->smp_state, need_state));
    CF_CUDA(p, dalloc(p->smp_allocs, &p->smp_err, (size_t)1));
    p->smp_cap = warps;
  }
  const int kc = ptr_kind(codons, p->device), kp = ptr_kind(partner, p->device);
  if (kc < 0 || kp < 0) return fail(p, CF_EINVAL, "cf_sample: output is device memory of another device");
  const bool dc = kc > 0, dpn = kp > 0;
  int32_t *ocod = codons, *opar = partner;
  std::vector<void *> tmp;
  cudaError_t ea = cudaSuccess;
  if (!dc) ea = dalloc(tmp, &ocod, (size_t)ns * m);
  if (ea == cudaSuccess && !dpn) ea = dalloc(tmp, &opar, (size_t)ns * n);
  if (ea != cudaSuccess) {
    free_list(tmp);
    return cuda_fail(p, ea, "cf_sample: output staging");
  }
  CF_CUDA(p, cudaMemsetAsync(p->smp_err, 0, sizeof(int), st));
  SampleArgs<T> a;
  a.p = t.dp;
  a.cid = p->dcid;
  a.sctab = p->layout == 1 ? p->dsctab : nullptr;
  a.nsamples = ns;
  a.seed = seed;
  a.stack = p->smp_stack;
  a.state = p->smp_state;
  a.codons = ocod;
  a.partner = opar;
  a.err = p->smp_err;
  k_sample<T><<<(warps + 3) / 4, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p->smp_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !dc) e = cudaMemcpyAsync(codons, ocod, sizeof(int32_t) * ns * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !dpn) e = cudaMemcpyAsync(partner, opar, sizeof(int32_t) * ns * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free_list(tmp);
  if (e != cudaSuccess) return cuda_fail(p, e, "cf_sample");
  if (err) return fail(p, CF_ENUMERIC, "cf_sample: traceback inconsistency code " + std::to_string(err));
  return CF_OK;
}

// The codon-pair tensor train along the backbone (Eq. pair-tt), made on the
// device by k_transfers from the weights (NULL = all zero): binary64 masters
// of T_p and X_p, residue 0's weights u0 and the per-boundary log rescales.
// The tables of each allocated precision are refreshed by upload_transfers.
cf_status device_transfers(cf_problem *p, const double *lw, const double *pb) {
  const int n = p->n, m = p->m;
  cudaStream_t st = p->stream;
  if (p->layout == 1) {
    // single-codon layout: T_{3r}[a][b] = 1 where state a's base at 3r is
    // state b's first base at 3r+1, T_{3r+1}[b][c] = s_r e^{lw[r][codon]} for
    // the codon whose first and second bases are state b at 3r+1 and whose
    // third base is state c at 3r+2 (s_r makes the average row sum one;
    // exact, undone in log Z), T_{3r+2} = 1 into every state of the next
    // residue; u0 = 1
    std::vector<double> T((size_t)n * BLK, 0.0), u0(NS, 0.0), ls((size_t)std::max(m, 1), 0.0);
    for (int r = 0; r < m; r++) {
      const int q = 3 * r;
      double sum = 0;
      for (int s2 = 0; s2 < 6; s2++) {
        const int sm = p->smap[(size_t)r * 6 + s2];
        if (sm < 0) continue;
        const double w = std::exp(lw ? lw[(size_t)r * 6 + s2] : 0.0);
        T[(size_t)(q + 1) * BLK + (sm & 15) * NS + ((sm >> 4) & 15)] = w;
        sum += w;
      }
      const double sr = p->M[q + 1] / sum;
      for (int e = 0; e < BLK; e++) T[(size_t)(q + 1) * BLK + e] *= sr;
      ls[r] = std::log(sr);
      for (int a = 0; a < p->M[q]; a++)
        for (int b2 = 0; b2 < p->M[q + 1]; b2++)
          if (p->base[(size_t)q * NS + a] == p->sc1[(size_t)(q + 1) * NS + b2]) T[(size_t)q * BLK + a * NS + b2] = 1.0;
      if (r + 1 < m)
        for (int c = 0; c < p->M[q + 2]; c++)
          for (int d = 0; d < p->M[q + 3]; d++) T[(size_t)(q + 2) * BLK + c * NS + d] = 1.0;
    }
    for (int a0 = 0; a0 < p->M[0]; a0++) u0[a0] = 1.0;
    if (lw) CF_CUDA(p, cudaMemcpyAsync(p->dlw, lw, sizeof(double) * (size_t)m * 6, cudaMemcpyHostToDevice, st));
    else CF_CUDA(p, cudaMemsetAsync(p->dlw, 0, sizeof(double) * (size_t)m * 6, st));
    CF_CUDA(p, cudaMemsetAsync(p->dpb, 0, sizeof(double) * 61 * 61, st));
    CF_CUDA(p, cudaMemcpyAsync(p->dTr64, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice, st));
    CF_CUDA(p, cudaMemcpyAsync(p->du0, u0.data(), sizeof(double) * NS, cudaMemcpyHostToDevice, st));
    CF_CUDA(p, cudaMemcpyAsync(p->dls, ls.data(), sizeof(double) * ls.size(), cudaMemcpyHostToDevice, st));
    k_typed_x<<<(n + 127) / 128, 128, 0, st>>>(n, p->dM, p->dbase, p->den64, p->dTr64, p->dX64);
    CF_CUDA(p, cudaGetLastError());
    CF_CUDA(p, cudaStreamSynchronize(st));  // the host arrays go out of scope
    (void)pb;
    return CF_OK;
  }
  if (lw) CF_CUDA(p, cudaMemcpyAsync(p->dlw, lw, sizeof(double) * (size_t)m * 6, cudaMemcpyHostToDevice, st));
  else CF_CUDA(p, cudaMemsetAsync(p->dlw, 0, sizeof(double) * (size_t)m * 6, st));
  if (pb) CF_CUDA(p, cudaMemcpyAsync(p->dpb, pb, sizeof(double) * 61 * 61, cudaMemcpyHostToDevice, st));
  else CF_CUDA(p, cudaMemsetAsync(p->dpb, 0, sizeof(double) * 61 * 61, st));
  CF_CUDA(p, cudaMemsetAsync(p->dls, 0, sizeof(double) * (size_t)std::max(m - 1, 1), st));
  k_transfers<<<(n + 127) / 128, 128, 0, st>>>(n, p->dM, p->dbase, p->dcid, p->den64, p->dlw, p->dpb, p->dTr64,
                                               p->dX64, p->du0, p->dls);
  CF_CUDA(p, cudaGetLastError());
  return CF_OK;
}

cf_status check_weights(cf_problem *p, int m, const double *lw, const double *pb) {
  if (lw)
    for (size_t k = 0; k < (size_t)m * 6; k++)
      if (!std::isfinite(lw[k])) return fail(p, CF_EINVAL, "non-finite codon weight");
  if (pb)
    for (size_t k = 0; k < 61 * 61; k++)
      if (!std::isfinite(pb[k])) return fail(p, CF_EINVAL, "non-finite pair bonus");
  return CF_OK;
}

// Zero every table of a precision (a new protein of the same length reuses
// them: the kernels leave the padding of a block beyond the codon-state
// counts untouched, so it must not keep the previous protein's values).
template <typename T>
cf_status clear_tables(cf_problem *p, PrecTables<T> &t) {
  const int n = p->n;
  const size_t nc = ncells(n) * BLK;
  cudaStream_t st = p->stream;
  DP<T> &d = t.dp;
  if (t.inside_alloc) {
    T *tabs[] = {d.CH, d.QB, d.XI, d.HB, d.QMpp, d.QMpu, d.G, d.QM2pp, d.QM2pu, d.QM2up, d.QM2uu};
    for (T *q : tabs) CF_CUDA(p, cudaMemsetAsync(q, 0, nc * sizeof(T), st));
    CF_CUDA(p, cudaMemsetAsync(d.YY, 0, yy_inside_elems(n, d.yyck) * sizeof(T), st));
    if (d.YYck) CF_CUDA(p, cudaMemsetAsync(d.YYck, 0, yy_ck_elems(n) * sizeof(T), st));
    if (d.YYb) CF_CUDA(p, cudaMemsetAsync(d.YYb, 0, yy_block_elems(n) * sizeof(T), st));
    T *ext[] = {d.Q5U, d.Q5P, d.Gx};
    for (T *q : ext) CF_CUDA(p, cudaMemsetAsync(q, 0, (size_t)n * BLK * sizeof(T), st));
  }
  if (t.outside_alloc) {
    T *tabs[] = {d.hCH, d.hQB, d.hGc, d.hXI, d.hHB, d.hQMpp, d.hQMpu, d.hG, d.hQM2pp, d.hQM2pu, d.hQM2up, d.hQM2uu};
    for (T *q : tabs) CF_CUDA(p, cudaMemsetAsync(q, 0, nc * sizeof(T), st));
    CF_CUDA(p, cudaMemsetAsync(d.hYY, 0, (size_t)YRING * n * NYY * BLK * sizeof(T), st));
    T *ext[] = {d.hQ5U, d.hQ5P, d.hGx};
    for (T *q : ext) CF_CUDA(p, cudaMemsetAsync(q, 0, (size_t)n * BLK * sizeof(T), st));
  }
  return CF_OK;
}

template <typename T>
cf_status upload_transfers(cf_problem *p, PrecTables<T> &t) {
  if (!t.inside_alloc) return CF_OK;  // cast when the tables are first made
  const int n = p->n;
  k_cast<T><<<148, 256, 0, p->stream>>>(p->dTr64, (T *)t.dp.Tr, (size_t)n * BLK);
  k_cast<T><<<148, 256, 0, p->stream>>>(p->dX64, (T *)t.dp.X, (size_t)n * 4 * BLK);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaStreamSynchronize(p->stream));
  return CF_OK;
}

// ---- minimum free energy (min-sum recursions on integer costs)

// cost of an energy in kcal/mol on the 2^-32 kcal/mol grid, rounded half away
// from zero (the rounding every implementation of the model applies once per
// elementary term)
long long qcost(double e) { return std::llround(e * 4294967296.0); }

cf_status mfe_alloc(cf_problem *p) {
  MfeTables &t = p->mfe;
  if (t.alloc) return CF_OK;
  const int n = p->n;
  const size_t nc = ncells(n) * BLK;
  MfeDP &d = t.dp;
  d.n = n;
  d.m = p->m;
  d.Mp = p->dM;
  d.base = p->dbase;
  d.cid = p->dcid;
  d.err = p->derr;
  auto &L = t.allocs;
  mq *tau, *chi, *en, *hq, *u0;
  CF_CUDA(p, dalloc(L, &tau, (size_t)n * BLK));
  CF_CUDA(p, dalloc(L, &chi, (size_t)n * 4 * BLK));
  CF_CUDA(p, dalloc(L, &en, (size_t)EN_N));
  CF_CUDA(p, dalloc(L, &hq, (size_t)n + 2));
  CF_CUDA(p, dalloc(L, &u0, (size_t)NS));
  d.tau = tau;
  d.chi = chi;
  d.en = en;
  d.hq = hq;
  d.u0 = u0;
  mq **tabs[] = {&d.CH, &d.QB, &d.XI, &d.QMP, &d.QMU, &d.GP, &d.BP, &d.M2PU, &d.M2UP, &d.M2UU};
  for (mq **q : tabs) CF_CUDA(p, dalloc(L, q, nc));
  CF_CUDA(p, dalloc(L, &d.W, (size_t)3 * n * MW * BLK));
  CF_CUDA(p, dalloc(L, &d.R, (size_t)3 * n * MRF * BLK));
  CF_CUDA(p, dalloc(L, &d.F, (size_t)3 * n * MRF * BLK));
  mq **ext[] = {&d.Q5U, &d.Q5P, &d.GX, &d.X5};
  for (mq **q : ext) CF_CUDA(p, dalloc(L, q, (size_t)n * BLK));
  CF_CUDA(p, dalloc(L, &d.best, (size_t)1));
  CF_CUDA(p, dalloc(L, &t.stack, (size_t)4 * n + 64));
  CF_CUDA(p, dalloc(L, &t.state, (size_t)n));
  CF_CUDA(p, dalloc(L, &t.codons, (size_t)p->m));
  CF_CUDA(p, dalloc(L, &t.partner, (size_t)n));
  // every table starts "infinite" (byte pattern 0x10 = MQINF); entries the
  // pass never writes (bifurcations of short diagonals) keep that value
  for (mq **q : tabs) CF_CUDA(p, cudaMemset(*q, 0x10, nc * sizeof(mq)));
  for (mq **q : ext) CF_CUDA(p, cudaMemset(*q, 0x10, (size_t)n * BLK * sizeof(mq)));
  // model costs: the energy-factor layout with each term as an integer cost
  const double *pr = p->model->params;
  std::vector<mq> ec(EN_N, 0), hc((size_t)n + 2, 0);
  for (int k = 0; k < 36; k++) ec[EN_STK + k] = qcost(pr[k]);
  for (int l = 0; l <= MAXLOOP; l++) {
    ec[EN_BU + l] = qcost(pr[67 + l]);
    ec[EN_IN + l] = qcost(pr[98 + l]);
  }
  for (int k = 0; k < 16; k++) {
    ec[EN_TM + k] = qcost(pr[129 + k]);
    ec[EN_D5 + k] = qcost(pr[145 + k]);
    ec[EN_D3 + k] = qcost(pr[161 + k]);
  }
  ec[EN_EA] = qcost(pr[177]);
  ec[EN_EB] = qcost(pr[178]);
  ec[EN_EC] = qcost(pr[179]);
  const double H30 = pr[36 + MAXLOOP];
  for (int l = 0; l < n + 2; l++)
    hc[l] = l <= MAXLOOP ? qcost(pr[36 + l]) : qcost(H30 + 1.07856 * std::log((double)l / MAXLOOP));
  CF_CUDA(p, cudaMemcpy(en, ec.data(), sizeof(mq) * EN_N, cudaMemcpyHostToDevice));
  CF_CUDA(p, cudaMemcpy(hq, hc.data(), sizeof(mq) * hc.size(), cudaMemcpyHostToDevice));
  t.alloc = true;
  return CF_OK;
}

// The pass as one CUDA graph: a chain of light kernels, one per diagonal
// (consecutive ones joined by programmatic edges), and the bifurcation kernel
// of diagonal d hanging off the light kernel of d - 4.
cf_status mfe_graph(cf_problem *p) {
  MfeTables &t = p->mfe;
  if (t.g) return CF_OK;
  const int n = p->n;
  cudaGraph_t g;
  CF_CUDA(p, cudaGraphCreate(&g, 0));
  std::vector<cudaGraphNode_t> kl(n), kb(n);
  MfeDP dp = t.dp;
  cudaError_t e = cudaSuccess;
  int nodes = 0;
  const int slots = offchain_ctas(p, 2);  // two bifurcation CTAs per SM
  for (int d = 0; d < n && e == cudaSuccess; d++) {
    int dd = d;
    void *args[] = {&dp, &dd};
    if (d >= 8) {
      // warps per cell: more on the long diagonals, until the launch fills
      // the SMs or a warp would have fewer than 32 split points
      const int cells = n - d + 1;
      int wpc = 1;
      while (wpc < 8 && (long long)cells * wpc < 8LL * slots && 64 * wpc <= d - 8) wpc *= 2;
      int wp = wpc;
      void *bargs[] = {&dp, &dd, &wp};
      cudaKernelNodeParams kp = {};
      kp.func = n <= MFE_BIF2_MAXN ? (void *)k_mfe_bif<2> : (void *)k_mfe_bif<1>;
      kp.gridDim = dim3((cells + 8 / wpc - 1) / (8 / wpc));
      kp.blockDim = dim3(256);
      kp.kernelParams = bargs;
      e = cudaGraphAddKernelNode(&kb[d], g, &kl[d - 4], 1, &kp);
      if (e == cudaSuccess) e = set_priority(kb[d], false);
      nodes++;
    }
    if (e != cudaSuccess) break;
    cudaGraphNode_t deps[1];
    int nd = 0;
    if (d >= 8) deps[nd++] = kb[d];
    cudaKernelNodeParams kp = {};
    kp.func = n <= MFE_BIF2_MAXN ? (void *)k_mfe_light<5> : (void *)k_mfe_light<4>;
    kp.gridDim = dim3(n - d);
    kp.blockDim = dim3(MFE_NT);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&kl[d], g, deps, nd, &kp);
    if (e == cudaSuccess && d > 0) e = add_programmatic_edge(g, kl[d - 1], kl[d]);  // the chain
    if (e == cudaSuccess) e = set_priority(kl[d], true);
    nodes++;
  }
  if (e == cudaSuccess) {
    void *args[] = {&dp};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_mfe_final;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    cudaGraphNode_t fin;
    e = cudaGraphAddKernelNode(&fin, g, &kl[n - 1], 1, &kp);
    nodes++;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&t.g, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(p, e, "mfe graph");
  t.nodes = nodes;
  return CF_OK;
}

cf_status run_mfe(cf_problem *p, int64_t *cost, double *kcal, int32_t *codons, int32_t *partner) {
  const int kc = ptr_kind(codons, p->device), kp = ptr_kind(partner, p->device);
  if (kc < 0 || kp < 0) return fail(p, CF_EINVAL, "cf_mfe: output is device memory of another device");
  cf_status s = mfe_alloc(p);
  if (s != CF_OK) {
    free_mfe(p->mfe);
    return s;
  }
  s = mfe_graph(p);
  if (s != CF_OK) return s;
  MfeTables &t = p->mfe;
  cudaStream_t st = p->stream;
  const int n = p->n, m = p->m;
  CF_CUDA(p, cudaMemsetAsync(p->derr, 0, sizeof(int), st));
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  // the transfer costs of the current weights (cf_set_weights may have changed them)
  k_mfe_transfers<<<(n + 127) / 128, 128, 0, st>>>(n, p->dM, p->dbase, p->dcid, t.dp.en, p->model->kT, p->dlw,
                                                    p->dpb, (mq *)t.dp.tau, (mq *)t.dp.chi, (mq *)t.dp.u0,
                                                    p->layout == 1 ? p->dsmap : nullptr, p->layout == 1 ? p->dsc1 : nullptr);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaGraphLaunch(t.g, st));
  const bool trace = codons || partner;
  if (trace) {
    MfeTrace tr;
    tr.p = t.dp;
    tr.stack = t.stack;
    tr.cap = 4 * n + 64;
    tr.state = t.state;
    tr.codons = kc > 0 ? codons : t.codons;
    tr.partner = kp > 0 ? partner : t.partner;
    tr.sctab = p->layout == 1 ? p->dsctab : nullptr;
    k_mfe_trace<<<1, 256, 0, st>>>(tr);
    CF_CUDA(p, cudaGetLastError());
  }
  CF_CUDA(p, cudaEventRecord(p->ev[1], st));
  long long q = 0;
  int err = 0;
  CF_CUDA(p, cudaMemcpyAsync(&q, t.dp.best, sizeof(q), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaMemcpyAsync(&err, p->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (codons && kc == 0)
    CF_CUDA(p, cudaMemcpyAsync(codons, t.codons, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, st));
  if (partner && kp == 0)
    CF_CUDA(p, cudaMemcpyAsync(partner, t.partner, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  CF_CUDA(p, cudaEventElapsedTime(&p->t_mfe, p->ev[0], p->ev[1]));
  if (q >= MQHALF) return fail(p, CF_ENUMERIC, "cf_mfe: no configuration has a finite cost");
  if (err) return fail(p, CF_ENUMERIC, "cf_mfe: traceback inconsistency (error word " + std::to_string(err) + ")");
  if (cost) *cost = q;
  if (kcal) *kcal = (double)q / 4294967296.0;
  return CF_OK;
}

// Every configuration within `gap` (integer cost) of the minimum, depth first
// (cf_subopt.cuh): the MFE tables first, then one CTA enumerates.
cf_status run_subopt(cf_problem *p, long long gap, int max_out, long long *cost, int32_t *codons, int32_t *partner,
                     int *count) {
  cf_status s = mfe_alloc(p);
  if (s != CF_OK) {
    free_mfe(p->mfe);
    return s;
  }
  s = mfe_graph(p);
  if (s != CF_OK) return s;
  MfeTables &t = p->mfe;
  cudaStream_t st = p->stream;
  const int n = p->n, m = p->m;
  CF_CUDA(p, cudaMemsetAsync(p->derr, 0, sizeof(int), st));
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  k_mfe_transfers<<<(n + 127) / 128, 128, 0, st>>>(n, p->dM, p->dbase, p->dcid, t.dp.en, p->model->kT, p->dlw,
                                                    p->dpb, (mq *)t.dp.tau, (mq *)t.dp.chi, (mq *)t.dp.u0,
                                                    p->layout == 1 ? p->dsmap : nullptr, p->layout == 1 ? p->dsc1 : nullptr);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaGraphLaunch(t.g, st));
  SubArgs a;
  a.p = t.dp;
  a.sctab = p->layout == 1 ? p->dsctab : nullptr;
  a.gap = gap;
  a.max_out = max_out;
  a.pcap = 4 * n + 64;
  a.depth_cap = 4 * n + 64;
  a.max_steps = 50000000ll;
  a.max_ns = 30ull * 1000000000ull;  // 30 s
  std::vector<void *> tmp;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    free_list(tmp);
  };
  cudaError_t e = dalloc(tmp, &a.frames, (size_t)a.depth_cap);
  if (e == cudaSuccess) e = dalloc(tmp, &a.pend, (size_t)a.pcap);
  if (e == cudaSuccess) e = dalloc(tmp, &a.pendw, (size_t)a.pcap);
  if (e == cudaSuccess) e = dalloc(tmp, &a.codons, (size_t)std::max(max_out, 1) * m);
  if (e == cudaSuccess) e = dalloc(tmp, &a.partner, (size_t)std::max(max_out, 1) * n);
  if (e == cudaSuccess) e = dalloc(tmp, &a.cost, (size_t)std::max(max_out, 1));
  if (e == cudaSuccess) e = dalloc(tmp, &a.count, (size_t)2);
  const size_t nc = ncells(n);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.QB, nc);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.CH, nc);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.XI, nc);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.GP, nc);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.tau, (size_t)n);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.chie, (size_t)n);
  if (e == cudaSuccess) e = dalloc(tmp, &a.mn.q5, (size_t)n * NS);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(p, e, "cf_subopt: scratch");
  }
  k_sub_mins<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(t.dp, a.mn);
  e = cudaGetLastError();
  const size_t ssm = sub_smem(n);  // the states and partners, the frame ring
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void *)k_mfe_subopt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
  if (e == cudaSuccess) k_mfe_subopt<<<1, SUB_NT, ssm, st>>>(a);
  if (e == cudaSuccess) e = cudaGetLastError();
  long long cnt[2] = {0, 0};
  int err = 0;
  long long best = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, a.count, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p->derr, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&best, t.dp.best, sizeof(best), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const long long nw = std::min<long long>(cnt[0], max_out);
  if (e == cudaSuccess && nw > 0) {
    if (cost) e = cudaMemcpy(cost, a.cost, sizeof(long long) * nw, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && codons) e = cudaMemcpy(codons, a.codons, sizeof(int32_t) * nw * m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && partner)
      e = cudaMemcpy(partner, a.partner, sizeof(int32_t) * nw * n, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) e = cudaEventRecord(p->ev[1], st);
  if (e == cudaSuccess) e = cudaEventSynchronize(p->ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&p->t_mfe, p->ev[0], p->ev[1]);
  release();
  if (e != cudaSuccess) return cuda_fail(p, e, "cf_subopt");
  if (best >= MQHALF) return fail(p, CF_ENUMERIC, "cf_subopt: no configuration has a finite cost");
  if (err) return fail(p, CF_ENUMERIC, "cf_subopt: enumeration inconsistency (error word " + std::to_string(err) + ")");
  *count = (int)std::min<long long>(cnt[0], (long long)max_out + 1);
  p->sub_steps = cnt[1];
  return CF_OK;
}

// ---- batched fixed-sequence windows

cf_status window_tables(cf_problem *p) {
  if (p->win_en) return CF_OK;
  std::vector<float> en(p->model->en, p->model->en + EN_N), ehl(WMAXN + 2);
  const double kT = p->model->kT, H30 = p->model->params[36 + MAXLOOP];
  for (int L = 0; L < WMAXN + 2; L++) {
    double e = (L <= MAXLOOP) ? p->model->params[36 + L] : H30 + 1.07856 * std::log((double)L / MAXLOOP);
    ehl[L] = (float)std::exp(-e / kT);
  }
  CF_CUDA(p, dalloc(p->win_allocs, &p->win_en, (size_t)EN_N));
  CF_CUDA(p, dalloc(p->win_allocs, &p->win_ehl, (size_t)WMAXN + 2));
  CF_CUDA(p, dalloc(p->win_allocs, &p->win_err, (size_t)1));
  CF_CUDA(p, cudaMemcpy(p->win_en, en.data(), sizeof(float) * EN_N, cudaMemcpyHostToDevice));
  CF_CUDA(p, cudaMemcpy(p->win_ehl, ehl.data(), sizeof(float) * ehl.size(), cudaMemcpyHostToDevice));
  return CF_OK;
}

cf_status run_windows(cf_problem *p, const uint8_t *bases, const int64_t *offsets, int nwin, double *logz) {
  cf_status s = window_tables(p);
  if (s != CF_OK) return s;
  cudaStream_t st = p->stream;
  const int ko = ptr_kind(offsets, p->device), kb = ptr_kind(bases, p->device), kl = ptr_kind(logz, p->device);
  if (ko < 0 || kb < 0 || kl < 0)
    return fail(p, CF_EINVAL, "cf_window_logz: a buffer is device memory of another device");
  const bool off_dev = ko > 0, bases_dev = kb > 0, out_dev = kl > 0;
  std::vector<int64_t> off((size_t)nwin + 1);
  if (off_dev) {
    CF_CUDA(p, cudaMemcpyAsync(off.data(), offsets, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost, st));
    CF_CUDA(p, cudaStreamSynchronize(st));
  } else {
    std::memcpy(off.data(), offsets, sizeof(int64_t) * off.size());
  }
  int nmax = 0;
  if (off[0] < 0) return fail(p, CF_EINVAL, "cf_window_logz: offsets[0] < 0");
  for (int w = 0; w < nwin; w++) {
    const int64_t len = off[w + 1] - off[w];
    if (len < 0) return fail(p, CF_EINVAL, "cf_window_logz: offsets must not decrease");
    if (len > WMAXN)
      return fail(p, CF_EINVAL, "cf_window_logz: window " + std::to_string(w) + " longer than CF_WINDOW_MAX_N");
    nmax = std::max(nmax, (int)len);
  }
  const size_t total = (size_t)off[nwin];
  int dev_sms = 148, per_sm = 1;
  CF_CUDA(p, cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device));
  CF_CUDA(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_window, WT, 0));
  const int grid = std::max(1, std::min(nwin, dev_sms * std::max(per_sm, 1)));
  const size_t stride = (3 * ncells(nmax) + 63) / 64 * 64;
  // buffers grow monotonically and are reused by later calls
  if (p->win_scratch_cap < stride * grid || (!bases_dev && p->win_bases_cap < total) || p->win_nwin_cap < (size_t)nwin + 1) {
    CF_CUDA(p, cudaStreamSynchronize(st));
    free_list(p->win_buf_allocs);
    p->win_scratch_cap = std::max(p->win_scratch_cap, stride * grid);
    p->win_bases_cap = std::max(p->win_bases_cap, bases_dev ? (size_t)16 : std::max(total, (size_t)16));
    p->win_nwin_cap = std::max(p->win_nwin_cap, (size_t)nwin + 1);
    CF_CUDA(p, dalloc(p->win_buf_allocs, &p->win_scratch, p->win_scratch_cap));
    CF_CUDA(p, dalloc(p->win_buf_allocs, &p->win_bases, p->win_bases_cap));
    CF_CUDA(p, dalloc(p->win_buf_allocs, &p->win_off, p->win_nwin_cap));
    CF_CUDA(p, dalloc(p->win_buf_allocs, &p->win_logz, p->win_nwin_cap));
  }
  // host inputs and outputs go through pinned buffers owned by the problem
  // (every call ends with a stream synchronisation, so they are free here)
  const bool host_io = !bases_dev || !off_dev || !out_dev;
  if (host_io && (p->win_hbases_cap < total || p->win_hnwin_cap < (size_t)nwin + 1)) {
    if (p->win_hbases) cudaFreeHost(p->win_hbases);
    if (p->win_hoff) cudaFreeHost(p->win_hoff);
    if (p->win_hlogz) cudaFreeHost(p->win_hlogz);
    p->win_hbases = nullptr;
    p->win_hoff = nullptr;
    p->win_hlogz = nullptr;
    p->win_hbases_cap = std::max(p->win_hbases_cap, std::max(total, (size_t)16));
    p->win_hnwin_cap = std::max(p->win_hnwin_cap, (size_t)nwin + 1);
    CF_CUDA(p, cudaHostAlloc((void **)&p->win_hbases, p->win_hbases_cap, cudaHostAllocDefault));
    CF_CUDA(p, cudaHostAlloc((void **)&p->win_hoff, p->win_hnwin_cap * sizeof(int64_t), cudaHostAllocDefault));
    CF_CUDA(p, cudaHostAlloc((void **)&p->win_hlogz, p->win_hnwin_cap * sizeof(double), cudaHostAllocDefault));
  }
  WinArgs a;
  a.bases = bases;
  if (!bases_dev) {
    std::memcpy(p->win_hbases, bases, total);
    CF_CUDA(p, cudaMemcpyAsync(p->win_bases, p->win_hbases, total, cudaMemcpyHostToDevice, st));
    a.bases = p->win_bases;
  }
  a.off = offsets;
  if (!off_dev) {
    std::memcpy(p->win_hoff, off.data(), sizeof(int64_t) * off.size());
    CF_CUDA(p, cudaMemcpyAsync(p->win_off, p->win_hoff, sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st));
    a.off = p->win_off;
  }
  a.nwin = nwin;
  a.en = p->win_en;
  a.eHL = p->win_ehl;
  a.log2eb = (float)std::log2(p->model->en[EN_EB]);
  a.scratch = p->win_scratch;
  a.stride = stride;
  a.logz = out_dev ? logz : p->win_logz;
  a.err = p->win_err;
  CF_CUDA(p, cudaMemsetAsync(p->win_err, 0, sizeof(int), st));
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  k_window<<<grid, WT, 0, st>>>(a);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaEventRecord(p->ev[1], st));
  if (!out_dev)
    CF_CUDA(p, cudaMemcpyAsync(p->win_hlogz, p->win_logz, sizeof(double) * nwin, cudaMemcpyDeviceToHost, st));
  int err = 0;
  CF_CUDA(p, cudaMemcpyAsync(&err, p->win_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  if (!out_dev) std::memcpy(logz, p->win_hlogz, sizeof(double) * nwin);
  CF_CUDA(p, cudaEventElapsedTime(&p->t_win, p->ev[0], p->ev[1]));
  if (err & 1) return fail(p, CF_EINVAL, "cf_window_logz: base code outside 0..3");
  if (err & 2) return fail(p, CF_ENUMERIC, "cf_window_logz: non-finite table entry after scaling");
  return CF_OK;
}

}  // namespace

namespace cf {
// error text for calls without a problem handle (read by cf_last_error(NULL))
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace cf

// ------------------------------------------------------------------ C ABI

extern "C" {

cf_status cf_load_model(const double *params, size_t nparams, cf_model **out) {
  if (!params || !out) return fail(nullptr, CF_EINVAL, "cf_load_model: NULL argument");
  if (nparams != CF_NPARAMS) return fail(nullptr, CF_EINVAL, "cf_load_model: expected 181 parameters");
  for (size_t k = 0; k < nparams; k++)
    if (!std::isfinite(params[k])) return fail(nullptr, CF_EINVAL, "cf_load_model: non-finite parameter");
  cf_model *m = new (std::nothrow) cf_model;
  if (!m) return fail(nullptr, CF_ENOMEM, "cf_load_model: out of host memory");
  std::memcpy(m->params, params, sizeof(m->params));
  m->kT = 1.98717e-3 * (params[180] + 273.15);
  auto bz = [&](double e) { return std::exp(-e / m->kT); };
  for (int k = 0; k < 36; k++) m->en[EN_STK + k] = bz(params[k]);
  for (int L = 0; L <= MAXLOOP; L++) {
    m->en[EN_BU + L] = bz(params[67 + L]);
    m->en[EN_IN + L] = bz(params[98 + L]);
  }
  for (int k = 0; k < 16; k++) {
    m->en[EN_TM + k] = bz(params[129 + k]);
    m->en[EN_D5 + k] = bz(params[145 + k]);
    m->en[EN_D3 + k] = bz(params[161 + k]);
  }
  m->en[EN_EA] = bz(params[177]);
  m->en[EN_EB] = bz(params[178]);
  m->en[EN_EC] = bz(params[179]);
  *out = m;
  return CF_OK;
}

cf_status cf_model_free(cf_model *model) {
  delete model;
  return CF_OK;
}

cf_status cf_problem_create(const cf_model *model, int device, void *stream, cf_problem **out) {
  if (!model || !out) return fail(nullptr, CF_EINVAL, "cf_problem_create: NULL argument");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
  cf_problem *p = new (std::nothrow) cf_problem;
  if (!p) return fail(nullptr, CF_ENOMEM, "cf_problem_create: out of host memory");
  p->model = model;
  p->device = device;
  p->stream = (cudaStream_t)stream;
  for (auto &ev : p->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(nullptr, e, "cudaEventCreate");
    }
  }
  *out = p;
  return CF_OK;
}

extern "C++" {
template <typename T>
static void free_tm(TmTables<T> &t) {
  if (t.g) cudaGraphExecDestroy(t.g);
  t = TmTables<T>();
}
}

static void release_protein(cf_problem *p) {
  free_prec(p->f32);
  free_prec(p->f64);
  free_mfe(p->mfe);
  free_tm(p->tm32);
  free_tm(p->tm64);
  free_list(p->tm_allocs);
  free_list(p->shared_allocs);
  free_list(p->smp_allocs);
  p->smp_cap = 0;
  p->dM = p->dbase = p->dbnd = p->dE = p->derr = nullptr;
  p->ddmax = nullptr;
  p->du0 = p->dZm = p->dtrans = p->dp0 = nullptr;
  p->dcm = p->dbm = p->dpg = nullptr;
  p->dcid = nullptr;
  p->dsmap = p->dsctab = p->dsc1 = nullptr;
  p->dlw = p->dpb = p->dTr64 = p->dX64 = p->den64 = p->dls = p->dlogz = nullptr;
  p->dP = nullptr;
  p->have_inside = false;
  p->n = p->m = 0;
}

cf_status cf_problem_free(cf_problem *p) {
  if (!p) return CF_OK;
  cudaSetDevice(p->device);
  release_protein(p);
  free_list(p->win_allocs);
  free_list(p->win_buf_allocs);
  if (p->win_hbases) cudaFreeHost(p->win_hbases);
  if (p->win_hoff) cudaFreeHost(p->win_hoff);
  if (p->win_hlogz) cudaFreeHost(p->win_hlogz);
  for (auto &ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  delete p;
  return CF_OK;
}

static cf_status set_protein_tables(cf_problem *p, const std::vector<int> &res, const double *lw,
                                    const double *pb);

cf_status cf_set_protein(cf_problem *p, const char *aa, int m, const double *lw, const double *pb) {
  CfRange nvtx_range("cf_set_protein");
  if (!p || !aa) return fail(p, CF_EINVAL, "cf_set_protein: NULL argument");
  if (m < 1) return fail(p, CF_EINVAL, "cf_set_protein: m must be >= 1");
  std::vector<int> res(m);
  for (int r = 0; r < m; r++) {
    const char *q = std::strchr(kAminoAcids, aa[r]);
    if (!aa[r] || !q) return fail(p, CF_EINVAL, std::string("cf_set_protein: invalid amino acid at residue ") + std::to_string(r));
    res[r] = (int)(q - kAminoAcids);
  }
  if (check_weights(p, m, lw, pb) != CF_OK) return fail(p, CF_EINVAL, "cf_set_protein: " + p->err);
  if (pb && p->layout_req == 1)
    return fail(p, CF_EINVAL, "cf_set_protein: the single-codon layout has no codon-pair bonuses");
  CF_CUDA(p, cudaSetDevice(p->device));
  // past validation the old protein is gone: a failure below (an allocation
  // that does not fit, a CUDA error) releases everything, so that the problem
  // is empty and usable (the next cf_set_protein starts from scratch)
  const cf_status s = set_protein_tables(p, res, lw, pb);
  if (s != CF_OK) {
    cudaStreamSynchronize(p->stream);
    cudaGetLastError();
    release_protein(p);
  }
  return s;
}

static cf_status set_protein_tables(cf_problem *p, const std::vector<int> &res, const double *lw,
                                    const double *pb) {
  const int m = (int)res.size();
  const GeneticCode &gc = gcode();
  // a protein of the same length reuses the device tables and the pass graphs
  // (they depend on the length only): no allocation, no device-wide sync
  const bool reuse = p->n == 3 * m && p->dM != nullptr && p->layout == p->layout_req;
  if (reuse) {
    CF_CUDA(p, cudaStreamSynchronize(p->stream));  // no pass may still read the old protein
    p->have_inside = false;
  } else {
    release_protein(p);
  }
  const int n = 3 * m;
  p->n = n;
  p->m = m;
  p->layout = p->layout_req;
  p->M.assign(n, 0);
  p->base.assign((size_t)n * NS, 0);
  p->cid.assign((size_t)n * NS, -1);
  p->bnd.assign(n, 0);
  p->smap.assign((size_t)m * 6, -1);
  p->sc1.assign((size_t)n * NS, -1);
  p->sctab.assign((size_t)m * BLK, -1);
  for (int r = 0; r < m; r++) {
    const auto &cods = gc.codons[res[r]];
    if (p->layout == 0) {
      for (int off = 0; off < 3; off++) {
        int q = 3 * r + off;
        p->M[q] = (int)cods.size();
        for (size_t a = 0; a < cods.size(); a++) {
          p->base[(size_t)q * NS + a] = (cods[a] >> (2 * (2 - off))) & 3;
          p->cid[(size_t)q * NS + a] = gc.sense_id[cods[a]];
        }
        p->bnd[q] = (off == 2 && q + 1 < n) ? 1 : 0;  // T_q crosses into residue r+1
      }
    } else {
      // single-codon layout (Eq. single-tt): the states of the first position
      // are the distinct first bases, of the second the distinct (first,
      // second) base pairs, of the third the distinct third bases, in
      // ascending order; the codon is fixed by the transfer 3r+1 -> 3r+2.
      // A position state must fix its base (the loop energies read it), so
      // each position has at least as many states as distinct bases; the
      // (first, second) pair never has more states than the (second, third)
      // pair under the standard code (serine: 2 against 6)
      std::vector<int> f, pr, l;
      for (int c : cods) {
        f.push_back(c >> 4 & 3);
        pr.push_back(c >> 2 & 15);
        l.push_back(c & 3);
      }
      auto uniq = [](std::vector<int> v) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        return v;
      };
      const std::vector<int> F = uniq(f), PR = uniq(pr), L = uniq(l);
      const int q = 3 * r;
      p->M[q] = (int)F.size();
      p->M[q + 1] = (int)PR.size();
      p->M[q + 2] = (int)L.size();
      for (size_t a = 0; a < F.size(); a++) p->base[(size_t)q * NS + a] = F[a];
      for (size_t a = 0; a < PR.size(); a++) {
        p->base[(size_t)(q + 1) * NS + a] = PR[a] & 3;
        p->sc1[(size_t)(q + 1) * NS + a] = PR[a] >> 2;
      }
      for (size_t a = 0; a < L.size(); a++) p->base[(size_t)(q + 2) * NS + a] = L[a];
      p->bnd[q + 1] = 1;  // T_{q+1} carries the codon and its weight
      for (size_t s2 = 0; s2 < cods.size(); s2++) {
        const int c = cods[s2];
        const int a = (int)(std::lower_bound(PR.begin(), PR.end(), c >> 2 & 15) - PR.begin());
        const int b = (int)(std::lower_bound(L.begin(), L.end(), c & 3) - L.begin());
        p->smap[(size_t)r * 6 + s2] = a | (b << 4) | ((c >> 4 & 3) << 8) | ((c >> 2 & 3) << 10) | ((c & 3) << 12);
        const int a0 = (int)(std::lower_bound(F.begin(), F.end(), c >> 4 & 3) - F.begin());
        p->sctab[(size_t)r * BLK + a * NS + b] = gc.sense_id[c] | (a0 << 8);
      }
    }
  }
  p->nls = p->layout == 0 ? m - 1 : m;
  p->eHL.assign((size_t)n + 2, 0.0);
  const double kT = p->model->kT, H30 = p->model->params[36 + MAXLOOP];
  for (int L = 0; L < n + 2; L++) {
    double e = (L <= MAXLOOP) ? p->model->params[36 + L] : H30 + 1.07856 * std::log((double)L / MAXLOOP);
    p->eHL[L] = std::exp(-e / kT);
  }
  if (!reuse) {
    auto &S = p->shared_allocs;
    CF_CUDA(p, dalloc(S, &p->dM, (size_t)n));
    CF_CUDA(p, dalloc(S, &p->dbase, (size_t)n * NS));
    CF_CUDA(p, dalloc(S, &p->dbnd, (size_t)n));
    CF_CUDA(p, dalloc(S, &p->dE, (size_t)n));
    CF_CUDA(p, dalloc(S, &p->derr, (size_t)1));
    CF_CUDA(p, dalloc(S, &p->ddmax, (size_t)n));
    CF_CUDA(p, dalloc(S, &p->du0, (size_t)NS));
    CF_CUDA(p, dalloc(S, &p->dZm, (size_t)1));
    CF_CUDA(p, dalloc(S, &p->dtrans, (size_t)std::max(m - 1, 1) * BLK));
    CF_CUDA(p, dalloc(S, &p->dp0, (size_t)NS));
    CF_CUDA(p, dalloc(S, &p->dP, (size_t)n * n));
    CF_CUDA(p, dalloc(S, &p->dcm, (size_t)m * 6));
    CF_CUDA(p, dalloc(S, &p->dbm, (size_t)n * 4));
    CF_CUDA(p, dalloc(S, &p->dpg, (size_t)61 * 61));
    CF_CUDA(p, dalloc(S, &p->dcid, (size_t)n * NS));
    CF_CUDA(p, dalloc(S, &p->dlw, (size_t)m * 6));
    CF_CUDA(p, dalloc(S, &p->dpb, (size_t)61 * 61));
    CF_CUDA(p, dalloc(S, &p->dTr64, (size_t)n * BLK));
    CF_CUDA(p, dalloc(S, &p->dX64, (size_t)n * 4 * BLK));
    CF_CUDA(p, dalloc(S, &p->den64, (size_t)EN_N));
    CF_CUDA(p, dalloc(S, &p->dls, (size_t)std::max(m, 1)));
    CF_CUDA(p, dalloc(S, &p->dsmap, (size_t)m * 6));
    CF_CUDA(p, dalloc(S, &p->dsctab, (size_t)m * BLK));
    CF_CUDA(p, dalloc(S, &p->dsc1, (size_t)n * NS));
    CF_CUDA(p, dalloc(S, &p->dlogz, (size_t)1));
    CF_CUDA(p, cudaMemcpy(p->den64, p->model->en, sizeof(double) * EN_N, cudaMemcpyHostToDevice));
  }
  cudaStream_t st = p->stream;
  CF_CUDA(p, cudaMemcpyAsync(p->dM, p->M.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dbase, p->base.data(), sizeof(int) * n * NS, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dbnd, p->bnd.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dcid, p->cid.data(), sizeof(int) * n * NS, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dsmap, p->smap.data(), sizeof(int) * m * 6, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dsctab, p->sctab.data(), sizeof(int) * m * BLK, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemcpyAsync(p->dsc1, p->sc1.data(), sizeof(int) * n * NS, cudaMemcpyHostToDevice, st));
  CF_CUDA(p, cudaMemsetAsync(p->dE, 0, sizeof(int) * n, st));
  if (cf_status ts = device_transfers(p, lw, pb); ts != CF_OK) return ts;
  CF_CUDA(p, cudaStreamSynchronize(st));
  if (reuse) {
    // the tables of each precision are cleared by its next inside pass
    p->f32.stale = p->f32.inside_alloc;
    p->f64.stale = p->f64.inside_alloc;
    cf_status s = upload_transfers(p, p->f32);
    if (s == CF_OK) s = upload_transfers(p, p->f64);
    if (s != CF_OK) return s;
  }
  return CF_OK;
}

cf_status cf_set_weights(cf_problem *p, const double *lw, const double *pb) {
  CfRange nvtx_range("cf_set_weights");
  if (!p) return fail(p, CF_EINVAL, "cf_set_weights: NULL problem");
  if (p->n == 0) return fail(p, CF_ESTATE, "cf_set_weights: no protein set");
  if (check_weights(p, p->m, lw, pb) != CF_OK) return fail(p, CF_EINVAL, "cf_set_weights: " + p->err);
  if (pb && p->layout == 1) return fail(p, CF_EINVAL, "cf_set_weights: the single-codon layout has no codon-pair bonuses");
  CF_CUDA(p, cudaSetDevice(p->device));
  CF_CUDA(p, cudaStreamSynchronize(p->stream));  // no pass may still read the old transfers
  p->have_inside = false;
  if (cf_status ts = device_transfers(p, lw, pb); ts != CF_OK) return ts;
  cf_status s = upload_transfers(p, p->f32);
  if (s == CF_OK) s = upload_transfers(p, p->f64);
  if (s != CF_OK) return s;
  CF_CUDA(p, cudaStreamSynchronize(p->stream));
  return CF_OK;
}

cf_status cf_inside(cf_problem *p, cf_precision prec, double *logZ) {
  CfRange nvtx_range("cf_inside");
  if (!p || !logZ) return fail(p, CF_EINVAL, "cf_inside: NULL argument");
  if (p->n == 0) return fail(p, CF_ESTATE, "cf_inside: no protein set");
  if (prec != CF_FP64 && prec != CF_FP32_SCALED) return fail(p, CF_EINVAL, "cf_inside: unknown precision");
  CF_CUDA(p, cudaSetDevice(p->device));
  p->have_inside = false;
  cf_status s = (prec == CF_FP64) ? run_inside(p, p->f64, logZ) : run_inside(p, p->f32, logZ);
  if (s != CF_OK) return s;
  p->last_prec = (int)prec;
  p->have_inside = true;
  return CF_OK;
}

cf_status cf_outside(cf_problem *p, float *pair_prob, double *codon_marg, double *base_marg, double *pair_grad) {
  CfRange nvtx_range("cf_outside");
  if (!p) return fail(p, CF_EINVAL, "cf_outside: NULL problem");
  if (!p->have_inside) return fail(p, CF_ESTATE, "cf_outside: run cf_inside first");
  if (pair_grad && p->layout == 1)
    return fail(p, CF_EINVAL, "cf_outside: no codon-pair gradient in the single-codon layout");
  CF_CUDA(p, cudaSetDevice(p->device));
  cf_status s = (p->last_prec == CF_FP64) ? run_outside(p, p->f64) : run_outside(p, p->f32);
  if (s != CF_OK) return s;
  const int n = p->n, m = p->m;
  cudaStream_t st = p->stream;
  if (pair_prob) {
    s = copy_out(p, pair_prob, p->dP, sizeof(float) * (size_t)n * n, true);
    if (s != CF_OK) return s;
  }
  if (codon_marg) {
    s = copy_out(p, codon_marg, p->dcm, sizeof(double) * (size_t)m * 6, true);
    if (s != CF_OK) return s;
  }
  if (base_marg) {
    s = copy_out(p, base_marg, p->dbm, sizeof(double) * (size_t)n * 4, true);
    if (s != CF_OK) return s;
  }
  if (pair_grad) {
    s = copy_out(p, pair_grad, p->dpg, sizeof(double) * 61 * 61, true);
    if (s != CF_OK) return s;
  }
  int err = 0;
  CF_CUDA(p, cudaMemcpyAsync(&err, p->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  CF_CUDA(p, cudaEventElapsedTime(&p->t_out, p->ev[2], p->ev[3]));
  if (err & ERR_STAGE_TIMEOUT) return fail(p, CF_ETIMEOUT, "outside: a bounded wait for staged inputs gave up");
  if (err & ERR_OUT_NONFINITE) return fail(p, CF_ENUMERIC, "outside: a pair probability or marginal is not finite");
  return CF_OK;
}

cf_status cf_window_logz(cf_problem *p, const uint8_t *bases, const int64_t *offsets, int nwin, double *logz) {
  CfRange nvtx_range("cf_window_logz");
  if (!p) return fail(p, CF_EINVAL, "cf_window_logz: NULL problem");
  if (nwin < 0) return fail(p, CF_EINVAL, "cf_window_logz: nwin < 0");
  if (nwin == 0) return CF_OK;
  if (!bases || !offsets || !logz) return fail(p, CF_EINVAL, "cf_window_logz: NULL argument");
  CF_CUDA(p, cudaSetDevice(p->device));
  return run_windows(p, bases, offsets, nwin, logz);
}

float cf_window_last_ms(const cf_problem *p) { return p ? p->t_win : 0.f; }

cf_status cf_last_timing(const cf_problem *p, float *inside_ms, float *outside_ms, int *inside_launches,
                         int *outside_launches) {
  if (!p) return CF_EINVAL;
  if (inside_ms) *inside_ms = p->t_in;
  if (outside_ms) *outside_ms = p->t_out;
  if (inside_launches) *inside_launches = p->l_in;
  if (outside_launches) *outside_launches = p->l_out;
  return CF_OK;
}

int cf_problem_length(const cf_problem *p) { return p ? p->n : 0; }

const char *cf_last_error(const cf_problem *p) {
  if (p) return p->err.c_str();
  return g_last_error.c_str();
}

cf_status cf_mfe(cf_problem *p, int64_t *cost, double *mfe_kcal, int32_t *codons, int32_t *partner) {
  CfRange nvtx_range("cf_mfe");
  if (!p) return fail(p, CF_EINVAL, "cf_mfe: NULL problem");
  if (p->n == 0) return fail(p, CF_ESTATE, "cf_mfe: no protein set");
  CF_CUDA(p, cudaSetDevice(p->device));
  return run_mfe(p, cost, mfe_kcal, codons, partner);
}

float cf_mfe_last_ms(const cf_problem *p) { return p ? p->t_mfe : 0.f; }
long long cf_subopt_steps(const cf_problem *p) { return p ? p->sub_steps : 0; }

cf_status cf_subopt(cf_problem *p, double gap_kcal, int max_out, int64_t *cost, int32_t *codons, int32_t *partner,
                    int *count) {
  CfRange nvtx_range("cf_subopt");
  if (!p || !count) return fail(p, CF_EINVAL, "cf_subopt: NULL argument");
  if (!(gap_kcal >= 0) || gap_kcal > 1e6 || max_out < 0) return fail(p, CF_EINVAL, "cf_subopt: bad gap or max_out");
  if (p->n == 0) return fail(p, CF_ESTATE, "cf_subopt: no protein set");
  if (ptr_kind(cost, p->device) != 0 || ptr_kind(codons, p->device) != 0 || ptr_kind(partner, p->device) != 0)
    return fail(p, CF_EINVAL, "cf_subopt: outputs must be host memory");
  if (p->n > CF_SUBOPT_MAX_N) return fail(p, CF_EINVAL, "cf_subopt: protein longer than CF_SUBOPT_MAX_N nt");
  CF_CUDA(p, cudaSetDevice(p->device));
  const long long gap = (long long)std::floor(gap_kcal * 4294967296.0);  // on the 2^-32 kcal/mol grid
  return run_subopt(p, gap, max_out, (long long *)cost, codons, partner, count);
}

// ------------------------------------------------------------------ tensor-based model

struct cf_tm_model {
  int device = 0, gamma = 0, nrho = 0;
  TmModelDev *d = nullptr;
  double radius[4] = {0, 0, 0, 0};
};

// Spectral radius by Gelfand's formula r = lim ||A^m||^(1/m) over m = 2^s:
// repeated squaring of A scaled to unit norm (max row sum of |entries|), the
// logarithm of the scale carried separately, 48 squarings.
cf_status cf_tm_spectral_radius(const double *A, int dim, double *radius) {
  if (!A || !radius || dim < 1 || dim > 64) return fail(nullptr, CF_EINVAL, "cf_tm_spectral_radius: bad argument");
  std::vector<double> M(A, A + (size_t)dim * dim), P((size_t)dim * dim);
  for (double v : M)
    if (!std::isfinite(v)) return fail(nullptr, CF_EINVAL, "cf_tm_spectral_radius: non-finite entry");
  auto norm = [&](const std::vector<double> &X) {
    double m = 0;
    for (int i = 0; i < dim; i++) {
      double s = 0;
      for (int j = 0; j < dim; j++) s += std::fabs(X[(size_t)i * dim + j]);
      m = std::max(m, s);
    }
    return m;
  };
  double nrm = norm(M);
  if (nrm == 0) {
    *radius = 0;
    return CF_OK;
  }
  for (double &v : M) v /= nrm;
  double logc = std::log(nrm);  // log of ||A^(2^s)|| as (scale) * ||M|| with ||M|| = 1
  double m = 1;                 // 2^s
  for (int s = 0; s < 48; s++) {
    for (int i = 0; i < dim; i++)
      for (int j = 0; j < dim; j++) {
        double acc = 0;
        for (int k = 0; k < dim; k++) acc += M[(size_t)i * dim + k] * M[(size_t)k * dim + j];
        P[(size_t)i * dim + j] = acc;
      }
    const double np = norm(P);
    if (np == 0) {
      *radius = 0;
      return CF_OK;
    }
    for (size_t q = 0; q < P.size(); q++) M[q] = P[q] / np;
    logc = 2 * logc + std::log(np);
    m *= 2;
  }
  *radius = std::exp(logc / m);
  return CF_OK;
}

cf_status cf_tm_model_create(int device, int gamma, int nrho, const double *V, const double *B, const double *S,
                             int normalize, cf_tm_model **out) {
  if (!out || !V || !B || !S || gamma < 1 || gamma > TM_G || nrho < 1 || nrho > TM_R)
    return fail(nullptr, CF_EINVAL, "cf_tm_model_create: bad argument (1 <= gamma <= 4, 1 <= nrho <= 4)");
  *out = nullptr;
  const size_t g2 = (size_t)gamma * gamma;
  for (size_t q = 0; q < 4 * g2; q++)
    if (!std::isfinite(V[q])) return fail(nullptr, CF_EINVAL, "cf_tm_model_create: non-finite V");
  for (size_t q = 0; q < (size_t)nrho * 16 * g2; q++)
    if (!std::isfinite(B[q])) return fail(nullptr, CF_EINVAL, "cf_tm_model_create: non-finite B");
  for (size_t q = 0; q < g2; q++)
    if (!std::isfinite(S[q])) return fail(nullptr, CF_EINVAL, "cf_tm_model_create: non-finite S");
  cf_tm_model *m = new (std::nothrow) cf_tm_model;
  if (!m) return fail(nullptr, CF_ENOMEM, "cf_tm_model_create: host memory");
  m->device = device;
  m->gamma = gamma;
  m->nrho = nrho;
  double r[4] = {1, 1, 1, 1};
  if (normalize)
    for (int x = 0; x < 4; x++) {
      cf_status st = cf_tm_spectral_radius(V + x * g2, gamma, &r[x]);
      if (st != CF_OK || !(r[x] > 0)) {
        delete m;
        return fail(nullptr, CF_EINVAL, "cf_tm_model_create: an unpaired matrix has spectral radius 0");
      }
    }
  for (int x = 0; x < 4; x++) m->radius[x] = r[x];
  // padded to TM_G with zeros; V / r_x and B / sqrt(r_x r_y) when normalising
  TmModelDev h;
  std::memset(&h, 0, sizeof(h));
  for (int x = 0; x < 4; x++)
    for (int a = 0; a < gamma; a++)
      for (int b = 0; b < gamma; b++) h.V[x][a][b] = V[x * g2 + a * gamma + b] / r[x];
  for (int a = 0; a < gamma; a++)
    for (int b = 0; b < gamma; b++) h.S[a][b] = S[a * gamma + b];
  for (int k = 0; k < nrho; k++)
    for (int x = 0; x < 4; x++)
      for (int y = 0; y < 4; y++) {
        const double sc = 1.0 / std::sqrt(r[x] * r[y]);
        for (int a = 0; a < gamma; a++)
          for (int b = 0; b < gamma; b++)
            h.B[k][x][y][a][b] = B[(((size_t)k * 4 + x) * 4 + y) * g2 + a * gamma + b] * sc;
        for (int a = 0; a < gamma; a++)
          for (int b = 0; b < gamma; b++) {
            double s = 0;
            for (int c = 0; c < gamma; c++) s += h.S[a][c] * h.B[k][x][y][c][b];
            h.SB[k][x][y][a][b] = s;
          }
      }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&m->d, sizeof(TmModelDev));
  if (e == cudaSuccess) e = cudaMemcpy(m->d, &h, sizeof(TmModelDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (m->d) cudaFree(m->d);
    delete m;
    return cuda_fail(nullptr, e, "cf_tm_model_create");
  }
  *out = m;
  return CF_OK;
}

cf_status cf_tm_model_radius(const cf_tm_model *m, double *radius4) {
  if (!m || !radius4) return fail(nullptr, CF_EINVAL, "cf_tm_model_radius: NULL argument");
  for (int x = 0; x < 4; x++) radius4[x] = m->radius[x];
  return CF_OK;
}

cf_status cf_tm_model_free(cf_tm_model *m) {
  if (!m) return CF_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  if (m->d) cudaFree(m->d);
  delete m;
  return CF_OK;
}

extern "C++" {
template <typename T>
static cf_status tm_run(cf_problem *p, const cf_tm_model *mod, TmTables<T> &t, double *logZ) {
  const int n = p->n;
  cudaStream_t st = p->stream;
  if (!t.alloc) {
    const size_t cells = ncells(n) * TM_BLK;
    CF_CUDA(p, dalloc(p->tm_allocs, &t.Q, cells));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.L, cells));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.F, cells));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.E, (size_t)n + 1));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.dmax, (size_t)n + 1));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.err, (size_t)1));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.Zm, (size_t)1));
    CF_CUDA(p, dalloc(p->tm_allocs, &t.logz, (size_t)1));
    CF_CUDA(p, cudaMemsetAsync(t.F, 0, cells * sizeof(T), st));  // pairs closer than 4 are never written
    t.alloc = true;
  }
  if (!t.g || t.gmodel != (const void *)mod->d || t.gnrho != mod->nrho) {
    if (t.g) {
      cudaGraphExecDestroy(t.g);
      t.g = nullptr;
    }
    TmArgs<T> a;
    a.n = n;
    a.nrho = mod->nrho;
    a.Mp = p->dM;
    a.base = p->dbase;
    a.Tr = p->dTr64;
    a.u0 = p->du0;
    a.ls = p->dls;
    a.nls = p->nls;
    a.mod = mod->d;
    a.Q = t.Q;
    a.L = t.L;
    a.F = t.F;
    a.E = t.E;
    a.dmax = t.dmax;
    a.Zm = t.Zm;
    a.logz = t.logz;
    a.err = t.err;
    CF_CUDA(p, cudaFuncSetAttribute((const void *)k_tm_cell<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tm_cell_smem<T>()));
    // captured on a private stream (the problem's may be the legacy default
    // stream, which cannot be captured); the graph runs on the problem's
    cudaStream_t cs = nullptr;
    CF_CUDA(p, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(t.E, 0, sizeof(int) * (n + 1), cs);
      cudaMemsetAsync(t.dmax, 0, sizeof(unsigned long long) * (n + 1), cs);
      cudaMemsetAsync(t.err, 0, sizeof(int), cs);
      k_tm_init<T><<<n, TM_NT, 0, cs>>>(a);
      for (int len = 2; len <= n; len++) {
        if (len - 1 >= 4) k_tm_fold<T><<<n - (len - 1), TM_NT, 0, cs>>>(a, len);
        // few long cells: each cell's groups split over a cluster of two CTAs
        const int cells = n - len + 1, ngroups = std::max(0, (len - 5 + tm_kc<T>() - 1) / tm_kc<T>());
        const int split = cells <= TM_SPLIT8_CELLS && ngroups >= TM_SPLIT8_GROUPS   ? 8
                          : cells <= TM_SPLIT4_CELLS && ngroups >= TM_SPLIT4_GROUPS ? 4
                          : cells <= TM_SPLIT_CELLS && ngroups >= TM_SPLIT_GROUPS   ? 2
                                                                                     : 1;
        const int nst = tm_cell_stages<T>(n, len, split);
        if (split == 1) {
          k_tm_cell<T><<<cells, TM_NTH, (size_t)nst * tm_stage_bytes<T>(), cs>>>(a, len, nst, 1);
        } else {
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3((unsigned)(split * cells));
          cfg.blockDim = dim3(TM_NTH);
          cfg.dynamicSmemBytes = (size_t)nst * tm_stage_bytes<T>();
          cfg.stream = cs;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = (unsigned)split;
          at[0].val.clusterDim.y = 1;
          at[0].val.clusterDim.z = 1;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          cudaLaunchKernelEx(&cfg, k_tm_cell<T>, a, len, nst, split);
        }
      }
      k_tm_finish<T><<<1, 32, 0, cs>>>(a);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&t.g, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(p, e, "cf_tm_inside: graph");
    t.gmodel = mod->d;
    t.gnrho = mod->nrho;
  }
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  CF_CUDA(p, cudaGraphLaunch(t.g, st));
  CF_CUDA(p, cudaEventRecord(p->ev[1], st));
  double lz = 0;
  int err = 0;
  CF_CUDA(p, cudaMemcpyAsync(&lz, t.logz, sizeof(double), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaMemcpyAsync(&err, t.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  CF_CUDA(p, cudaEventElapsedTime(&p->t_tm, p->ev[0], p->ev[1]));
  if (err & ERR_STAGE_TIMEOUT) return fail(p, CF_ETIMEOUT, "cf_tm_inside: a bounded wait for staged inputs gave up");
  if (err || !std::isfinite(lz))
    return fail(p, CF_ENUMERIC, "cf_tm_inside: non-finite or zero partition function (try CF_FP64)");
  *logZ = lz;
  return CF_OK;
}

}  // extern "C++"

cf_status cf_tm_inside(cf_problem *p, const cf_tm_model *mod, cf_precision prec, double *logZ) {
  CfRange nvtx_range("cf_tm_inside");
  if (!p || !mod || !logZ) return fail(p, CF_EINVAL, "cf_tm_inside: NULL argument");
  if (prec != CF_FP64 && prec != CF_FP32_SCALED) return fail(p, CF_EINVAL, "cf_tm_inside: unknown precision");
  if (mod->device != p->device) return fail(p, CF_EINVAL, "cf_tm_inside: model and problem on different devices");
  if (p->n == 0) return fail(p, CF_ESTATE, "cf_tm_inside: no protein set");
  if (p->batch > 1) return fail(p, CF_EINVAL, "cf_tm_inside: not available on a batch");
  CF_CUDA(p, cudaSetDevice(p->device));
  return prec == CF_FP64 ? tm_run(p, mod, p->tm64, logZ) : tm_run(p, mod, p->tm32, logZ);
}

float cf_tm_last_ms(const cf_problem *p) { return p ? p->t_tm : 0.f; }

cf_status cf_set_checkpoint(cf_problem *p, int mode) {
  if (!p || mode < -1 || mode > 1) return fail(p, CF_EINVAL, "cf_set_checkpoint: bad argument");
  if (mode == p->ck_request) return CF_OK;
  CF_CUDA(p, cudaSetDevice(p->device));
  CF_CUDA(p, cudaStreamSynchronize(p->stream));
  p->ck_request = mode;
  // the tables of both precisions are rebuilt in the requested form
  free_prec(p->f32);
  free_prec(p->f64);
  p->have_inside = false;
  return CF_OK;
}

cf_status cf_set_layout(cf_problem *p, int layout) {
  if (!p || layout < 0 || layout > 1) return fail(p, CF_EINVAL, "cf_set_layout: bad argument");
  if (p->batch > 1 && layout != 0) return fail(p, CF_EINVAL, "cf_set_layout: a batch keeps codon states");
  p->layout_req = layout;  // the next cf_set_protein builds the states
  return CF_OK;
}

cf_status cf_layout_states(const cf_problem *p, int *layout, int *states) {
  if (!p) return fail(nullptr, CF_EINVAL, "cf_layout_states: NULL problem");
  if (layout) *layout = p->layout;
  if (states)
    for (int q = 0; q < p->n; q++) states[q] = p->M[q];
  return CF_OK;
}

int cf_checkpointed(const cf_problem *p) {
  if (!p) return 0;
  if (p->f32.inside_alloc) return p->f32.dp.yyck;
  if (p->f64.inside_alloc) return p->f64.dp.yyck;
  return yy_checkpointed(p) ? 1 : 0;
}

cf_status cf_sample(cf_problem *p, int nsamples, uint64_t seed, int32_t *codons, int32_t *partner) {
  CfRange nvtx_range("cf_sample");
  if (!p) return fail(p, CF_EINVAL, "cf_sample: NULL problem");
  if (nsamples < 0 || (nsamples > 0 && (!codons || !partner))) return fail(p, CF_EINVAL, "cf_sample: bad arguments");
  if (!p->have_inside) return fail(p, CF_ESTATE, "cf_sample: run cf_inside first");
  if (nsamples == 0) return CF_OK;
  CF_CUDA(p, cudaSetDevice(p->device));
  return (p->last_prec == CF_FP64) ? run_sample(p, p->f64, nsamples, seed, codons, partner)
                                   : run_sample(p, p->f32, nsamples, seed, codons, partner);
}

}  // extern "C"

// ------------------------------------------------------------------ no-allocation sampler
// Static scratch of cf_sample_noalloc (see include/codonfold.h): error word,
// per-warp states and per-warp traceback stacks for CF_NOALLOC_WARPS warps and
// sequences of up to CF_NOALLOC_MAX_N bases.  The codon ids of the positions
// are read from the problem's own device copy.
namespace {
constexpr size_t kNaErrBytes = 256;
constexpr size_t kNaStateBytes = ((size_t)CF_NOALLOC_WARPS * CF_NOALLOC_MAX_N * sizeof(int) + 255) / 256 * 256;
constexpr size_t kNaStackBytes = (size_t)CF_NOALLOC_WARPS * (CF_NOALLOC_MAX_N + 64) * sizeof(int2);
constexpr size_t kNaBytes = kNaErrBytes + kNaStateBytes + kNaStackBytes;
static_assert(kNaBytes == CF_NOALLOC_SCRATCH_BYTES, "the header states the static scratch size");
static_assert(sizeof(int2) == 8 && sizeof(int) == 4, "scratch layout");
}  // namespace

static __device__ __align__(256) unsigned char g_cf_noalloc_scratch[kNaBytes];

namespace {
std::mutex g_na_mutex;
void *g_na_ptr[64] = {nullptr};

// Device address of the static scratch on `device` (looked up once per device,
// with that device current).
cudaError_t noalloc_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_cf_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[device] = ptr;
  }
  *out = (unsigned char *)g_na_ptr[device];
  return cudaSuccess;
}

template <typename T>
cf_status run_sample_noalloc(cf_problem *p, PrecTables<T> &t, int ns, uint64_t seed, int32_t *codons,
                             int32_t *partner) {
  cudaStream_t st = p->stream;
  unsigned char *base = nullptr;
  CF_CUDA(p, noalloc_scratch(p->device, &base));
  int *err = (int *)base;
  int *state = (int *)(base + kNaErrBytes);
  int2 *stack = (int2 *)(base + kNaErrBytes + kNaStateBytes);
  // the error word must start at zero (states and stacks are written before
  // they are read by every sample)
  CF_CUDA(p, cudaMemsetAsync(err, 0, sizeof(int), st));
  const int warps = std::min(ns, CF_NOALLOC_WARPS);
  SampleArgs<T> a;
  a.p = t.dp;
  a.cid = p->dcid;
  a.sctab = p->layout == 1 ? p->dsctab : nullptr;
  a.nsamples = ns;
  a.seed = seed;
  a.stack = stack;
  a.state = state;
  a.codons = codons;
  a.partner = partner;
  a.err = err;
  k_sample<T><<<(warps + 3) / 4, 128, 0, st>>>(a);
  CF_CUDA(p, cudaGetLastError());
  int herr = 0;
  CF_CUDA(p, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  if (herr) return fail(p, CF_ENUMERIC, "cf_sample_noalloc: traceback inconsistency code " + std::to_string(herr));
  return CF_OK;
}
}  // namespace

extern "C" cf_status cf_sample_noalloc(cf_problem *p, int nsamples, uint64_t seed, int32_t *codons,
                                       int32_t *partner) {
  CfRange nvtx_range("cf_sample_noalloc");
  if (!p) return fail(p, CF_EINVAL, "cf_sample_noalloc: NULL problem");
  if (p->n > CF_NOALLOC_MAX_N)
    return fail(p, CF_EINVAL, "cf_sample_noalloc: sequence length " + std::to_string(p->n) +
                                  " exceeds CF_NOALLOC_MAX_N = " + std::to_string(CF_NOALLOC_MAX_N));
  if (nsamples < 0) return fail(p, CF_EINVAL, "cf_sample_noalloc: nsamples < 0");
  if (!p->have_inside) return fail(p, CF_ESTATE, "cf_sample_noalloc: run cf_inside first");
  if (nsamples == 0) return CF_OK;
  CF_CUDA(p, cudaSetDevice(p->device));
  if (ptr_kind(codons, p->device) != 1 || ptr_kind(partner, p->device) != 1)
    return fail(p, CF_EINVAL, "cf_sample_noalloc: codons and partner must be device memory of the problem's device");
  return (p->last_prec == CF_FP64) ? run_sample_noalloc(p, p->f64, nsamples, seed, codons, partner)
                                   : run_sample_noalloc(p, p->f32, nsamples, seed, codons, partner);
}

// ------------------------------------------------------------------ diagnostics and test hooks

extern "C" cf_status cf_far_band_info(const cf_problem *p, int *in_max_dev, int *in_untiled, int *out_max_dev,
                                      int *out_untiled, int *spread_bits) {
  if (!p) return CF_EINVAL;
  int idev = 0, iun = 0, odev = 0, oun = 0, spr = 0;
  const PrecTables<float> &t = p->f32;
  if (cudaSetDevice(p->device) != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(const_cast<cf_problem *>(p), CF_ECUDA, "cf_far_band_info: device not usable");
  }
  int far_max = 48;
  if (cudaMemcpyFromSymbol(&far_max, g_cf_far_dev_max, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(const_cast<cf_problem *>(p), CF_ECUDA, "cf_far_band_info: bound");
  }
  if (t.inside_alloc && t.bb.gdev) {
    const int n = p->n;
    std::vector<int> dev((size_t)n / FARD + 1, 0);
    if (cudaMemcpy(dev.data(), t.bb.gdev, dev.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(const_cast<cf_problem *>(p), CF_ECUDA, "cf_far_band_info: copy");
    for (int d0 = 0; d0 < n; d0 += FARD)
      if (far_band(d0)) {
        const int v = dev[(size_t)d0 / FARD];
        idev = std::max(idev, v);
        iun += v > far_max ? 1 : 0;
      }
  }
  if (t.outside_alloc && t.ob.fdev) {
    if (cudaMemcpy(&odev, t.ob.fdev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(const_cast<cf_problem *>(p), CF_ECUDA, "cf_far_band_info: copy");
    oun = odev > far_max ? 1 : 0;
  }
  if (in_max_dev) *in_max_dev = idev;
  if (in_untiled) *in_untiled = iun;
  if (t.inside_alloc && t.bb.spread &&
      cudaMemcpy(&spr, t.bb.spread, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(const_cast<cf_problem *>(p), CF_ECUDA, "cf_far_band_info: copy");
  if (out_max_dev) *out_max_dev = odev;
  if (out_untiled) *out_untiled = oun;
  if (spread_bits) *spread_bits = spr;
  return CF_OK;
}

extern "C" cf_status cf_debug_set_range_limit(int device, int bits, int max_length) {
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cf_range_limit, &bits, sizeof(bits));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cf_range_maxlen, &max_length, sizeof(max_length));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cf_debug_set_range_limit");
  return CF_OK;
}

extern "C" cf_status cf_debug_set_wait_polls(int device, unsigned long long polls) {
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();  // no kernel of this process is still waiting
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cf_wait_polls, &polls, sizeof(polls));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cf_debug_set_wait_polls");
  return CF_OK;
}

extern "C" cf_status cf_debug_set_far_dev_max(int device, int bound) {
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cf_far_dev_max, &bound, sizeof(bound));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cf_debug_set_far_dev_max");
  return CF_OK;
}

extern "C" cf_status cf_debug_fail_alloc(long long after) {
  g_fail_alloc_after.store(after < 0 ? -1 : after);
  return CF_OK;
}

extern "C" int cf_debug_classify_pointer(int memory_type, int pointer_device, int problem_device) {
  return classify_ptr(memory_type, pointer_device, problem_device);
}

// ------------------------------------------------------------------ batches of small proteins
// B proteins of one length m <= CF_BATCH_MAX_M in one launch per kernel: every
// array of protein 0 is placed in one slab (the same allocation sequence as a
// single problem, bump-allocated from an arena), the other proteins' slabs
// follow at a fixed stride, and each kernel of the inside and outside graphs
// covers all proteins' cells of its diagonal (blockIdx.y = protein; the
// kernels move their pointers by the protein's slab offset).

namespace {

__global__ void k_replicate(const uint4 *src, size_t n16, long long stride16, int nprot) {
  const int b = blockIdx.y + 1;
  if (b >= nprot) return;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n16; k += (size_t)gridDim.x * blockDim.x)
    (const_cast<uint4 *>(src))[(size_t)b * stride16 + k] = src[k];
}

}  // namespace

struct cf_batch {
  cf_problem *p = nullptr;
  char *buf = nullptr;
  size_t slab = 0;
  int B = 0, m = 0, n = 0, prec = 0;
  bool have = false;
  float t_ms = 0;
};

namespace {

template <typename T>
cf_status batch_layout(cf_problem *p, PrecTables<T> &t, int m) {
  std::vector<int> res(m, 0);  // any letters: the layout depends on the length only
  cf_status s = set_protein_tables(p, res, nullptr, nullptr);
  if (s == CF_OK) s = alloc_inside(p, t);
  if (s == CF_OK) s = alloc_outside(p, t);
  return s;
}

template <typename T>
cf_status batch_clear(cf_batch *b, PrecTables<T> &t) {
  cf_problem *p = b->p;
  const int n = b->n, B = b->B;
  const size_t nc = ncells(n) * BLK, S = b->slab;
  cudaStream_t st = p->stream;
  DP<T> &d = t.dp;
  auto z = [&](void *ptr, size_t bytes) { return cudaMemset2DAsync(ptr, S, 0, bytes, B, st); };
  T *tabs[] = {d.CH, d.QB, d.XI, d.HB, d.QMpp, d.QMpu, d.G, d.QM2pp, d.QM2pu, d.QM2up, d.QM2uu,
               d.hCH, d.hQB, d.hGc, d.hXI, d.hHB, d.hQMpp, d.hQMpu, d.hG, d.hQM2pp, d.hQM2pu, d.hQM2up, d.hQM2uu};
  for (T *q : tabs) CF_CUDA(p, z(q, nc * sizeof(T)));
  CF_CUDA(p, z(d.YY, yy_inside_elems(n, d.yyck) * sizeof(T)));
  CF_CUDA(p, z(d.hYY, (size_t)YRING * n * NYY * BLK * sizeof(T)));
  T *ext[] = {d.Q5U, d.Q5P, d.Gx, d.hQ5U, d.hQ5P, d.hGx};
  for (T *q : ext) CF_CUDA(p, z(q, (size_t)n * BLK * sizeof(T)));
  return CF_OK;
}

template <typename T>
cf_status batch_run(cf_batch *b, PrecTables<T> &t, double *logZ, float *P, double *cm) {
  cf_problem *p = b->p;
  const int n = b->n, m = b->m, B = b->B;
  const size_t S = b->slab;
  cudaStream_t st = p->stream;
  cf_status s = build_inside_graph(p, t);
  if (s == CF_OK) s = build_outside_graph(p, t);
  if (s != CF_OK) return s;
  CF_CUDA(p, cudaMemset2DAsync(p->derr, S, 0, sizeof(int), B, st));
  CF_CUDA(p, cudaEventRecord(p->ev[0], st));
  CF_CUDA(p, cudaGraphLaunch(t.gin, st));
  k_logz<<<dim3(1, B), 32, 0, st>>>(p->dZm, p->dE + (n - 1), p->dls, m - 1, p->dlogz, (long long)S);
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaGraphLaunch(t.gout, st));
  CF_CUDA(p, cudaEventRecord(p->ev[1], st));
  std::vector<int> err(B);
  std::vector<double> lz(B);
  CF_CUDA(p, cudaMemcpy2DAsync(lz.data(), sizeof(double), p->dlogz, S, sizeof(double), B, cudaMemcpyDeviceToHost, st));
  CF_CUDA(p, cudaMemcpy2DAsync(err.data(), sizeof(int), p->derr, S, sizeof(int), B, cudaMemcpyDeviceToHost, st));
  if (P) CF_CUDA(p, cudaMemcpy2DAsync(P, (size_t)n * n * 4, p->dP, S, (size_t)n * n * 4, B, cudaMemcpyDefault, st));
  if (cm) CF_CUDA(p, cudaMemcpy2DAsync(cm, (size_t)m * 48, p->dcm, S, (size_t)m * 48, B, cudaMemcpyDefault, st));
  CF_CUDA(p, cudaStreamSynchronize(st));
  CF_CUDA(p, cudaEventElapsedTime(&b->t_ms, p->ev[0], p->ev[1]));
  for (int k = 0; k < B; k++) {
    if (err[k] & ERR_STAGE_TIMEOUT) return fail(p, CF_ETIMEOUT, "cf_batch_run: a bounded wait for staged inputs gave up");
    if (err[k] || !std::isfinite(lz[k]))
      return fail(p, CF_ENUMERIC, "cf_batch_run: protein " + std::to_string(k) + ": non-finite result");
  }
  std::memcpy(logZ, lz.data(), sizeof(double) * B);
  return CF_OK;
}

}  // namespace

extern "C" cf_status cf_batch_create(const cf_model *model, int device, void *stream, int nprot, int m,
                                     cf_precision prec, cf_batch **out) {
  if (!model || !out || nprot < 1 || m < 1 || m > CF_BATCH_MAX_M || (prec != CF_FP64 && prec != CF_FP32_SCALED))
    return fail(nullptr, CF_EINVAL, "cf_batch_create: bad argument (1 <= m <= CF_BATCH_MAX_M, nprot >= 1)");
  *out = nullptr;
  cf_problem *p = nullptr;
  cf_status s = cf_problem_create(model, device, stream, &p);
  if (s != CF_OK) return s;
  cf_batch *b = new (std::nothrow) cf_batch;
  if (!b) {
    cf_problem_free(p);
    return fail(nullptr, CF_ENOMEM, "cf_batch_create: host memory");
  }
  b->p = p;
  b->B = nprot;
  b->m = m;
  b->n = 3 * m;
  b->prec = (int)prec;
  p->batch = nprot;
  p->ck_request = 0;
  // 1. the slab size: protein 0's allocation sequence in a scratch arena
  char *scratch = nullptr;
  const size_t scap = (size_t)256 << 20;
  cudaError_t e = cudaMalloc(&scratch, scap);
  if (e != cudaSuccess) {
    cf_batch_free(b);
    return cuda_fail(nullptr, e, "cf_batch_create: scratch arena");
  }
  Arena a1{scratch, scap, 0};
  g_arena = &a1;
  s = prec == CF_FP64 ? batch_layout(p, p->f64, m) : batch_layout(p, p->f32, m);
  g_arena = nullptr;
  cudaStreamSynchronize(p->stream);
  release_protein(p);
  cudaFree(scratch);
  if (s != CF_OK) {
    cf_batch_free(b);
    return s;
  }
  b->slab = (a1.used + 4095) / 4096 * 4096;
  // 2. the batch buffer, protein 0 laid out in its first slab, copied to all
  e = cudaMalloc(&b->buf, b->slab * (size_t)nprot);
  if (e == cudaSuccess) e = cudaMemset(b->buf, 0, b->slab * (size_t)nprot);
  if (e != cudaSuccess) {
    cf_batch_free(b);
    return cuda_fail(nullptr, e, "cf_batch_create: batch buffer");
  }
  Arena a2{b->buf, b->slab, 0};
  g_arena = &a2;
  s = prec == CF_FP64 ? batch_layout(p, p->f64, m) : batch_layout(p, p->f32, m);
  g_arena = nullptr;
  if (s == CF_OK && a2.used != a1.used) s = fail(p, CF_ECUDA, "cf_batch_create: layout mismatch");
  if (s != CF_OK) {
    cf_batch_free(b);
    return s;
  }
  p->bstride = (long long)b->slab;
  p->f32.dp.bstride = p->f64.dp.bstride = (long long)b->slab;
  if (nprot > 1) {
    k_replicate<<<dim3(148, nprot - 1), 256, 0, p->stream>>>((const uint4 *)b->buf, b->slab / 16,
                                                             (long long)(b->slab / 16), nprot);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    cf_batch_free(b);
    return cuda_fail(nullptr, e, "cf_batch_create: replicate");
  }
  *out = b;
  return CF_OK;
}

extern "C" cf_status cf_batch_set_proteins(cf_batch *b, const char *aa, const double *lw, const double *pb) {
  CfRange nvtx_range("cf_batch_set_proteins");
  if (!b || !aa) return fail(nullptr, CF_EINVAL, "cf_batch_set_proteins: NULL argument");
  cf_problem *p = b->p;
  const int B = b->B, m = b->m, n = b->n;
  const size_t S = b->slab;
  if (lw)
    for (size_t k = 0; k < (size_t)B * m * 6; k++)
      if (!std::isfinite(lw[k])) return fail(p, CF_EINVAL, "cf_batch_set_proteins: non-finite codon weight");
  if (pb)
    for (size_t k = 0; k < 61 * 61; k++)
      if (!std::isfinite(pb[k])) return fail(p, CF_EINVAL, "cf_batch_set_proteins: non-finite pair bonus");
  const GeneticCode &gc = gcode();
  std::vector<int> M((size_t)B * n), base((size_t)B * n * NS, 0), cid((size_t)B * n * NS, -1), bnd((size_t)B * n);
  for (int k = 0; k < B; k++)
    for (int r = 0; r < m; r++) {
      const char *q = aa[(size_t)k * m + r] ? std::strchr(kAminoAcids, aa[(size_t)k * m + r]) : nullptr;
      if (!q) return fail(p, CF_EINVAL, "cf_batch_set_proteins: invalid amino acid");
      const auto &cods = gc.codons[q - kAminoAcids];
      for (int off = 0; off < 3; off++) {
        const size_t i = (size_t)k * n + 3 * r + off;
        M[i] = (int)cods.size();
        for (size_t a = 0; a < cods.size(); a++) {
          base[i * NS + a] = (cods[a] >> (2 * (2 - off))) & 3;
          cid[i * NS + a] = gc.sense_id[cods[a]];
        }
        bnd[i] = (off == 2 && 3 * r + off + 1 < n) ? 1 : 0;
      }
    }
  CF_CUDA(p, cudaSetDevice(p->device));
  cudaStream_t st = p->stream;
  CF_CUDA(p, cudaStreamSynchronize(st));
  b->have = false;
  auto up = [&](void *dst, const void *src, size_t w) {
    return cudaMemcpy2DAsync(dst, S, src, w, w, B, cudaMemcpyHostToDevice, st);
  };
  CF_CUDA(p, up(p->dM, M.data(), sizeof(int) * n));
  CF_CUDA(p, up(p->dbase, base.data(), sizeof(int) * n * NS));
  CF_CUDA(p, up(p->dcid, cid.data(), sizeof(int) * n * NS));
  CF_CUDA(p, up(p->dbnd, bnd.data(), sizeof(int) * n));
  if (lw) CF_CUDA(p, up(p->dlw, lw, sizeof(double) * m * 6));
  else CF_CUDA(p, cudaMemset2DAsync(p->dlw, S, 0, sizeof(double) * m * 6, B, st));
  if (pb) {
    CF_CUDA(p, cudaMemcpyAsync(p->dpb, pb, sizeof(double) * 61 * 61, cudaMemcpyHostToDevice, st));
    if (B > 1) {  // the same bonuses in every slab
      // (the last 16-byte chunk reaches into the allocation's 256-byte padding)
      k_replicate<<<dim3(8, B - 1), 256, 0, st>>>((const uint4 *)p->dpb, (61 * 61 * 8 + 15) / 16, (long long)(S / 16),
                                                  B);
      CF_CUDA(p, cudaGetLastError());
    }
  } else {
    CF_CUDA(p, cudaMemset2DAsync(p->dpb, S, 0, sizeof(double) * 61 * 61, B, st));
  }
  CF_CUDA(p, cudaMemset2DAsync(p->dls, S, 0, sizeof(double) * std::max(m - 1, 1), B, st));
  CF_CUDA(p, cudaMemset2DAsync(p->dE, S, 0, sizeof(int) * n, B, st));
  k_transfers<<<dim3((n + 127) / 128, B), 128, 0, st>>>(n, p->dM, p->dbase, p->dcid, p->den64, p->dlw, p->dpb,
                                                         p->dTr64, p->dX64, p->du0, p->dls, (long long)S);
  CF_CUDA(p, cudaGetLastError());
  cf_status s;
  if (b->prec == CF_FP64) {
    k_cast<double><<<dim3(8, B), 256, 0, st>>>(p->dTr64, (double *)p->f64.dp.Tr, (size_t)n * BLK, (long long)S);
    k_cast<double><<<dim3(8, B), 256, 0, st>>>(p->dX64, (double *)p->f64.dp.X, (size_t)n * 4 * BLK, (long long)S);
    s = batch_clear(b, p->f64);
  } else {
    k_cast<float><<<dim3(8, B), 256, 0, st>>>(p->dTr64, (float *)p->f32.dp.Tr, (size_t)n * BLK, (long long)S);
    k_cast<float><<<dim3(8, B), 256, 0, st>>>(p->dX64, (float *)p->f32.dp.X, (size_t)n * 4 * BLK, (long long)S);
    s = batch_clear(b, p->f32);
  }
  if (s != CF_OK) return s;
  CF_CUDA(p, cudaGetLastError());
  CF_CUDA(p, cudaStreamSynchronize(st));
  b->have = true;
  return CF_OK;
}

extern "C" cf_status cf_batch_run(cf_batch *b, double *logZ, float *pair_prob, double *codon_marg) {
  CfRange nvtx_range("cf_batch_run");
  if (!b || !logZ) return fail(nullptr, CF_EINVAL, "cf_batch_run: NULL argument");
  if (!b->have) return fail(b->p, CF_ESTATE, "cf_batch_run: set the proteins first");
  CF_CUDA(b->p, cudaSetDevice(b->p->device));
  return b->prec == CF_FP64 ? batch_run(b, b->p->f64, logZ, pair_prob, codon_marg)
                            : batch_run(b, b->p->f32, logZ, pair_prob, codon_marg);
}

extern "C" float cf_batch_last_ms(const cf_batch *b) { return b ? b->t_ms : 0.f; }

extern "C" cf_status cf_batch_free(cf_batch *b) {
  if (!b) return CF_OK;
  if (b->p) {
    cudaSetDevice(b->p->device);
    cudaStreamSynchronize(b->p->stream);
    cf_problem_free(b->p);  // the slab arrays belong to buf: the problem's lists are empty
  }
  if (b->buf) cudaFree(b->buf);
  delete b;
  return CF_OK;
}
