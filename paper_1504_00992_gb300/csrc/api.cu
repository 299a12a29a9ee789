// C ABI of the TEBD / RRSVD library: handles, device memory, and the launch
// sequence of a sweep.  See include/tebd_gb300.h for the contract.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tebd_gb300.h"
#include "adjoint.cuh"
#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"
#include "workspace.cuh"

using namespace tg;

namespace {

const size_t ALIGN = 256;
// the precisions that run the mixed form (mixed.cu)
inline bool prec_mixed(int p) { return p == TEBD_PREC_TF32 || p == TEBD_PREC_BF16; }
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

struct ErrState {
  int code = TEBD_OK;
  std::string msg;
  void set(int c, const char* fmt, ...) {
    if (code != TEBD_OK) return;  // sticky: keep the first
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    code = c;
    msg = buf;
  }
};

#define CU_OR(h, x)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) {                                                              \
      (h)->err.set(TEBD_ECUDA, "%s failed: %s", #x, cudaGetErrorString(e_));               \
      return (h)->err.code;                                                               \
    }                                                                                     \
  } while (0)

bool all_finite(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return false;
  return true;
}

}  // namespace

namespace tg {
WsLayout ws_layout(int m, int n, int k, int l, bool own_U, bool own_V, int r) {
  WsLayout w;
  size_t o = 0;
  const size_t c = sizeof(cplx);
  w.omega = o; o += align_up(c * (size_t)n * l);
  w.Y = o; o += align_up(c * (size_t)m * l);
  w.Q = o; o += align_up(c * (size_t)m * l);
  w.Yt = o; o += align_up(c * (size_t)n * l);
  w.Qt = o; o += align_up(c * (size_t)n * l);
  // R and J also hold the scratch of the many-CTA QR (partial products in R,
  // alpha, tau and the panels' T in J), which a bond batched with larger
  // ones may run even when its own l is small
  w.R = o; o += align_up(c * std::max((size_t)l * l, qr_multi_scratch_r(l)));
  w.J = o; o += align_up(c * std::max((size_t)l * l, qr_multi_scratch_j(l)));
  w.Jk = o; o += align_up(c * (size_t)l * k);
  w.Wk = o; o += align_up(c * (size_t)l * k);
  w.U = o; if (own_U) o += align_up(c * (size_t)m * k);
  w.V = o; if (own_V) o += align_up(c * (size_t)k * n);
  w.sigma = o; o += align_up(sizeof(double) * (size_t)l);
  w.part = o; o += align_up(sizeof(double) * NPART);
  w.scal = o; o += align_up(sizeof(double) * 4);
  w.Dr = o; o += align_up(c * (size_t)m * r);
  w.total = o;
  return w;
}

static std::atomic<int> g_fault_alloc{0}, g_fault_tc{0};

bool fault_take(int kind) {
  std::atomic<int>& f = (kind == TEBD_FAULT_ALLOC) ? g_fault_alloc : g_fault_tc;
  int armed = 1;
  return f.compare_exchange_strong(armed, 0);
}
}  // namespace tg

extern "C" int tebd_fault_inject(int kind) {
  switch (kind) {
    case TEBD_FAULT_NONE: g_fault_alloc = 0; g_fault_tc = 0; return TEBD_OK;
    case TEBD_FAULT_ALLOC: g_fault_alloc = 1; return TEBD_OK;
    case TEBD_FAULT_TC_STALL: g_fault_tc = 1; return TEBD_OK;
    default: return TEBD_EINVAL;
  }
}

namespace {
// Device blocks of a handle: the caller's allocator, or cudaMalloc / cudaFree.
struct DevAlloc {
  tebd_alloc_fn fn = nullptr;
  tebd_release_fn rel = nullptr;
  void* ctx = nullptr;
  // TEBD_OK, TEBD_ENOMEM (no memory, or an injected allocation fault) or
  // TEBD_EINVAL (a block that is not 256-byte aligned; returned at once)
  int get(size_t bytes, void** out) const {
    *out = nullptr;
    if (fault_take(TEBD_FAULT_ALLOC)) return TEBD_ENOMEM;
    if (fn) {
      void* q = fn(bytes, ctx);
      if (!q) return TEBD_ENOMEM;
      if ((uintptr_t)q % ALIGN) {
        rel(q, ctx);
        return TEBD_EINVAL;
      }
      *out = q;
      return TEBD_OK;
    }
    if (cudaMalloc(out, bytes) != cudaSuccess) {
      cudaGetLastError();
      *out = nullptr;
      return TEBD_ENOMEM;
    }
    return TEBD_OK;
  }
  void put(void* q) const {
    if (!q) return;
    if (fn) rel(q, ctx);
    else cudaFree(q);
  }
};
}  // namespace

// ===========================================================================
// TEBD handle: one or many chains, all bonds of a parity updated together
// ===========================================================================
struct ChainH {
  int N = 0;
  int64_t chain_index = 0;  // Philox chain word
  std::vector<int> d, chi_cap, cap_ext;
  std::vector<size_t> gamma_off, lam_off, gate_off;
  size_t gamma_lo = 0, gamma_hi = 0;  // the chain's Gamma block in the arena
  size_t tab_off = 0, int_off = 0, wb_off = 0;
  std::vector<cplx*> gamma_ptr;       // N
  std::vector<double*> lam_ptr;       // N+1, outer ones -> the constant 1.0
  int* chi_ext = nullptr;             // device, N+1
  int* dsite_dev = nullptr;
  int* cap_ext_dev = nullptr;
  cplx** gamma_tab = nullptr;
  double** lam_tab = nullptr;
  double* wbond = nullptr;            // device, N-1: w of each bond's latest update
  bool gates_set[2] = {false, false};
  ChainDev dev{};
};

struct Wave {
  int first = 0, count = 0;
  Caps cap{};
  int tiles[6] = {0, 0, 0, 0, 0, 0};
  int fused = 0;    // 1: the whole update of every bond in one persistent launch (fused.cu)
  MixedKnobs mk{0, 0, 0, 0};  // launch choices of the mixed form (TF32 handles)
  float tune_ms[2] = {0.f, 0.f};  // tuner timings of the staged and fused RRSVD (0: not timed)
  MixedSizes ms{};  // TF32 handles: the wave's FP32 arrays at its capacities
};

struct ParitySet {
  int batch = 0;
  Dims* dims = nullptr;     // device
  ProbPtr* ptrs = nullptr;  // device
  std::vector<std::pair<int, int>> bonds;  // (chain slot, bond)
  std::vector<Wave> waves;
};

// Byte offsets of the handle's arena, from the plan of tebd_create_multi.
struct HandlePlan {
  size_t one_off = 0, st_off = 0, wacc_off = 0, sweep_off = 0, tcerr_off = 0, op_off = 0, wout_off = 0, queue_off = 0;
  size_t desc_off = 0, desc_per = 0, ws_off = 0, mixed_off = 0, total = 0;
  std::vector<WsLayout> lay[2];
  int max_batch = 0;
};

struct tebd_s {
  ErrState err;
  DevAlloc alloc;
  HandlePlan plan;
  int p = 0, q = 0, precision = 0;
  uint64_t seed = 0;
  double cutoff = 1e-14;
  int64_t sweeps = 0;
  cudaStream_t stream = 0;
  std::vector<ChainH> ch;
  int cur = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  ParitySet par[2];
  int* status = nullptr;
  double* wacc = nullptr;   // 2 per chain: sum w, prod (1 - w)
  double* wout = nullptr;   // per problem of the larger parity
  uint64_t* sweep_dev = nullptr;
  int* queue = nullptr;        // work counter of the persistent fused launch
  int* tcerr = nullptr;        // tensor-core wait timeout flag (TF32 handles)
  char* mixed = nullptr;       // FP32 arrays of the current wave (TF32 handles)
  cplx* op_dev = nullptr;
  cplx* out_dev = nullptr;
  double* one_lam = nullptr;
  bool use_graph = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaStream_t own_stream = nullptr;  // used for graphs when the caller gives the legacy stream 0
  // reverse pass: checkpoints of the chain's state before every recorded sweep
  bool recording = false;
  struct Ckpt {
    int parity;
    int64_t sweep;
    char* buf;
  };
  std::vector<Ckpt> ckpts;
  char* adj_arena = nullptr;
  AdjPtr* adj_dev[2] = {nullptr, nullptr};
  cplx* gbar0 = nullptr;  // cotangent state (Gamma block, then lambdas)
  size_t cot_bytes = 0;
};

static size_t chain_region_end(const ChainH& C) {
  return C.int_off + 3 * align_up(sizeof(int) * (C.N + 1));
}

static void free_ckpts(tebd_s* h) {
  for (auto& c : h->ckpts) h->alloc.put(c.buf);
  h->ckpts.clear();
}

static int tebd_check_status(tebd_t h) {
  int st = 0, te = 0;
  CU_OR(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (h->tcerr) CU_OR(h, cudaMemcpyAsync(&te, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  if (te) h->err.set(TEBD_ETIMEOUT, "a tensor-core pipeline wait timed out");
  else if (st & 4)
    h->err.set(TEBD_ENUMERIC, "the re-orthonormalisation of an FP32 basis met a non-finite or far from orthonormal "
                              "basis");
  else if (st & 1)
    h->err.set(TEBD_ENUMERIC, "a bond update met a zero or non-finite theta");
  return h->err.code;
}

static void tebd_free(tebd_s* h) {
  // a caller's allocator may hand the blocks out again at once
  if (h->alloc.fn) cudaStreamSynchronize(h->stream);
  free_ckpts(h);
  h->alloc.put(h->adj_arena);
  for (int i = 0; i < 2; ++i)
    if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
  h->alloc.put(h->arena);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

// GEMM tile autotuner: times the 16x16 and 32x32 variants of every GEMM stage
// on the wave's capacity sizes (the saturated regime) and keeps the faster.
// Results are cached per (stage, rows, cols, inner, batch) for the process.
static std::map<std::vector<long long>, int> g_tile_cache;
static std::map<std::vector<long long>, std::pair<MixedKnobs, std::vector<float>>> g_knob_cache;
static std::mutex g_tile_mu;

static int tune_wave(tebd_s* h, const ParitySet& ps, Wave& w, cudaStream_t st, Dims* scratch_dims, const int p_os,
                     int fused_mode) {
  // capacity-sized descriptors of the wave's problems
  std::vector<Dims> hd(w.count);
  std::vector<ProbPtr> hp(w.count);
  if (cudaMemcpy(hp.data(), ps.ptrs + w.first, sizeof(ProbPtr) * w.count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return -1;
  for (int i = 0; i < w.count; ++i) {
    Dims& D = hd[i];
    memset(&D, 0, sizeof D);
    D.dl = hp[i].dl_s; D.dr = hp[i].dr_s;
    D.cl = hp[i].cap_l; D.cm = hp[i].cap_m; D.cr = hp[i].cap_r;
    D.m = D.dl * D.cl; D.n = D.dr * D.cr;
    D.k = std::min(hp[i].chicap, std::min(D.m, D.n));
    D.l = std::min(D.k + p_os, std::min(D.m, D.n));
    D.active = 1;
  }
  if (cudaMemcpy(scratch_dims, hd.data(), sizeof(Dims) * w.count, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int inner[6] = {w.cap.n, w.cap.m, w.cap.n, w.cap.m, w.cap.l, w.cap.l};
  for (int stage = 0; stage < 6; ++stage) {
    std::vector<long long> key = {stage, w.cap.m, w.cap.n, w.cap.l, w.cap.k, inner[stage], w.count};
    {
      std::lock_guard<std::mutex> g(g_tile_mu);
      auto it = g_tile_cache.find(key);
      if (it != g_tile_cache.end()) { w.tiles[stage] = it->second; continue; }
    }
    float best = 1e30f;
    int pick = 0;
    for (int tile : {16, 32}) {
      launch_zgemm_tile(stage, tile, scratch_dims, ps.ptrs + w.first, w.count, w.cap, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2; ++r) launch_zgemm_tile(stage, tile, scratch_dims, ps.ptrs + w.first, w.count, w.cap, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; pick = tile; }
    }
    w.tiles[stage] = pick;
    std::lock_guard<std::mutex> g(g_tile_mu);
    g_tile_cache[key] = pick;
  }
  // the whole RRSVD of the wave, staged (tuned tiles) against the persistent
  // fused kernel, on synthetic theta at the capacity sizes (the two give the
  // same results; the data only sets the QR and Jacobi work)
  if (fused_mode == 0 && fused_fits(w.cap)) {
    if (launch_tune_theta(scratch_dims, ps.ptrs + w.first, w.count, st) != cudaSuccess) return -1;
    float ms[2] = {1e30f, 1e30f};
    for (int variant = 0; variant < 2; ++variant)
      for (int r = 0; r < 2; ++r) {  // the first run warms up
        cudaEventRecord(e0, st);
        const cudaError_t e =
            variant == 0 ? run_rrsvd(scratch_dims, ps.ptrs + w.first, w.count, w.cap, h->q, h->seed, 0, 0, -1,
                                     h->status, st, h->sweep_dev, w.tiles)
                         : launch_bond_fused(ps.ptrs + w.first, nullptr, scratch_dims, w.count, p_os, h->q, h->seed,
                                             h->sweep_dev, h->cutoff, nullptr, h->status, h->queue, st);
        if (e != cudaSuccess) return -1;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r == 1) ms[variant] = t;
      }
    w.tune_ms[0] = ms[0];
    w.tune_ms[1] = ms[1];
    w.fused = ms[1] < ms[0] ? 1 : 0;
    if (cudaMemsetAsync(h->status, 0, sizeof(int), st) != cudaSuccess) return -1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Coordinate search over the mixed form's launch choices (MixedKnobs): one
// knob at a time, each candidate timed once on the current best of the
// others; `run` launches the whole RRSVD with the given knobs on `st`.
// Returns the timings of the size rules and of the choice kept.
template <class Run>
static int tune_knobs(Run run, cudaStream_t st, const Caps& cap, int batch, MixedKnobs& best, float ms_out[2]) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_of = [&](const MixedKnobs& k, float& ms) -> bool {
    cudaEventRecord(e0, st);
    if (run(k) != cudaSuccess) return false;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return false;
    cudaEventElapsedTime(&ms, e0, e1);
    return true;
  };
  best = MixedKnobs{0, 0, 0, 0, 0};
  float t_best = 0.f, t_rule = 0.f;
  bool ok = run(best) == cudaSuccess && time_of(best, t_best);  // warm-up, then the size rules
  t_rule = t_best;
  const bool multi_ok = cap.n >= 1024 && cap.l >= 16;  // the many-CTA QR's structure (its own rule adds the batch)
  const bool cl_ok = cap.l >= 64 && cap.l <= 512;
  std::vector<std::vector<int>> cand = {{0, 1}, {0, 512, 256, 128}, {0, 1, 2, 3}, {0, 1, 2, 3}, {0, 1, 2}};
  for (int knob = 0; knob < 5 && ok; ++knob)
    for (int v : cand[knob]) {
      MixedKnobs k = best;
      int* f = knob == 0 ? &k.tc_half : knob == 1 ? &k.qr_threads : knob == 2 ? &k.qrbh : knob == 3 ? &k.jac : &k.dfg;
      if (*f == v || (knob == 2 && v == 2 && !multi_ok) || (knob == 3 && v == 2 && !cl_ok)) continue;
      *f = v;
      float t = 0.f;
      if (!time_of(k, t)) { ok = false; break; }
      if (t < 0.97f * t_best) { best = k; t_best = t; }  // a clear gain only
    }
  (void)batch;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ms_out[0] = t_rule;
  ms_out[1] = t_best;
  return ok && cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static int tebd_reset_state(tebd_t h, int slot, const double* psi);


// Validates the chain descriptors and plans the handle on the host: the
// chains' capacities and Gamma/lambda/gate regions, the bonds of each parity
// (grouped by shape in the mixed form), their waves under the workspace
// budget and the arena's offsets.  Makes no CUDA call.
static int plan_handle(tebd_s* h, int n_chains, const tebd_desc_t* descs, HandlePlan& lay_plan) {
  if (n_chains < 1 || !descs) return TEBD_EINVAL;
  const tebd_desc_t& d0 = descs[0];
  if (d0.p < 0 || d0.q < 0) return TEBD_EINVAL;
  if (d0.precision != TEBD_PREC_FP64 && !prec_mixed(d0.precision)) return TEBD_ENOTIMPL;
  if ((d0.alloc == nullptr) != (d0.release == nullptr)) return TEBD_EINVAL;
  if (d0.fused < -1 || d0.fused > 1) return TEBD_EINVAL;
  for (int c = 0; c < n_chains; ++c) {
    const tebd_desc_t& dc = descs[c];
    if (dc.N < 2 || dc.p != d0.p || dc.q != d0.q || dc.seed != d0.seed || dc.precision != d0.precision)
      return TEBD_EINVAL;
  }
  h->p = d0.p;
  h->q = d0.q;
  h->seed = d0.seed;
  h->precision = d0.precision;
  h->cutoff = d0.sv_cutoff > 0 ? d0.sv_cutoff : 1e-14;
  h->use_graph = d0.use_graph != 0;
  h->ch.resize(n_chains);
  size_t off = 0;
  for (int c = 0; c < n_chains; ++c) {
    const tebd_desc_t& dc = descs[c];
    ChainH& C = h->ch[c];
    const int N = dc.N;
    C.N = N;
    C.chain_index = (n_chains == 1) ? dc.chain : (int64_t)dc.chain + c;
    C.d.resize(N);
    for (int s = 0; s < N; ++s) {
      const int ds = dc.d_site ? dc.d_site[s] : dc.d;
      if (ds < 2 || ds > 64) { return TEBD_EINVAL; }
      C.d[s] = ds;
    }
    C.chi_cap.resize(N - 1);
    for (int b = 0; b < N - 1; ++b) {
      const int cc = dc.chi_bond ? dc.chi_bond[b] : dc.chi_max;
      if (cc < 1) { return TEBD_EINVAL; }
      C.chi_cap[b] = cc;
    }
    // chi_b <= min(cap_b, prod_{s<=b} d_s, prod_{s>b} d_s)
    C.cap_ext.assign(N + 1, 1);
    for (int b = 0; b < N - 1; ++b) {
      double left = 1, right = 1;
      for (int s = 0; s <= b; ++s) left = std::min(left * C.d[s], 1e9);
      for (int s = b + 1; s < N; ++s) right = std::min(right * C.d[s], 1e9);
      C.cap_ext[b + 1] = (int)std::min<double>(C.chi_cap[b], std::min(left, right));
    }
    C.gamma_off.resize(N);
    C.gamma_lo = off;
    for (int s = 0; s < N; ++s) {
      C.gamma_off[s] = off;
      off += align_up(sizeof(cplx) * (size_t)C.d[s] * C.cap_ext[s] * C.cap_ext[s + 1]);
    }
    C.gamma_hi = off;
    C.lam_off.resize(N - 1);
    for (int b = 0; b < N - 1; ++b) {
      C.lam_off[b] = off;
      off += align_up(sizeof(double) * C.cap_ext[b + 1]);
    }
    C.gate_off.resize(N - 1);
    for (int b = 0; b < N - 1; ++b) {
      C.gate_off[b] = off;
      const size_t dd = (size_t)C.d[b] * C.d[b + 1];
      off += align_up(sizeof(cplx) * dd * dd);
    }
    C.tab_off = off;
    off += align_up(sizeof(cplx*) * N) + align_up(sizeof(double*) * (N + 1));
    C.int_off = off;
    off += 3 * align_up(sizeof(int) * (N + 1));
    C.wb_off = off;
    off += align_up(sizeof(double) * (N - 1));
  }
  lay_plan.one_off = off; off += ALIGN;
  lay_plan.st_off = off; off += ALIGN;
  lay_plan.wacc_off = off; off += align_up(sizeof(double) * 2 * n_chains);
  lay_plan.sweep_off = off; off += ALIGN;
  lay_plan.tcerr_off = off; off += ALIGN;
  lay_plan.queue_off = off; off += ALIGN;
  lay_plan.op_off = off; off += align_up(sizeof(cplx) * 64 * 64) + ALIGN;
  // problems of each parity, chain-major, and their waves under the budget
  const size_t budget = d0.workspace_budget;
  size_t ws_max = 0;
  std::vector<WsLayout>* lay = lay_plan.lay;
  std::vector<size_t> pbytes[2];
  int max_batch = 0;
  const bool tf32 = prec_mixed(h->precision);
  const int bf16 = h->precision == TEBD_PREC_BF16;
  size_t mixed_max = 0;
  auto bond_caps = [&](const ChainH& C, int b, int& mc, int& nc, int& kc, int& lc) {
    mc = C.d[b] * C.cap_ext[b];
    nc = C.d[b + 1] * C.cap_ext[b + 2];
    kc = std::min(C.cap_ext[b + 1], std::min(mc, nc));
    lc = std::min(kc + h->p, std::min(mc, nc));
  };
  for (int par = 0; par < 2; ++par) {
    ParitySet& ps = h->par[par];
    for (int c = 0; c < n_chains; ++c) {
      const ChainH& C = h->ch[c];
      for (int b = par; b < C.N - 1; b += 2) {
        int mc, nc, kc, lc;
        bond_caps(C, b, mc, nc, kc, lc);
        if (lc > 512) { return TEBD_ENOTIMPL; }
        ps.bonds.push_back({c, b});
      }
    }
    if (tf32) {
      // the FP32 arrays of a wave are laid out at its capacities: group bonds
      // of similar shape (largest first) so that little of them is padding
      std::stable_sort(ps.bonds.begin(), ps.bonds.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        int m1, n1, k1, l1, m2, n2, k2, l2;
        bond_caps(h->ch[x.first], x.second, m1, n1, k1, l1);
        bond_caps(h->ch[y.first], y.second, m2, n2, k2, l2);
        if (l1 != l2) return l1 > l2;
        return (long long)m1 * n1 > (long long)m2 * n2;
      });
    }
    for (const auto& cb : ps.bonds) {
      int mc, nc, kc, lc;
      bond_caps(h->ch[cb.first], cb.second, mc, nc, kc, lc);
      lay[par].push_back(ws_layout(mc, nc, kc, lc, true, true));
      const ChainH& Cb = h->ch[cb.first];
      const bool gemm_gate = Cb.d[cb.second] * Cb.d[cb.second + 1] >= GATE_GEMM_MIN;  // pre-gate theta buffer
      pbytes[par].push_back(align_up(sizeof(cplx) * (size_t)mc * nc) * (gemm_gate ? 2 : 1) + lay[par].back().total);
    }
    ps.batch = (int)ps.bonds.size();
    max_batch = std::max(max_batch, ps.batch);
    size_t acc = 0;
    Wave w;
    w.first = 0;
    for (int i = 0; i < ps.batch; ++i) {
      const int c = ps.bonds[i].first, b = ps.bonds[i].second;
      const ChainH& C = h->ch[c];
      int mc, nc, kc, lc;
      bond_caps(C, b, mc, nc, kc, lc);
      Caps cp = w.cap;
      cp.m = std::max(cp.m, mc); cp.n = std::max(cp.n, nc); cp.k = std::max(cp.k, kc); cp.l = std::max(cp.l, lc);
      cp.cl = std::max(cp.cl, C.cap_ext[b]); cp.cr = std::max(cp.cr, C.cap_ext[b + 2]);
      cp.cm = std::max(cp.cm, C.cap_ext[b + 1]);
      cp.dl = std::max(cp.dl, C.d[b]); cp.dr = std::max(cp.dr, C.d[b + 1]);
      const size_t mix = tf32 ? mixed_bytes(mixed_sizes(cp.m, cp.n, cp.k, cp.l, bf16, &cp), w.count + 1) : 0;
      if (w.count > 0 && budget > 0 && acc + pbytes[par][i] + mix > budget) {
        ps.waves.push_back(w);
        ws_max = std::max(ws_max, acc);
        w = Wave();
        w.first = i;
        acc = 0;
        cp = w.cap;
        cp.m = mc; cp.n = nc; cp.k = kc; cp.l = lc;
        cp.cl = C.cap_ext[b]; cp.cr = C.cap_ext[b + 2]; cp.dl = C.d[b]; cp.dr = C.d[b + 1];
        cp.cm = C.cap_ext[b + 1];
      }
      w.cap = cp;
      acc += pbytes[par][i];
      w.count++;
    }
    if (w.count > 0) {
      ps.waves.push_back(w);
      ws_max = std::max(ws_max, acc);
    }
    if (tf32)
      for (Wave& wv : ps.waves) {
        wv.ms = mixed_sizes(wv.cap.m, wv.cap.n, wv.cap.k, wv.cap.l, bf16, &wv.cap);
        mixed_max = std::max(mixed_max, mixed_bytes(wv.ms, wv.count));
      }
  }
  lay_plan.wout_off = off; off += align_up(sizeof(double) * std::max(1, max_batch));
  lay_plan.desc_off = off;
  lay_plan.desc_per = align_up(sizeof(Dims) * std::max(1, max_batch)) + align_up(sizeof(ProbPtr) * std::max(1, max_batch));
  off += 2 * lay_plan.desc_per + align_up(sizeof(Dims) * std::max(1, max_batch));  // + autotuner scratch dims
  lay_plan.ws_off = off;
  off += ws_max;
  lay_plan.mixed_off = off;
  off += align_up(mixed_max);
  lay_plan.total = off;
  lay_plan.max_batch = max_batch;
  h->arena_bytes = off;
  return TEBD_OK;
}

extern "C" int tebd_plan_query(int n_chains, const tebd_desc_t* descs, size_t* arena_bytes, int* waves_even,
                               int* waves_odd) {
  tebd_s* h = new tebd_s();
  HandlePlan lay_plan;
  const int rc = plan_handle(h, n_chains, descs, lay_plan);
  if (rc == TEBD_OK) {
    if (arena_bytes) *arena_bytes = lay_plan.total;
    if (waves_even) *waves_even = (int)h->par[0].waves.size();
    if (waves_odd) *waves_odd = (int)h->par[1].waves.size();
  }
  delete h;
  return rc;
}

// Points every pointer of the handle (host copies and device tables) into
// its arena h->arena from the offsets of h->plan, and uploads the pointer
// tables and the constant lambda = 1 of the outer bonds; the arena's other
// contents are left as they are.  Runs at creation and after
// tebd_set_allocator moved the arena.  Synchronous.
static bool bind_arena(tebd_s* h) {
  const HandlePlan& L = h->plan;
  char* A = h->arena;
  const bool tf32 = prec_mixed(h->precision);
  h->one_lam = (double*)(A + L.one_off);
  h->status = (int*)(A + L.st_off);
  h->wacc = (double*)(A + L.wacc_off);
  h->sweep_dev = (uint64_t*)(A + L.sweep_off);
  h->queue = (int*)(A + L.queue_off);
  h->tcerr = tf32 ? (int*)(A + L.tcerr_off) : nullptr;
  h->mixed = tf32 ? A + L.mixed_off : nullptr;
  h->op_dev = (cplx*)(A + L.op_off);
  h->out_dev = (cplx*)(A + L.op_off + align_up(sizeof(cplx) * 64 * 64));
  h->wout = (double*)(A + L.wout_off);
  bool ok = true;
  for (size_t c = 0; c < h->ch.size() && ok; ++c) {
    ChainH& C = h->ch[c];
    const int N = C.N;
    C.gamma_ptr.resize(N);
    for (int s = 0; s < N; ++s) C.gamma_ptr[s] = (cplx*)(A + C.gamma_off[s]);
    C.lam_ptr.resize(N + 1);
    C.lam_ptr[0] = h->one_lam;
    C.lam_ptr[N] = h->one_lam;
    for (int b = 0; b < N - 1; ++b) C.lam_ptr[b + 1] = (double*)(A + C.lam_off[b]);
    C.gamma_tab = (cplx**)(A + C.tab_off);
    C.lam_tab = (double**)(A + C.tab_off + align_up(sizeof(cplx*) * N));
    C.chi_ext = (int*)(A + C.int_off);
    C.dsite_dev = (int*)(A + C.int_off + align_up(sizeof(int) * (N + 1)));
    C.cap_ext_dev = (int*)(A + C.int_off + 2 * align_up(sizeof(int) * (N + 1)));
    C.wbond = (double*)(A + C.wb_off);
    ok = cudaMemcpy(C.gamma_tab, C.gamma_ptr.data(), sizeof(cplx*) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(C.lam_tab, C.lam_ptr.data(), sizeof(double*) * (N + 1), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(C.dsite_dev, C.d.data(), sizeof(int) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(C.cap_ext_dev, C.cap_ext.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice) == cudaSuccess;
    C.dev.N = N;
    C.dev.chi_ext = C.chi_ext;
    C.dev.dsite = C.dsite_dev;
    C.dev.lam_ext = C.lam_tab;
    C.dev.gamma = C.gamma_tab;
    C.dev.cap_ext = C.cap_ext_dev;
  }
  const double one = 1.0;
  ok = ok && cudaMemcpy(h->one_lam, &one, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  char* ws = A + L.ws_off;
  const int max_batch = L.max_batch;
  for (int par = 0; par < 2 && ok; ++par) {
    ParitySet& ps = h->par[par];
    ps.dims = (Dims*)(A + L.desc_off + par * L.desc_per);
    ps.ptrs = (ProbPtr*)((char*)ps.dims + align_up(sizeof(Dims) * std::max(1, max_batch)));
    std::vector<ProbPtr> hp(ps.batch);
    for (const Wave& w : ps.waves) {
      size_t o = 0;
      for (int i = w.first; i < w.first + w.count; ++i) {
        const int c = ps.bonds[i].first, b = ps.bonds[i].second;
        ChainH& C = h->ch[c];
        ProbPtr& P = hp[i];
        memset(&P, 0, sizeof P);
        P.gl = C.gamma_ptr[b];
        P.gr = C.gamma_ptr[b + 1];
        P.laml = C.lam_ptr[b];
        P.lamm = C.lam_ptr[b + 1];
        P.lamr = C.lam_ptr[b + 2];
        P.gate = (const cplx*)(A + C.gate_off[b]);
        P.cap_l = C.cap_ext[b];
        P.cap_m = C.cap_ext[b + 1];
        P.cap_r = C.cap_ext[b + 2];
        P.chi_l = C.chi_ext + b;
        P.chi_m = C.chi_ext + b + 1;
        P.chi_r = C.chi_ext + b + 2;
        P.dl_s = C.d[b];
        P.dr_s = C.d[b + 1];
        P.chicap = C.chi_cap[b];
        P.bond_s = b;
        P.chain_s = (int)C.chain_index;
        P.slot = c;
        P.wbond = C.wbond + b;
        P.theta = (const cplx*)(ws + o);
        o += align_up(sizeof(cplx) * (size_t)C.d[b] * C.cap_ext[b] * C.d[b + 1] * C.cap_ext[b + 2]);
        if (C.d[b] * C.d[b + 1] >= GATE_GEMM_MIN) {
          P.Cpre = (cplx*)(ws + o);
          o += align_up(sizeof(cplx) * (size_t)C.d[b] * C.cap_ext[b] * C.d[b + 1] * C.cap_ext[b + 2]);
        }
        fill_ptrs(P, ws + o, L.lay[par][i]);
        o += L.lay[par][i].total;
      }
    }
    if (ps.batch > 0)
      ok = cudaMemcpy(ps.ptrs, hp.data(), sizeof(ProbPtr) * ps.batch, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  return ok;
}

extern "C" int tebd_create_multi(int n_chains, const tebd_desc_t* descs, tebd_t* out) {
  if (!out) return TEBD_EINVAL;
  *out = nullptr;
  tebd_s* h = new tebd_s();
  {
    const int rc = plan_handle(h, n_chains, descs, h->plan);
    if (rc != TEBD_OK) { delete h; return rc; }
  }
  const tebd_desc_t& d0 = descs[0];
  h->alloc.fn = d0.alloc;
  h->alloc.rel = d0.release;
  h->alloc.ctx = d0.alloc_ctx;
  if (h->use_graph) {
    // the legacy default stream cannot be captured: run on a blocking stream
    // of our own (it still orders with stream 0)
    if (cudaStreamCreate(&h->own_stream) != cudaSuccess) { cudaGetLastError(); delete h; return TEBD_ECUDA; }
    h->stream = h->own_stream;
  }
  {
    void* blk = nullptr;
    const int rc = h->alloc.get(h->arena_bytes, &blk);
    if (rc != TEBD_OK) {
      tebd_free(h);  // also the stream of our own
      return rc;
    }
    h->arena = (char*)blk;
  }
  if (cudaMemset(h->arena, 0, h->plan.ws_off) != cudaSuccess) { tebd_free(h); return TEBD_ECUDA; }
  if (prec_mixed(h->precision))
    for (int par = 0; par < 2; ++par)
      for (const Wave& w : h->par[par].waves)
        if (mixed_prepare(w.cap) != cudaSuccess) { cudaGetLastError(); tebd_free(h); return TEBD_ECUDA; }
  if (fused_prepare() != cudaSuccess) { cudaGetLastError(); tebd_free(h); return TEBD_ECUDA; }
  if (!bind_arena(h)) { tebd_free(h); return TEBD_ECUDA; }
  // every chain starts in |0...0>
  for (int c = 0; c < n_chains; ++c) {
    std::vector<double> psi;
    for (int s = 0; s < h->ch[c].N; ++s) {
      psi.push_back(1.0);
      psi.push_back(0.0);
      for (int i = 1; i < h->ch[c].d[s]; ++i) { psi.push_back(0.0); psi.push_back(0.0); }
    }
    const int rc = tebd_reset_state(h, c, psi.data());
    if (rc != TEBD_OK) { tebd_free(h); return rc; }
  }
  if (d0.fused == 1 && h->precision == TEBD_PREC_FP64)
    for (int par = 0; par < 2; ++par)
      for (Wave& w : h->par[par].waves) w.fused = fused_fits(w.cap) ? 1 : 0;
  if (d0.autotune && h->precision == TEBD_PREC_FP64) {
    Dims* scratch = (Dims*)(h->arena + h->plan.desc_off + 2 * h->plan.desc_per);
    for (int par = 0; par < 2; ++par)
      for (Wave& w : h->par[par].waves)
        if (tune_wave(h, h->par[par], w, h->stream, scratch, h->p, d0.fused) != 0) { tebd_free(h); return TEBD_ECUDA; }
    if (cudaDeviceSynchronize() != cudaSuccess) { tebd_free(h); return TEBD_ECUDA; }
  }
  if (d0.autotune && prec_mixed(h->precision)) {
    // the mixed form's launch choices, timed on synthetic theta at each
    // wave's capacity sizes (cached per wave shape for the process)
    Dims* scratch = (Dims*)(h->arena + h->plan.desc_off + 2 * h->plan.desc_per);
    for (int par = 0; par < 2; ++par)
      for (Wave& w : h->par[par].waves) {
        const ParitySet& ps = h->par[par];
        std::vector<long long> key = {100, w.cap.m, w.cap.n, w.cap.l, w.cap.k, w.count, h->q};
        {
          std::lock_guard<std::mutex> g(g_tile_mu);
          auto it = g_knob_cache.find(key);
          if (it != g_knob_cache.end()) { w.mk = it->second.first; w.tune_ms[0] = it->second.second[0]; w.tune_ms[1] = it->second.second[1]; continue; }
        }
        std::vector<Dims> hd(w.count);
        std::vector<ProbPtr> hp(w.count);
        bool ok = cudaMemcpy(hp.data(), ps.ptrs + w.first, sizeof(ProbPtr) * w.count, cudaMemcpyDeviceToHost) == cudaSuccess;
        for (int i = 0; i < w.count && ok; ++i) {
          Dims& D = hd[i];
          memset(&D, 0, sizeof D);
          D.dl = hp[i].dl_s; D.dr = hp[i].dr_s;
          D.cl = hp[i].cap_l; D.cm = hp[i].cap_m; D.cr = hp[i].cap_r;
          D.m = D.dl * D.cl; D.n = D.dr * D.cr;
          D.k = std::min(hp[i].chicap, std::min(D.m, D.n));
          D.l = std::min(D.k + h->p, std::min(D.m, D.n));
          D.active = 1;
        }
        ok = ok && cudaMemcpy(scratch, hd.data(), sizeof(Dims) * w.count, cudaMemcpyHostToDevice) == cudaSuccess &&
             launch_tune_theta(scratch, ps.ptrs + w.first, w.count, h->stream) == cudaSuccess;
        const MixedPtrs mp = mixed_carve(h->mixed, w.ms, w.count);
        auto run = [&](const MixedKnobs& k) {
          return run_rrsvd_mixed(scratch, ps.ptrs + w.first, w.count, w.cap, mp, h->q, h->seed, 0, 0, -1, h->status,
                                 h->tcerr, h->stream, h->sweep_dev, &k, h->precision == TEBD_PREC_BF16);
        };
        float ms[2] = {0.f, 0.f};
        if (!ok || tune_knobs(run, h->stream, w.cap, w.count, w.mk, ms) != 0) { tebd_free(h); return TEBD_ECUDA; }
        w.tune_ms[0] = ms[0];
        w.tune_ms[1] = ms[1];
        std::lock_guard<std::mutex> g(g_tile_mu);
        g_knob_cache[key] = {w.mk, {ms[0], ms[1]}};
      }
    if (cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess || cudaMemset(h->tcerr, 0, sizeof(int)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) { tebd_free(h); return TEBD_ECUDA; }
  }
  *out = h;
  return TEBD_OK;
}

extern "C" int tebd_create_ex(const tebd_desc_t* desc, tebd_t* out) { return tebd_create_multi(1, desc, out); }

extern "C" int tebd_create(int N, int d, int chi_max, int p, int q, uint64_t seed, tebd_t* out) {
  tebd_desc_t desc;
  memset(&desc, 0, sizeof desc);
  desc.N = N;
  desc.d = d;
  desc.chi_max = chi_max;
  desc.p = p;
  desc.q = q;
  desc.seed = seed;
  desc.precision = TEBD_PREC_FP64;
  return tebd_create_ex(&desc, out);
}

extern "C" int tebd_destroy(tebd_t h) {
  if (!h) return TEBD_OK;
  tebd_free(h);
  return TEBD_OK;
}

extern "C" int tebd_set_stream(tebd_t h, void* s) {
  if (!h) return TEBD_EINVAL;
  if (!s && h->own_stream) s = h->own_stream;
  if ((cudaStream_t)s != h->stream)
    for (int i = 0; i < 2; ++i)
      if (h->gexec[i]) { cudaGraphExecDestroy(h->gexec[i]); h->gexec[i] = nullptr; }
  h->stream = (cudaStream_t)s;
  return TEBD_OK;
}

extern "C" int tebd_set_allocator(tebd_t h, tebd_alloc_fn fn, tebd_release_fn rel, void* ctx) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if ((fn == nullptr) != (rel == nullptr)) {
    h->err.set(TEBD_EINVAL, "allocator: give both alloc and release, or neither");
    return h->err.code;
  }
  DevAlloc na;
  na.fn = fn;
  na.rel = rel;
  na.ctx = ctx;
  CU_OR(h, cudaStreamSynchronize(h->stream));
  // new blocks first: on failure the handle keeps its old ones
  void* nb = nullptr;
  int rc = na.get(h->arena_bytes, &nb);
  if (rc != TEBD_OK) {
    h->err.set(rc, "allocator: arena of %zu bytes %s", h->arena_bytes,
               rc == TEBD_ENOMEM ? "not available" : "not 256-byte aligned");
    return h->err.code;
  }
  const size_t cbytes = h->ch.empty() ? 0 : chain_region_end(h->ch[0]) - h->ch[0].gamma_lo;
  std::vector<char*> nck(h->ckpts.size(), nullptr);
  for (size_t i = 0; i < nck.size(); ++i) {
    void* q = nullptr;
    rc = na.get(cbytes, &q);
    if (rc != TEBD_OK) {
      for (size_t j = 0; j < i; ++j) na.put(nck[j]);
      na.put(nb);
      h->err.set(rc, "allocator: checkpoint of %zu bytes %s", cbytes,
                 rc == TEBD_ENOMEM ? "not available" : "not 256-byte aligned");
      return h->err.code;
    }
    nck[i] = (char*)q;
  }
  bool ok = cudaMemcpyAsync(nb, h->arena, h->arena_bytes, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess;
  for (size_t i = 0; i < nck.size() && ok; ++i)
    ok = cudaMemcpyAsync(nck[i], h->ckpts[i].buf, cbytes, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
  if (!ok) {
    for (char* q : nck) na.put(q);
    na.put(nb);
    h->err.set(TEBD_ECUDA, "allocator: copy into the new blocks failed");
    return h->err.code;
  }
  const DevAlloc old = h->alloc;
  char* old_arena = h->arena;
  h->arena = (char*)nb;
  ok = bind_arena(h);
  // the checkpoints carry copies of the chain's pointer tables, which a
  // restore writes back: point them at the new arena too
  for (size_t i = 0; i < nck.size() && ok; ++i) {
    const ChainH& C = h->ch[0];
    char* t = nck[i] + (C.tab_off - C.gamma_lo);
    ok = cudaMemcpy(t, C.gamma_ptr.data(), sizeof(cplx*) * C.N, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t + align_up(sizeof(cplx*) * C.N), C.lam_ptr.data(), sizeof(double*) * (C.N + 1),
                    cudaMemcpyHostToDevice) == cudaSuccess;
  }
  for (size_t i = 0; i < nck.size(); ++i) {
    old.put(h->ckpts[i].buf);
    h->ckpts[i].buf = nck[i];
  }
  old.put(h->adj_arena);  // made again from the new allocator when needed
  h->adj_arena = nullptr;
  h->gbar0 = nullptr;
  h->adj_dev[0] = h->adj_dev[1] = nullptr;
  old.put(old_arena);
  h->alloc = na;
  for (int i = 0; i < 2; ++i)
    if (h->gexec[i]) { cudaGraphExecDestroy(h->gexec[i]); h->gexec[i] = nullptr; }
  if (!ok) { h->err.set(TEBD_ECUDA, "allocator: rebinding the arena failed"); return h->err.code; }
  return TEBD_OK;
}

extern "C" int tebd_num_chains(tebd_t h, int* out) {
  if (!h || !out) return TEBD_EINVAL;
  *out = (int)h->ch.size();
  return TEBD_OK;
}

extern "C" int tebd_select_chain(tebd_t h, int chain) {
  if (!h) return TEBD_EINVAL;
  if (chain < 0 || chain >= (int)h->ch.size()) { h->err.set(TEBD_EINVAL, "chain %d out of range", chain); return h->err.code; }
  h->cur = chain;
  return TEBD_OK;
}

static int tebd_reset_state(tebd_t h, int slot, const double* psi) {
  ChainH& C = h->ch[slot];
  const int N = C.N;
  std::vector<char> gam(C.gamma_hi - C.gamma_lo, 0);
  size_t o = 0;
  for (int s = 0; s < N; ++s) {
    const int ds = C.d[s];
    double nrm = 0.0;
    for (int i = 0; i < 2 * ds; ++i) nrm += psi[o + i] * psi[o + i];
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      h->err.set(TEBD_ENUMERIC, "site %d: zero or non-finite amplitudes", s);
      return h->err.code;
    }
    nrm = 1.0 / sqrt(nrm);
    cplx* g = (cplx*)(gam.data() + (C.gamma_off[s] - C.gamma_lo));
    const size_t stride = (size_t)C.cap_ext[s] * C.cap_ext[s + 1];
    for (int i = 0; i < ds; ++i) g[i * stride] = cmk(psi[o + 2 * i] * nrm, psi[o + 2 * i + 1] * nrm);
    o += 2 * ds;
  }
  CU_OR(h, cudaMemcpyAsync(h->arena + C.gamma_lo, gam.data(), gam.size(), cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < N - 1; ++b) {
    std::vector<double> lam(C.cap_ext[b + 1], 0.0);
    lam[0] = 1.0;
    CU_OR(h, cudaMemcpyAsync(C.lam_ptr[b + 1], lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                             h->stream));
  }
  std::vector<int> chi(N + 1, 1);
  CU_OR(h, cudaMemcpyAsync(C.chi_ext, chi.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->stream));
  const double w0[2] = {0.0, 1.0};
  CU_OR(h, cudaMemcpyAsync(h->wacc + 2 * slot, w0, sizeof w0, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, cudaMemsetAsync(C.wbond, 0, sizeof(double) * (N - 1), h->stream));
  CU_OR(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  CU_OR(h, cudaMemsetAsync(h->sweep_dev, 0, sizeof(uint64_t), h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  h->sweeps = 0;
  return TEBD_OK;
}

extern "C" int tebd_set_product_state(tebd_t h, const double* psi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!psi) { h->err.set(TEBD_EINVAL, "psi is NULL"); return h->err.code; }
  return tebd_reset_state(h, h->cur, psi);
}

extern "C" int tebd_set_mps(tebd_t h, const double* const* gamma, const double* const* lambda, const int* chi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!gamma || !lambda || !chi) { h->err.set(TEBD_EINVAL, "NULL argument"); return h->err.code; }
  ChainH& C = h->ch[h->cur];
  const int N = C.N;
  std::vector<int> ce(N + 1, 1);
  for (int b = 0; b < N - 1; ++b) {
    if (chi[b] < 1 || chi[b] > C.cap_ext[b + 1]) {
      h->err.set(TEBD_EINVAL, "bond %d: chi %d outside [1, %d]", b, chi[b], C.cap_ext[b + 1]);
      return h->err.code;
    }
    ce[b + 1] = chi[b];
  }
  std::vector<char> gam(C.gamma_hi - C.gamma_lo, 0);
  for (int s = 0; s < N; ++s) {
    if (!gamma[s]) { h->err.set(TEBD_EINVAL, "gamma[%d] is NULL", s); return h->err.code; }
    cplx* g = (cplx*)(gam.data() + (C.gamma_off[s] - C.gamma_lo));
    const int cl = ce[s], cr = ce[s + 1], capl = C.cap_ext[s], capr = C.cap_ext[s + 1];
    for (int i = 0; i < C.d[s]; ++i)
      for (int a = 0; a < cl; ++a)
        for (int c = 0; c < cr; ++c) {
          const size_t src = 2 * (((size_t)i * cl + a) * cr + c);
          g[((size_t)i * capl + a) * capr + c] = cmk(gamma[s][src], gamma[s][src + 1]);
        }
  }
  CU_OR(h, cudaMemcpyAsync(h->arena + C.gamma_lo, gam.data(), gam.size(), cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < N - 1; ++b) {
    if (!lambda[b]) { h->err.set(TEBD_EINVAL, "lambda[%d] is NULL", b); return h->err.code; }
    std::vector<double> lam(C.cap_ext[b + 1], 0.0);
    for (int i = 0; i < chi[b]; ++i) lam[i] = lambda[b][i];
    CU_OR(h, cudaMemcpyAsync(C.lam_ptr[b + 1], lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                             h->stream));
  }
  CU_OR(h, cudaMemcpyAsync(C.chi_ext, ce.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->stream));
  const double w0[2] = {0.0, 1.0};
  CU_OR(h, cudaMemcpyAsync(h->wacc + 2 * h->cur, w0, sizeof w0, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, cudaMemsetAsync(C.wbond, 0, sizeof(double) * (N - 1), h->stream));
  CU_OR(h, cudaMemsetAsync(h->sweep_dev, 0, sizeof(uint64_t), h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  h->sweeps = 0;
  return TEBD_OK;
}

extern "C" int tebd_get_mps(tebd_t h, double* const* gamma, double* const* lambda, int* chi) {
  if (!h) return TEBD_EINVAL;
  if (tebd_check_status(h)) return h->err.code;
  ChainH& C = h->ch[h->cur];
  const int N = C.N;
  std::vector<int> ce(N + 1);
  CU_OR(h, cudaMemcpy(ce.data(), C.chi_ext, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost));
  if (chi)
    for (int b = 0; b < N - 1; ++b) chi[b] = ce[b + 1];
  if (gamma) {
    std::vector<char> gam(C.gamma_hi - C.gamma_lo);
    CU_OR(h, cudaMemcpy(gam.data(), h->arena + C.gamma_lo, gam.size(), cudaMemcpyDeviceToHost));
    for (int s = 0; s < N; ++s) {
      if (!gamma[s]) continue;
      const cplx* g = (const cplx*)(gam.data() + (C.gamma_off[s] - C.gamma_lo));
      const int cl = ce[s], cr = ce[s + 1], capl = C.cap_ext[s], capr = C.cap_ext[s + 1];
      for (int i = 0; i < C.d[s]; ++i)
        for (int a = 0; a < cl; ++a)
          for (int c = 0; c < cr; ++c) {
            const cplx v = g[((size_t)i * capl + a) * capr + c];
            const size_t dst = 2 * (((size_t)i * cl + a) * cr + c);
            gamma[s][dst] = v.x;
            gamma[s][dst + 1] = v.y;
          }
    }
  }
  if (lambda)
    for (int b = 0; b < N - 1; ++b) {
      if (!lambda[b]) continue;
      CU_OR(h, cudaMemcpy(lambda[b], C.lam_ptr[b + 1], sizeof(double) * ce[b + 1], cudaMemcpyDeviceToHost));
    }
  return TEBD_OK;
}

extern "C" int tebd_set_gates(tebd_t h, int parity, const double* gates) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if ((parity != 0 && parity != 1) || !gates) { h->err.set(TEBD_EINVAL, "bad parity or NULL gates"); return h->err.code; }
  ChainH& C = h->ch[h->cur];
  size_t o = 0;
  for (int b = 0; b < C.N - 1; ++b) {
    const size_t dd = (size_t)C.d[b] * C.d[b + 1];
    if (b % 2 == parity) {
      if (!all_finite(gates + o, 2 * dd * dd)) {
        h->err.set(TEBD_ENUMERIC, "gate of bond %d has a non-finite entry", b);
        return h->err.code;
      }
      CU_OR(h, cudaMemcpyAsync(h->arena + C.gate_off[b], gates + o, sizeof(cplx) * dd * dd, cudaMemcpyHostToDevice,
                               h->stream));
    }
    o += 2 * dd * dd;
  }
  CU_OR(h, cudaStreamSynchronize(h->stream));
  C.gates_set[parity] = true;
  return TEBD_OK;
}

// The launch sequence of one sweep: per wave, sizes -> theta -> RRSVD ->
// rebuild -> weights; then the device sweep counter advances.
static cudaError_t enqueue_sweep(tebd_t h, int parity) {
  ParitySet& ps = h->par[parity];
  for (const Wave& w : ps.waves) {
    Dims* dims = ps.dims + w.first;
    ProbPtr* ptrs = ps.ptrs + w.first;
    const bool tuned = w.tiles[0] != 0;
    cudaError_t e;
    if (w.fused) {
      // the whole update of every bond of the wave in one persistent launch
      if ((e = launch_bond_fused(ptrs, dims, nullptr, w.count, h->p, h->q, h->seed, h->sweep_dev, h->cutoff,
                                 h->wout + w.first, h->status, h->queue, h->stream)) != cudaSuccess)
        return e;
      if ((e = launch_wacc(dims, ptrs, h->wout + w.first, w.count, h->wacc, h->stream)) != cudaSuccess) return e;
      continue;
    }
    if ((e = launch_plan(ptrs, dims, w.count, h->p, h->stream)) != cudaSuccess) return e;
    if (prec_mixed(h->precision)) {
      // bonds of large local dimensions: contraction and gate as GEMMs, on
      // the tensor cores from digit splits or in double-float arithmetic
      if ((e = launch_theta(dims, ptrs, w.count, w.cap, h->stream, 0, 1)) != cudaSuccess) return e;
      if (oz_gate_rule(w.cap) && w.mk.dfg != 2) {
        const MixedPtrs mp = mixed_carve(h->mixed, w.ms, w.count);
        const OzScratch oz{mp.gad, mp.gas, mp.gbd, mp.gbs};
        if ((e = launch_oz_stage(OZ_THETA_STAGE, dims, ptrs, w.count, w.cap, oz, h->tcerr, h->stream)) != cudaSuccess)
          return e;
        if ((e = launch_oz_stage(OZ_GATE_STAGE, dims, ptrs, w.count, w.cap, oz, h->tcerr, h->stream)) != cudaSuccess)
          return e;
      } else {
        if ((e = launch_theta_df(dims, ptrs, w.count, w.cap, h->stream)) != cudaSuccess) return e;
        if ((e = launch_gate_gemm_df(dims, ptrs, w.count, w.cap, h->stream)) != cudaSuccess) return e;
      }
    } else {
      if ((e = launch_theta(dims, ptrs, w.count, w.cap, h->stream)) != cudaSuccess) return e;
      if ((e = launch_gate_gemm(dims, ptrs, w.count, w.cap, h->stream)) != cudaSuccess) return e;
    }
    if (prec_mixed(h->precision)) {
      const MixedPtrs mp = mixed_carve(h->mixed, w.ms, w.count);
      if ((e = run_rrsvd_mixed(dims, ptrs, w.count, w.cap, mp, h->q, h->seed, 0, 0, -1, h->status, h->tcerr,
                               h->stream, h->sweep_dev, &w.mk, h->precision == TEBD_PREC_BF16)) != cudaSuccess)
        return e;
    } else if ((e = run_rrsvd(dims, ptrs, w.count, w.cap, h->q, h->seed, 0, 0, -1, h->status, h->stream,
                              h->sweep_dev, tuned ? w.tiles : nullptr)) != cudaSuccess) {
      return e;
    }
    if ((e = launch_rebuild(dims, ptrs, w.count, h->cutoff, h->wout + w.first, h->status, h->stream)) != cudaSuccess)
      return e;
    if ((e = launch_wacc(dims, ptrs, h->wout + w.first, w.count, h->wacc, h->stream)) != cudaSuccess) return e;
  }
  return launch_sweep_tick(h->sweep_dev, h->stream);
}

static int tebd_step(tebd_t h, int parity) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  for (size_t c = 0; c < h->ch.size(); ++c)
    if (!h->ch[c].gates_set[parity]) {
      h->err.set(TEBD_ESTATE, "gates of parity %d not set (chain %d)", parity, (int)c);
      return h->err.code;
    }
  if (h->recording) {
    const ChainH& C = h->ch[0];
    const size_t bytes = chain_region_end(C) - C.gamma_lo;
    void* blk = nullptr;
    const int rc = h->alloc.get(bytes, &blk);
    if (rc != TEBD_OK) {
      h->err.set(rc, "checkpoint of %zu bytes failed", bytes);
      return h->err.code;
    }
    char* buf = (char*)blk;
    h->ckpts.push_back({parity, h->sweeps, buf});
    CU_OR(h, cudaMemcpyAsync(buf, h->arena + C.gamma_lo, bytes, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (h->use_graph && !prof_on()) {
    if (!h->gexec[parity]) {
      cudaGraph_t g = nullptr;
      CU_OR(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t e = enqueue_sweep(h, parity);
      const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        h->err.set(TEBD_ECUDA, "sweep capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        return h->err.code;
      }
      const cudaError_t e3 = cudaGraphInstantiate(&h->gexec[parity], g, 0);
      cudaGraphDestroy(g);
      if (e3 != cudaSuccess) {
        h->gexec[parity] = nullptr;
        h->err.set(TEBD_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e3));
        return h->err.code;
      }
    }
    CU_OR(h, cudaGraphLaunch(h->gexec[parity], h->stream));
  } else {
    CU_OR(h, enqueue_sweep(h, parity));
  }
  h->sweeps++;
  return TEBD_OK;
}

extern "C" int tebd_step_even(tebd_t h) { return tebd_step(h, 0); }
extern "C" int tebd_step_odd(tebd_t h) { return tebd_step(h, 1); }

extern "C" int tebd_expect(tebd_t h, int site, const double* op, double* out) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  ChainH& C = h->ch[h->cur];
  if (site < 0 || site >= C.N || !op || !out) { h->err.set(TEBD_EINVAL, "bad site or NULL pointer"); return h->err.code; }
  const int d = C.d[site];
  CU_OR(h, cudaMemcpyAsync(h->op_dev, op, sizeof(cplx) * d * d, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, launch_expect(C.dev, site, h->op_dev, d, h->out_dev, h->stream));
  CU_OR(h, cudaMemcpyAsync(out, h->out_dev, sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  return tebd_check_status(h);
}

extern "C" int tebd_get_lambda(tebd_t h, int bond, double* out, int* chi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  ChainH& C = h->ch[h->cur];
  if (bond < 0 || bond >= C.N - 1 || !out) { h->err.set(TEBD_EINVAL, "bad bond or NULL pointer"); return h->err.code; }
  int c = 0;
  CU_OR(h, cudaMemcpyAsync(&c, C.chi_ext + bond + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU_OR(h, cudaMemcpyAsync(out, C.lam_ptr[bond + 1], sizeof(double) * C.cap_ext[bond + 1], cudaMemcpyDeviceToHost,
                           h->stream));
  if (tebd_check_status(h)) return h->err.code;
  if (chi) *chi = c;
  return TEBD_OK;
}

extern "C" int tebd_discarded_weight(tebd_t h, double* out) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!out) { h->err.set(TEBD_EINVAL, "NULL pointer"); return h->err.code; }
  CU_OR(h, cudaMemcpyAsync(out, h->wacc + 2 * h->cur, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return tebd_check_status(h);
}

extern "C" int tebd_sweep_count(tebd_t h, int64_t* out) {
  if (!h || !out) return TEBD_EINVAL;
  *out = h->sweeps;
  return TEBD_OK;
}

extern "C" int tebd_set_sweep_count(tebd_t h, int64_t count) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (count < 0) { h->err.set(TEBD_EINVAL, "sweep count %lld < 0", (long long)count); return h->err.code; }
  const uint64_t c = (uint64_t)count;
  CU_OR(h, cudaMemcpyAsync(h->sweep_dev, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  h->sweeps = count;
  return TEBD_OK;
}

extern "C" int tebd_bond_weights(tebd_t h, double* out) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!out) { h->err.set(TEBD_EINVAL, "NULL pointer"); return h->err.code; }
  const ChainH& C = h->ch[h->cur];
  CU_OR(h, cudaMemcpyAsync(out, C.wbond, sizeof(double) * (C.N - 1), cudaMemcpyDeviceToHost, h->stream));
  return tebd_check_status(h);
}

extern "C" int tebd_wave_info(tebd_t h, int parity, int wave, int* info, double* ms) {
  if (!h) return TEBD_EINVAL;
  if (parity < 0 || parity > 1 || wave < 0 || wave >= (int)h->par[parity].waves.size()) return TEBD_EINVAL;
  const Wave& w = h->par[parity].waves[wave];
  if (info) {
    memset(info, 0, sizeof(int) * 20);
    info[0] = w.count;
    info[1] = w.cap.m; info[2] = w.cap.n; info[3] = w.cap.k; info[4] = w.cap.l;
    info[5] = w.fused;
    for (int i = 0; i < 6; ++i) info[6 + i] = w.tiles[i];
    info[12] = w.mk.tc_half; info[13] = w.mk.qr_threads; info[14] = w.mk.qrbh; info[15] = w.mk.jac;
    info[16] = w.mk.dfg;
  }
  if (ms) {
    ms[0] = w.tune_ms[0];
    ms[1] = w.tune_ms[1];
  }
  return TEBD_OK;
}

extern "C" int tebd_workspace_info(tebd_t h, size_t* arena_bytes, int* waves_even, int* waves_odd) {
  if (!h) return TEBD_EINVAL;
  if (arena_bytes) *arena_bytes = h->arena_bytes;
  if (waves_even) *waves_even = (int)h->par[0].waves.size();
  if (waves_odd) *waves_odd = (int)h->par[1].waves.size();
  return TEBD_OK;
}

// Adjoint scratch and cotangent buffers of a single-chain handle (capacity sizes).
static int tebd_adj_alloc(tebd_t h) {
  if (h->adj_arena) return TEBD_OK;
  const ChainH& C = h->ch[0];
  const int N = C.N;
  const size_t c16 = sizeof(cplx), c8 = sizeof(double);
  // cotangent state: Gamma_bar per site, lambda_bar per bond
  std::vector<size_t> goff(N), loff(N - 1);
  size_t off = 0;
  for (int s = 0; s < N; ++s) {
    goff[s] = off;
    off += align_up(c16 * (size_t)C.d[s] * C.cap_ext[s] * C.cap_ext[s + 1]);
  }
  for (int b = 0; b < N - 1; ++b) {
    loff[b] = off;
    off += align_up(c8 * C.cap_ext[b + 1]);
  }
  const size_t cot_bytes = off;
  struct Sz { size_t th, ur, vr, kk, pb, rb, sb, xb, yb, zb, gb; };
  std::vector<Sz> sz[2];
  std::vector<size_t> poff[2];
  for (int par = 0; par < 2; ++par)
    for (const auto& bb : h->par[par].bonds) {
      const int b = bb.second;
      const size_t m = (size_t)C.d[b] * C.cap_ext[b], n = (size_t)C.d[b + 1] * C.cap_ext[b + 2];
      const size_t kc = std::min<size_t>(C.cap_ext[b + 1], std::min(m, n)), cm = C.cap_ext[b + 1];
      const size_t dd = (size_t)C.d[b] * C.d[b + 1];
      Sz z{align_up(c16 * m * n), align_up(c16 * m * kc), align_up(c16 * n * kc), align_up(c16 * kc * kc),
           align_up(c16 * m * cm), align_up(c16 * cm * n), align_up(c8 * kc), align_up(c8 * C.cap_ext[b]),
           align_up(c8 * cm), align_up(c8 * C.cap_ext[b + 2]), align_up(c16 * dd * dd)};
      sz[par].push_back(z);
      poff[par].push_back(off);
      off += 3 * z.th + 2 * z.ur + 2 * z.vr + 3 * z.kk + z.pb + z.rb + z.sb + z.xb + z.yb + z.zb + z.gb;
    }
  const size_t desc_off = off;
  for (int par = 0; par < 2; ++par) off += align_up(sizeof(AdjPtr) * std::max<size_t>(1, h->par[par].bonds.size()));
  {
    void* blk = nullptr;
    const int rc = h->alloc.get(off, &blk);
    if (rc != TEBD_OK) {
      h->adj_arena = nullptr;
      h->err.set(rc, "reverse-pass buffers of %zu bytes failed", off);
      return h->err.code;
    }
    h->adj_arena = (char*)blk;
  }
  char* A = h->adj_arena;
  h->gbar0 = (cplx*)A;
  h->cot_bytes = cot_bytes;
  size_t doff = desc_off;
  for (int par = 0; par < 2; ++par) {
    ParitySet& ps = h->par[par];
    std::vector<AdjPtr> hp(ps.bonds.size());
    for (size_t i = 0; i < ps.bonds.size(); ++i) {
      const int b = ps.bonds[i].second;
      const Sz& z = sz[par][i];
      char* q = A + poff[par][i];
      AdjPtr& P = hp[i];
      P.th0 = (cplx*)q; q += z.th;
      P.Mbar = (cplx*)q; q += z.th;
      P.Tbar = (cplx*)q; q += z.th;
      P.Ubar = (cplx*)q; q += z.ur;
      P.T1 = (cplx*)q; q += z.ur;
      P.Vbar = (cplx*)q; q += z.vr;
      P.Pv = (cplx*)q; q += z.vr;
      P.Gu = (cplx*)q; q += z.kk;
      P.Gv = (cplx*)q; q += z.kk;
      P.Cm = (cplx*)q; q += z.kk;
      P.Pbar = (cplx*)q; q += z.pb;
      P.Rbar = (cplx*)q; q += z.rb;
      P.Sbar = (double*)q; q += z.sb;
      P.xbar = (double*)q; q += z.xb;
      P.ybar = (double*)q; q += z.yb;
      P.zbar = (double*)q; q += z.zb;
      P.Gbar = (cplx*)q; q += z.gb;
      P.gbar_l = (cplx*)(A + goff[b]);
      P.gbar_r = (cplx*)(A + goff[b + 1]);
      P.lbar = (double*)(A + loff[b]);
      P.lbar_l = b > 0 ? (double*)(A + loff[b - 1]) : nullptr;
      P.lbar_r = b + 1 < N - 1 ? (double*)(A + loff[b + 1]) : nullptr;
    }
    h->adj_dev[par] = (AdjPtr*)(A + doff);
    doff += align_up(sizeof(AdjPtr) * std::max<size_t>(1, ps.bonds.size()));
    if (!hp.empty() && cudaMemcpy(h->adj_dev[par], hp.data(), sizeof(AdjPtr) * hp.size(), cudaMemcpyHostToDevice) !=
                           cudaSuccess) {
      h->err.set(TEBD_ECUDA, "reverse-pass descriptors upload failed");
      return h->err.code;
    }
  }
  return TEBD_OK;
}

extern "C" int tebd_record(tebd_t h, int on) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (h->ch.size() != 1) { h->err.set(TEBD_ENOTIMPL, "recording needs a single-chain handle"); return h->err.code; }
  if (h->precision != TEBD_PREC_FP64) {
    h->err.set(TEBD_ENOTIMPL, "the reverse pass differentiates the FP64 form");
    return h->err.code;
  }
  if (on) {
    CU_OR(h, cudaStreamSynchronize(h->stream));
    free_ckpts(h);
    if (tebd_adj_alloc(h) != TEBD_OK) return h->err.code;
  }
  h->recording = on != 0;
  return TEBD_OK;
}

extern "C" int tebd_backward(tebd_t h, int site, const double* op, double* dgates_even, double* dgates_odd) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (h->ch.size() != 1) { h->err.set(TEBD_ENOTIMPL, "the reverse pass needs a single-chain handle"); return h->err.code; }
  ChainH& C = h->ch[0];
  const int N = C.N;
  if (site < 0 || site >= N || !op) { h->err.set(TEBD_EINVAL, "bad site or NULL op"); return h->err.code; }
  if (h->ckpts.empty()) { h->err.set(TEBD_ESTATE, "no recorded sweeps"); return h->err.code; }
  if (tebd_adj_alloc(h) != TEBD_OK) return h->err.code;
  if (tebd_check_status(h)) return h->err.code;
  cudaStream_t st = h->stream;
  const size_t rbytes = chain_region_end(C) - C.gamma_lo;
  char* region = h->arena + C.gamma_lo;
  // keep the final state, sweep counter and weights to restore them afterwards
  char* save = nullptr;
  {
    void* blk = nullptr;
    const int arc = h->alloc.get(rbytes + 2 * ALIGN + align_up(sizeof(double) * 2 * h->ch.size()), &blk);
    if (arc != TEBD_OK) {
      h->err.set(arc, "reverse-pass save buffer failed");
      return h->err.code;
    }
    save = (char*)blk;
  }
  int rc = TEBD_OK;
  do {
    if (cudaMemcpyAsync(save, region, rbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(save + rbytes, h->sweep_dev, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(save + rbytes + ALIGN, h->wacc, sizeof(double) * 2 * h->ch.size(), cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess ||
        cudaMemsetAsync(h->gbar0, 0, h->cot_bytes, st) != cudaSuccess) { rc = TEBD_ECUDA; break; }
    for (int par = 0; par < 2 && rc == TEBD_OK; ++par) {
      std::vector<AdjPtr> hp(h->par[par].bonds.size());
      if (!hp.empty() && cudaMemcpy(hp.data(), h->adj_dev[par], sizeof(AdjPtr) * hp.size(), cudaMemcpyDeviceToHost) != cudaSuccess) rc = TEBD_ECUDA;
      for (size_t i = 0; i < hp.size() && rc == TEBD_OK; ++i) {
        const int b = h->par[par].bonds[i].second;
        const size_t dd = (size_t)C.d[b] * C.d[b + 1];
        if (cudaMemsetAsync(hp[i].Gbar, 0, sizeof(cplx) * dd * dd, st) != cudaSuccess) rc = TEBD_ECUDA;
      }
    }
    if (rc) break;
    // L = Re <O_site> with the Hermitian part of O
    const int d = C.d[site];
    std::vector<cplx> oh(d * d);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        oh[i * d + j] = cmk(0.5 * (op[2 * (i * d + j)] + op[2 * (j * d + i)]),
                            0.5 * (op[2 * (i * d + j) + 1] - op[2 * (j * d + i) + 1]));
    std::vector<int> ce(N + 1);
    if (cudaMemcpyAsync(h->op_dev, oh.data(), sizeof(cplx) * d * d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ce.data(), C.chi_ext, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = TEBD_ECUDA; break; }
    // cotangent buffers of site and its bonds: the Gamma block comes first,
    // then the lambdas in bond order (same layout as tebd_adj_alloc)
    std::vector<size_t> goff(N), loff(N - 1);
    size_t off = 0;
    for (int s = 0; s < N; ++s) { goff[s] = off; off += align_up(sizeof(cplx) * (size_t)C.d[s] * C.cap_ext[s] * C.cap_ext[s + 1]); }
    for (int b = 0; b < N - 1; ++b) { loff[b] = off; off += align_up(sizeof(double) * C.cap_ext[b + 1]); }
    char* cb = (char*)h->gbar0;
    if (launch_adj_expect(C.gamma_ptr[site], d, ce[site], ce[site + 1], C.cap_ext[site], C.cap_ext[site + 1],
                          C.lam_ptr[site], C.lam_ptr[site + 1], h->op_dev, (cplx*)(cb + goff[site]),
                          site > 0 ? (double*)(cb + loff[site - 1]) : nullptr,
                          site < N - 1 ? (double*)(cb + loff[site]) : nullptr, st) != cudaSuccess) { rc = TEBD_ECUDA; break; }
    for (int k = (int)h->ckpts.size() - 1; k >= 0 && rc == TEBD_OK; --k) {
      const tebd_s::Ckpt& ck = h->ckpts[k];
      const uint64_t sw = (uint64_t)ck.sweep;
      if (cudaMemcpyAsync(region, ck.buf, rbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(h->sweep_dev, &sw, sizeof sw, cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = TEBD_ECUDA; break; }
      ParitySet& ps = h->par[ck.parity];
      for (const Wave& w : ps.waves) {
        Dims* dims = ps.dims + w.first;
        ProbPtr* ptrs = ps.ptrs + w.first;
        AdjPtr* adj = h->adj_dev[ck.parity] + w.first;
        const bool tuned = w.tiles[0] != 0;
        if (launch_plan(ptrs, dims, w.count, h->p, st) != cudaSuccess ||
            launch_theta(dims, ptrs, w.count, w.cap, st, 1) != cudaSuccess ||
            launch_adj_keep_theta(dims, ptrs, adj, w.count, st) != cudaSuccess ||
            launch_theta(dims, ptrs, w.count, w.cap, st) != cudaSuccess ||
            launch_gate_gemm(dims, ptrs, w.count, w.cap, st) != cudaSuccess ||
            run_rrsvd(dims, ptrs, w.count, w.cap, h->q, h->seed, 0, 0, -1, h->status, st, h->sweep_dev,
                      tuned ? w.tiles : nullptr) != cudaSuccess ||
            launch_rebuild(dims, ptrs, w.count, h->cutoff, h->wout + w.first, h->status, st) != cudaSuccess ||
            launch_adj_bond(dims, ptrs, adj, w.count, region, region + rbytes, ck.buf, h->cutoff, 1e-24, 1e-24,
                            st) != cudaSuccess ||
            launch_adj_accum(dims, adj, w.count, st) != cudaSuccess) { rc = TEBD_ECUDA; break; }
      }
    }
    if (rc) break;
    // gate cotangents, summed over the applications of each parity
    for (int par = 0; par < 2 && rc == TEBD_OK; ++par) {
      double* out = par == 0 ? dgates_even : dgates_odd;
      if (!out) continue;
      std::vector<AdjPtr> hp(h->par[par].bonds.size());
      if (!hp.empty() && cudaMemcpy(hp.data(), h->adj_dev[par], sizeof(AdjPtr) * hp.size(), cudaMemcpyDeviceToHost) != cudaSuccess) { rc = TEBD_ECUDA; break; }
      size_t o = 0;
      std::vector<size_t> boff(N - 1);
      for (int b = 0; b < N - 1; ++b) { boff[b] = o; o += 2 * (size_t)C.d[b] * C.d[b + 1] * C.d[b] * C.d[b + 1]; }
      memset(out, 0, sizeof(double) * o);
      for (size_t i = 0; i < hp.size(); ++i) {
        const int b = h->par[par].bonds[i].second;
        const size_t dd = (size_t)C.d[b] * C.d[b + 1];
        if (cudaMemcpy(out + boff[b], hp[i].Gbar, sizeof(cplx) * dd * dd, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = TEBD_ECUDA; break; }
      }
    }
  } while (0);
  // restore the forward state whatever happened above
  cudaMemcpyAsync(region, save, rbytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(h->sweep_dev, save + rbytes, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(h->wacc, save + rbytes + ALIGN, sizeof(double) * 2 * h->ch.size(), cudaMemcpyDeviceToDevice, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  h->alloc.put(save);
  if (rc == TEBD_OK && e != cudaSuccess) rc = TEBD_ECUDA;
  if (rc != TEBD_OK) {
    h->err.set(rc, "reverse pass failed: %s", cudaGetErrorString(cudaGetLastError()));
    return h->err.code;
  }
  return tebd_check_status(h);
}

extern "C" const char* tebd_last_error(tebd_t h) { return h ? h->err.msg.c_str() : "NULL handle"; }

// ===========================================================================
// Standalone RRSVD plan
// ===========================================================================
struct rrsvd_plan_s {
  ErrState err;
  int m = 0, n = 0, k = 0, l = 0, p = 0, q = 0, batch = 0, precision = 0;
  uint64_t seed = 0;
  Caps cap{};
  WsLayout lay{};
  size_t per = 0, ws_bytes = 0;
  char* meta = nullptr;  // device: dims, ptrs, status, tensor-core error flag
  Dims* dims = nullptr;
  ProbPtr* ptrs = nullptr;
  int* status = nullptr;
  int* tcerr = nullptr;
  size_t mixed_off = 0;  // start of the mixed-precision arrays in the workspace
  MixedSizes ms{};
  // accuracy check (Alg. 2); check_r == 0: fixed rank
  int check_r = 0, l_max = 0, rounds = 0, k0 = 0, l0 = 0;
  double eps = 0.0;
  // host-path staging (allocated on first use) and the streams / events of
  // its pipelined sub-batches (created on first use)
  char* stage = nullptr;
  size_t stage_bytes = 0;
  static const int HCH = 4;
  cudaStream_t hs[HCH] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t hev[HCH + 1] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // asynchronous host path: two staging slots (theta in, results out) used in
  // turn, one workspace, copy-in and copy-out streams, and per slot the
  // events "copied in", "computed", "copied out"
  char* aslot[2] = {nullptr, nullptr};
  char* aws = nullptr;
  cudaStream_t acs = nullptr, aos = nullptr, astream = nullptr;
  cudaEvent_t a_call = nullptr, a_in[2] = {nullptr, nullptr}, a_comp[2] = {nullptr, nullptr},
              a_out[2] = {nullptr, nullptr};
  int anext = 0, apending = 0;
  // autotuner choices (rrsvd_plan_autotune): FP64 GEMM tiles, mixed-form knobs
  int tiles[6] = {0, 0, 0, 0, 0, 0};
  MixedKnobs mk{0, 0, 0, 0, 0};
  float tune_ms[2] = {0.f, 0.f};
  int tuned = 0;
};

namespace tg {
__global__ void k_rrsvd_bind(ProbPtr* ptrs, int batch, char* ws, size_t per, WsLayout lay, const cplx* theta,
                             size_t theta_stride, cplx* U, size_t U_stride, cplx* Vh, size_t V_stride, Dims* dims,
                             int dims_m, int dims_n, int dims_k, int dims_l, int* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (dims_m > 0 && p == 0) *status = 0;
  if (p >= batch) return;
  ProbPtr P;
  memset(&P, 0, sizeof P);
  fill_ptrs(P, ws + per * (size_t)p, lay);
  P.theta = theta + theta_stride * p;
  if (U) P.U = U + U_stride * p;
  if (Vh) P.V = Vh + V_stride * p;
  ptrs[p] = P;
  if (dims_m > 0) {
    Dims D;
    memset(&D, 0, sizeof D);
    D.m = dims_m; D.n = dims_n; D.k = dims_k; D.l = dims_l; D.bond = 0; D.active = 1;
    dims[p] = D;
  }
}
}  // namespace tg

extern "C" int rrsvd_plan_create_ex(int m, int n, int k_max, int p, int q, int batch, int precision,
                                    uint64_t seed, int check_r, double check_eps, int l_max, rrsvd_plan_t* out) {
  if (!out) return TEBD_EINVAL;
  *out = nullptr;
  if (m < 1 || n < 1 || k_max < 1 || p < 0 || q < 0 || batch < 1 || check_r < 0) return TEBD_EINVAL;
  if (precision != TEBD_PREC_FP64 && !prec_mixed(precision)) return TEBD_ENOTIMPL;
  if (check_r > 0 && (precision != TEBD_PREC_FP64 || !(check_eps > 0.0))) return check_eps > 0.0 ? TEBD_ENOTIMPL : TEBD_EINVAL;
  rrsvd_plan_s* P = new rrsvd_plan_s();
  P->m = m; P->n = n; P->p = p; P->q = q; P->batch = batch; P->precision = precision; P->seed = seed;
  P->k = std::min(k_max, std::min(m, n));
  P->l = std::min(P->k + p, std::min(m, n));
  P->k0 = P->k;
  P->l0 = P->l;
  if (check_r > 0) {
    P->check_r = check_r;
    P->eps = check_eps;
    P->l_max = std::min(std::max(l_max, P->l), std::min(m, n));
    P->rounds = (P->l_max - P->l0) / check_r + 1;
    P->l = P->l_max;                           // capacities
    P->k = std::max(1, P->l_max - p);
    if (P->k < P->k0) P->k = P->k0;
  }
  if (P->l > 512) { delete P; return TEBD_ENOTIMPL; }
  P->cap.m = m; P->cap.n = n; P->cap.k = P->k; P->cap.l = P->l; P->cap.r = check_r;
  // workspace always holds U and Vh so that either may be NULL at execute
  P->lay = ws_layout(m, n, P->k, P->l, true, true, check_r);
  P->per = P->lay.total;
  P->ws_bytes = P->per * (size_t)batch;
  if (prec_mixed(precision)) {
    P->ms = mixed_sizes(m, n, P->k, P->l, precision == TEBD_PREC_BF16);
    P->mixed_off = P->ws_bytes;
    P->ws_bytes += mixed_bytes(P->ms, batch);
  }
  const size_t meta = align_up(sizeof(Dims) * batch) + align_up(sizeof(ProbPtr) * batch) + 2 * ALIGN;
  if (fault_take(TEBD_FAULT_ALLOC) || cudaMalloc(&P->meta, meta) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return TEBD_ENOMEM;
  }
  P->dims = (Dims*)P->meta;
  P->ptrs = (ProbPtr*)(P->meta + align_up(sizeof(Dims) * batch));
  P->status = (int*)(P->meta + align_up(sizeof(Dims) * batch) + align_up(sizeof(ProbPtr) * batch));
  P->tcerr = (int*)((char*)P->status + ALIGN);
  std::vector<Dims> hd(batch);
  for (int i = 0; i < batch; ++i) {
    Dims& D = hd[i];
    memset(&D, 0, sizeof D);
    D.m = m; D.n = n; D.k = P->k; D.l = P->l; D.bond = 0; D.active = 1;
  }
  if (cudaMemcpy(P->dims, hd.data(), sizeof(Dims) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(P->status, 0, 2 * ALIGN) != cudaSuccess) {
    cudaFree(P->meta);
    delete P;
    return TEBD_ECUDA;
  }
  *out = P;
  return TEBD_OK;
}

extern "C" int rrsvd_plan_create(int m, int n, int k_max, int p, int q, int batch, int precision, uint64_t seed,
                                 rrsvd_plan_t* out) {
  return rrsvd_plan_create_ex(m, n, k_max, p, q, batch, precision, seed, 0, 0.0, 0, out);
}

extern "C" int rrsvd_plan_destroy(rrsvd_plan_t P) {
  if (!P) return TEBD_OK;
  if (P->meta) cudaFree(P->meta);
  if (P->stage) cudaFree(P->stage);
  for (cudaStream_t& h : P->hs)
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t& e : P->hev)
    if (e) cudaEventDestroy(e);
  if (P->apending) {  // finish the pending calls before their buffers go
    if (P->astream) cudaStreamSynchronize(P->astream);
    if (P->aos) cudaStreamSynchronize(P->aos);
  }
  for (char* b : P->aslot)
    if (b) cudaFree(b);
  if (P->aws) cudaFree(P->aws);
  for (cudaStream_t h : {P->acs, P->aos})
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t e : {P->a_call, P->a_in[0], P->a_in[1], P->a_comp[0], P->a_comp[1], P->a_out[0], P->a_out[1]})
    if (e) cudaEventDestroy(e);
  delete P;
  return TEBD_OK;
}

extern "C" int rrsvd_workspace_size(rrsvd_plan_t P, size_t* bytes) {
  if (!P || !bytes) return TEBD_EINVAL;
  *bytes = P->ws_bytes;
  return TEBD_OK;
}

extern "C" int rrsvd_plan_widths(rrsvd_plan_t P, int* l_out) {
  if (!P || !l_out) return TEBD_EINVAL;
  std::vector<Dims> hd(P->batch);
  CU_OR(P, cudaMemcpy(hd.data(), P->dims, sizeof(Dims) * P->batch, cudaMemcpyDeviceToHost));
  for (int i = 0; i < P->batch; ++i) l_out[i] = hd[i].l;
  return TEBD_OK;
}

extern "C" int rrsvd_plan_dims(rrsvd_plan_t P, int* k, int* l) {
  if (!P) return TEBD_EINVAL;
  if (k) *k = P->k;
  if (l) *l = P->l;
  return TEBD_OK;
}

// The fixed-rank truncation of instances z0 .. z0 + cnt - 1 of a bound plan
// (k_rrsvd_bind has run): sigma, Vh, w and rank point at instance z0's
// entries.  Sub-batches of one plan may run concurrently on different streams.
static cudaError_t exec_range(rrsvd_plan_t P, int z0, int cnt, int64_t chain0, double* sigma, double* Vh, double* w,
                              int* rank, void* workspace, cudaStream_t st, const MixedKnobs& kn) {
  Dims* dims = P->dims + z0;
  const ProbPtr* ptrs = P->ptrs + z0;
  cudaError_t e;
  if (prec_mixed(P->precision)) {
    const MixedPtrs mp =
        mixed_offset(mixed_carve((char*)workspace + P->mixed_off, P->ms, P->batch), P->ms, z0);
    e = run_rrsvd_mixed(dims, ptrs, cnt, P->cap, mp, P->q, P->seed, 0, chain0 + z0, 1, P->status, P->tcerr, st,
                        nullptr, &kn, P->precision == TEBD_PREC_BF16);
  } else {
    e = run_rrsvd(dims, ptrs, cnt, P->cap, P->q, P->seed, 0, chain0 + z0, 1, P->status, st, nullptr,
                  P->tuned ? P->tiles : nullptr);
  }
  if (e != cudaSuccess) return e;
  return launch_rrsvd_finalize(dims, ptrs, cnt, P->cap, 1e-14, sigma, Vh, w, rank, P->status, st);
}

extern "C" int rrsvd_execute(rrsvd_plan_t P, const double* theta, int64_t chain0, double* sigma, double* U, double* Vh,
                             double* w, int* rank, void* workspace, size_t workspace_bytes, void* stream) {
  if (!P) return TEBD_EINVAL;
  if (P->err.code) return P->err.code;
  if (!theta || !sigma || !workspace || chain0 < 0) { P->err.set(TEBD_EINVAL, "NULL argument or chain0 < 0"); return P->err.code; }
  if (workspace_bytes < P->ws_bytes) {
    P->err.set(TEBD_EINVAL, "workspace of %zu bytes, %zu needed", workspace_bytes, P->ws_bytes);
    return P->err.code;
  }
  if (((uintptr_t)workspace) % ALIGN) { P->err.set(TEBD_EINVAL, "workspace not 256-byte aligned"); return P->err.code; }
  cudaStream_t st = (cudaStream_t)stream;
  const bool checked = P->check_r > 0;
  {
  ProfScope ps("k_rrsvd_bind", st);
  k_rrsvd_bind<<<(P->batch + 127) / 128, 128, 0, st>>>(P->ptrs, P->batch, (char*)workspace, P->per, P->lay,
                                                     (const cplx*)theta, (size_t)P->m * P->n,
                                                     checked ? nullptr : (cplx*)U, (size_t)P->m * P->k, (cplx*)Vh,
                                                     (size_t)P->k * P->n, nullptr, 0, 0, 0, 0, nullptr);
  }
  CU_OR(P, cudaGetLastError());
  if (checked) {
    Dims t;
    memset(&t, 0, sizeof t);
    t.m = P->m; t.n = P->n; t.k = P->k0; t.l = P->l0; t.active = 1; t.r = P->check_r;
    t.chk = (P->l0 + P->check_r <= P->l_max) ? 1 : 0;
    CU_OR(P, launch_checked_init(P->dims, P->batch, t, st));
    CU_OR(P, run_rrsvd_checked(P->dims, P->ptrs, P->batch, P->cap, P->q, P->rounds, P->eps, P->l_max, P->p, P->seed,
                               chain0, P->status, st));
    CU_OR(P, launch_finalize_checked(P->dims, P->ptrs, P->batch, P->k, 1e-14, sigma, U, w, rank, nullptr, P->status,
                                     st));
    return TEBD_OK;
  }
  CU_OR(P, exec_range(P, 0, P->batch, chain0, sigma, Vh, w, rank, workspace, st, P->mk));
  return TEBD_OK;
}

// Status flags raised by the truncations since they were last read: the
// plan's error (and return code) for them.
static int plan_flags(rrsvd_plan_t P, int stv, int tce) {
  if (tce) { P->err.set(TEBD_ETIMEOUT, "a tensor-core pipeline wait expired"); return P->err.code; }
  if (stv & 4) {
    P->err.set(TEBD_ENUMERIC, "the re-orthonormalisation of an FP32 basis met a non-finite or far from orthonormal "
                              "basis");
    return P->err.code;
  }
  if (stv & 1) { P->err.set(TEBD_ENUMERIC, "an instance had a zero or non-finite theta"); return P->err.code; }
  return TEBD_OK;
}

extern "C" int rrsvd_host_wait(rrsvd_plan_t P);

extern "C" int rrsvd_execute_host(rrsvd_plan_t P, const double* theta, int64_t chain0, double* sigma, double* U,
                                  double* Vh, double* w, int* rank, void* stream) {
  if (!P) return TEBD_EINVAL;
  if (P->apending) {
    const int rc = rrsvd_host_wait(P);
    if (rc) return rc;
  }
  if (P->err.code) return P->err.code;
  if (!theta || !sigma) { P->err.set(TEBD_EINVAL, "NULL theta or sigma"); return P->err.code; }
  const size_t B = P->batch, c = sizeof(cplx);
  const size_t th = align_up(c * (size_t)P->m * P->n * B), sg = align_up(sizeof(double) * P->k * B),
               uu = align_up(c * (size_t)P->m * P->k * B), vv = align_up(c * (size_t)P->k * P->n * B),
               ww = align_up(sizeof(double) * B), rr = align_up(sizeof(int) * B);
  const size_t need = th + sg + uu + vv + ww + rr + P->ws_bytes;
  if (!P->stage) {
    if (fault_take(TEBD_FAULT_ALLOC) || cudaMalloc(&P->stage, need) != cudaSuccess) {
      cudaGetLastError();
      P->stage = nullptr;
      P->err.set(TEBD_ENOMEM, "staging allocation of %zu bytes failed", need);
      return P->err.code;
    }
    P->stage_bytes = need;
  }
  char* s = P->stage;
  double* d_th = (double*)s;
  double* d_sg = (double*)(s + th);
  double* d_u = (double*)(s + th + sg);
  double* d_v = (double*)(s + th + sg + uu);
  double* d_w = (double*)(s + th + sg + uu + vv);
  int* d_r = (int*)(s + th + sg + uu + vv + ww);
  void* d_ws = s + th + sg + uu + vv + ww + rr;
  cudaStream_t st = (cudaStream_t)stream;
  // sub-batches for mixed-form plans of 16 instances or more (their launch
  // choices fixed as the whole batch's size rules make them, so that the
  // results equal rrsvd_execute's bit for bit)
  const int nch = (P->check_r > 0 || !prec_mixed(P->precision) || P->batch < 16) ? 1 : rrsvd_plan_s::HCH;
  if (nch == 1) {
    {
      ProfScope ps("copy[h2d]", st);
      CU_OR(P, cudaMemcpyAsync(d_th, theta, c * (size_t)P->m * P->n * B, cudaMemcpyHostToDevice, st));
    }
    int rc = rrsvd_execute(P, d_th, chain0, d_sg, U ? d_u : nullptr, Vh ? d_v : nullptr, w ? d_w : nullptr,
                           rank ? d_r : nullptr, d_ws, P->ws_bytes, stream);
    if (rc) return rc;
    ProfScope ps("copy[d2h]", st);
    CU_OR(P, cudaMemcpyAsync(sigma, d_sg, sizeof(double) * P->k * B, cudaMemcpyDeviceToHost, st));
    if (U) CU_OR(P, cudaMemcpyAsync(U, d_u, c * (size_t)P->m * P->k * B, cudaMemcpyDeviceToHost, st));
    if (Vh) CU_OR(P, cudaMemcpyAsync(Vh, d_v, c * (size_t)P->k * P->n * B, cudaMemcpyDeviceToHost, st));
    if (w) CU_OR(P, cudaMemcpyAsync(w, d_w, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    if (rank) CU_OR(P, cudaMemcpyAsync(rank, d_r, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  } else {
    // Pipelined: the batch in HCH sub-batches, each on a stream of its own
    // (copy in, truncation, copy out), so that copies of one overlap the
    // kernels of the others and the kernels of the sub-batches share the SMs.
    if (chain0 < 0) { P->err.set(TEBD_EINVAL, "chain0 < 0"); return P->err.code; }
    for (int i = 0; i < nch; ++i)
      if (!P->hs[i]) CU_OR(P, cudaStreamCreateWithFlags(&P->hs[i], cudaStreamNonBlocking));
    for (int i = 0; i <= nch; ++i)
      if (!P->hev[i]) CU_OR(P, cudaEventCreateWithFlags(&P->hev[i], cudaEventDisableTiming));
    {
      ProfScope ps("k_rrsvd_bind", st);
      k_rrsvd_bind<<<(P->batch + 127) / 128, 128, 0, st>>>(P->ptrs, P->batch, (char*)d_ws, P->per, P->lay,
                                                         (const cplx*)d_th, (size_t)P->m * P->n,
                                                         U ? (cplx*)d_u : nullptr, (size_t)P->m * P->k,
                                                         Vh ? (cplx*)d_v : nullptr, (size_t)P->k * P->n, nullptr, 0,
                                                         0, 0, 0, nullptr);
      CU_OR(P, cudaGetLastError());
    }
    CU_OR(P, cudaEventRecord(P->hev[nch], st));
    MixedKnobs kc = P->mk;
    if (kc.qrbh == 0) kc.qrbh = qr_multi_chosen(QR_BH, P->cap, P->batch, 0) ? 2 : 3;
    if (kc.jac == 0) kc.jac = jacobi_cluster_chosen(P->cap, P->batch, 0) ? 2 : 3;
    const size_t mn = (size_t)P->m * P->n, mk = (size_t)P->m * P->k, kn = (size_t)P->k * P->n;
    const int per = (P->batch + nch - 1) / nch;
    for (int i = 0; i < nch; ++i) {
      const int z0 = i * per, cnt = std::min(per, P->batch - z0);
      if (cnt <= 0) break;
      cudaStream_t hs = P->hs[i];
      CU_OR(P, cudaStreamWaitEvent(hs, P->hev[nch], 0));
      {
        ProfScope ps("copy[h2d]", hs);
        CU_OR(P, cudaMemcpyAsync(d_th + 2 * mn * z0, theta + 2 * mn * z0, c * mn * cnt, cudaMemcpyHostToDevice, hs));
      }
      CU_OR(P, exec_range(P, z0, cnt, chain0, d_sg + (size_t)P->k * z0, Vh ? d_v + 2 * kn * z0 : nullptr,
                          w ? d_w + z0 : nullptr, rank ? d_r + z0 : nullptr, d_ws, hs, kc));
      {
        ProfScope ps("copy[d2h]", hs);
        CU_OR(P, cudaMemcpyAsync(sigma + (size_t)P->k * z0, d_sg + (size_t)P->k * z0, sizeof(double) * P->k * cnt,
                                 cudaMemcpyDeviceToHost, hs));
        if (U) CU_OR(P, cudaMemcpyAsync(U + 2 * mk * z0, d_u + 2 * mk * z0, c * mk * cnt, cudaMemcpyDeviceToHost, hs));
        if (Vh) CU_OR(P, cudaMemcpyAsync(Vh + 2 * kn * z0, d_v + 2 * kn * z0, c * kn * cnt, cudaMemcpyDeviceToHost, hs));
        if (w) CU_OR(P, cudaMemcpyAsync(w + z0, d_w + z0, sizeof(double) * cnt, cudaMemcpyDeviceToHost, hs));
        if (rank) CU_OR(P, cudaMemcpyAsync(rank + z0, d_r + z0, sizeof(int) * cnt, cudaMemcpyDeviceToHost, hs));
      }
      CU_OR(P, cudaEventRecord(P->hev[i], hs));
      CU_OR(P, cudaStreamWaitEvent(st, P->hev[i], 0));
    }
  }
  int stv = 0, tce = 0;
  CU_OR(P, cudaMemcpyAsync(&stv, P->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU_OR(P, cudaMemcpyAsync(&tce, P->tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU_OR(P, cudaStreamSynchronize(st));
  return plan_flags(P, stv, tce);
}

extern "C" int rrsvd_execute_host_async(rrsvd_plan_t P, const double* theta, int64_t chain0, double* sigma,
                                        double* U, double* Vh, double* w, int* rank, void* stream) {
  if (!P) return TEBD_EINVAL;
  if (P->err.code) return P->err.code;
  if (!theta || !sigma || chain0 < 0) { P->err.set(TEBD_EINVAL, "NULL theta or sigma, or chain0 < 0"); return P->err.code; }
  const size_t B = P->batch, c = sizeof(cplx);
  const size_t th = align_up(c * (size_t)P->m * P->n * B), sg = align_up(sizeof(double) * P->k * B),
               uu = align_up(c * (size_t)P->m * P->k * B), vv = align_up(c * (size_t)P->k * P->n * B),
               ww = align_up(sizeof(double) * B), rr = align_up(sizeof(int) * B);
  const size_t slot_bytes = th + sg + uu + vv + ww + rr;
  if (!P->aws) {
    if (fault_take(TEBD_FAULT_ALLOC) || cudaMalloc(&P->aws, P->ws_bytes) != cudaSuccess ||
        cudaMalloc(&P->aslot[0], slot_bytes) != cudaSuccess || cudaMalloc(&P->aslot[1], slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      for (char*& b : P->aslot)
        if (b) { cudaFree(b); b = nullptr; }
      if (P->aws) { cudaFree(P->aws); P->aws = nullptr; }
      P->err.set(TEBD_ENOMEM, "staging allocation of 2 x %zu + %zu bytes failed", slot_bytes, P->ws_bytes);
      return P->err.code;
    }
    CU_OR(P, cudaStreamCreateWithFlags(&P->acs, cudaStreamNonBlocking));
    CU_OR(P, cudaStreamCreateWithFlags(&P->aos, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&P->a_call, &P->a_in[0], &P->a_in[1], &P->a_comp[0], &P->a_comp[1], &P->a_out[0],
                           &P->a_out[1]})
      CU_OR(P, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  const int slot = P->anext;
  P->anext ^= 1;
  char* s = P->aslot[slot];
  double* d_th = (double*)s;
  double* d_sg = (double*)(s + th);
  double* d_u = (double*)(s + th + sg);
  double* d_v = (double*)(s + th + sg + uu);
  double* d_w = (double*)(s + th + sg + uu + vv);
  int* d_r = (int*)(s + th + sg + uu + vv + ww);
  cudaStream_t st = (cudaStream_t)stream;
  // copy in as soon as this slot's theta was last read (by the truncation
  // two calls back): not ordered after the work on `stream`, so that it
  // overlaps the previous call's truncation
  CU_OR(P, cudaStreamWaitEvent(P->acs, P->a_comp[slot], 0));
  {
    ProfScope ps("copy[h2d]", P->acs);
    CU_OR(P, cudaMemcpyAsync(d_th, theta, c * (size_t)P->m * P->n * B, cudaMemcpyHostToDevice, P->acs));
  }
  CU_OR(P, cudaEventRecord(P->a_in[slot], P->acs));
  // the truncation after the copy in and after this slot's results of two
  // calls back are copied out
  CU_OR(P, cudaStreamWaitEvent(st, P->a_in[slot], 0));
  CU_OR(P, cudaStreamWaitEvent(st, P->a_out[slot], 0));
  P->apending = 1;
  P->astream = st;
  int rc = rrsvd_execute(P, d_th, chain0, d_sg, U ? d_u : nullptr, Vh ? d_v : nullptr, w ? d_w : nullptr,
                         rank ? d_r : nullptr, P->aws, P->ws_bytes, stream);
  if (rc) return rc;
  CU_OR(P, cudaEventRecord(P->a_comp[slot], st));
  CU_OR(P, cudaStreamWaitEvent(P->aos, P->a_comp[slot], 0));
  {
    ProfScope ps("copy[d2h]", P->aos);
    CU_OR(P, cudaMemcpyAsync(sigma, d_sg, sizeof(double) * P->k * B, cudaMemcpyDeviceToHost, P->aos));
    if (U) CU_OR(P, cudaMemcpyAsync(U, d_u, c * (size_t)P->m * P->k * B, cudaMemcpyDeviceToHost, P->aos));
    if (Vh) CU_OR(P, cudaMemcpyAsync(Vh, d_v, c * (size_t)P->k * P->n * B, cudaMemcpyDeviceToHost, P->aos));
    if (w) CU_OR(P, cudaMemcpyAsync(w, d_w, sizeof(double) * B, cudaMemcpyDeviceToHost, P->aos));
    if (rank) CU_OR(P, cudaMemcpyAsync(rank, d_r, sizeof(int) * B, cudaMemcpyDeviceToHost, P->aos));
  }
  CU_OR(P, cudaEventRecord(P->a_out[slot], P->aos));
  return TEBD_OK;
}

extern "C" int rrsvd_host_wait(rrsvd_plan_t P) {
  if (!P) return TEBD_EINVAL;
  if (!P->apending) return P->err.code;
  P->apending = 0;
  CU_OR(P, cudaStreamSynchronize(P->aos));
  CU_OR(P, cudaStreamSynchronize(P->astream));
  int stv = 0, tce = 0;
  CU_OR(P, cudaMemcpy(&stv, P->status, sizeof(int), cudaMemcpyDeviceToHost));
  CU_OR(P, cudaMemcpy(&tce, P->tcerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (P->err.code) return P->err.code;
  return plan_flags(P, stv, tce);
}

extern "C" const char* rrsvd_last_error(rrsvd_plan_t P) { return P ? P->err.msg.c_str() : "NULL plan"; }

extern "C" int rrsvd_plan_autotune(rrsvd_plan_t P, const double* theta, void* workspace, size_t workspace_bytes,
                                   void* stream) {
  if (!P) return TEBD_EINVAL;
  if (P->err.code) return P->err.code;
  if (!theta || !workspace) { P->err.set(TEBD_EINVAL, "NULL theta or workspace"); return P->err.code; }
  if (workspace_bytes < P->ws_bytes || ((uintptr_t)workspace) % ALIGN) {
    P->err.set(TEBD_EINVAL, "workspace too small or not 256-byte aligned");
    return P->err.code;
  }
  if (P->check_r > 0) return TEBD_OK;  // the accuracy-check sequence has no launch choices to tune
  cudaStream_t st = (cudaStream_t)stream;
  k_rrsvd_bind<<<(P->batch + 127) / 128, 128, 0, st>>>(P->ptrs, P->batch, (char*)workspace, P->per, P->lay,
                                                     (const cplx*)theta, (size_t)P->m * P->n, nullptr, 0, nullptr, 0,
                                                     nullptr, 0, 0, 0, 0, nullptr);
  CU_OR(P, cudaGetLastError());
  if (prec_mixed(P->precision)) {
    const MixedPtrs mp = mixed_carve((char*)workspace + P->mixed_off, P->ms, P->batch);
    auto run = [&](const MixedKnobs& k) {
      return run_rrsvd_mixed(P->dims, P->ptrs, P->batch, P->cap, mp, P->q, P->seed, 0, 0, 1, P->status, P->tcerr, st,
                             nullptr, &k, P->precision == TEBD_PREC_BF16);
    };
    float ms[2] = {0.f, 0.f};
    if (tune_knobs(run, st, P->cap, P->batch, P->mk, ms) != 0) {
      P->err.set(TEBD_ECUDA, "autotuning failed: %s", cudaGetErrorString(cudaGetLastError()));
      return P->err.code;
    }
    P->tune_ms[0] = ms[0];
    P->tune_ms[1] = ms[1];
  } else {
    // GEMM tiles of every stage: the kernels alone (their time does not depend
    // on the data), after one whole RRSVD that fills every operand
    CU_OR(P, run_rrsvd(P->dims, P->ptrs, P->batch, P->cap, P->q, P->seed, 0, 0, 1, P->status, st));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int stage = 0; stage < 6; ++stage) {
      float best = 1e30f;
      for (int tile : {16, 32}) {
        launch_zgemm_tile(stage, tile, P->dims, P->ptrs, P->batch, P->cap, st);
        cudaEventRecord(e0, st);
        launch_zgemm_tile(stage, tile, P->dims, P->ptrs, P->batch, P->cap, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) { best = t; P->tiles[stage] = tile; }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  P->tuned = 1;
  // the timing runs raise no flag the next execute should see
  CU_OR(P, cudaMemsetAsync(P->status, 0, 2 * ALIGN, st));
  CU_OR(P, cudaStreamSynchronize(st));
  return TEBD_OK;
}

extern "C" int rrsvd_plan_set_tuning(rrsvd_plan_t P, const int* info) {
  if (!P || !info) return TEBD_EINVAL;
  for (int i = 0; i < 6; ++i)
    if (info[i] != 0 && info[i] != 16 && info[i] != 32) return TEBD_EINVAL;
  const int th = info[7];
  if (info[6] < 0 || info[6] > 1 || (th != 0 && th != 128 && th != 256 && th != 512) || info[8] < 0 ||
      info[8] > 3 || info[9] < 0 || info[9] > 3 || info[11] < 0 || info[11] > 2)
    return TEBD_EINVAL;
  for (int i = 0; i < 6; ++i) P->tiles[i] = info[i];
  P->mk = MixedKnobs{info[6], info[7], info[8], info[9], info[11]};
  P->tuned = 1;
  return TEBD_OK;
}

extern "C" int rrsvd_plan_tuning(rrsvd_plan_t P, int* info, double* ms) {
  if (!P) return TEBD_EINVAL;
  if (info) {
    memset(info, 0, sizeof(int) * 16);
    for (int i = 0; i < 6; ++i) info[i] = P->tiles[i];
    info[6] = P->mk.tc_half; info[7] = P->mk.qr_threads; info[8] = P->mk.qrbh; info[9] = P->mk.jac;
    info[10] = P->tuned;
    info[11] = P->mk.dfg;
  }
  if (ms) {
    ms[0] = P->tune_ms[0];
    ms[1] = P->tune_ms[1];
  }
  return TEBD_OK;
}

extern "C" int rrsvd_clear_error(rrsvd_plan_t P) {
  if (!P) return TEBD_EINVAL;
  P->err.code = TEBD_OK;
  P->err.msg.clear();
  // status and the tensor-core flag sit in the two ALIGN-sized slots after
  // the descriptors
  if (cudaMemset(P->status, 0, 2 * ALIGN) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    P->err.set(TEBD_ECUDA, "clearing the device flags failed");
    return P->err.code;
  }
  return TEBD_OK;
}
