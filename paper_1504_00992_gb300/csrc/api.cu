// C ABI of the TEBD / RRSVD library: handles, device memory, and the launch
// sequence of a sweep.  See include/tebd_gb300.h for the contract.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tebd_gb300.h"
#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"

using namespace tg;

namespace {

const size_t ALIGN = 256;
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

// Per-problem RRSVD workspace layout (byte offsets from a base).
struct WsLayout {
  size_t omega, Y, Q, Yt, Qt, R, J, Jk, Wk, U, V, sigma, part, scal, total;
};

WsLayout ws_layout(int m, int n, int k, int l, bool own_U, bool own_V) {
  WsLayout w;
  size_t o = 0;
  const size_t c = sizeof(cplx);
  w.omega = o; o += align_up(c * (size_t)n * l);
  w.Y = o; o += align_up(c * (size_t)m * l);
  w.Q = o; o += align_up(c * (size_t)m * l);
  w.Yt = o; o += align_up(c * (size_t)n * l);
  w.Qt = o; o += align_up(c * (size_t)n * l);
  w.R = o; o += align_up(c * (size_t)l * l);
  w.J = o; o += align_up(c * (size_t)l * l);
  w.Jk = o; o += align_up(c * (size_t)l * k);
  w.Wk = o; o += align_up(c * (size_t)l * k);
  w.U = o; if (own_U) o += align_up(c * (size_t)m * k);
  w.V = o; if (own_V) o += align_up(c * (size_t)k * n);
  w.sigma = o; o += align_up(sizeof(double) * (size_t)l);
  w.part = o; o += align_up(sizeof(double) * NPART);
  w.scal = o; o += align_up(sizeof(double) * 4);
  w.total = o;
  return w;
}

void fill_ptrs(ProbPtr& P, char* base, const WsLayout& w) {
  P.omega = (cplx*)(base + w.omega);
  P.Y = (cplx*)(base + w.Y);
  P.Q = (cplx*)(base + w.Q);
  P.Yt = (cplx*)(base + w.Yt);
  P.Qt = (cplx*)(base + w.Qt);
  P.R = (cplx*)(base + w.R);
  P.J = (cplx*)(base + w.J);
  P.Jk = (cplx*)(base + w.Jk);
  P.Wk = (cplx*)(base + w.Wk);
  P.U = (cplx*)(base + w.U);
  P.V = (cplx*)(base + w.V);
  P.sigma = (double*)(base + w.sigma);
  P.part = (double*)(base + w.part);
  P.scal = (double*)(base + w.scal);
}

bool all_finite(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return false;
  return true;
}

}  // namespace

// ===========================================================================
// TEBD handle
// ===========================================================================
struct ParitySet {
  int batch = 0;
  Dims* dims = nullptr;     // device
  ProbPtr* ptrs = nullptr;  // device
  Caps cap{};
  std::vector<int> bonds;
};

struct tebd_s {
  ErrState err;
  int N = 0, p = 0, q = 0, precision = 0;
  uint64_t seed = 0;
  double cutoff = 1e-14;
  int64_t chain = 0;
  int64_t sweeps = 0;
  cudaStream_t stream = 0;
  bool gates_set[2] = {false, false};
  std::vector<int> d, chi_cap, cap_ext;
  std::vector<size_t> gamma_off, lam_off, gate_off;
  size_t gamma_bytes = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // device views
  cplx** gamma_tab = nullptr;
  double** lam_tab = nullptr;
  int* chi_ext = nullptr;
  int* chi_cap_dev = nullptr;
  int* dsite_dev = nullptr;
  int* cap_ext_dev = nullptr;
  int* status = nullptr;
  double* wacc = nullptr;  // [0] sum w, [1] prod(1-w), [2..] per-sweep w
  cplx* gates = nullptr;
  cplx* op_dev = nullptr;
  cplx* out_dev = nullptr;
  std::vector<cplx*> gamma_ptr;
  std::vector<double*> lam_ptr;  // N+1 (outer ones -> one_lam)
  double* one_lam = nullptr;
  ParitySet par[2];
  ChainDev ch{};
};

static int tebd_check_status(tebd_t h) {
  int st = 0;
  CU_OR(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  if (st & 1) h->err.set(TEBD_ENUMERIC, "a bond update met a zero or non-finite theta");
  return h->err.code;
}

extern "C" int tebd_create_ex(const tebd_desc_t* desc, tebd_t* out) {
  if (!out) return TEBD_EINVAL;
  *out = nullptr;
  if (!desc) return TEBD_EINVAL;
  const int N = desc->N;
  if (N < 2 || desc->p < 0 || desc->q < 0) return TEBD_EINVAL;
  if (desc->precision != TEBD_PREC_FP64) return TEBD_ENOTIMPL;
  tebd_s* h = new tebd_s();
  h->N = N;
  h->p = desc->p;
  h->q = desc->q;
  h->seed = desc->seed;
  h->precision = desc->precision;
  h->cutoff = desc->sv_cutoff > 0 ? desc->sv_cutoff : 1e-14;
  h->chain = desc->chain;
  h->d.resize(N);
  for (int s = 0; s < N; ++s) {
    const int ds = desc->d_site ? desc->d_site[s] : desc->d;
    if (ds < 2 || ds > 64) { delete h; return TEBD_EINVAL; }
    h->d[s] = ds;
  }
  h->chi_cap.resize(N - 1);
  for (int b = 0; b < N - 1; ++b) {
    const int c = desc->chi_bond ? desc->chi_bond[b] : desc->chi_max;
    if (c < 1) { delete h; return TEBD_EINVAL; }
    h->chi_cap[b] = c;
  }
  // capacities: chi_b <= min(cap_b, prod_{s<=b} d_s, prod_{s>b} d_s)
  h->cap_ext.assign(N + 1, 1);
  for (int b = 0; b < N - 1; ++b) {
    double left = 1, right = 1;
    for (int s = 0; s <= b; ++s) left = std::min(left * h->d[s], 1e9);
    for (int s = b + 1; s < N; ++s) right = std::min(right * h->d[s], 1e9);
    h->cap_ext[b + 1] = (int)std::min<double>(h->chi_cap[b], std::min(left, right));
  }
  // --- sizes of every device buffer
  size_t off = 0;
  h->gamma_off.resize(N);
  for (int s = 0; s < N; ++s) {
    h->gamma_off[s] = off;
    off += align_up(sizeof(cplx) * (size_t)h->d[s] * h->cap_ext[s] * h->cap_ext[s + 1]);
  }
  h->gamma_bytes = off;
  h->lam_off.resize(N - 1);
  for (int b = 0; b < N - 1; ++b) {
    h->lam_off[b] = off;
    off += align_up(sizeof(double) * h->cap_ext[b + 1]);
  }
  const size_t one_off = off; off += ALIGN;
  h->gate_off.resize(N - 1);
  for (int b = 0; b < N - 1; ++b) {
    h->gate_off[b] = off;
    const size_t dd = (size_t)h->d[b] * h->d[b + 1];
    off += align_up(sizeof(cplx) * dd * dd);
  }
  const size_t tab_off = off;
  off += align_up(sizeof(cplx*) * N) + align_up(sizeof(double*) * (N + 1));
  const size_t int_off = off;
  off += 4 * align_up(sizeof(int) * (N + 1));
  const size_t st_off = off; off += ALIGN;
  const size_t wacc_off = off; off += align_up(sizeof(double) * (2 + N));
  const size_t op_off = off; off += align_up(sizeof(cplx) * 64 * 64) + ALIGN;
  // per-parity problem descriptors and shared workspace
  size_t ws_max = 0;
  std::vector<WsLayout> lay[2];
  for (int par = 0; par < 2; ++par) {
    ParitySet& ps = h->par[par];
    Caps c{};
    for (int b = par; b < N - 1; b += 2) {
      const int mc = h->d[b] * h->cap_ext[b], nc = h->d[b + 1] * h->cap_ext[b + 2];
      const int kc = std::min(h->cap_ext[b + 1], std::min(mc, nc));
      const int lc = std::min(kc + h->p, std::min(mc, nc));
      if (lc > 512) { delete h; return TEBD_ENOTIMPL; }
      ps.bonds.push_back(b);
      lay[par].push_back(ws_layout(mc, nc, kc, lc, true, true));
      c.m = std::max(c.m, mc); c.n = std::max(c.n, nc); c.k = std::max(c.k, kc); c.l = std::max(c.l, lc);
      c.cl = std::max(c.cl, h->cap_ext[b]); c.cr = std::max(c.cr, h->cap_ext[b + 2]);
      c.dl = std::max(c.dl, h->d[b]); c.dr = std::max(c.dr, h->d[b + 1]);
    }
    ps.batch = (int)ps.bonds.size();
    ps.cap = c;
    size_t tot = 0;
    for (size_t i = 0; i < ps.bonds.size(); ++i) {
      const int b = ps.bonds[i];
      tot += align_up(sizeof(cplx) * (size_t)h->d[b] * h->cap_ext[b] * h->d[b + 1] * h->cap_ext[b + 2]);
      tot += lay[par][i].total;
    }
    ws_max = std::max(ws_max, tot);
  }
  const size_t desc_off = off;
  off += 2 * (align_up(sizeof(Dims) * N) + align_up(sizeof(ProbPtr) * N));
  const size_t ws_off = off;
  off += ws_max;
  h->arena_bytes = off;
  if (cudaMalloc(&h->arena, h->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return TEBD_ENOMEM;
  }
  char* A = h->arena;
  h->gamma_ptr.resize(N);
  for (int s = 0; s < N; ++s) h->gamma_ptr[s] = (cplx*)(A + h->gamma_off[s]);
  h->one_lam = (double*)(A + one_off);
  h->lam_ptr.resize(N + 1);
  h->lam_ptr[0] = h->one_lam;
  h->lam_ptr[N] = h->one_lam;
  for (int b = 0; b < N - 1; ++b) h->lam_ptr[b + 1] = (double*)(A + h->lam_off[b]);
  h->gates = (cplx*)(A + h->gate_off[0]);
  h->gamma_tab = (cplx**)(A + tab_off);
  h->lam_tab = (double**)(A + tab_off + align_up(sizeof(cplx*) * N));
  h->chi_ext = (int*)(A + int_off);
  h->chi_cap_dev = (int*)(A + int_off + align_up(sizeof(int) * (N + 1)));
  h->dsite_dev = (int*)(A + int_off + 2 * align_up(sizeof(int) * (N + 1)));
  h->cap_ext_dev = (int*)(A + int_off + 3 * align_up(sizeof(int) * (N + 1)));
  h->status = (int*)(A + st_off);
  h->wacc = (double*)(A + wacc_off);
  h->op_dev = (cplx*)(A + op_off);
  h->out_dev = (cplx*)(A + op_off + align_up(sizeof(cplx) * 64 * 64));
  char* ws = A + ws_off;
  for (int par = 0; par < 2; ++par) {
    ParitySet& ps = h->par[par];
    ps.dims = (Dims*)(A + desc_off + par * (align_up(sizeof(Dims) * N) + align_up(sizeof(ProbPtr) * N)));
    ps.ptrs = (ProbPtr*)((char*)ps.dims + align_up(sizeof(Dims) * N));
    std::vector<ProbPtr> hp(ps.batch);
    size_t o = 0;
    for (int i = 0; i < ps.batch; ++i) {
      const int b = ps.bonds[i];
      ProbPtr& P = hp[i];
      memset(&P, 0, sizeof P);
      P.gl = h->gamma_ptr[b];
      P.gr = h->gamma_ptr[b + 1];
      P.laml = h->lam_ptr[b];
      P.lamm = h->lam_ptr[b + 1];
      P.lamr = h->lam_ptr[b + 2];
      P.gate = (const cplx*)(A + h->gate_off[b]);
      P.cap_l = h->cap_ext[b];
      P.cap_m = h->cap_ext[b + 1];
      P.cap_r = h->cap_ext[b + 2];
      P.theta = (const cplx*)(ws + o);
      o += align_up(sizeof(cplx) * (size_t)h->d[b] * h->cap_ext[b] * h->d[b + 1] * h->cap_ext[b + 2]);
      fill_ptrs(P, ws + o, lay[par][i]);
      o += lay[par][i].total;
    }
    if (ps.batch > 0 &&
        cudaMemcpy(ps.ptrs, hp.data(), sizeof(ProbPtr) * ps.batch, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(h->arena);
      delete h;
      return TEBD_ECUDA;
    }
  }
  std::vector<int> dsite(h->d), capv(h->chi_cap);
  const double one = 1.0;
  bool ok = cudaMemcpy(h->gamma_tab, h->gamma_ptr.data(), sizeof(cplx*) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->lam_tab, h->lam_ptr.data(), sizeof(double*) * (N + 1), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(h->dsite_dev, dsite.data(), sizeof(int) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->chi_cap_dev, capv.data(), sizeof(int) * (N - 1), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(h->cap_ext_dev, h->cap_ext.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(h->one_lam, &one, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaFree(h->arena);
    delete h;
    return TEBD_ECUDA;
  }
  h->ch.N = N;
  h->ch.chi_ext = h->chi_ext;
  h->ch.chi_cap = h->chi_cap_dev;
  h->ch.dsite = h->dsite_dev;
  h->ch.lam_ext = h->lam_tab;
  h->ch.gamma = h->gamma_tab;
  h->ch.cap_ext = h->cap_ext_dev;
  // |0...0>
  std::vector<double> psi;
  for (int s = 0; s < N; ++s) {
    psi.push_back(1.0);
    psi.push_back(0.0);
    for (int i = 1; i < h->d[s]; ++i) { psi.push_back(0.0); psi.push_back(0.0); }
  }
  int rc = tebd_set_product_state(h, psi.data());
  if (rc != TEBD_OK) {
    cudaFree(h->arena);
    delete h;
    return rc;
  }
  *out = h;
  return TEBD_OK;
}

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
  if (h->arena) cudaFree(h->arena);
  delete h;
  return TEBD_OK;
}

extern "C" int tebd_set_stream(tebd_t h, void* s) {
  if (!h) return TEBD_EINVAL;
  h->stream = (cudaStream_t)s;
  return TEBD_OK;
}

extern "C" int tebd_set_product_state(tebd_t h, const double* psi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!psi) { h->err.set(TEBD_EINVAL, "psi is NULL"); return h->err.code; }
  const int N = h->N;
  std::vector<char> gam(h->gamma_bytes, 0);
  size_t o = 0;
  for (int s = 0; s < N; ++s) {
    const int ds = h->d[s];
    double nrm = 0.0;
    for (int i = 0; i < 2 * ds; ++i) nrm += psi[o + i] * psi[o + i];
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      h->err.set(TEBD_ENUMERIC, "site %d: zero or non-finite amplitudes", s);
      return h->err.code;
    }
    nrm = 1.0 / sqrt(nrm);
    cplx* g = (cplx*)(gam.data() + h->gamma_off[s]);
    const size_t stride = (size_t)h->cap_ext[s] * h->cap_ext[s + 1];
    for (int i = 0; i < ds; ++i) g[i * stride] = cmk(psi[o + 2 * i] * nrm, psi[o + 2 * i + 1] * nrm);
    o += 2 * ds;
  }
  CU_OR(h, cudaMemcpyAsync(h->arena, gam.data(), h->gamma_bytes, cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < N - 1; ++b) {
    std::vector<double> lam(h->cap_ext[b + 1], 0.0);
    lam[0] = 1.0;
    CU_OR(h, cudaMemcpyAsync(h->lam_ptr[b + 1], lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                             h->stream));
  }
  std::vector<int> chi(N + 1, 1);
  CU_OR(h, cudaMemcpyAsync(h->chi_ext, chi.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->stream));
  const double w0[2] = {0.0, 1.0};
  CU_OR(h, cudaMemcpyAsync(h->wacc, w0, sizeof w0, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  h->sweeps = 0;
  return TEBD_OK;
}

extern "C" int tebd_set_mps(tebd_t h, const double* const* gamma, const double* const* lambda, const int* chi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!gamma || !lambda || !chi) { h->err.set(TEBD_EINVAL, "NULL argument"); return h->err.code; }
  const int N = h->N;
  std::vector<int> ce(N + 1, 1);
  for (int b = 0; b < N - 1; ++b) {
    if (chi[b] < 1 || chi[b] > h->cap_ext[b + 1]) {
      h->err.set(TEBD_EINVAL, "bond %d: chi %d outside [1, %d]", b, chi[b], h->cap_ext[b + 1]);
      return h->err.code;
    }
    ce[b + 1] = chi[b];
  }
  std::vector<char> gam(h->gamma_bytes, 0);
  for (int s = 0; s < N; ++s) {
    if (!gamma[s]) { h->err.set(TEBD_EINVAL, "gamma[%d] is NULL", s); return h->err.code; }
    cplx* g = (cplx*)(gam.data() + h->gamma_off[s]);
    const int cl = ce[s], cr = ce[s + 1], capl = h->cap_ext[s], capr = h->cap_ext[s + 1];
    for (int i = 0; i < h->d[s]; ++i)
      for (int a = 0; a < cl; ++a)
        for (int c = 0; c < cr; ++c) {
          const size_t src = 2 * (((size_t)i * cl + a) * cr + c);
          g[((size_t)i * capl + a) * capr + c] = cmk(gamma[s][src], gamma[s][src + 1]);
        }
  }
  CU_OR(h, cudaMemcpyAsync(h->arena, gam.data(), h->gamma_bytes, cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < N - 1; ++b) {
    if (!lambda[b]) { h->err.set(TEBD_EINVAL, "lambda[%d] is NULL", b); return h->err.code; }
    std::vector<double> lam(h->cap_ext[b + 1], 0.0);
    for (int i = 0; i < chi[b]; ++i) lam[i] = lambda[b][i];
    CU_OR(h, cudaMemcpyAsync(h->lam_ptr[b + 1], lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                             h->stream));
  }
  CU_OR(h, cudaMemcpyAsync(h->chi_ext, ce.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, cudaStreamSynchronize(h->stream));
  return TEBD_OK;
}

extern "C" int tebd_get_mps(tebd_t h, double* const* gamma, double* const* lambda, int* chi) {
  if (!h) return TEBD_EINVAL;
  if (tebd_check_status(h)) return h->err.code;
  const int N = h->N;
  std::vector<int> ce(N + 1);
  CU_OR(h, cudaMemcpy(ce.data(), h->chi_ext, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost));
  if (chi)
    for (int b = 0; b < N - 1; ++b) chi[b] = ce[b + 1];
  if (gamma) {
    std::vector<char> gam(h->gamma_bytes);
    CU_OR(h, cudaMemcpy(gam.data(), h->arena, h->gamma_bytes, cudaMemcpyDeviceToHost));
    for (int s = 0; s < N; ++s) {
      if (!gamma[s]) continue;
      const cplx* g = (const cplx*)(gam.data() + h->gamma_off[s]);
      const int cl = ce[s], cr = ce[s + 1], capl = h->cap_ext[s], capr = h->cap_ext[s + 1];
      for (int i = 0; i < h->d[s]; ++i)
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
      CU_OR(h, cudaMemcpy(lambda[b], h->lam_ptr[b + 1], sizeof(double) * ce[b + 1], cudaMemcpyDeviceToHost));
    }
  return TEBD_OK;
}

extern "C" int tebd_set_gates(tebd_t h, int parity, const double* gates) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if ((parity != 0 && parity != 1) || !gates) { h->err.set(TEBD_EINVAL, "bad parity or NULL gates"); return h->err.code; }
  size_t o = 0;
  for (int b = 0; b < h->N - 1; ++b) {
    const size_t dd = (size_t)h->d[b] * h->d[b + 1];
    if (b % 2 == parity) {
      if (!all_finite(gates + o, 2 * dd * dd)) {
        h->err.set(TEBD_ENUMERIC, "gate of bond %d has a non-finite entry", b);
        return h->err.code;
      }
      CU_OR(h, cudaMemcpyAsync(h->arena + h->gate_off[b], gates + o, sizeof(cplx) * dd * dd, cudaMemcpyHostToDevice,
                               h->stream));
    }
    o += 2 * dd * dd;
  }
  CU_OR(h, cudaStreamSynchronize(h->stream));
  h->gates_set[parity] = true;
  return TEBD_OK;
}

static int tebd_step(tebd_t h, int parity) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!h->gates_set[parity]) { h->err.set(TEBD_ESTATE, "gates of parity %d not set", parity); return h->err.code; }
  ParitySet& ps = h->par[parity];
  if (ps.batch > 0) {
    CU_OR(h, launch_plan(h->ch, parity, h->p, ps.dims, ps.ptrs, ps.batch, h->stream));
    CU_OR(h, launch_theta(ps.dims, ps.ptrs, ps.batch, ps.cap, h->stream));
    CU_OR(h, run_rrsvd(ps.dims, ps.ptrs, ps.batch, ps.cap, h->q, h->seed, (uint64_t)h->sweeps, h->chain, 0,
                       h->status, h->stream));
    CU_OR(h, launch_rebuild(h->ch, ps.dims, ps.ptrs, ps.batch, ps.cap, h->cutoff, h->wacc, h->status, h->stream));
  }
  h->sweeps++;
  return TEBD_OK;
}

extern "C" int tebd_step_even(tebd_t h) { return tebd_step(h, 0); }
extern "C" int tebd_step_odd(tebd_t h) { return tebd_step(h, 1); }

extern "C" int tebd_expect(tebd_t h, int site, const double* op, double* out) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (site < 0 || site >= h->N || !op || !out) { h->err.set(TEBD_EINVAL, "bad site or NULL pointer"); return h->err.code; }
  const int d = h->d[site];
  CU_OR(h, cudaMemcpyAsync(h->op_dev, op, sizeof(cplx) * d * d, cudaMemcpyHostToDevice, h->stream));
  CU_OR(h, launch_expect(h->ch, site, h->op_dev, d, h->out_dev, h->stream));
  CU_OR(h, cudaMemcpyAsync(out, h->out_dev, sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  return tebd_check_status(h);
}

extern "C" int tebd_get_lambda(tebd_t h, int bond, double* out, int* chi) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (bond < 0 || bond >= h->N - 1 || !out) { h->err.set(TEBD_EINVAL, "bad bond or NULL pointer"); return h->err.code; }
  int c = 0;
  CU_OR(h, cudaMemcpyAsync(&c, h->chi_ext + bond + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU_OR(h, cudaMemcpyAsync(out, h->lam_ptr[bond + 1], sizeof(double) * h->cap_ext[bond + 1], cudaMemcpyDeviceToHost,
                           h->stream));
  if (tebd_check_status(h)) return h->err.code;
  if (chi) *chi = c;
  return TEBD_OK;
}

extern "C" int tebd_discarded_weight(tebd_t h, double* out) {
  if (!h) return TEBD_EINVAL;
  if (h->err.code) return h->err.code;
  if (!out) { h->err.set(TEBD_EINVAL, "NULL pointer"); return h->err.code; }
  CU_OR(h, cudaMemcpyAsync(out, h->wacc, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return tebd_check_status(h);
}

extern "C" int tebd_sweep_count(tebd_t h, int64_t* out) {
  if (!h || !out) return TEBD_EINVAL;
  *out = h->sweeps;
  return TEBD_OK;
}

extern "C" int tebd_backward(tebd_t h, const double*, double*, double*) {
  if (!h) return TEBD_EINVAL;
  return TEBD_ENOTIMPL;
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
  // host-path staging (allocated on first use)
  char* stage = nullptr;
  size_t stage_bytes = 0;
};

namespace tg {
// Fills the per-instance pointers from the call's buffers.
__global__ void k_rrsvd_bind(ProbPtr* ptrs, int batch, char* ws, size_t per, WsLayout lay, const cplx* theta,
                             size_t theta_stride, cplx* U, size_t U_stride, cplx* Vh, size_t V_stride) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= batch) return;
  ProbPtr P;
  memset(&P, 0, sizeof P);
  char* base = ws + per * (size_t)p;
  P.theta = theta + theta_stride * p;
  P.omega = (cplx*)(base + lay.omega);
  P.Y = (cplx*)(base + lay.Y);
  P.Q = (cplx*)(base + lay.Q);
  P.Yt = (cplx*)(base + lay.Yt);
  P.Qt = (cplx*)(base + lay.Qt);
  P.R = (cplx*)(base + lay.R);
  P.J = (cplx*)(base + lay.J);
  P.Jk = (cplx*)(base + lay.Jk);
  P.Wk = (cplx*)(base + lay.Wk);
  P.U = U ? U + U_stride * p : (cplx*)(base + lay.U);
  P.V = Vh ? Vh + V_stride * p : (cplx*)(base + lay.V);
  P.sigma = (double*)(base + lay.sigma);
  P.part = (double*)(base + lay.part);
  P.scal = (double*)(base + lay.scal);
  ptrs[p] = P;
}
}  // namespace tg

extern "C" int rrsvd_plan_create(int m, int n, int k_max, int p, int q, int batch, int precision, uint64_t seed,
                                 rrsvd_plan_t* out) {
  if (!out) return TEBD_EINVAL;
  *out = nullptr;
  if (m < 1 || n < 1 || k_max < 1 || p < 0 || q < 0 || batch < 1) return TEBD_EINVAL;
  if (precision != TEBD_PREC_FP64 && precision != TEBD_PREC_TF32) return TEBD_ENOTIMPL;
  rrsvd_plan_s* P = new rrsvd_plan_s();
  P->m = m; P->n = n; P->p = p; P->q = q; P->batch = batch; P->precision = precision; P->seed = seed;
  P->k = std::min(k_max, std::min(m, n));
  P->l = std::min(P->k + p, std::min(m, n));
  if (P->l > 512) { delete P; return TEBD_ENOTIMPL; }
  P->cap.m = m; P->cap.n = n; P->cap.k = P->k; P->cap.l = P->l;
  // workspace always holds U and Vh so that either may be NULL at execute
  P->lay = ws_layout(m, n, P->k, P->l, true, true);
  P->per = P->lay.total;
  P->ws_bytes = P->per * (size_t)batch;
  if (precision == TEBD_PREC_TF32) {
    P->ms = mixed_sizes(m, n, P->k, P->l);
    P->mixed_off = P->ws_bytes;
    P->ws_bytes += mixed_bytes(P->ms, batch);
  }
  const size_t meta = align_up(sizeof(Dims) * batch) + align_up(sizeof(ProbPtr) * batch) + 2 * ALIGN;
  if (cudaMalloc(&P->meta, meta) != cudaSuccess) { cudaGetLastError(); delete P; return TEBD_ENOMEM; }
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

extern "C" int rrsvd_plan_destroy(rrsvd_plan_t P) {
  if (!P) return TEBD_OK;
  if (P->meta) cudaFree(P->meta);
  if (P->stage) cudaFree(P->stage);
  delete P;
  return TEBD_OK;
}

extern "C" int rrsvd_workspace_size(rrsvd_plan_t P, size_t* bytes) {
  if (!P || !bytes) return TEBD_EINVAL;
  *bytes = P->ws_bytes;
  return TEBD_OK;
}

extern "C" int rrsvd_plan_dims(rrsvd_plan_t P, int* k, int* l) {
  if (!P) return TEBD_EINVAL;
  if (k) *k = P->k;
  if (l) *l = P->l;
  return TEBD_OK;
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
  {
  ProfScope ps("k_rrsvd_bind", st);
  k_rrsvd_bind<<<(P->batch + 127) / 128, 128, 0, st>>>(P->ptrs, P->batch, (char*)workspace, P->per, P->lay,
                                                     (const cplx*)theta, (size_t)P->m * P->n, (cplx*)U,
                                                     (size_t)P->m * P->k, (cplx*)Vh, (size_t)P->k * P->n);
  }
  CU_OR(P, cudaGetLastError());
  if (P->precision == TEBD_PREC_TF32) {
    const MixedPtrs mp = mixed_carve((char*)workspace + P->mixed_off, P->ms, P->batch);
    CU_OR(P, run_rrsvd_mixed(P->dims, P->ptrs, P->batch, P->cap, mp, P->q, P->seed, 0, chain0, 1, P->status,
                             P->tcerr, st));
  } else {
    CU_OR(P, run_rrsvd(P->dims, P->ptrs, P->batch, P->cap, P->q, P->seed, 0, chain0, 1, P->status, st));
  }
  CU_OR(P, launch_rrsvd_finalize(P->dims, P->ptrs, P->batch, P->cap, 1e-14, sigma, Vh, w, rank, P->status, st));
  return TEBD_OK;
}

extern "C" int rrsvd_execute_host(rrsvd_plan_t P, const double* theta, int64_t chain0, double* sigma, double* U,
                                  double* Vh, double* w, int* rank, void* stream) {
  if (!P) return TEBD_EINVAL;
  if (P->err.code) return P->err.code;
  if (!theta || !sigma) { P->err.set(TEBD_EINVAL, "NULL theta or sigma"); return P->err.code; }
  const size_t B = P->batch, c = sizeof(cplx);
  const size_t th = align_up(c * (size_t)P->m * P->n * B), sg = align_up(sizeof(double) * P->k * B),
               uu = align_up(c * (size_t)P->m * P->k * B), vv = align_up(c * (size_t)P->k * P->n * B),
               ww = align_up(sizeof(double) * B), rr = align_up(sizeof(int) * B);
  const size_t need = th + sg + uu + vv + ww + rr + P->ws_bytes;
  if (!P->stage) {
    if (cudaMalloc(&P->stage, need) != cudaSuccess) {
      cudaGetLastError();
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
  CU_OR(P, cudaMemcpyAsync(d_th, theta, c * (size_t)P->m * P->n * B, cudaMemcpyHostToDevice, st));
  int rc = rrsvd_execute(P, d_th, chain0, d_sg, U ? d_u : nullptr, Vh ? d_v : nullptr, w ? d_w : nullptr,
                         rank ? d_r : nullptr, d_ws, P->ws_bytes, stream);
  if (rc) return rc;
  CU_OR(P, cudaMemcpyAsync(sigma, d_sg, sizeof(double) * P->k * B, cudaMemcpyDeviceToHost, st));
  if (U) CU_OR(P, cudaMemcpyAsync(U, d_u, c * (size_t)P->m * P->k * B, cudaMemcpyDeviceToHost, st));
  if (Vh) CU_OR(P, cudaMemcpyAsync(Vh, d_v, c * (size_t)P->k * P->n * B, cudaMemcpyDeviceToHost, st));
  if (w) CU_OR(P, cudaMemcpyAsync(w, d_w, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  if (rank) CU_OR(P, cudaMemcpyAsync(rank, d_r, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  int stv = 0, tce = 0;
  CU_OR(P, cudaMemcpyAsync(&stv, P->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU_OR(P, cudaMemcpyAsync(&tce, P->tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU_OR(P, cudaStreamSynchronize(st));
  if (tce) { P->err.set(TEBD_ETIMEOUT, "a tensor-core pipeline wait expired"); return P->err.code; }
  if (stv & 1) { P->err.set(TEBD_ENUMERIC, "an instance had a zero or non-finite theta"); return P->err.code; }
  return TEBD_OK;
}

extern "C" const char* rrsvd_last_error(rrsvd_plan_t P) { return P ? P->err.msg.c_str() : "NULL plan"; }
