/*
 * tebd_gb300.h -- C ABI of the GB300 (sm_103a) TEBD two-site bond update with
 * reduced-rank randomized SVD (RRSVD).
 *
 * Method: Tamascelli, Rosenbach, Plenio, "Improved scaling of Time-Evolving
 * Block-Decimation algorithm through Reduced-Rank Randomized Singular Value
 * Decomposition" (arXiv:1504.00992).
 *
 * Conventions shared by every call
 *   - Complex numbers are two doubles (re, im), interleaved, i.e. the memory
 *     layout of C99 `double _Complex` and numpy complex128.  Every complex
 *     pointer below is typed `double*` and points at the real part of the
 *     first element.
 *   - Matrices are row-major.
 *   - Local basis of a site: index i = 0..d-1.  A two-site operator (gate)
 *     of sites (b, b+1) is a (d_b d_{b+1}) x (d_b d_{b+1}) complex matrix
 *     with <i j|G|i' j'> at row i*d_{b+1} + j, column i'*d_{b+1} + j'.
 *   - Vidal form (Section II.A, Eq. defmps): Gamma[s] is a complex array
 *     [d_s][chi_{s-1}][chi_s]; lambda[b] (bond b between sites b and b+1,
 *     b = 0..N-2) holds chi_b Schmidt values, descending, sum of squares 1.
 *     The two outer bonds have dimension 1 and lambda = 1.
 *   - The blocked theta matrix of bond b (Section II.B) has row
 *     i*chi_{b-1} + alpha and column j*chi_{b+1} + beta.
 *   - Status: every call returns an int, TEBD_OK (0) on success or one of
 *     the negative codes below.  Errors are sticky per handle (the first one
 *     is kept and described by *_last_error) until the handle is destroyed.
 *     No exception crosses the ABI.  One host thread per handle.
 *   - Streams: device work is enqueued on the handle's CUDA stream (default
 *     stream 0 until tebd_set_stream / the stream argument says otherwise).
 *     Calls with host outputs synchronise that stream before returning.
 *   - Ownership: the library copies every host input before the call
 *     returns; the caller keeps its buffers.  Outputs go to caller buffers.
 *     Device pointers passed to rrsvd_execute stay owned by the caller.
 *
 * The sketch matrix Omega of Alg. 1 is drawn from Philox4x64-10
 * (Salmon et al., SC'11): element (r, c) of the n x l matrix uses counter
 * (r*l + c, bond, sweep, chain) and key (seed, 0); the 64-bit words w0, w1
 * become u = ((w >> 12) + 0.5) 2^-52 and Box-Muller gives
 * Re = sqrt(-2 ln u1) cos(2 pi u2), Im = sqrt(-2 ln u1) sin(2 pi u2).
 * `sweep` counts the tebd_step_* calls made on the handle so far; `chain` is
 * the chain (or instance) index.
 */
#ifndef TEBD_GB300_H
#define TEBD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TEBD_OK = 0,
  TEBD_EINVAL = -1,    /* bad argument (size, index, pointer, call order) */
  TEBD_ENOMEM = -2,    /* device or host allocation failed */
  TEBD_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  TEBD_ENUMERIC = -4,  /* non-finite input, or theta with zero norm */
  TEBD_ETIMEOUT = -5,  /* a bounded device wait gave up */
  TEBD_ENOTIMPL = -6,  /* mode not built */
  TEBD_ESTATE = -7     /* call out of order (e.g. a step before its gates) */
};

/* Arithmetic of the RRSVD (Alg. 1 and the steps after it).
 *   TEBD_PREC_FP64: the plain path, every step in FP64.
 *   TEBD_PREC_TF32: the mixed form.  Y0 = A Omega and power rounds 1..q-1
 *     on the tensor cores in TF32 with FP32 accumulation and FP32 QR;
 *     power round q (Y0 when q = 0) as the refinement pass in split 3xTF32
 *     products (FP32-level accuracy); the last basis re-orthonormalised
 *     FP64-accurately (FP32 QR and a double-float Loewdin correction);
 *     B = Q^H A on the tensor cores from exact BF16 digit splits of Q and
 *     A (products exact in FP32, digit levels summed in double-float:
 *     FP64-level accuracy); the QR of B^H by two Cholesky QR passes in
 *     double-float arithmetic (Householder QR in FP64 for an instance whose
 *     Gram matrix is too ill-conditioned); the Jacobi SVD, U, V and lambda
 *     FP64-accurate.  Omega comes from the same Philox words by an FP32
 *     Box-Muller.
 *   TEBD_PREC_BF16: the mixed form with the products before the refinement
 *     round (Y0 and power rounds 1..q-1) in BF16 with FP32 accumulation,
 *     from BF16 roundings of theta and of the FP32 Omega / bases; the
 *     refinement round and everything after it as TEBD_PREC_TF32.  With
 *     q = 0 it is TEBD_PREC_TF32.  The subspace the refinement round starts
 *     from is perturbed at the BF16 level (2^-9 relative), which the power
 *     iteration damps like any other sketch error.
 * Both mixed forms: standalone RRSVD plans and TEBD handles, autotune
 * allowed, not tebd_record. */
enum { TEBD_PREC_FP64 = 0, TEBD_PREC_TF32 = 2, TEBD_PREC_BF16 = 3 };

/* ------------------------------------------------------------------------
 * TEBD handle: an N-site chain in Vidal form resident on the device.
 * ---------------------------------------------------------------------- */
typedef struct tebd_s* tebd_t;

/* Device allocator of a handle (e.g. a framework's caching allocator, so that
 * the handle's memory comes from the same pool as the caller's tensors).
 * alloc(bytes, ctx) returns device memory of the current device, at least
 * 256-byte aligned, or NULL when out of memory; release(ptr, ctx) returns a
 * block.  Blocks are used on the handle's stream and released only after
 * that stream has been synchronised.  Both NULL: cudaMalloc / cudaFree. */
typedef void* (*tebd_alloc_fn)(size_t bytes, void* ctx);
typedef void (*tebd_release_fn)(void* ptr, void* ctx);

typedef struct {
  int N;                /* sites, >= 2 */
  int d;                /* local dimension of every site (used if d_site == NULL), 2..64 */
  const int* d_site;    /* optional: per-site local dimensions, length N */
  int chi_max;          /* bond-dimension cap of every bond (used if chi_bond == NULL) */
  const int* chi_bond;  /* optional: per-bond caps, length N-1 */
  int p;                /* RRSVD oversampling, >= 0 */
  int q;                /* RRSVD power iterations, >= 0 */
  uint64_t seed;        /* Philox key word 0 */
  int precision;        /* TEBD_PREC_* (TF32, BF16: every bond update in a mixed form) */
  double sv_cutoff;     /* keep s_i > sv_cutoff * s_1 among the first k; <= 0 selects 1e-14 */
  int chain;            /* chain index entering the Philox counter (default 0); with
                           tebd_create_multi, chain c uses chain + c */
  int use_graph;        /* nonzero: each sweep is captured once into a CUDA graph and
                           replayed (not while the kernel profiler is enabled); the
                           legacy stream 0 cannot be captured, so such a handle then
                           runs on a blocking stream of its own */
  int autotune;         /* nonzero: at creation, time each wave's launch choices at its
                           capacity sizes and keep the fastest (tebd_wave_info): FP64 --
                           the 16x16 or 32x32 GEMM tiles of every stage and (with
                           fused = 0) the staged sequence against the fused persistent
                           launch; TF32 -- the mixed form's choices as for
                           rrsvd_plan_autotune */
  size_t workspace_budget; /* bytes of per-bond workspace one wave may use (0 = all bonds
                              of a parity in one wave); larger batches run in waves */
  tebd_alloc_fn alloc;     /* optional: allocator of every device block of the handle
                              (read from descs[0]); with release, or both NULL */
  tebd_release_fn release;
  void* alloc_ctx;         /* passed to alloc and release */
  int fused;               /* persistent fused launch (FP64 handles; read from descs[0]):
                              every bond of a wave updated whole by one CTA of one
                              persistent launch, for waves whose bonds have
                              d_l d_r < 32 and m, n <= 512.  0: where the autotuner
                              finds it faster (never without autotune); 1: wherever
                              it fits; -1: never.  Same results as the staged launches,
                              bit for bit */
} tebd_desc_t;

/* Section II (Eq. defmps, deftheta, defupdatetheta) with the RRSVD of
 * Section IV.  Creates a handle for an N-site chain with uniform local
 * dimension d, bond cap chi_max, oversampling p and q power iterations.
 * The state is |0...0> until set.  Device memory is sized once here from
 * the caps (the bond dimension of bond b never exceeds
 * min(chi_max, prod_{s<=b} d_s, prod_{s>b} d_s)).
 * Errors: TEBD_EINVAL (N < 2, d < 2 or > 64, chi_max < 1, p < 0, q < 0,
 * out == NULL; only one of desc alloc / release given, or a block from alloc
 * that is not 256-byte aligned), TEBD_ENOMEM, TEBD_ECUDA.  On error *out is
 * NULL. */
int tebd_create(int N, int d, int chi_max, int p, int q, uint64_t seed, tebd_t* out);

/* As tebd_create, with per-site d, per-bond caps, precision and cutoff. */
int tebd_create_ex(const tebd_desc_t* desc, tebd_t* out);

/* Many independent chains in one handle (Section II.C sweeps, batched over
 * chains): descs[c] describes chain c (N, d, caps, chain index); p, q, seed
 * and precision must agree, use_graph / autotune / workspace_budget are read
 * from descs[0].  tebd_step_even/odd then update the bonds of that parity of
 * every chain in one launch sequence (in waves when a workspace budget is
 * set; with a mixed form the budget also covers the FP32 arrays, laid out
 * at each wave's largest bond, and the bonds are grouped by shape); the
 * per-chain calls (state, gates, expect, lambda, weights, MPS) act on the
 * chain chosen by tebd_select_chain (default 0).
 * Errors: TEBD_EINVAL (n_chains < 1, inconsistent p/q/seed/precision, as
 * tebd_create_ex), TEBD_ENOMEM, TEBD_ECUDA. */
int tebd_create_multi(int n_chains, const tebd_desc_t* descs, tebd_t* out);
int tebd_num_chains(tebd_t h, int* out);
int tebd_select_chain(tebd_t h, int chain);

/* Device bytes held by the handle and the number of waves per parity. */
int tebd_workspace_info(tebd_t h, size_t* arena_bytes, int* waves_even, int* waves_odd);

/* Plan and tuning of wave `wave` of a parity (0 <= wave < its count from
 * tebd_workspace_info).  info (20 ints): [0] bonds in the wave, [1..4] its
 * capacities m, n, k, l, [5] 1 if it runs as the persistent fused launch,
 * [6..11] the GEMM tile of stages Y0, Y~, Y, B^H, U, V (0: by grid size),
 * [12..15] the mixed form's launch choices of mixed-form handles (as
 * rrsvd_plan_tuning's [6..9]), [16] as rrsvd_plan_tuning's [11], [17..19]
 * zero.  ms (2 doubles): the autotuner's timings on
 * synthetic theta -- FP64: the wave's staged and fused RRSVD; TF32: the RRSVD
 * with the size rules and with the choices kept (0 when not timed).
 * Either may be NULL.  Errors: TEBD_EINVAL (parity, wave). */
int tebd_wave_info(tebd_t h, int parity, int wave, int* info, double* ms);

/* The plan tebd_create_multi(n_chains, descs, ...) would make, without
 * creating a handle: the device bytes it would allocate and its waves per
 * parity (what tebd_workspace_info reports for that handle).  Host only: no
 * CUDA call and no GPU needed, so a caller can size workspace_budget before
 * creating.  Any output pointer may be NULL.
 * Errors: as tebd_create_multi's argument checks (TEBD_EINVAL, TEBD_ENOTIMPL);
 * on error the outputs are left unchanged. */
int tebd_plan_query(int n_chains, const tebd_desc_t* descs, size_t* arena_bytes, int* waves_even,
                    int* waves_odd);

/* Frees all device and host memory of the handle (NULL is accepted). */
int tebd_destroy(tebd_t h);

/* Device work of later calls goes to `cuda_stream` (a cudaStream_t). */
int tebd_set_stream(tebd_t h, void* cuda_stream);

/* Moves every device block of the handle to `alloc` / `release` (both NULL:
 * cudaMalloc / cudaFree): the arena is allocated anew, the state (MPS, gates,
 * sweep counter, weights) and any recorded checkpoints are copied into the
 * new blocks, and the old blocks go back to the allocator they came from.
 * Later blocks (checkpoints, reverse-pass buffers) come from `alloc` too.
 * Captured sweep graphs are dropped and captured again at the next step.
 * Synchronises the handle's stream.  On error the handle keeps its old
 * blocks and allocator.
 * Errors: TEBD_EINVAL (only one of alloc / release NULL, a block that is not
 * 256-byte aligned), TEBD_ENOMEM (alloc returned NULL), TEBD_ECUDA. */
int tebd_set_allocator(tebd_t h, tebd_alloc_fn alloc, tebd_release_fn release, void* ctx);

/* Product state of the selected chain: psi is N blocks of d_s complex
 * amplitudes (host), each normalised by the library.  Resets the chain's bond
 * dimensions to 1 and its discarded-weight accumulators, and the handle's
 * sweep counter, to 0.
 * Errors: TEBD_EINVAL (NULL), TEBD_ENUMERIC (a zero or non-finite block). */
int tebd_set_product_state(tebd_t h, const double* psi);

/* Arbitrary Vidal-form state (host arrays, copied): gamma[s] points at a
 * [d_s][chi[s-1]][chi[s]] complex array (chi[-1] = chi[N-1] = 1 implied),
 * lambda[b] at chi[b] doubles, chi has N-1 entries each within the bond's cap.
 * Resets the chain's discarded-weight accumulators and the handle's sweep
 * counter to 0 (tebd_set_sweep_count restores a checkpointed counter).
 * Errors: TEBD_EINVAL. */
int tebd_set_mps(tebd_t h, const double* const* gamma, const double* const* lambda, const int* chi);

/* Copies the state out (checkpoint): chi[] receives N-1 bond dimensions;
 * gamma[s] / lambda[b] must have room for the caps' sizes
 * (d_s * cap_{s-1} * cap_s complex, cap_b doubles); the data are written
 * densely with the current dimensions.  Any of the three may be NULL. */
int tebd_get_mps(tebd_t h, double* const* gamma, double* const* lambda, int* chi);

/* Gates of one parity (Eq. defst3rd: even bonds b % 2 == 0 form F, odd form
 * G).  `gates` holds N-1 complex matrices back to back, gate b of size
 * (d_b d_{b+1})^2; only bonds with b % 2 == parity are read.  Copied to the
 * device.  Errors: TEBD_EINVAL (parity not 0/1, NULL), TEBD_ENUMERIC
 * (non-finite entry). */
int tebd_set_gates(tebd_t h, int parity, const double* gates);

/* One sweep over all bonds of the parity (Section II.C): for each such bond,
 * theta = lambda Gamma lambda Gamma lambda, gate, RRSVD truncation to
 * chi' <= min(cap, m, n) kept values, lambda' = s / ||s||, Gamma rebuilt,
 * discarded weight accumulated.  All bonds of the parity run in one batched
 * launch sequence; asynchronous on the handle's stream.
 * Errors: TEBD_ESTATE (gates of that parity not set), TEBD_ECUDA.  A theta
 * with zero norm is reported by the next synchronising call as
 * TEBD_ENUMERIC. */
int tebd_step_even(tebd_t h);
int tebd_step_odd(tebd_t h);

/* <O_site> = sum lam_l[a]^2 lam_r[c]^2 conj(Gamma^i[a,c]) O[i,i'] Gamma^i'[a,c]
 * (Vidal canonical form).  op: d x d complex (host); out: one complex (host,
 * 2 doubles).  Synchronises.  Errors: TEBD_EINVAL, TEBD_ENUMERIC (a step
 * met a zero theta). */
int tebd_expect(tebd_t h, int site, const double* op, double* out);

/* Schmidt values of a bond: out must hold the bond's cap doubles; *chi gets
 * the current dimension.  Synchronises. */
int tebd_get_lambda(tebd_t h, int bond, double* out, int* chi);

/* out[0] = sum over all bond updates of w_b (Eq. defdiscweigt),
 * out[1] = prod (1 - w_b).  Synchronises. */
int tebd_discarded_weight(tebd_t h, double* out);

/* Number of tebd_step_* calls made (the Philox sweep counter). */
int tebd_sweep_count(tebd_t h, int64_t* out);

/* Sets the sweep counter (count >= 0): Omega of the next step is drawn at
 * sweep `count`.  A run checkpointed with tebd_get_mps + tebd_sweep_count and
 * resumed with tebd_set_mps + tebd_set_sweep_count then draws the same sketch
 * matrices as the uninterrupted run and gives bit-identical states.
 * Errors: TEBD_EINVAL (count < 0), TEBD_ECUDA. */
int tebd_set_sweep_count(tebd_t h, int64_t count);

/* Discarded weight w_b = 1 - sum_kept s^2 / ||theta||_F^2 (Eq. defdiscweigt)
 * of the latest update of every bond b of the selected chain: out holds N-1
 * doubles (host); 0 for bonds not updated since the state was set.
 * Synchronises. */
int tebd_bond_weights(tebd_t h, double* out);

/* Recording for the reverse pass (single-chain handles): while on, every
 * tebd_step_* first stores a device checkpoint of the chain's tensors,
 * Schmidt values, gates and bond dimensions (one allocation per sweep,
 * freed by the next tebd_record(h, 1) or tebd_destroy).  Turning it on
 * clears earlier checkpoints.  Errors: TEBD_ENOTIMPL (several chains, or a
 * mixed-form handle: the reverse pass differentiates the FP64 form),
 * TEBD_ENOMEM. */
int tebd_record(tebd_t h, int on);

/* Gradient of L = Re <O_site> in the current state (O: d x d complex, host;
 * its Hermitian part is used) with respect to the gate matrices of the
 * recorded sweeps, summed over every application of each parity:
 * dgates_even / dgates_odd receive N-1 complex blocks in the tebd_set_gates
 * layout (bonds of the other parity zero; either may be NULL).  The
 * cotangent convention is G_bar = dL/dRe G + i dL/dIm G, so that
 * dL = Re sum conj(G_bar) dG.  Each recorded sweep is recomputed from its
 * checkpoint, then its bond updates are differentiated in reverse: the
 * Vidal extraction, the renormalisation, the truncated SVD the RRSVD
 * approximates (Omega held fixed; 1/(s_j^2 - s_i^2) and 1/s broadened as
 * x/(x^2 + 1e-24); the coupling to discarded singular vectors is neglected),
 * the gate and the contraction.  The forward state, sweep counter and
 * discarded weights are restored afterwards.  Synchronises.
 * Errors: TEBD_EINVAL, TEBD_ESTATE (nothing recorded), TEBD_ENOTIMPL
 * (several chains), TEBD_ENOMEM, TEBD_ECUDA. */
int tebd_backward(tebd_t h, int site, const double* op, double* dgates_even, double* dgates_odd);

/* Text of the first error recorded on the handle ("" if none). */
const char* tebd_last_error(tebd_t h);

/* ------------------------------------------------------------------------
 * Standalone RRSVD truncation of caller-given matrices (Section IV: Alg. 1
 * followed by B = Q^H A, B = U~ S V^H, U = Q U~), batched over instances.
 * ---------------------------------------------------------------------- */
typedef struct rrsvd_plan_s* rrsvd_plan_t;

/* Plan for `batch` complex m x n matrices truncated to k = min(k_max, m, n)
 * singular triplets with sketch width l = min(k + p, m, n) and q power
 * iterations.  Instance t of a call uses Philox counter chain = chain0 + t,
 * bond 0, sweep 0.  precision: TEBD_PREC_FP64, TEBD_PREC_TF32 or
 * TEBD_PREC_BF16 (the workspace then also holds FP32 copies of theta, about
 * 4 m n 8 bytes per instance, and with BF16 half as much again).  Errors: TEBD_EINVAL (m, n, batch < 1, k_max < 1, p < 0,
 * q < 0), TEBD_ENOTIMPL (precision, or l > 512). */
int rrsvd_plan_create(int m, int n, int k_max, int p, int q, int batch, int precision, uint64_t seed,
                      rrsvd_plan_t* out);
int rrsvd_plan_destroy(rrsvd_plan_t plan);

/* Fixed-precision plan (Alg. 1 with the accuracy check of Alg. 2, Thm 2):
 * after Y0 = A Omega and its QR, rounds of check_r Gaussian probes (Philox
 * key word 1 = 1; element (j, c) of round t at counter (t n + j) check_r + c)
 * measure MAX = max_i ||(I - Q Q^H) A w_i||; while MAX > check_eps the probe
 * images A w_i join the basis (re-orthonormalised, l += check_r), up to
 * l_max columns.  The q power iterations and the projection then act on the
 * enlarged basis and each instance keeps up to k = l - p values (its basis
 * width is read back with rrsvd_plan_widths).  Outputs use the capacity
 * k_cap = max(l_max - p, min(k_max, m, n)) (rrsvd_plan_dims), zero past each
 * instance's kept rank.  FP64 only.  check_r = 0 gives rrsvd_plan_create.
 * Errors: as rrsvd_plan_create; TEBD_EINVAL for check_r < 0 or
 * check_eps <= 0 with check_r > 0; TEBD_ENOTIMPL for TF32 with a check. */
int rrsvd_plan_create_ex(int m, int n, int k_max, int p, int q, int batch, int precision, uint64_t seed,
                         int check_r, double check_eps, int l_max, rrsvd_plan_t* out);

/* Basis width l of every instance after the last execute (host array of
 * `batch` ints); synchronises with the device. */
int rrsvd_plan_widths(rrsvd_plan_t plan, int* l_out);

/* Device workspace (bytes) that rrsvd_execute needs, and the plan's k, l. */
int rrsvd_workspace_size(rrsvd_plan_t plan, size_t* bytes);
int rrsvd_plan_dims(rrsvd_plan_t plan, int* k, int* l);

/* Truncates theta (device, batch x m x n complex, contiguous) into
 *   sigma (device, batch x k doubles, descending, zero past the kept rank),
 *   U     (device, batch x m x k complex; may be NULL),
 *   Vh    (device, batch x k x n complex; may be NULL),
 *   w     (device, batch doubles: 1 - sum_{kept} s^2 / ||theta||_F^2; may be NULL),
 *   rank  (device, batch ints: kept count chi' (s_i > 1e-14 s_1); may be NULL),
 * using `workspace` (device, >= rrsvd_workspace_size bytes, 256-byte
 * aligned).  theta is only read.  Asynchronous on `stream`.
 * Errors: TEBD_EINVAL (NULL theta/sigma/workspace, small workspace, chain0 < 0),
 * TEBD_ECUDA.  A bounded tensor-core pipeline wait that expires (TF32 plans)
 * is reported by the next rrsvd_execute_host as TEBD_ETIMEOUT. */
int rrsvd_execute(rrsvd_plan_t plan, const double* theta, int64_t chain0, double* sigma, double* U, double* Vh,
                  double* w, int* rank, void* workspace, size_t workspace_bytes, void* stream);

/* Same truncation from and to HOST buffers (same shapes): copies theta to
 * the device, runs, and copies the results back, all on `stream`, and
 * synchronises.  Device staging buffers and workspace are allocated on the
 * first call and kept by the plan.  Page-locked host buffers let the copies
 * run at the link's rate; pageable ones are staged by the CUDA runtime.
 * Mixed-form plans of 16 instances or more run as four sub-batches, each on
 * a stream of the plan's own (copy in, truncation, copy out), ordered after
 * the work already on `stream` and before the call returns, so that copies
 * overlap kernels; their launch choices are those of the whole batch and the
 * results equal rrsvd_execute's bit for bit.  Errors: TEBD_EINVAL (NULL theta
 * or sigma), TEBD_ENOMEM (staging), TEBD_ECUDA, TEBD_ETIMEOUT, TEBD_ENUMERIC
 * (a zero or non-finite theta, a failed re-orthonormalisation). */
int rrsvd_execute_host(rrsvd_plan_t plan, const double* theta, int64_t chain0, double* sigma, double* U,
                       double* Vh, double* w, int* rank, void* stream);

/* The same truncation from and to HOST buffers without waiting for it:
 * enqueues the copy in (on a copy stream of the plan's own, at once: theta
 * must hold its values when the call is made, whatever work `stream` still
 * has queued), the truncation (on `stream`) and the copy out (on a second
 * stream of the plan's own) and returns.  The plan keeps two staging
 * slots used in turn, so the copy in of a call runs while the previous
 * call's truncation computes; a call blocks only on the host while slots
 * are busy.  theta and the outputs must stay valid, and the outputs unread,
 * until rrsvd_host_wait.  Calls of one plan run their truncations in call
 * order on `stream` and share one device workspace: pass the same stream to
 * every call until rrsvd_host_wait, and do not mix them with rrsvd_execute on
 * the same plan on another stream before it.  Errors: TEBD_EINVAL (NULL theta or
 * sigma, chain0 < 0), TEBD_ENOMEM (two staging slots and a workspace on the
 * first call), TEBD_ECUDA. */
int rrsvd_execute_host_async(rrsvd_plan_t plan, const double* theta, int64_t chain0, double* sigma, double* U,
                             double* Vh, double* w, int* rank, void* stream);

/* Waits for every rrsvd_execute_host_async call of the plan since the last
 * wait; their outputs are then in place.  Returns the first error raised by
 * them: TEBD_ETIMEOUT (an expired tensor-core pipeline wait), TEBD_ENUMERIC
 * (a zero or non-finite theta, a failed re-orthonormalisation), TEBD_ECUDA.
 * rrsvd_execute_host waits for pending calls itself. */
int rrsvd_host_wait(rrsvd_plan_t plan);

const char* rrsvd_last_error(rrsvd_plan_t plan);

/* Autotuner of a plan (the batched launches of Section IV's steps): times
 * the launch choices on the caller's theta (device, as for rrsvd_execute) and
 * keeps the fastest for later executes.  FP64 plans: the GEMM tile of every
 * stage; mixed-form plans: the mixed form's choices (tensor-core tile width,
 * CTA size of the FP32 QRs, one-CTA or many-CTA QR of B^H, one-CTA or
 * cluster Jacobi, the products after the projection on the tensor cores or
 * the CUDA cores), one at a time, each kept only for a clear gain.  Results of a
 * tuned plan agree with an untuned one to rounding.  Synchronises `stream`.
 * Errors: as rrsvd_execute. */
int rrsvd_plan_autotune(rrsvd_plan_t plan, const double* theta, void* workspace, size_t workspace_bytes,
                        void* stream);

/* What the autotuner chose: info (16 ints): [0..5] the FP64 GEMM tile of
 * stages Y0, Y~, Y, B^H, U, V (0: by grid size), [6..9] the mixed form's
 * choices (tile split, FP32 QR threads, QR of B^H, Jacobi; 0: the size rule;
 * Jacobi 1: one CTA in FP64, 2: a cluster per instance in FP64, 3: one CTA
 * in double-float arithmetic),
 * [10] 1 once tuned, [11] the FP64-accurate products after the projection
 * (0: the size rule, 1: tensor cores from digit splits, 2: double-float
 * CUDA-core GEMMs), [12..15] zero; ms (2 doubles, TF32 plans): the step with the size
 * rules and with the choices kept.  Either may be NULL. */
int rrsvd_plan_tuning(rrsvd_plan_t plan, int* info, double* ms);

/* Sets a plan's launch choices (info: 16 ints laid out as rrsvd_plan_tuning
 * gives them; [10] and [12..15] are ignored), e.g. to restore choices tuned
 * in another process or to compare two of them.  The plan counts as tuned
 * afterwards.  Results agree with those of any other choice to rounding.
 * Errors: TEBD_EINVAL (NULL, a tile other than 0, 16 or 32, a choice out of
 * range: [6] 0..1, [7] 0, 128, 256 or 512, [8] 0..3, [9] 0..3, [11] 0..2). */
int rrsvd_plan_set_tuning(rrsvd_plan_t plan, const int* info);

/* Clears the plan's recorded error and its device status flags (a zero or
 * non-finite theta, an expired tensor-core wait): an execute that failed
 * that way leaves nothing behind that the next execute reads, since every
 * buffer of the workspace is written before it is read.  Synchronises the
 * legacy default stream. */
int rrsvd_clear_error(rrsvd_plan_t plan);


/* ------------------------------------------------------------------------
 * Kernel timing (tracing aid).  When enabled, every kernel launch of the
 * library is bracketed by CUDA events on its stream, grouped by kernel class
 * (e.g. "k_zgemm[sketch]", "k_qr", "k_jacobi"; the copies of
 * rrsvd_execute_host as "copy[h2d]" and "copy[d2h]").  Process-wide; not to
 * be enabled while a stream is being captured into a CUDA graph.
 * ---------------------------------------------------------------------- */
int tebd_profiler_enable(int enable);
/* Drops all accumulated timings. */
int tebd_profiler_reset(void);
/* Waits for the recorded events, then writes up to max_entries classes:
 * names (64 chars each, NUL-terminated), total milliseconds and launch
 * counts; *count receives the number of classes (may exceed max_entries). */
int tebd_profiler_read(int max_entries, char* names, double* total_ms, int64_t* launches, int* count);

/* ------------------------------------------------------------------------
 * Failure injection (test hook; the paper has no counterpart).  Faults are
 * made on the host, never by faulting the GPU:
 *   TEBD_FAULT_ALLOC:    the next device allocation of a handle or plan
 *                        (arena, checkpoint, reverse-pass or staging buffer,
 *                        plan descriptors) fails as if out of memory, so the
 *                        call returns TEBD_ENOMEM;
 *   TEBD_FAULT_TC_STALL: the next tensor-core product launched (mixed form)
 *                        outside a stream capture issues none of its operand
 *                        copies and polls its pipeline waits at most 2^12
 *                        times, so its bounded waits expire: the kernel
 *                        raises the timeout flag, writes zeros, frees its
 *                        tensor memory and returns, and the next
 *                        synchronising call reports TEBD_ETIMEOUT.
 * Each armed fault fires once; TEBD_FAULT_NONE disarms all.  Process-wide.
 * Errors: TEBD_EINVAL (unknown kind). */
enum { TEBD_FAULT_NONE = 0, TEBD_FAULT_ALLOC = 1, TEBD_FAULT_TC_STALL = 2 };
int tebd_fault_inject(int kind);

/* ------------------------------------------------------------------------
 * The sketch generator (Section IV, Alg. 1: Omega "drawn from the Gaussian
 * distribution"), exported so that its output can be checked against an
 * independent implementation of the same published generator.  Both calls
 * run the device functions the sketch kernels call, on device buffers owned
 * by the caller, asynchronously on `stream`; they allocate nothing.
 * ---------------------------------------------------------------------- */

/* Philox4x64-10 blocks: for i < count, counter (counters[4i], ..., [4i+3])
 * and key (key0, key1) give words[4i .. 4i+3].  counters and words are
 * device arrays of 4 * count uint64_t.
 * Errors: TEBD_EINVAL (count < 0, NULL buffer with count > 0), TEBD_ECUDA. */
int tebd_philox4x64_10(const uint64_t* counters, int64_t count, uint64_t key0, uint64_t key1, uint64_t* words,
                       void* stream);

/* The n x l sketch matrix of a truncation, row-major into `out` (device):
 * element (r, c) from counter (r*l + c, bond, sweep, chain), key (seed, 0),
 * as described at the top of this header.
 *   TEBD_PREC_FP64: complex128 (2 doubles per element), the Omega of the
 *     FP64 form: u = ((w >> 12) + 0.5) 2^-52, Box-Muller in FP64.
 *   TEBD_PREC_TF32, TEBD_PREC_BF16: complex64 (2 floats per element), the
 *     Omega of the mixed forms before their TF32 or BF16 rounding:
 *     u = ((w >> 40) + 0.5) 2^-24, Box-Muller in FP32.
 * Standalone plans use bond 0, sweep 0 and chain chain0 + instance; TEBD
 * handles use the bond index, the handle's sweep count at the step and the
 * chain index.  Errors: TEBD_EINVAL (negative size or index, NULL out with
 * n l > 0), TEBD_ENOTIMPL (precision), TEBD_ECUDA. */
int rrsvd_sketch_omega(int n, int l, uint64_t seed, int64_t bond, int64_t sweep, int64_t chain, int precision,
                       void* out, void* stream);

/* ------------------------------------------------------------------------
 * No-allocation variant of rrsvd_execute.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * running inside another library's scheduling loop or a host callback that
 * must not block (cudaMalloc may synchronise the device), or a process whose
 * device memory is reserved up front by a caching allocator or a fixed
 * budget -- and so can neither create an rrsvd plan nor supply a workspace.
 *
 * Same truncation, Omega and outputs as rrsvd_execute on a plan created
 * with (m, n, k_max, p, q, batch, TEBD_PREC_FP64, seed); theta, sigma, U,
 * Vh, w and rank are caller device buffers with the shapes given there (U,
 * Vh, w, rank may be NULL).  All scratch is one static 16 MiB device array
 * inside the library, held by every GPU that loads it until the process
 * exits; the call allocates nothing.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and caches it; make that first call before any
 *     stream capture.
 *   - Calls share the array: work of two calls that overlaps on the GPU
 *     (other streams, other host threads) races and corrupts both results.
 *     Order such calls on one stream.
 *   - Errors: TEBD_EINVAL for bad arguments or when descriptors plus
 *     batch x (per-instance workspace, about 16 (5 l (m + n)/2 + 2 l^2 +
 *     2 l k + k (m + n)) bytes) exceed 16 MiB -- e.g. one 512 x 512
 *     instance with k = 128, p = 10 (about 9 MB) fits, one 2048 x 2048 with
 *     k = 100, p = 20 (about 27 MB) does not;
 *     TEBD_ECUDA if a launch or the address lookup fails.
 * Asynchronous on `stream`; zero-norm instances report rank 0 as with
 * rrsvd_execute.
 * ---------------------------------------------------------------------- */
int rrsvd_execute_noalloc(int m, int n, int k_max, int p, int q, int batch, uint64_t seed, int64_t chain0,
                          const double* theta, double* sigma, double* U, double* Vh, double* w, int* rank,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TEBD_GB300_H */
