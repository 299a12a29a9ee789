// Internal descriptors and launch entry points of the bond-update pipeline.
//
// One "problem" is one bond update (TEBD) or one given matrix (standalone
// RRSVD).  Its sizes live on the device (Dims) because bond dimensions change
// from sweep to sweep without the host reading them back; its buffers
// (ProbPtr) are carved once from a workspace sized by the capacities.
// Every matrix is row-major and compact: its leading dimension is its actual
// column count.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tg {

struct Dims {
  int m, n;        // theta rows (d_l chi_l) and columns (d_r chi_r)
  int k, l;        // target rank min(chi_cap, m, n) and sketch width min(k + p, m, n)
  int dl, dr;      // local dimensions of the two sites
  int cl, cm, cr;  // bond dimensions left of, between and right of the two sites
  int bond;        // bond index (Philox counter word 1)
  int active;      // 0: skip this problem
  int chain;       // Philox chain index (counter word 3) of chain-driven launches
  int r;           // accuracy check: probes per round (0 = no check)
  int chk;         // accuracy check still running for this problem
  int qflag;       // this round extended the basis: re-orthonormalise it
};

struct ProbPtr {
  // operands of the theta contraction (TEBD only)
  const cplx* gl;     // Gamma[b]   [dl][cap_l][cap_m]
  const cplx* gr;     // Gamma[b+1] [dr][cap_m][cap_r]
  const double* laml; // lambda left  (cap_l)
  const double* lamm; // lambda middle (cap_m)
  const double* lamr; // lambda right (cap_r)
  const cplx* gate;   // (dl dr)^2
  int cap_l, cap_m, cap_r, pad0;
  // static description of a chain bond (TEBD only): where its bond
  // dimensions live on the device and its fixed sizes
  int* chi_l;         // bond dimension left of the two sites
  int* chi_m;         // bond dimension between them (rewritten by the rebuild)
  int* chi_r;
  int dl_s, dr_s;     // local dimensions
  int chicap;         // user cap on the kept rank
  int bond_s;         // bond index within its chain
  int chain_s;        // Philox chain index of the chain
  int slot;           // chain slot in the handle (discarded-weight accumulators)
  double* wbond;      // where the bond's latest discarded weight goes (TEBD only), or null
  // RRSVD buffers
  const cplx* theta;  // m x n (read only for the sketches)
  cplx* omega;        // n x l
  cplx* Y;            // m x l   (QR input, overwritten by reflectors)
  cplx* Q;            // m x l
  cplx* Yt;           // n x l   (QR input, overwritten by reflectors)
  cplx* Qt;           // n x l
  cplx* R;            // l x l   (R factor of B^H, then Jacobi working matrix)
  cplx* J;            // l x l   (accumulated Jacobi rotations)
  cplx* Jk;           // l x k   (sorted leading columns of J)
  cplx* Wk;           // l x k   (sorted leading normalised columns of R J)
  cplx* U;            // m x k   (Q Jk)
  cplx* V;            // n x k   (Qt Wk)
  double* sigma;      // l       (sorted descending)
  double* part;       // NPART partial sums of |theta|^2
  double* scal;       // per-problem scalars: [0] ||theta||_F^2, [1] w, [2] kept rank
  cplx* Dr;           // m x r: Q Q^H A Omega_r of the accuracy check
  cplx* Cpre;         // m x n pre-gate theta of a bond whose gate is applied as a GEMM (large d_l d_r), or null
};

enum { NPART = 64 };

// GEMM stages of the pipeline (op(A) op(B) -> C).
enum GemmStage { G_Y0 = 0, G_YT = 1, G_Y = 2, G_BH = 3, G_U = 4, G_V = 5,
                 // accuracy check: Br = A Omega_r (into Y after the basis), C1 = Q^H Br, Dr = Q C1
                 G_PR = 6, G_PQ = 7, G_PD = 8,
                 // Cholesky QR of B^H (the mixed form, cholqr.cu): G1 = B B^H into R,
                 // Q1 = B^H R1^-1 into omega, G2 = Q1^H Q1 into R, Qb = Q1 R2^-1 into Qt,
                 // X = B Qb (= Rb^H) into R; the inverse factors come in J
                 G_G1 = 9, G_Q1 = 10, G_G2 = 11, G_QB = 12, G_X = 13 };
// QR stages: which buffer is factored and where Q goes.
enum QrStage { QR_Y = 0, QR_YT = 1, QR_BH = 2 };

// Capacities (maxima over the batch) used to size grids.
struct Caps {
  int m, n, k, l;
  int cl, cr, dl, dr;
  int r;  // accuracy-check probes per round
  int cm;  // largest middle-bond capacity (TEBD waves)
};

// --- launchers (kernels.cu) ---------------------------------------------
// chain_stride >= 0: instance p uses Philox chain chain0 + p * chain_stride and
// the host-given sweep; chain_stride < 0: dims[p].chain and *sweep_dev.
cudaError_t launch_omega(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, uint64_t seed,
                         uint64_t sweep, int64_t chain0, int chain_stride, cudaStream_t st,
                         const uint64_t* sweep_dev = nullptr);
cudaError_t launch_zgemm(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                         cudaStream_t st);
cudaError_t launch_qr(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st,
                      int only_flagged = 0);
// the same, spread over many CTAs per instance (qr_multi.cu) when the batch
// is a few tall matrices (cap.m or cap.n rows, cap.l columns); every
// instance's R and J buffers must hold at least qr_multi_scratch_r(l) and
// qr_multi_scratch_j(l) complex words for its own l
// force: 0 the size rule, 1 the one-CTA kernel, 2 the many-CTA form wherever
// its structure allows (the autotuner's choices)
cudaError_t launch_qr_sized(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                           cudaStream_t st, int force = 0);
// true when launch_qr_sized(stage, ..., force) runs the many-CTA form
bool qr_multi_chosen(int stage, const Caps& cap, int batch, int force);
size_t qr_multi_scratch_r(int l);
size_t qr_multi_scratch_j(int l);
cudaError_t launch_jacobi(const Dims* dims, const ProbPtr* ptrs, int batch, int* status, cudaStream_t st);
// the same, each instance on a cluster of CTAs (jacobi_cluster.cu) when the
// batch is a few instances with cap.l >= 64
// force: 0 the size rule, 1 one CTA per matrix, 2 the cluster form wherever l allows
cudaError_t launch_jacobi_sized(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int* status,
                                cudaStream_t st, int force = 0);
// true when launch_jacobi_sized(..., force) runs the cluster form
bool jacobi_cluster_chosen(const Caps& cap, int batch, int force);
// the one-CTA Jacobi SVD in double-float arithmetic (jacobi_df.cu), the mixed
// form's: same outputs as launch_jacobi, FP64-accurate to 2^-48
// (lcap: the widest instance's l; X is held in shared memory where it fits)
cudaError_t launch_jacobi_df(const Dims* dims, const ProbPtr* ptrs, int batch, int lcap, int* status,
                             cudaStream_t st);
cudaError_t jacobi_df_prepare();
cudaError_t launch_frob2(const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st);
// identity_gate = 1 writes the pre-gate theta (reverse pass).  Otherwise a
// bond with ptrs[p].Cpre set gets its pre-gate theta written there, and
// launch_gate_gemm applies its gate; skip_pre = 1 leaves those bonds to
// launch_theta_df.
cudaError_t launch_theta(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st,
                         int identity_gate = 0, int skip_pre = 0);
// theta~ = G C for the bonds with Cpre set (a complex GEMM over the physical
// indices, FP64): local dimensions with d_l d_r >= GATE_GEMM_MIN take this path.
enum { GATE_GEMM_MIN = 32 };
cudaError_t launch_gate_gemm(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st);
// the same in double-float arithmetic on the FP32 pipes (FP64-accurate; df_gemm.cu)
cudaError_t launch_gate_gemm_df(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st);
// the pre-gate theta of the bonds with Cpre set, in double-float arithmetic (df_gemm.cu)
cudaError_t launch_theta_df(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st);

// standalone RRSVD epilogue: sigma/U/Vh/w/rank into caller buffers
cudaError_t launch_rrsvd_finalize(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, double cutoff,
                                  double* sigma, double* Vh, double* w, int* rank, int* status, cudaStream_t st);

// the whole RRSVD from theta to (sigma, Jk, Wk, U, V): Alg. 1 + steps i-iii
cudaError_t run_rrsvd(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int q, uint64_t seed,
                      uint64_t sweep, int64_t chain0, int chain_stride, int* status, cudaStream_t st,
                      const uint64_t* sweep_dev = nullptr, const int* tiles = nullptr);

// Accuracy check (Alg. 2) rounds between the first basis of Alg. 1 and the power
// iterations: rounds = host bound on the number of rounds; l grows on the
// device; eps the threshold; stream-1 Philox probes.
cudaError_t run_accuracy_check(const Dims* dims_mut, const ProbPtr* ptrs, int batch, const Caps& cap, int rounds,
                               double eps, int l_max, int p, uint64_t seed, uint64_t sweep, int64_t chain0,
                               int chain_stride, cudaStream_t st);
// the whole fixed-precision RRSVD (Alg. 1 + Alg. 2 + steps i-iii), FP64
cudaError_t run_rrsvd_checked(Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int q, int rounds,
                              double eps, int l_max, int p, uint64_t seed, int64_t chain0, int* status,
                              cudaStream_t st);

cudaError_t launch_finalize_checked(const Dims* dims, const ProbPtr* ptrs, int batch, int kcap, double cutoff,
                                    double* sigma, double* Uout, double* w, int* rank, int* lw, int* status,
                                    cudaStream_t st);
cudaError_t launch_checked_init(Dims* dims, int batch, const Dims& tmpl, cudaStream_t st);

// Double-float (FP32-pair) variant of the FP64 GEMM for G_U and G_V (U = Q J_k,
// V = Qb W_k of the mixed form); other stages return cudaErrorInvalidValue.
cudaError_t launch_zgemm_df(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                            cudaStream_t st);

// GEMM tile choice per stage (16 or 32); tiles == nullptr picks by grid size.
cudaError_t launch_zgemm_tile(int stage, int tile, const Dims* dims, const ProbPtr* ptrs, int batch,
                              const Caps& cap, cudaStream_t st);

// --- TEBD-specific (tebd_kernels.cu) -------------------------------------
struct ChainDev {
  int N;
  int* chi_ext;          // N+1 bond dims, chi_ext[0] = chi_ext[N] = 1, chi_ext[b+1] = chi of bond b
  const int* dsite;      // N local dims
  double** lam_ext;      // N+1 pointers, outer ones point at a constant 1.0
  cplx** gamma;          // N pointers
  const int* cap_ext;    // N+1 capacities of the bonds (outer = 1)
};

// per-bond sizes of a wave of problems from the current bond dimensions
cudaError_t launch_plan(const ProbPtr* ptrs, Dims* dims, int batch, int p, cudaStream_t st);
// truncation, renormalisation and Gamma rebuild; w of problem i goes to wout[i]
cudaError_t launch_rebuild(const Dims* dims, const ProbPtr* ptrs, int batch, double cutoff, double* wout,
                           int* status, cudaStream_t st);
// adds the w of a wave into the per-slot accumulators (2 doubles per chain slot)
cudaError_t launch_wacc(const Dims* dims, const ProbPtr* ptrs, const double* wout, int batch, double* wacc,
                        cudaStream_t st);
cudaError_t launch_sweep_tick(uint64_t* sweep_dev, cudaStream_t st);
cudaError_t launch_expect(const ChainDev& ch, int site, const cplx* op, int d, cplx* out, cudaStream_t st);

// --- persistent fused bond update (fused.cu) -------------------------------
// Bonds of a wave whose capacities satisfy fused_fits can be updated by one
// persistent launch instead of the staged sequence; `queue` is a device int
// that starts at zero (the kernel leaves it at zero).  With dims_in set, the
// RRSVD alone of theta already in place (the tuner's timing run).
enum { FUSED_MAXMN = 512 };
bool fused_fits(const Caps& cap);
cudaError_t fused_prepare();
cudaError_t launch_bond_fused(const ProbPtr* ptrs, Dims* dims, const Dims* dims_in, int batch, int p_os, int q,
                              uint64_t seed, const uint64_t* sweep_dev, double cutoff, double* wout, int* status,
                              int* queue, cudaStream_t st);
cudaError_t launch_tune_theta(const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st);

}  // namespace tg
