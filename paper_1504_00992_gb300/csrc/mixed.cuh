// Buffers and entry of the mixed-precision RRSVD (mixed.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "internal.cuh"

namespace tg {

// Padded sizes of the real-embedded operands of one instance.
struct MixedSizes {
  int bf16;      // 1: the products before the refinement round in BF16 (TEBD_PREC_BF16)
  int K1;        // 2n rounded up to 32: row length of theta's forward copy and of Bt for A X
  int K2;        // 2m rounded up to 32: row length of the adjoint copy and of Bt for A^H X
  int K1b, K2b;  // the same rounded up to 64 for the BF16 copies (128-byte rows)
  int Np;        // 2l rounded up to 16: rows of Bt (tensor-core N)
  int BN;        // tensor-core tile width, min(Np, 256)
  size_t thf, tha, bt, yf, ytf, df;  // bytes per instance
  size_t bd, bsc, ad, asc;  // BF16 digits and block scales of theta and of Q_f^H (tensor-core projection)
  size_t thfb, thab, btb;   // BF16 copies of theta, theta^H and Bt (bf16 only)
  size_t gad, gas, gbd, gbs;  // digit scratch of the other tensor-core products (oz_stage_bytes)
  size_t qs;     // bytes per instance of the many-CTA FP32 QR's scratch (0: not used)
  int ntile;     // 32 x 32 tiles of the theta conversion (partials of ||theta||_F^2)
};

// Batch-major arrays (instance z at base + z * per-instance size).
struct MixedPtrs {
  float* thf_hi;  // m x K1, TF32-rounded theta (Re, Im interleaved)
  float* thf_lo;  // TF32 remainder of theta
  float* tha_hi;  // n x K2, TF32-rounded theta^H
  float* tha_lo;
  float* bt_hi;   // Np x K (K1 or K2), real embedding of the right operand
  float* bt_lo;
  float2* Yf;     // m x l complex FP32, column-major
  float2* Qf;
  float2* Ytf;    // n x l
  float2* Qtf;
  float2* Df;     // l x l correction of the re-orthonormalisation
  uint16_t* bd;   // digits of theta for the tensor-core projection (oz_proj.cu)
  float* bsc;     // their block scales
  uint16_t* ad;   // digits of Q_f^H
  float* asc;
  uint16_t* thf_b;  // m x K1b BF16 theta (bf16 form), or null
  uint16_t* tha_b;  // n x K2b BF16 theta^H
  uint16_t* bt_b;   // Np x max(K1b, K2b) BF16 right operand
  uint16_t* gad;  // digit scratch of the Cholesky QR and U / V products (OzScratch)
  float* gas;
  uint16_t* gbd;
  float* gbs;
  double* tpart;  // ntile partial sums of |theta|^2 per instance
  float2* qscr;   // scratch of the many-CTA FP32 QR (qs bytes per instance), or null
};

MixedSizes mixed_sizes(int m, int n, int k, int l, int bf16 = 0, const Caps* gate = nullptr);
// The arrays of instances z0, z0 + 1, ... of a carve (every array advanced
// by z0 instances): run_rrsvd_mixed on a sub-batch starting at instance z0.
MixedPtrs mixed_offset(const MixedPtrs& p, const MixedSizes& s, int z0);
size_t mixed_bytes(const MixedSizes& s, int batch);
MixedPtrs mixed_carve(char* base, const MixedSizes& s, int batch);

// Blocked FP32 Householder QR (qr_blocked.cu): A (M x L column-major per
// instance, overwritten) -> Q; usable when qr_blk_f32_fits(M, L).  With
// dims, each instance factors only its own rows (D.n if use_n, else D.m) and
// D.l columns of the zero-padded M x L layout.
bool qr_blk_f32_fits(int M, int L);
// threads: 0 picks the CTA size by batch; 128, 256 or 512 force it (when its
// shared memory fits)
cudaError_t launch_qr_blk_f32(float2* A, float2* Q, int M, int L, int batch, cudaStream_t st,
                              const Dims* dims = nullptr, int use_n = 0, int threads = 0);
// The same QR spread over many CTAs per instance (qr_multi.cu), for matrices
// too tall for the blocked kernel's shared memory; scr holds
// qr_multi_f32_scratch(M, L) float2 per instance at the given stride; with
// dims each instance is factored at its own size, as above.
bool qr_multi_f32_fits(int M, int L);
size_t qr_multi_f32_scratch(int M, int L);
cudaError_t launch_qr_multi_f32(float2* A, float2* Q, float2* scr, size_t stride, int M, int L, int batch,
                                cudaStream_t st, const Dims* dims = nullptr, int use_n = 0);
// Q_f (FP32, M x L) -> ptrs[z].Q (FP64) orthonormal to ~1e-13, spanning
// range(Q_f), from E = Q_f^H Q_f - I already in ptrs[z].R (launch_oz_gram);
// usable when reorth_fits(M, L).
bool reorth_fits(int M, int L);
cudaError_t launch_reorth(const float2* Qf, float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int M, int L,
                          int batch, int* status, cudaStream_t st);
// B^H <- B^H (I + D) in place on ptrs[z].Yt (qr_blocked.cu).
cudaError_t launch_fold_bh(const float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int n, int l, int batch,
                           cudaStream_t st);

// B^H = A^H Q_f (I + D) into ptrs[z].Yt on the tensor cores from BF16 digits
// (oz_proj.cu): launch_oz_digits_theta once theta is in place, launch_proj_oz
// after launch_reorth.  Arrays at capacities m x n (theta) and m x l (Q_f).
int oz_kpad(int m);
size_t oz_digits_bytes(int rows, int m);
size_t oz_scales_bytes(int rows, int m);
cudaError_t oz_prepare();
// The other FP64-accurate products on the tensor cores (GemmStage G_G1 ..
// G_X of the Cholesky QR, G_U, G_V): digit scratch of both operands, sized
// by oz_stage_bytes for the capacities, reused by every stage.
struct OzScratch {
  uint16_t* ad;
  float* as;
  uint16_t* bd;
  float* bs;
};
struct OzStageBytes {
  size_t ad, as, bd, bs;  // per instance
};
// gate: the capacities of a TEBD wave whose bonds take the contraction and
// gate GEMMs (stages OZ_THETA, OZ_GATE of launch_oz_stage), or null
OzStageBytes oz_stage_bytes(int m, int n, int k, int l, const Caps* gate = nullptr);
// the contraction and gate GEMMs of a wave on the tensor cores: stages
// OZ_THETA (into the pre-gate buffers) and OZ_GATE (into theta) of
// launch_oz_stage; the wave's bonds without a pre-gate buffer are skipped
enum { OZ_THETA_STAGE = 102, OZ_GATE_STAGE = 103 };
bool oz_gate_rule(const Caps& cap);
cudaError_t launch_oz_stage(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                            const OzScratch& sc, int* err, cudaStream_t st);
// the size rule of MixedKnobs::dfg: the tensor-core products for bonds whose
// products are deep and wide enough to fill the digit-pair pipeline
bool oz_stage_rule(const Caps& cap);

// Cholesky QR (two passes) of B^H for well-conditioned instances, Householder
// for the others (cholqr.cu); writes dims[p].qflag.  oz: the products on the
// tensor cores (raising *err on a pipeline stall), or null for double-float
// GEMMs.
cudaError_t run_cholqr_bh(Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st,
                          const OzScratch* oz, int* err);
cudaError_t cholqr_prepare();
cudaError_t launch_oz_digits_theta(const Dims* dims, const ProbPtr* ptrs, uint16_t* Bd, float* Bs, int m, int n,
                                   int batch, cudaStream_t st);
// (digits_done: Q_f's digits already in Ad / As from launch_oz_digits_qf)
cudaError_t launch_proj_oz(const Dims* dims, const ProbPtr* ptrs, const float2* Qf, const float2* Dbuf,
                           uint16_t* Ad, float* As, const uint16_t* Bd, const float* Bs, int m, int n, int l, int batch,
                           int* err, cudaStream_t st, bool digits_done = false);
// Digits of conj(Q_f) (the projection's left operand) into Ad / As, and the
// Gram matrix E = Q_f^H Q_f - I of the re-orthonormalisation from them into
// ptrs[z].R (l x l column-major), FP64-accurate, on the tensor cores.
cudaError_t launch_oz_digits_qf(const Dims* dims, const float2* Qf, uint16_t* Ad, float* As, int m, int l, int batch,
                                cudaStream_t st);
cudaError_t launch_oz_gram(const Dims* dims, const ProbPtr* ptrs, const uint16_t* Ad, const float* As, int m, int l,
                           int batch, int* err, cudaStream_t st);

// Launch choices of the mixed form that the autotuner may override (0 keeps
// each size rule): tc_half = 1 splits the tensor-core products' columns over
// two CTAs; qr_threads sets the CTA size of the blocked FP32 QRs (128, 256,
// 512); qrbh forces the QR of B^H (1 one-CTA Householder, 2 many-CTA
// Householder, 3 Cholesky QR with Householder for ill-conditioned instances;
// the size rule takes the Cholesky QR wherever it would run the one-CTA
// kernel); jac forces the Jacobi SVD as in launch_jacobi_sized.
// Launch choices of the mixed form (0: the size rule).  jac: 1 the one-CTA
// FP64 Jacobi, 2 the cluster form, 3 the one-CTA double-float one.  dfg: the
// Cholesky QR
// and U / V products on the tensor cores (digit splits, 0 by rule / 1) or as
// double-float CUDA-core GEMMs (2).
struct MixedKnobs {
  int tc_half, qr_threads, qrbh, jac, dfg;
};

// Everything that must happen outside a stream capture before
// run_rrsvd_mixed runs on capacities `cap` (shared-memory limits, the
// tensor-map encoder entry point).
cudaError_t mixed_prepare(const Caps& cap);
cudaError_t qr_blocked_prepare(int M, int N, int L);

// Alg. 1 with tensor-core products and the FP64-accurate projection / FP64
// small SVD.  The FP32 arrays are laid out at the capacities `cap` (the
// maxima over the batch, which size mixed_sizes/mixed_carve); each instance
// uses its own (m, n, k, l) from dims, zero-padded up to them.  Instance z
// draws Omega from chain chain0 + z chain_stride at `sweep`, or, with
// chain_stride < 0, from its own chain index at *sweep_dev.
cudaError_t run_rrsvd_mixed(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, const MixedPtrs& mp,
                            int q, uint64_t seed, uint64_t sweep, int64_t chain0, int chain_stride, int* status,
                            int* err, cudaStream_t st, const uint64_t* sweep_dev = nullptr,
                            const MixedKnobs* knobs = nullptr, int bf16 = 0);

}  // namespace tg
