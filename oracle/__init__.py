"""CPU FP64 correctness oracle for the RRSVD-accelerated TEBD bond update.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test suite, the smoke check and the CPU-baseline
leg of the benchmark use it.  It shares no code with the CUDA path; the only
module both sides use is the seeded input generator, which holds none of the
method's arithmetic.

Modules
  philox   Philox4x64-10 counter-based generator and the complex Gaussian
           sketch matrix Omega drawn from it (Section IV, Alg. 1).
  rrsvd    Randomized SVD with power iterations (Alg. 1) followed by the
           projection B = Q^H A, the SVD of B and U = Q U~ (Section IV, steps
           i-iii); exact dense-SVD truncation (Eckart-Young, Section IV).
  tebd     Vidal-form MPS, theta (Eq. deftheta), gate (Eq. defupdatetheta),
           truncation / renormalisation (Eq. defdiscweigt), sweeps (Eq.
           defst3rd) and one-site expectation values.
  linalg   Hand-written Householder QR and one-sided Jacobi SVD used only as a
           second opinion on tiny cases.
  statevector  Dense state-vector time evolution with the same gates (pins
           TEBD without truncation).
"""
