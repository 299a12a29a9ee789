"""The oracle's reverse pass at the differentiable workload's full size
(transverse-field Ising N=40, chi_max=64, p=10, q=2, 50 second-order steps,
L = <sigma^z_19>) against the oracle's own central differences (eps = 1e-6)
stored by tests/golden/make_golden.py for every coupling: two independent
routes to dL/dJ (the adjoint of each bond update, Section IV's truncation
held fixed, chained through the Frechet derivative of each gate; and 78
forward runs).  The adjoint neglects the coupling to discarded singular
vectors and broadens 1/(s_j^2 - s_i^2); at this size that moves dL/dJ by
about 1e-8 near the site (the differences at eps = 1e-5 and 1e-4 agree with
the stored ones to 1e-9 there, so the gap is the adjoint's, not the
differences')."""
import os

import numpy as np

from oracle import adjoint as AD
from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c4_tfim_n40_dLdJ.txt")


def load_c4_golden():
    """(L, dL/dJ) stored for the workload: L from the header line '# L v'."""
    with open(GOLDEN) as f:
        L = next(float(line.split()[2]) for line in f if line.startswith("# L "))
    return L, np.loadtxt(GOLDEN)[:, 1]


def test_c4_oracle_reverse_pass_matches_stored_differences():
    N, hf, dt, steps, chi, p, q, seed, site = 40, 1.0, 0.02, 50, 64, 10, 2, 0, 19
    J = np.random.default_rng(0).uniform(0.5, 1.5, N - 1)
    hs = I.tfim_bond_terms(J, hf)
    ge, go = I.trotter_gates(hs, dt / 2), I.trotter_gates(hs, dt)
    _, _, sz = I.pauli()
    mps0 = T.product_state([np.array([1.0, 0.0]) for _ in range(N)])
    dG, L = AD.tebd_gradient(mps0, [0, 1, 0] * steps, {0: ge, 1: go}, chi, p, q, seed, site, sz)
    dh = I.tfim_bond_terms_dJ(N)
    g = np.array([np.real(np.vdot(dG[b % 2][b], I.gate_derivative(hs[b], dt / 2 if b % 2 == 0 else dt, dh[b])))
                  for b in range(N - 1)])
    L_fd, fd = load_c4_golden()
    assert abs(L - L_fd) <= 1e-12
    assert np.abs(g - fd).max() <= 5e-8
    # the light cone: couplings far from the site barely move it, the two next to it most
    assert np.argsort(-np.abs(fd))[:2].tolist() in ([19, 18], [18, 19])
    assert np.abs(fd[:14]).max() < 1e-8 and np.abs(fd[24:]).max() < 1e-8
