"""Writes the stored expected values under tests/golden/ from the oracle only.

  c1_xxz_n20_sz_t1.txt  <S^z_k> at t = 1 for the XXZ chain N = 20, d = 2,
      J = 1, Delta = 0.5, dt = 0.01, 100 second-order Trotter steps (Eq.
      defst3rd: half-step even, odd, half-step even), Neel initial state,
      from the dense 2^20 state vector (oracle.statevector): the exact
      Trotterised state that TEBD approximates when its discarded weight is
      negligible.  Columns: site, <S^z>.

  c4_tfim_n40_dLdJ.txt  the transverse-field Ising chain N = 40, chi_max = 64,
      p = 10, q = 2, seed 0, h = 1, dt = 0.02, 50 second-order steps from
      |0...0>, couplings J_b ~ U[0.5, 1.5] (numpy default_rng(0)),
      L = <sigma^z_19>: L at J and the central differences
      (L(J + eps e_b) - L(J - eps e_b)) / (2 eps), eps = 1e-6, for every b,
      from the oracle's RRSVD-TEBD with the same Omega streams (the
      differentiable workload's reference gradient).  Columns: b, dL/dJ_b;
      L in the header.

Run:  python tests/golden/make_golden.py [c1] [c4]   (c1: about two minutes
on 8 cores; c4: 78 oracle runs of ~5 s each on a pool of worker processes)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import statevector as SV          # noqa: E402
from oracle import tebd as T                  # noqa: E402
from paper_1504_00992_gb300 import inputs as I  # noqa: E402


def c1_statevector():
    N, d, dt, steps = 20, 2, 0.01, 100
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    ge, go = I.trotter_gates(hs, dt / 2), I.trotter_gates(hs, dt)
    psi = SV.product(I.neel_state(N, d))
    for _ in range(steps):
        psi = SV.sweep(psi, N, d, 0, ge)
        psi = SV.sweep(psi, N, d, 1, go)
        psi = SV.sweep(psi, N, d, 0, ge)
    _, _, sz = I.spin_ops(d)
    return [SV.expect_onesite(psi, N, d, k, sz).real for k in range(N)]


C4 = dict(N=40, hf=1.0, dt=0.02, steps=50, chi=64, p=10, q=2, seed=0, site=19, eps=1e-6)


def c4_couplings():
    return np.random.default_rng(0).uniform(0.5, 1.5, C4["N"] - 1)


def c4_observable(J):
    """<sigma^z_site> after the C4 evolution with couplings J (oracle TEBD)."""
    c = C4
    hs = I.tfim_bond_terms(J, c["hf"])
    sim = T.TEBD(T.product_state([np.array([1.0, 0.0]) for _ in range(c["N"])]), c["chi"], c["p"], c["q"],
                 c["seed"])
    sim.set_gates(0, I.trotter_gates(hs, c["dt"] / 2))
    sim.set_gates(1, I.trotter_gates(hs, c["dt"]))
    for _ in range(c["steps"]):
        sim.second_order_step()
    _, _, sz = I.pauli()
    return float(np.real(sim.expect(c["site"], sz)))


def c4_difference(b):
    """Central difference of the C4 observable along coupling b."""
    J0, eps = c4_couplings(), C4["eps"]
    Jp, Jm = J0.copy(), J0.copy()
    Jp[b] += eps
    Jm[b] -= eps
    return (c4_observable(Jp) - c4_observable(Jm)) / (2 * eps)


def write_c1():
    vals = c1_statevector()
    with open(os.path.join(HERE, "c1_xxz_n20_sz_t1.txt"), "w") as f:
        f.write("# <S^z_k>(t=1), XXZ N=20 d=2 J=1 Delta=0.5 dt=0.01, 100 Strang steps, Neel; "
                "dense state vector (tests/golden/make_golden.py)\n")
        for k, v in enumerate(vals):
            f.write(f"{k} {v:.17e}\n")


def write_c4():
    os.environ["OPENBLAS_NUM_THREADS"] = "1"      # one thread per worker; the workers inherit it
    L = c4_observable(c4_couplings())
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 16)) as pool:
        d = pool.map(c4_difference, range(C4["N"] - 1))
    c = C4
    with open(os.path.join(HERE, "c4_tfim_n40_dLdJ.txt"), "w") as f:
        f.write(f"# TFIM N={c['N']} chi={c['chi']} p={c['p']} q={c['q']} seed={c['seed']} h={c['hf']} "
                f"dt={c['dt']} steps={c['steps']} site={c['site']} J~U[0.5,1.5] default_rng(0); "
                f"oracle central differences eps={c['eps']} (tests/golden/make_golden.py)\n")
        f.write(f"# L {L:.17e}\n")
        for b, v in enumerate(d):
            f.write(f"{b} {v:.17e}\n")


def main():
    which = sys.argv[1:] or ["c1", "c4"]
    if "c1" in which:
        write_c1()
    if "c4" in which:
        write_c4()


if __name__ == "__main__":
    main()
