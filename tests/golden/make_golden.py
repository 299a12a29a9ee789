"""Writes the stored expected values under tests/golden/ from the oracle only.

  c1_xxz_n20_sz_t1.txt  <S^z_k> at t = 1 for the XXZ chain N = 20, d = 2,
      J = 1, Delta = 0.5, dt = 0.01, 100 second-order Trotter steps (Eq.
      defst3rd: half-step even, odd, half-step even), Neel initial state,
      from the dense 2^20 state vector (oracle.statevector): the exact
      Trotterised state that TEBD approximates when its discarded weight is
      negligible.  Columns: site, <S^z>.

Run:  python tests/golden/make_golden.py   (about two minutes on 8 cores)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import statevector as SV          # noqa: E402
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


def main():
    vals = c1_statevector()
    with open(os.path.join(HERE, "c1_xxz_n20_sz_t1.txt"), "w") as f:
        f.write("# <S^z_k>(t=1), XXZ N=20 d=2 J=1 Delta=0.5 dt=0.01, 100 Strang steps, Neel; "
                "dense state vector (tests/golden/make_golden.py)\n")
        for k, v in enumerate(vals):
            f.write(f"{k} {v:.17e}\n")


if __name__ == "__main__":
    main()
