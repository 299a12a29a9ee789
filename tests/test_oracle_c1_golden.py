"""The oracle's RRSVD-TEBD on the XXZ chain N=20 (chi_max=32, p=10, q=2)
reproduces the exact Trotterised state-vector observables stored by
tests/golden/make_golden.py: the discarded weight of this run is ~1e-23, so
the two agree to well within 1e-8."""
import os

import numpy as np

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def test_c1_oracle_matches_state_vector_golden():
    N, d, dt = 20, 2, 0.01
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim = T.TEBD(T.product_state(I.neel_state(N, d)), 32, 10, 2, 0)
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(100):
        sim.second_order_step()
    _, _, sz = I.spin_ops(d)
    got = np.array([sim.expect(k, sz).real for k in range(N)])
    golden = np.loadtxt(os.path.join(HERE, "golden", "c1_xxz_n20_sz_t1.txt"))
    assert np.abs(got - golden[:, 1]).max() <= 1e-8
    assert sim.w_sum < 1e-15
    assert max(len(l) for l in sim.mps.lam) == 32      # the cap is reached in the bulk
