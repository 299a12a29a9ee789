"""The persistent fused bond update (every bond of a wave updated whole by
one CTA of one persistent launch; Section II.B with the RRSVD of Section IV,
all bonds of a parity at once by Section II.C, Eq. defst3rd).

It runs the staged kernels' stage code with their per-element summation
orders, so it must give the staged path's states bit for bit, and hence the
oracle's to the FP64 tolerances."""
import numpy as np
import pytest

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _xxz(B, N, d, chi, p, q, seed, steps, dt, fused, **kw):
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim = B.Tebd(N, d, chi, p, q, seed, fused=fused, **kw)
    sim.set_product_state(I.neel_state(N, d))
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    _, _, sz = I.spin_ops(d)
    lam = [sim.get_lambda(b) for b in range(N - 1)]
    ex = np.array([sim.expect(k, sz) for k in range(N)])
    w = sim.discarded_weight()
    wb = sim.bond_weights()
    table = sim.tuning_table()
    sim.close()
    return lam, ex, w, wb, table


@pytest.mark.parametrize("N,d,chi,p,q,steps", [
    (20, 2, 32, 10, 2, 30),    # the XXZ chain of the benchmark (theta 64 x 64), 90 sweeps
    (11, 3, 20, 6, 1, 6),      # spin-1, ragged sizes (theta 60 x 60), odd chain length
    (8, 4, 12, 4, 3, 4),       # d = 4, q = 3
])
def test_fused_equals_staged_bit_for_bit_and_matches_oracle(lib, N, d, chi, p, q, steps):
    from paper_1504_00992_gb300 import binding as B
    dt, seed = 0.02, 7
    fl, fe, fw, fwb, table = _xxz(B, N, d, chi, p, q, seed, steps, dt, fused=1, use_graph=1)
    assert all(w["fused"] == 1 for par in (0, 1) for w in table[par])   # every wave took the fused launch
    sl, se, sw, swb, table_s = _xxz(B, N, d, chi, p, q, seed, steps, dt, fused=-1)
    assert all(w["fused"] == 0 for par in (0, 1) for w in table_s[par])
    for a, b in zip(fl, sl):
        assert np.array_equal(a, b)
    assert np.array_equal(fe, se) and fw == sw and np.array_equal(fwb, swb)
    # and the oracle, to the FP64 bars (observables 1e-8 after the steps)
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    ref = T.TEBD(T.product_state(I.neel_state(N, d)), chi, p, q, seed)
    ref.set_gates(0, I.trotter_gates(hs, dt / 2))
    ref.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        ref.second_order_step()
    _, _, sz = I.spin_ops(d)
    exp = np.array([ref.expect(k, sz) for k in range(N)])
    assert np.abs(fe - exp).max() <= 1e-8
    for b in range(N - 1):
        lo = ref.mps.lam[b]
        r = max(len(lo), len(fl[b]))
        x, y = np.zeros(r), np.zeros(r)
        x[:len(lo)], y[:len(fl[b])] = lo, fl[b]
        assert np.abs(x - y).max() <= 1e-10, b
    assert abs(fw[0] - ref.w_sum) <= 1e-10


def test_fused_many_chain_waves_equal_staged(lib):
    """Uneven chains in one handle, several waves per parity (a workspace
    budget): the persistent launch balances bonds of different sizes and
    still gives the staged states bit for bit."""
    from paper_1504_00992_gb300 import binding as B
    specs = I.many_chain_specs(24, 3)
    chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
    out = {}
    for fused in (1, -1):
        sim = B.MultiTebd(chains, 10, 1, 0, use_graph=1, workspace_budget=256 << 20, fused=fused)
        info = sim.workspace_info()
        assert info[1] > 1 and info[2] > 1
        for c, (N, d, chi, delta) in enumerate(specs):
            hs = I.xxz_bond_terms(N, d, 1.0, delta)
            sim.set_product_state(c, I.neel_state(N, d))
            sim.set_gates(c, 0, I.trotter_gates(hs, 0.005))
            sim.set_gates(c, 1, I.trotter_gates(hs, 0.01))
        for _ in range(8):
            sim.step_even(); sim.step_odd(); sim.step_even()
        res = []
        for c, (N, d, _, _) in enumerate(specs):
            _, _, sz = I.spin_ops(d)
            res.append(([sim.get_lambda(c, b) for b in range(N - 1)],
                        np.array([sim.expect(c, k, sz) for k in range(N)]), sim.discarded_weight(c)))
        out[fused] = (res, sim.tuning_table())
        sim.close()
    assert any(w["fused"] for par in (0, 1) for w in out[1][1][par])
    for (la, ea, wa), (lb, eb, wb) in zip(out[1][0], out[-1][0]):
        for x, y in zip(la, lb):
            assert np.array_equal(x, y)
        assert np.array_equal(ea, eb) and wa == wb


def test_autotuner_times_both_launches(lib):
    from paper_1504_00992_gb300 import binding as B
    hs = I.xxz_bond_terms(20, 2, 1.0, 0.5)
    sim = B.Tebd(20, 2, 32, 10, 2, 0, autotune=1, use_graph=1)
    table = sim.tuning_table()
    for par in (0, 1):
        for w in table[par]:
            staged, fused = w["tune_ms"]
            assert staged > 0 and fused > 0
            assert w["fused"] == (1 if fused < staged else 0)
            assert all(t in (16, 32) for t in w["tiles"])
    sim.set_product_state(I.neel_state(20, 2))
    sim.set_gates(0, I.trotter_gates(hs, 0.005))
    sim.set_gates(1, I.trotter_gates(hs, 0.01))
    for _ in range(3):
        sim.step_even(); sim.step_odd(); sim.step_even()
    assert sim.discarded_weight()[0] < 1e-10
    sim.close()
