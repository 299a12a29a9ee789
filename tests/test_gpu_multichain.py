"""Batched form (many chains per launch, CUDA-graph replay, waves under a
workspace budget, autotuned GEMM tiles): every chain agrees with its own
oracle run, and graph replay, waves and tile choices change nothing."""
import numpy as np
import pytest

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _chains(count, seed):
    """Uneven XXZ chains in the style of the many-chain batch: N, d, chi_max,
    Delta drawn per chain."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(6, 13))
        d = int(rng.choice([2, 3]))
        chi = int(rng.choice([4, 8, 12]))
        delta = float(rng.random())
        out.append((N, d, chi, delta))
    return out


def _run_multi(B, specs, steps, dt, p, q, seed, **kw):
    chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
    sim = B.MultiTebd(chains, p, q, seed, **kw)
    for c, (N, d, chi, delta) in enumerate(specs):
        hs = I.xxz_bond_terms(N, d, 1.0, delta)
        sim.set_product_state(c, I.neel_state(N, d))
        sim.set_gates(c, 0, I.trotter_gates(hs, dt / 2))
        sim.set_gates(c, 1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    res = []
    for c, (N, d, chi, delta) in enumerate(specs):
        _, _, sz = I.spin_ops(d)
        res.append((np.array([sim.expect(c, k, sz).real for k in range(N)]),
                    [sim.get_lambda(c, b) for b in range(N - 1)], sim.discarded_weight(c)))
    info = sim.workspace_info()
    sim.close()
    return res, info


def test_multichain_matches_oracle_per_chain(lib):
    from paper_1504_00992_gb300 import binding as B
    specs = _chains(7, 3)
    steps, dt, p, q, seed = 8, 0.1, 4, 2, 9
    res, _ = _run_multi(B, specs, steps, dt, p, q, seed)
    for c, (N, d, chi, delta) in enumerate(specs):
        hs = I.xxz_bond_terms(N, d, 1.0, delta)
        ref = T.TEBD(T.product_state(I.neel_state(N, d)), chi, p, q, seed, chain=c)
        ref.set_gates(0, I.trotter_gates(hs, dt / 2))
        ref.set_gates(1, I.trotter_gates(hs, dt))
        for _ in range(steps):
            ref.second_order_step()
        _, _, sz = I.spin_ops(d)
        exp = np.array([ref.expect(k, sz).real for k in range(N)])
        assert np.abs(res[c][0] - exp).max() <= 1e-8, c
        # these chains truncate hard (d = 3, chi = 8, dt = 0.1): the oracle
        # against itself with another Householder QR moves their Schmidt
        # values by up to 1.8e-9 after 24 sweeps, so 1e-8 is the bar
        for b in range(N - 1):
            lg, lo = res[c][1][b], ref.mps.lam[b]
            r = min(len(lg), len(lo))
            assert np.abs(lg[:r] - lo[:r]).max() <= 1e-8
        assert abs(res[c][2][0] - ref.w_sum) <= 1e-10


def test_graph_waves_and_autotune_change_nothing(lib):
    from paper_1504_00992_gb300 import binding as B
    specs = _chains(9, 5)
    args = (specs, 5, 0.1, 3, 2, 4)
    base, info0 = _run_multi(B, *args)
    assert info0[1] == 1 and info0[2] == 1
    for kw in ({"use_graph": 1}, {"workspace_budget": 200_000}, {"autotune": 1},
               {"use_graph": 1, "workspace_budget": 300_000, "autotune": 1}):
        got, info = _run_multi(B, *args, **kw)
        if "workspace_budget" in kw:
            assert info[1] > 1 and info[2] > 1       # the budget split the sweeps into waves
        # the host-only plan is the plan the handle was created with
        chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
        assert B.tebd_plan_query(chains, 3, 2, 4, autotune=kw.get("autotune", 0),
                                 workspace_budget=kw.get("workspace_budget", 0)) == info
        for (e0, l0, w0), (e1, l1, w1) in zip(base, got):
            assert np.array_equal(e0, e1)
            assert all(np.array_equal(a, b) for a, b in zip(l0, l1))
            assert w0 == w1


def test_single_chain_graph_replay_is_bit_identical(lib):
    from paper_1504_00992_gb300 import binding as B
    N, d = 12, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    outs = []
    for g in (0, 1):
        sim = B.Tebd(N, d, 16, 4, 2, 1, use_graph=g)
        sim.set_product_state(I.neel_state(N, d))
        sim.set_gates(0, I.trotter_gates(hs, 0.025))
        sim.set_gates(1, I.trotter_gates(hs, 0.05))
        for _ in range(10):
            sim.step_even(); sim.step_odd(); sim.step_even()
        _, _, sz = I.spin_ops(d)
        outs.append(np.array([sim.expect(k, sz).real for k in range(N)]))
        assert sim.sweeps() == 30
        sim.close()
    assert np.array_equal(outs[0], outs[1])
