"""TEBD handles at the full sizes and in the launch configurations the
benchmark times, on sampled outputs the oracle computes one by one.

Spin-boson chain (spin + 100 bosons, d 32 -> 4, caps 256 -> 64; graphs,
40 GB wave budget): one even sweep from a full-size state on the device, then
sampled even bonds -- the spin bond, the largest theta of the sweep
(~7800 x 7500), a middle and the last one -- against the oracle's update of
the same bond from the same state and the same Omega (Section II.B with the
RRSVD of Section IV).  Even bonds touch disjoint sites, so each sampled
bond's result depends on the pre-sweep state alone.  The state is a seeded
random Vidal form at the caps, not brought into canonical form: the update's
arithmetic does not need it, and it keeps the generation cheap at this size.
Its spectra have no gap at the caps, so the smallest kept Schmidt values of
any randomized truncation move with the rounding order (up to ~5e-6 between
two FP64 codes on the same Omega): they are held to 1e-5, the spin bond (no
truncation) to the form's tolerance.

Many-chain batch (256 uneven XXZ chains, p = 10, q = 1, dt = 0.01; graphs,
16 GB wave budget, waves on both parities): two second-order steps, then
sampled chains against their own oracle runs at the form's tolerances.  Their
Schmidt spectra reach the 1e-14 cutoff (a value of 1.00006e-14 relative is
kept by the FP64 oracle and rounds below the cutoff in the TF32 form), so the
kept ranks may differ by such values and the lists are compared zero-padded."""
import numpy as np
import pytest

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SB_SIZE = (100, 32, 4, 256, 64)
SB_DT, SB_P, SB_Q, SB_SEED = 0.05, 10, 2, 3


def _random_vidal_state(dims, caps, seed):
    """Gamma[s] complex Gaussian (d, chi_{s-1}, chi_s) scaled to O(1) bond
    norms; lambda[b] decaying as exp(-j / (chi/8)), unit 2-norm; every bond at
    its cap min(chi_b, prod_{s<=b} d_s, prod_{s>b} d_s)."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    chi = [1]
    for b in range(N - 1):
        chi.append(int(min(caps[b], np.prod(np.array(dims[:b + 1], dtype=float)),
                           np.prod(np.array(dims[b + 1:], dtype=float)))))
    chi.append(1)
    gam = []
    for s in range(N):
        shape = (dims[s], chi[s], chi[s + 1])
        gam.append((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0 * dims[s] * chi[s]))
    lam = []
    for b in range(N - 1):
        x = np.exp(-np.arange(chi[b + 1]) / max(1.0, chi[b + 1] / 8.0))
        lam.append(x / np.linalg.norm(x))
    return gam, lam, chi


@pytest.fixture(scope="module")
def spin_boson_case():
    dims, caps = I.spin_boson_sizes(*SB_SIZE)
    g0, lam0, chi = _random_vidal_state(dims, caps, 5)
    gates = I.trotter_gates(I.spin_boson_bond_terms(dims), SB_DT / 2)
    N = len(dims)
    even = list(range(0, N - 1, 2))
    size = {b: dims[b] * chi[b] * dims[b + 1] * chi[b + 2] for b in even}
    largest = max(even, key=lambda b: size[b])
    sample = sorted({0, 2, largest, 50, even[-1]})
    ref = {}
    for b in sample:
        mps = T.VidalMPS(g0, lam0)
        info = T.bond_update(mps, b, gates[b], caps[b], SB_P, SB_Q, SB_SEED, 0)
        nb = I.boson_ops(dims[b + 1])[2]
        ref[b] = (mps.lam[b].copy(), T.expect_onesite(mps, b + 1, nb).real, info["theta"].shape)
    return dims, caps, g0, lam0, gates, sample, ref


@pytest.mark.parametrize("prec,tol_spin", [(0, 1e-8), (2, 2e-7)])
def test_spin_boson_full_size_sampled_bonds(lib, spin_boson_case, prec, tol_spin):
    from paper_1504_00992_gb300 import binding as B
    dims, caps, g0, lam0, gates, sample, ref = spin_boson_case
    assert max(np.prod(ref[b][2]) for b in sample) > 7000 * 7000   # the largest theta is in the sample
    sim = B.Tebd(len(dims), 2, 0, SB_P, SB_Q, SB_SEED, d_site=dims, chi_bond=caps, precision=prec,
                 use_graph=1, workspace_budget=40 << 30)
    try:
        sim.set_mps(g0, lam0)
        sim.set_gates(0, gates)
        sim.set_gates(1, gates)
        sim.step_even()
        for b in sample:
            lam_o, n_o, _ = ref[b]
            lg = sim.get_lambda(b)
            assert len(lg) == len(lam_o), b
            assert np.abs(lg - lam_o).max() <= (tol_spin if b == 0 else 1e-5), b
            # the rebuilt Gamma of site b+1 (V^H / lambda_r): its boson number,
            # a gauge-invariant function of the new tensors
            n_g = sim.expect(b + 1, I.boson_ops(dims[b + 1])[2]).real
            assert abs(n_g - n_o) <= (tol_spin if b == 0 else 1e-5) * (dims[b + 1] - 1), b
    finally:
        sim.close()


def _xxz_oracle(N, d, chi, delta, steps, dt, p, q, seed, chain):
    hs = I.xxz_bond_terms(N, d, 1.0, delta)
    ref = T.TEBD(T.product_state(I.neel_state(N, d)), chi, p, q, seed, chain=chain)
    ref.set_gates(0, I.trotter_gates(hs, dt / 2))
    ref.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        ref.second_order_step()
    _, _, sz = I.spin_ops(d)
    return np.array([ref.expect(k, sz).real for k in range(N)]), ref.mps.lam, ref.w_sum


@pytest.mark.parametrize("prec,tol_obs,tol_lam,extra", [
    (0, 1e-8, 1e-8, {"autotune": 1}),
    (2, 1e-7, 2e-7, {}),
])
def test_many_chain_batch_full_size_sampled(lib, prec, tol_obs, tol_lam, extra):
    from paper_1504_00992_gb300 import binding as B
    specs = I.many_chain_specs(256, 0)
    steps, dt, p, q, seed = 2, 0.01, 10, 1, 0
    chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
    sim = B.MultiTebd(chains, p, q, seed, use_graph=1, workspace_budget=16 << 30, precision=prec, **extra)
    try:
        info = sim.workspace_info()
        assert info[1] > 1 and info[2] > 1
        for c, (N, d, chi, delta) in enumerate(specs):
            hs = I.xxz_bond_terms(N, d, 1.0, delta)
            sim.set_product_state(c, I.neel_state(N, d))
            sim.set_gates(c, 0, I.trotter_gates(hs, dt / 2))
            sim.set_gates(c, 1, I.trotter_gates(hs, dt))
        for _ in range(steps):
            sim.step_even(); sim.step_odd(); sim.step_even()
        for c in (0, 131, 255):
            N, d, chi, delta = specs[c]
            exp, lam_o, w_o = _xxz_oracle(N, d, chi, delta, steps, dt, p, q, seed, c)
            _, _, sz = I.spin_ops(d)
            got = np.array([sim.expect(c, k, sz).real for k in range(N)])
            assert np.abs(got - exp).max() <= tol_obs, c
            for b in range(N - 1):
                lg, lo = sim.get_lambda(c, b), lam_o[b]
                # a Schmidt value within rounding of the 1e-14 cutoff may be
                # kept on one side only: the shorter list is padded with zeros,
                # and the values only one side kept must lie at the cutoff
                r = max(len(lg), len(lo))
                pg, po = np.zeros(r), np.zeros(r)
                pg[:len(lg)], po[:len(lo)] = lg, lo
                assert np.abs(pg - po).max() <= tol_lam, (c, b)
                tail = min(len(lg), len(lo))
                assert np.all(np.concatenate([lg[tail:], lo[tail:]]) <= 2e-14 * lo[0]), (c, b)
            assert abs(sim.discarded_weight(c)[0] - w_o) <= 1e-10, c
    finally:
        sim.close()
