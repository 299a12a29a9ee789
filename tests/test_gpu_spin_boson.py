"""Spin-boson chain (star-to-chain form) on the GPU: per-site local
dimensions falling along the chain, per-bond caps falling along the chain, a
canonical random MPS that starts every bond at its cap.  The FP64 handle
matches the oracle (same gates, same Omega); the TF32 form stays within its
stated tolerance of it.  Observable tolerances are relative to the operator
norm of the measured operator (sigma^z: 1; the boson number n on a site of
local dimension d: d - 1), the scale of the error a relative perturbation of
the state produces in <O>."""
import numpy as np
import pytest

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(B, precision, dims, caps, g0, lam0, steps, dt, p, q, seed):
    hs = I.spin_boson_bond_terms(dims)
    N = len(dims)
    sim = B.Tebd(N, 2, 0, p, q, seed, d_site=dims, chi_bond=caps, precision=precision)
    sim.set_mps(g0, lam0)
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    _, _, sz = I.pauli()
    obs = [sim.expect(0, sz).real] + [sim.expect(s, I.boson_ops(dims[s])[2]).real for s in range(1, N)]
    lam = [sim.get_lambda(b) for b in range(N - 1)]
    w = sim.discarded_weight()[0]
    sim.close()
    return np.array(obs), lam, w


def _oracle(dims, caps, g0, lam0, steps, dt, p, q, seed):
    hs = I.spin_boson_bond_terms(dims)
    ref = T.TEBD(T.VidalMPS(g0, lam0), caps, p, q, seed)
    ref.set_gates(0, I.trotter_gates(hs, dt / 2))
    ref.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        ref.second_order_step()
    _, _, sz = I.pauli()
    N = len(dims)
    obs = [ref.expect(0, sz).real] + [ref.expect(s, I.boson_ops(dims[s])[2]).real for s in range(1, N)]
    return np.array(obs), ref.mps.lam, ref.w_sum


@pytest.mark.parametrize("prec,tol_obs,tol_lam", [(0, 1e-8, 1e-8), (2, 1e-7, 2e-7)])
def test_spin_boson_chain_matches_oracle(lib, prec, tol_obs, tol_lam):
    from paper_1504_00992_gb300 import binding as B
    dims, caps = I.spin_boson_sizes(6, 8, 4, 32, 12)
    g0, lam0 = I.random_canonical_mps(dims, caps, 0)
    steps, dt, p, q, seed = 4, 0.05, 10, 2, 3
    obs, lam, w = _run(B, prec, dims, caps, g0, lam0, steps, dt, p, q, seed)
    obs_o, lam_o, w_o = _oracle(dims, caps, g0, lam0, steps, dt, p, q, seed)
    scale = np.array([1.0] + [dims[s] - 1.0 for s in range(1, len(dims))])
    assert np.all(np.abs(obs - obs_o) <= tol_obs * scale)
    for b in range(len(dims) - 1):
        r = min(len(lam[b]), len(lam_o[b]))
        assert np.abs(lam[b][:r] - lam_o[b][:r]).max() <= tol_lam, b
    assert abs(w - w_o) <= 1e-10


@pytest.mark.parametrize("size", [(6, 16, 16, 64, 64), (6, 7, 7, 200, 200)])
@pytest.mark.parametrize("prec,tol_spin", [(0, 1e-8), (2, 2e-7)])
def test_spin_boson_wave_mixes_tiny_and_tall_bonds(lib, prec, tol_spin, size):
    """Head of a chain with d = 16: one parity's wave holds the spin bond
    (theta 2 x 512, l = 2, no truncation) next to bonds of 1024 rows whose QRs
    run over many CTAs per instance, so every instance's scratch must fit its
    own buffers.  One Strang step against the oracle: every kept rank equal,
    the spin bond's Schmidt values to the form's tolerance, the discarded
    weight to 1e-8.  The other bonds start from a random MPS whose spectra
    have no gap at the cap, so the smallest kept values of any randomized
    truncation move with the rounding order (up to ~5e-6 between two FP64
    codes on the same Omega); they are held to 1e-5.  The second chain (d = 7,
    caps 200) has bases of l = 210: the TF32 form re-orthonormalises them with
    the correction read through L1."""
    from paper_1504_00992_gb300 import binding as B
    dims, caps = I.spin_boson_sizes(*size)
    g0, lam0 = I.random_canonical_mps(dims, caps, 0)
    _, lam, w = _run(B, prec, dims, caps, g0, lam0, 1, 0.05, 10, 2, 3)
    _, lam_o, w_o = _oracle(dims, caps, g0, lam0, 1, 0.05, 10, 2, 3)
    for b in range(len(dims) - 1):
        assert len(lam[b]) == len(lam_o[b]), b
        assert np.abs(lam[b] - lam_o[b]).max() <= (tol_spin if b == 0 else 1e-5), b
    assert abs(w - w_o) <= 1e-8
