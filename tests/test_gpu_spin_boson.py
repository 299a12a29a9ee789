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
