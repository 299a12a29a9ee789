"""The oracle's pins are sensitive: each plausible mistake, planted in the
oracle on the CPU, makes at least one pin fail."""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle import statevector as SV
from oracle import tebd as T
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I


def _tebd_vs_statevector_error():
    N, d = 8, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    ge, go = I.trotter_gates(hs, 0.05), I.trotter_gates(hs, 0.1)
    rng = np.random.default_rng(0)
    ge = [g @ I.random_unitary(4, rng) for g in ge]      # generic, non-symmetric gates
    psi0 = I.neel_state(N, d)
    sim = T.TEBD(T.product_state(psi0), 64, 10, 2, 0)
    sim.set_gates(0, ge)
    sim.set_gates(1, go)
    psi = SV.product(psi0)
    for _ in range(4):
        sim.second_order_step()
        for par, gs in ((0, ge), (1, go), (0, ge)):
            psi = SV.sweep(psi, N, d, par, gs)
    v = T.to_statevector(sim.mps)
    return abs(abs(np.vdot(v, psi)) - 1.0)


def _exp_spectrum_error():
    n, k, p, q = 200, 40, 10, 2
    sig = I.exp_spectrum(n, 8.0)
    A = I.synthetic_theta(n, n, sig, seed=1)
    _, s, _ = R.rrsvd(A, gaussian_omega(n, k + p, seed=1), q)
    return np.abs(s[:k // 2] - sig[:k // 2]).max()


def _lambda_norm_error():
    N, d = 8, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim = T.TEBD(T.product_state(I.neel_state(N, d)), 3, 2, 2, 0)
    sim.set_gates(0, I.trotter_gates(hs, 0.2))
    sim.set_gates(1, I.trotter_gates(hs, 0.4))
    for _ in range(5):
        sim.second_order_step()
    return max(abs(np.sum(l ** 2) - 1.0) for l in sim.mps.lam)


def test_unmutated_baselines():
    assert _tebd_vs_statevector_error() < 1e-12
    assert _exp_spectrum_error() < 1e-12
    assert _lambda_norm_error() < 1e-13


def test_dropped_middle_lambda_is_caught(monkeypatch):
    orig = T.theta_tensor
    monkeypatch.setattr(T, "theta_tensor", lambda gl, ll, lm, gr, lr: orig(gl, ll, np.ones_like(lm), gr, lr))
    assert _tebd_vs_statevector_error() > 1e-6


def test_transposed_gate_is_caught(monkeypatch):
    orig = T.apply_gate
    monkeypatch.setattr(T, "apply_gate", lambda Tt, G: orig(Tt, np.asarray(G).T))
    assert _tebd_vs_statevector_error() > 1e-6


def test_swapped_gate_legs_are_caught(monkeypatch):
    orig = T.apply_gate

    def swapped(Tt, G):
        d = Tt.shape[0]
        G4 = np.asarray(G).reshape(d, d, d, d).transpose(1, 0, 3, 2)
        return orig(Tt, G4.reshape(d * d, d * d))
    monkeypatch.setattr(T, "apply_gate", swapped)
    assert _tebd_vs_statevector_error() > 1e-6


def test_missing_conjugate_in_power_iteration_is_caught(monkeypatch):
    def bad_range_finder(A, Omega, q):
        Q = R._qr_q(A @ Omega)
        for _ in range(q):
            Qt = R._qr_q(A.T @ Q)           # A^T instead of A^H
            Q = R._qr_q(A @ Qt)
        return Q
    monkeypatch.setattr(R, "range_finder", bad_range_finder)
    assert _exp_spectrum_error() > 1e-8


def test_missing_renormalisation_is_caught(monkeypatch):
    orig = R.truncate
    monkeypatch.setattr(R, "truncate", lambda U, s, Vh, k, cutoff=1e-14: orig(U, s, Vh, k, cutoff))
    orig_bu = T.bond_update

    def no_renorm(mps, b, *a, **kw):
        info = orig_bu(mps, b, *a, **kw)
        mps.lam[b] = info["s"]                 # skip lambda / ||lambda||
        return info
    monkeypatch.setattr(T, "bond_update", no_renorm)
    assert _lambda_norm_error() > 1e-8


def test_wrong_rebuild_division_is_caught(monkeypatch):
    monkeypatch.setattr(T, "_safe_inv", lambda lam: np.ones_like(lam))
    assert _tebd_vs_statevector_error() > 1e-6


def _eckart_young_gap():
    """|A - A_k|_F of the oracle's exact truncation against the closed form
    sqrt(sum_{i>k} sigma_i^2) of a matrix built with known singular values."""
    n, k = 60, 12
    sig = I.exp_spectrum(n, 5.0)
    A = I.synthetic_theta(n, n, sig, seed=4)
    Uk, sk, Vhk, _ = R.exact_truncate(A, k)
    return abs(np.linalg.norm(A - (Uk * sk) @ Vhk) - np.sqrt(np.sum(sig[k:] ** 2)))


def _weight_vs_kept_norm():
    """1 - w against the squared norm of the kept part, formed directly
    (Eq. defdiscweigt for a normalised theta)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 24)) + 1j * rng.standard_normal((30, 24))
    A /= np.linalg.norm(A)
    Uk, sk, Vhk, w = R.exact_truncate(A, 7)
    return abs((1.0 - w) - np.linalg.norm((Uk * sk) @ Vhk) ** 2)


def test_unmutated_truncation_baselines():
    assert _eckart_young_gap() < 1e-13
    assert _weight_vs_kept_norm() < 1e-14


def test_projection_without_conjugate_is_caught(monkeypatch):
    def bad_rrsvd(A, Omega, q):
        Q = R.range_finder(A, Omega, q)
        Ut, s, Vh = np.linalg.svd(Q.T @ A, full_matrices=False)   # Q^T instead of Q^H
        return Q @ Ut, s, Vh
    monkeypatch.setattr(R, "rrsvd", bad_rrsvd)
    assert _exp_spectrum_error() > 1e-8


def test_kept_rank_off_by_one_is_caught(monkeypatch):
    orig = R.kept_rank
    monkeypatch.setattr(R, "kept_rank", lambda s, k, cutoff: max(orig(s, k, cutoff) - 1, 0))
    assert _eckart_young_gap() > 1e-6


def test_weight_from_unsquared_values_is_caught(monkeypatch):
    def bad_weight(s_kept, normF2):
        return 1.0 - float(np.sum(np.asarray(s_kept))) / normF2
    monkeypatch.setattr(R, "discarded_weight", bad_weight)
    assert _weight_vs_kept_norm() > 1e-3
