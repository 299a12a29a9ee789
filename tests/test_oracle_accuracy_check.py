"""Pins of the oracle's accuracy check (Alg. 2, Thm 2) and of the exact
Frobenius residual identity (Section IV, the Fact 1 discussion)."""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I


def _problem(m=160, n=120, scale=6.0, seed=3):
    sig = I.exp_spectrum(n, scale)
    return I.synthetic_theta(m, n, sig, seed), sig


def test_thm2_probe_bound_holds_after_the_check():
    """Thm 2: ||(I - QQ^H)A|| <= 10 sqrt(2/pi) max_i ||(I - QQ^H) A w_i|| with
    probability >= 1 - 10^-r; after a check that passed, the spectral residual
    of the enlarged basis is below 10 sqrt(2/pi) eps."""
    A, sig = _problem()
    k, p, r, eps = 10, 5, 4, 1e-4
    bound = 10 * np.sqrt(2 / np.pi) * eps
    for t in range(40):
        Q = R._qr_q(A @ gaussian_omega(120, k + p, seed=t))
        Q2, rounds, mx = R.accuracy_check(A, Q, r, eps, 120, seed=t)
        assert mx <= eps
        assert np.linalg.norm(A - Q2 @ (Q2.conj().T @ A), 2) <= bound
        assert Q2.shape[1] == k + p + r * (rounds - 1)


def test_check_grows_the_basis_only_as_needed():
    A, sig = _problem()
    Q = R._qr_q(A @ gaussian_omega(120, 15, seed=1))
    loose = R.accuracy_check(A, Q, 4, 1.0, 120, seed=1)
    assert loose[0].shape[1] == 15 and loose[1] == 1
    widths = [R.accuracy_check(A, Q, 4, eps, 120, seed=1)[0].shape[1] for eps in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert widths == sorted(widths) and widths[-1] > widths[0]
    # the width tracks the exponential spectrum: sigma_j < eps for j >= the width, roughly
    for eps, wdt in zip((1e-2, 1e-4, 1e-6, 1e-8), widths):
        assert sig[wdt - 1] < 50 * eps or wdt + 4 > 120


def test_check_stops_at_l_max():
    A, _ = _problem()
    Q = R._qr_q(A @ gaussian_omega(120, 15, seed=2))
    Q2, rounds, mx = R.accuracy_check(A, Q, 4, 1e-14, 31, seed=2)
    assert Q2.shape[1] == 31 and mx > 1e-14


def test_probe_layout():
    full = R.probe_omega(7, 3, 2, 5)
    flat = gaussian_omega(1, 3 * 7 * 3, 5, stream=1).ravel()[2 * 21:]
    assert np.array_equal(full.ravel(), flat)
    assert not np.allclose(R.probe_omega(7, 3, 0, 5), gaussian_omega(7, 3, 5))   # other stream than Omega


def test_exact_frobenius_residual_identity():
    """||(I - QQ^H)A||_F^2 = ||A||_F^2 - ||A^H Q||_F^2 for orthonormal Q."""
    A, _ = _problem(80, 60)
    Q = R._qr_q(A @ gaussian_omega(60, 12, seed=4))
    lhs = np.linalg.norm(A - Q @ (Q.conj().T @ A)) ** 2
    rhs = np.linalg.norm(A) ** 2 - np.linalg.norm(A.conj().T @ Q) ** 2
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(A) ** 2


def test_fixed_precision_rrsvd_reaches_the_tolerance():
    A, sig = _problem(200, 150, 8.0, 9)
    k, p, q, r, eps = 8, 4, 1, 6, 1e-6
    U, s, Vh, l, kk, resid = R.rrsvd_fixed_precision(A, gaussian_omega(150, k + p, seed=9), q, r, eps, 150, p,
                                                     seed=9)
    assert l > k + p and kk == l - p
    assert abs(resid - np.linalg.norm(A - (U * s) @ Vh)) <= 1e-9
    assert resid <= 10 * np.sqrt(2 / np.pi) * eps * np.sqrt(l)
    assert np.abs(s[:kk] - sig[:kk]).max() <= 1e-8
