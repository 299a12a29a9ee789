"""Pins of the oracle's RRSVD (Section IV) against facts fixed by the
mathematics: brute force on tiny cases, hand-written QR/Jacobi as a second
opinion on LAPACK, Eckart-Young (Section IV), the power relation of Eq. powSV,
the expectation bound of Thm 1 and the tail bound of Cor. 1, and closed-form
spectra."""
import numpy as np
import pytest

from oracle import linalg as L
from oracle import rrsvd as R
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I


def _cgauss(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _lowrank(rng, m, n, r):
    return _cgauss(rng, m, r) @ _cgauss(rng, r, n)


@pytest.mark.parametrize("m,n,r,k,p,q", [
    (8, 6, 3, 3, 2, 0), (12, 16, 5, 4, 2, 1), (16, 16, 6, 6, 3, 2), (5, 9, 5, 5, 0, 2), (10, 4, 4, 2, 8, 1)])
def test_exact_when_sketch_covers_rank(m, n, r, k, p, q):
    """Brute force: if l >= rank(A), range(A Omega) = range(A) and RRSVD is
    exact up to rounding (the sketch captures the whole range)."""
    rng = np.random.default_rng(m * 100 + n)
    A = _lowrank(rng, m, n, r)
    kk, l = R.sketch_sizes(m, n, k, p)
    assert l >= min(r, m, n) or l == min(m, n)
    om = gaussian_omega(n, l, seed=5)
    U, s, Vh = R.rrsvd(A, om, q)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(s[:r] - s_ref[:r]).max() <= 1e-13 * s_ref[0]
    assert np.linalg.norm((U * s) @ Vh - A) <= 1e-13 * np.linalg.norm(A)
    # truncated products agree with the dense truncation
    Uk, sk, Vhk, w = R.rrsvd_truncate(A, om, kk, q)
    Ue, se, Vhe, we = R.exact_truncate(A, kk)
    assert np.linalg.norm((Uk * sk) @ Vhk - (Ue * se) @ Vhe) <= 1e-12 * np.linalg.norm(A)
    assert abs(w - we) <= 1e-13


def test_hand_written_qr_and_jacobi_agree_with_lapack():
    rng = np.random.default_rng(1)
    A = _cgauss(rng, 9, 5)
    Q, Rr = L.householder_qr(A)
    assert np.abs(Q @ Rr - A).max() < 1e-14 * 10
    assert np.abs(Q.conj().T @ Q - np.eye(5)).max() < 1e-14 * 10
    U, s, Vh = L.jacobi_svd(A)
    assert np.abs(s - np.linalg.svd(A, compute_uv=False)).max() < 1e-14 * 10
    assert np.abs((U * s) @ Vh - A).max() < 1e-14 * 10


def test_rrsvd_with_hand_written_kernels(monkeypatch):
    """Re-running the RRSVD with the hand-written QR and Jacobi SVD in place of
    LAPACK gives the same truncation: the library calls are used as stated."""
    rng = np.random.default_rng(2)
    sig = np.exp(-np.arange(10) / 2.0)
    A = I.synthetic_theta(14, 10, sig, seed=3)
    om = gaussian_omega(10, 6, seed=9)
    Uk, sk, Vhk, w = R.rrsvd_truncate(A, om, 4, 2)
    monkeypatch.setattr(R, "_qr_q", lambda Y: L.householder_qr(Y)[0])
    monkeypatch.setattr(R.np.linalg, "svd", lambda B, full_matrices=False, compute_uv=True: L.jacobi_svd(B.conj().T)[::-1] if False else _svd_via_jacobi(B))
    Uk2, sk2, Vhk2, w2 = R.rrsvd_truncate(A, om, 4, 2)
    assert np.abs(sk - sk2).max() < 1e-13
    assert np.linalg.norm((Uk * sk) @ Vhk - (Uk2 * sk2) @ Vhk2) < 1e-13
    assert abs(w - w2) < 1e-13


def _svd_via_jacobi(B):
    l, n = B.shape
    if l <= n:
        # B^H = W S Z^H  ->  B = Z S W^H
        W, s, Zh = L.jacobi_svd(B.conj().T)
        return Zh.conj().T, s, W.conj().T
    return L.jacobi_svd(B)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_eckart_young(q):
    """||A - A~||_F >= sqrt(sum_{j>k} s_j^2) for the RRSVD truncation, with
    equality for the dense truncation (Section IV)."""
    rng = np.random.default_rng(10 + q)
    A = _cgauss(rng, 40, 30) * np.exp(-np.arange(30) / 6.0)[None, :]
    k = 8
    s = np.linalg.svd(A, compute_uv=False)
    opt = np.sqrt(np.sum(s[k:] ** 2))
    Uk, sk, Vhk, _ = R.rrsvd_truncate(A, gaussian_omega(30, k + 4, seed=q), k, q)
    err = np.linalg.norm(A - (Uk * sk) @ Vhk)
    assert err >= opt * (1 - 1e-12)
    assert err >= s[k] * (1 - 1e-12)
    Ue, se, Vhe, _ = R.exact_truncate(A, k)
    assert abs(np.linalg.norm(A - (Ue * se) @ Vhe) - opt) <= 1e-12 * s[0]


@pytest.mark.parametrize("q", [1, 2, 3])
def test_power_relation(q):
    """Eq. powSV: s_j((A A^H)^q A) = s_j(A)^(2q+1)."""
    rng = np.random.default_rng(20 + q)
    A = _cgauss(rng, 12, 9) / 4.0
    s = np.linalg.svd(A, compute_uv=False)
    Bq = np.linalg.matrix_power(A @ A.conj().T, q) @ A
    sb = np.linalg.svd(Bq, compute_uv=False)
    assert np.allclose(sb, s ** (2 * q + 1), rtol=1e-10, atol=1e-14 * sb[0])


def test_thm1_expected_error_bound():
    """Thm 1 (Halko Cor. 10.10): the mean spectral error of the range finder
    with q power iterations stays below the stated bound."""
    m, n, k, p, q = 120, 90, 10, 5, 1
    sig = 1.0 / (1.0 + np.arange(n)) ** 0.7
    A = I.synthetic_theta(m, n, sig, seed=4)
    tail = sig[k:]
    bound = ((1 + np.sqrt(k / (p - 1))) * sig[k] ** (2 * q + 1)
             + np.e * np.sqrt(k + p) / p * np.sqrt(np.sum(tail ** (2 * (2 * q + 1))))) ** (1.0 / (2 * q + 1))
    errs = []
    for t in range(200):
        Q = R.range_finder(A, gaussian_omega(n, k + p, seed=1000 + t), q)
        errs.append(np.linalg.norm(A - Q @ (Q.conj().T @ A), 2))
    errs = np.array(errs)
    assert errs.min() >= sig[k + p] * (1 - 1e-10)   # no rank-(k+p) projection beats sigma_{k+p+1}
    assert errs.mean() <= bound


def test_cor1_tail_bound():
    """Cor. 1: with probability >= 1 - 6/p^p the spectral error is below
    alpha^(1/(2q+1)) sigma_{k+1} + beta^(1/(2q+1)) ||tail||_F (the proof's
    constant 6 is used; reading of the garbled statement)."""
    m, n, k, p, q = 100, 80, 8, 4, 1
    sig = np.exp(-np.arange(n) / 10.0)
    A = I.synthetic_theta(m, n, sig, seed=6)
    alpha = 1 + 6 * np.sqrt((k + p) * p * np.log(p))
    beta = 3 * np.sqrt(k + p)
    e = 1.0 / (2 * q + 1)
    bound = alpha ** e * sig[k] + beta ** e * np.sqrt(np.sum(sig[k:] ** 2))
    fails = 0
    trials = 300
    for t in range(trials):
        Q = R.range_finder(A, gaussian_omega(n, k + p, seed=t, chain=1), q)
        if np.linalg.norm(A - Q @ (Q.conj().T @ A), 2) > bound:
            fails += 1
    assert fails / trials <= 6.0 / p ** p + 3.0 / np.sqrt(trials)


def test_exp_spectrum_accuracy():
    """Closed-form spectrum sigma_k = exp(-(k-1)/15) (the single-bond stress
    spectrum, at reduced size): RRSVD with p=20, q=2 meets the accuracy bar
    of the truncation, |ds_i|/s_1 <= 1e-8 for i <= k and an excess Frobenius
    error <= 1e-8 relative, while q=0 misses it."""
    m = n = 400
    k, p, q = 100, 20, 2
    sig = I.exp_spectrum(n)
    A = I.synthetic_theta(m, n, sig, seed=7)
    Uk, sk, Vhk, w = R.rrsvd_truncate(A, gaussian_omega(n, k + p, seed=7), k, q)
    assert np.abs(sk - sig[:k]).max() <= 1e-8 * sig[0]
    assert np.abs(sk[:50] - sig[:50]).max() <= 1e-13 * sig[0]
    opt = np.sqrt(np.sum(sig[k:] ** 2))
    err = np.linalg.norm(A - (Uk * sk) @ Vhk)
    assert (err - opt) / np.linalg.norm(A) <= 1e-8
    w_exact = np.sum(sig[k:] ** 2) / np.sum(sig ** 2)
    # w = 1 - sum s~_i^2 / ||A||_F^2 moves by at most 2 sum s_i |ds_i| (+ rounding)
    assert abs(w - w_exact) <= 2.0 * np.sum(sig[:k] * np.abs(sk - sig[:k])) + 1e-14
    _, s0, _ = R.rrsvd(A, gaussian_omega(n, k + p, seed=7), 0)
    assert np.abs(s0[:k] - sig[:k]).max() > 1e-8 * sig[0]


def test_critical_spectrum_trend():
    """Fig. 2 trend on sigma_i = 1/i: the error of the top-k singular values
    shrinks as q grows, and q = 10 resolves the leading values."""
    m, n, k, p = 300, 150, 20, 20
    sig = 1.0 / (1.0 + np.arange(n))
    A = I.synthetic_theta(m, n, sig, seed=8)
    errs = []
    for q in (0, 2, 10):
        _, s, _ = R.rrsvd(A, gaussian_omega(n, k + p, seed=8), q)
        errs.append(np.abs(s[:k] - sig[:k]).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3 * sig[0]


def test_kept_rank_and_weight_rules():
    s = np.array([1.0, 0.5, 1e-15, 0.0])
    assert R.kept_rank(s, 4, 1e-14) == 2
    assert R.kept_rank(s, 1, 1e-14) == 1
    assert R.kept_rank(np.zeros(3), 3, 1e-14) == 0
    assert R.sketch_sizes(64, 64, 32, 10) == (32, 42)
    assert R.sketch_sizes(2, 2, 32, 10) == (2, 2)
    assert R.sketch_sizes(2000, 2000, 100, 20) == (100, 120)
    assert abs(R.discarded_weight([0.6, 0.6], 1.0) - 0.28) < 1e-15
