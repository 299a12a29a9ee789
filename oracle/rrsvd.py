"""Reduced-rank randomized SVD (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Section IV of the paper in its own order:
  * Alg. 1 (randomized range finder with q power iterations, each product
    re-orthonormalised by a QR factorisation);
  * the three closing steps of Section IV: B = Q^H A, the SVD B = U~ S V^H,
    and U = Q U~;
  * the fixed-rank truncation to the first k singular triplets and the exact
    alternative, the dense SVD truncated to rank k, whose optimality is the
    Eckart-Young statement of Section IV (Frobenius error
    sqrt(sum_{i>k} s_i^2)).

NumPy's LAPACK QR and SVD serve as library steps; nothing is blocked, fused or
reordered beyond the algorithm as stated.
"""
import numpy as np


def sketch_sizes(m, n, k_max, p):
    """k = min(k_max, m, n) and l = min(k + p, m, n).

    Reading of the paper: Alg. 1 assumes k + p < n; when the oversampled rank
    reaches min(m, n) the sketch is simply the whole range and the method is
    exact up to rounding.
    """
    k = min(k_max, m, n)
    l = min(k + p, m, n)
    return k, l


def _qr_q(Y):
    """Orthonormal factor of the reduced QR factorisation Y = Q R."""
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def range_finder(A, Omega, q):
    """Alg. 1: Q with orthonormal columns spanning approx. the range of A.

    Y0 = A Omega, Y0 = Q0 R0; for j = 1..q: Y~j = A^H Q_{j-1} = Q~j R~j,
    Yj = A Q~j = Qj Rj.  Returns Q_q.
    """
    Y = A @ Omega
    Q = _qr_q(Y)
    for _ in range(q):
        Yt = A.conj().T @ Q
        Qt = _qr_q(Yt)
        Y = A @ Qt
        Q = _qr_q(Y)
    return Q


def rrsvd(A, Omega, q):
    """Alg. 1 followed by the projection steps i-iii of Section IV.

    Returns (U, s, Vh) with U = Q U~ (m x l), s (l, descending), Vh (l x n),
    so that A ~= U diag(s) Vh.
    """
    Q = range_finder(A, Omega, q)
    B = Q.conj().T @ A                                   # step i
    Ut, s, Vh = np.linalg.svd(B, full_matrices=False)    # step ii
    U = Q @ Ut                                           # step iii
    return U, s, Vh


def dense_svd(A):
    """Exact mode: the full SVD of A (what RRSVD approximates)."""
    return np.linalg.svd(A, full_matrices=False)


def kept_rank(s, k, cutoff):
    """Number of leading singular values kept.

    The first k values are candidates (fixed-rank problem, Section IV); of
    those, only values above cutoff * s[0] are kept so that the Vidal-form
    division by lambda stays defined (reading of the paper, which is silent on
    exact zeros in fixed-rank mode).  Returns 0 only if s[0] == 0.
    """
    kk = min(k, len(s))
    if kk == 0 or not (s[0] > 0.0):
        return 0
    thr = cutoff * s[0]
    r = 0
    while r < kk and s[r] > thr:
        r += 1
    return r


def truncate(U, s, Vh, k, cutoff=1e-14):
    """Keep the leading chi' <= k singular triplets."""
    r = kept_rank(s, k, cutoff)
    return U[:, :r], s[:r], Vh[:r, :]


def frob2(A):
    """Squared Frobenius norm ||A||_F^2 = sum |a_ij|^2 (Eq. frobNorm)."""
    return float(np.vdot(A, A).real)


def discarded_weight(s_kept, normF2):
    """w = 1 - sum_{i<=chi'} s_i^2 / ||A||_F^2 (Eq. defdiscweigt for a state
    whose squared Schmidt values sum to ||A||_F^2)."""
    if normF2 <= 0.0:
        return 0.0
    return 1.0 - float(np.sum(np.asarray(s_kept) ** 2)) / normF2


def rrsvd_truncate(A, Omega, k, q, cutoff=1e-14):
    """RRSVD then truncation: (U_k, s_k, Vh_k, w)."""
    U, s, Vh = rrsvd(A, Omega, q)
    Uk, sk, Vhk = truncate(U, s, Vh, k, cutoff)
    return Uk, sk, Vhk, discarded_weight(sk, frob2(A))


def exact_truncate(A, k, cutoff=1e-14):
    """Dense SVD truncation (the Eckart-Young optimum): (U_k, s_k, Vh_k, w)."""
    U, s, Vh = dense_svd(A)
    Uk, sk, Vhk = truncate(U, s, Vh, k, cutoff)
    return Uk, sk, Vhk, discarded_weight(sk, frob2(A))


def probe_omega(n, r, t, seed, bond=0, sweep=0, chain=0):
    """Probe matrix of accuracy-check round t (n x r): Philox stream 1, probe
    element (j, c) at counter index (t n + j) r + c."""
    from .philox import gaussian_omega
    full = gaussian_omega(1, (t + 1) * n * r, seed, bond, sweep, chain, stream=1).ravel()
    return full[t * n * r:(t + 1) * n * r].reshape(n, r)


def accuracy_check(A, Q, r, eps, l_max, seed, bond=0, sweep=0, chain=0):
    """Alg. 2 (accuracy check): while the largest probe residual
    max_i ||(I - Q Q^H) A w_i|| exceeds eps, append the r probe images A Omega_r
    to Q and re-orthonormalise (l += r); stop when the check passes or when
    l + r would exceed l_max (the paper's l <= n - r, with n >= l_max).
    Returns (Q, rounds, last MAX)."""
    t = 0
    while True:
        Om = probe_omega(A.shape[1], r, t, seed, bond, sweep, chain)
        Br = A @ Om
        D = Br - Q @ (Q.conj().T @ Br)
        mx = float(np.max(np.linalg.norm(D, axis=0)))
        t += 1
        if mx > eps:
            Q = _qr_q(np.concatenate([Q, Br], axis=1))
        if not (mx > eps and Q.shape[1] + r <= l_max):
            return Q, t, mx


def rrsvd_fixed_precision(A, Omega, q, r, eps, l_max, p, seed, bond=0, sweep=0, chain=0):
    """Alg. 1's sketch and first basis, the accuracy check of Alg. 2 on Q0, the q power
    iterations of Alg. 1 on the (possibly enlarged) basis, then steps i-iii.
    The kept rank follows the basis: k = l - p.  Returns (U, s, Vh, l, k,
    exact Frobenius residual of the final Q)."""
    Q = _qr_q(A @ Omega)
    Q, _, _ = accuracy_check(A, Q, r, eps, l_max, seed, bond, sweep, chain)
    for _ in range(q):
        Qt = _qr_q(A.conj().T @ Q)
        Q = _qr_q(A @ Qt)
    B = Q.conj().T @ A
    Ut, s, Vh = np.linalg.svd(B, full_matrices=False)
    l = Q.shape[1]
    resid = np.sqrt(max(frob2(A) - frob2(B), 0.0))   # ||(I - Q Q^H) A||_F = sqrt(||A||^2 - ||Q^H A||^2)
    return Q @ Ut, s, Vh, l, max(l - p, 1), resid
