"""Hand-written Householder QR and one-sided Jacobi SVD (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Used only as a second opinion on LAPACK for tiny matrices, so that a wrong
library call (a transposed operand, a lost conjugate) in the oracle cannot
hide behind the library itself.  Textbook algorithms: Householder reflectors
H = I - 2 v v^H / (v^H v) (Golub & Van Loan, Sec. 5.1-5.2) and Hestenes'
one-sided Jacobi rotations (Golub & Van Loan, Sec. 8.6.3).
"""
import numpy as np


def householder_qr(A):
    """Reduced QR of an m x l complex matrix (m >= l): returns (Q, R)."""
    A = np.array(A, dtype=np.complex128)
    m, l = A.shape
    vs = []
    for j in range(l):
        x = A[j:, j].copy()
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * nx
        v = x.copy()
        v[0] -= alpha
        vv = np.vdot(v, v).real
        if vv == 0.0:
            vs.append(None)
            continue
        A[j:, j:] -= np.outer(v, (2.0 / vv) * (v.conj() @ A[j:, j:]))
        vs.append(v)
    R = np.triu(A[:l, :l])
    Q = np.zeros((m, l), dtype=np.complex128)
    Q[np.arange(l), np.arange(l)] = 1.0
    for j in reversed(range(l)):
        v = vs[j]
        if v is None:
            continue
        vv = np.vdot(v, v).real
        Q[j:, :] -= np.outer(v, (2.0 / vv) * (v.conj() @ Q[j:, :]))
    return Q, R


def jacobi_svd(A, tol=1e-15, max_sweeps=60):
    """One-sided Jacobi SVD of an m x n complex matrix (m >= n).

    Rotates column pairs until all are mutually orthogonal: A J = U S, so that
    A = U S J^H.  Returns (U, s, Vh) with s descending.
    """
    X = np.array(A, dtype=np.complex128)
    m, n = X.shape
    J = np.eye(n, dtype=np.complex128)
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                a = np.vdot(X[:, i], X[:, i]).real
                b = np.vdot(X[:, j], X[:, j]).real
                g = np.vdot(X[:, i], X[:, j])
                ag = abs(g)
                if ag <= tol * np.sqrt(a * b) or ag == 0.0:
                    continue
                rotated = True
                e = g / ag
                zeta = (b - a) / (2.0 * ag)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                xi, xj = X[:, i].copy(), X[:, j].copy()
                X[:, i] = c * xi - s * np.conj(e) * xj
                X[:, j] = s * e * xi + c * xj
                ji, jj = J[:, i].copy(), J[:, j].copy()
                J[:, i] = c * ji - s * np.conj(e) * jj
                J[:, j] = s * e * ji + c * jj
        if not rotated:
            break
    s = np.linalg.norm(X, axis=0)
    order = np.argsort(-s, kind="stable")
    s = s[order]
    X = X[:, order]
    J = J[:, order]
    U = np.zeros_like(X)
    nz = s > 0
    U[:, nz] = X[:, nz] / s[nz]
    return U, s, J.conj().T
