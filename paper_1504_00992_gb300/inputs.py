"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the
oracle.

This module holds none of the bond update's arithmetic: it builds the
caller-side inputs of the method (Hamiltonian bond terms and their Trotter
gates, initial product states, random Vidal-form tensors and synthetic theta
matrices with a prescribed singular spectrum).  Random numbers come from
NumPy's PCG64 generator seeded by the caller.

Conventions
  * local basis index i = 0..d-1 is the spin projection m = s - i with
    s = (d - 1) / 2 (index 0 is "up");
  * a two-site operator is a (d_l d_r) x (d_l d_r) matrix with <ij|O|i'j'> at
    [i*d_r + j, i'*d_r + j'];
  * complex arrays are numpy complex128 (interleaved re, im in memory).
"""
import numpy as np


def spin_ops(d):
    """(Sx, Sy, Sz) for spin s = (d-1)/2 in the basis m = s, s-1, ..., -s."""
    s = (d - 1) / 2.0
    m = s - np.arange(d)
    sz = np.diag(m).astype(np.complex128)
    sp = np.zeros((d, d), dtype=np.complex128)   # S+ |m> = sqrt(s(s+1) - m(m+1)) |m+1>
    for i in range(1, d):
        mm = m[i]
        sp[i - 1, i] = np.sqrt(s * (s + 1) - mm * (mm + 1))
    sm = sp.conj().T
    sx = 0.5 * (sp + sm)
    sy = -0.5j * (sp - sm)
    return sx, sy, sz


def pauli():
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return sx, sy, sz


def xxz_bond_terms(N, d=2, J=1.0, Delta=0.5):
    """h_b = J (Sx Sx + Sy Sy + Delta Sz Sz) on bond (b, b+1), b = 0..N-2."""
    sx, sy, sz = spin_ops(d)
    h = J * (np.kron(sx, sx) + np.kron(sy, sy) + Delta * np.kron(sz, sz))
    return [h.copy() for _ in range(N - 1)]


def tfim_bond_terms(Js, h=1.0):
    """Transverse-field Ising, H = -sum_b J_b Z_b Z_{b+1} - h sum_i X_i
    (Pauli operators).  The field on an inner site is split 1/2 : 1/2 between
    its two bonds; the end sites carry their full field on their only bond."""
    sx, _, sz = pauli()
    N = len(Js) + 1
    eye = np.eye(2, dtype=np.complex128)
    out = []
    for b, Jb in enumerate(Js):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b + 1 == N - 1 else 0.5
        out.append(-Jb * np.kron(sz, sz) - h * (wl * np.kron(sx, eye) + wr * np.kron(eye, sx)))
    return out


def tfim_bond_terms_dJ(N):
    """d h_b / d J_b = -Z Z (the same for every bond)."""
    _, _, sz = pauli()
    return [-np.kron(sz, sz) for _ in range(N - 1)]


def unitary_from_hermitian(h, tau):
    """exp(-i h tau) through the eigendecomposition of the Hermitian h."""
    e, V = np.linalg.eigh(h)
    return (V * np.exp(-1j * tau * e)) @ V.conj().T


def trotter_gates(bond_terms, tau):
    return [unitary_from_hermitian(h, tau) for h in bond_terms]


def neel_state(N, d=2):
    """Site k in m = +s for even k, m = -s for odd k."""
    out = []
    for k in range(N):
        v = np.zeros(d, dtype=np.complex128)
        v[0 if k % 2 == 0 else d - 1] = 1.0
        out.append(v)
    return out


def random_unitary(dim, rng):
    """Haar-random unitary (QR of a complex Gaussian with the phase fix)."""
    Z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def random_bond(dl, dr, chi_l, chi_m, chi_r, rng, decay=4.0):
    """Random operands of one bond update: Gamma_l (dl, chi_l, chi_m),
    Gamma_r (dr, chi_m, chi_r), positive descending lambdas normalised to
    sum(lambda^2) = 1, and a Haar-random two-site gate."""
    def lam(c):
        v = np.exp(-np.arange(c) / max(c / decay, 1e-300)) * (1.0 + 0.1 * rng.random(c))
        v = np.sort(v)[::-1]
        return v / np.sqrt(np.sum(v ** 2))

    gl = (rng.standard_normal((dl, chi_l, chi_m)) + 1j * rng.standard_normal((dl, chi_l, chi_m)))
    gr = (rng.standard_normal((dr, chi_m, chi_r)) + 1j * rng.standard_normal((dr, chi_m, chi_r)))
    return {
        "gamma_l": gl, "gamma_r": gr,
        "lam_l": lam(chi_l), "lam_m": lam(chi_m), "lam_r": lam(chi_r),
        "gate": random_unitary(dl * dr, rng),
    }


def exp_spectrum(n, scale=15.0):
    """sigma_k = exp(-(k-1)/scale), k = 1..n."""
    return np.exp(-np.arange(n) / scale)


def _reflector_apply_left(X, v):
    """(I - 2 v v^H / v^H v) X."""
    return X - np.outer(v, (2.0 / np.vdot(v, v).real) * (v.conj() @ X))


def synthetic_theta(m, n, sigma, seed, reflectors=4):
    """theta = U diag(sigma) V^H with U, V products of `reflectors` Householder
    reflectors built from complex Gaussian vectors (exactly unitary, O(mn)
    work each).  len(sigma) <= min(m, n)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    X = np.zeros((m, n), dtype=np.complex128)
    X[np.arange(r), np.arange(r)] = sigma
    for _ in range(reflectors):
        v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        X = _reflector_apply_left(X, v)
    Xt = X.conj().T                               # apply V^H from the right via its adjoint
    for _ in range(reflectors):
        v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        Xt = _reflector_apply_left(Xt, v)
    return np.ascontiguousarray(Xt.conj().T)


def haar_theta(m, n, sigma, seed):
    """theta = U diag(sigma) V^H with Haar-random U (m x r) and V (n x r)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = random_unitary(m, rng)[:, :r]
    V = random_unitary(n, rng)[:, :r]
    return (U * sigma[None, :]) @ V.conj().T


def many_chain_specs(count=256, seed=0):
    """Uneven XXZ chains of the many-chain batch: N ~ U{16..128},
    d in {2, 3, 4}, chi_max in {32, 64, 128}, Delta ~ U[0, 1]; returns a list of
    (N, d, chi_max, Delta)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(16, 129))
        d = int(rng.choice([2, 3, 4]))
        chi = int(rng.choice([32, 64, 128]))
        out.append((N, d, chi, float(rng.random())))
    return out


def gate_derivative(h, tau, dh):
    """Frechet derivative of the gate G = exp(-i tau h) along dh (h Hermitian), the
    caller-side chain rule from gate cotangents to Hamiltonian couplings: with
    h = W diag(e) W^H, dG = W [ (W^H dh W) o Phi ] W^H, Phi_ij the divided
    difference of exp(-i tau e) between e_i and e_j."""
    e, W = np.linalg.eigh(h)
    f = np.exp(-1j * tau * e)
    de = e[:, None] - e[None, :]
    same = np.abs(de) < 1e-12 * max(1.0, np.abs(e).max())
    Phi = np.where(same, -1j * tau * f[:, None] * np.ones_like(de), (f[:, None] - f[None, :]) / np.where(same, 1.0, de))
    return W @ ((W.conj().T @ dh @ W) * Phi) @ W.conj().T


# ---------------------------------------------------------------------------
# Spin-boson chain (star-to-chain form of the paper's TEDOPA applications; the
# chain coefficients are simple stand-ins): a spin coupled through sigma^z to
# the first of n bosonic sites,
#   H = (Delta_s/2) sx + t0 sz (a_1 + a_1^+) + sum_n omega n_n
#       + sum_n t_n (a_n^+ a_{n+1} + a_n a_{n+1}^+),   t_n = t0 / (1 + n),
# bosons truncated to d_n levels falling linearly from d_first to d_last.
# ---------------------------------------------------------------------------
def boson_ops(d):
    """(a, a^+, n) on a boson truncated to d levels |0>..|d-1>."""
    a = np.diag(np.sqrt(np.arange(1, d)), 1).astype(np.complex128)
    return a, a.conj().T, np.diag(np.arange(d)).astype(np.complex128)


def spin_boson_sizes(n_bosons, d_first, d_last, chi_first, chi_last):
    """Local dimensions [2, d_1 .. d_n] and per-bond caps chi_b, both falling
    linearly (rounded) along the chain."""
    nb = n_bosons
    ds = [2] + [int(round(d_first - (d_first - d_last) * (k - 1) / max(1, nb - 1))) for k in range(1, nb + 1)]
    chis = [int(round(chi_first - (chi_first - chi_last) * b / max(1, nb - 1))) for b in range(nb)]
    return ds, chis


def spin_boson_bond_terms(dims, omega=1.0, t0=0.5, delta_s=1.0):
    """Bond Hamiltonians h_b on sites (b, b+1) of the spin-boson chain with
    local dimensions dims = [2, d_1, ...]; on-site terms split half and half
    between the two bonds of a site, with full weight at the chain ends."""
    N = len(dims)
    sx, _, sz = pauli()
    out = []
    for b in range(N - 1):
        dl, dr = dims[b], dims[b + 1]
        il, ir = np.eye(dl), np.eye(dr)
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b + 1 == N - 1 else 0.5
        ar, adr, nr = boson_ops(dr)
        if b == 0:
            h = t0 * np.kron(sz, ar + adr) + wl * 0.5 * delta_s * np.kron(sx, ir)
        else:
            al, adl, nl = boson_ops(dl)
            tb = t0 / (1.0 + b)
            h = tb * (np.kron(adl, ar) + np.kron(al, adr)) + wl * omega * np.kron(nl, ir)
        h = h + wr * omega * np.kron(il, nr)
        out.append(h)
    return out


def spin_boson_product_state(dims):
    """|up> (x) |0 ... 0>."""
    out = []
    for d in dims:
        v = np.zeros(d, dtype=np.complex128)
        v[0] = 1.0
        out.append(v)
    return out


def random_canonical_mps(dims, chi_caps, seed, return_raw=False):
    """Seeded random MPS brought into Vidal form: bond b carries
    chi_b = min(cap_b, prod_{s<=b} d_s, prod_{s>b} d_s); column j of each
    random tensor is weighted by exp(-j / (chi/8)) so the Schmidt values decay;
    a right QR sweep then a left SVD sweep give Gamma[s] (d, chi_{s-1}, chi_s)
    and Schmidt vectors lambda[b] (sum lambda^2 = 1).  A caller-side fixture:
    it makes every bond start at its cap.  return_raw also returns the random
    tensors (the same state, unnormalised and not canonical)."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    chi = [1]
    for b in range(N - 1):
        left = float(np.prod([float(x) for x in dims[: b + 1]]))
        right = float(np.prod([float(x) for x in dims[b + 1:]]))
        chi.append(int(min(chi_caps[b], left, right)))
    chi.append(1)
    A = []
    for s in range(N):
        t = rng.standard_normal((dims[s], chi[s], chi[s + 1])) + 1j * rng.standard_normal((dims[s], chi[s], chi[s + 1]))
        w = np.exp(-np.arange(chi[s + 1]) / max(1.0, chi[s + 1] / 8.0))
        A.append(t * w[None, None, :])
    # right sweep: A[s] -> right-orthonormal B[s] (rows a of the chi_{s-1} x (d chi_s) matrix orthonormal)
    B = [None] * N
    carry = None
    for s in range(N - 1, -1, -1):
        t = A[s] if carry is None else np.einsum("iag,gh->iah", A[s], carry)
        d, cl, cr = t.shape
        M = t.transpose(1, 0, 2).reshape(cl, d * cr)          # rows alpha, columns (i, gamma)
        if s == 0:
            B[s] = t / np.linalg.norm(M)
            break
        Qt, Rt = np.linalg.qr(M.conj().T)                      # M = Rt^H Qt^H, Qt^H with orthonormal rows
        k = Qt.shape[1]
        B[s] = Qt.conj().T.reshape(k, d, cr).transpose(1, 0, 2)
        carry = Rt.conj().T                                    # cl x k, absorbed into A[s-1]
        if k != cl:
            raise ValueError("bond %d lost rank in the QR sweep" % s)
    # left sweep: SVDs give the Schmidt values and Gamma
    gam, lam = [], []
    psi = B[0]
    lam_prev = np.ones(1)
    for s in range(N - 1):
        d, cl, cr = psi.shape
        M = psi.reshape(d * cl, cr)                            # rows (i, alpha), i-major
        U, S, Vh = np.linalg.svd(M, full_matrices=False)
        nrm = np.linalg.norm(S)
        U, S, Vh = U[:, :cr], S[:cr] / nrm, Vh[:cr]
        inv = np.where(lam_prev > 0, 1.0 / np.where(lam_prev > 0, lam_prev, 1.0), 0.0)
        gam.append(U.reshape(d, cl, cr) * inv[None, :, None])
        lam.append(S)
        psi = np.einsum("g,gh,jhc->jgc", S, Vh, B[s + 1])
        lam_prev = S
    inv = np.where(lam_prev > 0, 1.0 / np.where(lam_prev > 0, lam_prev, 1.0), 0.0)
    gam.append(psi * inv[None, :, None])
    if return_raw:
        return gam, lam, A
    return gam, lam
