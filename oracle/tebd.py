"""Vidal-form TEBD with RRSVD truncation (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

State (Section II.A, Eq. defmps / relcoefmat): for N sites, Gamma[k] is a
(d_k, chi_{k-1}, chi_k) complex array and lambda[k] (k = 0..N-2) holds the
Schmidt values of the bond between sites k and k+1.  The outer bonds of the
chain have dimension 1 and lambda = [1].

Two-site update of bond b (sites b, b+1), Section II.B:
  1. Theta(i,j,a,c) = sum_g lam_l[a] Gam_b^i[a,g] lam_m[g] Gam_{b+1}^j[g,c] lam_r[c]
     (Eq. deftheta);
  2. Theta~(i,j,a,c) = sum_{i'j'} <ij|G|i'j'> Theta(i',j',a,c)
     (Eq. defupdatetheta);
  3. reshape to the blocked matrix with row (i, a) -> i*chi_l + a and column
     (j, c) -> j*chi_r + c;
  4. truncated SVD to rank chi' <= chi_max, by RRSVD (Section IV) or by the
     dense SVD (exact mode);
  5. lambda'[b] = s_kept / ||s_kept|| (renormalisation after truncation,
     Eq. defdiscweigt; the state norm is rescaled by 1/sqrt(1 - w)),
     Gamma'[b]^i[a,g] = U[(i,a), g] / lam_l[a],
     Gamma'[b+1]^j[g,c] = Vh[g, (j,c)] / lam_r[c]   (division only where
     lambda > 0, else 0).
Sweeps (Section II.C, Eq. defst3rd): all bonds of one parity are updated in
one sweep; the caller sequences even/odd sweeps.  Each sweep increments the
sweep counter that enters the sketch generator.
"""
import numpy as np

from . import rrsvd as _rr
from .philox import gaussian_omega


class VidalMPS:
    """Gamma tensors and Schmidt values of a chain in Vidal form."""

    def __init__(self, gammas, lambdas):
        self.gamma = [np.asarray(g, dtype=np.complex128) for g in gammas]
        self.lam = [np.asarray(l, dtype=np.float64) for l in lambdas]
        self.N = len(self.gamma)
        assert len(self.lam) == self.N - 1

    def copy(self):
        return VidalMPS([g.copy() for g in self.gamma], [l.copy() for l in self.lam])

    def lam_left(self, site):
        """Schmidt values to the left of a site ([1] at the left end)."""
        return self.lam[site - 1] if site > 0 else np.ones(1)

    def lam_right(self, site):
        """Schmidt values to the right of a site ([1] at the right end)."""
        return self.lam[site] if site < self.N - 1 else np.ones(1)

    def dims(self):
        return [g.shape[0] for g in self.gamma]

    def chis(self):
        return [len(l) for l in self.lam]


def product_state(psis):
    """Vidal form of a product state: Gamma^i = psi_i as 1x1 matrices."""
    gam = []
    for v in psis:
        v = np.asarray(v, dtype=np.complex128)
        gam.append(v.reshape(-1, 1, 1).copy())
    return VidalMPS(gam, [np.ones(1) for _ in range(len(psis) - 1)])


def theta_tensor(gl, lam_l, lam_m, gr, lam_r):
    """Eq. deftheta, as a plain sum over the middle index gamma."""
    return np.einsum("a,iag,g,jgc,c->ijac", lam_l, gl, lam_m, gr, lam_r, optimize=True)


def apply_gate(T, G):
    """Eq. defupdatetheta: G is (dl*dr) x (dl*dr) with <ij|G|i'j'> at
    [i*dr + j, i'*dr + j']."""
    dl, dr = T.shape[0], T.shape[1]
    G4 = np.asarray(G, dtype=np.complex128).reshape(dl, dr, dl, dr)
    return np.einsum("ijkl,klac->ijac", G4, T, optimize=True)


def theta_matrix(Tt):
    """Blocked matrix: row i*chi_l + a, column j*chi_r + c."""
    dl, dr, cl, cr = Tt.shape
    return Tt.transpose(0, 2, 1, 3).reshape(dl * cl, dr * cr)


def bond_theta(mps, b, G):
    """Theta~ of bond b as the (d_l chi_l) x (d_r chi_r) matrix."""
    T = theta_tensor(mps.gamma[b], mps.lam_left(b), mps.lam[b], mps.gamma[b + 1], mps.lam_right(b + 1))
    return theta_matrix(apply_gate(T, G))


def _safe_inv(lam):
    out = np.zeros_like(lam)
    nz = lam > 0.0
    out[nz] = 1.0 / lam[nz]
    return out


def bond_update(mps, b, G, chi_max, p, q, seed, sweep, chain=0, method="rrsvd", cutoff=1e-14):
    """One two-site update of bond b, in place.  Returns a dict with the
    diagnostics compared against the GPU path: the blocked Theta~, its
    truncated singular values s (before renormalisation), the truncated
    Theta~_k = U_k diag(s) Vh_k, and the discarded weight w."""
    dl, dr = mps.gamma[b].shape[0], mps.gamma[b + 1].shape[0]
    lam_l = mps.lam_left(b)
    lam_r = mps.lam_right(b + 1)
    cl, cr = len(lam_l), len(lam_r)
    A = bond_theta(mps, b, G)
    m, n = A.shape
    k, l = _rr.sketch_sizes(m, n, chi_max, p)
    if method == "rrsvd":
        Om = gaussian_omega(n, l, seed, bond=b, sweep=sweep, chain=chain)
        Uk, sk, Vhk, w = _rr.rrsvd_truncate(A, Om, k, q, cutoff)
    elif method == "exact":
        Uk, sk, Vhk, w = _rr.exact_truncate(A, k, cutoff)
    else:
        raise ValueError(method)
    r = len(sk)
    if r == 0:
        raise FloatingPointError("theta is zero: the state has no norm left")
    nrm = np.sqrt(np.sum(sk ** 2))
    mps.lam[b] = sk / nrm
    mps.gamma[b] = (Uk.reshape(dl, cl, r) * _safe_inv(lam_l)[None, :, None]).copy()
    mps.gamma[b + 1] = (Vhk.reshape(r, dr, cr).transpose(1, 0, 2) * _safe_inv(lam_r)[None, None, :]).copy()
    return {"theta": A, "s": sk, "theta_k": (Uk * sk) @ Vhk, "w": w, "k": k, "l": l}


def sweep(mps, parity, gates, chi_max, p, q, seed, sweep_index, chain=0, method="rrsvd", cutoff=1e-14):
    """All bonds b with b % 2 == parity, left to right (they commute).
    gates[b] is the gate of bond b; chi_max is one cap for every bond or a
    sequence of per-bond caps.  Returns the list of discarded weights."""
    ws = []
    for b in range(parity, mps.N - 1, 2):
        cap = chi_max[b] if hasattr(chi_max, "__len__") else chi_max
        info = bond_update(mps, b, gates[b], cap, p, q, seed, sweep_index, chain, method, cutoff)
        ws.append(info["w"])
    return ws


class TEBD:
    """Driver with the call sequence of the C ABI: set_gates per parity, then
    step_even / step_odd; the sweep counter counts step calls."""

    def __init__(self, mps, chi_max, p, q, seed, method="rrsvd", cutoff=1e-14, chain=0):
        self.mps = mps
        self.chi_max, self.p, self.q, self.seed = chi_max, p, q, seed
        self.method, self.cutoff, self.chain = method, cutoff, chain
        self.gates = {0: None, 1: None}
        self.sweeps = 0
        self.w_sum = 0.0
        self.norm_prod = 1.0   # prod (1 - w_b)

    def set_gates(self, parity, gates):
        self.gates[parity] = [None if g is None else np.asarray(g, dtype=np.complex128) for g in gates]

    def _step(self, parity):
        ws = sweep(self.mps, parity, self.gates[parity], self.chi_max, self.p, self.q, self.seed,
                   self.sweeps, self.chain, self.method, self.cutoff)
        self.sweeps += 1
        for w in ws:
            self.w_sum += w
            self.norm_prod *= (1.0 - w)
        return ws

    def step_even(self):
        return self._step(0)

    def step_odd(self):
        return self._step(1)

    def second_order_step(self):
        """One Strang step: half-step even, full odd, half-step even (the
        caller must have set the even gates for dt/2 and the odd for dt)."""
        self.step_even()
        self.step_odd()
        self.step_even()

    def expect(self, site, op):
        return expect_onesite(self.mps, site, op)


def expect_onesite(mps, site, op):
    """<O_k> = sum lam_l[a]^2 lam_r[c]^2 conj(Gam^i[a,c]) O[i,i'] Gam^{i'}[a,c]
    (valid in Vidal canonical form)."""
    g = mps.gamma[site]
    ll = mps.lam_left(site) ** 2
    lr = mps.lam_right(site) ** 2
    og = np.einsum("ij,jac->iac", np.asarray(op, dtype=np.complex128), g)
    return complex(np.einsum("a,c,iac,iac->", ll, lr, g.conj(), og))


def to_statevector(mps):
    """Full contraction of Eq. relcoefmat into the d^N coefficient vector
    (site 0 most significant).  Small N only."""
    cur = mps.gamma[0][:, 0, :]                 # (d0, chi0)
    for k in range(1, mps.N):
        cur = cur * mps.lam[k - 1][None, :]
        g = mps.gamma[k]                         # (d, cl, cr)
        cur = np.einsum("pa,iac->pic", cur, g).reshape(-1, g.shape[2])
    return cur[:, 0]


def norm_by_transfer(mps):
    """<psi|psi> by left-to-right transfer matrices of A^i = Gamma^i lambda."""
    E = np.ones((1, 1), dtype=np.complex128)
    for k in range(mps.N):
        A = mps.gamma[k] * mps.lam_right(k)[None, None, :]
        E = np.einsum("ab,iac,ibd->cd", E, A.conj(), A)
    return float(E[0, 0].real)
