"""Reverse-mode derivative of the TEBD bond update (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Convention: for a real loss L and a complex quantity z, the cotangent is
z_bar = dL/dRe z + i dL/dIm z, so that dL = Re sum conj(z_bar) dz.

Forward of one bond (Section II.B, Eq. deftheta / defupdatetheta, the
truncation of Section IV and the Vidal extraction):
  Theta(i,j,a,c) = x_a A^i[a,g] y_g B^j[g,c] z_c          (x, y, z the lambdas)
  Theta~ = G Theta (physical indices), M = blocked Theta~, M ~ U S V^H (rank k)
  y' = S / ||S||,  A'^i[a,g] = U[(i,a), g] / x_a,  B'^j[g,c] = conj(V[(j,c), g]) / z_c
The derivative of the truncated factorisation is that of the truncated SVD
the RRSVD approximates (Omega held fixed): with F_ij = (s_j^2 - s_i^2) /
((s_j^2 - s_i^2)^2 + eps_F) (broadened 1/(s_j^2 - s_i^2)), S^-1 broadened as
s / (s^2 + eps_S) (both 1e-24 by default: a broadening of 1e-12 biased
gradients of an Ising chain by 1e-5 relative, 1e-16 and below leave
2e-9), Gu = U^H U_bar, Gv = V^H V_bar:
  M_bar = U [ (F o (Gu - Gu^H)) S + diag(S_bar) + S (F o (Gv - Gv^H))
              + 1/2 S^-1 (I o (Gu - Gu^H)) ] V^H
          + (I - U U^H) U_bar S^-1 V^H + U S^-1 V_bar^H (I - V V^H)
(Townsend 2016 for the real case; Wan & Zhang 2019 for the complex gauge
term), then the linear adjoints of the gate and of the contraction.
"""
import numpy as np

from . import rrsvd as _rr
from . import tebd as _t
from .philox import gaussian_omega


def _binv(s, eps_s):
    return s / (s * s + eps_s)


def svd_vjp(U, S, V, Ubar, Sbar, Vbar, eps_f=1e-24, eps_s=1e-24):
    """Cotangent of M from those of its truncated SVD M ~ U diag(S) V^H."""
    s2 = S ** 2
    dsq = s2[None, :] - s2[:, None]            # s_j^2 - s_i^2 at (i, j)
    den = dsq ** 2 + eps_f
    np.fill_diagonal(den, 1.0)
    F = dsq / den
    np.fill_diagonal(F, 0.0)
    Gu = U.conj().T @ Ubar
    Gv = V.conj().T @ Vbar
    Sinv = _binv(S, eps_s)
    Ju = F * (Gu - Gu.conj().T)
    Jv = F * (Gv - Gv.conj().T)
    C = Ju * S[None, :] + np.diag(Sbar) + S[:, None] * Jv
    C += 0.5 * np.diag(Sinv * np.diag(Gu - Gu.conj().T))
    Pu = (Ubar - U @ Gu) * Sinv[None, :]       # (I - U U^H) U_bar S^-1
    Pv = (Vbar - V @ Gv) * Sinv[None, :]       # (I - V V^H) V_bar S^-1
    return (U @ C + Pu) @ V.conj().T + U @ Pv.conj().T


def bond_forward(A, B, x, y, z, G, chi_max, p, q, seed, sweep, bond, chain=0, cutoff=1e-14):
    """One bond update with its cache for the reverse pass."""
    dl, dr = A.shape[0], B.shape[0]
    cl, cr = len(x), len(z)
    T = _t.theta_tensor(A, x, y, B, z)
    Tt = _t.apply_gate(T, G)
    M = _t.theta_matrix(Tt)
    m, n = M.shape
    k, l = _rr.sketch_sizes(m, n, chi_max, p)
    Uf, sf, Vhf = _rr.rrsvd(M, gaussian_omega(n, l, seed, bond=bond, sweep=sweep, chain=chain), q)
    r = _rr.kept_rank(sf, k, cutoff)
    U, S, V = Uf[:, :r], sf[:r], Vhf[:r].conj().T
    nrm = np.sqrt(np.sum(S ** 2))
    inv_x = np.where(x > 0, 1.0 / np.where(x > 0, x, 1.0), 0.0)
    inv_z = np.where(z > 0, 1.0 / np.where(z > 0, z, 1.0), 0.0)
    A2 = U.reshape(dl, cl, r) * inv_x[None, :, None]
    B2 = V.conj().T.reshape(r, dr, cr).transpose(1, 0, 2) * inv_z[None, None, :]
    cache = dict(A=A, B=B, x=x, y=y, z=z, G=G, T=T, U=U, S=S, V=V, nrm=nrm, inv_x=inv_x, inv_z=inv_z,
                 dl=dl, dr=dr, cl=cl, cr=cr)
    return A2, B2, S / nrm, cache


def bond_vjp(c, A2bar, B2bar, y2bar, eps_f=1e-24, eps_s=1e-24):
    """Cotangents (A_bar, B_bar, x_bar, y_bar, z_bar, G_bar) of one bond
    update from those of its outputs (A', B', y')."""
    dl, dr, cl, cr = c["dl"], c["dr"], c["cl"], c["cr"]
    U, S, V, x, z = c["U"], c["S"], c["V"], c["x"], c["z"]
    r = len(S)
    A2 = U.reshape(dl, cl, r) * c["inv_x"][None, :, None]
    B2 = V.conj().T.reshape(r, dr, cr).transpose(1, 0, 2) * c["inv_z"][None, None, :]
    # Vidal extraction
    Ubar = (A2bar * c["inv_x"][None, :, None]).reshape(dl * cl, r)
    xbar = -np.real(np.einsum("iag,iag->a", A2bar.conj(), A2)) * c["inv_x"]
    Vbar = (B2bar * c["inv_z"][None, None, :]).transpose(1, 0, 2).reshape(r, dr * cr).T.conj()
    zbar = -np.real(np.einsum("jgc,jgc->c", B2bar.conj(), B2)) * c["inv_z"]
    # renormalisation y' = S / ||S||
    nrm = c["nrm"]
    Sbar = y2bar / nrm - np.dot(y2bar, S) * S / nrm ** 3
    Mbar = svd_vjp(U, S, V, Ubar, Sbar, Vbar, eps_f, eps_s)
    Ttbar = Mbar.reshape(dl, cl, dr, cr).transpose(0, 2, 1, 3)      # (i, j, a, c)
    G4 = c["G"].reshape(dl, dr, dl, dr)
    Tbar = np.einsum("ijkl,ijac->klac", G4.conj(), Ttbar)
    Gbar = np.einsum("ijac,klac->ijkl", Ttbar, c["T"].conj()).reshape(dl * dr, dl * dr)
    # contraction Theta = x A y B z
    A, B, y = c["A"], c["B"], c["y"]
    P = A * x[None, :, None] * y[None, None, :]           # (i, a, g)
    R = B * z[None, None, :]                              # (j, g, c)
    Pbar = np.einsum("ijac,jgc->iag", Tbar, R.conj())
    Rbar = np.einsum("iag,ijac->jgc", P.conj(), Tbar)
    Abar = Pbar * x[None, :, None] * y[None, None, :]
    xbar = xbar + np.real(np.einsum("iag,iag,g->a", Pbar.conj(), A, y))
    ybar = np.real(np.einsum("iag,iag,a->g", Pbar.conj(), A, x))
    Bbar = Rbar * z[None, None, :]
    zbar = zbar + np.real(np.einsum("jgc,jgc->c", Rbar.conj(), B))
    return Abar, Bbar, xbar, ybar, zbar, Gbar


def expect_vjp(mps, site, op):
    """Cotangents of L = Re <O_site> (local Vidal formula) with respect to
    Gamma[site] and the two lambdas around it."""
    g = mps.gamma[site]
    ll = mps.lam_left(site)
    lr = mps.lam_right(site)
    opg = np.einsum("ij,jac->iac", op, g)
    w = (ll ** 2)[:, None] * (lr ** 2)[None, :]
    # L = Re sum w conj(g) O g; O Hermitian -> dL/dconj(g) = w O g, cotangent 2 w O g
    gbar = 2.0 * w[None, :, :] * opg
    dens = np.real(np.einsum("iac,iac->ac", g.conj(), opg))
    llbar = 2.0 * ll * np.sum(dens * (lr ** 2)[None, :], axis=1)
    lrbar = 2.0 * lr * np.sum(dens * (ll ** 2)[:, None], axis=0)
    return gbar, llbar, lrbar


def tebd_gradient(mps0, schedule, gates, chi_max, p, q, seed, site, op, chain=0, eps_f=1e-24, eps_s=1e-24):
    """Gradient of L = Re <O_site> after the sweeps in `schedule` (a list of
    parities, 0 = even, 1 = odd; sweep s uses Philox sweep index s) with
    respect to the gate matrices: returns {parity: [G_bar per bond]} summed
    over all applications, plus L.  Checkpoints the state before every
    sweep and recomputes the sweep during the reverse pass."""
    N = mps0.N
    ckpts = []
    mps = mps0.copy()
    for s, par in enumerate(schedule):
        ckpts.append(mps.copy())
        _t.sweep(mps, par, gates[par], chi_max, p, q, seed, s, chain)
    L = float(np.real(_t.expect_onesite(mps, site, op)))
    gbar = [np.zeros_like(g) for g in mps.gamma]
    lbar = [np.zeros_like(l) for l in mps.lam]
    gs, lls, lrs = expect_vjp(mps, site, op)
    gbar[site] = gbar[site] + gs
    if site > 0:
        lbar[site - 1] = lbar[site - 1] + lls
    if site < N - 1:
        lbar[site] = lbar[site] + lrs
    dG = {0: [None] * (N - 1), 1: [None] * (N - 1)}
    for b in range(N - 1):
        for par in (0, 1):
            if gates[par] is not None and b % 2 == par:
                dG[par][b] = np.zeros_like(gates[par][b])
    for s in reversed(range(len(schedule))):
        par = schedule[s]
        pre = ckpts[s]
        new_lbar = [l.copy() for l in lbar]
        for b in range(par, N - 1, 2):
            x = pre.lam_left(b)
            z = pre.lam_right(b + 1)
            _, _, _, cache = bond_forward(pre.gamma[b], pre.gamma[b + 1], x, pre.lam[b], z, gates[par][b],
                                          chi_max, p, q, seed, s, b, chain)
            Ab, Bb, xb, yb, zb, Gb = bond_vjp(cache, gbar[b], gbar[b + 1], lbar[b], eps_f, eps_s)
            gbar[b], gbar[b + 1] = Ab, Bb
            new_lbar[b] = yb
            if b > 0:
                new_lbar[b - 1] = new_lbar[b - 1] + xb
            if b + 1 < N - 1:
                new_lbar[b + 1] = new_lbar[b + 1] + zb
            dG[par][b] = dG[par][b] + Gb
        lbar = new_lbar
    return dG, L
