"""Dense state-vector evolution with two-site gates (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Applies <ij|G|i'j'> to sites (b, b+1) of a d^N coefficient vector exactly
(Eq. deftsgate without any decomposition): this is what TEBD computes when no
Schmidt value is discarded.
"""
import numpy as np


def apply_two_site(psi, N, d, b, G):
    t = psi.reshape((d,) * N)
    G4 = np.asarray(G).reshape(d, d, d, d)
    t = np.tensordot(G4, t, axes=([2, 3], [b, b + 1]))   # new axes 0,1 = sites b, b+1
    t = np.moveaxis(t, [0, 1], [b, b + 1])
    return t.reshape(-1)


def product(psis):
    out = np.ones(1, dtype=np.complex128)
    for v in psis:
        out = np.kron(out, np.asarray(v, dtype=np.complex128))
    return out


def expect_onesite(psi, N, d, site, op):
    t = psi.reshape((d,) * N)
    ot = np.tensordot(np.asarray(op), t, axes=([1], [site]))
    ot = np.moveaxis(ot, 0, site)
    return complex(np.vdot(t.reshape(-1), ot.reshape(-1)))


def sweep(psi, N, d, parity, gates):
    for b in range(parity, N - 1, 2):
        psi = apply_two_site(psi, N, d, b, gates[b])
    return psi


def apply_two_site_dims(psi, dims, b, G):
    """apply_two_site for per-site local dimensions dims."""
    N = len(dims)
    t = psi.reshape(tuple(dims))
    G4 = np.asarray(G).reshape(dims[b], dims[b + 1], dims[b], dims[b + 1])
    t = np.tensordot(G4, t, axes=([2, 3], [b, b + 1]))
    t = np.moveaxis(t, [0, 1], [b, b + 1])
    return t.reshape(-1)


def expect_onesite_dims(psi, dims, site, op):
    t = psi.reshape(tuple(dims))
    ot = np.tensordot(np.asarray(op), t, axes=([1], [site]))
    ot = np.moveaxis(ot, 0, site)
    return complex(np.vdot(t.reshape(-1), ot.reshape(-1)))


def sweep_dims(psi, dims, parity, gates):
    for b in range(parity, len(dims) - 1, 2):
        psi = apply_two_site_dims(psi, dims, b, gates[b])
    return psi
