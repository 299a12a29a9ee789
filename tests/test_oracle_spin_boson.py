"""Spin-boson chain inputs (star-to-chain form, per-site local dimensions,
per-bond caps) and the oracle's TEBD on them, pinned against dense
constructions: the bond terms sum to the chain Hamiltonian written out
directly, the canonical random-MPS fixture is the Vidal form of its random
state, and untruncated TEBD equals gate-by-gate state-vector evolution."""
import numpy as np
import pytest

from oracle import statevector as SV
from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I


def _embed(op, dims, sites):
    """op acting on consecutive sites, identity elsewhere."""
    left = int(np.prod(dims[: sites[0]])) if sites[0] > 0 else 1
    right = int(np.prod(dims[sites[-1] + 1:])) if sites[-1] + 1 < len(dims) else 1
    return np.kron(np.kron(np.eye(left), op), np.eye(right))


def test_bond_terms_sum_to_the_chain_hamiltonian():
    dims = [2, 4, 3, 3]
    omega, t0, ds = 1.3, 0.5, 0.8
    hs = I.spin_boson_bond_terms(dims, omega=omega, t0=t0, delta_s=ds)
    H = sum(_embed(h, dims, [b, b + 1]) for b, h in enumerate(hs))
    sx, _, sz = I.pauli()
    a1, ad1, n1 = I.boson_ops(4)
    a2, ad2, n2 = I.boson_ops(3)
    a3, ad3, n3 = I.boson_ops(3)
    Hd = 0.5 * ds * _embed(sx, dims, [0]) + t0 * _embed(np.kron(sz, a1 + ad1), dims, [0, 1])
    Hd = Hd + omega * (_embed(n1, dims, [1]) + _embed(n2, dims, [2]) + _embed(n3, dims, [3]))
    Hd = Hd + (t0 / 2) * _embed(np.kron(ad1, a2) + np.kron(a1, ad2), dims, [1, 2])
    Hd = Hd + (t0 / 3) * _embed(np.kron(ad2, a3) + np.kron(a2, ad3), dims, [2, 3])
    assert np.abs(H - Hd).max() < 1e-14
    assert np.abs(H - H.conj().T).max() == 0.0


def test_sizes_fall_linearly():
    ds, chis = I.spin_boson_sizes(100, 32, 4, 256, 64)
    assert ds[0] == 2 and ds[1] == 32 and ds[-1] == 4 and len(ds) == 101
    assert chis[0] == 256 and chis[-1] == 64 and len(chis) == 100
    assert all(a >= b for a, b in zip(ds[1:], ds[2:]))


def test_random_canonical_mps_is_the_vidal_form_of_its_random_state():
    dims = [2, 4, 4, 3, 3]
    caps = [6, 8, 7, 3]
    g, lam, raw = I.random_canonical_mps(dims, caps, 11, return_raw=True)
    N = len(dims)
    for s in range(N):
        ll = lam[s - 1] if s > 0 else np.ones(1)
        lr = lam[s] if s < N - 1 else np.ones(1)
        left = np.einsum("a,iab,iac->bc", ll ** 2, g[s].conj(), g[s])
        right = np.einsum("iab,b,icb->ac", g[s], lr ** 2, g[s].conj())
        assert np.abs(left - np.eye(len(lr))).max() < 1e-12
        assert np.abs(right - np.eye(len(ll))).max() < 1e-12
    for b in range(N - 1):
        assert abs(np.sum(lam[b] ** 2) - 1.0) < 1e-12
        assert np.all(np.diff(lam[b]) <= 0)
    v = T.to_statevector(T.VidalMPS(g, lam))
    w = raw[0][:, 0, :]
    for s in range(1, N):
        w = np.einsum("pa,iac->pic", w, raw[s]).reshape(-1, raw[s].shape[2])
    w = w[:, 0] / np.linalg.norm(w[:, 0])
    assert abs(abs(np.vdot(v, w)) - 1.0) < 1e-12
    # each bond's Schmidt values are those of the state vector's bipartition
    for b in range(N - 1):
        M = v.reshape(int(np.prod(dims[: b + 1])), -1)
        s = np.linalg.svd(M, compute_uv=False)[: len(lam[b])]
        assert np.abs(s - lam[b]).max() < 1e-12


@pytest.mark.parametrize("method", ["rrsvd", "exact"])
def test_untruncated_spin_boson_tebd_equals_state_vector(method):
    dims, _ = I.spin_boson_sizes(3, 4, 3, 8, 8)
    big = [64] * (len(dims) - 1)
    g, lam = I.random_canonical_mps(dims, [3, 4, 3], 5)
    hs = I.spin_boson_bond_terms(dims)
    ge, go = I.trotter_gates(hs, 0.05), I.trotter_gates(hs, 0.1)
    sim = T.TEBD(T.VidalMPS(g, lam), big, 6, 2, 3, method=method)
    sim.set_gates(0, ge)
    sim.set_gates(1, go)
    psi = T.to_statevector(T.VidalMPS(g, lam))
    for _ in range(4):
        sim.second_order_step()
        psi = SV.sweep_dims(psi, dims, 0, ge)
        psi = SV.sweep_dims(psi, dims, 1, go)
        psi = SV.sweep_dims(psi, dims, 0, ge)
    v = T.to_statevector(sim.mps)
    assert abs(abs(np.vdot(v, psi)) - 1.0) < 1e-11
    _, _, sz = I.pauli()
    assert abs(sim.expect(0, sz) - SV.expect_onesite_dims(psi, dims, 0, sz)) < 1e-11
    for s in range(1, len(dims)):
        n = I.boson_ops(dims[s])[2]
        assert abs(sim.expect(s, n) - SV.expect_onesite_dims(psi, dims, s, n)) < 1e-11


def test_per_bond_caps_bound_each_bond():
    dims, caps = I.spin_boson_sizes(5, 6, 4, 10, 4)
    g, lam = I.random_canonical_mps(dims, caps, 2)
    hs = I.spin_boson_bond_terms(dims)
    sim = T.TEBD(T.VidalMPS(g, lam), caps, 4, 1, 7)
    sim.set_gates(0, I.trotter_gates(hs, 0.05))
    sim.set_gates(1, I.trotter_gates(hs, 0.1))
    sim.second_order_step()
    for b, l in enumerate(sim.mps.lam):
        assert len(l) <= caps[b]
        assert abs(np.sum(l ** 2) - 1.0) < 1e-12
