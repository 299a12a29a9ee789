"""Pins of the oracle's TEBD bond update (Section II) against exact results:
brute-force loops for theta (Eq. deftheta / defupdatetheta), the dense state
vector when nothing is truncated, the free-fermion closed form of the XX chain
with the Trotter order of Eq. defst3rd, and the norm rules of Eq.
defdiscweigt."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import statevector as SV
from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I


def test_theta_brute_force():
    rng = np.random.default_rng(0)
    dl, dr, cl, cm, cr = 2, 3, 3, 4, 2
    bd = I.random_bond(dl, dr, cl, cm, cr, rng)
    Tt = T.theta_tensor(bd["gamma_l"], bd["lam_l"], bd["lam_m"], bd["gamma_r"], bd["lam_r"])
    G = bd["gate"]
    ref = np.zeros((dl, dr, cl, cr), dtype=complex)
    for i in range(dl):
        for j in range(dr):
            for a in range(cl):
                for c in range(cr):
                    acc = 0j
                    for g in range(cm):
                        acc += (bd["lam_l"][a] * bd["gamma_l"][i, a, g] * bd["lam_m"][g]
                                * bd["gamma_r"][j, g, c] * bd["lam_r"][c])
                    ref[i, j, a, c] = acc
    assert np.abs(Tt - ref).max() < 1e-13
    Tg = T.apply_gate(Tt, G)
    ref2 = np.zeros_like(ref)
    for i in range(dl):
        for j in range(dr):
            for ip in range(dl):
                for jp in range(dr):
                    ref2[i, j] += G[i * dr + j, ip * dr + jp] * ref[ip, jp]
    assert np.abs(Tg - ref2).max() < 1e-13
    M = T.theta_matrix(Tg)
    for i in range(dl):
        for j in range(dr):
            for a in range(cl):
                for c in range(cr):
                    assert M[i * cl + a, j * cr + c] == Tg[i, j, a, c]


def _evolve_both(N, d, gates_e, gates_o, steps, chi_max, method="rrsvd", p=10, q=2, seed=0):
    psi0 = I.neel_state(N, d)
    sim = T.TEBD(T.product_state(psi0), chi_max, p, q, seed, method=method)
    sim.set_gates(0, gates_e)
    sim.set_gates(1, gates_o)
    psi = SV.product(psi0)
    for _ in range(steps):
        sim.second_order_step()
        psi = SV.sweep(psi, N, d, 0, gates_e)
        psi = SV.sweep(psi, N, d, 1, gates_o)
        psi = SV.sweep(psi, N, d, 0, gates_e)
    return sim, psi


@pytest.mark.parametrize("method", ["rrsvd", "exact"])
def test_untruncated_tebd_equals_state_vector(method):
    """With chi_max above every Schmidt rank, TEBD is the exact Trotterised
    state (Eq. deftsgate applied gate by gate)."""
    N, d = 10, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim, psi = _evolve_both(N, d, I.trotter_gates(hs, 0.05), I.trotter_gates(hs, 0.1), 15, 64, method)
    _, _, sz = I.spin_ops(d)
    for k in range(N):
        assert abs(sim.expect(k, sz) - SV.expect_onesite(psi, N, d, k, sz)) < 1e-12
    v = T.to_statevector(sim.mps)
    assert abs(abs(np.vdot(v, psi)) - 1.0) < 1e-12
    assert sim.w_sum < 1e-12      # w = 1 - sum s^2/||theta||^2 carries rounding only


def test_random_gates_spin1():
    """Generic Haar-random gates, d = 3, uneven bond dimensions."""
    N, d = 6, 3
    rng = np.random.default_rng(5)
    ge = [I.random_unitary(d * d, rng) for _ in range(N - 1)]
    go = [I.random_unitary(d * d, rng) for _ in range(N - 1)]
    sim, psi = _evolve_both(N, d, ge, go, 3, 81)
    v = T.to_statevector(sim.mps)
    assert abs(abs(np.vdot(v, psi)) - 1.0) < 1e-11
    sx, _, _ = I.spin_ops(d)
    for k in range(N):
        assert abs(sim.expect(k, sx) - SV.expect_onesite(psi, N, d, k, sx)) < 1e-11


def _xx_free_fermion_sz(N, J, t, occ):
    """XX chain, H = J sum (Sx Sx + Sy Sy) = (J/2) sum (c+_i c_{i+1} + h.c.):
    <Sz_i(t)> = sum_j |[exp(-i h t)]_ij|^2 n_j(0) - 1/2 for a Fock state."""
    h = np.zeros((N, N))
    for i in range(N - 1):
        h[i, i + 1] = h[i + 1, i] = J / 2.0
    Ut = expm(-1j * h * t)
    return (np.abs(Ut) ** 2) @ occ - 0.5


def test_xx_chain_free_fermions_and_trotter_order():
    N, J, Tf = 10, 1.0, 1.0
    occ = np.array([1.0 if k % 2 == 0 else 0.0 for k in range(N)])   # Neel: up = occupied
    exact = _xx_free_fermion_sz(N, J, Tf, occ)
    hs = I.xxz_bond_terms(N, 2, J, 0.0)
    _, _, sz = I.spin_ops(2)
    errs = []
    for dt in (0.1, 0.05):
        steps = int(round(Tf / dt))
        sim, _ = _evolve_both(N, 2, I.trotter_gates(hs, dt / 2), I.trotter_gates(hs, dt), steps, 64)
        got = np.array([sim.expect(k, sz).real for k in range(N)])
        errs.append(np.abs(got - exact).max())
    assert errs[1] < 5e-3
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0     # second-order splitting: global error O(dt^2)


def test_norm_rules_under_truncation():
    """Truncating: every lambda is renormalised (sum lambda^2 = 1) and stays
    sorted, the chain stays normalised up to the truncation, and weights add."""
    N, d = 10, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim, psi = _evolve_both(N, d, I.trotter_gates(hs, 0.1), I.trotter_gates(hs, 0.2), 10, 4)
    for lam in sim.mps.lam:
        assert abs(np.sum(lam ** 2) - 1.0) < 1e-13
        assert np.all(np.diff(lam) <= 0)
    assert abs(T.norm_by_transfer(sim.mps) - 1.0) < 1e-3
    assert sim.w_sum > 1e-8
    assert abs((1 - sim.norm_prod) - sim.w_sum) < sim.w_sum ** 2


@pytest.mark.parametrize("method", ["exact", "rrsvd"])
def test_single_truncation_fidelity_is_one_minus_w(method):
    """Eq. defdiscweigt: from a canonical state, truncating one bond to chi'
    Schmidt values keeps overlap^2 = 1 - w with the untruncated state (exact
    for the dense SVD; RRSVD with q = 2 is within its approximation error)."""
    N, d = 8, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    sim, _ = _evolve_both(N, d, I.trotter_gates(hs, 0.1), I.trotter_gates(hs, 0.2), 6, 64)
    b = 3
    gate = I.trotter_gates(hs, 0.3)[b]
    ref = sim.mps.copy()
    T.bond_update(ref, b, gate, 64, 10, 2, 0, 99, method="exact")
    v_ref = T.to_statevector(ref)
    trunc = sim.mps.copy()
    info = T.bond_update(trunc, b, gate, 3, 2, 2, 0, 99, method=method)
    v = T.to_statevector(trunc)
    fid = abs(np.vdot(v, v_ref)) ** 2 / (np.vdot(v, v).real * np.vdot(v_ref, v_ref).real)
    assert info["w"] > 1e-6
    tol = 1e-12 if method == "exact" else 1e-4 * info["w"]
    assert abs(fid - (1 - info["w"])) < tol
    assert abs(np.vdot(v, v).real - 1.0) < 1e-12   # renormalised


def test_product_state_and_expect():
    psi = [np.array([np.cos(0.3), np.sin(0.3) * np.exp(0.2j)]) for _ in range(4)]
    mps = T.product_state(psi)
    sx, sy, sz = I.spin_ops(2)
    v = SV.product(psi)
    for k in range(4):
        for op in (sx, sy, sz):
            assert abs(T.expect_onesite(mps, k, op) - SV.expect_onesite(v, 4, 2, k, op)) < 1e-15


def test_spin_ops_algebra():
    for d in (2, 3, 4):
        sx, sy, sz = I.spin_ops(d)
        s = (d - 1) / 2
        assert np.allclose(sx @ sy - sy @ sx, 1j * sz)
        assert np.allclose(sx @ sx + sy @ sy + sz @ sz, s * (s + 1) * np.eye(d))
