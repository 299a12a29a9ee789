"""Pins of the oracle's reverse-mode bond update against central finite
differences of the forward oracle (the truncated-SVD adjoint with Omega held
fixed, the gate and contraction adjoints), and of the gate Frechet
derivative against finite differences of the matrix exponential."""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _out_loss(A2, B2, y2, wA, wy, xw, zw):
    """Gauge-invariant function of the outputs alone: sum_g xw_a A'[a,g] y'_g
    B'[g,c] zw_c (blocked) paired with wA, plus sum wy y'^2; xw, zw are fixed
    weights (constants of the loss, not the bond's inputs) that keep it well
    scaled when some lambda is tiny."""
    th = T.theta_matrix(T.theta_tensor(A2, xw, np.real(y2).astype(complex), B2, zw))
    return float(np.real(np.vdot(wA, th)) + np.dot(wy[:len(y2)], np.real(y2) ** 2))


def _loss_bond(A, B, x, y, z, G, wA, wy, xw, zw, chi, p, q):
    A2, B2, y2, _ = AD.bond_forward(A, B, x, y, z, G, chi, p, q, 5, 2, 1)
    return _out_loss(A2, B2, y2, wA, wy, xw, zw)


@pytest.mark.parametrize("decay,chi", [
    (4.0, 6),     # nothing discarded: the SVD adjoint is exact
    (30.0, 2),    # truncated across a gap sigma_3 / sigma_2 ~ 5e-10: the neglected
                  # coupling to the discarded vectors is of that order
])
def test_bond_vjp_matches_finite_differences(decay, chi):
    rng = np.random.default_rng(0 if decay > 10 else 1)
    dl = dr = 2
    cl, cm, cr = 3, 4, 3
    bd = I.random_bond(dl, dr, cl, cm, cr, rng, decay=decay)
    A, B, x, y, z, G = bd["gamma_l"], bd["gamma_r"], bd["lam_l"], bd["lam_m"], bd["lam_r"], bd["gate"]
    p, q = 2, 2
    wA = _rand_c(rng, dl * cl, dr * cr)
    wy = rng.standard_normal(8)
    A2, B2, y2, cache = AD.bond_forward(A, B, x, y, z, G, chi, p, q, 5, 2, 1)
    h = 1e-5

    def num_bar(arr, f, rel=False):
        """Central differences; rel=True steps each entry by h |entry| (the
        lambdas have entries near 1e-9, where an absolute step would cross
        zero)."""
        bar = np.zeros(arr.shape, dtype=complex)
        for idx in np.ndindex(arr.shape):
            step = h * abs(arr[idx]) if rel else h
            for unit, fac in ((1.0, 1.0), (1j, 1j)):
                if fac == 1j and not np.iscomplexobj(arr):
                    continue
                ap, am = arr.astype(complex).copy(), arr.astype(complex).copy()
                ap[idx] += unit * step
                am[idx] -= unit * step
                bar[idx] += (f(ap) - f(am)) / (2 * step) * fac
        return bar

    xw, zw = x.copy(), z.copy()
    L_of = lambda A2_, B2_, y2_: _out_loss(A2_, B2_, y2_, wA, wy, xw, zw)
    A2bar = num_bar(A2, lambda a: L_of(a, B2, y2))
    B2bar = num_bar(B2, lambda b: L_of(A2, b, y2))
    y2bar = np.real(num_bar(y2, lambda yy: L_of(A2, B2, yy), rel=True))
    with np.errstate(invalid="ignore"):
        Abar, Bbar, xbar, ybar, zbar, Gbar = AD.bond_vjp(cache, A2bar, B2bar, y2bar, eps_f=0.0, eps_s=0.0)
    full = lambda A_, B_, x_, y_, z_, G_: _loss_bond(A_, B_, x_, y_, z_, G_, wA, wy, xw, zw, chi, p, q)
    nA = num_bar(A, lambda a: full(a, B, x, y, z, G))
    nB = num_bar(B, lambda b: full(A, b, x, y, z, G))
    nG = num_bar(G, lambda g: full(A, B, x, y, z, g))
    ny = np.real(num_bar(y, lambda yy: full(A, B, x, np.real(yy), z, G), rel=True))
    nx = np.real(num_bar(x, lambda xx: full(A, B, np.real(xx), y, z, G), rel=True))
    nz = np.real(num_bar(z, lambda zz: full(A, B, x, y, np.real(zz), G), rel=True))
    for got, ref in ((Abar, nA), (Bbar, nB), (Gbar, nG)):
        assert np.abs(got - ref).max() <= 1e-7 * max(1.0, np.abs(ref).max())
    # lambda entries below 1e-6 (down to 1e-10 here) are not resolvable by
    # central differences in FP64 (a relative step of 1e-15 drowns in rounding)
    for got, ref, lam in ((ybar, ny, y), (xbar, nx, x), (zbar, nz, z)):
        ok = lam >= 1e-6
        assert np.abs(got[ok] - ref[ok]).max() <= 1e-6 * max(1.0, np.abs(ref[ok]).max())


def test_gate_derivative_matches_finite_differences():
    rng = np.random.default_rng(2)
    hs = I.tfim_bond_terms([0.7, 1.3, 0.9], 1.0)
    dh = I.tfim_bond_terms_dJ(4)[1]
    tau, eps = 0.05, 1e-6
    h = hs[1]
    ref = (I.unitary_from_hermitian(h + eps * dh, tau) - I.unitary_from_hermitian(h - eps * dh, tau)) / (2 * eps)
    assert np.abs(I.gate_derivative(h, tau, dh) - ref).max() < 1e-9
    # a degenerate spectrum (equal eigenvalues) takes the limit branch
    h0 = np.kron(np.diag([1.0, 1.0]), np.eye(2)).astype(complex)
    ref0 = (I.unitary_from_hermitian(h0 + eps * dh, tau) - I.unitary_from_hermitian(h0 - eps * dh, tau)) / (2 * eps)
    assert np.abs(I.gate_derivative(h0, tau, dh) - ref0).max() < 1e-9


def _tfim_observable(J, N, h, dt, steps, chi, p, q, seed, site):
    hs = I.tfim_bond_terms(J, h)
    sim = T.TEBD(T.product_state([np.array([1.0, 0.0]) for _ in range(N)]), chi, p, q, seed)
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.second_order_step()
    _, _, sz = I.pauli()
    return float(np.real(sim.expect(site, sz)))


def test_tebd_gradient_matches_finite_differences_of_the_oracle():
    """dL/dJ_b of L = <sigma^z_site>(T) for the transverse-field Ising chain,
    through the reverse pass, against central differences (h = 1e-6) of the
    forward oracle."""
    N, hfield, dt, steps, chi, p, q, seed, site = 6, 1.0, 0.05, 6, 8, 4, 2, 3, 2
    rng = np.random.default_rng(4)
    J = rng.uniform(0.5, 1.5, N - 1)
    hs = I.tfim_bond_terms(J, hfield)
    ge, go = I.trotter_gates(hs, dt / 2), I.trotter_gates(hs, dt)
    schedule = [0, 1, 0] * steps
    _, _, sz = I.pauli()
    mps0 = T.product_state([np.array([1.0, 0.0]) for _ in range(N)])
    dG, L = AD.tebd_gradient(mps0, schedule, {0: ge, 1: go}, chi, p, q, seed, site, sz)
    assert abs(L - _tfim_observable(J, N, hfield, dt, steps, chi, p, q, seed, site)) < 1e-13
    dh = I.tfim_bond_terms_dJ(N)
    grad = np.zeros(N - 1)
    for b in range(N - 1):
        par = b % 2
        tau = dt / 2 if par == 0 else dt
        grad[b] = np.real(np.vdot(dG[par][b], I.gate_derivative(hs[b], tau, dh[b])))
    fd = np.zeros(N - 1)
    eps = 1e-6
    for b in range(N - 1):
        Jp, Jm = J.copy(), J.copy()
        Jp[b] += eps
        Jm[b] -= eps
        fd[b] = (_tfim_observable(Jp, N, hfield, dt, steps, chi, p, q, seed, site)
                 - _tfim_observable(Jm, N, hfield, dt, steps, chi, p, q, seed, site)) / (2 * eps)
    assert np.abs(grad - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())
