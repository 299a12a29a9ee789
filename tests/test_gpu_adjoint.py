"""The differentiable form: gate cotangents from tebd_backward against the
oracle's reverse pass, and dL/dJ through the torch.autograd.Function against
central finite differences (h = 1e-6) of the GPU forward and of the oracle."""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _gpu_L(J, N, hf, dt, steps, chi, p, q, seed, site):
    from paper_1504_00992_gb300 import binding as B
    hs = I.tfim_bond_terms(J, hf)
    sim = B.Tebd(N, 2, chi, p, q, seed)
    sim.set_product_state([np.array([1.0, 0.0]) for _ in range(N)])
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    _, _, sz = I.pauli()
    v = sim.expect(site, sz).real
    sim.close()
    return v


def _oracle_L(J, N, hf, dt, steps, chi, p, q, seed, site):
    hs = I.tfim_bond_terms(J, hf)
    sim = T.TEBD(T.product_state([np.array([1.0, 0.0]) for _ in range(N)]), chi, p, q, seed)
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.second_order_step()
    _, _, sz = I.pauli()
    return float(np.real(sim.expect(site, sz)))


CFG = dict(N=8, hf=1.0, dt=0.05, steps=8, chi=8, p=4, q=2, seed=3, site=3)


def test_gate_cotangents_match_the_oracle_reverse_pass(lib):
    from paper_1504_00992_gb300 import binding as B
    c = CFG
    rng = np.random.default_rng(0)
    J = rng.uniform(0.5, 1.5, c["N"] - 1)
    hs = I.tfim_bond_terms(J, c["hf"])
    ge, go = I.trotter_gates(hs, c["dt"] / 2), I.trotter_gates(hs, c["dt"])
    sim = B.Tebd(c["N"], 2, c["chi"], c["p"], c["q"], c["seed"])
    sim.set_product_state([np.array([1.0, 0.0]) for _ in range(c["N"])])
    sim.set_gates(0, ge)
    sim.set_gates(1, go)
    sim.record(True)
    for _ in range(c["steps"]):
        sim.step_even(); sim.step_odd(); sim.step_even()
    _, _, sz = I.pauli()
    L_gpu = sim.expect(c["site"], sz).real
    dge, dgo = sim.backward(c["site"], sz)
    assert sim.expect(c["site"], sz).real == L_gpu          # forward state restored
    assert sim.sweeps() == 3 * c["steps"]
    sim.close()
    mps0 = T.product_state([np.array([1.0, 0.0]) for _ in range(c["N"])])
    dG, L = AD.tebd_gradient(mps0, [0, 1, 0] * c["steps"], {0: ge, 1: go}, c["chi"], c["p"], c["q"], c["seed"],
                             c["site"], sz)
    assert abs(L - L_gpu) <= 1e-10
    scale = max(np.abs(g).max() for par in (0, 1) for g in dG[par] if g is not None)
    for b in range(c["N"] - 1):
        ref = dG[b % 2][b]
        got = (dge if b % 2 == 0 else dgo)[b]
        assert np.abs(got - ref).max() <= 1e-8 * scale, b
        other = (dgo if b % 2 == 0 else dge)[b]
        assert np.all(other == 0)


def test_coupling_gradient_matches_finite_differences(lib):
    import torch
    from paper_1504_00992_gb300.autograd import tfim_observable
    c = CFG
    rng = np.random.default_rng(1)
    J0 = rng.uniform(0.5, 1.5, c["N"] - 1)
    J = torch.tensor(J0, requires_grad=True)
    L = tfim_observable(J, c["N"], c["hf"], c["dt"], c["steps"], c["chi"], c["p"], c["q"], c["seed"], c["site"])
    L.backward()
    g = J.grad.numpy()
    eps = 1e-6
    args = (c["N"], c["hf"], c["dt"], c["steps"], c["chi"], c["p"], c["q"], c["seed"], c["site"])
    fd_gpu = np.zeros_like(J0)
    fd_orc = np.zeros_like(J0)
    for b in range(len(J0)):
        Jp, Jm = J0.copy(), J0.copy()
        Jp[b] += eps
        Jm[b] -= eps
        fd_gpu[b] = (_gpu_L(Jp, *args) - _gpu_L(Jm, *args)) / (2 * eps)
        fd_orc[b] = (_oracle_L(Jp, *args) - _oracle_L(Jm, *args)) / (2 * eps)
    sc = max(1.0, np.abs(fd_orc).max())
    assert np.abs(g - fd_gpu).max() <= 1e-6 * sc
    assert np.abs(g - fd_orc).max() <= 1e-6 * sc


def test_ising_n40_gradient_full_size(lib):
    """The differentiable workload at full size: transverse-field Ising chain
    N=40, chi=64, dt=0.02, 50 steps, d<sigma^z_19>/dJ_b with J ~ U[0.5, 1.5]
    (seed 0), against the oracle's central differences (h = 1e-6) stored for
    every coupling, and against central differences of the GPU forward on
    couplings near and far from the site."""
    import torch
    from paper_1504_00992_gb300.autograd import tfim_observable
    from tests.test_oracle_c4_golden import load_c4_golden
    N, hf, dt, steps, chi, p, q, seed, site = 40, 1.0, 0.02, 50, 64, 10, 2, 0, 19
    J0 = np.random.default_rng(0).uniform(0.5, 1.5, N - 1)
    J = torch.tensor(J0, requires_grad=True)
    L = tfim_observable(J, N, hf, dt, steps, chi, p, q, seed, site)
    L.backward()
    g = J.grad.numpy()
    L_orc, fd_orc = load_c4_golden()
    assert abs(L.item() - L_orc) <= 1e-10
    assert np.abs(g - fd_orc).max() <= 1e-7
    for b in (0, 17, 18, 19, 20, 38):
        Jp, Jm = J0.copy(), J0.copy()
        Jp[b] += 1e-6
        Jm[b] -= 1e-6
        fd = (_gpu_L(Jp, N, hf, dt, steps, chi, p, q, seed, site)
              - _gpu_L(Jm, N, hf, dt, steps, chi, p, q, seed, site)) / 2e-6
        assert abs(g[b] - fd) <= 1e-7, b
