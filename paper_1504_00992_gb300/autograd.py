"""torch.autograd.Function over the library's forward and reverse passes.

`TfimObservable.apply(J, ...)` evolves the transverse-field Ising chain
H = -sum_b J_b Z_b Z_{b+1} - h sum_i X_i from |0...0> with second-order
Trotter sweeps through the C ABI (recording checkpoints) and returns
<sigma^z_site>; its backward calls tebd_backward for the gate cotangents and
chains them to the couplings with the Frechet derivative of each gate
exponential (the caller-side step of the chain rule):
  dL/dJ_b = sum_parity Re sum conj(G_bar_b) dG_b/dJ_b.
"""
import numpy as np
import torch

from . import binding as B
from . import inputs as I


class TfimObservable(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, N, h, dt, steps, chi, p, q, seed, site):
        Jn = J.detach().cpu().double().numpy()
        hs = I.tfim_bond_terms(Jn, h)
        sim = B.Tebd(N, 2, chi, p, q, seed)
        sim.set_product_state([np.array([1.0, 0.0]) for _ in range(N)])
        sim.set_gates(0, I.trotter_gates(hs, dt / 2))
        sim.set_gates(1, I.trotter_gates(hs, dt))
        sim.record(True)
        for _ in range(steps):
            sim.step_even()
            sim.step_odd()
            sim.step_even()
        _, _, sz = I.pauli()
        val = sim.expect(site, sz).real
        ctx.sim, ctx.hs, ctx.dt, ctx.site = sim, hs, dt, site
        return torch.tensor(val, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        _, _, sz = I.pauli()
        ge, go = ctx.sim.backward(ctx.site, sz)
        dh = I.tfim_bond_terms_dJ(len(ctx.hs) + 1)
        grad = np.zeros(len(ctx.hs))
        for b in range(len(ctx.hs)):
            gbar, tau = (ge[b], ctx.dt / 2) if b % 2 == 0 else (go[b], ctx.dt)
            grad[b] = np.real(np.vdot(gbar, I.gate_derivative(ctx.hs[b], tau, dh[b])))
        ctx.sim.close()
        return (gL * torch.from_numpy(grad),) + (None,) * 9


def tfim_observable(J, N, h=1.0, dt=0.02, steps=50, chi=64, p=10, q=2, seed=0, site=19):
    return TfimObservable.apply(J, N, h, dt, steps, chi, p, q, seed, site)
