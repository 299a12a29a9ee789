"""TEBD handles in the mixed-precision form (TEBD_PREC_TF32): every bond
update runs the TF32 sketch, the FP64-accurate re-orthonormalisation and
projection and the FP64 small SVD, on batches of bonds of uneven shape
(each instance at its own (m, n, l) inside arrays laid out at the wave's
capacities).

Stated tolerance of the form against the FP64 oracle.  Its Omega is the
oracle's rounded to TF32 and its refinement pass is 3xTF32 (FP32-level), so
the sketched range is resolved to ~1e-7 sigma_1: directions whose singular
values lie below that level (TEBD spectra reach 1e-14) are captured only to
FP32 accuracy.  On the single-bond stress spectrum this is invisible (the
form's singular values are as close to the exact ones as the FP64 method's),
but over a TEBD run it leaves differences of a few 1e-8 in observables and
Schmidt values: after the 36 sweeps here they stay within 1e-7 (observables)
and 2e-7 (Schmidt values) of the FP64 oracle, and the discarded weights
within 1e-10."""
import numpy as np
import pytest

from oracle import tebd as T
from paper_1504_00992_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _oracle(N, d, chi, delta, steps, dt, p, q, seed, chain=0):
    hs = I.xxz_bond_terms(N, d, 1.0, delta)
    ref = T.TEBD(T.product_state(I.neel_state(N, d)), chi, p, q, seed, chain=chain)
    ref.set_gates(0, I.trotter_gates(hs, dt / 2))
    ref.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        ref.second_order_step()
    _, _, sz = I.spin_ops(d)
    return np.array([ref.expect(k, sz).real for k in range(N)]), ref.mps.lam, ref.w_sum


# (observables, Schmidt values) bars of each form after the 36 sweeps
BARS = {"tf32": (1e-7, 2e-7), "bf16": (1e-6, 2e-6)}


@pytest.mark.parametrize("form", ["tf32", "bf16"])
def test_single_chain_mixed_matches_fp64_oracle(lib, form):
    from paper_1504_00992_gb300 import binding as B
    N, d, chi, delta, steps, dt, p, q, seed = 14, 2, 16, 0.5, 12, 0.05, 6, 2, 5
    hs = I.xxz_bond_terms(N, d, 1.0, delta)
    prec = B.TEBD_PREC_BF16 if form == "bf16" else B.TEBD_PREC_TF32
    sim = B.Tebd(N, d, chi, p, q, seed, precision=prec)
    sim.set_product_state(I.neel_state(N, d))
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    _, _, sz = I.spin_ops(d)
    got = np.array([sim.expect(k, sz).real for k in range(N)])
    lam = [sim.get_lambda(b) for b in range(N - 1)]
    w = sim.discarded_weight()
    sim.close()
    exp, lam_o, w_o = _oracle(N, d, chi, delta, steps, dt, p, q, seed)
    bo, bl = BARS[form]
    d_obs = np.abs(got - exp).max()
    d_lam = max(np.abs(lam[b][:min(len(lam[b]), len(lam_o[b]))] - lam_o[b][:min(len(lam[b]), len(lam_o[b]))]).max()
                for b in range(N - 1))
    print(f"{form}: observables {d_obs:.2e}, Schmidt values {d_lam:.2e}, weight {abs(w[0] - w_o):.2e}")
    assert d_obs <= bo
    assert d_lam <= bl
    assert abs(w[0] - w_o) <= 1e-10


def test_multichain_tf32_waves_and_graphs(lib):
    """Uneven chains (d in {2, 3}, chi_max in {4, 8, 12}) in one TF32 handle,
    split into waves by a workspace budget and replayed from CUDA graphs:
    every chain agrees with its own FP64 oracle run within the form's
    tolerance."""
    from paper_1504_00992_gb300 import binding as B
    rng = np.random.default_rng(11)
    specs = []
    for _ in range(6):
        specs.append((int(rng.integers(6, 11)), int(rng.choice([2, 3])), int(rng.choice([4, 8, 12])),
                      float(rng.random())))
    steps, dt, p, q, seed = 6, 0.05, 4, 1, 21
    chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
    sim = B.MultiTebd(chains, p, q, seed, use_graph=1, workspace_budget=300_000, precision=B.TEBD_PREC_TF32)
    for c, (N, d, chi, delta) in enumerate(specs):
        hs = I.xxz_bond_terms(N, d, 1.0, delta)
        sim.set_product_state(c, I.neel_state(N, d))
        sim.set_gates(c, 0, I.trotter_gates(hs, dt / 2))
        sim.set_gates(c, 1, I.trotter_gates(hs, dt))
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    info = sim.workspace_info()
    assert info[1] > 1 and info[2] > 1           # the budget split the sweeps into waves
    for c, (N, d, chi, delta) in enumerate(specs):
        _, _, sz = I.spin_ops(d)
        got = np.array([sim.expect(c, k, sz).real for k in range(N)])
        exp, lam_o, w_o = _oracle(N, d, chi, delta, steps, dt, p, q, seed, chain=c)
        assert np.abs(got - exp).max() <= 1e-7, c
        for b in range(N - 1):
            lg = sim.get_lambda(c, b)
            r = min(len(lg), len(lam_o[b]))
            assert np.abs(lg[:r] - lam_o[b][:r]).max() <= 2e-7, (c, b)
        assert abs(sim.discarded_weight(c)[0] - w_o) <= 1e-10
    sim.close()


def test_tf32_handle_rejects_recording_and_tunes_its_launches(lib):
    """The reverse pass differentiates the FP64 form, so recording is refused
    on TF32 handles; the autotuner times the mixed form's launch choices and
    a tuned handle agrees with an untuned one to the form's tolerance."""
    from paper_1504_00992_gb300 import binding as B
    sim = B.Tebd(6, 2, 4, 2, 1, 0, precision=B.TEBD_PREC_TF32)
    with pytest.raises(B.TebdError) as ei:
        sim.record(True)
    assert ei.value.code == B.TEBD_ENOTIMPL
    sim.close()
    N, d, chi = 12, 2, 8
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)
    out = []
    for tune in (1, 0):
        sim = B.Tebd(N, d, chi, 4, 1, 0, autotune=tune, precision=B.TEBD_PREC_TF32)
        table = sim.tuning_table()
        if tune:
            assert all(w["tune_ms"][0] > 0 and w["tune_ms"][1] > 0 for par in (0, 1) for w in table[par])
        sim.set_product_state(I.neel_state(N, d))
        sim.set_gates(0, I.trotter_gates(hs, 0.025))
        sim.set_gates(1, I.trotter_gates(hs, 0.05))
        for _ in range(4):
            sim.step_even(); sim.step_odd(); sim.step_even()
        _, _, sz = I.spin_ops(d)
        out.append(np.array([sim.expect(k, sz).real for k in range(N)]))
        sim.close()
    assert np.abs(out[0] - out[1]).max() <= 1e-7
