"""The C-ABI boundary of TEBD handles on the GPU: device memory from the
caller's allocator (PyTorch's caching allocator), checkpoint and resume,
per-bond discarded weights, and failure detection made on the host.

Every kernel of the update is deterministic (fixed reduction orders, no
atomics on floating-point values), so runs that differ only in where their
memory lives, or in having been interrupted and resumed with the same sweep
counter, must agree bit for bit (Section II.C: the sweeps; Section IV: Omega
keyed on the sweep counter)."""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle import tebd as T
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

N, D, CHI, P, Q, SEED, DT = 14, 2, 16, 6, 2, 5, 0.05


def _chain(B, chi=CHI, **kw):
    hs = I.xxz_bond_terms(N, D, 1.0, 0.7)
    sim = B.Tebd(N, D, chi, P, Q, SEED, **kw)
    sim.set_product_state(I.neel_state(N, D))
    sim.set_gates(0, I.trotter_gates(hs, DT / 2))
    sim.set_gates(1, I.trotter_gates(hs, DT))
    return sim


def _steps(sim, n):
    for _ in range(n):
        sim.step_even(); sim.step_odd(); sim.step_even()


def _state(sim):
    _, _, sz = I.spin_ops(D)
    lam = [sim.get_lambda(b) for b in range(N - 1)]
    ex = np.array([sim.expect(k, sz) for k in range(N)])
    return lam, ex, sim.discarded_weight()


def _identical(a, b):
    (la, ea, wa), (lb, eb, wb) = a, b
    assert len(la) == len(lb)
    for x, y in zip(la, lb):
        assert x.shape == y.shape and np.array_equal(x, y)
    assert np.array_equal(ea, eb)
    assert wa == wb


def test_torch_allocated_handle_matches_cudamalloc_handle_bit_for_bit(lib):
    from paper_1504_00992_gb300 import binding as B
    torch = torch_cuda()
    ref = _chain(B)
    _steps(ref, 12)
    s_ref = _state(ref)
    ref.close()
    alloc = B.TorchAllocator()
    before = torch.cuda.memory_allocated()
    sim = _chain(B, allocator=alloc, use_graph=1)
    # the arena is one block of the caching allocator, of the planned size
    arena = B.tebd_workspace_info(sim.h)[0]
    assert list(alloc.live.values()) == [arena]
    assert torch.cuda.memory_allocated() - before >= arena
    _steps(sim, 12)
    _identical(_state(sim), s_ref)
    sim.close()
    assert not alloc.live   # every block went back to the pool


def test_moving_a_live_handle_keeps_its_state_and_checkpoints(lib):
    from paper_1504_00992_gb300 import binding as B
    _, _, sz = I.spin_ops(D)
    ref = _chain(B)
    ref.record(True)
    _steps(ref, 6)
    s_ref = _state(ref)
    g_ref = ref.backward(7, sz)
    ref.close()
    alloc = B.TorchAllocator()
    sim = _chain(B, use_graph=0)
    sim.record(True)
    _steps(sim, 3)
    sim.set_allocator(alloc)        # cudaMalloc -> torch, with 9 checkpoints
    assert len(alloc.live) == 1 + 9
    _steps(sim, 2)
    sim.set_allocator(None)         # and back: every block returned to torch
    assert not alloc.live
    _steps(sim, 1)
    _identical(_state(sim), s_ref)
    g = sim.backward(7, sz)        # the moved checkpoints drive the reverse pass
    for par in range(2):
        for x, y in zip(g[par], g_ref[par]):
            assert np.array_equal(x, y)
    sim.close()


def test_resume_from_checkpoint_is_bit_identical(lib):
    from paper_1504_00992_gb300 import binding as B
    full = _chain(B)
    _steps(full, 20)
    s_full = _state(full)
    w_full = full.bond_weights()
    full.close()
    first = _chain(B)
    _steps(first, 10)
    g, lam = first.get_mps()
    sweeps = first.sweeps()
    first.close()
    assert sweeps == 30
    hs = I.xxz_bond_terms(N, D, 1.0, 0.7)
    for restore in (True, False):
        sim = B.Tebd(N, D, CHI, P, Q, SEED)
        sim.set_mps(g, lam)
        assert sim.sweeps() == 0        # set_mps resets the counter ...
        sim.set_gates(0, I.trotter_gates(hs, DT / 2))
        sim.set_gates(1, I.trotter_gates(hs, DT))
        if restore:
            sim.set_sweep_count(sweeps)  # ... and the checkpointed one is restored
        _steps(sim, 10)
        st = _state(sim)
        if restore:
            lam_r, ex_r, _ = st
            for x, y in zip(lam_r, s_full[0]):
                assert np.array_equal(x, y)
            assert np.array_equal(ex_r, s_full[1])
            assert np.array_equal(sim.bond_weights(), w_full)
        else:
            # another sweep counter draws other sketches: the truncated
            # states differ (slightly), so the counter is what resume needs
            assert any(not np.array_equal(x, y) for x, y in zip(st[0], s_full[0]))
        sim.close()


def test_bond_weights_match_the_oracle(lib):
    from paper_1504_00992_gb300 import binding as B
    hs = I.xxz_bond_terms(N, D, 1.0, 0.7)
    ge, go = I.trotter_gates(hs, DT / 2), I.trotter_gates(hs, DT)
    chi = 3    # small enough that the central bonds truncate within the run
    sim = _chain(B, chi=chi)
    ref = T.TEBD(T.product_state(I.neel_state(N, D)), chi, P, Q, SEED)
    ref.set_gates(0, ge)
    ref.set_gates(1, go)
    assert np.array_equal(sim.bond_weights(), np.zeros(N - 1))
    latest = np.zeros(N - 1)
    for _ in range(8):
        for par, s, r in ((0, sim.step_even, ref.step_even), (1, sim.step_odd, ref.step_odd),
                          (0, sim.step_even, ref.step_even)):
            s()
            ws = r()
            for i, b in enumerate(range(par, N - 1, 2)):
                latest[b] = ws[i]
    got = sim.bond_weights()
    assert np.abs(got - latest).max() <= 1e-12
    assert abs(got.sum() - sum(latest)) <= 1e-11
    assert got.max() > 1e-8    # the chain truncates
    sim.close()


def test_injected_tensor_core_stall_reports_timeout_and_recovers(lib):
    """The mixed form's tensor-core product with no operand copies: its
    bounded pipeline waits expire, the kernel frees its tensor memory and
    returns, TEBD_ETIMEOUT is reported, and the same plan (error cleared)
    then truncates exactly as a fresh plan does -- a later allocation of
    tensor memory would block if the stalled kernel had not freed it."""
    from paper_1504_00992_gb300 import binding as B
    m = n = 256
    k, p, q, batch = 40, 10, 1, 3
    sig = I.exp_spectrum(n, 10.0)
    th = np.stack([I.synthetic_theta(m, n, sig, seed=300 + t) for t in range(batch)])

    def run(plan):
        kk, _ = B.rrsvd_plan_dims(plan)
        sg, U = np.zeros((batch, kk)), np.zeros((batch, m, kk), dtype=np.complex128)
        B.rrsvd_execute_host(plan, th, 0, sg, U)
        return sg, U

    fresh = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_TF32, 17)
    try:
        ref_s, ref_u = run(fresh)
    finally:
        B.rrsvd_plan_destroy(fresh)
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_TF32, 17)
    try:
        B.tebd_fault_inject(B.TEBD_FAULT_TC_STALL)
        with pytest.raises(B.TebdError) as ei:
            run(plan)
        assert ei.value.code == B.TEBD_ETIMEOUT
        with pytest.raises(B.TebdError):   # errors are sticky until cleared
            run(plan)
        B.rrsvd_clear_error(plan)
        for _ in range(2):   # every later product runs normally
            sg, U = run(plan)
            assert np.array_equal(sg, ref_s) and np.array_equal(U, ref_u)
    finally:
        B.tebd_fault_inject(B.TEBD_FAULT_NONE)
        B.rrsvd_plan_destroy(plan)


def test_injected_stall_in_a_tebd_handle_reports_timeout(lib):
    from paper_1504_00992_gb300 import binding as B
    ref = _chain(B, precision=B.TEBD_PREC_TF32)
    _steps(ref, 2)
    s_ref = _state(ref)
    ref.close()
    sim = _chain(B, precision=B.TEBD_PREC_TF32)
    try:
        _steps(sim, 2)
        sim.discarded_weight()
        B.tebd_fault_inject(B.TEBD_FAULT_TC_STALL)
        sim.step_even()
        with pytest.raises(B.TebdError) as ei:
            sim.discarded_weight()
        assert ei.value.code == B.TEBD_ETIMEOUT
    finally:
        B.tebd_fault_inject(B.TEBD_FAULT_NONE)
        sim.close()
    # the context is intact: a fresh handle runs exactly as before
    sim = _chain(B, precision=B.TEBD_PREC_TF32)
    _steps(sim, 2)
    _identical(_state(sim), s_ref)
    sim.close()


def test_injected_allocation_faults_on_the_gpu(lib):
    from paper_1504_00992_gb300 import binding as B
    try:
        B.tebd_fault_inject(B.TEBD_FAULT_ALLOC)
        with pytest.raises(B.TebdError) as ei:
            _chain(B)
        assert ei.value.code == B.TEBD_ENOMEM
        sim = _chain(B)                 # the next allocation succeeds
        sim.record(True)
        sim.step_even()
        B.tebd_fault_inject(B.TEBD_FAULT_ALLOC)
        with pytest.raises(B.TebdError) as ei:
            sim.step_odd()              # its checkpoint cannot be allocated
        assert ei.value.code == B.TEBD_ENOMEM
        sim.close()
        plan = B.rrsvd_plan_create(32, 32, 4, 2, 1, 1, B.TEBD_PREC_FP64, 0)
        B.tebd_fault_inject(B.TEBD_FAULT_ALLOC)
        with pytest.raises(B.TebdError) as ei:
            B.rrsvd_execute_host(plan, np.zeros((1, 32, 32), dtype=np.complex128) + 1.0, 0, np.zeros((1, 4)))
        assert ei.value.code == B.TEBD_ENOMEM   # the staging buffers
        B.rrsvd_plan_destroy(plan)
    finally:
        B.tebd_fault_inject(B.TEBD_FAULT_NONE)
