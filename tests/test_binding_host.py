"""Host-side marshalling of the binding's host-buffer calls (no GPU: the
library is replaced by a recording fake): the numpy arrays are checked
against the extents the library reads and writes before any call is made,
and the arrays of asynchronous calls are held by the binding until the
plan's wait."""
import ctypes
import gc
import weakref

import numpy as np
import pytest

from paper_1504_00992_gb300 import binding as B

K = 4


class FakeLib:
    def __init__(self):
        self.calls = []

    def rrsvd_plan_dims(self, plan, k, l):
        k._obj.value = K
        l._obj.value = K + 2
        return 0

    def rrsvd_execute_host(self, *a):
        self.calls.append("host")
        return 0

    def rrsvd_execute_host_async(self, *a):
        self.calls.append("async")
        return 0

    def rrsvd_host_wait(self, plan):
        self.calls.append("wait")
        return 0

    def rrsvd_plan_destroy(self, plan):
        self.calls.append("destroy")
        return 0

    def rrsvd_last_error(self, plan):
        return b""


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(B, "load", lambda path=None: f)
    B._IN_FLIGHT.clear()
    yield f
    B._IN_FLIGHT.clear()


def _arrays(batch=3, m=10, n=8):
    return (np.zeros((batch, m, n), dtype=np.complex128), np.zeros((batch, K)),
            np.zeros((batch, m, K), dtype=np.complex128), np.zeros((batch, K, n), dtype=np.complex128),
            np.zeros(batch), np.zeros(batch, dtype=np.int32))


def test_well_formed_arrays_reach_the_library(fake):
    plan = ctypes.c_void_p(0x1000)
    B.rrsvd_execute_host(plan, *_arrays()[:1], 0, *_arrays()[1:])
    B.rrsvd_execute_host(plan, _arrays()[0], 0, _arrays()[1])          # optional outputs left out
    assert fake.calls == ["host", "host"]


@pytest.mark.parametrize("slot,bad", [
    (0, lambda a: a.astype(np.complex64)),                  # theta in single precision
    (0, lambda a: a[:, :, ::2]),                            # theta not contiguous
    (0, lambda a: a[0]),                                    # theta without a batch axis
    (1, lambda a: np.zeros((a.shape[0], K + 1))),           # sigma wider than the plan's k
    (1, lambda a: a.astype(np.float32)),
    (2, lambda a: np.asfortranarray(a)),                    # U in column-major order
    (3, lambda a: a[:, :, :-1].copy()),                     # Vh too small
    (4, lambda a: np.zeros(a.size + 1)),                    # w of the wrong length
    (5, lambda a: a.astype(np.int64)),                      # rank as 64-bit integers
])
def test_malformed_arrays_are_refused_before_the_call(fake, slot, bad):
    args = list(_arrays())
    args[slot] = bad(args[slot])
    for call in (B.rrsvd_execute_host, B.rrsvd_execute_host_async):
        with pytest.raises(B.TebdError) as ei:
            call(ctypes.c_void_p(0x1000), args[0], 0, *args[1:])
        assert ei.value.code == B.TEBD_EINVAL
    assert fake.calls == []


def test_read_only_output_is_refused(fake):
    args = list(_arrays())
    args[1].flags.writeable = False
    with pytest.raises(B.TebdError) as ei:
        B.rrsvd_execute_host(ctypes.c_void_p(0x1000), args[0], 0, *args[1:])
    assert ei.value.code == B.TEBD_EINVAL and fake.calls == []
    ro_theta = _arrays()[0]
    ro_theta.flags.writeable = False                        # theta is only read
    B.rrsvd_execute_host(ctypes.c_void_p(0x1000), ro_theta, 0, _arrays()[1])
    assert fake.calls == ["host"]


def test_async_arrays_live_until_the_wait(fake):
    plan, other = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000)
    refs = []
    for p in (plan, plan, other):
        arrs = _arrays()
        refs.append([weakref.ref(a) for a in arrs])
        B.rrsvd_execute_host_async(p, arrs[0], 0, *arrs[1:])
        del arrs
    gc.collect()
    assert all(r() is not None for rs in refs for r in rs)    # the caller dropped them; the binding holds them
    B.rrsvd_host_wait(plan)
    gc.collect()
    assert all(r() is None for rs in refs[:2] for r in rs)    # released by this plan's wait
    assert all(r() is not None for r in refs[2])              # the other plan's call still in flight
    B.rrsvd_plan_destroy(other)                               # destroy waits in the library, then releases
    gc.collect()
    assert all(r() is None for r in refs[2])
    assert fake.calls == ["async", "async", "async", "wait", "destroy"]


def test_blocking_call_releases_pending_async_arrays(fake):
    plan = ctypes.c_void_p(0x1000)
    arrs = _arrays()
    ref = weakref.ref(arrs[0])
    B.rrsvd_execute_host_async(plan, arrs[0], 0, *arrs[1:])
    del arrs
    B.rrsvd_execute_host(plan, *_arrays()[:1], 0, _arrays()[1])   # the library waits for pending calls first
    gc.collect()
    assert ref() is None and B._IN_FLIGHT == {}
