"""Failure detection made on the host (no GPU fault, no GPU needed): an
injected allocation failure turns into TEBD_ENOMEM before any CUDA call, and
the argument checks of the allocator hook and the fault hook."""
import ctypes

import pytest

from paper_1504_00992_gb300 import binding as B
from paper_1504_00992_gb300 import build as _build


@pytest.fixture(scope="module")
def L():
    return B.load(_build.build())


def test_injected_allocation_fault_reports_enomem(L):
    h = ctypes.c_void_p()
    try:
        assert L.tebd_fault_inject(B.TEBD_FAULT_ALLOC) == B.TEBD_OK
        # the handle's arena is its first device allocation: it fails before
        # the library makes any CUDA call, and nothing is left behind
        assert L.tebd_create(6, 2, 4, 2, 1, 0, ctypes.byref(h)) == B.TEBD_ENOMEM
        assert not h.value
        # armed once: the next failure would be a real one (an argument error
        # is still reported first and consumes nothing)
        assert L.tebd_fault_inject(B.TEBD_FAULT_ALLOC) == B.TEBD_OK
        assert L.tebd_create(1, 2, 4, 2, 1, 0, ctypes.byref(h)) == B.TEBD_EINVAL
        assert L.rrsvd_plan_create(8, 8, 2, 1, 1, 1, B.TEBD_PREC_FP64, 0, ctypes.byref(h)) == B.TEBD_ENOMEM
        assert not h.value
    finally:
        L.tebd_fault_inject(B.TEBD_FAULT_NONE)


def test_fault_hook_rejects_unknown_kinds(L):
    assert L.tebd_fault_inject(7) == B.TEBD_EINVAL
    assert L.tebd_fault_inject(-1) == B.TEBD_EINVAL
    assert L.tebd_fault_inject(B.TEBD_FAULT_NONE) == B.TEBD_OK


def test_allocator_callbacks_come_in_pairs(L):
    calls = []

    def alloc(nbytes, ctx):
        calls.append(nbytes)
        return None

    fa = B.ALLOC_FN(alloc)
    d = B._desc(6, [2] * 6, [4] * 5, 2, 1, 0)
    d.alloc = fa          # no release: refused while planning, nothing allocated
    h = ctypes.c_void_p()
    assert L.tebd_create_ex(ctypes.byref(d), ctypes.byref(h)) == B.TEBD_EINVAL
    assert not calls and not h.value
    B._KEEP.clear()
    assert L.tebd_set_allocator(None, fa, B.RELEASE_FN(), None) == B.TEBD_EINVAL


def test_allocator_returning_null_reports_enomem(L):
    calls = []

    class NoMemory:
        def __init__(self):
            self.alloc = B.ALLOC_FN(lambda nbytes, ctx: calls.append(nbytes))
            self.release = B.RELEASE_FN(lambda ptr, ctx: None)

    a = NoMemory()
    d = B._desc(6, [2] * 6, [4] * 5, 2, 1, 0, allocator=a)
    h = ctypes.c_void_p()
    # the arena request reaches the caller's allocator; NULL means out of memory
    assert L.tebd_create_ex(ctypes.byref(d), ctypes.byref(h)) == B.TEBD_ENOMEM
    size = ctypes.c_size_t()
    assert L.tebd_plan_query(1, ctypes.byref(d), ctypes.byref(size), None, None) == B.TEBD_OK
    B._KEEP.clear()
    assert calls == [size.value]
    assert not h.value
