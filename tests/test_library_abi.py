"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/tebd_gb300.h (no compute calls: no GPU needed)."""
import ctypes
import os

import pytest

from paper_1504_00992_gb300 import binding
from paper_1504_00992_gb300 import build as B


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_function(libpath):
    L = ctypes.CDLL(libpath)
    names = binding.header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(binding._SIGS), set(names) ^ set(binding._SIGS)


def test_library_is_built_for_sm_103a_only(libpath):
    # every translation unit and the link get exactly one -gencode: real
    # sm_103a code, no PTX for other targets to JIT from
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(libpath) > 0


def test_argument_errors_need_no_device(libpath):
    L = binding.load(libpath)
    h = ctypes.c_void_p()
    assert L.tebd_create(1, 2, 4, 2, 1, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.tebd_create(4, 1, 4, 2, 1, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.tebd_create(4, 2, 0, 2, 1, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.tebd_create(4, 2, 4, -1, 1, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.tebd_create(4, 2, 4, 2, 1, 0, None) == binding.TEBD_EINVAL
    assert L.rrsvd_plan_create(0, 4, 2, 1, 1, 1, 0, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.rrsvd_plan_create(4, 4, 2, 1, 1, 1, 7, 0, ctypes.byref(h)) == binding.TEBD_ENOTIMPL
    # an empty batch, negative oversampling or power rounds
    assert L.rrsvd_plan_create(8, 8, 2, 1, 1, 0, 0, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.rrsvd_plan_create(8, 8, 2, -1, 1, 1, 0, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.rrsvd_plan_create(8, 8, 2, 1, -1, 1, 0, 0, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert not h.value                                  # *out cleared on every refusal
    # a sketch wider than 512 columns (l = min(k + p, m, n) = 620)
    assert L.rrsvd_plan_create(2000, 2000, 600, 20, 2, 1, 0, 0, ctypes.byref(h)) == binding.TEBD_ENOTIMPL
    # Alg. 2's accuracy check: FP64 only, and a positive threshold
    assert L.rrsvd_plan_create_ex(64, 64, 8, 4, 1, 1, binding.TEBD_PREC_TF32, 0, 4, 1e-3, 32,
                                  ctypes.byref(h)) == binding.TEBD_ENOTIMPL
    assert L.rrsvd_plan_create_ex(64, 64, 8, 4, 1, 1, 0, 0, 4, 0.0, 32, ctypes.byref(h)) == binding.TEBD_EINVAL
    assert L.rrsvd_plan_create_ex(64, 64, 8, 4, 1, 1, 0, 0, -1, 1e-3, 32, ctypes.byref(h)) == binding.TEBD_EINVAL
    info = (ctypes.c_int * 16)()
    assert L.rrsvd_plan_set_tuning(None, info) == binding.TEBD_EINVAL
    assert L.tebd_destroy(None) == binding.TEBD_OK
    assert L.rrsvd_plan_destroy(None) == binding.TEBD_OK
