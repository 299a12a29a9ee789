"""Host planning of a TEBD handle (tebd_plan_query): the bonds of each parity,
their waves under a workspace budget and the device arena, as the library
plans them for tebd_create_multi, computed on the host with no GPU."""
import ctypes

import numpy as np
import pytest

from paper_1504_00992_gb300 import binding as B
from paper_1504_00992_gb300 import build as BLD
from paper_1504_00992_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def lib():
    return B.load(BLD.build())


def _chain(N, d, chi):
    return (N, [d] * N, [chi] * (N - 1))


def _caps(ds, chi_bond):
    """Bond dimensions the state can reach (Section II): bond b is capped by
    chi_b and by the dimensions of the sites on either side of it."""
    N = len(ds)
    ext = [1] * (N + 1)
    for b in range(N - 1):
        ext[b + 1] = int(min(chi_bond[b], np.prod(ds[:b + 1], dtype=float), np.prod(ds[b + 1:], dtype=float)))
    return ext


def test_one_wave_per_parity_without_a_budget():
    for prec in (B.TEBD_PREC_FP64, B.TEBD_PREC_TF32):
        _, we, wo = B.tebd_plan_query([_chain(20, 2, 32)], 10, 2, 0, precision=prec)
        assert (we, wo) == (1, 1)


@pytest.mark.parametrize("N", [2, 3, 20, 21])
def test_a_one_byte_budget_puts_every_bond_in_its_own_wave(N):
    full, _, _ = B.tebd_plan_query([_chain(N, 2, 32)], 10, 2, 0)
    tiny, we, wo = B.tebd_plan_query([_chain(N, 2, 32)], 10, 2, 0, workspace_budget=1)
    # even bonds 0, 2, ..; odd bonds 1, 3, ..; a parity without bonds has no wave
    assert (we, wo) == (N // 2, (N - 1) // 2)
    if N > 3:
        assert tiny < full  # workspace of the largest wave, not of all bonds


def test_arena_holds_the_state_and_every_theta_of_a_parity():
    """Lower bound from first principles: Gamma of every site, a gate per
    bond and, with one wave, the theta matrix (m x n complex) of every bond
    of the larger parity at its capacity."""
    N, d, chi = 12, 3, 20
    ds, cb = [d] * N, [chi] * (N - 1)
    ext = _caps(ds, cb)
    gam = sum(16 * ds[s] * ext[s] * ext[s + 1] for s in range(N))
    gates = sum(16 * (ds[b] * ds[b + 1]) ** 2 for b in range(N - 1))
    theta = max(sum(16 * ds[b] * ext[b] * ds[b + 1] * ext[b + 2] for b in range(par, N - 1, 2)) for par in (0, 1))
    arena, _, _ = B.tebd_plan_query([(N, ds, cb)], 6, 2, 0)
    assert arena >= gam + gates + theta
    # and it is not wildly above it: the RRSVD workspace of a bond is a few
    # m x l and n x l blocks, below 8 theta matrices here
    assert arena <= gam + gates + 8 * theta + (1 << 20)


def test_waves_never_fewer_when_the_budget_shrinks():
    specs = I.many_chain_specs(64, 0)
    chains = [_chain(N, d, chi) for N, d, chi, _ in specs]
    for prec in (B.TEBD_PREC_FP64, B.TEBD_PREC_TF32, B.TEBD_PREC_BF16):
        prev = (1, 1)
        for gb in (64, 16, 4, 1, 0.25):
            _, we, wo = B.tebd_plan_query(chains, 10, 1, 0, precision=prec, workspace_budget=int(gb * (1 << 30)))
            assert we >= prev[0] and wo >= prev[1], (prec, gb)
            prev = (we, wo)
        assert prev[0] > 1 and prev[1] > 1


def test_argument_errors():
    with pytest.raises(B.TebdError) as e:
        B.tebd_plan_query([_chain(6, 65, 8)], 4, 1, 0)            # d > 64
    assert e.value.code == B.TEBD_EINVAL
    with pytest.raises(B.TebdError) as e:
        B.tebd_plan_query([_chain(6, 2, 0)], 4, 1, 0)             # chi cap < 1
    assert e.value.code == B.TEBD_EINVAL
    with pytest.raises(B.TebdError) as e:
        B.tebd_plan_query([_chain(6, 2, 8)], 4, 1, 0, precision=7)
    assert e.value.code == B.TEBD_ENOTIMPL
    # the BF16 form holds its BF16 copies beside the FP32 arrays
    a_tf = B.tebd_plan_query([_chain(20, 2, 64)], 4, 1, 0, precision=B.TEBD_PREC_TF32)[0]
    a_bf = B.tebd_plan_query([_chain(20, 2, 64)], 4, 1, 0, precision=B.TEBD_PREC_BF16)[0]
    assert a_bf > a_tf
    # the autotuner covers the mixed form too: the plan is the same as untuned
    assert B.tebd_plan_query([_chain(6, 2, 8)], 4, 1, 0, precision=B.TEBD_PREC_TF32, autotune=1) == \
        B.tebd_plan_query([_chain(6, 2, 8)], 4, 1, 0, precision=B.TEBD_PREC_TF32)
    with pytest.raises(B.TebdError) as e:                           # sketch width l = 1024 + 4 > 512
        B.tebd_plan_query([_chain(4, 64, 1024)], 4, 1, 0)
    assert e.value.code == B.TEBD_ENOTIMPL
    # chains that disagree on p
    L = B.load()
    arr = (B.TebdDesc * 2)()
    keep = []
    for c, p in enumerate((4, 5)):
        ds = (ctypes.c_int * 6)(*([2] * 6))
        cb = (ctypes.c_int * 5)(*([8] * 5))
        keep.append((ds, cb))
        arr[c] = B.TebdDesc(6, 2, ds, 8, cb, p, 1, 0, B.TEBD_PREC_FP64, 0.0, 0, 0, 0, 0)
    nb = ctypes.c_size_t(7)
    assert L.tebd_plan_query(2, arr, ctypes.byref(nb), None, None) == B.TEBD_EINVAL
    assert nb.value == 7  # outputs untouched on error
    assert L.tebd_plan_query(0, arr, None, None, None) == B.TEBD_EINVAL
    assert L.tebd_plan_query(1, None, None, None, None) == B.TEBD_EINVAL


def test_a_handle_larger_than_any_device_reports_enomem():
    """Allocation failure is reported as a status, not a crash: 20 chains of
    60 sites with d = 64 and caps of 500 plan a 20 TB arena, more than any
    device holds, so creation fails with TEBD_ENOMEM and returns no handle.
    Without a device the allocation fails the same way, so this runs on the
    host too."""
    chains = [_chain(60, 64, 500)] * 20
    arena, _, _ = B.tebd_plan_query(chains, 10, 2, 0)
    assert arena > 10 * (1 << 40)
    with pytest.raises(B.TebdError) as e:
        B.tebd_create_multi(chains, 10, 2, 0)
    assert e.value.code == B.TEBD_ENOMEM
