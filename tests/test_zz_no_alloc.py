"""The no-allocation truncation entry point, for callers that cannot call
cudaMalloc (code inside another library's scheduling loop or a host callback
that must not block, or a process whose device memory is reserved up front):
it gives the oracle's truncation (Alg. 1 and the projection steps of
Section IV, same Omega) and the same results as the workspace-based
rrsvd_execute, on calls in a row that reuse its static scratch, and the
device's free memory does not move across a call.

The file name sorts last so that a run stopping at the first failure has run
every other test first: the entry point's one-time set-up (the lookup of its
static array's device address) then also happens after the rest of the suite
has used the device, as well as in a fresh process when run alone."""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I
from tests.gpu_util import rrsvd_device, torch_cuda, truncated

pytestmark = pytest.mark.gpu


def _noalloc(B, theta, k, p, q, seed, chain0, outputs=True):
    torch = torch_cuda()
    batch, m, n = theta.shape
    kk = min(k, m, n)
    dev = torch.device("cuda:0")
    th = torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    sg = torch.full((batch, kk), -1.0, dtype=torch.float64, device=dev)
    U = torch.zeros((batch, m, kk), dtype=torch.complex128, device=dev)
    Vh = torch.zeros((batch, kk, n), dtype=torch.complex128, device=dev)
    w = torch.zeros(batch, dtype=torch.float64, device=dev)
    rk = torch.zeros(batch, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream().cuda_stream

    def call():
        if outputs:
            B.rrsvd_execute_noalloc(m, n, k, p, q, batch, seed, chain0, th.data_ptr(), sg.data_ptr(),
                                    U.data_ptr(), Vh.data_ptr(), w.data_ptr(), rk.data_ptr(), st)
        else:   # sigma only: U and V^H stay in the static array, w and rank are not written
            B.rrsvd_execute_noalloc(m, n, k, p, q, batch, seed, chain0, th.data_ptr(), sg.data_ptr(), 0, 0, 0, 0,
                                    st)

    # the same call twice in a row; the first may load kernel code on first
    # use (lazy module loading), so the device's free memory is read across
    # the second, which must not move it
    call()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    call()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return {"sigma": sg.cpu().numpy(), "U": U.cpu().numpy(), "Vh": Vh.cpu().numpy(), "w": w.cpu().numpy(),
            "rank": rk.cpu().numpy(), "free_delta": free0 - free1}


def _reference(B, theta, k, p, q, seed, chain0):
    batch, m, n = theta.shape
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_FP64, seed)
    try:
        return rrsvd_device(B, plan, theta, chain0=chain0)
    finally:
        B.rrsvd_plan_destroy(plan)


def _same(a, b, theta):
    for t in range(theta.shape[0]):
        s0 = b["sigma"][t][0]
        assert a["rank"][t] == b["rank"][t]
        assert np.abs(a["sigma"][t] - b["sigma"][t]).max() <= 1e-10 * s0
        d = truncated(a["U"][t], a["sigma"][t], a["Vh"][t]) - truncated(b["U"][t], b["sigma"][t], b["Vh"][t])
        assert np.linalg.norm(d) <= 1e-10 * np.linalg.norm(theta[t])
        assert abs(a["w"][t] - b["w"][t]) <= 1e-12


def _matches_oracle(a, theta, k, p, q, seed, chain0):
    """Element-wise parity with the oracle on the same Omega: kept values to
    1e-10 s_1, the truncated theta to 1e-10 in Frobenius norm, w to 1e-12."""
    batch, m, n = theta.shape
    kk, l = R.sketch_sizes(m, n, k, p)
    for t in range(batch):
        Uk, sk, Vhk, w = R.rrsvd_truncate(theta[t], gaussian_omega(n, l, seed, chain=chain0 + t), kk, q)
        r = len(sk)
        assert a["rank"][t] == r
        assert np.abs(a["sigma"][t][:r] - sk).max() <= 1e-10 * sk[0]
        assert np.all(a["sigma"][t][r:] == 0.0)
        d = truncated(a["U"][t], a["sigma"][t], a["Vh"][t]) - (Uk * sk) @ Vhk
        assert np.linalg.norm(d) <= 1e-10 * np.linalg.norm(theta[t])
        assert abs(a["w"][t] - w) <= 1e-12


def test_noalloc_matches_oracle_and_workspace_entry_point_twice(lib):
    from paper_1504_00992_gb300 import binding as B
    # two 96 x 80 instances
    sig = I.exp_spectrum(80, 6.0)
    th1 = np.stack([I.synthetic_theta(96, 80, sig, seed=40 + t) for t in range(2)])
    a1 = _noalloc(B, th1, 20, 7, 2, 99, 3)
    _matches_oracle(a1, th1, 20, 7, 2, 99, 3)
    _same(a1, _reference(B, th1, 20, 7, 2, 99, 3), th1)
    # second call right after, other sizes and chains, same static scratch
    sig2 = I.exp_spectrum(64, 5.0)
    th2 = np.stack([I.synthetic_theta(64, 64, sig2, seed=77)])
    a2 = _noalloc(B, th2, 32, 10, 2, 5, 11)
    _matches_oracle(a2, th2, 32, 10, 2, 5, 11)
    _same(a2, _reference(B, th2, 32, 10, 2, 5, 11), th2)
    # the device's free memory did not move across the repeated calls
    assert a1["free_delta"] == 0 and a2["free_delta"] == 0


def test_noalloc_without_optional_outputs(lib):
    from paper_1504_00992_gb300 import binding as B
    sig = I.exp_spectrum(100, 8.0)
    th = np.stack([I.synthetic_theta(120, 100, sig, seed=90 + t) for t in range(3)])
    full = _noalloc(B, th, 24, 8, 1, 7, 0)
    bare = _noalloc(B, th, 24, 8, 1, 7, 0, outputs=False)
    assert np.array_equal(bare["sigma"], full["sigma"])   # same kernels, same Omega: bit for bit
    assert bare["free_delta"] == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_1504_00992_gb300 import binding as B
    torch = torch_cuda()
    th = torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda:0")
    sg = torch.zeros((1, 4), dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.TebdError) as ei:
        B.rrsvd_execute_noalloc(2048, 2048, 100, 20, 2, 1, 0, 0, th.data_ptr(), sg.data_ptr())
    assert ei.value.code == B.TEBD_EINVAL
