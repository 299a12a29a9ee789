"""The library's sketch generator against the oracle's (Section IV, Alg. 1:
the Gaussian test matrix Omega).

Parity of every truncation with the oracle rests on both sides drawing the
identical Omega.  These tests check the generator directly rather than
through the truncation results, which can be insensitive to Omega (l =
min(m, n) makes the RRSVD exact for any Omega):
  - the Philox4x64-10 words are integers: equal bit for bit;
  - the FP64 Omega: the uniforms are exact in both, so the values differ only
    by the rounding of log, sqrt and the sine/cosine (NumPy rounds 2 pi u2
    before its cos/sin, CUDA's sincospi takes u2 itself), a few ulp of |Omega|;
  - the FP32 Omega of the mixed form against its definition (24-bit uniforms,
    Box-Muller) evaluated in FP64 from the oracle's words: FP32 rounding;
  - the Omega an FP64 plan actually used (its workspace after rrsvd_execute)
    equals the exported one bit for bit.
"""
import numpy as np
import pytest

from oracle import philox as P
from paper_1504_00992_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


def _words_gpu(B, counters, key):
    torch = torch_cuda()
    c = np.array(counters, dtype=np.uint64).reshape(-1, 4)
    ct = torch.from_numpy(c.view(np.int64).copy()).to("cuda:0")
    out = torch.zeros_like(ct)
    B.tebd_philox4x64_10(ct.data_ptr(), c.shape[0], key[0], key[1], out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def test_philox_words_bit_exact(lib):
    from paper_1504_00992_gb300 import binding as B
    rng = np.random.default_rng(7)
    special = [(0, 0, 0, 0), (1, 0, 0, 0), (MASK, MASK, MASK, MASK), (123456789, 42, 7, 999),
               (2**63, 1, 2**32 - 1, 2**40 + 3)]
    rand = [tuple(int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)) for _ in range(251)]
    counters = special + rand
    for key in [(0, 0), (2024, 0), (2024, 1), (MASK, MASK), (0xDEADBEEF, 0xFEEDFACE)]:
        got = _words_gpu(B, counters, key)
        for i, c in enumerate(special):
            assert [int(x) for x in got[i]] == list(P.philox4x64_10(c, key)), (c, key)
        c = np.array(counters, dtype=np.uint64)
        exp = np.stack(P.philox4x64_10_array(c[:, 0], c[:, 1], c[:, 2], c[:, 3], key[0], key[1]), axis=1)
        assert np.array_equal(got, exp), key


def _omega_gpu(B, n, l, seed, bond, sweep, chain, precision):
    torch = torch_cuda()
    dt = torch.complex128 if precision == B.TEBD_PREC_FP64 else torch.complex64
    out = torch.zeros((n, l), dtype=dt, device="cuda:0")
    B.rrsvd_sketch_omega(n, l, seed, bond, sweep, chain, precision, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [  # (n, l, seed, bond, sweep, chain)
    (1, 1, 0, 0, 0, 0),
    (80, 26, 99, 0, 0, 3),
    (2000, 120, 2024, 0, 0, 10_000_151),   # the single-bond stress sketch of a bench instance
    (64, 42, 0, 9, 217, 0),                # an XXZ-chain bond late in the run
    (517, 33, 2**63 + 5, 50, 1, 131),
]


@pytest.mark.parametrize("n,l,seed,bond,sweep,chain", CASES)
def test_fp64_omega_matches_oracle(lib, n, l, seed, bond, sweep, chain):
    from paper_1504_00992_gb300 import binding as B
    got = _omega_gpu(B, n, l, seed, bond, sweep, chain, B.TEBD_PREC_FP64)
    exp = P.gaussian_omega(n, l, seed, bond=bond, sweep=sweep, chain=chain)
    assert got.shape == exp.shape
    # |Omega| <= 8.6 (u >= 2^-53); log, sqrt and sin/cos each within 2 ulp,
    # and NumPy's rounding of 2 pi u2 moves its cos/sin by <= 2 pi 2^-53
    bound = 3e-15 * np.abs(exp) + 1e-300
    assert np.all(np.abs(got.real - exp.real) <= bound)
    assert np.all(np.abs(got.imag - exp.imag) <= bound)
    # most entries agree exactly or to one ulp
    if n * l >= 100:
        ulp = np.spacing(np.abs(exp.real))
        assert np.mean(np.abs(got.real - exp.real) <= ulp) > 0.5


def _omega_f32_definition(n, l, seed, bond, sweep, chain):
    idx = np.arange(n * l, dtype=np.uint64)
    z = np.zeros_like(idx)
    w0, w1, _, _ = P.philox4x64_10_array(idx, z + np.uint64(bond), z + np.uint64(sweep), z + np.uint64(chain),
                                         seed & MASK, 0)
    # the 24-bit integer plus one half is rounded to FP32 (to nearest even)
    # before the exact scaling by 2^-24, as the mixed form computes it
    half = np.float32(0.5)
    u1 = ((w0 >> np.uint64(40)).astype(np.float32) + half).astype(np.float64) * 2.0 ** -24
    u2 = ((w1 >> np.uint64(40)).astype(np.float32) + half).astype(np.float64) * 2.0 ** -24
    rho = np.sqrt(-2.0 * np.log(u1))
    return (rho * np.cos(2 * np.pi * u2) + 1j * rho * np.sin(2 * np.pi * u2)).reshape(n, l), rho.reshape(n, l)


@pytest.mark.parametrize("n,l,seed,bond,sweep,chain", CASES)
def test_fp32_omega_of_the_mixed_form(lib, n, l, seed, bond, sweep, chain):
    from paper_1504_00992_gb300 import binding as B
    got = _omega_gpu(B, n, l, seed, bond, sweep, chain, B.TEBD_PREC_TF32).astype(np.complex128)
    exp, rho = _omega_f32_definition(n, l, seed, bond, sweep, chain)
    # logf, sqrtf and sincospif within 2 ulp each, and the FP32 products:
    # a few ulp of FP32 (6e-8) relative to rho
    bound = 6e-7 * rho + 1e-30
    assert np.all(np.abs(got.real - exp.real) <= bound)
    assert np.all(np.abs(got.imag - exp.imag) <= bound)
    # and it is the FP64 Omega to FP32 accuracy except where the 24-bit
    # uniform differs from the 52-bit one by a relative amount that matters
    exp64 = P.gaussian_omega(n, l, seed, bond=bond, sweep=sweep, chain=chain)
    assert np.median(np.abs(got - exp64)) <= 1e-6


def test_plan_workspace_holds_the_exported_omega(lib):
    """The FP64 path's own buffer: each instance's block of an FP64 plan's
    workspace begins with the Omega it sketched with (column-major n x l)."""
    from paper_1504_00992_gb300 import binding as B
    torch = torch_cuda()
    m, n, k, p, q, batch, seed, chain0 = 96, 80, 20, 6, 1, 3, 77, 41
    sig = I.exp_spectrum(n, 6.0)
    th = torch.from_numpy(np.stack([I.synthetic_theta(m, n, sig, seed=t) for t in range(batch)])).to("cuda:0")
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_FP64, seed)
    try:
        kk, ll = B.rrsvd_plan_dims(plan)
        wsb = B.rrsvd_workspace_size(plan)
        per = wsb // batch
        ws = torch.zeros(wsb + 256, dtype=torch.uint8, device="cuda:0")
        base = (ws.data_ptr() + 255) // 256 * 256
        off = base - ws.data_ptr()
        sg = torch.zeros((batch, kk), dtype=torch.float64, device="cuda:0")
        B.rrsvd_execute(plan, th.data_ptr(), chain0, sg.data_ptr(), 0, 0, 0, 0, base, wsb,
                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        raw = ws.cpu().numpy()
        for t in range(batch):
            blk = raw[off + t * per: off + t * per + 16 * n * ll].view(np.complex128)
            used = blk.reshape(ll, n).T   # column-major n x l
            exported = _omega_gpu(B, n, ll, seed, 0, 0, chain0 + t, B.TEBD_PREC_FP64)
            assert np.array_equal(used, exported), t
    finally:
        B.rrsvd_plan_destroy(plan)
