"""Fixed-precision RRSVD (Alg. 1 + the accuracy check of Alg. 2) on the GPU
against the oracle with identical sketch and probes: the same basis widths
(decisions taken far from the threshold), then the FP64 parity tolerances."""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I
from tests.gpu_util import rrsvd_device, truncated

pytestmark = pytest.mark.gpu
SEED = 77


def _oracle_with_margins(A, k, p, q, r, eps, l_max, chain):
    """Oracle run that also checks every MAX is far from eps (so that a
    different rounding order cannot flip a decision)."""
    m, n = A.shape
    kk, l0 = R.sketch_sizes(m, n, k, p)
    Q = R._qr_q(A @ gaussian_omega(n, l0, SEED, chain=chain))
    t = 0
    while Q.shape[1] + r <= l_max:
        Om = R.probe_omega(n, r, t, SEED, chain=chain)
        Br = A @ Om
        mx = np.max(np.linalg.norm(Br - Q @ (Q.conj().T @ Br), axis=0))
        assert abs(mx - eps) > 1e-6 * eps, "test case sits on the decision threshold"
        t += 1
        if mx <= eps:
            break
        Q = R._qr_q(np.concatenate([Q, Br], axis=1))
    return R.rrsvd_fixed_precision(A, gaussian_omega(n, l0, SEED, chain=chain), q, r, eps, l_max, p, SEED,
                                   chain=chain)


@pytest.mark.parametrize("m,n,k,p,q,r,eps,l_max,scale", [
    (160, 120, 8, 4, 1, 6, 1e-5, 100, 6.0),
    (96, 130, 10, 5, 2, 8, 1e-8, 90, 5.0),
    (200, 200, 12, 6, 1, 4, 1e-3, 120, 10.0),
])
def test_checked_plan_matches_oracle(lib, m, n, k, p, q, r, eps, l_max, scale):
    from paper_1504_00992_gb300 import binding as B
    batch = 3
    sig = I.exp_spectrum(min(m, n), scale)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=60 + t) for t in range(batch)])
    plan = B.rrsvd_plan_create_ex(m, n, k, p, q, batch, B.TEBD_PREC_FP64, SEED, r, eps, l_max)
    try:
        res = rrsvd_device(B, plan, theta, chain0=4)
        widths = B.rrsvd_plan_widths(plan, batch)
    finally:
        B.rrsvd_plan_destroy(plan)
    grew = False
    for t in range(batch):
        U, s, Vh, l, kk, resid = _oracle_with_margins(theta[t], k, p, q, r, eps, l_max, 4 + t)
        assert widths[t] == l
        grew |= l > min(k + p, m, n)
        Uk, sk, Vhk = U[:, :kk], s[:kk], Vh[:kk]
        rank = R.kept_rank(sk, kk, 1e-14)
        assert res["rank"][t] == rank
        assert np.abs(res["sigma"][t][:rank] - sk[:rank]).max() <= 1e-10 * sk[0]
        assert np.all(res["sigma"][t][rank:] == 0.0)
        d = truncated(res["U"][t], res["sigma"][t], res["Vh"][t]) - truncated(Uk[:, :rank], sk[:rank], Vhk[:rank])
        assert np.linalg.norm(d) <= 1e-10 * np.linalg.norm(theta[t])
    assert grew
