"""The mixed-precision RRSVD form (TEBD_PREC_TF32): TF32 tensor-core sketch
and power iterations with FP32 Householder QRs, 3xTF32 refinement of the last
power round, an FP64-accurate re-orthonormalisation of the last Q (FP64
Householder when l > 512), double-float projection and FP64 small SVD.

Its stated tolerances: with Omega rounded to TF32 and the sketch in TF32 the
mixed form is a different (equally valid) randomized truncation than the FP64
oracle, so it is held to the FP64 method's accuracy, not to its rounding
(exact spectra are known by construction):
  * max_i |s_i(mixed) - s_i(exact)| <= max_i |s_i(oracle) - s_i(exact)| + 1e-8 s_1;
  * excess error (||A - A_k||_F - ||A - A_k(exact)||_F) / ||A||_F no more
    than 1e-8 above the oracle's;
  * where the FP64 method meets the 1e-8 bar, the mixed form meets it too;
  * the returned factors are orthonormal to 1e-11 (re-orthonormalised last Q,
    FP64 Jacobi, double-float U = Q J_k and V = Qb W_k).

TEBD_PREC_BF16 runs the products before the refinement round in BF16: the
subspace the refinement round starts from is perturbed at 2^-9, which moves
the method's own approximation error by a few percent where that error is
large (slowly decaying spectra, q = 1), so its first two bars read
err_m <= 1.05 err_o + 1e-8 s_1 (and likewise for the excess error); the
others are unchanged.
"""
import numpy as np
import pytest

from oracle import rrsvd as R
from oracle.philox import gaussian_omega
from paper_1504_00992_gb300 import inputs as I
from tests.gpu_util import repeat_on_device, rrsvd_device, truncated

pytestmark = pytest.mark.gpu
SEED = 4321


@pytest.mark.parametrize("m,n,k,p,q,scale", [
    (400, 400, 60, 20, 2, 12.0),   # the single-bond stress spectrum shape, reduced
    (300, 200, 40, 10, 1, 8.0),    # ragged: no size is a multiple of 128 / 32
    (130, 70, 20, 6, 0, 4.0),      # q = 0: the sketch itself is the refinement pass
    (96, 96, 24, 8, 2, 5.0),
    (400, 360, 120, 20, 1, 30.0),  # l = 140: the widest correction held in shared memory
    (3700, 200, 20, 10, 1, 6.0),   # Y too tall for the blocked FP32 QR: unblocked fallback
    (1200, 400, 140, 20, 1, 12.0), # l = 160: correction read through L1 (tiled Loewdin and fold)
    (3700, 300, 30, 10, 1, 6.0),   # Y too tall for the blocked FP32 QR, l = 40: FP32 QR over many CTAs
])
@pytest.mark.parametrize("form", ["tf32", "bf16"])
def test_mixed_form_meets_its_tolerances(lib, m, n, k, p, q, scale, form):
    from paper_1504_00992_gb300 import binding as B
    batch = 3
    sig = I.exp_spectrum(min(m, n), scale)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=200 + t) for t in range(batch)])
    prec = B.TEBD_PREC_BF16 if form == "bf16" else B.TEBD_PREC_TF32
    rel = 1.05 if form == "bf16" else 1.0
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, prec, SEED)
    try:
        res = rrsvd_device(B, plan, theta, chain0=2)
    finally:
        B.rrsvd_plan_destroy(plan)
    kk, l = R.sketch_sizes(m, n, k, p)
    opt = np.sqrt(np.sum(sig[kk:] ** 2))
    for t in range(batch):
        A = theta[t]
        nA = np.linalg.norm(A)
        s = res["sigma"][t]
        assert res["rank"][t] == kk
        Uk, sk, Vhk, w = R.rrsvd_truncate(A, gaussian_omega(n, l, SEED, chain=2 + t), kk, q)
        err_o = np.abs(sk - sig[:kk]).max()
        err_m = np.abs(s - sig[:kk]).max()
        assert err_m <= rel * err_o + 1e-8 * sig[0]
        if err_o <= 1e-8:
            assert err_m <= 1e-8
        exc_o = (np.linalg.norm(A - truncated(Uk, sk, Vhk)) - opt) / nA
        exc_m = (np.linalg.norm(A - truncated(res["U"][t], s, res["Vh"][t])) - opt) / nA
        assert exc_m <= rel * max(exc_o, 0.0) + 1e-8
        U = res["U"][t]
        assert np.abs(U.conj().T @ U - np.eye(kk)).max() < 1e-11
        V = res["Vh"][t]
        assert np.abs(V @ V.conj().T - np.eye(kk)).max() < 1e-11
        assert abs(res["w"][t] - w) <= 1e-8 + abs(w - (np.sum(sig[kk:] ** 2) / np.sum(sig ** 2)))


@pytest.mark.parametrize("batch,form", [(2, "tf32"), (152, "tf32"), (152, "bf16")])
def test_mixed_form_full_size_sampled(lib, batch, form):
    """2000 x 2000, k=100, p=20, q=2 (the single-bond stress workload): kept
    singular values within 1e-8 of the exact spectrum and excess truncation
    error within 1e-8, on the first and last instance.  The batch of 152 (two
    distinct matrices repeated, each instance with its own Omega) is the
    launch configuration the benchmark times (one-CTA QR of B^H and Jacobi
    SVD); two instances take the many-CTA QR and the cluster Jacobi."""
    from paper_1504_00992_gb300 import binding as B
    m = n = 2000
    sig = I.exp_spectrum(n)
    base = [I.synthetic_theta(m, n, sig, seed=t) for t in range(2)]
    prec = B.TEBD_PREC_BF16 if form == "bf16" else B.TEBD_PREC_TF32
    plan = B.rrsvd_plan_create(m, n, 100, 20, 2, batch, prec, SEED)
    try:
        res = rrsvd_device(B, plan, repeat_on_device(base, batch))
    finally:
        B.rrsvd_plan_destroy(plan)
    for t in (0, batch - 1):
        th = base[t % 2]
        assert np.abs(res["sigma"][t] - sig[:100]).max() <= 1e-8
        opt = np.sqrt(np.sum(sig[100:] ** 2))
        err = np.linalg.norm(th - truncated(res["U"][t], res["sigma"][t], res["Vh"][t]))
        assert (err - opt) / np.linalg.norm(th) <= 1e-8


@pytest.mark.parametrize("m,n,k,p,rank", [
    (3700, 300, 30, 10, 12),   # FP32 QR of Y over a cluster panel: columns 13..40 collapse to rounding noise
    (2000, 160, 24, 8, 5),     # blocked FP32 QR in shared memory
])
def test_mixed_form_rank_deficient(lib, m, n, k, p, rank):
    """Exact rank below the sketch width: the FP32 QRs meet columns at the
    rounding level (the tiny-column rules keep every reflector unitary), the
    basis stays orthonormal, the singular values are the exact ones to
    1e-8 s_1 and the rest fall to the noise level.  The rank-r reconstruction
    carries the form's first-order range error (the refinement pass resolves
    the sketched range to FP32 level, ~1e-7 relative; singular values feel it
    only to second order): it is held to 3e-6 relative."""
    from paper_1504_00992_gb300 import binding as B
    rng = np.random.default_rng(17)
    batch = 2
    theta = np.stack([(rng.standard_normal((m, rank)) + 1j * rng.standard_normal((m, rank))) @
                      (rng.standard_normal((rank, n)) + 1j * rng.standard_normal((rank, n))) for _ in range(batch)])
    plan = B.rrsvd_plan_create(m, n, k, p, 1, batch, B.TEBD_PREC_TF32, SEED)
    try:
        res = rrsvd_device(B, plan, theta)
    finally:
        B.rrsvd_plan_destroy(plan)
    for t in range(batch):
        s_ref = np.linalg.svd(theta[t], compute_uv=False)
        s = res["sigma"][t]
        assert np.all(np.isfinite(s)) and res["rank"][t] >= rank
        assert np.abs(s[:rank] - s_ref[:rank]).max() <= 1e-8 * s_ref[0]
        assert np.all(s[rank:] <= 1e-6 * s_ref[0])
        r = rank
        rec = truncated(res["U"][t][:, :r], s[:r], res["Vh"][t][:r])
        assert np.linalg.norm(rec - theta[t]) <= 3e-6 * np.linalg.norm(theta[t])
        U = res["U"][t][:, :r]
        assert np.abs(U.conj().T @ U - np.eye(r)).max() < 1e-11
        V = res["Vh"][t][:r]
        assert np.abs(V @ V.conj().T - np.eye(r)).max() < 1e-11


@pytest.mark.parametrize("m,n,k,scale_rows", [
    (120, 200, 120, False),   # l = m: the basis is a whole unitary of C^m
    (150, 300, 150, True),    # rows scaled over 2^-40 .. 2^40 (the digits' block scales)
    (500, 600, 500, False),   # l = 500: a 500-deep projection, 16 exact k blocks
])
def test_mixed_projection_is_fp64_accurate(lib, m, n, k, scale_rows):
    """When the sketch width reaches m the basis Q is a whole unitary matrix
    (re-orthonormalised FP64-accurately), so B = Q^H A carries all of A and
    the mixed form's singular values and reconstruction are limited by its
    FP64-accurate steps alone: the projection on the tensor cores (48-bit
    BF16 digits of both operands, exact FP32 sums per 32-deep k block), the
    basis and the FP64 small SVD.  Held to 1e-11 relative (normwise), where
    an FP32-level projection would miss by 1e-7 and the digit product with
    a single inexact group for levels 4+ by 3e-10."""
    from paper_1504_00992_gb300 import binding as B
    batch = 2
    rng = np.random.default_rng(31)
    r = min(m, n)
    sig = np.exp(-np.arange(r) / (r / 12.0))
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=500 + t) for t in range(batch)])
    if scale_rows:
        theta = theta * (2.0 ** rng.integers(-40, 41, size=(1, m, 1)))
    plan = B.rrsvd_plan_create(m, n, k, 10, 1, batch, B.TEBD_PREC_TF32, SEED)
    try:
        res = rrsvd_device(B, plan, theta)
    finally:
        B.rrsvd_plan_destroy(plan)
    kk = min(k, m, n)
    for t in range(batch):
        s_ref = np.linalg.svd(theta[t], compute_uv=False)
        s = res["sigma"][t]
        r_t = res["rank"][t]
        # values below the 1e-14 cutoff are dropped (scaled rows give such
        # values); at 1e-11 s_1 accuracy a value within 1e-11 s_1 of the
        # cutoff may fall on either side, so the kept rank lies between the
        # counts of values clearly above and not clearly below it
        cut, tol = 1e-14 * s_ref[0], 1e-11 * s_ref[0]
        r_lo, r_hi = np.sum(s_ref[:kk] > cut + tol), np.sum(s_ref[:kk] > cut - tol)
        assert r_lo <= r_t <= r_hi
        if not scale_rows:
            assert r_t == kk
        assert np.abs(s[:r_t] - s_ref[:r_t]).max() <= tol
        rec = truncated(res["U"][t], s, res["Vh"][t])
        assert np.linalg.norm(rec - theta[t]) <= 1e-11 * np.linalg.norm(theta[t])


def test_mixed_qr_of_bh_cholesky_and_householder_in_one_batch(lib):
    """The QR of B^H (Section IV, step ii) takes Cholesky QR (two passes,
    double-float Grams, FP64 Cholesky) for well-conditioned instances and the
    Householder QR for the others, chosen per instance in the same launch:
    instances 0 and 2 have kappa(B) ~ e^(39/10) ~ 50, instances 1 and 3 a
    spectrum falling to 1e-13.  All meet the form's tolerances against the
    exact spectrum, and the returned factors are orthonormal to 1e-11."""
    from paper_1504_00992_gb300 import binding as B
    m, n, k, p, q = 600, 500, 40, 10, 2
    mild = np.exp(-np.arange(n) / 10.0)
    steep = np.exp(-np.arange(n) / 1.5)
    sigs = [mild, steep, mild, steep]
    theta = np.stack([I.synthetic_theta(m, n, s, seed=700 + t) for t, s in enumerate(sigs)])
    plan = B.rrsvd_plan_create(m, n, k, p, q, 4, B.TEBD_PREC_TF32, SEED)
    try:
        res = rrsvd_device(B, plan, theta)
    finally:
        B.rrsvd_plan_destroy(plan)
    kk, l = R.sketch_sizes(m, n, k, p)
    for t in range(4):
        sig = sigs[t]
        r = res["rank"][t]
        Uk, sk, Vhk, w = R.rrsvd_truncate(theta[t], gaussian_omega(n, l, SEED, chain=t), kk, q)
        err_o = np.abs(sk - sig[:len(sk)]).max()
        s = res["sigma"][t][:r]
        assert abs(r - len(sk)) <= 1
        rr = min(r, len(sk))
        assert np.abs(s[:rr] - sig[:rr]).max() <= err_o + 1e-8 * sig[0]
        U = res["U"][t][:, :r]
        assert np.abs(U.conj().T @ U - np.eye(r)).max() < 1e-11
        V = res["Vh"][t][:r]
        assert np.abs(V @ V.conj().T - np.eye(r)).max() < 1e-11


def test_products_after_the_projection_on_either_unit(lib):
    """The Cholesky QR of B^H and U = Q J_k, V = Qb W_k run on the tensor
    cores from exact BF16 digit splits (48-bit digits, the projection's
    kernel) or as double-float CUDA-core GEMMs; both are FP64-accurate, so a
    plan forced to either gives the same truncation to rounding (1e-12 s_1),
    and both meet the form's tolerances.  A choice out of range is refused."""
    from paper_1504_00992_gb300 import binding as B
    m, n, k, p, q, batch = 600, 520, 60, 20, 1, 3
    sig = I.exp_spectrum(min(m, n), 10.0)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=700 + t) for t in range(batch)])
    out = {}
    for unit in (1, 2):
        plan = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_TF32, SEED)
        try:
            B.rrsvd_plan_set_tuning(plan, {"products": unit})
            assert B.rrsvd_plan_tuning(plan)["products"] == unit
            with pytest.raises(B.TebdError):
                B.rrsvd_plan_set_tuning(plan, {"products": 3})
            out[unit] = rrsvd_device(B, plan, theta, chain0=5)
        finally:
            B.rrsvd_plan_destroy(plan)
    kk, l = R.sketch_sizes(m, n, k, p)
    for t in range(batch):
        a, b = out[1], out[2]
        assert np.abs(a["sigma"][t] - b["sigma"][t]).max() <= 1e-12 * sig[0]
        ra = truncated(a["U"][t], a["sigma"][t], a["Vh"][t])
        rb = truncated(b["U"][t], b["sigma"][t], b["Vh"][t])
        assert np.linalg.norm(ra - rb) <= 1e-11 * np.linalg.norm(theta[t])
        for r in (a, b):
            U, V = r["U"][t], r["Vh"][t]
            assert np.abs(U.conj().T @ U - np.eye(kk)).max() < 1e-11
            assert np.abs(V @ V.conj().T - np.eye(kk)).max() < 1e-11
            _, sk, _, _ = R.rrsvd_truncate(theta[t], gaussian_omega(n, l, SEED, chain=5 + t), kk, q)
            assert np.abs(r["sigma"][t] - sig[:kk]).max() <= np.abs(sk - sig[:kk]).max() + 1e-8 * sig[0]


@pytest.mark.parametrize("m,n,k,p", [(600, 520, 60, 20), (300, 260, 230, 20)])
def test_double_float_jacobi_agrees_with_fp64(lib, m, n, k, p):
    """The small SVD of the mixed form (one-sided Jacobi on Rb^H) in
    double-float arithmetic against the FP64 kernel on the same B: singular
    values within 1e-12 s_1 (2^-48 arithmetic over a few hundred rotations per
    column), both factor sets orthonormal to 1e-11, and the same truncation.
    The second case keeps l = 250 columns, the spectrum falling to 1e-11."""
    from paper_1504_00992_gb300 import binding as B
    batch = 3
    sig = I.exp_spectrum(min(m, n), 10.0)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=900 + t) for t in range(batch)])
    out = {}
    for jac in (1, 3):
        plan = B.rrsvd_plan_create(m, n, k, p, 1, batch, B.TEBD_PREC_TF32, SEED)
        try:
            B.rrsvd_plan_set_tuning(plan, {"jacobi": jac})
            out[jac] = rrsvd_device(B, plan, theta, chain0=11)
        finally:
            B.rrsvd_plan_destroy(plan)
    kk, _ = R.sketch_sizes(m, n, k, p)
    for t in range(batch):
        a, b = out[3], out[1]
        assert a["rank"][t] == b["rank"][t]
        r = a["rank"][t]
        assert np.abs(a["sigma"][t][:r] - b["sigma"][t][:r]).max() <= 1e-12 * sig[0]
        for res in (a, b):
            U, V = res["U"][t][:, :r], res["Vh"][t][:r]
            assert np.abs(U.conj().T @ U - np.eye(r)).max() < 1e-11
            assert np.abs(V @ V.conj().T - np.eye(r)).max() < 1e-11
        ra = truncated(a["U"][t], a["sigma"][t], a["Vh"][t])
        rb = truncated(b["U"][t], b["sigma"][t], b["Vh"][t])
        assert np.linalg.norm(ra - rb) <= 1e-11 * np.linalg.norm(theta[t])


@pytest.mark.parametrize("form", ["tf32", "bf16"])
def test_host_path_sub_batches_equal_device_path(lib, form):
    """rrsvd_execute_host runs a mixed-form batch of 16 or more as four
    sub-batches on streams of their own (copies overlapping kernels); with the
    launch choices of the whole batch its results equal rrsvd_execute's bit
    for bit, here with an uneven split (18 = 5 + 5 + 5 + 3)."""
    from paper_1504_00992_gb300 import binding as B
    m, n, k, p, q, batch = 300, 260, 40, 10, 1, 18
    sig = I.exp_spectrum(min(m, n), 8.0)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=40 + t) for t in range(batch)])
    prec = B.TEBD_PREC_BF16 if form == "bf16" else B.TEBD_PREC_TF32
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, prec, SEED)
    try:
        dev = rrsvd_device(B, plan, theta, chain0=3)
        sg = np.zeros((batch, k))
        U = np.zeros((batch, m, k), dtype=np.complex128)
        Vh = np.zeros((batch, k, n), dtype=np.complex128)
        w = np.zeros(batch)
        rk = np.zeros(batch, dtype=np.int32)
        B.rrsvd_execute_host(plan, theta, 3, sg, U, Vh, w, rk)
        # again: the plan's streams and staging are reused
        sg2 = np.zeros((batch, k))
        B.rrsvd_execute_host(plan, theta, 3, sg2)
    finally:
        B.rrsvd_plan_destroy(plan)
    assert np.array_equal(sg, dev["sigma"]) and np.array_equal(U, dev["U"]) and np.array_equal(Vh, dev["Vh"])
    assert np.array_equal(w, dev["w"]) and np.array_equal(rk, dev["rank"]) and np.array_equal(sg2, sg)


def test_async_host_calls_overlap_and_equal_device_path(lib):
    """rrsvd_execute_host_async: three calls in flight on one plan (two
    staging slots used in turn, the third call waiting for the first slot),
    each with its own chain0 and output arrays, equal the device path bit for
    bit after rrsvd_host_wait; the wait reports nothing when nothing failed
    and returns at once when nothing is pending."""
    from paper_1504_00992_gb300 import binding as B
    m, n, k, p, q, batch = 200, 180, 30, 8, 1, 5
    sig = I.exp_spectrum(min(m, n), 6.0)
    theta = np.stack([I.synthetic_theta(m, n, sig, seed=70 + t) for t in range(batch)])
    plan = B.rrsvd_plan_create(m, n, k, p, q, batch, B.TEBD_PREC_TF32, SEED)
    try:
        outs = []
        for call in range(3):
            o = {"sigma": np.zeros((batch, k)), "U": np.zeros((batch, m, k), dtype=np.complex128),
                 "Vh": np.zeros((batch, k, n), dtype=np.complex128), "w": np.zeros(batch),
                 "rank": np.zeros(batch, dtype=np.int32)}
            B.rrsvd_execute_host_async(plan, theta, 100 * call, o["sigma"], o["U"], o["Vh"], o["w"], o["rank"])
            outs.append(o)
        B.rrsvd_host_wait(plan)
        B.rrsvd_host_wait(plan)
        for call in range(3):
            dev = rrsvd_device(B, plan, theta, chain0=100 * call)
            for key in ("sigma", "U", "Vh", "w", "rank"):
                assert np.array_equal(outs[call][key], dev[key]), (call, key)
        # a zero theta is reported by the wait
        B.rrsvd_execute_host_async(plan, np.zeros_like(theta), 0, np.zeros((batch, k)))
        with pytest.raises(B.TebdError) as ei:
            B.rrsvd_host_wait(plan)
        assert ei.value.code == B.TEBD_ENUMERIC
    finally:
        B.rrsvd_plan_destroy(plan)
