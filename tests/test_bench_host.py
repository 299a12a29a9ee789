"""Host-side arithmetic of bench.py's roofline object (no GPU): achieved
flops per launch over the mean launch time, the derived ceilings, and DRAM
traffic taken from the committed ncu record only while
that record was captured on the current kernel source."""
import json
import os

import pytest

import bench


def _res(prof):
    return {"prof": prof, "l": 120, "k": 100}


def test_fp32_qr_roofline_arithmetic():
    batch = 152
    # five launches of the FP32 QRs at 4.9 ms each, the projection beside them
    r = bench.roofline(_res({"k_qr_f32": (24.5, 5), "k_oz_proj[project]": (15.1, 1)}), batch)
    flops = (16.0 * bench.M * 120 * 120 - 16.0 * 120 ** 3 / 3) * batch
    assert r["kernel"] == "k_qr_f32" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(flops / 0.0049 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07 / 1e3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_traffic_only_from_a_matching_capture():
    r = bench.roofline(_res({"k_oz_proj[project]": (15.0, 1)}), 152)
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_oz_proj[project]"]
    if rec["src_sha256_16"] == bench._src_hash("oz_proj.cu"):
        assert r["traffic"] == rec["dram_bytes_per_instance"] * 152
        # the capture moved about the algorithmic bytes: theta's six digits
        # (24 bytes per complex element, k padded to 64), Q_f's digits, B^H
        alg = 24 * bench.N_ * 2048 + 24 * 120 * 2048 + bench.N_ * 120 * 16
        assert 0.95 * alg <= rec["dram_bytes_per_instance"] <= 1.1 * alg
    else:
        assert r["traffic"] is None


def test_fp32_qr_traffic_only_at_its_capture_batch():
    """The FP32 QR's DRAM traffic depends on how many instances share L2, so
    its capture (one launch at batch 152) is reported at that batch only."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_qr_f32"]
    assert rec["captured_batch"] == 152 and rec["proportional"] is False
    r152 = bench.roofline(_res({"k_qr_f32": (24.5, 5)}), 152)
    r4 = bench.roofline(_res({"k_qr_f32": (18.7, 5)}), 4)
    assert r4["traffic"] is None
    if rec["src_sha256_16"] == bench._src_hash("qr_blocked.cu"):
        assert r152["traffic"] == rec["dram_bytes_per_instance"] * 152
        # far above the algorithmic bytes (Y read, Q written: 2 x 2000 x 120 x 8 B per instance): the
        # trailing columns of every panel come from DRAM once the batch's working set exceeds L2
        assert rec["dram_bytes_per_instance"] > 10 * 2 * bench.M * 120 * 8
    else:
        assert r152["traffic"] is None


def test_unknown_dominant_kernel_has_no_roofline():
    assert bench.roofline(_res({"k_unlisted": (40.0, 1)}), 152) is None


def test_tensor_core_projection_roofline_uses_the_digit_product_ceiling():
    r = bench.roofline(_res({"k_oz_proj[project]": (10.0, 2), "k_qr": (3.0, 1)}), 152)
    assert r["kernel"] == "k_oz_proj[project]" and r["bound"] == "tensor"
    # 8 m n l flop per instance over the 5 ms launch, against BF16 x 8 / 168
    # (21 digit pairs x 4 real products x 2 flop per complex multiply-add)
    assert abs(r["achieved"] - 8.0 * 2000 * 2000 * 120 * 152 / 5e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - (bench.measured_peaks().get("bf16_tflops_sustained") or 1700.0) * 8 / 168) < 1e-9
    assert set(r["by_kernel"]) == {"k_oz_proj[project]", "k_qr"}
    # with the Cholesky QR of B^H in the step, k_qr (flagged instances only) has no fixed count
    r = bench.roofline(_res({"k_oz_proj[project]": (10.0, 2), "k_qr": (0.01, 1), "k_oz_gemm[cholqr]": (3.0, 5)}), 152)
    assert set(r["by_kernel"]) == {"k_oz_proj[project]", "k_oz_gemm[cholqr]"}


def _bench(args, env_extra=None):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                          cwd=root, env=env, timeout=600)


def test_reference_arm_prints_its_line_on_the_host():
    """bench.py --impl reference: the oracle timed on the host cores on a
    bounded sample of the single-bond stress workload, one JSON line with the
    contract's keys; no GPU involved."""
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "bond updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "2000x2000" in d["config"]["workload"]


def test_reference_arm_other_ranks_exit_without_work():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "1"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""
