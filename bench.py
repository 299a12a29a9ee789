#!/usr/bin/env python
"""Benchmark of the RRSVD bond-update path on one GB300 (or N replicas).

Workload (N=1 line): the single-bond stress case -- complex theta of size
2000 x 2000 (d = 20, chi = 100) with singular values exp(-(k-1)/15), truncated
to rank 100 by RRSVD with p = 20, q = 2 (Section IV; Alg. 1 plus the
projection steps), a batch of instances per step, theta resident in HBM.
Every instance uses its own Philox chain index, so each step is a batch of
new randomized truncations.  A second object reports the whole two-site
update (theta build + gate + RRSVD + rebuild) on the XXZ chain N=20, chi=32.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own batch
(replicas, weak scaling; there is no data exchange between ranks).
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

# the oracle's CPU leg runs LAPACK/BLAS through OpenBLAS on every host core;
# the thread count must be fixed before NumPy loads the library
os.environ.setdefault("OPENBLAS_NUM_THREADS", str(os.cpu_count() or 1))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bond updates/s (theta+RRSVD) vs plain FP64 GPU at <=1e-8 trunc err; % roofline"
M = N_ = 2000
K_MAX, P_OS, Q_PI = 100, 20, 2
POOL = 16            # distinct synthetic theta matrices, tiled over the batch
SEED = 2024
# FP64 peak of GB300 derived from its unit counts and clock: 152 SMs x 2 FP64
# FMA per clock x 2 flop x 2.07 GHz.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# arithmetic of each form of the single-bond measurement
DTYPES = {"fp64": "f64", "tf32": "tf32+f32+bf16x6+df64+f64", "bf16": "bf16+tf32+f32+bf16x6+df64+f64"}
_MIXED_TAIL = ("3xTF32 refinement round, FP32 Householder QRs, FP64-accurate re-orthonormalisation of the last "
               "Q, projection B = Q^H theta on the tensor cores from exact BF16 digit splits (FP64-accurate), "
               "two Cholesky QR passes of B^H and U, V on the same digit-split tensor-core products, "
               "double-float Jacobi SVD")
FORMS = {"fp64": "plain path, every step in FP64",
         "tf32": "TF32 sketch and power rounds before the last, " + _MIXED_TAIL,
         "bf16": "BF16 sketch and power rounds before the last, " + _MIXED_TAIL}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=152)
    ap.add_argument("--precision", default="all", choices=["all", "both", "tf32", "bf16", "fp64"],
                    help="forms of the single-bond measurement (all: fp64, tf32 and bf16; both: fp64 and tf32)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-autotune", action="store_true",
                    help="single-bond plans keep the size rules instead of timing their launch choices first "
                         "(for runs under a profiler, whose replays distort the tuner's timings)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tebd", action="store_true")
    ap.add_argument("--no-spin-boson", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the nvidia-smi clock samples of the timed regions (default: a temp dir)")
    ap.add_argument("--spin-boson-only", action="store_true",
                    help="run only the spin-boson chain measurement (for kernel launch lists)")
    ap.add_argument("--sb-size", default="100,32,4,256,64",
                    help="spin-boson chain: bosons, first and last local dimension, first and last bond cap")
    ap.add_argument("--sb-precision", default="tf32", choices=["tf32", "fp64"],
                    help="form of the spin-boson chain measurement")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_offset(rank):
    """First Philox chain index of a rank's instances: ranks draw disjoint
    ranges (replicas share no data; there is no exchange between them)."""
    return rank * 10_000_000


def max_over_ranks(x, world, device=None):
    """The slowest rank's value (whole-job timing); identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / seconds


def flops_rrsvd(m, n, k, l, q):
    """Algorithmic flops of one RRSVD truncation (complex MAC = 8 flop)."""
    gemm = (2 * q + 2) * 8.0 * m * n * l                      # A Omega, q x (A^H Q, A Q~), A^H Q for B^H
    qr = (2 * q + 1) * (16.0 * m * l * l - 16.0 * l ** 3 / 3)  # range finder QRs (R + explicit Q)
    qr += 16.0 * n * l * l - 16.0 * l ** 3 / 3                 # QR of B^H
    uv = 8.0 * (m + n) * l * k                                 # U = Q J_k, V = Qb W_k
    return gemm, qr, uv


class ClockSampler:
    def __init__(self, index, path):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2][1:5]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def synthetic_pool(count):
    from paper_1504_00992_gb300 import inputs as I
    sig = I.exp_spectrum(N_)
    return np.stack([I.synthetic_theta(M, N_, sig, seed=SEED + t) for t in range(count)]), sig


def cpu_baseline(theta_pool, seconds):
    """The oracle as it stands, timed on this host's cores on a bounded sample."""
    from oracle import rrsvd as R
    from oracle.philox import gaussian_omega
    k, l = R.sketch_sizes(M, N_, K_MAX, P_OS)
    done = 0
    t0 = time.perf_counter()
    while True:
        A = theta_pool[done % len(theta_pool)]
        R.rrsvd_truncate(A, gaussian_omega(N_, l, SEED, chain=done), k, Q_PI)
        done += 1
        el = time.perf_counter() - t0
        if (el >= seconds and done >= 2) or done >= 200:
            break
    return done / el, done, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    pool, _ = synthetic_pool(4)
    from oracle import rrsvd as R
    from oracle.philox import gaussian_omega
    k, l = R.sketch_sizes(M, N_, K_MAX, P_OS)
    per_step = 2
    for w in range(args.warmup):
        R.rrsvd_truncate(pool[w % 4], gaussian_omega(N_, l, SEED, chain=w), k, Q_PI)
    t0 = time.perf_counter()
    for s in range(args.steps):
        for j in range(per_step):
            i = s * per_step + j
            R.rrsvd_truncate(pool[i % 4], gaussian_omega(N_, l, SEED, chain=i), k, Q_PI)
    el = time.perf_counter() - t0
    val = args.steps * per_step / el
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "bond updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "single-bond stress: RRSVD truncation of given 2000x2000 complex128 theta, "
                                   "sigma_k = exp(-(k-1)/15), k=100, p=20, q=2",
                       "per_step_instances": per_step},
            "cpu_baseline": {"value": val, "unit": "bond updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps * per_step} instances (oracle RRSVD, NumPy/LAPACK FP64)"},
            "e2e": {"value": val, "unit": "bond updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_tebd_c1(B, I, torch):
    """Whole two-site updates: XXZ N=20, chi=32, p=10, q=2, 100 Strang steps;
    each sweep replayed from a CUDA graph (value) and launched kernel by kernel
    (no_graph_value)."""
    N, d = 20, 2
    hs = I.xxz_bond_terms(N, d, 1.0, 0.5)

    tuning = []

    def run(use_graph):
        sim = B.Tebd(N, d, 32, 10, 2, 0, stream=torch.cuda.current_stream().cuda_stream, use_graph=use_graph,
                     autotune=1)
        tuning.append(sim.tuning_table())
        sim.set_product_state(I.neel_state(N, d))
        sim.set_gates(0, I.trotter_gates(hs, 0.005))
        sim.set_gates(1, I.trotter_gates(hs, 0.01))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(100):
            sim.step_even(); sim.step_odd(); sim.step_even()
        ws, _ = sim.discarded_weight()
        el = time.perf_counter() - t0
        sim.close()
        return el, ws

    el_g, ws_g = run(1)
    el, ws = run(0)
    updates = 100 * (10 + 9 + 10)
    return {"value": updates / el_g, "unit": "bond updates/s", "seconds": el_g, "updates": updates,
            "no_graph_value": updates / el,
            "workload": "XXZ chain N=20 d=2 J=1 Delta=0.5 dt=0.01, 100 second-order steps, chi_max=32 "
                        "(theta 64x64), p=10, q=2, Neel, seed 0; whole update theta+gate+RRSVD+rebuild; "
                        "the first sweeps capture the graphs inside the timed region",
            "discarded_weight": ws_g, "discarded_weight_no_graph": ws,
            "tuning": [{"parity": par, "bonds": w["bonds"], "m": w["m"], "l": w["l"], "fused": w["fused"],
                        "tiles": w["tiles"], "tune_ms": w["tune_ms"]} for par in (0, 1) for w in tuning[0][par]]}


def measure(B, torch, dev, theta, sig, batch, prec, args, rank, world, local):
    """Device-timed steps of one precision form; inputs resident in HBM."""
    code = {"tf32": B.TEBD_PREC_TF32, "bf16": B.TEBD_PREC_BF16}.get(prec, B.TEBD_PREC_FP64)
    plan = B.rrsvd_plan_create(M, N_, K_MAX, P_OS, Q_PI, batch, code, SEED)
    k, l = B.rrsvd_plan_dims(plan)
    wsb = B.rrsvd_workspace_size(plan)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    sg = torch.zeros((batch, k), dtype=torch.float64, device=dev)
    U = torch.empty((batch, M, k), dtype=torch.complex128, device=dev)
    Vh = torch.empty((batch, k, N_), dtype=torch.complex128, device=dev)
    w = torch.zeros(batch, dtype=torch.float64, device=dev)
    rk = torch.zeros(batch, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    inst0 = replica_offset(rank)

    def step(s):
        B.rrsvd_execute(plan, theta.data_ptr(), inst0 + s * batch, sg.data_ptr(), U.data_ptr(), Vh.data_ptr(),
                        w.data_ptr(), rk.data_ptr(), wsp, wsb, sp)

    # the plan's launch choices, timed on this workload before the warm-up
    if not args.no_autotune:
        B.rrsvd_plan_autotune(plan, theta.data_ptr(), wsp, wsb, sp)
    tuning = B.rrsvd_plan_tuning(plan)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    # accuracy of this launch configuration against the exact spectrum, and
    # the excess Frobenius error of one instance: (||theta - theta_k||_F -
    # ||theta - theta_k(exact)||_F) / ||theta||_F
    sig_err = float(np.abs(sg.cpu().numpy() - sig[:k][None, :]).max())
    u0, s0, v0 = U[0].cpu().numpy(), sg[0].cpu().numpy(), Vh[0].cpu().numpy()
    th0 = theta[0].cpu().numpy()
    excess = (np.linalg.norm(th0 - (u0 * s0) @ v0) - np.sqrt(np.sum(sig[k:] ** 2))) / np.linalg.norm(th0)
    sampler = ClockSampler(local, os.path.join(args.clocks_dir or tempfile.gettempdir(),
                                               f"clocks_{prec}_rank{rank}.csv"))
    B.tebd_profiler_reset()
    B.tebd_profiler_enable(True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        step(args.warmup + s)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    B.tebd_profiler_enable(False)
    prof = B.tebd_profiler_read()
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world, dev)
    B.rrsvd_plan_destroy(plan)
    del ws, U, Vh
    torch.cuda.empty_cache()
    return {"prec": prec, "code": code, "value": whole_job_rate(args.steps * batch, world, ms / 1e3), "ms": ms,
            "prof": prof, "tuning": tuning,
            "clocks": clocks, "sig_err": sig_err, "excess_err": float(excess), "k": k, "l": l}


def e2e_host_buffers(torch, batch, pool):
    """Pinned host buffers of the end-to-end measurement, allocated before any
    device memory (as a serving process would set up its staging once); the
    host theta is written by the CPU from the pool of distinct matrices."""
    k = min(K_MAX, M, N_)
    th_h = torch.empty((batch, M, N_), dtype=torch.complex128, pin_memory=True)
    th_np = th_h.numpy()
    for t in range(batch):
        th_np[t] = pool[t % len(pool)]
    return {"theta": th_h,
            "sigma": torch.empty((batch, k), dtype=torch.float64, pin_memory=True),
            "U": torch.empty((batch, M, k), dtype=torch.complex128, pin_memory=True),
            "Vh": torch.empty((batch, k, N_), dtype=torch.complex128, pin_memory=True),
            "w": torch.empty(batch, dtype=torch.float64, pin_memory=True),
            "rank": torch.empty(batch, dtype=torch.int32, pin_memory=True)}


def e2e_measure(B, torch, theta, batch, code, args, rank, world, host):
    """Through the host-buffer entry point: pinned host theta in, results out,
    copies inside the timed region."""
    th_h, sg_h, U_h, Vh_h, w_h, rk_h = (host[x] for x in ("theta", "sigma", "U", "Vh", "w", "rank"))
    sp = torch.cuda.current_stream().cuda_stream
    inst0 = replica_offset(rank) + 5_000_000
    hp = B.rrsvd_plan_create(M, N_, K_MAX, P_OS, Q_PI, batch, code, SEED)
    # one call first: it allocates the two staging slots and the workspace
    B.rrsvd_execute_host_async(hp, th_h.numpy(), inst0, sg_h.numpy(), U_h.numpy(), Vh_h.numpy(), w_h.numpy(),
                               rk_h.numpy(), sp)
    B.rrsvd_host_wait(hp)
    if world > 1:
        torch.distributed.barrier()
    # back-to-back calls: each step's copy in overlaps the previous step's
    # truncation; every step copies its theta in and its results out
    t0 = time.perf_counter()
    for s in range(args.e2e_steps):
        B.rrsvd_execute_host_async(hp, th_h.numpy(), inst0 + (s + 1) * batch, sg_h.numpy(), U_h.numpy(),
                                   Vh_h.numpy(), w_h.numpy(), rk_h.numpy(), sp)
    B.rrsvd_host_wait(hp)
    el = max_over_ranks(time.perf_counter() - t0, world, theta.device)
    B.rrsvd_plan_destroy(hp)
    bi = th_h.numel() * 16
    bo = sg_h.numel() * 8 + U_h.numel() * 16 + Vh_h.numel() * 16 + w_h.numel() * 8 + rk_h.numel() * 4
    return {"value": whole_job_rate(args.e2e_steps * batch, world, el), "unit": "bond updates/s",
            "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo}


# Double-float (FP32-pair) arithmetic of the projection kernel: per complex
# multiply-add three double-float products by Gauss's rule, 37 FP32
# instructions.  Its ceiling is the FP32 issue rate (152 SMs x 128 lanes x
# 2.07 GHz) / 37 instructions x 8 FP64-equivalent flop.
DF_OPS_PER_CMAC = 37
DF_PEAK_GFLOPS = 152 * 128 * 2.07 / DF_OPS_PER_CMAC * 8


def _src_hash(name):
    import hashlib
    src = open(os.path.join(ROOT, "paper_1504_00992_gb300", "csrc", name), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


# The tensor-core projection forms each complex multiply-add of C = Q_f^H A
# from 21 pairs of BF16 digits (six 8-bit digits per operand, pairs t + u <=
# 7) x 4 real products: 168 BF16 flop per 8 FP64-equivalent flop, so its
# FP64-equivalent ceiling is the measured BF16 rate x 8 / 168.
OZ_BF16_FLOP_PER_CMAC = 21 * 4 * 2
# FP32 CUDA-core peak of GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07


def measured_peaks():
    """Measured GB300 peaks (HBM GB/s, dense BF16 TFLOP/s) from MEASURED_PEAKS.json, if present."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def roofline(res, batch):
    """Roofline object of the dominant kernel class of one measured form:
    algorithmic flops of one launch (per instance x batch) over its mean
    CUDA-event duration, against the derived ceiling of the pipe it runs on;
    traffic = DRAM bytes per launch from the committed ncu capture of that
    kernel (scaled by instances), or null when the source has changed since."""
    prof = res["prof"]
    l, k = res["l"], res["k"]
    dom = max(prof, key=lambda kk: prof[kk][0]) if prof else None
    fp64_peak = FP64_PEAK_GFLOPS / 1e3
    df_peak = DF_PEAK_GFLOPS / 1e3
    fp64_src = "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived)"
    df_src = ("FP32 issue rate 152 SMs x 128 lanes x 2.07 GHz / %d FP32 instructions per double-float complex "
              "multiply-add x 8 flop (derived)" % DF_OPS_PER_CMAC)
    # kernel -> (algorithmic flops per launch, bound, peak, peak source, file holding the kernel)
    pk = measured_peaks()
    bf16 = pk.get("bf16_tflops_sustained") or 1700.0
    oz_peak = bf16 * 8.0 / OZ_BF16_FLOP_PER_CMAC
    oz_src = ("measured sustained BF16 %.0f TFLOP/s (MEASURED_PEAKS.json) x 8 FP64-equivalent flop / %d BF16 flop "
              "per complex multiply-add of the digit products" % (bf16, OZ_BF16_FLOP_PER_CMAC))
    fp32_peak = FP32_PEAK_GFLOPS / 1e3
    fp32_src = "FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (derived)"
    tf32 = bf16 * 1.1 / 2.25
    tf32_src = "measured sustained BF16 %.0f TFLOP/s (MEASURED_PEAKS.json) x nominal TF32:BF16 ratio 1.1:2.25" % bf16
    bf16_src = "measured sustained BF16 %.0f TFLOP/s (MEASURED_PEAKS.json)" % bf16
    # per launch: (algorithmic flops, bound, peak, peak source, file, flops
    # counted in the kernel's own unit when it differs from the algorithmic
    # FP64-equivalent figure)
    per_launch = {
        "k_zgemm[sketch]": (8.0 * M * N_ * l * batch, "alu", fp64_peak, fp64_src, "kernels.cu"),
        # the QR of B^H (n x l) of the mixed form, R and Q
        "k_qr": ((16.0 * N_ * l * l - 16.0 * l ** 3 / 3) * batch, "alu", fp64_peak, fp64_src, "stages.cuh"),
        "k_jacobi": (60.0 * l ** 3 * batch, "alu", fp64_peak, fp64_src, "stages.cuh"),
        # the mixed form's Jacobi in double-float arithmetic: the same
        # algorithmic flops against the double-float ceiling
        "k_jacobi[df]": (60.0 * l ** 3 * batch, "alu", df_peak, df_src, "jacobi_df.cu"),
        # the FP32 Householder QRs of the sketch rounds (R and explicit Q of an
        # m x l complex matrix, m = n here)
        "k_qr_f32": ((16.0 * M * l * l - 16.0 * l ** 3 / 3) * batch, "alu", fp32_peak, fp32_src, "qr_blocked.cu"),
        "k_zgemm[uv]": (8.0 * M * l * k * batch, "alu", fp64_peak, fp64_src, "kernels.cu"),
        "k_oz_proj[project]": (8.0 * M * N_ * l * batch, "tensor", oz_peak, oz_src, "oz_proj.cu"),
        # the Cholesky QR of B^H (Gram matrices, triangular products, B Qb:
        # each n l^2 complex multiply-adds as computed) and U, V, on the same
        # digit-pair kernel
        "k_oz_gemm[cholqr]": (8.0 * N_ * l * l * batch, "tensor", oz_peak, oz_src, "oz_proj.cu"),
        "k_oz_gemm[uv]": (8.0 * M * l * k * batch, "tensor", oz_peak, oz_src, "oz_proj.cu"),
        # E = Q_f^H Q_f - I of the re-orthonormalisation (full l x l product)
        "k_oz_gemm[gram]": (8.0 * M * l * l * batch, "tensor", oz_peak, oz_src, "oz_proj.cu"),
        "k_zgemm_df[cholqr]": (8.0 * N_ * l * l * batch, "alu", df_peak, df_src, "kernels.cu"),
        "k_zgemm_df[uv]": (8.0 * M * l * k * batch, "alu", df_peak, df_src, "kernels.cu"),
        # the sketch products (one complex m x n x l product per launch; the
        # 3xTF32 launch does three TF32 products for the same algorithmic flops)
        "k_tc_gemm[tf32]": (8.0 * M * N_ * l * batch, "tensor", tf32, tf32_src, "tc_gemm.cuh"),
        "k_tc_gemm[3xtf32]": (8.0 * M * N_ * l * batch, "tensor", tf32, tf32_src, "tc_gemm.cuh"),
        "k_tc_gemm[bf16]": (8.0 * M * N_ * l * batch, "tensor", bf16, bf16_src, "tc_gemm.cuh"),
    }
    if dom not in per_launch:
        return None
    fl, bound, peak, psrc, srcfile = per_launch[dom]
    avg_ms = prof[dom][0] / prof[dom][1]
    achieved = fl / (avg_ms / 1e3) / 1e12
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        rec = json.load(open(tp)).get(dom)
        # counters taken on this exact kernel source; a capture at another batch
        # only where the record states that the traffic grows in proportion
        # (per-instance data above L2 either way), not where the batch decides
        # what stays in L2
        if rec and rec.get("src_sha256_16") == _src_hash(srcfile) and (
                rec.get("captured_batch") == batch or rec.get("proportional", False)):
            traffic = rec["dram_bytes_per_instance"] * batch
    out = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic, "peak_source": psrc}
    # every kernel class of the step against its own ceiling (same units)
    out["by_kernel"] = {}
    cholqr = "k_oz_gemm[cholqr]" in prof or "k_zgemm_df[cholqr]" in prof
    for kk, (flk, bd, pkk, _, _) in per_launch.items():
        # with the Cholesky QR of B^H, k_qr factors only the instances it
        # flags as ill-conditioned (usually none): no fixed flop count
        if kk == "k_qr" and cholqr:
            continue
        if kk in prof and prof[kk][1] > 0:
            a = flk / (prof[kk][0] / prof[kk][1] / 1e3) / 1e12
            out["by_kernel"][kk] = {"bound": bd, "achieved": a, "peak": pkk, "frac": a / pkk,
                                    "ms_per_step": prof[kk][0] / max(1, prof[kk][1]) * prof[kk][1]}
    return out


def run_rrsvd_checked(B, torch, dev, theta, sig, batch, steps=2, warm=1):
    """Fixed-precision RRSVD (Alg. 2 accuracy check) on the single-bond stress
    matrices: start at k=40, p=10 (l=50), rounds of r=10 probes until the
    largest probe residual is below eps=1e-3 (the paper's setting; sigma_1=1)
    or l reaches 200; q=2 power rounds on the grown basis; FP64.  Timed like
    the headline (device buffers, CUDA events)."""
    kk, p, q, r, eps, lmax = 40, 10, 2, 10, 1e-3, 200
    plan = B.rrsvd_plan_create_ex(M, N_, kk, p, q, batch, B.TEBD_PREC_FP64, SEED, r, eps, lmax)
    kcap, lcap = B.rrsvd_plan_dims(plan)
    wsb = B.rrsvd_workspace_size(plan)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device=dev)
    wsp = (ws.data_ptr() + 255) // 256 * 256
    sg = torch.zeros((batch, kcap), dtype=torch.float64, device=dev)
    rk = torch.zeros(batch, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(s):
        B.rrsvd_execute(plan, theta.data_ptr(), 7_000_000 + s * batch, sg.data_ptr(), 0, 0, 0, rk.data_ptr(), wsp,
                        wsb, stream.cuda_stream)

    for s in range(warm):
        step(s)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        step(warm + s)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    widths = B.rrsvd_plan_widths(plan, batch)
    ranks = rk.cpu().numpy()
    s_h = sg.cpu().numpy()
    err = max(float(np.abs(s_h[t, :ranks[t]] - sig[:ranks[t]]).max()) for t in range(batch))
    B.rrsvd_plan_destroy(plan)
    del ws
    torch.cuda.empty_cache()
    return {"value": steps * batch / (ms / 1e3), "unit": "truncations/s", "ms_per_step": ms / steps,
            "widths_l": {"min": int(min(widths)), "max": int(max(widths)), "mean": float(np.mean(widths))},
            "kept_rank_mean": float(np.mean(ranks)), "max_abs_sigma_err_vs_exact": err,
            "workload": "single-bond stress 2000x2000, Alg. 2 accuracy check: k0=40, p=10, r=10 probes per round, "
                        "eps=1e-3, l_max=200, q=2, FP64, %d instances per step" % batch}


def _canonical_fixture(spec):
    """Worker of the fixture pool: a seeded random MPS of one chain at its
    bond caps, in Vidal canonical form (host input generation, untimed)."""
    from paper_1504_00992_gb300 import inputs as I
    N, d, chi, seed = spec
    return I.random_canonical_mps([d] * N, [chi] * (N - 1), seed)


def canonical_fixtures(specs, seed0=1000):
    """Canonical random MPS of every chain (seed seed0 + c), built by a pool
    of spawned processes on the host cores (one BLAS thread each)."""
    import multiprocessing as mp
    saved = os.environ.get("OPENBLAS_NUM_THREADS")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
            return pool.map(_canonical_fixture, [(N, d, chi, seed0 + c) for c, (N, d, chi, _) in enumerate(specs)],
                            chunksize=2)
    finally:
        if saved is None:
            del os.environ["OPENBLAS_NUM_THREADS"]
        else:
            os.environ["OPENBLAS_NUM_THREADS"] = saved


def run_tebd_many(B, I, torch, n_chains=256, steps=2, warm=1, unbatched_chains=16, fixtures=None, fix_seconds=0.0):
    """Many-chain batch: the chains of I.many_chain_specs (seed 0), dt = 0.01,
    p = 10, q = 1, every chain starting from a canonical random MPS at its
    bond caps (the regime of the configuration's 100 steps), all bonds of a
    parity of all chains per launch sequence, sweeps replayed from CUDA
    graphs, 16 GB wave budget, launch choices autotuned; in the mixed form
    (TF32, as the configuration asks) and in the FP64 form, the latter also
    against the first chains stepped one handle at a time.  A second mixed
    run from Neel states (bonds far below their caps) is reported beside."""
    specs = I.many_chain_specs(n_chains, 0)
    dt, p, q = 0.01, 10, 1
    t0 = time.perf_counter()
    fix = fixtures if fixtures is not None else canonical_fixtures(specs)
    if fixtures is None:
        fix_seconds = time.perf_counter() - t0
    chi_lo = min(min(len(l) for l in lam) for _, lam in fix)
    chi_hi = max(max(len(l) for l in lam) for _, lam in fix)

    def setup(sim_set_state, sim_set_gates, subset, canonical=True):
        for c, (N, d, chi, delta) in enumerate(subset):
            hs = I.xxz_bond_terms(N, d, 1.0, delta)
            if canonical:
                sim_set_state(c, *fix[c])
            else:
                sim_set_state(c, I.neel_state(N, d))
            sim_set_gates(c, 0, I.trotter_gates(hs, dt / 2))
            sim_set_gates(c, 1, I.trotter_gates(hs, dt))

    def updates(subset, steps_):
        return steps_ * sum(2 * ((N - 1 + 1) // 2) + (N - 1) // 2 for N, _, _, _ in subset)

    chains = [(N, [d] * N, [chi] * (N - 1)) for N, d, chi, _ in specs]
    tables = {}

    def batched(prec, canonical=True, steps_=steps, warm_=warm):
        sim = B.MultiTebd(chains, p, q, 0, use_graph=1, workspace_budget=16 << 30, precision=prec, autotune=1)
        tables[prec] = sim.tuning_table()
        if canonical:
            setup(sim.set_mps, sim.set_gates, specs)
        else:
            setup(sim.set_product_state, sim.set_gates, specs, canonical=False)
        for _ in range(warm_):
            sim.step_even(); sim.step_odd(); sim.step_even()
        sim.discarded_weight(0)   # synchronises
        t0 = time.perf_counter()
        for _ in range(steps_):
            sim.step_even(); sim.step_odd(); sim.step_even()
        sim.discarded_weight(0)
        el = time.perf_counter() - t0
        info = sim.workspace_info()
        _, _, sz = I.spin_ops(specs[0][1])
        probe = [sim.expect(0, k, sz).real for k in range(specs[0][0])]
        sim.close()
        return updates(specs, steps_) / el, info, np.array(probe)

    mixed, info_m, probe_m = batched(B.TEBD_PREC_TF32)
    fp64, info, probe_d = batched(B.TEBD_PREC_FP64, steps_=1)
    neel, _, _ = batched(B.TEBD_PREC_TF32, canonical=False, steps_=2, warm_=2)
    # unbatched: the first chains, each in its own handle, stepped in turn
    sub = specs[:unbatched_chains]
    sims = []
    for N, d, chi, delta in sub:
        s1 = B.Tebd(N, d, chi, p, q, 0)
        sims.append(s1)
    setup(lambda c, g, lam: sims[c].set_mps(g, lam), lambda c, par, g: sims[c].set_gates(par, g), sub)
    for s1 in sims:
        s1.step_even(); s1.step_odd(); s1.step_even()
    sims[0].discarded_weight()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s1 in sims:
        s1.step_even(); s1.step_odd(); s1.step_even()
    for s1 in sims:
        s1.discarded_weight()
    el2 = time.perf_counter() - t0
    for s1 in sims:
        s1.close()
    unbatched = updates(sub, 1) / el2
    # the same first chains in the batched FP64 form, for the like-for-like ratio
    return {"value": mixed, "unit": "bond updates/s", "precision": "tf32 (mixed form)", "chains": n_chains,
            "steps_timed": steps, "arena_bytes": info_m[0], "waves": [info_m[1], info_m[2]],
            "start": "canonical random MPS at every bond cap (inputs.random_canonical_mps, seed 1000 + chain), "
                     "built on the host in %.1f s" % fix_seconds,
            "chi_range_at_start": [chi_lo, chi_hi],
            "fp64_value": fp64, "fp64_steps_timed": 1, "fp64_arena_bytes": info[0], "fp64_waves": [info[1], info[2]],
            "speedup_mixed_vs_fp64": mixed / fp64,
            "chain0_max_abs_sz_diff_mixed_vs_fp64": float(np.abs(probe_m - probe_d[:len(probe_m)]).max())
            if len(probe_d) else None,
            "neel_start_value": neel,
            "unbatched_fp64_value": unbatched, "unbatched_chains": unbatched_chains,
            "speedup_fp64_batched_vs_unbatched": fp64 / unbatched,
            "tuning": {"tf32": [{"parity": par, "bonds": w["bonds"], "m": w["m"], "n": w["n"], "l": w["l"],
                                 "mixed": w["mixed"], "tune_ms": w["tune_ms"]}
                                for par in (0, 1) for w in tables[B.TEBD_PREC_TF32][par]],
                       "fp64": [{"parity": par, "bonds": w["bonds"], "m": w["m"], "n": w["n"], "l": w["l"],
                                 "fused": w["fused"], "tiles": w["tiles"], "tune_ms": w["tune_ms"]}
                                for par in (0, 1) for w in tables[B.TEBD_PREC_FP64][par]]},
            "workload": "256 XXZ chains, N~U{16..128}, d in {2,3,4}, chi_max in {32,64,128}, Delta~U[0,1], "
                        "dt=0.01, p=10, q=1, from canonical random MPS at the caps; graphs + 16 GB wave budget, "
                        "autotuned; %d warm-up step(s), %d timed (FP64: 1)" % (warm, steps)}


def run_tebd_spin_boson(B, I, torch, steps=1, warm=1, size=(100, 32, 4, 256, 64), precision="tf32"):
    """Spin-boson chain in star-to-chain form: a spin and 100 bosonic sites
    whose local dimension falls from 32 to 4, couplings 1/(1+n), per-bond
    caps falling from 256 to 64, from a canonical random MPS at the caps
    (seed 0), dt = 0.05, p = 10, q = 2; the TF32 form (TF32 sketches with FP32
    QRs, FP64-accurate tail; the configuration's precision) or the plain FP64
    form, all bonds of a parity per launch sequence replayed from CUDA graphs,
    40 GB wave budget, launch choices autotuned per wave shape at creation.
    One second-order step = even, odd, even sweep."""
    dims, caps = I.spin_boson_sizes(*size)
    g0, lam0 = I.random_canonical_mps(dims, caps, 0)
    hs = I.spin_boson_bond_terms(dims)
    dt, p, q = 0.05, 10, 2
    code = B.TEBD_PREC_TF32 if precision == "tf32" else B.TEBD_PREC_FP64
    t_tune = time.perf_counter()
    sim = B.Tebd(len(dims), 2, 0, p, q, 3, d_site=dims, chi_bond=caps, precision=code, use_graph=1,
                 workspace_budget=40 << 30, autotune=1)
    t_tune = time.perf_counter() - t_tune
    table = sim.tuning_table()
    sim.set_mps(g0, lam0)
    sim.set_gates(0, I.trotter_gates(hs, dt / 2))
    sim.set_gates(1, I.trotter_gates(hs, dt))
    for _ in range(warm):
        sim.step_even(); sim.step_odd(); sim.step_even()
    sim.discarded_weight()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step_even(); sim.step_odd(); sim.step_even()
    w = sim.discarded_weight()
    el = time.perf_counter() - t0
    nb = len(dims) - 1
    upd = steps * (2 * ((nb + 1) // 2) + nb // 2)
    info = sim.workspace_info() if hasattr(sim, "workspace_info") else None
    sim.close()
    return {"value": upd / el, "unit": "bond updates/s", "seconds_per_step": el / steps, "steps_timed": steps,
            "precision": "tf32 (mixed form)" if precision == "tf32" else "fp64 (plain)",
            "discarded_weight": float(w[0]), "workspace": info,
            "creation_and_tuning_seconds": t_tune,
            "tuning": [{"parity": par, "bonds": wv["bonds"], "m": wv["m"], "n": wv["n"], "l": wv["l"],
                        "mixed": wv["mixed"], "fused": wv["fused"], "tune_ms": wv["tune_ms"]}
                       for par in (0, 1) for wv in table[par]],
            "workload": "spin-boson chain: spin + %d bosons, d %d -> %d, chi caps %d -> %d, dt=0.05, p=10, q=2, "
                        "canonical random MPS at the caps (seed 0); graphs, 40 GB wave budget, autotuned, after %d "
                        "warm-up step(s)" % (tuple(size) + (warm,))}


def run_tebd_gradient(B, I, torch):
    """Differentiable form: gradient of <sigma^z_19>(t=1) of the transverse-field
    Ising chain N=40, chi=64, dt=0.02, 50 steps with respect to its 39
    couplings, by the recorded forward + reverse pass, against the cost of the
    same gradient by central differences of the plain forward (78 runs)."""
    from paper_1504_00992_gb300.autograd import tfim_observable
    N, hf, dt, steps, chi, p, q, seed, site = 40, 1.0, 0.02, 50, 64, 10, 2, 0, 19
    J0 = np.random.default_rng(0).uniform(0.5, 1.5, N - 1)
    hs = I.tfim_bond_terms(J0, hf)

    def forward(J):
        sim = B.Tebd(N, 2, chi, p, q, seed)
        sim.set_product_state([np.array([1.0, 0.0]) for _ in range(N)])
        h2 = I.tfim_bond_terms(J, hf)
        sim.set_gates(0, I.trotter_gates(h2, dt / 2))
        sim.set_gates(1, I.trotter_gates(h2, dt))
        for _ in range(steps):
            sim.step_even(); sim.step_odd(); sim.step_even()
        v = sim.expect(site, I.pauli()[2]).real
        sim.close()
        return v

    forward(J0)   # warm-up
    t0 = time.perf_counter()
    forward(J0)
    t_fwd = time.perf_counter() - t0
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        J = torch.tensor(J0, requires_grad=True)
        tfim_observable(J, N, hf, dt, steps, chi, p, q, seed, site).backward()
    t_grad = (time.perf_counter() - t0) / reps
    updates = steps * (20 + 19 + 20)
    return {"value": 1.0 / t_grad, "unit": "gradients/s", "seconds_per_gradient": t_grad,
            "bond_updates_per_s": 2 * updates / t_grad, "forward_seconds": t_fwd,
            "central_difference_seconds": 2 * (N - 1) * t_fwd,
            "speedup_vs_central_differences": 2 * (N - 1) * t_fwd / t_grad,
            "workload": "transverse-field Ising N=40 d=2 chi=64 dt=0.02, 50 steps, d<sigma^z_19>/dJ_b (39 couplings), "
                        "J~U[0.5,1.5] seed 0; recorded forward + reverse pass (tebd_backward)"}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1504_00992_gb300 import binding as B
    from paper_1504_00992_gb300 import inputs as I
    if args.spin_boson_only:
        if rank == 0:
            size = tuple(int(x) for x in args.sb_size.split(","))
            print(json.dumps({"tebd_spin_boson": run_tebd_spin_boson(B, I, torch, size=size,
                                                                     precision=args.sb_precision)}), flush=True)
        return

    batch = args.batch
    # host fixtures of the many-chain batch, built by spawned workers before
    # any device work of the measurements
    t_fix = time.perf_counter()
    fixtures = canonical_fixtures(I.many_chain_specs(256, 0)) if not args.no_tebd else None
    t_fix = time.perf_counter() - t_fix
    pool, sig = synthetic_pool(POOL)
    host = e2e_host_buffers(torch, batch, pool) if args.e2e_steps > 0 else None
    theta = torch.empty((batch, M, N_), dtype=torch.complex128, device=dev)
    pool_dev = torch.from_numpy(pool).to(dev)
    for t in range(batch):
        theta[t].copy_(pool_dev[t % POOL])
    del pool_dev
    precs = {"all": ["fp64", "tf32", "bf16"], "both": ["fp64", "tf32"]}.get(args.precision, [args.precision])
    results = {p: measure(B, torch, dev, theta, sig, batch, p, args, rank, world, local) for p in precs}
    # headline: the fastest form that meets the 1e-8 truncation-accuracy bar
    ok = [r for r in results.values() if r["sig_err"] <= 1e-8 and r["excess_err"] <= 1e-8]
    head = max(ok or list(results.values()), key=lambda r: r["value"])
    e2e = e2e_measure(B, torch, theta, batch, head["code"], args, rank, world, host) if args.e2e_steps > 0 else None
    roof = roofline(head, batch)
    prof = head["prof"]
    shares = {kk: {"ms": v[0], "launches": v[1]} for kk, v in sorted(prof.items(), key=lambda x: -x[1][0])}
    launches = sum(v[1] for v in prof.values())
    k, l = head["k"], head["l"]
    gemm_f, qr_f, uv_f = flops_rrsvd(M, N_, k, l, Q_PI)

    tebd = many = grad = checked = sb = None
    if not args.no_tebd:
        checked = run_rrsvd_checked(B, torch, dev, theta, sig, batch)
        tebd = run_tebd_c1(B, I, torch)
        many = run_tebd_many(B, I, torch, fixtures=fixtures, fix_seconds=t_fix)
        grad = run_tebd_gradient(B, I, torch)
        if not args.no_spin_boson:
            del theta
            torch.cuda.empty_cache()
            sb = run_tebd_spin_boson(B, I, torch)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        val, done, el = cpu_baseline(pool, args.cpu_seconds)
        cpu = {"value": val, "unit": "bond updates/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} instances of the same workload in {el:.1f} s (oracle RRSVD, NumPy/LAPACK FP64, "
                         f"OPENBLAS_NUM_THREADS={os.environ['OPENBLAS_NUM_THREADS']}, nproc={os.cpu_count()})"}
    if rank == 0:
        forms = {p: {"value": r["value"], "ms_per_step": r["ms"] / args.steps,
                     "max_abs_sigma_err_vs_exact": r["sig_err"], "excess_frobenius_err": r["excess_err"],
                     "tuning": r["tuning"]}
                 for p, r in results.items()}
        line = {"metric": METRIC, "value": head["value"], "unit": "bond updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES[head["prec"]], "data": "synthetic",
                "config": {"workload": "single-bond stress: RRSVD truncation of given 2000x2000 complex128 theta, "
                                       "sigma_k = exp(-(k-1)/15), k=100, p=20, q=2 (theta given directly)",
                           "precision": head["prec"] + " (" + FORMS[head["prec"]] + ")",
                           "batch_per_gpu": batch, "distinct_theta": POOL, "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2: %.1f GB of theta read per step" % (batch * M * N_ * 16 / 1e9),
                           "max_abs_sigma_err_vs_exact": head["sig_err"],
                           "excess_frobenius_err": head["excess_err"],
                           # the metric's anchor: the plain FP64 GPU path on the same workload
                           "fp64_value": results["fp64"]["value"] if "fp64" in results else None,
                           "speedup_vs_plain_fp64": (head["value"] / results["fp64"]["value"])
                           if "fp64" in results else None},
                "forms": forms,
                "speedup_vs_plain_fp64": (head["value"] / results["fp64"]["value"]) if "fp64" in results else None,
                "roofline": roof, "kernel_time_ms": shares, "gpu_launches": launches,
                "flops_per_update": {"gemm": gemm_f, "qr": qr_f, "uv": uv_f},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": head["clocks"], "tebd_c1": tebd,
                "tebd_many_chains": many, "tebd_gradient": grad, "rrsvd_accuracy_check": checked,
                "tebd_spin_boson": sb}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
