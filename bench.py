"""Benchmark: Reduced Basis Decomposition of the 8192 x 8192 image-like FP64 matrix on GB300.

One step = one complete rbd_compress (Algorithm 1 to tolerance: the initial norm pass, then per
basis the orthogonalisation and the fused pass over X) followed by the out-of-sample map of 64
vectors (rbd_project).  Metric: GB/s of X streamed by the compression, i.e.
(passes over X) * m * n * 8 bytes / step time, passes = d + 1 (the initial pass and one per
basis), reported against the measured HBM bandwidth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun) runs N independent replicas, one per GPU ("replicas only": one matrix does not
shard in this build), value = total bytes of all ranks / max over ranks of the timed region.
--impl reference times the FP64 CPU oracle (the plain implementation of Algorithm 1) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = 8192
D_MAX = 512
TOL = 1e-3
TOL_MODE = "fro_rel"
N_OOS = 64
METRIC = "RBD compress GB/s of X to tol (HBM % of peak); mixed/batched vs FP64 speedup"
UNIT = "GB/s"
WORKLOAD = ("image-like 8192x8192 field (200 Gaussian bumps + 20 sinusoids, uint8-quantised, /255) "
            "in FP64; d_max=512, tol=1e-3 relative Frobenius, start column 0; + projection of 64 "
            "out-of-sample vectors")
PASS_SOURCES = ["paper_1503_05947_gb300/csrc/rbd_defer.cu", "paper_1503_05947_gb300/csrc/rbd_loop.cuh",
                "paper_1503_05947_gb300/csrc/rbd_tile.cuh", "paper_1503_05947_gb300/csrc/rbd_device.cuh",
                "paper_1503_05947_gb300/csrc/rbd_work.h"]


def _code_only(src: str) -> str:
    """C/C++/CUDA source without its comments and blank lines (string literals here hold no
    comment markers), so that a change of wording does not read as a change of the kernel."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())


def pass_kernel_hash() -> str:
    """Hash of the loop kernel's code (comments excluded) that the committed traffic figure was
    measured on."""
    h = hashlib.sha256()
    for p in PASS_SOURCES:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def ncu_traffic() -> dict | None:
    """DRAM bytes per launch of the persistent loop kernel on this workload, from the committed
    ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "defer_kernel_image8192_f64_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != pass_kernel_hash():
        return None
    return d


def make_inputs(device):
    import torch

    import gen
    q = gen.image_like_u8(M, seed=1)
    qt = torch.from_numpy(np.ascontiguousarray(q.T))  # (n, m) row-major == column-major X
    X = (qt.to(device=device, dtype=torch.float64) / 255.0).t()
    V = gen.out_of_sample(M, N_OOS, seed=11)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).to(device).t()
    return q, X, Vd


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier_max(world: int, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample(X64: np.ndarray, steps: int, threads: int = 0) -> tuple[float, float]:
    """Time the FP64 CPU oracle on the first `steps` bases of Algorithm 1 for this matrix
    (threads > 0: its OpenMP build on that many threads).  Returns (seconds, bytes of X the
    sample represents = steps * m * n * 8)."""
    import oracle
    oracle.build(omp=threads > 0)
    t0 = time.perf_counter()
    r = oracle.compress(X64, 0.0, steps, threads=threads)
    dt = time.perf_counter() - t0
    assert r["d"] == steps
    return dt, steps * X64.shape[0] * X64.shape[1] * 8.0


def host_cpu() -> dict:
    """The host's CPU model and core count (the CPU baseline's label)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    return {"model": model or "unknown", "cores": os.cpu_count() or 1}


def omp_available() -> bool:
    import oracle
    try:
        oracle.build(omp=True)
        return True
    except Exception:  # noqa: BLE001
        return False


def run_reference(args, world, rank):
    """Reference arm: the oracle on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return
    import gen
    q = gen.image_like_u8(M, seed=1)
    X64 = gen.u8_to_unit_f64(q)
    steps_per_sample = args.ref_steps
    cpu = host_cpu()
    threads = cpu["cores"] if omp_available() else 0
    for _ in range(args.warmup):
        oracle_sample(X64, steps_per_sample, threads)
    times, nbytes = [], 0.0
    for _ in range(args.steps):
        dt, b = oracle_sample(X64, steps_per_sample, threads)
        times.append(dt)
        nbytes += b
    total = sum(times)
    value = nbytes / total / 1e9
    sample = (f"first {steps_per_sample} bases of Algorithm 1 on the full 8192x8192 matrix per step "
              f"(oracle: explicit FP64 residual, MGS twice), "
              + (f"OpenMP build on {threads} threads" if threads else "single thread") + f", {cpu['model']}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "m": M, "n": N, "d_max": D_MAX, "tol": TOL,
                                            "tol_mode": TOL_MODE, "sample_bases": steps_per_sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(threads, 1), "kind": "oracle", "sample": sample,
                             "cpu_model": cpu["model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch

    import paper_1503_05947_gb300 as rbd
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rbd.load()
    q, X, V = make_inputs(dev)
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(rbd.workspace_bytes(M, N, D_MAX), dtype=torch.uint8, device=dev)

    def step():
        r = rbd.compress(X, TOL, D_MAX, tol_mode=TOL_MODE, workspace=ws)
        C = rbd.project(r.Y, V)
        return r, C

    for _ in range(args.warmup):
        r, _ = step()
    torch.cuda.synchronize(dev)

    rbd.set_profiling(True)
    pass_ms, pass_n, orth_ms, init_ms = 0.0, 0, 0.0, 0.0
    loop_ms, loop_n, loop_passes = 0.0, 0, 0
    passes_total = 0
    launches = 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            r, C = step()
            pf = rbd.get_profile()
            pass_ms += pf["pass_ms"]
            pass_n += pf["pass_launches"]
            orth_ms += pf["orth_ms"]
            if pf["loop_kernel"]:
                loop_ms += pf["loop_ms"]
                loop_n += pf["loop_launches"]
                loop_passes += pf["pass_launches"]
            init_ms += pf["init_ms"]
            passes_total += r.d + 1
            launches += r.launches + 2  # + the projection: row-split partial products and their sum
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    rbd.set_profiling(False)
    t_local = e0.elapsed_time(e1) / 1e3
    t = barrier_max(world, t_local)
    bytes_per_pass = M * N * 8.0
    value = world * passes_total * bytes_per_pass / t / 1e9

    e2e = None
    if not args.no_e2e:
        # end to end through the host-buffer entry point (pinned host X, copies inside the region)
        Xh = torch.from_numpy(np.ascontiguousarray(q.T)).to(torch.float64).div_(255.0).pin_memory().t()
        outs = {"Y": torch.empty((D_MAX, M), dtype=torch.float64).pin_memory().t(),
                "T": torch.empty((N, D_MAX), dtype=torch.float64).pin_memory().t(),
                "pivots": torch.empty(D_MAX, dtype=torch.int64).pin_memory(),
                "err": torch.empty(D_MAX, dtype=torch.float64).pin_memory(),
                "nu": torch.empty(D_MAX, dtype=torch.float64).pin_memory()}
        rh = rbd.compress_host(Xh, TOL, D_MAX, tol_mode=TOL_MODE, device=dev, out=outs)  # warm-up
        e2e_steps = max(1, min(args.steps, 5))
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_passes = 0
        for _ in range(e2e_steps):
            rh = rbd.compress_host(Xh, TOL, D_MAX, tol_mode=TOL_MODE, device=dev, out=outs)
            e2e_passes += rh.d + 1
        t_e2e = barrier_max(world, time.perf_counter() - t0)
        e2e = {"value": world * e2e_passes * bytes_per_pass / t_e2e / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": M * N * 8, "d2h_bytes_per_step": M * rh.d * 8 + rh.d * N * 8 + rh.d * 8 * 3,
               "steps": e2e_steps}

    peaks = measured_peaks()
    tr = ncu_traffic()
    if loop_n:
        # the persistent kernel runs the whole greedy loop: per launch it streams X once per basis
        kern_s = loop_ms / loop_n / 1e3
        bytes_per_launch = bytes_per_pass * loop_passes / loop_n
        kname = ("rbd::loop_kernel<0, 0> (persistent greedy loop, four grid barriers per basis)"
                 if os.environ.get("RBD_LOOP_CLASSIC", "0") not in ("", "0") else
                 "rbd::defer_kernel<0> (persistent greedy loop, two grid barriers per basis)")
    else:
        kern_s = pass_ms / max(pass_n, 1) / 1e3
        bytes_per_launch = bytes_per_pass
        kname = "rbd::pass_kernel<2> (fused pass, FP64 data as float-float planes)"
    achieved = bytes_per_launch / kern_s / 1e9 if kern_s > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
            "traffic": tr["dram_bytes_per_launch"] if tr else None,
            "kernel": kname, "peak_source": peaks["source"], "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": kern_s * 1e3}

    forms = {}
    if rank == 0 and not args.no_forms:
        forms["decode"] = decode_form(r, dev)
        forms["weighted"] = weighted_form(X, ws, dev, (loop_ms / loop_passes) if loop_passes else None)
        forms["precision"] = precision_forms(dev, peaks)
        forms["batched"] = batched_forms(dev)
        forms["paper_5001"] = paper_5001_form(dev)
        forms["small"] = small_form(dev)
        forms["grad"] = grad_form(dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        X64 = gen_x64(q)
        hc = host_cpu()
        dt1, b1 = oracle_sample(X64, args.cpu_steps)
        one = {"value": b1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
               "sample": f"first {args.cpu_steps} bases of Algorithm 1 on the full matrix, single thread ({dt1:.1f} s)"}
        if omp_available():
            # the whole step on all cores: every basis of the benchmarked compression (d_max of them)
            nth = hc["cores"]
            dt, b = oracle_sample(X64, args.d_max, nth)
            cpu = {"value": b / dt / 1e9, "unit": UNIT, "cores": nth, "kind": "oracle",
                   "sample": f"the whole step: all {args.d_max} bases of Algorithm 1 on the full matrix, OpenMP "
                             f"build on {nth} threads ({dt:.1f} s)", "cpu_model": hc["model"], "single_thread": one}
        else:
            cpu = dict(one, kind="oracle", cpu_model=hc["model"])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "m": M, "n": N, "d_max": D_MAX, "tol": TOL, "tol_mode": TOL_MODE,
                           "bases": r.d, "passes_per_step": r.d + 1, "stop_reason": r.stop_reason,
                           "fro_rel_residual": r.fro_last / r.x_fro, "oos_vectors": N_OOS,
                           "l2": "inputs larger than L2 (X 512 MiB vs 129 MB L2)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": launches,
                "forms": forms,
                "breakdown_ms_per_step": {"loop_kernel": loop_ms / args.steps, "stepwise_pass": pass_ms / args.steps,
                                          "stepwise_orth": orth_ms / args.steps, "init": init_ms / args.steps},
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def decode_form(r, dev) -> dict:
    """Uncompress (Section 3.1): the full 8192 x 8192 approximation Y T from the benchmark's
    compression (d = 512), CUDA events around rbd_reconstruct after one warm-up call."""
    import torch

    import paper_1503_05947_gb300 as rbd
    out = rbd.reconstruct(r.Y, r.T)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    rbd.reconstruct(r.Y, r.T, out=out)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    m, d = r.Y.shape
    n = r.T.shape[1]
    del out
    fma = m * n * d / (ms * 1e-3)
    # ceiling: every float-float product-accumulate (ff_mac2) is 12 FP32 instructions, and the SMs
    # issue 128 FP32 lanes per clock: 128 / 12 products per SM and clock at the sampled SM clock
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    ceil_fma = sm_count * 2.07e9 * 128 / 12
    return {"workload": f"Xr = Y T, {m} x {d} times {d} x {n} (the benchmark's compression)", "ms": ms,
            "fma_per_s": fma, "out_gbs": m * n * 8 / (ms * 1e-3) / 1e9,
            "arith": "float-float products on the FP32 pipes (FP64-grade)",
            "roofline": {"bound": "alu", "achieved": fma, "peak": ceil_fma, "unit": "FMA/s", "frac": fma / ceil_fma,
                         "peak_source": f"{sm_count} SMs x 2070 MHz x 128 FP32 lanes / 12 FP32 instructions "
                                        "per float-float product (ff_mac2)"}}


def weighted_form(X, ws, dev, plain_pass_ms) -> dict:
    """The diagonal A-norm form (Section 3.2): the benchmark's matrix and tolerance with row
    weights (gen.row_weights, seed 7: a smooth bump up to 10x over a third of the rows times a
    0.5-2x jitter), CUDA events around one rbd_compress_weighted call after a warm-up call, and
    the persistent kernel's time per pass against the unweighted run's."""
    import torch

    import gen
    import paper_1503_05947_gb300 as rbd
    w = torch.as_tensor(gen.row_weights(M, seed=7), device=dev)
    rbd.compress(X, TOL, D_MAX, tol_mode=TOL_MODE, workspace=ws, weights=w)
    rbd.set_profiling(True)
    stream = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    r = rbd.compress(X, TOL, D_MAX, tol_mode=TOL_MODE, workspace=ws, weights=w)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    pf = rbd.get_profile()
    rbd.set_profiling(False)
    ms = ev0.elapsed_time(ev1)
    pass_ms = pf["loop_ms"] / max(r.d, 1)
    out = {"workload": f"A = diag(w) on the benchmark matrix ({M}x{N} FP64, d_max {D_MAX}, {TOL_MODE} {TOL})",
           "ms": ms, "bases": r.d, "stop_reason": r.stop_reason, "fro_rel_residual_A": r.fro_last / r.x_fro,
           "gbs": r.d * M * N * 8 / (pf["loop_ms"] * 1e-3) / 1e9, "pass_ms": pass_ms}
    if plain_pass_ms:
        out["pass_time_vs_unweighted"] = pass_ms / plain_pass_ms
    return out


PREC_M, PREC_N, PREC_DMAX = 65536, 16384, 256
PREC_WORKLOAD = ("parametric snapshots 65536x16384, X_ij = 1/sqrt((s_i - mu1_j)^2 + mu2_j^2), s uniform on [0, 1], "
                 "mu1 ~ U[-1,-0.01], mu2 ~ U[0.01,1] (seed 2); d_max 256, relative Frobenius tolerance")


def precision_forms(dev, peaks: dict) -> dict:
    """The precision form on the parametric snapshots 65536 x 16384, stored in FP64, FP32 (with
    FP64-grade float-float dot products, or with FP32 accumulation per tile) and BF16:

    * to_tolerance: one whole rbd_compress call per form to a relative Frobenius tolerance (1e-6;
      1e-2 for BF16, whose storage alone carries ~2^-9), CUDA events, inputs resident; bases,
      relative reconstruction error against the FP64 matrix;
    * equal_d: every form at the FP64 run's number of bases d (tol 0, d_max d): time, time per
      pass over X, algorithmic GB/s (m n bytes-per-element per pass) and its fraction of the
      measured HBM peak, speedup over FP64, relative error against the FP64 matrix;
    * passes_256: the stated d_max 256 (the stored values of FP32 and BF16 keep X's numerical rank
      above the rank floor, so tol 0 runs all 256 passes; FP64 in the no-tolerance mode, which
      takes the four-barrier kernel): time per pass, GB/s, fraction of peak;
    * vs_oracle: on a 16384 x 4096 instance of the same family, the FP64 oracle at 1e-6 and each
      form at the oracle's d: the forms' relative errors against the oracle's own."""
    import torch

    import gen
    import oracle
    import paper_1503_05947_gb300 as rbd
    hbm_gbs = peaks["hbm_gbs"]
    X64 = gen.parametric_snapshots_torch(PREC_M, PREC_N, device=dev)
    x64n = X64.norm().item()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)

    def rel_err(Xref, r, xn):
        err2 = 0.0
        for j0 in range(0, Xref.shape[1], 2048):
            blk = Xref[:, j0:j0 + 2048] - r.Y @ r.T[:, j0:j0 + 2048]
            err2 += float(blk.norm()) ** 2
        return (err2 ** 0.5) / xn

    def timed(X, tol, dmax, mode, acc):
        rbd.compress(X, tol, dmax, tol_mode=mode, accumulate=acc)
        rbd.set_profiling(True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        r = rbd.compress(X, tol, dmax, tol_mode=mode, accumulate=acc)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        pf = rbd.get_profile()
        rbd.set_profiling(False)
        return r, ev0.elapsed_time(ev1), pf

    def stats(X, r, ms, pf, esize):
        pass_us = 1e3 * pf["loop_ms"] / max(r.d, 1) if pf["loop_kernel"] else 1e3 * pf["pass_ms"] / max(r.d, 1)
        gbs = PREC_M * PREC_N * esize / (pass_us * 1e-6) / 1e9
        return {"bases": r.d, "stop_reason": r.stop_reason, "ms": ms, "pass_us": pass_us, "pass_gbs": gbs,
                "pass_frac_of_hbm_peak": gbs / hbm_gbs}

    X32 = X64.t().contiguous().to(torch.float32).t()
    Xb = X64.t().contiguous().to(torch.bfloat16).t()
    forms = {"f64": (X64, "exact", 8, 1e-6), "f32": (X32, "exact", 4, 1e-6), "f32_acc32": (X32, "fp32", 4, 1e-6),
             "bf16": (Xb, "exact", 2, 1e-2)}
    out = {"workload": PREC_WORKLOAD, "timing": "CUDA events, inputs resident in HBM, after one warm-up call",
           "hbm_peak": {"gbs": hbm_gbs, "source": peaks.get("source", "measured")},
           "to_tolerance": {}, "equal_d": {}, "passes_256": {}}
    for k, (X, acc, es, tol) in forms.items():
        r, ms, pf = timed(X, tol, PREC_DMAX, "fro_rel", acc)
        out["to_tolerance"][k] = dict(stats(X, r, ms, pf, es), tol=tol, rel_err_vs_f64=rel_err(X64, r, x64n))
    d_eq = out["to_tolerance"]["f64"]["bases"]
    for k, (X, acc, es, tol) in forms.items():
        r, ms, pf = timed(X, 0.0, d_eq, "maxcol_abs", acc)
        out["equal_d"][k] = dict(stats(X, r, ms, pf, es), rel_err_vs_f64=rel_err(X64, r, x64n))
    for k in out["equal_d"]:
        out["equal_d"][k]["speedup_vs_f64"] = out["equal_d"]["f64"]["ms"] / out["equal_d"][k]["ms"]
        out["to_tolerance"][k]["speedup_vs_f64"] = out["to_tolerance"]["f64"]["ms"] / out["to_tolerance"][k]["ms"]
    for k, (X, acc, es, tol) in forms.items():
        mode = "none" if k == "f64" else "maxcol_abs"
        r, ms, pf = timed(X, 0.0, PREC_DMAX, mode, acc)
        out["passes_256"][k] = dict(stats(X, r, ms, pf, es),
                                    kernel="four-barrier (no-tolerance mode)" if k == "f64" else "two-barrier")
    del X32, Xb, X64
    torch.cuda.empty_cache()
    # against the FP64 oracle's own error at the same d, on a smaller instance of the family
    ms_, ns_ = 16384, 4096
    Xo = gen.parametric_snapshots(ms_, ns_, seed=2)
    nth = host_cpu()["cores"] if omp_available() else 0
    t0 = time.perf_counter()
    ref = oracle.compress(Xo, 1e-6, 64, mode="fro_rel", threads=nth)
    t_or = time.perf_counter() - t0
    e_or = np.linalg.norm(Xo - ref["Y"] @ ref["T"]) / np.linalg.norm(Xo)
    Xs64 = torch.from_numpy(np.ascontiguousarray(Xo.T)).to(dev).t()
    vs = {"instance": f"parametric snapshots {ms_}x{ns_} (seed 2)", "oracle_bases": ref["d"],
          "oracle_rel_err": e_or, "oracle_s": t_or, "oracle_threads": max(nth, 1)}
    for k, (dt, acc) in {"f64": (torch.float64, "exact"), "f32": (torch.float32, "exact"),
                         "f32_acc32": (torch.float32, "fp32"), "bf16": (torch.bfloat16, "exact")}.items():
        Xd = Xs64 if dt == torch.float64 else Xs64.t().contiguous().to(dt).t()
        r = rbd.compress(Xd, 0.0, ref["d"], accumulate=acc)
        e = rel_err(Xs64, r, float(Xs64.norm()))
        vs[k] = {"bases": r.d, "rel_err": e, "rel_err_over_oracle": e / e_or, "rel_err_minus_oracle": e - e_or}
    out["vs_oracle"] = vs
    return out


def small_form(dev) -> dict:
    """The small FP64 workload (1024 x 512 = U diag(s) V' with s_i = 2^(-i/4), noise sd 1e-5, d_max
    64, tol 1e-6 on the max column residual): one rbd_compress on the device (CUDA events, median
    of 10 calls, X resident; X fits in L2, so the rate is an effective one), the FP64 oracle on one
    host core and on all of them, and the largest deviations from the oracle."""
    import statistics

    import torch

    import gen
    import oracle
    import paper_1503_05947_gb300 as rbd
    Xn = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)
    m, n = Xn.shape
    X = torch.from_numpy(np.ascontiguousarray(Xn.T)).to(dev).t()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for i in range(12):
        torch.cuda.synchronize(dev)
        ev0.record()
        r = rbd.compress(X, 1e-6, 64)
        ev1.record()
        torch.cuda.synchronize(dev)
        if i >= 2:
            ts.append(ev0.elapsed_time(ev1))
    ms = statistics.median(ts)
    t0 = time.perf_counter()
    ref = oracle.compress(Xn, 1e-6, 64)
    t1 = time.perf_counter() - t0
    nth = host_cpu()["cores"] if omp_available() else 0
    t0 = time.perf_counter()
    oracle.compress(Xn, 1e-6, 64, threads=nth)
    tall = time.perf_counter() - t0
    scale = np.linalg.norm(Xn, axis=0)
    Y = r.Y.cpu().numpy()
    T = r.T.cpu().numpy()
    return {"workload": "1024x512 U diag(2^(-i/4)) V' + N(0, 1e-10) noise (sd 1e-5), FP64, d_max 64, tol 1e-6 max column",
            "bases": r.d, "ms": ms, "effective_gbs": (r.d + 1) * m * n * 8 / (ms * 1e-3) / 1e9,
            "note": "X (4 MiB) is L2-resident: an effective rate, not an HBM one",
            "pivots_equal_oracle": bool(np.array_equal(r.pivots.cpu().numpy(), ref["pivots"])),
            "max_dY": float(np.linalg.norm(Y - ref["Y"], axis=0).max()),
            "max_dT_rel": float((np.abs(T - ref["T"]) / scale[None, :]).max()),
            "oracle_s_1core": t1, "oracle_s_all_cores": tall, "oracle_threads": max(nth, 1)}


def grad_form(dev) -> dict:
    """The differentiation workload: 64 FP32 matrices 1024 x 512 (decay 0.1), d = 32, 256
    out-of-sample vectors each.  Device time (CUDA events) of the 64 forward compressions and of
    the 64 adjoints (loss and gradient), as a batch (one batched compression launch, one
    rbd_grad_batched call) and one instance at a time (rbd_compress, rbd_grad); the oracle's adjoint
    on two instances (one host core), scaled to 64, and the largest deviation from it."""
    import torch

    import gen
    import oracle
    import paper_1503_05947_gb300 as rbd
    inst = []
    for i in range(64):
        X = gen.lowrank_haar(1024, 512, np.exp(-0.1 * np.arange(512)), seed=1000 + i).astype(np.float32)
        Xo = gen.out_of_sample(1024, 256, seed=2000 + i).astype(np.float32)
        inst.append((torch.from_numpy(np.ascontiguousarray(X.T)).to(dev).t(),
                     torch.from_numpy(np.ascontiguousarray(Xo.T)).to(dev).t()))
    # one instance at a time
    for X, Xo in inst[:2]:
        r = rbd.compress(X, 0.0, 32)
        rbd.grad(X, r.Y, r.T, r.pivots, Xo)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    e[0].record()
    fw = [rbd.compress(X, 0.0, 32) for X, _ in inst]
    e[1].record()
    outs = [rbd.grad(X, r.Y, r.T, r.pivots, Xo) for (X, Xo), r in zip(inst, fw)]
    e[2].record()
    torch.cuda.synchronize(dev)
    one = (e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]))
    # as a batch
    plan = rbd.BatchPlan([{"X": X, "tol": 0.0, "d_max": 32} for X, _ in inst])
    plan.run()
    res = plan.results()
    gi = []
    for i, ((X, Xo), r) in enumerate(zip(inst, res)):
        c = plan.compressed(i, r)
        gi.append({"X": X, "Y": c.Y, "T": c.T, "pivots": c.pivots, "Xo": Xo})
    rbd.grad_batched(gi)
    torch.cuda.synchronize(dev)
    fb, ab = [], []
    for _ in range(3):
        e[0].record()
        plan.run()
        e[1].record()
        bouts = rbd.grad_batched(gi)
        e[2].record()
        torch.cuda.synchronize(dev)
        fb.append(e[0].elapsed_time(e[1]))
        ab.append(e[1].elapsed_time(e[2]))
    same_piv = all(torch.equal(g["pivots"], r.pivots) for g, r in zip(gi, fw))
    worst, worst_b, t_or = 0.0, 0.0, 0.0
    for i in (0, 37):
        X, Xo = inst[i]
        r = fw[i]
        t0 = time.perf_counter()
        Gref, _ = oracle.grad(X.double().cpu().numpy(), r.Y.cpu().numpy(), r.T.cpu().numpy(), r.pivots.cpu().numpy(),
                              Xo.double().cpu().numpy())
        t_or += time.perf_counter() - t0
        worst = max(worst, float(np.abs(outs[i][0].cpu().numpy() - Gref).max() / np.abs(Gref).max()))
        g = gi[i]
        Gb, _ = oracle.grad(X.double().cpu().numpy(), g["Y"].cpu().numpy(), g["T"].cpu().numpy(),
                            g["pivots"].cpu().numpy(), Xo.double().cpu().numpy())
        worst_b = max(worst_b, float(np.abs(bouts[i][0].cpu().numpy() - Gb).max() / np.abs(Gb).max()))
    del plan
    return {"workload": "64 FP32 matrices 1024x512 (decay 0.1), d = 32, 256 out-of-sample vectors each",
            "batched": {"forward_ms": float(np.median(fb)), "adjoint_ms": float(np.median(ab)),
                        "note": "one batched compression launch (tol 0, d_max 32) and one rbd_grad_batched call "
                                "(through the Python binding), median of 3",
                        "pivots_equal_one_by_one": same_piv, "adjoint_max_rel_dev_vs_oracle": worst_b},
            "one_by_one": {"forward_ms": one[0], "adjoint_ms": one[1], "adjoint_max_rel_dev_vs_oracle": worst},
            "oracle_adjoint_s_1core_est_64": t_or / 2 * 64,
            "fd_check": "against FP64 central differences in tests/test_gpu_grad.py (<= 1e-6 relative)"}


PAPER5001_N, PAPER5001_D = 5001, 22


def paper_5001_form(dev) -> dict:
    """Section 4.2.2 (approximate reconstruction): f = 0.6 f1 + 0.1 f2 + 0.01 f3 on a 5001 x 5001
    grid of [-1, 1]^2, d = 22.  The GPU's time to d = 22 (rbd_compress, CUDA events, FP64 input
    resident), the FP64 oracle's time on the host, a truncated SVD of the same rank on the host
    (scipy.sparse.linalg.svds, k = 22: the paper compares with Matlab's svds), and the pointwise
    and relative Frobenius errors of both decompositions."""
    import torch

    import gen
    import oracle
    import paper_1503_05947_gb300 as rbd
    X = gen.paper_approx_function(PAPER5001_N)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev).t()
    rbd.compress(Xd, 0.0, PAPER5001_D)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record()
    r = rbd.compress(Xd, 0.0, PAPER5001_D)
    ev1.record()
    torch.cuda.synchronize(dev)
    gpu_ms = ev0.elapsed_time(ev1)
    Xr = rbd.reconstruct(r.Y, r.T)
    pw = float((Xd - Xr).abs().max())
    fr = float((Xd - Xr).norm() / Xd.norm())
    del Xr
    t0 = time.perf_counter()
    ro = oracle.compress(X, 0.0, PAPER5001_D)
    t_or = time.perf_counter() - t0
    out = {"workload": f"f = 0.6 f1 + 0.1 f2 + 0.01 f3 on a {PAPER5001_N}^2 grid of [-1,1]^2, d = {PAPER5001_D}",
           "bases": r.d, "gpu_ms": gpu_ms, "gpu_pointwise_err": pw, "gpu_rel_fro_err": fr,
           "oracle_s_single_thread": t_or, "oracle_bases": ro["d"],
           "compression_ratio": PAPER5001_N * PAPER5001_N / (2 * PAPER5001_N * r.d),
           "paper": "RBD pointwise error < 1e-6 at d = 22; RBD 16x faster than svds (Matlab 2014a, 2011 iMac)"}
    try:
        from scipy.sparse.linalg import svds
        t0 = time.perf_counter()
        u, sv, vt = svds(X, k=PAPER5001_D)
        t_svd = time.perf_counter() - t0
        Xs = (u * sv) @ vt
        out.update({"svds_s_host": t_svd, "svds_pointwise_err": float(np.abs(X - Xs).max()),
                    "svds_rel_fro_err": float(np.linalg.norm(X - Xs) / np.linalg.norm(X)),
                    "gpu_speedup_vs_svds": t_svd / (gpu_ms * 1e-3), "host_cpu": host_cpu()})
        del u, vt, Xs
    except Exception as exc:  # noqa: BLE001
        out["svds"] = f"unavailable: {exc}"
    del Xd
    torch.cuda.empty_cache()
    return out


BATCH_WORKLOAD = ("2048 FP32 matrices U diag(s) V' (Haar U, V; s_i = exp(-r i), r ~ U[0.05, 0.5], truncated at 1e-9), "
                  "m log-uniform in [256, 4096], n log-uniform in [64, 2048], tol log-uniform in [1e-6, 1e-2] "
                  "(relative max-column), d_max = min(m, n, 512) (seed 3)")


def batched_forms(dev) -> dict:
    """The batched form: the 2048-matrix workload compressed by one persistent launch captured in a
    CUDA graph, with the default launch shape and with the one the plan's autotuner picks (column
    group width, tile rows, team sizing, ring depth; the tuning time is reported), against the
    single-matrix path
    (rbd_compress per matrix, FP32 and FP64 copies) timed on a seeded sample of 64 matrices and
    scaled to the whole batch by sum((d + 1) m n)."""
    import torch

    import gen
    import paper_1503_05947_gb300 as rbd
    specs = gen.batch_specs(2048, seed=3)
    items = []
    for sp in specs:
        s = gen.decay_spectrum(sp["rate"], min(sp["m"], sp["n"]))
        X = gen.lowrank_torch(sp["m"], sp["n"], s, sp["seed"], device=dev, dtype=torch.float32)
        items.append({"X": X, "tol": sp["tol"], "tol_mode": "maxcol_rel", "d_max": sp["d_max"],
                          "d_hint": sp["d_hint"]})
    plan = rbd.BatchPlan(items)

    def graph_ms(reps=3):
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            plan.run()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.run()
        graph.replay()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    untuned = plan.config()
    ms_untuned = graph_ms()
    import tempfile
    t0 = time.perf_counter()
    tuned = plan.tune(cache=os.path.join(tempfile.mkdtemp(), "batch_tune.json"))  # a fresh tuning
    tune_s = time.perf_counter() - t0
    ms = graph_ms()
    res = plan.results()
    cost = [(r["d"] + 1) * it["X"].shape[0] * it["X"].shape[1] for r, it in zip(res, items)]
    xbytes = 4.0 * sum(cost)
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(len(items), 64, replace=False).tolist())
    scale = sum(cost) / sum(cost[i] for i in sample)

    def single(dtype):
        Xs = [items[i]["X"] if dtype == torch.float32 else items[i]["X"].t().contiguous().double().t() for i in sample]
        for i, X in zip(sample[:2], Xs[:2]):
            rbd.compress(X, items[i]["tol"], items[i]["d_max"], tol_mode="maxcol_rel")
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i, X in zip(sample, Xs):
            rbd.compress(X, items[i]["tol"], items[i]["d_max"], tol_mode="maxcol_rel")
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) * 1e3 * scale

    s32 = single(torch.float32)
    s64 = single(torch.float64)
    out = {"workload": BATCH_WORKLOAD, "matrices": len(items), "graph": True,
           "launch_shape_default": untuned, "ms_default": ms_untuned,
           "launch_shape_tuned": {k: tuned[k] for k in ("cols", "tile_rows", "team_pct", "stages")},
           "tune_s": tune_s, "bucket": plan.bucket(), "speedup_tuned_vs_default": ms_untuned / ms, "ms": ms,
           "bases_total": int(sum(r["d"] for r in res)), "x_bytes_streamed": xbytes, "gbs": xbytes / (ms * 1e-3) / 1e9,
           "single_matrix_f32_ms_est": s32, "speedup_vs_single_f32": s32 / ms,
           "single_matrix_f64_ms_est": s64, "speedup_vs_single_f64": s64 / ms,
           "single_sample": "64 seeded matrices compressed one by one (rbd_compress, synchronous calls), "
                            "scaled by sum((d + 1) m n)"}
    del plan, items
    torch.cuda.empty_cache()
    return out


def profile_case(name: str, shape: str | None = None):
    """Short, fixed launches of one kernel for profiler captures (not a bench line):
    bf16-small: the persistent kernel on the parametric snapshots 16384 x 4096 stored in BF16;
    batched-small / batched-full: two runs of the batched form on the first 256 matrices / all 2048
    of the 2048-matrix workload, in the launch shape `shape` ("cols,tile_rows,team_pct,stages"; the
    plan's default without it)."""
    import torch

    import gen
    import paper_1503_05947_gb300 as rbd
    dev = torch.device("cuda", 0)
    if name == "bf16-small":
        X = gen.parametric_snapshots_torch(16384, 4096, device=dev).t().contiguous().to(torch.bfloat16).t()
        for _ in range(2):
            r = rbd.compress(X, 0.0, 32)
        torch.cuda.synchronize(dev)
        print(json.dumps({"case": name, "bases": r.d}))
    elif name in ("batched-small", "batched-full"):
        items = []
        for sp in gen.batch_specs(2048, seed=3)[:256 if name == "batched-small" else 2048]:
            s = gen.decay_spectrum(sp["rate"], min(sp["m"], sp["n"]))
            X = gen.lowrank_torch(sp["m"], sp["n"], s, sp["seed"], device=dev, dtype=torch.float32)
            items.append({"X": X, "tol": sp["tol"], "tol_mode": "maxcol_rel", "d_max": sp["d_max"],
                          "d_hint": sp["d_hint"]})
        plan = rbd.BatchPlan(items)
        if shape:
            c, r_, t, st = (int(v) for v in shape.split(","))
            plan.set_config({"cols": c, "tile_rows": r_, "team_pct": t, "stages": st})
        for _ in range(2):
            plan.run()
        torch.cuda.synchronize(dev)
        res = plan.results()
        xbytes = 4.0 * sum((r["d"] + 1) * it["X"].shape[0] * it["X"].shape[1] for r, it in zip(res, items))
        print(json.dumps({"case": name, "shape": plan.config(), "bases": int(sum(r["d"] for r in res)),
                          "x_bytes_streamed_per_run": xbytes}))
    else:
        raise SystemExit(f"unknown profile case {name}")


def gen_x64(q):
    import gen
    return gen.u8_to_unit_f64(q)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=64, help="bases in the single-thread oracle sample")
    ap.add_argument("--ref-steps", type=int, default=32, help="bases per step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--d-max", type=int, default=512,
                    help="basis limit; values below 512 give the short profiling case, not a bench line")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (end-to-end) measurement")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision / batched form measurements")
    ap.add_argument("--batch-shape", default=None, help="cols,tile_rows,team_pct,stages for the batched profile cases")
    ap.add_argument("--profile-case", choices=["bf16-small", "batched-small", "batched-full"], default=None,
                    help="run one short fixed case for a profiler capture instead of the bench")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case, args.batch_shape)
        return
    world, rank, local = dist_setup()
    global D_MAX
    D_MAX = args.d_max
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
