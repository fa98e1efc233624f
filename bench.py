#!/usr/bin/env python3
"""Benchmark of the HOSCF hot path on GB300.

One step = one HOSCF iteration (Algorithm 1 lines 4-9) on the headline
workload: all coupling blocks from one read of the tensor (TTVc pass and its
reduction), the KKT certificate of the current point, the largest-magnitude
eigen step and the block normalisation - through the library's C ABI
(hoscf_ttvc_blocks + hoscf_eig_step).  Every step starts from the same
seeded initial guess, so every step is the first (most expensive) iteration
of the solve and does identical work; full solves are reported separately.

Workload (default): order-3 1024^3 FP32 tensor, planted rank-5 CP
sum_r 2^-r a_r o b_r o c_r (unit Gaussian factors) plus i.i.d. Gaussian noise
with ||E||_F = 0.05 ||L||_F; generated on the device from fixed seeds.  The
4 GiB tensor is larger than L2, so no flush is needed between steps.

Metric: TTVc-pass HBM GB/s = algorithmic bytes of one pass (tensor + factors
+ blocks) per step time.  `roofline` reports the pass alone against the
measured HBM peak; `e2e` repeats the step with the tensor copied from pinned
host memory every step; `cpu_baseline` times the FP64 CPU oracle on a bounded
sample of the same workload.  Extra keys report time-to-residual 1e-6 of the
solve variants.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2a_1024cube_rank5")
    ap.add_argument("--no-extras", action="store_true", help="skip time-to-residual extras")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--dims", default=None,
                    help="comma-separated dims: same planted rank-5 recipe at another size")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
def make_workload(name, seed, device, dims=None):
    import workloads as W
    if dims:
        T, _ = W.planted_cp(dims, [2.0 ** -r for r in range(5)], seed=seed, noise_rel=0.05,
                            device=device)
    else:
        T = W.config_tensor(name, seed=seed, device=device)
    u0 = __import__("torch").cat(W.unit_gaussian_vectors(T.shape, seed + 1, device=device))
    return T, u0


def pass_bytes(dims, elem_bytes=4):
    N = math.prod(dims)
    n = sum(dims)
    P = sum(dims[m] * dims[k] for m in range(len(dims)) for k in range(m + 1, len(dims)))
    return N * elem_bytes + 4 * n + 4 * P


# ------------------------------------------------------------------ CPU baseline
def cpu_baseline(workload, seconds, seed=0):
    """FP64 oracle (as it stands) on a bounded slab of the workload: the first
    S mode-1 slices of the same seeded tensor; one oracle HOSCF step on it
    (blocks by definition + dense eigen step).  Returns GB/s of tensor bytes."""
    import numpy as np
    import torch
    import oracle
    import workloads as W
    T = W.config_tensor(workload, seed=seed, device="cpu")
    dims = list(T.shape)
    u0 = [v.numpy() for v in W.unit_gaussian_vectors(dims, seed + 1)]
    cores = len(os.sched_getaffinity(0))
    S = 4
    elapsed = 0.0
    while True:
        sub = np.ascontiguousarray(T[:S].numpy())
        us = [u0[0][:S] / np.linalg.norm(u0[0][:S])] + u0[1:]
        t0 = time.perf_counter()
        Hp = oracle.blocks(sub, us, nthreads=cores)
        J = oracle.nepv_matrix(Hp, [S] + dims[1:])
        oracle.largest_magnitude_eigpair(J, np.concatenate(us) / math.sqrt(len(dims)))
        elapsed = time.perf_counter() - t0
        if elapsed * 2 > seconds or S * 2 > dims[0]:
            break
        S *= 2
    del T
    nbytes = sub.nbytes
    return {"value": nbytes / elapsed / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"first {S} of {dims[0]} mode-1 slices ({nbytes / 1e6:.0f} MB), one FP64 "
                      f"HOSCF step (blocks by definition + dense eigh), {elapsed:.2f} s"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import workloads as W
    oracle.build()
    T = W.config_tensor(args.workload, seed=0, device="cpu")
    dims = list(T.shape)
    u0 = [v.numpy() for v in W.unit_gaussian_vectors(dims, 1)]
    cores = len(os.sched_getaffinity(0))
    # each step: one oracle HOSCF step on a bounded slab (sized for ~10 s)
    S = max(1, min(dims[0], 8))
    sub = np.ascontiguousarray(T[:S].numpy())
    us = [u0[0][:S] / np.linalg.norm(u0[0][:S])] + u0[1:]
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Hp = oracle.blocks(sub, us, nthreads=cores)
        J = oracle.nepv_matrix(Hp, [S] + dims[1:])
        oracle.largest_magnitude_eigpair(J, np.concatenate(us) / math.sqrt(len(dims)))
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = sub.nbytes * len(times) / tot / 1e9
    line = {"impl": "reference", "metric": "TTVc pass HBM GB/s", "value": v, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dims": dims, "sample_slices": S},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {S} of {dims[0]} mode-1 slices per step"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2403_01778_gb300 as P
    from paper_2403_01778_gb300 import build
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    dims_arg = [int(v) for v in args.dims.split(",")] if args.dims else None
    T, u0 = make_workload(args.workload, seed=rank, device=dev, dims=dims_arg)
    dims = tuple(T.shape)
    d = len(dims)
    nb = pass_bytes(dims, T.element_size())
    stream = torch.cuda.current_stream()
    H = torch.empty(P.n_blocks(dims), device=dev, dtype=torch.float32)

    def normalise(u):
        out, o = [], 0
        for n in dims:
            v = u[o:o + n]
            out.append(v / v.norm())
            o += n
        return torch.cat(out)

    u_start = normalise(u0)
    x_start = P.balanced(u_start, dims)
    state = {"u": u_start.clone()}
    pass_ev = []

    def step(record=False):
        u = u_start
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        P.hoscf_ttvc_blocks(T, u, H)
        if record:
            e1.record(stream)
            pass_ev.append((e0, e1))
        x, un, lam = P.hoscf_eig_step(dims, H, x_start)
        state["u"] = un
        return lam

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    state["u"] = u_start.clone()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    clocks = clk.stop()
    pass_ms = [a.elapsed_time(b) for a, b in pass_ev]
    pass_avg = sum(pass_ms) / len(pass_ms)
    if dist:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    value = nb * args.steps * world / (ms / 1e3) / 1e9

    # ---- end to end: tensor copied from pinned host memory every step
    e2e = None
    if not args.no_e2e:
        host = torch.empty(T.shape, dtype=T.dtype, pin_memory=True)
        host.copy_(T)
        Td = torch.empty_like(T)
        u_host = u_start.cpu().pin_memory()
        res_host = torch.empty(sum(dims), dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize()
        ue = u_start.clone()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k_e2e = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(k_e2e):
            Td.copy_(host, non_blocking=True)
            ue.copy_(u_host, non_blocking=True)
            P.hoscf_ttvc_blocks(Td, ue, H)
            _, un, lam = P.hoscf_eig_step(dims, H, P.balanced(ue, dims))
            res_host.copy_(un, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / k_e2e
        e2e = {"value": nb / (ms_e2e / 1e3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": T.numel() * T.element_size() + 4 * sum(dims),
               "d2h_bytes_per_step": 4 * sum(dims), "ms_per_step": ms_e2e, "steps": k_e2e}
        del host, Td

    extras = {}
    if not args.no_extras and rank == 0:
        for variant in ("hoscf", "ihoscf"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = P.hoscf_solve(T, u0, tol=1e-6, max_iter=200, variant=variant)
            torch.cuda.synchronize()
            extras[f"time_to_residual_1e-6_{variant}"] = {
                "seconds": time.perf_counter() - t0, "iters": r.iters, "passes": r.passes,
                "resid": r.resid, "sigma": r.sigma, "converged": r.converged}

    peak, peak_kind = load_peaks()
    achieved = nb / (pass_avg / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": "TTVc pass HBM GB/s", "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if T.dtype == torch.float32 else str(T.dtype),
            "data": "synthetic",
            "config": {"workload": args.workload if not args.dims else "planted rank-5 + 5% noise",
                       "dims": list(dims), "order": d,
                       "step": "one HOSCF iteration from the seeded x0: TTVc pass + reduce + "
                               "Lanczos eigen step + block normalisation",
                       "l2": "inputs larger than L2 (4 GiB tensor), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "TTVc pass (streaming kernel + its reduce kernels), "
                                   f"avg {pass_avg:.4f} ms over the timed steps",
                         "peak_kind": peak_kind},
            "pass_ms_avg": pass_avg,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps * (4 + 2 if d == 3 else 8),
        }
        if extras:
            line["extras"] = extras
        if world == 1 and not args.no_cpu:
            try:
                line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
            except Exception as exc:   # report, do not hide
                line["cpu_baseline"] = {"error": repr(exc)}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
