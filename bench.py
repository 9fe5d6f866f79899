"""Benchmark: full RQRCP (Alg. 4) of a 16384 x 16384 graded matrix on GB300.

One step = one RQRCP of A (FP64, b = 64, p = 8, k = n) through the C ABI,
preceded by a device copy that restores A (A is factorised in place).  The
metric is TFLOP/s with the algorithmic count 4/3 n^3 of Householder QR (the
same count is used for the unpivoted QR timed beside it, so the ratio is a
time ratio).  Inputs are 2.1 GB, larger than L2.

Extra legs (rank 0): unpivoted blocked QR of the same matrix, the FP32 path,
an end-to-end number with host buffers, per-phase timing with CUDA events,
the CPU oracle on a bounded sample.  ``--impl reference`` times the CPU
oracle alone.  Under torchrun every rank factorises its own matrix (replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RQRCP s & TFLOP/s vs unpivoted QR on GB300; TUXV req/s, p99 at fixed error"
# FP64 is bound by the FP64 pipe: 152 SMs x 2070 MHz x 2 DFMA/clk x 2 flop.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--decades", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip QR / FP32 / e2e / CPU legs")
    ap.add_argument("--cpu-n", type=int, default=2048)
    return ap.parse_args()


def flops_qr(m, n):
    """Householder QR flops: 4mnk - 2(m+n)k^2 + 4k^3/3, k = min(m, n) (= 4/3 n^3 for m = n)."""
    k = min(m, n)
    return 4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 * k ** 3 / 3.0


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.proc = None
        self.dev = dev

    def start(self):
        import torch
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            cmd += ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 6]
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].strip() == "Active"})
        load = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(n, b, p, decades):
    """The oracle as it stands, on a bounded n x n sample of the same workload."""
    import numpy as np  # noqa: F401
    import oracle as O
    from paper_2008_04447_gb300 import inputs as I
    a = I.graded(n, n, decades, seed=0)
    om = I.omega(b + p, n, seed=1)
    t0 = time.perf_counter()
    O.rqrcp(a, om, b)
    dt = time.perf_counter() - t0
    return {"value": flops_qr(n, n) / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle RQRCP of one {n}x{n} FP64 graded matrix (10^-{decades:g} spread), b={b}, p={p}: "
                      f"{dt:.1f} s; numpy with its BLAS threads"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n = args.cpu_n
    times = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(n, args.b, args.p, args.decades)
        if i >= args.warmup:
            times.append(flops_qr(n, n) / (r["value"] * 1e12))
    t = sum(times)
    val = args.steps * flops_qr(n, n) / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rqrcp_fp64_graded_{n}x{n}_b{args.b}_p{args.p} (bounded CPU sample of the "
                                   f"{args.n}x{args.n} workload)", "m": n, "n": n, "b": args.b, "p": args.p},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} oracle RQRCP runs of {n}x{n} FP64"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    torch.cuda.set_device(local)
    from paper_2008_04447_gb300 import Handle, colmajor, build as B
    from paper_2008_04447_gb300 import inputs as I
    if rank == 0:
        B.build()
    barrier(ws)
    n, b, p = args.n, args.b, args.p
    m = n
    l = b + p
    fl = flops_qr(m, n)

    A0 = colmajor(I.graded_torch(m, n, args.decades, seed=rank))          # pristine FP64 input
    Om = colmajor(I.omega_torch(l, m, seed=1000 + rank))
    A = torch.empty_like(A0)
    torch.cuda.synchronize()
    h = Handle()

    def step():
        A.copy_(A0)
        h.rqrcp(A, Om, b, p)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    clk = Clocks(local)
    clk.start()
    h.profile(True)
    la0 = h.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = h.launches - la0
    prof = h.profile_read()
    h.profile(False)
    ms = e0.elapsed_time(e1)
    barrier(ws)
    ms = max_over_ranks(ms, ws)
    ms_step = ms / args.steps
    value = ws * args.steps * fl / (ms / 1e3) / 1e12

    tr = prof["trailing"]
    tot_ms = sum(v[0] for v in prof.values())
    phases = {k: {"ms_per_step": v[0] / args.steps, "share": v[0] / tot_ms if tot_ms else None,
                  "tflops": (v[1] / (v[0] / 1e3) / 1e12) if v[0] > 0 and v[1] > 0 else None,
                  "gbs": (v[2] / (v[0] / 1e3) / 1e9) if v[0] > 0 else None, "launches": v[3] // args.steps}
              for k, v in prof.items()}
    achieved = tr[1] / (tr[0] / 1e3) / 1e12 if tr[0] > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                "kernel": "trailing update (block reflector GEMMs), FP64",
                "peak_source": "derived: 152 SMs x 2070 MHz x 2 DFMA/clk/SM x 2 flop (FP64 pipe, nominal)"}

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rqrcp_fp64_graded_{m}x{n}_b{b}_p{p}", "m": m, "n": n, "b": b, "p": p, "k": n,
                       "spectrum": f"U diag(10^(-{args.decades:g} i/n)) V^T, Haar U, V",
                       "l2": "inputs larger than L2 (A is 2.1 GB)",
                       "step": "device copy restoring A (2.1 GB) + rq_rqrcp", "parallelism": f"replicas x{ws}"},
            "rqrcp_s": ms_step / 1e3, "roofline": roofline, "phases": phases, "gpu_launches": launches,
            "clocks": clocks}

    if rank == 0 and not args.no_extras:
        # unpivoted blocked QR of the same matrix, same kernels (the paper's comparison)
        def qr_step():
            A.copy_(A0)
            h.qr(A, b)
        qr_step()
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record()
        for _ in range(2):
            qr_step()
        q1.record()
        torch.cuda.synchronize()
        qr_ms = q0.elapsed_time(q1) / 2
        line["qr"] = {"s": qr_ms / 1e3, "tflops": fl / (qr_ms / 1e3) / 1e12,
                      "rqrcp_over_qr": ms_step / qr_ms}

        # end to end through the C ABI with host buffers (pinned; column-major A is
        # copied as its contiguous transpose so each copy is one cudaMemcpyAsync)
        Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A0.t())
        Ao = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
        tau_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
        jp_h = torch.empty(n, dtype=torch.int32, pin_memory=True)

        def e2e_step():
            A.t().copy_(Ah, non_blocking=True)
            tau, jpvt, info = h.rqrcp(A, Om, b, p)
            Ao.copy_(A.t(), non_blocking=True)
            tau_h.copy_(tau, non_blocking=True)
            jp_h.copy_(jpvt, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = 2
        for _ in range(E):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / E
        line["e2e"] = {"value": fl / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * m * n,
                       "d2h_bytes_per_step": 8 * m * n + 12 * n, "s_per_step": e2e_s}
        del Ah, Ao

        # FP32 path on the same matrix (FP32 storage and updates, FP64 reflectors and norms)
        A32 = A0.float()
        A32 = colmajor(A32)
        Om32 = colmajor(Om.float())
        W = torch.empty_like(A32)

        def f32(fn):
            W.copy_(A32)
            fn()
        for _ in range(2):
            f32(lambda: h.rqrcp(W, Om32, b, p))
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(3):
            f32(lambda: h.rqrcp(W, Om32, b, p))
        g1.record()
        torch.cuda.synchronize()
        r32 = g0.elapsed_time(g1) / 3
        f32(lambda: h.qr(W, b))
        g0.record()
        for _ in range(3):
            f32(lambda: h.qr(W, b))
        g1.record()
        torch.cuda.synchronize()
        q32 = g0.elapsed_time(g1) / 3
        line["fp32"] = {"rqrcp_s": r32 / 1e3, "rqrcp_tflops": fl / (r32 / 1e3) / 1e12, "qr_s": q32 / 1e3,
                        "qr_tflops": fl / (q32 / 1e3) / 1e12, "rqrcp_over_qr": r32 / q32}
        del A32, W

        line["cpu_baseline"] = cpu_baseline(args.cpu_n, b, p, args.decades)
    barrier(ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
