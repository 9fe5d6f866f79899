"""Benchmark: full RQRCP (Alg. 4) of a 16384 x 16384 graded matrix on GB300.

One step = one RQRCP of A (FP64, b = 64, p = 8, k = n) through the C ABI,
preceded by a device copy that restores A (A is factorised in place).  The
metric is TFLOP/s with the algorithmic count 4/3 n^3 of Householder QR (the
same count is used for the unpivoted QR timed beside it, so the ratio is a
time ratio).  Inputs are 2.1 GB, larger than L2.

Extra legs (rank 0): unpivoted blocked QR of the same matrix, the FP32 path,
an end-to-end number with host buffers, per-phase timing with CUDA events,
repeated sampling (RSRQRCP) against the update formula on the same matrix,
the CPU oracle on a bounded sample, truncated TUXV of a 32768 x 16384 matrix,
the batched TUXV of 4096 small problems and the Poisson serving sweep.  ``--impl reference`` times the CPU
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


def hbm_peak_gbs():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else
    the earlier GB300 measurement the profiling notes give as the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback: 6.8 TB/s, an earlier GB300 copy measurement"


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
    ap.add_argument("--no-extras", action="store_true", help="skip every leg but the timed RQRCP")
    ap.add_argument("--legs", default="qr,e2e,fp32,rsrqrcp,cpu,fp64peak,slices,tuxv,batched,serving",
                    help="extra legs to run (comma list); --no-extras clears it")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"], help="precision of the timed RQRCP")
    ap.add_argument("--only-batched", action="store_true", help="run only the batched leg (profiling)")
    ap.add_argument("--only", default="", choices=["", "tuxv", "batched", "serving", "fp64peak"],
                    help="run only this leg and print its JSON (profiling)")
    ap.add_argument("--cpu-n", type=int, default=2048)
    ap.add_argument("--batch", type=int, default=4096, help="problems in the batched leg")
    ap.add_argument("--no-tune", action="store_true", help="batched leg: keep the default tile policy (profiling)")
    ap.add_argument("--tuxv-shape", default="32768,16384,512", help="m,n,k of the TUXV leg")
    ap.add_argument("--sweep", default="", help="paper-shaped timing sweeps instead of the bench line (comma list of "
                    + ", ".join(SWEEPS) + ", or 'all'); one JSON line per point")
    args = ap.parse_args()
    args.legs = set() if args.no_extras else {x.strip() for x in args.legs.split(",") if x.strip()}
    return args


# Paper-shaped timing sweeps (Sec. 5.1 full decompositions, Sec. 5.2 truncated):
# (m, n, k) per point, k = None for a full factorisation.  The paper scales
# around 12000 x 12000 with truncation rank 1200.
SWEEPS = {
    "full-order": [(n, n, None) for n in (2000, 4000, 6000, 8000, 10000, 12000)],
    "full-cols": [(12000, n, None) for n in (3000, 6000, 12000, 24000)],
    "full-rows": [(m, 12000, None) for m in (3000, 6000, 12000, 24000)],
    "trunc-rank": [(12000, 12000, k) for k in (150, 300, 600, 1200, 2400)],
    "trunc-cols": [(12000, n, 1200) for n in (3000, 6000, 12000, 24000)],
    "trunc-rows": [(m, 12000, 1200) for m in (3000, 6000, 12000, 24000)],
}


def run_sweep(args):
    """Times each algorithm once (after one untimed call at the same size) on an
    i.i.d. Gaussian matrix (the paper's timing matrices are random), FP64 unless
    --prec fp32.  Full points: RQRCP, RSRQRCP, unpivoted QR, and cuSOLVER geqrf
    through torch as context.  Truncated points: RQRCP, RSRQRCP (both with the
    trailing update, halted at k), TRQRCP and TUXV (j_max = 1)."""
    import torch
    from paper_2008_04447_gb300 import Handle, build as B
    B.build()
    names = list(SWEEPS) if args.sweep == "all" else [x.strip() for x in args.sweep.split(",") if x.strip()]
    dt = torch.float64 if args.prec == "fp64" else torch.float32
    h = Handle()
    b, p = args.b, args.p
    l = b + p
    gen = torch.Generator(device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(prep, run):
        out = []
        for _ in range(2):
            prep()
            torch.cuda.synchronize()
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return out[-1]

    for name in names:
        for (m, n, k) in SWEEPS[name]:
            gen.manual_seed(m * 100003 + n)
            A0 = torch.randn((n, m), generator=gen, device="cuda", dtype=dt).t()    # column-major m x n
            A = torch.empty_like(A0.t()).t()
            Om = h.gaussian(l, m, 1, dtype=dt)
            kk = min(m, n) if k is None else k
            res = {}

            def restore():
                A.copy_(A0)
            res["rqrcp"] = timed(restore, lambda: h.rqrcp(A, Om, b, p, kk))
            res["rsrqrcp"] = timed(restore, lambda: h.rsrqrcp(A, 7, b, p, kk))
            if k is None:
                res["qr"] = timed(restore, lambda: h.qr(A, b))
                res["cusolver_geqrf_via_torch"] = timed(restore, lambda: torch.geqrf(A))
            else:
                res["trqrcp"] = timed(lambda: None, lambda: h.trqrcp(A0, Om, b, p, kk))
                res["tuxv"] = timed(lambda: None, lambda: h.tuxv(A0, Om, b, p, kk))
            fl = flops_qr(m, n) if k is None else 4.0 * m * n * kk - 2.0 * (m + n) * kk * kk + 4.0 * kk ** 3 / 3.0
            line = {"sweep": name, "m": m, "n": n, "k": kk, "b": b, "p": p, "dtype": args.prec, "data": "synthetic",
                    "matrix": "i.i.d. N(0,1)", "seconds": res,
                    "tflops_householder_count": {a: fl / t / 1e12 for a, t in res.items()}}
            print(json.dumps(line), flush=True)
            del A0, A
            torch.cuda.empty_cache()


def bf16_peak_tflops():
    """(TFLOP/s, source): the measured sustained bfloat16 dense rate of
    MEASURED_PEAKS.json (the trailing update runs inside a seconds-long step),
    else the sustained figure the profiling notes give as the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        for key in ("bf16_tflops_sustained", "bf16_tflops"):
            if key in d:
                return float(d[key]), f"MEASURED_PEAKS.json {key} (measured cuBLAS bf16)"
    except (OSError, KeyError, ValueError):
        pass
    return 1700.0, "fallback: 1.7 PFLOP/s, an earlier sustained GB300 bf16 measurement"


# DRAM bytes per trailing entry (m_t n2 of a block) moved by the two FP64
# tensor-core products, from the ncu capture of a 6144 x 6144 factorisation
# summarised in profiles/oz_gemm_fp64_6144_ncu.md: W = A2^T (Y T) reads A2's
# slice planes once (1.035 x 16 B) and the update reads and writes A2
# (0.905 x 16 B).  Valid while those kernels are unchanged.
OZ_DRAM_BYTES_PER_ENTRY = 16.0 * (1.035 + 0.905)


def trailing_entries(m, n, b, k=None):
    """sum over blocks of m_t n2: the entries the trailing update touches."""
    k = min(m, n) if k is None else k
    return sum(float(m - j0) * (n - j0 - min(b, k - j0)) for j0 in range(0, k, b))


def slice_pair_flops(m, n, b, k=None):
    """bfloat16 tensor-core flops of the FP64 trailing update through slices:
    36 slice-pair products for each of the two block reflector products
    (W^T = (Y T)^T A2 and A2 -= Y W^T, 2 m_t n2 b_J flops each) per block."""
    k = min(m, n) if k is None else k
    tot = 0.0
    for j0 in range(0, k, b):
        bj = min(b, k - j0)
        tot += 2 * 2.0 * (m - j0) * (n - j0 - bj) * bj
    return 36.0 * tot


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
    """Max of a per-rank timing over all ranks (the slowest replica sets the pace)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
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


def cpu_context(m=8192, n=4096, k=128, b=64, p=8, nq=4096):
    """Host timings beside the CPU baseline, for context only (not targets):
    the oracle's TUXV on the truncated workload's recipe scaled to m x n at
    rank k (the size the oracle finishes in seconds), and LAPACK's unpivoted
    and pivoted QR (dgeqrf, dgeqp3 through scipy; the paper's own comparison
    routines) on an nq x nq graded matrix, with the host's BLAS threads."""
    import scipy.linalg as sla
    import oracle as O
    from paper_2008_04447_gb300 import inputs as I
    out = {"cores": os.cpu_count()}
    a = I.lowrank_plus_noise(m, n, 1024, 1e-6, seed=3)
    om = I.omega(b + p, m, seed=4)
    t0 = time.perf_counter()
    O.tuxv(a, om, b, k)
    out[f"oracle_tuxv_{m}x{n}_k{k}_s"] = time.perf_counter() - t0
    g = I.graded(nq, nq, 12, seed=5)
    t0 = time.perf_counter()
    sla.qr(g, mode="r", check_finite=False)
    out[f"lapack_dgeqrf_{nq}_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sla.qr(g, mode="r", pivoting=True, check_finite=False)
    out[f"lapack_dgeqp3_{nq}_s"] = time.perf_counter() - t0
    return out


def batch_inputs(count, seed, threads=16):
    """The many-small-problems workload: graded spectra 10^(-6 i/n), Haar factors,
    (m, n, k) from the batch recipe; generated on the host (FP64) in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2008_04447_gb300 import inputs as I
    shapes = I.batch_shapes(count, seed)

    def one(i):
        m, n, k = shapes[i]
        b = min(32, k)
        return (I.graded(m, n, 6, seed=seed * 100000 + i), I.omega(b + 8, m, seed=seed * 100000 + 50000 + i), b, 8, k)
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, range(count)))


def to_device_f32(host):
    import torch
    from paper_2008_04447_gb300 import colmajor
    return [(colmajor(torch.as_tensor(a, dtype=torch.float32)).cuda(),
             colmajor(torch.as_tensor(om, dtype=torch.float32)).cuda(), b, p, k) for a, om, b, p, k in host]


def leg_rsrqrcp(h, A0, A, Om, b, p, fl, rqrcp_ms, prec):
    """RSRQRCP (fresh Gaussian per block, Sec. 3.4) against RQRCP with the update
    formula on the same matrix: FP64 (one timed step) and FP32 (three)."""
    import torch
    from paper_2008_04447_gb300 import colmajor
    m, n = A0.shape
    l = b + p
    ex = sum(2.0 * l * (m - j0 - b) * (n - j0 - b) for j0 in range(0, min(m, n) - b, b))
    out = {"extra_sketch_flops": ex}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def rs(W, src):
        W.copy_(src)
        h.rsrqrcp(W, 1234, b, p)
    ms = timed(lambda: rs(A, A0), 1)
    out[prec] = {"rsrqrcp_s": ms / 1e3, "rqrcp_s": rqrcp_ms / 1e3, "rsrqrcp_over_rqrcp": ms / rqrcp_ms,
                 "tflops_counting_4n3_3": fl / (ms / 1e3) / 1e12}
    if prec == "fp64":
        A32 = colmajor(A0.float())
        Om32 = colmajor(Om.float())
        W = torch.empty_like(A32)

        def up(W, src):
            W.copy_(src)
            h.rqrcp(W, Om32, b, p)
        r32 = timed(lambda: up(W, A32), 3)
        s32 = timed(lambda: rs(W, A32), 3)
        out["fp32"] = {"rsrqrcp_s": s32 / 1e3, "rqrcp_s": r32 / 1e3, "rsrqrcp_over_rqrcp": s32 / r32}
        del A32, W
    return out


def leg_slices(h):
    """Exactness of 8-bit slice products on the tensor cores: integer matrices
    with entries in [-255, 255] (the slices of an exact FP64 split) through
    rq_gemm_bf16, against the exact integer product.  Every sum stays below
    2^24 up to K = 256 (also with all entries 255), so those results are exact
    if the tensor core's FP32 accumulation keeps every bit of them; K = 2048 is
    past that bound and shows the rounding of FP32 sums that large."""
    import numpy as np
    import torch
    from paper_2008_04447_gb300 import colmajor
    out = {}
    g = np.random.default_rng(0)
    M = N = 128
    for kind in ("random", "max"):
        for K in (32, 64, 128, 256, 2048):
            if kind == "random":
                a, b = g.integers(-255, 256, (M, K)), g.integers(-255, 256, (K, N))
            else:
                a, b = np.full((M, K), 255), np.full((K, N), 255)
            exact = a.astype(np.int64) @ b.astype(np.int64)
            A = colmajor(torch.as_tensor(a, dtype=torch.float32)).cuda()
            B = colmajor(torch.as_tensor(b, dtype=torch.float32)).cuda()
            C, info = h.gemm_bf16(A, B)
            torch.cuda.synchronize()
            err = np.abs(C.cpu().double().numpy() - exact)
            out[f"{kind}_k{K}"] = {"max_abs_err": float(err.max()), "max_abs": float(np.abs(exact).max()),
                                   "info": int(info.cpu()[0])}
    out["exact_below_2^24"] = all(v["max_abs_err"] == 0 for key, v in out.items() if not key.endswith("k2048"))
    return out


def leg_fp64_peak(n=8192, reps=3):
    """FP64 throughput of cuBLAS DGEMM (through torch) on n x n operands, timed
    with CUDA events with the SM clocks sampled: a measured reference for the
    FP64 trailing update's derived peak (152 SMs x 2 DFMA/clk x 2 flop x clock)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = clk.stop()
    best = min(times)
    del a, b, c
    return {"cublas_dgemm_tflops": 2.0 * n ** 3 / (best / 1e3) / 1e12, "n": n, "ms": best,
            "derived_peak_tflops": FP64_PEAK_TFLOPS, "clocks": clocks}


def leg_tuxv(h, steps=3, warmup=3, shape=(32768, 16384, 512)):
    """Truncated RQRCP + TUXV of one m x n matrix (low rank + noise; default
    32768 x 16384, k = 512): the FP32 path (FP32 sketch; the reduced-precision
    path that keeps each rank-k error within 1.05x the FP64 oracle's) and,
    beside it, the mixed mode (sketch from bfloat16-rounded inputs)."""
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, RQ_MIXED, colmajor
    from paper_2008_04447_gb300 import inputs as I
    m, n, k = shape
    b, p = 64, 8
    A = colmajor(I.lowrank_plus_noise_torch(m, n, 2048, 1e-6, seed=7).float())
    Om = colmajor(I.omega_torch(b + p, m, seed=8, dtype=torch.float32))
    peak, peak_src = hbm_peak_gbs()
    flops = 4.0 * k * m * n + 2.0 * (b + p) * m * n
    byts = 4.0 * m * n * (2 + k // b)

    def arm(prec):
        for _ in range(warmup):
            h.tuxv(A, Om, b, p, k, prec=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h.profile(True)
        e0.record()
        for _ in range(steps):
            U, X, V, _, info = h.tuxv(A, Om, b, p, k, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        prof = h.profile_read()
        h.profile(False)
        ms = e0.elapsed_time(e1) / steps
        gbs = byts / (ms / 1e3) / 1e9
        tr = prof["trailing"]
        return {"s": ms / 1e3, "tflops": flops / (ms / 1e3) / 1e12, "info": int(info.abs().sum()),
                "phases_ms": {kk: v[0] / steps for kk, v in prof.items()},
                # per phase: the algorithmic bytes and flops the library accounts, over the phase's event time
                "phases_gbs": {kk: v[2] / (v[0] / 1e3) / 1e9 for kk, v in prof.items() if v[0] > 0 and v[2] > 0},
                "phases_tflops": {kk: v[1] / (v[0] / 1e3) / 1e12 for kk, v in prof.items() if v[0] > 0 and v[1] > 0},
                "gbs_algorithmic": gbs, "hbm_frac": gbs / peak,
                "trailing_tflops": tr[1] / (tr[0] / 1e3) / 1e12 if tr[0] > 0 else None}, (U, X, V)

    out = {"workload": f"tuxv_lowrank_plus_noise_{m}x{n}_k{k}_b{b}_p{p}", "hbm_bytes_algorithmic": byts,
           "hbm_peak_source": peak_src}
    res = {}
    for name, prec in (("fp32", RQ_FP32), ("mixed", RQ_MIXED)):
        out[name], res[name] = arm(prec)
    # rank-k error in FP64 against the FP64 input
    A64 = I.lowrank_plus_noise_torch(m, n, 2048, 1e-6, seed=7)
    for name, (U, X, V) in res.items():
        R = A64 - U.double() @ (X.double() @ V.double().T)
        out[name]["rel_error"] = float(torch.linalg.norm(R) / torch.linalg.norm(A64))
        del R
    out["mixed_over_fp32_time"] = out["mixed"]["s"] / out["fp32"]["s"]
    del A, A64, res
    return out


def _rank_k_errors(host, order, idx, outs_by_arm, limit=600 * 400):
    """Per sampled problem: the rank-k error ||A - U X V^T||_F / ||A||_F of each
    arm's result, in FP64 against the FP64 input (problems of at most limit
    entries)."""
    import numpy as np
    rows = []
    for j in idx:
        a = host[order[j]][0]
        if a.shape[0] * a.shape[1] > limit:
            continue
        na = float(np.linalg.norm(a))
        row = {}
        for arm, outs in outs_by_arm.items():
            U, X, V = (t.cpu().double().numpy() for t in outs[j][:3])
            row[arm] = float(np.linalg.norm(a - U @ X @ V.T)) / na
        rows.append(row)
    return rows


def leg_batched(h, host, dev, steps=3, warmup=2, quality_sample=24, tune=True, fp64=True):
    """4096 uneven problems in one persistent launch: the FP32 path (tile policy
    autotuned on the batch first, outside the timed region; every policy gives
    the same bits), the mixed mode beside it, and the plain FP64 path (rq_tuxv
    in FP64, problem after problem: the batched kernel is FP32-only).  A step
    is one launch of the prepared batch (`problems_per_s`); `call_problems_per_s`
    times the full Python call, whose per-problem marshalling is host-bound, and
    `graph_problems_per_s` the launch captured in a CUDA graph.

    Quality, per sampled problem: each reduced-precision result's rank-k error
    over the FP64 path's on the same problem (the FP64 path matches the oracle
    to 1e-12 in the tests), and over the optimal rank-k error (numpy's SVD of
    the FP64 input)."""
    import numpy as np
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, RQ_MIXED
    order = sorted(range(len(dev)), key=lambda i: -(dev[i][0].shape[0] * dev[i][0].shape[1] * dev[i][4]))
    probs = [dev[i] for i in order]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tuning = {"tiles": list(h.batch_tiles)}
    outs = None
    if tune:
        try:
            t0 = time.perf_counter()
            tiles, tuned_ms, outs, _ = h.tune_batched(probs, prec=RQ_FP32, reps=1, passes=2)
            tuning = {"tiles": list(tiles), "tune_s": time.perf_counter() - t0, "tuned_ms": tuned_ms}
        except Exception as exc:  # the policy stays as it was; the leg is still measured
            tuning["tune_error"] = f"{type(exc).__name__}: {exc}"[:200]

    def timed(prec, outs):
        # the descriptors are built once (the batch's buffers stay the same);
        # each step is one persistent launch
        plan = h.prepare_batched(probs, outputs=outs)
        for _ in range(warmup):
            h.launch_prepared(plan, prec=prec)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            outs, info = h.launch_prepared(plan, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, outs, info

    def timed_calls(prec, outs):
        # the whole Python call per step: descriptors rebuilt and copied every time
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            outs, info = h.tuxv_batched(probs, prec=prec, outputs=outs)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms, outs, info = timed(RQ_FP32, outs)
    call_ms = timed_calls(RQ_FP32, outs)
    mms, mouts, minfo = timed(RQ_MIXED, None)
    # the same launch captured once in a CUDA graph and replayed (the call issues
    # one memset and one kernel, so the graph mainly removes host work)
    graph = {}
    try:
        from paper_2008_04447_gb300 import rq_tuxv_batched
        outs, info = h.tuxv_batched(probs, prec=RQ_FP32, outputs=outs)
        desc = h._keep                     # the descriptors of the last call (outputs = outs)
        dims = (max(int(t[0].shape[0]) for t in probs), max(int(t[0].shape[1]) for t in probs),
                max(int(t[4]) for t in probs), max(int(t[2]) for t in probs), max(int(t[3]) for t in probs))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            rc = rq_tuxv_batched(h.h, RQ_FP32, len(probs), desc, *dims)
        if rc != 0:
            raise RuntimeError(f"rq_tuxv_batched failed under capture with status {rc}")
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1) / steps
        graph = {"graph_s": gms / 1e3, "graph_problems_per_s": len(probs) / (gms / 1e3)}
    except Exception as exc:  # context only
        graph = {"graph_error": f"{type(exc).__name__}: {exc}"[:200]}
    flops = sum(4.0 * k * A.shape[0] * A.shape[1] + 2.0 * (b + p) * A.shape[0] * A.shape[1] for A, Om, b, p, k in probs)
    byts = sum(4.0 * A.shape[0] * A.shape[1] * (3 + (k + b - 1) // b) for A, Om, b, p, k in probs)
    out = {"workload": f"batched_tuxv_{len(probs)}_problems", "problems": len(probs), "s": ms / 1e3,
           "problems_per_s": len(probs) / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12,
           "gbs_algorithmic": byts / (ms / 1e3) / 1e9, "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm_peak_gbs()[0],
           "info_nonzero": int((info != 0).sum()), **tuning, **graph,
           "call_s": call_ms / 1e3, "call_problems_per_s": len(probs) / (call_ms / 1e3),
           "mixed": {"s": mms / 1e3, "problems_per_s": len(probs) / (mms / 1e3), "info_nonzero": int((minfo != 0).sum())}}
    g = np.random.default_rng(0)
    idx = g.choice(len(probs), size=min(quality_sample, len(probs)), replace=False)
    arms = {"fp32": outs, "mixed": mouts}
    if fp64:
        # the plain FP64 path: rq_tuxv in FP64 on every problem, one after another
        import torch as _t
        from paper_2008_04447_gb300 import colmajor
        d64 = [(colmajor(_t.as_tensor(host[i][0])).cuda(), colmajor(_t.as_tensor(host[i][1])).cuda(),
                host[i][2], host[i][3], host[i][4]) for i in order]
        for A, Om, b, p, k in d64[:16]:
            h.tuxv(A, Om, b, p, k)
        _t.cuda.synchronize()
        e0.record()
        o64 = [h.tuxv(A, Om, b, p, k)[:3] for A, Om, b, p, k in d64]
        e1.record()
        _t.cuda.synchronize()
        f64ms = e0.elapsed_time(e1)
        out["fp64"] = {"s": f64ms / 1e3, "problems_per_s": len(probs) / (f64ms / 1e3),
                       "path": "rq_tuxv FP64 per problem, one stream"}
        out["fp32_over_fp64_throughput"] = f64ms / ms
        arms["fp64"] = o64
    rows = _rank_k_errors(host, order, idx, arms)
    if fp64 and rows:
        r32 = [r["fp32"] / r["fp64"] for r in rows if r["fp64"] > 0]
        rmx = [r["mixed"] / r["fp64"] for r in rows if r["fp64"] > 0]
        out["error_over_fp64_path"] = {"n": len(r32), "fp32_max": max(r32), "fp32_median": float(np.median(r32)),
                                       "mixed_max": max(rmx), "mixed_median": float(np.median(rmx))}
    # rank-k error over the optimal rank-k error (Eckart-Young) of the FP32 results
    opt = []
    for j, row in zip([j for j in idx if host[order[j]][0].size <= 600 * 400], rows):
        a, k = host[order[j]][0], host[order[j]][4]
        sv = np.linalg.svd(a, compute_uv=False)
        e_opt = float(np.sqrt(np.sum(sv[k:] ** 2))) / float(np.linalg.norm(a))
        if e_opt > 0:
            opt.append(row["fp32"] / e_opt)
    out["error_over_svd_optimum"] = {"n": len(opt), "median": float(np.median(opt)) if opt else None,
                                     "max": float(np.max(opt)) if opt else None}
    return out


def leg_serving(dev, rates=(100, 200, 500, 1000, 2000, 5000), seconds=1.0, large_frac=0.1, budget=120e9,
                tiles=None, host=None, quality_sample=12, prec=None):
    """Poisson arrivals of TUXV requests: the batch mix plus 10% 8192 x 4096, k = 256
    (tiles: the batched kernel's tile policy for the server's lanes).  prec:
    RQ_FP32 (default; small requests batched, large ones through rq_tuxv) or
    RQ_FP64 (dev then holds FP64 inputs; every request through rq_tuxv)."""
    import numpy as np
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, RQ_FP64, Handle, colmajor
    from paper_2008_04447_gb300 import inputs as I
    from paper_2008_04447_gb300.serve import Server
    prec = RQ_FP32 if prec is None else prec
    dt_big = torch.float64 if prec == RQ_FP64 else torch.float32
    big = [(colmajor(I.lowrank_plus_noise_torch(8192, 4096, 1024, 1e-6, seed=40 + i).to(dt_big)),
            colmajor(I.omega_torch(72, 8192, seed=50 + i, dtype=dt_big)), 64, 8, 256) for i in range(2)]
    import sys
    results = []
    g = np.random.default_rng(1)
    # the client sleeps until just before each arrival and the interpreter
    # switches threads every 0.1 ms, so the load generator does not starve the
    # server's scheduling thread of the GIL
    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    for rate in rates:
        srv = Server(budget_bytes=budget, lanes=3, tiles=tiles, prec=prec)
        # warm the lanes' workspaces
        for lane_h, st in srv.lanes:
            if prec != RQ_FP64:
                lane_h.tuxv_batched(dev[:8], stream=st, prec=prec)
            lane_h.tuxv(*big[0][:2], 64, 8, 256, stream=st, prec=prec)
        torch.cuda.synchronize()
        srv.start()
        n = max(20, int(rate * seconds))
        gaps = g.exponential(1.0 / rate, size=n)
        t0 = time.perf_counter()
        tnext = t0
        reqs, sources = [], []
        for i in range(n):
            tnext += gaps[i]
            dt = tnext - time.perf_counter()
            if dt > 3e-4:
                time.sleep(dt - 2e-4)
            while time.perf_counter() < tnext:
                pass
            src = None
            if g.random() < large_frac:
                A, Om, b, p, k = big[i % len(big)]
            else:
                src = int(g.integers(len(dev)))
                A, Om, b, p, k = dev[src]
            reqs.append(srv.submit(A, Om, b, p, k))
            sources.append(src)
        for r in reqs:
            r.wait(300)
        srv.stop()
        st_ = srv.stats()
        st_["offered_rate"] = rate
        results.append(st_)
        torch.cuda.synchronize()
    sys.setswitchinterval(old_switch)
    out = {"workload": "poisson TUXV requests: 90% batch mix (m<=2048, n<=1024, k<=128), 10% 8192x4096 k=256",
           "prec": {RQ_FP32: "fp32", RQ_FP64: "fp64"}.get(prec, str(prec)), "budget_gb": budget / 1e9,
           "by_rate": results}
    # quality of served results (last rate), on a sample of the small requests:
    # the rank-k error (FP64, against the FP64 input) over that of the FP64 path
    # (rq_tuxv in FP64 on the same problem) and over the optimal rank-k error
    # (numpy's SVD of the FP64 input)
    if host is not None and prec != RQ_FP64:
        h64 = Handle()
        r64, ropt = [], []
        small = [(r, j) for r, j in zip(reqs, sources) if j is not None
                 and host[j][0].shape[0] * host[j][0].shape[1] <= 600 * 400]
        for r, j in small[:quality_sample]:
            a, om, b, p, k = host[j]
            na = float(np.linalg.norm(a))
            U, X, V = (t.cpu().double().numpy() for t in r.out)
            e = float(np.linalg.norm(a - U @ X @ V.T)) / na
            U6, X6, V6, _, _ = h64.tuxv(colmajor(torch.as_tensor(a)).cuda(), colmajor(torch.as_tensor(om)).cuda(),
                                        b, p, k)
            U6, X6, V6 = (t.cpu().numpy() for t in (U6, X6, V6))
            e64 = float(np.linalg.norm(a - U6 @ X6 @ V6.T)) / na
            sv = np.linalg.svd(a, compute_uv=False)
            e_opt = float(np.sqrt(np.sum(sv[k:] ** 2))) / na
            if e64 > 0:
                r64.append(e / e64)
            if e_opt > 0:
                ropt.append(e / e_opt)
        h64.close()
        out["error_over_fp64_path"] = {"n": len(r64), "median": float(np.median(r64)) if r64 else None,
                                       "max": float(np.max(r64)) if r64 else None}
        out["error_over_svd_optimum"] = {"n": len(ropt), "median": float(np.median(ropt)) if ropt else None,
                                         "max": float(np.max(ropt)) if ropt else None}
    return out


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
    if args.sweep:
        run_sweep(args)
        return
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
    if args.only_batched or args.only == "batched":
        host = batch_inputs(args.batch, seed=0)
        print(json.dumps({"batched": leg_batched(Handle(), host, to_device_f32(host), quality_sample=0, tune=not args.no_tune)}), flush=True)
        return
    if args.only == "serving":
        host = batch_inputs(args.batch, seed=0)
        print(json.dumps({"serving": leg_serving(to_device_f32(host), host=host)}), flush=True)
        return
    if args.only == "fp64peak":
        print(json.dumps({"fp64_peak": leg_fp64_peak()}), flush=True)
        return
    if args.only == "tuxv":
        shape = tuple(int(x) for x in args.tuxv_shape.split(","))
        print(json.dumps({"tuxv": leg_tuxv(Handle(), steps=args.steps, warmup=args.warmup, shape=shape)}), flush=True)
        return
    n, b, p = args.n, args.b, args.p
    m = n
    l = b + p
    fl = flops_qr(m, n)

    A0 = colmajor(I.graded_torch(m, n, args.decades, seed=rank))          # pristine FP64 input
    Om = colmajor(I.omega_torch(l, m, seed=1000 + rank))
    if args.prec == "fp32":
        A0 = colmajor(A0.float())
        Om = colmajor(Om.float())
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
    f64_tc = args.prec == "fp64" and os.environ.get("RQ_F64_TC", "2")[:1] not in ("0", "1")
    if f64_tc and tr[0] > 0:
        # the FP64 block reflector products run as bfloat16 slice-pair MMAs (oz_gemm_kernel)
        pk, pk_src = bf16_peak_tflops()
        tc_rate = slice_pair_flops(m, n, b) * args.steps / (tr[0] / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": tc_rate, "peak": pk, "unit": "TFLOP/s", "frac": tc_rate / pk,
                    "traffic": OZ_DRAM_BYTES_PER_ENTRY * trailing_entries(m, n, b),
                    "traffic_scope": "DRAM bytes per step of the two tensor-core products (W and the update), "
                                     "scaled by m_t n2 from an ncu capture of a 6144^2 factorisation",
                    "kernel": "trailing update: oz_gemm_kernel (FP64 block reflector products as 36 bfloat16 "
                              "slice-pair MMAs) + the Y T product; operand slicing is its own phase",
                    "achieved_is": "bfloat16 slice-pair flops per second over the trailing phase's CUDA-event time",
                    "fp64_equivalent_tflops": achieved, "frac_of_fp64_pipe": achieved / FP64_PEAK_TFLOPS,
                    "algorithmic_bytes": tr[2] / args.steps, "peak_source": pk_src}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                    "algorithmic_bytes": tr[2] / args.steps,
                    "kernel": "trailing update (block reflector GEMMs), FP64 pipe",
                    "peak_source": "derived: 152 SMs x 2070 MHz x 2 DFMA/clk/SM x 2 flop (FP64 pipe, nominal)"}

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": f"rqrcp_{args.prec}_graded_{m}x{n}_b{b}_p{p}", "m": m, "n": n, "b": b, "p": p, "k": n,
                       "spectrum": f"U diag(10^(-{args.decades:g} i/n)) V^T, Haar U, V",
                       "l2": "inputs larger than L2 (A is 2.1 GB)",
                       "step": "device copy restoring A (2.1 GB) + rq_rqrcp", "parallelism": f"replicas x{ws}"},
            "rqrcp_s": ms_step / 1e3, "roofline": roofline, "phases": phases, "gpu_launches": launches,
            "clocks": clocks}

    if args.prec == "fp32":
        peak, src = hbm_peak_gbs()
        roofline.update({"bound": "hbm", "peak": peak, "unit": "GB/s", "achieved": tr[2] / (tr[0] / 1e3) / 1e9,
                         "kernel": "trailing update (tensor-core 3xTF32 GEMMs), FP32", "peak_source": src})
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
    legs = args.legs if rank == 0 else set()
    if "e2e" in legs:
        try:
            # end to end through the C ABI with host buffers (pinned; column-major A is
            # copied as its contiguous transpose so each copy is one cudaMemcpyAsync)
            Ah = torch.empty((n, m), dtype=A0.dtype, pin_memory=True)
            Ah.copy_(A0.t())
            Ao = torch.empty((n, m), dtype=A0.dtype, pin_memory=True)
            tau_h = torch.empty(n, dtype=A0.dtype, pin_memory=True)
            jp_h = torch.empty(n, dtype=torch.int32, pin_memory=True)

            from paper_2008_04447_gb300 import rq_copy
            nbytes = A0.element_size() * m * n

            def e2e_step(sm_copy):
                # the 2.1 GB transfers by the library's SM copy (rq_copy) or the copy engines
                if sm_copy:
                    rc = rq_copy(A, Ah, nbytes, torch.cuda.current_stream().cuda_stream)
                    if rc != 0:
                        raise RuntimeError(f"rq_copy failed with status {rc}")
                else:
                    A.t().copy_(Ah, non_blocking=True)
                tau, jpvt, info = h.rqrcp(A, Om, b, p)
                if sm_copy:
                    rc = rq_copy(Ao, A, nbytes, torch.cuda.current_stream().cuda_stream)
                    if rc != 0:
                        raise RuntimeError(f"rq_copy failed with status {rc}")
                else:
                    Ao.copy_(A.t(), non_blocking=True)
                tau_h.copy_(tau, non_blocking=True)
                jp_h.copy_(jpvt, non_blocking=True)

            def e2e_run(sm_copy):
                e2e_step(sm_copy)
                torch.cuda.synchronize()
                eclk = Clocks(local)
                eclk.start()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                ev0.record()
                E = 2
                for _ in range(E):
                    e2e_step(sm_copy)
                ev1.record()
                torch.cuda.synchronize()
                return (time.perf_counter() - t0) / E, ev0.elapsed_time(ev1) / 1e3 / E, eclk.stop()

            e2e_s, e2e_dev_s, e2e_clocks = e2e_run(True)
            esz = A0.element_size()
            line["e2e"] = {"value": fl / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": esz * m * n,
                           "d2h_bytes_per_step": esz * m * n + (esz + 4) * n, "s_per_step": e2e_s,
                           "device_s_per_step": e2e_dev_s, "clocks": e2e_clocks,
                           "copies": "A in and R out by rq_copy (SM loads and stores through the pinned "
                                     "buffers' device mapping); tau and jpvt by cudaMemcpyAsync"}
            ce_s, ce_dev_s, _ = e2e_run(False)
            line["e2e"]["copy_engine"] = {"value": fl / ce_s / 1e12, "s_per_step": ce_s,
                                          "device_s_per_step": ce_dev_s}
            Ah_check = Ao.clone()
            e2e_step(True)
            torch.cuda.synchronize()
            line["e2e"]["sm_copy_matches_copy_engine"] = bool(torch.equal(Ao, Ah_check))
            del Ah_check
            del Ah, Ao
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["e2e"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()

    if "qr" in legs:
        try:
            # unpivoted blocked QR of the same matrix, same kernels (the paper's comparison)
            def qr_step():
                A.copy_(A0)
                h.qr(A, b)
            qr_step()
            torch.cuda.synchronize()
            qclk = Clocks(local)
            qclk.start()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record()
            for _ in range(2):
                qr_step()
            q1.record()
            torch.cuda.synchronize()
            qr_ms = q0.elapsed_time(q1) / 2
            line["qr"] = {"s": qr_ms / 1e3, "tflops": fl / (qr_ms / 1e3) / 1e12,
                          "rqrcp_over_qr": ms_step / qr_ms, "clocks": qclk.stop()}
            try:
                # cuSOLVER's geqrf (through torch) on the same matrix, as context
                torch.geqrf(A0)
                torch.cuda.synchronize()
                q0.record()
                torch.geqrf(A0)
                q1.record()
                torch.cuda.synchronize()
                g_ms = q0.elapsed_time(q1)
                line["qr"].update({"cusolver_geqrf_s": g_ms / 1e3, "cusolver_geqrf_tflops": fl / (g_ms / 1e3) / 1e12,
                                   "rqrcp_over_cusolver_geqrf": ms_step / g_ms})
            except Exception as exc:  # context only
                line["qr"]["cusolver_geqrf_error"] = f"{type(exc).__name__}: {exc}"[:200]
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["qr"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()

    if "fp32" in legs and args.prec == "fp64":
        try:
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
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["fp32"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()

    if "rsrqrcp" in legs:
        try:
            # ablation of the sample update (Sec. 3.4): repeated sampling re-sketches the
            # trailing matrix with fresh device draws at every block; same matrix
            line["rsrqrcp"] = leg_rsrqrcp(h, A0, A, Om, b, p, fl, ms_step, args.prec)
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["rsrqrcp"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()

    if "cpu" in legs:
        try:
            line["cpu_baseline"] = cpu_baseline(args.cpu_n, b, p, args.decades)
            line["cpu_context"] = cpu_context()
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line.setdefault("cpu_baseline", {"error": f"{type(exc).__name__}: {exc}"[:300]})
            line["cpu_context"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()
    del A0, A
    torch.cuda.empty_cache()
    if "fp64peak" in legs:
        try:
            pk = leg_fp64_peak()
            line["fp64_peak"] = pk
            if args.prec == "fp64" and achieved:
                # FP64 rate of the trailing update over cuBLAS DGEMM's on this GPU
                roofline["fp64_over_cublas_dgemm"] = achieved / pk["cublas_dgemm_tflops"]
        except Exception as exc:  # context only
            line["fp64_peak"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    if "slices" in legs:
        try:
            line["slices"] = leg_slices(h)
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["slices"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    if "tuxv" in legs:
        try:
            line["tuxv"] = leg_tuxv(h)
            torch.cuda.empty_cache()
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["tuxv"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()
    if "batched" in legs or "serving" in legs:
        try:
            host = batch_inputs(args.batch, seed=0)
            dev = to_device_f32(host)
            if "batched" in legs:
                line["batched"] = leg_batched(h, host, dev, tune=not args.no_tune)
            if "serving" in legs:
                line["serving"] = leg_serving(dev, tiles=line.get("batched", {}).get("tiles"), host=host)
            del dev
            torch.cuda.empty_cache()
            if "serving" in legs:
                # the plain FP64 path under the same arrivals (every request through rq_tuxv)
                from paper_2008_04447_gb300 import RQ_FP64
                d64 = [(colmajor(torch.as_tensor(a)).cuda(), colmajor(torch.as_tensor(om)).cuda(), bb, pp, kk)
                       for a, om, bb, pp, kk in host]
                s64 = leg_serving(d64, rates=(100, 500, 1000), prec=RQ_FP64)
                line["serving"]["fp64"] = s64
                by32 = {r["offered_rate"]: r for r in line["serving"]["by_rate"]}
                line["serving"]["fp32_over_fp64"] = [
                    {"offered_rate": r["offered_rate"],
                     "req_per_s": by32[r["offered_rate"]]["req_per_s"] / r["req_per_s"],
                     "p99": by32[r["offered_rate"]]["p99_ms"] / r["p99_ms"]}
                    for r in s64["by_rate"] if r["offered_rate"] in by32]
                del d64
        except Exception as exc:  # a failing extra leg must not lose the headline line
            line["batched+serving"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()
    barrier(ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
