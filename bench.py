"""Benchmark of the randomized block Krylov truncated T-SVD (arXiv 2504.04989).

Workload (one step = one whole T-SVD, every stage of Alg. 2): the video-like
2048 x 2048 x 128 float32 tensor with per-Fourier-slice singular values
sigma_i = 1/i plus Gaussian noise of 1e-4 x the RMS entry, R = 100, P = 20,
q = 3, synthetic (seeded), the input resident in HBM.  Metric: rank-R T-SVD
approximations per second on the mixed-precision path (Krylov products on the
tensor cores in TF32), next to the FP64 path on the same tensor at equal
reconstruction error, and the t-product TFLOP/s on the paper-shaped products.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32|bf16|fp32|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Under torchrun every rank runs its own independent tensor (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="video-like 2048x2048x128 fp32, sigma_i=1/i + noise 1e-4 x RMS, R=100 P=20 q=3",
                n1=2048, n2=2048, n3=128, R=100, P=20, q=3)
C2 = dict(name="image-like 512x512x64 fp32, sigma_i=i^-1.5 full rank, R=50 P=10 q=4",
          n1=512, n2=512, n3=64, R=50, P=10, q=4)
METRIC = "rank-R T-SVD approximations/s"
DF_FMA_INSTR = 15  # FP32 instructions per double-float multiply-add (TwoProduct, cross terms, TwoSum, renormalisation)
# DRAM bytes per launch of a kernel from an ncu capture, valid only while the
# source file the capture was taken on is unchanged (sha256 prefix of that
# file); reported as null otherwise.  eig_hetrd: the double-float
# tridiagonalisation with its rows in L2 for m = 480 on 65 Fourier slices (the
# eigen-problem of the 2048 x 2048 x 128 workload, captured on a 512 x 512 x 128
# tensor with the same R, P, q, whose eigen-problem has the same sizes).
NCU_TRAFFIC = {"eig_hetrd": {"src": "paper_2504_04989_gb300/csrc/eig.cu", "sha16": "6cdc60faafe65bcc",
                             "bytes_per_launch": 5.819092e9 + 11.789736e9}}


def peaks_file():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


def src_sha16(relpath):
    try:
        return hashlib.sha256(open(os.path.join(ROOT, relpath), "rb").read()).hexdigest()[:16]
    except OSError:
        return None


def ncu_traffic(stage):
    t = NCU_TRAFFIC.get(stage)
    if t and src_sha16(t["src"]) == t["sha16"]:
        return t["bytes_per_launch"]
    return None


def measure_alu_peaks(torch, dev, stream):
    """Dense-matmul peaks measured here (cuBLAS, the same kind of denominator as
    the driver's bf16 number): FP64, FP32 without TF32 and TF32, TFLOP/s."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, n, tf32 in (("fp64", torch.float64, 8192, False), ("fp32", torch.float32, 8192, False),
                              ("tf32", torch.float32, 8192, True)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        c = a @ b
        torch.cuda.synchronize(dev)
        reps = 3 if name == "fp64" else 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out[name] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = prev
    out["double_float"] = out["fp32"] / DF_FMA_INSTR * 2  # FP64-accuracy flops on the FP32 pipe
    return out


def algorithmic(stage, d, precision):
    """Algorithmic work of one stage for one T-SVD (flops; bytes for transforms)."""
    n1, n2, n3, R, b, m = d["n1"], d["n2"], d["n3"], d["R"], d["R"] + d["P"], d["m"]
    h = n3 // 2 + 1
    q = d["q"]
    cm = 8.0  # real flops per complex multiply-add
    blocks = [min(b, m - i * b) for i in range(q + 1) if i * b < m]
    c_before = np.cumsum([0] + blocks[:-1])
    if stage == "eig_hetrd":      # Householder tridiagonalisation of the m x m Hermitian Gram
        return {"flops": 16.0 / 3.0 * m ** 3 * h}
    if stage == "gram_c":         # G = C C^H (Hermitian: half of the m x m outputs)
        return {"flops": cm * n2 * m * (m + 1) / 2 * h}
    if stage == "orth_cgs":       # two classical Gram-Schmidt sweeps per block pass (3 passes)
        return {"flops": sum(3 * 2 * cm * n1 * c * nb for c, nb in zip(c_before, blocks)) * h}
    if stage == "orth_gram":
        return {"flops": sum(3 * cm * n1 * nb * (nb + 1) / 2 for nb in blocks) * h}
    if stage == "orth_trsm":
        return {"flops": sum(3 * cm * n1 * nb * nb / 2 for nb in blocks) * h}
    if stage in ("krylov_gemm", "krylov_gemm_tc"):  # A Omega, A^H Q and A Y per Krylov step, the last A^H Q
        return {"flops": cm * n1 * n2 * (sum(blocks) + sum(blocks[:-1]) + blocks[-1]) * h}
    s = 8 if precision == "fp64" else 4
    if stage == "rfft":
        return {"bytes": s * (n1 * n2 * n3 + 2 * n1 * n2 * h)}
    if stage == "irfft":
        return {"bytes": s * (2 * (n1 + n2) * R * h + (n1 + n2) * R * n3)}
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_slices(X, d, slices):
    """The FP64 CPU oracle, as it stands, on the listed Fourier slices of one
    T-SVD of X (each slice: its DFT, the Krylov basis, the projection and the
    small SVD; OpenMP across the slices).  Returns the wall time."""
    import oracle
    t0 = time.perf_counter()
    oracle.rtsvd_fourier(X, d["R"], d["P"], d["q"], seed=0, slices=list(slices))
    return time.perf_counter() - t0, oracle.num_threads()


def cpu_baseline(X, d):
    """One full wave of the oracle: as many Fourier slices as host threads, run
    at once by the oracle's loop over slices.  value = the T-SVD work done
    (slices / h) / wall time; a single T-SVD needs ceil(h / threads) waves."""
    import oracle
    h = d["n3"] // 2 + 1
    cores = oracle.num_threads()
    ns = min(cores, h)
    dt, cores = oracle_slices(X, d, range(ns))
    return {"value": (ns / h) / dt, "unit": "T-SVD/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the %d Fourier slices of one T-SVD (their DFT, Krylov basis, projection and SVD; FP64), "
                      "run at once on %d host threads in %.1f s; value = (%d/%d T-SVD) / wall time; one whole T-SVD "
                      "takes ceil(%d/%d) = %d such waves, %.0f s" % (ns, h, cores, dt, ns, h, h, cores,
                                                                    math.ceil(h / cores), math.ceil(h / cores) * dt),
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


def run_reference(args, d, rank, world):
    """The oracle on the bench workload: W warm-up steps, then K timed steps,
    each step the oracle's Alg. 2 on one Fourier slice (1/h of a T-SVD); the K
    steps go to the oracle's OpenMP loop over slices as one call, timed as a
    whole."""
    if rank != 0:
        return
    from paper_2504_04989_gb300 import workloads as wl
    X = wl.make_c3(0).astype(np.float64)
    h = d["n3"] // 2 + 1
    if args.warmup > 0:
        oracle_slices(X, d, [i % h for i in range(args.warmup)])
    dt, cores = oracle_slices(X, d, [(args.warmup + i) % h for i in range(args.steps)])
    val = (args.steps / h) / dt
    sample = ("each step: the oracle's Alg. 2 on one of the %d Fourier slices of one T-SVD (1/%d of the T-SVD: "
              "the slice's DFT, Krylov basis, projection, SVD; FP64); the %d steps run as one call of the oracle's "
              "OpenMP loop over slices on %d threads, %.1f s wall" % (h, h, args.steps, cores, dt))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "T-SVD/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": d["name"], "precision": "fp64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": "T-SVD/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": val, "unit": "T-SVD/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, device=None):
    """The largest x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, world, seconds):
    """Whole-job throughput: every rank runs `steps` units of its own tensor
    (weak scaling), timed by the slowest rank."""
    return world * steps / seconds


def timed_calls(torch, fn, k, flush, stream, dev):
    """k calls of fn, each bracketed by CUDA events on `stream` after an L2
    flush; mean milliseconds."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize(dev)
    return sum(a.elapsed_time(b) for a, b in ev) / k


def batched_bench(api, wl, dev, count, lanes, steps, flush, stream):
    """Uneven batch (n1, n2 ~ U{32..512}, n3 ~ U{8,16,32,64}, tubal rank
    r ~ U{5..40}, R = r, P = 5, q = 2, FP32): `count` tensors as one
    tsvd_rbk_batched call over `lanes` streams, captured in a CUDA graph and
    replayed; also one eager single-stream pass for comparison."""
    import torch
    items = wl.make_c4(0, count)
    shapes = [(it["X"].shape[1], it["X"].shape[2], it["X"].shape[0]) for it in items]
    Rs = [it["R"] for it in items]
    xs = [torch.from_numpy(it["X"].astype(np.float32)).to(dev) for it in items]
    del items
    eager = api.RbkBatchPlan(shapes, Rs, P=5, q=2, seed=0, precision="fp32", lanes=1, device=dev)
    eager(xs)
    ms_eager = timed_calls(torch, eager, 1, flush, stream, dev)
    del eager
    plan = api.RbkBatchPlan(shapes, Rs, P=5, q=2, seed=0, precision="fp32", lanes=lanes, device=dev, graph=True)
    plan(xs)
    torch.cuda.synchronize(dev)
    timed_calls(torch, plan, 1, flush, stream, dev)
    ms = timed_calls(torch, plan, steps, flush, stream, dev)
    return {"workload": "uneven batch: n1, n2 ~ U{32..512}, n3 ~ U{8,16,32,64}, rank ~ U{5..40}, P=5, q=2, fp32",
            "tensors": count, "lanes": lanes, "graph": True, "ms_per_batch": ms,
            "tsvd_per_s": count * 1000.0 / ms, "eager_single_stream_ms": ms_eager}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-count", type=int, default=256,
                    help="tensors of the uneven batch timed after the main workload (0: skip)")
    ap.add_argument("--n", type=int, default=2048,
                    help="n1 = n2 of the main workload (smaller cases for profiling; n3, R, P, q unchanged)")
    ap.add_argument("--quick", action="store_true",
                    help="only the main path (and its end-to-end and stage times): no other paths, peaks, "
                         "t-products or batch")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    d = dict(WORKLOAD)
    if args.n != 2048:
        d.update(n1=args.n, n2=args.n, name=d["name"].replace("2048x2048", "%dx%d" % (args.n, args.n)))
    d["m"] = min((d["q"] + 1) * (d["R"] + d["P"]), d["n1"], d["n2"])
    if args.impl == "reference":
        return run_reference(args, d, rank, world)

    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2504_04989_gb300 import api
    from paper_2504_04989_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    X = wl.make_c3(seed=rank, n=d["n1"])             # float32 (n3, n1, n2), 2.1 GB at n = 2048
    Xd = torch.from_numpy(X).to(dev)
    if args.precision == "fp64":
        Xd = Xd.double()
    n1, n2, n3, R, P, q = (d[k] for k in ("n1", "n2", "n3", "R", "P", "q"))
    plan = api.RbkPlan(n1, n2, n3, R, P, q, seed=0, precision=args.precision, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        plan(Xd)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        l0 = api.launch_count()
        for a, b in ev:
            flush.zero_()          # evict the previous step's working set from L2
            a.record(stream)
            plan(Xd)
            b.record(stream)
        barrier()
        launches_timed = api.launch_count() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(step_ms) / 1000.0, dev)
    value = job_value(args.steps, world, total_s)
    ms_step = 1000 * total_s / args.steps

    # end to end through the public API: pinned host input -> device -> T-SVD -> host outputs
    Xh = torch.from_numpy(X).pin_memory() if args.precision != "fp64" else torch.from_numpy(
        X.astype(np.float64)).pin_memory()
    outs_h = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (plan.U, plan.S, plan.V, plan.sig)]
    Xe = torch.empty_like(Xd)
    h2d = Xh.numel() * Xh.element_size()
    d2h = sum(t.numel() * t.element_size() for t in outs_h)
    barrier()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in e2e_ev:
        flush.zero_()
        a.record(stream)
        Xe.copy_(Xh, non_blocking=True)
        U, S, V, sg = plan(Xe)
        for src, dst in zip((U, S, V, sg), outs_h):
            dst.copy_(src, non_blocking=True)
        b.record(stream)
    barrier()
    e2e_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1000.0, dev)
    e2e_value = job_value(args.steps, world, e2e_s)
    del Xe, Xh

    # per-stage times (CUDA events recorded by the library on this stream)
    with api.profile() as pr:
        for _ in range(2):
            flush.zero_()
            plan(Xd)
    stages = {k: v[0] / 2 for k, v in pr.stages.items()}
    dom = max(stages, key=stages.get)
    pk = peaks_file()
    props = torch.cuda.get_device_properties(dev)
    alu = measure_alu_peaks(torch, dev, stream) if not args.quick else \
        {"fp64": None, "fp32": None, "tf32": None, "double_float": None}

    def roofline_of(stage):
        work = algorithmic(stage, d, args.precision)
        t = stages[stage] * 1e-3
        if "flops" in work:
            if args.precision == "fp64":
                peak, src = alu["fp64"], "measured here: cuBLAS FP64 GEMM"
            elif stage == "eig_hetrd":
                peak, src = alu["double_float"], "measured FP32 GEMM rate / 15 instructions per double-float FMA x 2"
            elif stage == "krylov_gemm_tc":
                peak, src = alu["tf32"], "measured here: cuBLAS TF32 GEMM"
            elif stage in ("orth_gram", "orth_trsm", "orth_cgs") and d["n1"] >= 1024:
                # tcgen05 in split TF32 from n1 = 1024 on: three TF32 products per FP32-accurate one
                peak, src = alu["tf32"] and alu["tf32"] / 3, "measured here: cuBLAS TF32 GEMM / 3 (split TF32)"
            elif stage == "gram_c" and d["n2"] <= 4096:
                # the exact Gram in base-64 digits on the BF16 tensor cores: of the 16 digit-pair
                # products about 8 are computed (the symmetric half skipped)
                peak = pk.get("bf16_tflops")
                peak, src = peak and peak / 8, "MEASURED_PEAKS.json bf16_tflops / 8 (digit-pair products)"
            else:
                peak, src = alu["fp32"], "measured here: cuBLAS FP32 GEMM (no TF32)"
            a = work["flops"] / t / 1e12
            return {"kernel": stage, "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                    "frac": a / peak if peak else None, "traffic": ncu_traffic(stage), "peak_source": src}
        if "bytes" in work:
            a = work["bytes"] / t / 1e9
            return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": a / pk["hbm_gbs"], "traffic": ncu_traffic(stage),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
        return None

    roof = roofline_of(dom) or {"kernel": dom, "bound": None}
    roof["stage_ms"] = {k: round(v, 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1])}
    roof["stages"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in r.items()
                          if kk in ("bound", "achieved", "peak", "unit", "frac")}
                      for k in stages for r in [roofline_of(k)] if r}
    roof["measured_peaks_tflops"] = {k: (round(v, 2) if v else None) for k, v in alu.items()}
    roof["sms"] = props.multi_processor_count

    # reconstruction errors: this path, the other mixed path, the configuration's
    # FP64 orthonormalisation, and the FP64 path on the same (FP32-rounded) tensor
    X64 = Xd.double() if Xd.dtype != torch.float64 else Xd
    xnorm2 = float(torch.linalg.vector_norm(X64) ** 2)

    def rel_err(pl):
        e2 = api.tsvd_error(X64, pl.U.double(), pl.S.double(), pl.V.double(), "fp64").item()
        return math.sqrt(max(e2, 0.0) / xnorm2)

    err_this = rel_err(plan)
    paths = {"this": {"precision": args.precision, "ms_per_tsvd": ms_step, "rel_error": err_this}}
    del plan
    torch.cuda.empty_cache()

    def time_path(tag, precision, k, xin, **kw):
        pl = api.RbkPlan(n1, n2, n3, R, P, q, seed=0, precision=precision, device=dev, **kw)
        pl(xin)
        torch.cuda.synchronize(dev)
        ms = timed_calls(torch, lambda: pl(xin), k, flush, stream, dev)
        paths[tag] = {"ms_per_tsvd": ms, "tsvd_per_s": 1000.0 / ms, "rel_error": rel_err(pl)}
        del pl
        torch.cuda.empty_cache()

    X32 = Xd if Xd.dtype == torch.float32 else Xd.float()
    if args.quick:  # the main path only
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "T-SVD/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "data": "synthetic", "config": {"workload": d["name"], "precision": args.precision},
                              "e2e": {"value": e2e_value, "unit": "T-SVD/s", "h2d_bytes_per_step": h2d,
                                      "d2h_bytes_per_step": d2h},
                              "gpu_launches": launches_timed, "roofline": roof, "paths": paths}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    for prec in ("tf32", "bf16", "fp32"):
        if prec != args.precision:
            time_path(prec, prec, 3, X32)
    time_path(args.precision + "+fp64_qr" if args.precision != "fp64" else "tf32+fp64_qr",
              args.precision if args.precision != "fp64" else "tf32", 2, X32, fp64_qr=True)
    time_path("alg1_" + ("tf32" if args.precision == "fp64" else args.precision),
              "tf32" if args.precision == "fp64" else args.precision, 3, X32, alg1=True)
    if args.precision != "fp64":
        time_path("fp64", "fp64", 2, X64)
        e64 = paths["fp64"]["rel_error"]
        paths["speedup_vs_fp64"] = paths["fp64"]["ms_per_tsvd"] / ms_step
        paths["error_rel_diff_vs_fp64"] = abs(err_this - e64) / e64
        paths["equal_error"] = abs(err_this - e64) / e64 <= 1e-3
    del X64

    # the image-like 512 x 512 x 64 configuration (FP32 and FP64 paths) with its Eckart-Young optimum
    Xc2 = torch.from_numpy(wl.make_c2(0).astype(np.float32)).to(dev)
    c2 = {}
    for prec in ("fp32", "fp64"):
        xin = Xc2 if prec == "fp32" else Xc2.double()
        pl = api.RbkPlan(512, 512, 64, 50, 10, 4, seed=0, precision=prec, device=dev)
        pl(xin)
        torch.cuda.synchronize(dev)
        ms = timed_calls(torch, lambda: pl(xin), 5 if prec == "fp32" else 2, flush, stream, dev)
        e2 = api.tsvd_error(Xc2.double(), pl.U.double(), pl.S.double(), pl.V.double(), "fp64").item()
        c2[prec] = {"ms_per_tsvd": ms, "rel_error": math.sqrt(e2) / float(torch.linalg.vector_norm(Xc2.double()))}
        del pl
    c2["eckart_young_optimum_rel_error"] = float(np.sqrt(wl.optimal_error2(wl.c2_sigma(512), 50)) /
                                                 torch.linalg.vector_norm(Xc2.double()).item())
    c2["workload"] = C2["name"]
    paths["c2"] = c2
    del Xc2

    # t-product throughput on the paper-shaped products (flops 8 n1 n2 n4 h, whole call incl. FFTs)
    tprod_tflops = {}
    for name, a1, a2, a4, a3 in (("2048x2048x128*2048x120x128", 2048, 2048, 120, 128),
                                 ("1024x1024x64*1024x1024x64", 1024, 1024, 1024, 64),
                                 ("256x20x100*20x256x100", 256, 20, 256, 100)):
        fl = 8.0 * a1 * a2 * a4 * (a3 // 2 + 1)
        row = {}
        for prec in ("fp64", "fp32", "tf32x3", "tf32", "bf16"):
            dt = torch.float64 if prec == "fp64" else torch.float32
            A = torch.randn(a3, a1, a2, device=dev, dtype=dt)
            B = torch.randn(a3, a2, a4, device=dev, dtype=dt)
            api.tprod(A, B, prec)
            ts = []
            for _ in range(3):
                ts.append(timed_calls(torch, lambda: api.tprod(A, B, prec), 1, flush, stream, dev))
            row[prec] = round(fl / (min(ts) * 1e-3) / 1e12, 3)
            del A, B
        tprod_tflops[name] = row

    batched = None
    if args.batched_count > 0 and args.precision != "fp64":
        batched = batched_bench(api, wl, dev, args.batched_count, 8, 3, flush, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "T-SVD/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32(tcgen05 %s)+i64+f64" % args.precision,
                "data": "synthetic",
                "config": {"workload": d["name"], "precision": args.precision, "m_eff": d["m"],
                           "l2": "inputs larger than L2 (2.1 GB); L2 also flushed between steps (256 MB write)",
                           "parallelism": "dp%d" % world},
                "e2e": {"value": e2e_value, "unit": "T-SVD/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_timed, "roofline": roof, "clocks": clk.summary(),
                "paths": paths, "tprod_tflops": tprod_tflops, "batched": batched}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(X.astype(np.float64), d)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
