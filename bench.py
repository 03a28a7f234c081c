"""Benchmark of the randomized block Krylov truncated T-SVD (arXiv 2504.04989).

Workload (one step = one whole T-SVD, every stage of Alg. 2): the image-like
512 x 512 x 64 float32 tensor with per-Fourier-slice singular values
sigma_i = i^-1.5 (full rank), R = 50, P = 10, q = 4, synthetic (seeded), the
input resident in HBM.  Metric: rank-R T-SVD approximations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Under torchrun every rank runs its own independent tensor (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="image-like 512x512x64 fp32, sigma_i=i^-1.5 full rank, R=50 P=10 q=4",
                n1=512, n2=512, n3=64, R=50, P=10, q=4)
METRIC = "rank-R T-SVD approximations/s"
# ALU peaks from unit counts and clocks (GB300: 152 SMs at 2.07 GHz; per SM and
# clock 2 FP64 FMA lanes, 128 FP32 FMA lanes).
SMS, CLOCK_GHZ = 152, 2.07
FP64_PEAK_TFLOPS = SMS * CLOCK_GHZ * 2 * 2 / 1e3            # 1.259
FP32_ISSUE_TINST = SMS * CLOCK_GHZ * 128 / 1e3               # 40.3 T FP32 instructions/s
DF_FMA_INSTR = 15                                            # FP32 instructions per double-float multiply-add
DF_PEAK_TFLOPS = FP32_ISSUE_TINST / DF_FMA_INSTR * 2         # 5.37 (FP64-accuracy flops on the FP32 pipe)
# DRAM bytes per launch of the dominant kernel from the committed ncu capture of
# the same kernel and workload (profiles/k_hetrd_df_512x512x64_fp32.md); None
# once the kernel changes.
NCU_TRAFFIC = {"eig_hetrd": 24.80e6}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


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
    if stage == "orth_cgs":       # two classical Gram-Schmidt sweeps per block
        return {"flops": sum(2 * 2 * cm * n1 * c * nb for c, nb in zip(c_before, blocks)) * h}
    if stage == "orth_gram":
        return {"flops": sum(2 * cm * n1 * nb * (nb + 1) / 2 for nb in blocks) * h}
    if stage == "orth_trsm":
        return {"flops": sum(2 * cm * n1 * nb * nb / 2 for nb in blocks) * h}
    if stage == "krylov_gemm":    # A Omega, then A^H Q and A Y per Krylov step, and the last A^H Q
        return {"flops": cm * n1 * n2 * (sum(blocks) + sum(blocks[:-1]) + blocks[-1]) * h}
    if stage in ("rfft", "irfft"):
        s = 8 if precision == "fp64" else 4
        if stage == "rfft":
            return {"bytes": s * (n1 * n2 * n3 + 2 * n1 * n2 * h)}
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


ORACLE_SLICES = 16  # bounded sample: this many of the workload's Fourier slices per oracle run


def oracle_sample(X, d, nslices=ORACLE_SLICES):
    """The FP64 CPU oracle, as it stands, on `nslices` of the workload's
    h = n3/2 + 1 independent Fourier slices (OpenMP across slices); the time
    of a whole T-SVD is that of the sample scaled by h / nslices."""
    import oracle
    h = d["n3"] // 2 + 1
    om = oracle.gaussian(0, d["n3"] * d["n2"] * (d["R"] + d["P"])).reshape(d["n3"], d["n2"], d["R"] + d["P"])
    t0 = time.perf_counter()
    oracle.rtsvd_fourier(X, d["R"], d["P"], d["q"], omega=om, slices=list(range(nslices)))
    dt = time.perf_counter() - t0
    return dt * h / nslices, dt, oracle.num_threads()


def cpu_baseline(X, d):
    per_tsvd, dt, cores = oracle_sample(X.astype(np.float64), d)
    return {"value": 1.0 / per_tsvd, "unit": "T-SVD/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the %d Fourier slices of one T-SVD of the workload (FP64, %.1f s), scaled to the whole "
                      "T-SVD" % (ORACLE_SLICES, d["n3"] // 2 + 1, dt)}


def run_reference(args, d, rank, world):
    if rank != 0:
        return
    from paper_2504_04989_gb300 import workloads as wl
    X = wl.make_c2(0).astype(np.float32).astype(np.float64)
    steps = []
    for i in range(args.warmup + args.steps):
        per, dt, cores = oracle_sample(X, d)
        if i >= args.warmup:
            steps.append(per)
    t = sum(steps)
    val = args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "T-SVD/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": d["name"], "precision": "fp64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": "T-SVD/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: %d of the %d Fourier slices of one T-SVD, scaled to the whole "
                                       "T-SVD" % (ORACLE_SLICES, d["n3"] // 2 + 1)},
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

    def timed(plan, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev) / k

    eager = api.RbkBatchPlan(shapes, Rs, P=5, q=2, seed=0, precision="fp32", lanes=1, device=dev)
    eager(xs)
    ms_eager = timed(eager, 1)
    del eager
    plan = api.RbkBatchPlan(shapes, Rs, P=5, q=2, seed=0, precision="fp32", lanes=lanes, device=dev, graph=True)
    plan(xs)
    torch.cuda.synchronize(dev)
    timed(plan, 1)
    ms = timed(plan, steps)
    return {"workload": "uneven batch: n1, n2 ~ U{32..512}, n3 ~ U{8,16,32,64}, rank ~ U{5..40}, P=5, q=2, fp32",
            "tensors": count, "lanes": lanes, "graph": True, "ms_per_batch": ms,
            "tsvd_per_s": count * 1000.0 / ms, "eager_single_stream_ms": ms_eager}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-count", type=int, default=64,
                    help="tensors of the uneven batch timed after the main workload (0: skip)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    d = dict(WORKLOAD)
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
    X = wl.make_c2(seed=rank).astype(np.float32 if args.precision == "fp32" else np.float64)
    Xd = torch.from_numpy(X).to(dev)
    plan = api.RbkPlan(d["n1"], d["n2"], d["n3"], d["R"], d["P"], d["q"], seed=0, precision=args.precision,
                       device=dev)
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

    # end to end through the public API: pinned host input -> device -> T-SVD -> host outputs
    Xh = torch.from_numpy(X).pin_memory()
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

    # per-stage times (CUDA events recorded by the library on this stream)
    with api.profile() as pr:
        for _ in range(3):
            flush.zero_()
            plan(Xd)
    stages = {k: v[0] / 3 for k, v in pr.stages.items()}
    launches = {k: v[1] // 3 for k, v in pr.stages.items()}
    dom = max(stages, key=stages.get)
    pk = peaks()

    def roofline_of(stage):
        work = algorithmic(stage, d, args.precision)
        t = stages[stage] * 1e-3
        if "flops" in work:
            if args.precision == "fp64":
                peak, src = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz"
            elif stage == "eig_hetrd":
                peak, src = DF_PEAK_TFLOPS, "derived: FP32 issue rate / 15 instructions per double-float FMA"
            elif stage == "gram_c":
                peak, src = 2 * FP32_ISSUE_TINST, "derived: one 32x32->64-bit multiply-add per lane and clock"
            else:
                peak, src = 2 * FP32_ISSUE_TINST, "derived: 152 SMs x 128 FP32 FMA/clk x 2.07 GHz"
            a = work["flops"] / t / 1e12
            return {"kernel": stage, "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                    "frac": a / peak, "traffic": NCU_TRAFFIC.get(stage), "peak_source": src}
        if "bytes" in work:
            a = work["bytes"] / t / 1e9
            return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": a / pk["hbm_gbs"], "traffic": NCU_TRAFFIC.get(stage),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
        return None

    roof = roofline_of(dom) or {"kernel": dom, "bound": None}
    roof["stage_ms"] = {k: round(v, 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1])}
    roof["stages"] = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in r.items()
                          if kk in ("bound", "achieved", "peak", "unit", "frac")}
                      for k in stages for r in [roofline_of(k)] if r}

    # reconstruction error of this path and of the FP64 path on the same tensor ("equal error")
    def rel_err(U, S, V, Xref):
        Sf = torch.zeros((d["n3"], d["R"], d["R"]), dtype=torch.float64, device=dev)
        Sf.diagonal(dim1=1, dim2=2).copy_(S.double())
        VT = torch.zeros((d["n3"], d["R"], d["n2"]), dtype=torch.float64, device=dev)
        VT[0] = V[0].double().T
        VT[1:] = V.double().flip(0)[:-1].transpose(1, 2)      # tensor transpose (Sec. 2)
        Xr = api.tprod(api.tprod(U.double(), Sf, "fp64"), VT, "fp64")
        return float(torch.linalg.vector_norm(Xref - Xr) / torch.linalg.vector_norm(Xref))

    X64 = Xd.double()
    err_path = rel_err(plan.U, plan.S, plan.V, X64)
    plan64 = api.RbkPlan(d["n1"], d["n2"], d["n3"], d["R"], d["P"], d["q"], seed=0, precision="fp64", device=dev)
    plan64(X64)
    torch.cuda.synchronize(dev)
    ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for a, b in ev64:
        flush.zero_()
        a.record(stream)
        plan64(X64)
        b.record(stream)
    torch.cuda.synchronize(dev)
    fp64_ms = sum(a.elapsed_time(b) for a, b in ev64) / len(ev64)
    err_fp64 = rel_err(plan64.U, plan64.S, plan64.V, X64)
    opt = float(np.sqrt(wl.optimal_error2(wl.c2_sigma(d["n1"]), d["R"])) / torch.linalg.vector_norm(X64).item())

    # mixed paths (basis-building products on tcgen05, TF32 / BF16, the rest as on the FP32 path)
    # and Alg. 1 of the paper on the FP32 path
    mixed = {}
    if args.precision == "fp32":
        for prec in ("tf32", "bf16", "alg1"):
            # "alg1": Alg. 1 of the paper (power iteration) on the FP32 path, same Omega
            pl = api.RbkPlan(d["n1"], d["n2"], d["n3"], d["R"], d["P"], d["q"], seed=0,
                             precision="fp32" if prec == "alg1" else prec, device=dev, alg1=prec == "alg1")
            pl(Xd)
            torch.cuda.synchronize(dev)
            evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            for a, b in evm:
                flush.zero_()
                a.record(stream)
                pl(Xd)
                b.record(stream)
            torch.cuda.synchronize(dev)
            ms_m = sum(a.elapsed_time(b) for a, b in evm) / len(evm)
            mixed[prec] = {"ms_per_tsvd": ms_m, "tsvd_per_s": 1000.0 / ms_m,
                           "rel_error": rel_err(pl.U, pl.S, pl.V, X64)}
            del pl

    # t-product throughput on the paper-shaped products (flops 8 n1 n2 n4 h, whole call incl. FFTs)
    tprod_tflops = {}
    for name, n1, n2, n4, n3 in (("2048x2048x128*2048x120x128", 2048, 2048, 120, 128),
                                 ("1024x1024x64*1024x1024x64", 1024, 1024, 1024, 64),
                                 ("256x20x100*20x256x100", 256, 20, 256, 100)):
        fl = 8.0 * n1 * n2 * n4 * (n3 // 2 + 1)
        row = {}
        for prec in ("fp64", "fp32", "tf32", "bf16"):
            dt = torch.float64 if prec == "fp64" else torch.float32
            A = torch.randn(n3, n1, n2, device=dev, dtype=dt)
            B = torch.randn(n3, n2, n4, device=dev, dtype=dt)
            api.tprod(A, B, prec)
            ts = []
            for _ in range(3):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                api.tprod(A, B, prec)
                b.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(a.elapsed_time(b))
            row[prec] = round(fl / (min(ts) * 1e-3) / 1e12, 3)
            del A, B
        tprod_tflops[name] = row

    batched = None
    if args.batched_count > 0 and args.precision == "fp32":
        batched = batched_bench(api, wl, dev, args.batched_count, 8, 3, flush, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "T-SVD/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64+f64" if args.precision == "fp32" else "f64",
                "data": "synthetic",
                "config": {"workload": d["name"], "precision": args.precision, "m_eff": d["m"],
                           "l2": "flushed between steps (256 MB write)", "parallelism": "dp%d" % world},
                "e2e": {"value": e2e_value, "unit": "T-SVD/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_timed, "roofline": roof, "clocks": clk.summary(),
                "paths": {"this": {"precision": args.precision, "ms_per_tsvd": 1000 * total_s / args.steps,
                                   "rel_error": err_path},
                          "fp64": {"ms_per_tsvd": fp64_ms, "tsvd_per_s": 1000.0 / fp64_ms, "rel_error": err_fp64},
                          **mixed,
                          "speedup_vs_fp64": fp64_ms / (1000 * total_s / args.steps),
                          "eckart_young_optimum_rel_error": opt},
                "tprod_tflops": tprod_tflops, "batched": batched}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(X, d)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
