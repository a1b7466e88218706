"""Benchmark: H^2-ULV factor + refined solve on one GB300.

One step = h2_factor (mixed precision) + h2_solve refined to a relative H^2
residual of 1e-10, on N = 2^20 points on a union of 16 ellipsoid and 16
torus surfaces (Laplace kernel 1/(r + 1e-3), leaf 256, eta 1, tol 1e-6).
The inputs (points, right-hand side) are resident in HBM and the per-step
working set (tens of GB of near blocks) is far larger than L2.

Prints ONE JSON line (rank 0).  --impl reference runs the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "H²-ULV factor s + solve ms at N=2^20, mixed vs FP64 GPU at rel. residual 1e-10"
WORKLOAD = dict(name="surfaces1m", n=1 << 20, kernel="laplace", leaf=256, eta=1.0, tol=1e-6, max_rank=128,
                far_s0=16, far_smin=2, target=1e-10, seed=4, rhs_seed=40)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 7 for k in range(4)
                          if r[3 + k].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def cpu_oracle_sample(n_sample, repeats=1):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload:
    the same generator, kernel and parameters at N = n_sample; the method is
    O(N), so the time is scaled by 2^20 / n_sample."""
    from oracle import h2ulv_oracle as O
    W = WORKLOAD
    X = synth.surface_union(n_sample, W["seed"])
    b = synth.rhs(n_sample, 1, W["rhs_seed"])[:, 0].copy()
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        pb = O.Problem(X, W["kernel"], W["leaf"], W["eta"], W["tol"], W["max_rank"], W["far_s0"], W["far_smin"])
        op = O.H2Operator(pb)
        t1 = time.perf_counter()
        fac = O.ULVFactor(pb)
        x, rel, it = O.refine(op, fac, b, W["target"], 30)
        t2 = time.perf_counter()
        ts.append((t1 - t0, t2 - t1))
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max(i.get("num_threads", 1) for i in threadpool_info()) or cores
    except Exception:
        pass
    fac_solve = float(np.median([t[1] for t in ts]))
    return dict(value=fac_solve * W["n"] / n_sample, unit="s", cores=int(cores), kind="oracle",
                cpu_model=cpu_model(), measured_s=fac_solve, n_sample=n_sample,
                sample=f"oracle factor+refined solve on N={n_sample} points of the same surface union "
                       f"(leaf 256, tol 1e-6), {fac_solve:.2f} s measured, scaled x{W['n'] / n_sample:.0f} "
                       f"to N=2^20 (O(N) method); construct {np.median([t[0] for t in ts]):.2f} s not included")


# DRAM traffic of a kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), as bytes per algorithmic unit (flop or byte) of the
# captured launch, keyed by kernel@site; a launch's traffic is that ratio x
# its algorithmic units (the captures ran on N = 65 536, where the same
# per-pair products run on the same block sizes).  Remove an entry when its
# kernel changes.
NCU_TRAFFIC = {
    # tcgen05 GEMM, first leaf fill-in launch (8 192 products 256x256x256 =
    # 274.9 GFLOP): 3.438 GB read + 2.108 GB write
    "gemm_tc3xtf32@fillin": {"per_unit": (3.438254e9 + 2.108418e9) / 274.878e9,
                             "source": "ncu dram__bytes_read/write.sum, N=65536 leaf fill-in launch, "
                                       "scaled by flops per launch"},
    # double-float near matvec, one launch over 4.61 GB of stored blocks:
    # 4.62 GB read + 0.048 GB write
    "symv_pairs_df@mv_near": {"per_unit": (4.62e9 + 0.048e9) / 4.61e9,
                              "source": "ncu dram__bytes_read/write.sum, N=65536 near matvec, "
                                        "scaled by algorithmic bytes per launch"},
}

FP32_PREFIX = ("gemm_f32", "kgram_f32", "getrf_f32", "trsm_f32", "hqr_f32")
FP64_PREFIX = ("gemm_f64", "getrf_f64", "trsm_f64", "pchol_f64", "pqr_f64", "fold_f64", "hqr_f64", "kgram_f64")


def roofline_of(name, ks, pk, tot_ms):
    """Achieved = algorithmic flops or bytes the host declared for the
    kernel's launches / their summed CUDA-event time; peak by the bound."""
    secs = ks["ms"] * 1e-3
    clock = (pk["sm_max_mhz"] if pk else 2070.0) * 1e6
    if name.startswith("gemm_tc3xtf32"):
        # split 3xTF32: three tf32 products per useful product; tf32 peak =
        # measured sustained bf16 x nominal tf32/bf16 (1.1 / 2.25)
        peak = (pk["bf16_tflops_sustained"] if pk else 1700.0) * (1.1 / 2.25) / 3.0
        bound, unit, ach = "tensor", "TFLOP/s", ks["flops"] / secs / 1e12
        src = "measured sustained bf16 x tf32/bf16 nominal / 3 products" + ("" if pk else " (fallback)")
    elif name.startswith(FP32_PREFIX) and ks["flops"] > 0:
        peak = 152 * 128 * 2 * clock / 1e12
        bound, unit, ach = "alu", "TFLOP/s", ks["flops"] / secs / 1e12
        src = "152 SM x 128 FP32 lanes x 2 x max SM clock"
    elif name.startswith(FP64_PREFIX) and ks["flops"] > 0:
        peak = 1.25 * clock / 2.07e9
        bound, unit, ach = "alu", "TFLOP/s", ks["flops"] / secs / 1e12
        src = "GB300 nominal FP64 1.25 TFLOP/s at the max SM clock"
    else:
        peak = pk["hbm_gbs"] if pk else 6800.0
        bound, unit, ach = "hbm", "GB/s", ks["bytes"] / secs / 1e9
        src = "measured HBM copy bandwidth" if pk else "fallback 6.8 TB/s"
    tr = NCU_TRAFFIC.get(name)
    units = (ks["flops"] if bound != "hbm" else ks["bytes"]) / max(1, ks["launches"])
    return {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
            "frac": ach / peak if peak else None, "traffic": tr["per_unit"] * units if tr else None,
            "traffic_source": tr["source"] if tr else None, "launches": ks["launches"],
            "ms_total": ks["ms"], "share": ks["ms"] / tot_ms, "per_launch_ms": ks["ms"] / max(1, ks["launches"]),
            "algorithmic_per_launch": units,
            "peak_source": src}


def dense_rows(X, rows, v, delta=1e-3):
    """(K v)_i on sampled rows of the workload's dense matrix, K = 1/(r +
    delta) (Laplace), one FP64 row at a time."""
    return np.array([(1.0 / (np.sqrt(((X - X[i]) ** 2).sum(1)) + delta)) @ v for i in rows])


def accuracy(h, H, b_dev, b_host, X, rows, x_ref):
    """The factorization's own accuracy: x_u = ULV^-1 b (no refinement); its
    dense residual on sampled rows, its distance to the refined solution
    x_ref (which solves the H2 system to 1e-10), and the dense residual of
    x_ref itself."""
    import torch
    n = len(b_host)
    xu = torch.zeros_like(b_dev)
    st, ach, it = H.h2_solve(h, b_dev, xu, 1, n, 1e300, 0)
    xu = xu.cpu().numpy()
    assert WORKLOAD["kernel"] == "laplace"
    r_u = b_host[rows] - dense_rows(X, rows, xu)
    r_x = b_host[rows] - dense_rows(X, rows, x_ref)
    nb = np.linalg.norm(b_host[rows])
    return {"unrefined_h2_residual": float(ach[0]),
            "unrefined_dense_residual_rows": float(np.linalg.norm(r_u) / nb),
            "unrefined_vs_refined": float(np.linalg.norm(xu - x_ref) / np.linalg.norm(x_ref)),
            "refined_dense_residual_rows": float(np.linalg.norm(r_x) / nb)}


def cpu_model():
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True).stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def dist_init(world):
    """One process per GPU over NCCL; gloo when CUDA is absent (CPU tests of
    the multi-rank path).  Replicas: no collective touches the data path,
    only the barrier and the max over ranks of the step time."""
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def max_over_ranks(x, world, device=None):
    """The largest value of x over all ranks (the step time of the job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_sample = args.cpu_sample
    vals = []
    cb = None
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up effects worth timing separately
    for _ in range(args.steps):
        cb = cpu_oracle_sample(n_sample)
        vals.append(cb["value"])
    v = float(np.median(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "surfaces1m: N=2^20 on 16 ellipsoid + 16 torus surfaces, Laplace 1/(r+1e-3), "
                                   "leaf 256, eta 1, tol 1e-6, refined to 1e-10", "n": WORKLOAD["n"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """The batched workload: 64 independent problems (N log-uniform in
    [2048, 65536], cube / sphere / ellipsoid surfaces, Laplace, leaf 256,
    tol 1e-8), one batched handle; a step is the mixed-precision factor of
    all problems plus the solve of each problem's own right-hand sides (1 to
    256 columns) refined to 1e-10."""
    import torch
    from paper_2208_10907_gb300 import h2ulv as H
    probs = synth.batched_problems(64)
    Xs = [p["points"] for p in probs]
    nr = [p["nrhs"] for p in probs]
    Ns = [len(X) for X in Xs]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    hb = H.h2_construct_batched([torch.from_numpy(X).to(dev) for X in Xs], H.make_kernel("laplace"),
                                H.make_options(leaf=256, tol=1e-8, max_rank=128), stream.cuda_stream)
    torch.cuda.synchronize()
    t_con = time.perf_counter() - t0
    bt = [torch.from_numpy(np.ascontiguousarray(synth.rhs(N, k, 500 + q).T)).to(dev) for q, (N, k) in enumerate(zip(Ns, nr))]
    xt = [torch.zeros_like(b) for b in bt]

    def step():
        H.h2_factor(hb, H.H2_MIXED)
        return H.h2_solve_batched(hb, bt, xt, nr, Ns, 1e-10, 60)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    res = []
    e[0].record(stream)
    for k in range(args.steps):
        H.h2_factor(hb, H.H2_MIXED)
        e[2 * k + 1].record(stream)
        st, ach, it = H.h2_solve_batched(hb, bt, xt, nr, Ns, 1e-10, 60)
        e[2 * k + 2].record(stream)
        res.append((int(st), float(np.max(ach)), int(it)))
    torch.cuda.synchronize()
    total = e[0].elapsed_time(e[-1]) / args.steps
    f_ms = [e[2 * k].elapsed_time(e[2 * k + 1]) for k in range(args.steps)]
    s_ms = [e[2 * k + 1].elapsed_time(e[2 * k + 2]) for k in range(args.steps)]
    line = {"metric": "batched H2-ULV: mixed factor of 64 problems + per-problem solve refined to 1e-10",
            "value": total / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batched64: 64 problems, N log-uniform in [2048, 65536], cube/sphere/ellipsoid "
                                   "surfaces, Laplace 1/(r+1e-3), leaf 256, eta 1, tol 1e-8, 1-256 rhs each",
                       "n_total": int(sum(Ns)), "rhs_total": int(sum(nr)), "rhs_max": int(max(nr))},
            "factor_s": float(np.median(f_ms)) / 1e3, "solve_s": float(np.median(s_ms)) / 1e3,
            "construct_s": t_con, "refine": [{"status": a, "max_residual": b, "iters": c} for a, b, c in res]}
    print(json.dumps(line), flush=True)
    H.h2_destroy(hb)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink N (debugging only)")
    ap.add_argument("--cpu-sample", type=int, default=8192)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64-path steps (0 = skip)")
    ap.add_argument("--kernel-table", action="store_true", help="print the per-kernel event table to stderr")
    ap.add_argument("--max-rank", type=int, default=None,
                    help="rank cap per box (default: the workload's 128; at most 256)")
    ap.add_argument("--partition", default="bisection", choices=["bisection", "kmeans"],
                    help="cluster tree of the headline workload (the default is the workload's bisection)")
    ap.add_argument("--workload", default="surfaces1m", choices=["surfaces1m", "batched64"],
                    help="batched64: the 64 independent problems of the batched workload (not the headline)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched64":
        return run_batched(args)

    import torch
    import torch.distributed as dist
    from paper_2208_10907_gb300 import h2ulv as H

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = dict(WORKLOAD)
    if args.max_rank is not None:
        W["max_rank"] = args.max_rank
    n = max(4096, int(W["n"] * args.scale))
    X = synth.surface_union(n, W["seed"])
    b_host = synth.rhs(n, 1, W["rhs_seed"])[:, 0].copy()
    pts = torch.from_numpy(X).to(dev)
    b = torch.from_numpy(b_host).to(dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream(dev)
    kern = H.make_kernel(W["kernel"])
    opt = H.make_options(eta=W["eta"], leaf=W["leaf"], tol=W["tol"], max_rank=W["max_rank"], far_s0=W["far_s0"],
                         far_smin=W["far_smin"], hbm_budget_bytes=180 * 10**9, partition=args.partition)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = H.h2_construct(pts, n, kern, opt, stream.cuda_stream)
    torch.cuda.synchronize()
    t_construct = time.perf_counter() - t0

    def step(prec, bb, xx):
        H.h2_factor(h, prec)
        st, ach, it = H.h2_solve(h, bb, xx, 1, n, W["target"], 30)
        return st, ach, it

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    for _ in range(args.warmup):
        step(H.H2_MIXED, b, x)
    # ---- timed region: device-resident inputs, no instrumentation (the
    # solve plans run as captured CUDA graphs)
    H.h2_profile(0, 1)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evf = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = []
    evs[0].record(stream)
    for k in range(args.steps):
        H.h2_factor(h, H.H2_MIXED)
        evf[k].record(stream)
        st, ach, it = H.h2_solve(h, b, x, 1, n, W["target"], 30)
        evs[k + 1].record(stream)
        iters.append((int(st), float(ach[0]), int(it)))
    barrier()
    clk = clocks.stop()
    launches_timed = int(json.loads(H.h2_stats(h)).get("launches", 0))
    total_ms = evs[0].elapsed_time(evs[-1])
    f_ms = [evs[k].elapsed_time(evf[k]) for k in range(args.steps)]
    s_ms = [evf[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    step_ms = total_ms / args.steps
    solve_ms = float(np.mean(s_ms))
    step_ms = max_over_ranks(step_ms, world, dev)

    # ---- per-kernel times: the same step repeated with every launch
    # bracketed by CUDA events on its stream (rooflines below)
    prof_steps = min(args.steps, 3)
    H.h2_profile(1, 1)
    barrier()
    for _ in range(prof_steps):
        step(H.H2_MIXED, b, x)
    barrier()
    stats = json.loads(H.h2_stats(h))
    H.h2_profile(0, 0)
    kern_stats = stats.get("kernels", {})
    if args.kernel_table:
        ks_ = sorted(kern_stats.items(), key=lambda kv: -kv[1]["ms"])
        tot_ = sum(v["ms"] for _, v in ks_) or 1.0
        print(f"per-kernel CUDA-event times over {prof_steps} instrumented step(s)", file=sys.stderr)
        for k_, v_ in ks_[:48]:
            print(f"{k_:32s} launches {v_['launches']:6d} ms {v_['ms']:10.2f} ({100 * v_['ms'] / tot_:5.1f}%) "
                  f"GFLOP {v_['flops'] / 1e9:10.1f} GB {v_['bytes'] / 1e9:9.2f}", file=sys.stderr)
        print("GEMM autotuner choices:", json.dumps(stats.get("autotune", [])), file=sys.stderr)

    # ---- roofline of every kernel (algorithmic flops or bytes per launch
    # over its event time); the dominant one goes in "roofline"
    pk = peaks()
    tot_ms = sum(v["ms"] for v in kern_stats.values()) or 1.0
    ranked = sorted(kern_stats.items(), key=lambda kv: -kv[1]["ms"])
    roof_all = [roofline_of(k, v, pk, tot_ms) for k, v in ranked if v["ms"] > 0]
    roof = roof_all[0] if roof_all else None

    # ---- accuracy of the factorization itself (the paper's protocol: the
    # unrefined ULV solution), on sampled rows of the dense kernel matrix
    rows = np.sort(np.random.default_rng(77).choice(n, 48, replace=False))
    x_ref = x.cpu().numpy()
    acc = {"rows": len(rows), "mixed": accuracy(h, H, b, b_host, X, rows, x_ref)}

    # ---- FP64 path, same GPU (fewer steps: FP64 throughput is 1/60 of FP32)
    fp64 = None
    if args.fp64_steps > 0:
        step(H.H2_FP64, b, x)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        fs, ss, its = [], [], []
        for _ in range(args.fp64_steps):
            e0.record(stream)
            H.h2_factor(h, H.H2_FP64)
            e1.record(stream)
            st, ach, it = H.h2_solve(h, b, x, 1, n, W["target"], 30)
            e2.record(stream)
            torch.cuda.synchronize()
            fs.append(e0.elapsed_time(e1))
            ss.append(e1.elapsed_time(e2))
            its.append(it)
        st64 = json.loads(H.h2_stats(h))
        fp64 = {"factor_s": float(np.median(fs)) / 1e3, "solve_ms": float(np.median(ss)), "iters": its,
                "step_s": (float(np.median(fs)) + float(np.median(ss))) / 1e3,
                "basis_route": st64.get("basis_route"), "tol_basis": st64.get("tol_basis")}
        acc["fp64"] = accuracy(h, H, b, b_host, X, rows, x.cpu().numpy())
        H.h2_factor(h, H.H2_MIXED)

    # ---- end to end through the C ABI with host buffers (pinned)
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.zeros_like(b_pin).pin_memory()
    step(H.H2_MIXED, b_pin, x_pin)
    barrier()
    t_e2e = time.perf_counter()
    for _ in range(args.steps):
        step(H.H2_MIXED, b_pin, x_pin)
    barrier()
    e2e_ms = (time.perf_counter() - t_e2e) * 1e3 / args.steps

    # ---- CPU baseline (oracle) on rank 0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.cpu_sample)

    if rank == 0:
        st_m = json.loads(H.h2_stats(h))
        line = {
            "metric": METRIC, "value": step_ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "surfaces1m: N=2^20 on 16 ellipsoid + 16 torus surfaces, Laplace 1/(r+1e-3), "
                                   "leaf 256, eta 1, tol 1e-6, mixed factor refined to H2 residual 1e-10",
                       "n": n, "leaf": W["leaf"], "eta": W["eta"], "tol": W["tol"], "max_rank": W["max_rank"],
                       "far_sample": [W["far_s0"], W["far_smin"]], "l2": "inputs larger than L2 (tens of GB)",
                       "partition": args.partition,
                       "residual": "FP64 H2 operator; its near field for one right-hand side in double-float "
                                   "(FP64 entries split exactly into FP32 pairs, about 2^-46 per product)",
                       "basis": {"route": st_m.get("basis_route"), "tol_basis": st_m.get("tol_basis")},
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "factor_s": float(np.mean(f_ms)) / 1e3, "solve_ms": solve_ms,
            "step_s_median": float(np.median(per_step)) / 1e3,
            "step_s_all": [round(v / 1e3, 4) for v in per_step],
            "refine": [{"status": s_, "residual": a_, "iters": i_} for s_, a_, i_ in iters],
            "construct_s": t_construct,
            "fp64": fp64,
            "mixed_vs_fp64_speedup": (fp64["step_s"] / (step_ms / 1e3)) if fp64 else None,
            "accuracy": acc,
            "roofline": roof,
            "roofline_all": roof_all,
            "roofline_steps": prof_steps,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": launches_timed,
            "clocks": clk,
            "levels": stats.get("levels"),
        }
        print(json.dumps(line), flush=True)
    H.h2_destroy(h)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
