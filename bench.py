"""Benchmark of the GB300 H^2 product Z <- Z + X Y.

One step = one h2_mul_add call (the whole hot path: basis products, weights,
compressed induced bases, the couplings on T^XY, coarsening, final
couplings) on the n = 32768 unit-sphere workload: Laplace kernel, leaf 64,
eta 2, Chebyshev order 4 (rank 64), X = Y = Z, eps = 1e-6.  The metric is
rows per second (n / time).  The line's `value` is the FP64 GPU form (the
workload's stated precision); the mixed-precision form of the same workload
is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent product (the products of
a batch are independent: replicas only, weak scaling); value = all rows of
all ranks / max-over-ranks time.  `--impl reference` times the FP64 CPU
oracle (the reference for this method) on a bounded sample of the workload.
"""
import argparse
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

import synth  # noqa: E402

WORKLOAD = dict(name="sphere-n32768-laplace-leaf64-eta2-m4-eps1e-6", geometry="sphere", n=32768, kernel=0,
                leaf=64, eta=2.0, order=4, eps=1e-6, seed=2309090611)
# bounded CPU sample of the same workload for the oracle: same geometry,
# kernel, leaf, eta, order and eps at n = 4096 (about 10-20 s of CPU work)
CPU_SAMPLE_N = 4096
METRIC = "H2 Z<-Z+XY rows/s at eps (FP64 GPU form; mixed form beside it)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"], help="override n (testing only)")
    ap.add_argument("--workload", default="sphere32768", choices=["sphere32768", "batched64", "dlp49152"],
                    help="sphere32768: the default line; batched64: 64 independent products in one batched call")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(seed, rank):
    """Seed of rank `rank`'s points: every rank runs an independent product."""
    return seed + 1000 * rank


def max_over_ranks(x, world, tdist, device):
    """The largest x of all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def library_peaks(torch, dev):
    """FP64 and FP32 (no TF32) GEMM throughput of cuBLAS on this GPU, measured
    here: the denominators for the FP64 and FP32 contraction kernels, which
    MEASURED_PEAKS.json does not cover."""
    out = {}
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        n = 8192 if dt == torch.float32 else 4096
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        torch.backends.cuda.matmul.allow_tf32 = prev
        out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
        del a, b
    torch.cuda.empty_cache()
    return out


def run_cpu_sample():
    """The oracle as it stands on a bounded sample of the workload."""
    from oracle import h2_oracle as O
    w = WORKLOAD
    pts = synth.make_points(w["geometry"], CPU_SAMPLE_N, w["seed"])
    st = O.build_structure(pts, w["leaf"], w["eta"], w["order"])
    G = O.build_interp(st, w["kernel"])
    t0 = time.perf_counter()
    O.mul_add(G, G, G, w["eps"])
    dt = time.perf_counter() - t0
    return CPU_SAMPLE_N / dt, dt


def reference_arm(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    times = []
    for i in range(args.warmup + args.steps):
        v, dt = run_cpu_sample()
        if i >= args.warmup:
            times.append(dt)
    value = CPU_SAMPLE_N * len(times) / sum(times)
    cores = os.cpu_count()
    sample = (f"oracle (numpy FP64) on n={CPU_SAMPLE_N} points of the same workload "
              f"(sphere, Laplace, leaf 64, eta 2, order 4, eps 1e-6), X=Y=Z")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 points)",
            "config": {"workload": WORKLOAD["name"] + f" (CPU sample n={CPU_SAMPLE_N})", "n": CPU_SAMPLE_N},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours_arm(args):
    import torch
    import torch.distributed as tdist

    import paper_2309_09061_gb300 as P

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.build()
    P.load()
    w = dict(WORKLOAD)
    w["n"] = args.n
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    # each rank: its own independent product (seed offset by rank)
    pts = synth.make_points(w["geometry"], w["n"], rank_seed(w["seed"], rank))
    G = P.h2_build_interp(pts, w["kernel"], w["leaf"], w["eta"], w["order"], stream=sptr)

    def barrier():
        if world > 1:
            tdist.barrier()

    def timed(precision, steps, warmup):
        for _ in range(warmup):
            Zw = P.h2_clone(G, stream=sptr)
            P.h2_mul_add(Zw, G, G, w["eps"], precision, stream=sptr)
            del Zw
        Zs = [P.h2_clone(G, stream=sptr) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        t0 = time.perf_counter()
        e0.record(stream)
        for Z in Zs:
            stats.append(P.h2_mul_add(Z, G, G, w["eps"], precision, stream=sptr))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, tdist, dev)
        info = Zs[-1].info()
        # eps_2 of the last result (Sec. 7: relative spectral error, 20 power-iteration
        # steps through H^2 matrix-vector products), outside the timed region
        eps2 = P.h2_product_error(Zs[-1], G, G, G, steps=20, stream=sptr)[0] if rank == 0 else None
        for Z in Zs:
            Z.free()
        info["eps2"] = eps2
        return dt, wall, stats, info

    sampler = ClockSampler(local)
    sampler.start()
    dt64, wall64, st64, info64 = timed(P.H2_FP64, args.steps, args.warmup)
    clocks = sampler.stop()
    dtmx, wallmx, stmx, infomx = timed(P.H2_MIXED, args.steps, max(1, args.warmup // 2))
    dttc, walltc, sttc, infotc = timed(P.H2_TC, args.steps, max(1, args.warmup // 2))
    # end to end through the public API with host buffers: points host->device,
    # build, product, result structure (ranks) device->host, per step
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        X = P.h2_build_interp(pts, w["kernel"], w["leaf"], w["eta"], w["order"], stream=sptr)
        Z = P.h2_clone(X, stream=sptr)
        P.h2_mul_add(Z, X, X, w["eps"], P.H2_FP64, stream=sptr)
        _ = Z.structure()
        Z.free()
        X.free()
    torch.cuda.synchronize(dev)
    e2e_dt = (time.perf_counter() - t0) / e2e_steps
    nclusters = info64["nclusters"]
    d2h = w["n"] * 8 + 3 * nclusters * 8 + 2 * nclusters * 4

    # roofline of the dominant kernel family of each form
    peaks = measured_peaks()
    lib_peaks = library_peaks(torch, dev) if rank == 0 else {}
    names = P.FAMILIES
    kernel_of = {0: "k_gemm<double>", 1: "k_gemm_f32<false>", 2: "k_qr<double>", 3: "k_qr<float>", 4: "k_pchol",
                 5: "k_jacobi64", 6: "k_jacobi_pre / k_jacobi_pre_cluster", 7: "k_norm", 8: "k_copy",
                 9: "k_sumsq / k_finite", 10: "k_gemm_tc", 11: "k_gemm_f32<true>"}

    def sums(stats):
        out = {k: np.zeros(12) for k in ("ms", "fl", "by", "n")}
        for s in stats:
            out["ms"] += np.array(s["fam_ms"])
            out["fl"] += np.array(s["fam_flops"])
            out["by"] += np.array(s["fam_bytes"])
            out["n"] += np.array(s["fam_launches"])
        return out

    # DRAM traffic of k_gemm<double> from one ncu capture (sphere n=8192, the 61st
    # launch of the kernel; profiles/k_gemm_sphere-n8192_fp64.md): 45.77 MB of
    # dram__bytes_read.sum + dram__bytes_write.sum for 0.629 GFLOP of executed FP64 work
    # (314.6 M DFMA), scaled to the average launch here by its flops.  The kernel has not
    # changed since the capture.
    gemm64_capture = {"dram_bytes": 45.77e6, "flops": 0.629e9}

    def roofline(f):
        top = int(np.argmax(f["ms"]))
        rate = f["fl"][top] / (f["ms"][top] / 1e3) / 1e12
        if top in (0, 2, 4, 5, 7):  # FP64 arithmetic: bound by the FP64 pipe
            roof = {"kernel": kernel_of[top], "bound": "alu", "achieved": rate, "peak": lib_peaks.get("fp64_tflops"),
                    "unit": "TFLOP/s (FP64)",
                    "peak_source": "cuBLAS DGEMM 4096^3 measured in this run (MEASURED_PEAKS.json has no FP64 figure)"}
        elif top in (1, 3, 6):
            roof = {"kernel": kernel_of[top], "bound": "alu", "achieved": rate, "peak": lib_peaks.get("fp32_tflops"),
                    "unit": "TFLOP/s (FP32)", "peak_source": "cuBLAS SGEMM 8192^3 (no TF32) measured in this run"}
        elif top == 11:
            # double-float: 12 FP32 instructions per multiply-add (1 FMUL, 3 FFMA, 8 FADD),
            # i.e. 6 per algorithmic flop, each one lane operation; the SGEMM rate counts
            # an FFMA lane operation as 2 flops, so its lane-operation rate is half of it
            f32 = lib_peaks.get("fp32_tflops")
            roof = {"kernel": kernel_of[top], "bound": "alu", "achieved": 6.0 * rate,
                    "peak": f32 / 2.0 if f32 else None,
                    "unit": "T FP32 lane operations/s (FFMA, FADD, FMUL each one)",
                    "algorithmic_fp64_equivalent_tflops": rate,
                    "peak_source": "cuBLAS SGEMM 8192^3 (no TF32) measured in this run, / 2 (one FFMA = 2 flops)"}
        elif top == 10:
            roof = {"kernel": kernel_of[top], "bound": "tensor", "achieved": rate,
                    "peak": peaks.get("bf16_tflops", 1900.0) / 2.0, "unit": "TFLOP/s (algorithmic, TF32 x6)",
                    "peak_source": "MEASURED_PEAKS.json bf16 burst x 1/2 (nominal TF32:BF16 ratio)"}
        else:
            rate = f["by"][top] / (f["ms"][top] / 1e3) / 1e9
            roof = {"kernel": kernel_of[top], "bound": "hbm", "achieved": rate, "peak": peaks.get("hbm_gbs", 6800.0),
                    "unit": "GB/s", "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
        roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("peak") else None
        roof["traffic"] = None
        if top == 0 and f["n"][top] > 0:
            per_launch = f["fl"][top] / f["n"][top]
            roof["traffic"] = gemm64_capture["dram_bytes"] * per_launch / gemm64_capture["flops"]
            roof["traffic_unit"] = "bytes per launch"
            roof["traffic_source"] = ("ncu capture at n=8192 (45.77 MB for 0.629 GFLOP executed), "
                                      "scaled by the average launch's flops")
            roof["algorithmic_bytes_per_launch"] = f["by"][top] / f["n"][top]
        roof["avg_launch_ms"] = f["ms"][top] / max(1.0, f["n"][top])
        roof["share_of_step"] = float(f["ms"][top] / max(1e-9, f["ms"].sum()))
        return roof

    f64s, fmxs = sums(st64), sums(stmx)
    roof = roofline(f64s)
    roof["peaks_measured_here"] = lib_peaks
    roof_mx = roofline(fmxs)
    fam_report = {names[i]: {"ms_per_step": f64s["ms"][i] / len(st64), "launches_per_step": f64s["n"][i] / len(st64),
                             "gflop_per_step": f64s["fl"][i] / len(st64) / 1e9,
                             "gb_per_step": f64s["by"][i] / len(st64) / 1e9}
                  for i in range(12) if f64s["n"][i] > 0}
    fam_report_mx = {names[i]: {"ms_per_step": fmxs["ms"][i] / len(stmx), "launches_per_step": fmxs["n"][i] / len(stmx),
                                "gflop_per_step": fmxs["fl"][i] / len(stmx) / 1e9}
                     for i in range(12) if fmxs["n"][i] > 0}

    n_all = w["n"] * world
    value = n_all * args.steps / dt64
    line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt64 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 points on the unit sphere)",
            "config": {"workload": w["name"], "n": w["n"], "leaf": w["leaf"], "eta": w["eta"],
                       "order": w["order"], "rank": w["order"] ** 3, "eps": w["eps"], "X=Y=Z": True,
                       "precision": "FP64 products, FP64 QR/SVD",
                       "l2": "inputs larger than L2 (X: %.0f MB)" % (G.info()["device_bytes"] / 1e6),
                       "parallelism": f"replicas x{world}"},
            "mixed": {"value": w["n"] * world * args.steps / dtmx, "unit": "rows/s",
                      "ms_per_step": 1e3 * dtmx / args.steps, "speedup_vs_fp64": dt64 / dtmx,
                      "precision": "FP32 products on CUDA cores; Gram matrices and SVD finishing in "
                                   "double-float FP32 (FP64-accurate); FP64 rank decisions",
                      "roofline": roof_mx},
            "tensor_core": {"value": w["n"] * world * args.steps / dttc, "unit": "rows/s",
                            "ms_per_step": 1e3 * dttc / args.steps, "speedup_vs_fp64": dt64 / dttc,
                            "precision": "tcgen05 TF32 three-term products, FP32 accumulation in TMEM, FP64 rank decisions",
                            "gemm_tc_ms_per_step": sum(x["fam_ms"][10] for x in sttc) / len(sttc),
                            "gemm_tc_gflop_per_step": sum(x["fam_flops"][10] for x in sttc) / len(sttc) / 1e9},
            "e2e": {"value": n_all / e2e_dt, "unit": "rows/s", "h2d_bytes_per_step": int(pts.nbytes),
                    "d2h_bytes_per_step": int(d2h),
                    "note": "h2_build_interp from host points + h2_clone + h2_mul_add + h2_get_structure"},
            "gpu_launches": int(sum(s["kernel_launches"] for s in st64)),
            "accuracy": {"eps": w["eps"], "eps2_fp64": info64["eps2"], "eps2_mixed": infomx["eps2"],
                         "eps2_tensor_core": infotc["eps2"],
                         "definition": "||Zr - (Z + X Y)||_2 / ||Z + X Y||_2, 20 power-iteration steps "
                                       "through H2 matrix-vector products (h2_product_error)"},
            "roofline": roof,
            "kernel_families_fp64": fam_report,
            "kernel_families_mixed": fam_report_mx,
            "stats_fp64": {k: st64[-1][k] for k in ("t_rows_a_ms", "t_cols_a_ms", "t_mat_a_ms", "t_rows_b_ms",
                                                     "t_cols_b_ms", "t_mat_b_ms", "product_nodes", "triples",
                                                     "max_rank_a", "max_rank_b")},
            "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        v, dt = run_cpu_sample()
        line["cpu_baseline"] = {"value": v, "unit": "rows/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"oracle on n={CPU_SAMPLE_N} points of the same workload, one product, "
                                          f"{dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


BATCH = dict(count=64, nmin=2048, nmax=65536, eps=1e-5, leaf=64, eta=2.0, seed=2309090613)


def batch_members():
    """The 64 products of the batched workload: n_i = round(2048 * 32^u_i), u_i
    uniform, half on the sphere and half on the cube surface, Chebyshev order
    3, 4 or 5 uniformly (ranks 27, 64, 125), Laplace kernel, leaf 64, eta 2."""
    b = BATCH
    u = synth.uniform01(b["seed"], 2 * b["count"])
    out = []
    for i in range(b["count"]):
        n = int(round(b["nmin"] * (b["nmax"] / b["nmin"]) ** u[2 * i]))
        order = 3 + min(2, int(3 * u[2 * i + 1]))
        geom = "sphere" if i % 2 == 0 else "cube_surface"
        out.append((geom, n, order, b["seed"] + 1000 * i))
    return out


def batched_arm(args):
    import torch

    import paper_2309_09061_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.build()
    P.load()
    members = batch_members()
    Gs = [P.h2_build_interp(synth.make_points(g, n, seed + rank), 0, BATCH["leaf"], BATCH["eta"], m)
          for g, n, m, seed in members]
    rows = sum(n for _, n, _, _ in members) * world
    out = {}
    for name, prec in (("mixed", P.H2_MIXED), ("fp64", P.H2_FP64)):
        times, stats = [], None
        for it in range(args.warmup + args.steps):
            Zs = [P.h2_clone(G) for G in Gs]
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            stats, codes = P.h2_mul_add_batched(Zs, Gs, Gs, BATCH["eps"], prec)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            assert codes == [0] * len(Zs)
            for Z in Zs:
                Z.free()
            if it >= args.warmup:
                times.append(dt)
        out[name] = {"value": rows * len(times) / sum(times), "unit": "rows/s",
                     "ms_per_step": 1e3 * sum(times) / len(times), "kernel_launches": stats["kernel_launches"]}
    line = {"metric": "H2 Z<-Z+XY rows/s, 64 independent products in one batched call", "value": out["mixed"]["value"],
            "unit": "rows/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["mixed"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 products, f64 factorisations", "data": "synthetic",
            "config": {"workload": "batched64", "products": len(members), "rows": rows,
                       "n_range": [min(n for _, n, _, _ in members), max(n for _, n, _, _ in members)],
                       "orders": sorted(set(m for _, _, m, _ in members)), "eps": BATCH["eps"]},
            "fp64": out["fp64"], "speedup_mixed_vs_fp64": out["mixed"]["value"] / out["fp64"]["value"],
            "gpu_launches": out["mixed"]["kernel_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


DLP = dict(n=49152, leaf=64, eta=2.0, order=4, eps=1e-4, seed=2309090615)


def dlp_arm(args):
    """The double-layer workload: K + K K for the collocated double-layer
    operator on the cube surface (non-symmetric, V != W), n = 49152 (the size of
    the paper's cube-surface example), FP64 and mixed, with eps_2 of each."""
    import torch

    import paper_2309_09061_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    P.build()
    P.load()
    d = DLP
    pts = synth.cube_surface(d["n"], rank_seed(d["seed"], rank))
    nrm = synth.cube_surface_normals(pts)
    K = P.h2_build_interp(pts, P.H2_K_DLP, d["leaf"], d["eta"], d["order"], stream=sptr, normals=nrm)
    out = {}
    for name, prec in (("fp64", P.H2_FP64), ("mixed", P.H2_MIXED)):
        for _ in range(args.warmup):
            Zw = P.h2_clone(K, stream=sptr)
            P.h2_mul_add(Zw, K, K, d["eps"], prec, stream=sptr)
            Zw.free()
        Zs = [P.h2_clone(K, stream=sptr) for _ in range(args.steps)]
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for Z in Zs:
            P.h2_mul_add(Z, K, K, d["eps"], prec, stream=sptr)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        dt = e0.elapsed_time(e1) / 1e3
        e2 = P.h2_product_error(Zs[-1], K, K, K, steps=20, stream=sptr)[0]
        for Z in Zs:
            Z.free()
        out[name] = {"value": d["n"] * world * args.steps / dt, "unit": "rows/s", "ms_per_step": 1e3 * dt / args.steps,
                     "eps2": e2}
    line = {"metric": "H2 Z<-Z+XY rows/s, double-layer operator on the cube surface", "value": out["fp64"]["value"],
            "unit": "rows/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["fp64"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded points on the cube surface, face normals)",
            "config": {"workload": "dlp49152", "n": d["n"], "leaf": d["leaf"], "eta": d["eta"], "order": d["order"],
                       "eps": d["eps"], "X=Y=Z": True},
            "mixed": out["mixed"], "speedup_mixed_vs_fp64": out["mixed"]["value"] / out["fp64"]["value"],
            "accuracy": {"eps2_fp64": out["fp64"]["eps2"], "eps2_mixed": out["mixed"]["eps2"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl != "reference" and args.workload == "batched64":
        batched_arm(args)
        return
    if args.impl != "reference" and args.workload == "dlp49152":
        dlp_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
