"""Benchmark of the GB300 H^2 product Z <- Z + X Y.

One step = one h2_mul_add call (the whole hot path: basis products, weights,
compressed induced bases, the couplings on T^XY, coarsening, final
couplings) on the n = 32768 unit-sphere workload: Laplace kernel, leaf 64,
eta 2, Chebyshev order 4 (rank 64), X = Y = Z, eps = 1e-6.  The metric is
rows per second (n / time).  The line's `value` is the fast form (H2_AUTO,
which at eps = 1e-6 runs the FP32-class products on the tcgen05 tensor cores
in three-term TF32 pieces and keeps QR/SVD/ranks in FP64); the plain FP64 GPU
form of the same workload is timed beside it with the same steps, and the
other workloads (n = 2048 sphere, n = 131072 cube at eps 1e-4 and 1e-6, the
64-product batch, n = 524288 sphere) follow as compact records at the end of
the line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--configs all|none]

Under torchrun every rank runs its own independent product (the products of
a batch are independent: replicas only, weak scaling); value = all rows of
all ranks / max-over-ranks time.  `--impl reference` times the FP64 CPU
oracle (the reference for this method) on a bounded sample of the workload.
"""
import argparse
import json
import os
import platform
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
# the other workloads: parity-test cases that the line reports compactly
CONFIGS = {
    "sphere2048": dict(geometry="sphere", n=2048, kernel=0, leaf=32, eta=2.0, order=3, eps=1e-4, seed=2309090610),
    "cube131072_e4": dict(geometry="cube", n=131072, kernel=1, leaf=64, eta=1.5, order=4, eps=1e-4,
                          seed=2309090612),
    "cube131072_e6": dict(geometry="cube", n=131072, kernel=1, leaf=64, eta=1.5, order=4, eps=1e-6,
                          seed=2309090612),
    "sphere524288": dict(geometry="sphere", n=524288, kernel=0, leaf=64, eta=2.0, order=5, eps=1e-6,
                         seed=2309090614),
}
# bounded CPU sample of the same workload for the oracle: same geometry,
# kernel, leaf, eta, order and eps at n = 4096 (about 10-20 s of CPU work)
CPU_SAMPLE_N = 4096
METRIC = "H2 Z<-Z+XY rows/s at eps (fast form: tensor-core products, FP64 QR/SVD; FP64 GPU form beside it)"
MODE_NAMES = {0: "fp64", 1: "mixed", 2: "tf32x3", 3: "tf32", 4: "bf16x3", 5: "auto"}


def resolve_precision(p, eps):
    """The concrete mode of H2_AUTO for a tolerance (the library's rule)."""
    if p != 5:
        return p
    return 3 if eps >= 1e-3 else 4 if eps >= 1e-4 else 2 if eps >= 1e-7 else 0


def r4(x):
    """x rounded to 4 significant digits (short JSON)."""
    if x is None or x == 0:
        return x
    return float(f"{x:.4g}")


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="all: also time the other workloads and report them compactly")
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


ONE_THREAD = {v: "1" for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")}


def run_c1_one_thread():
    """The oracle on the whole n = 2048 sphere workload (leaf 32, eta 2, order 3,
    eps 1e-4) with its BLAS held to one thread, in a fresh process: seconds of
    the product (for comparison with the paper's sequential timings)."""
    code = ("import sys,time; sys.path.insert(0, %r); import synth; from oracle import h2_oracle as O; "
            "c = %r; p = synth.make_points(c['geometry'], c['n'], c['seed']); "
            "st = O.build_structure(p, c['leaf'], c['eta'], c['order']); G = O.build_interp(st, c['kernel']); "
            "t = time.perf_counter(); O.mul_add(G, G, G, c['eps']); print(time.perf_counter() - t)"
            % (ROOT, CONFIGS["sphere2048"]))
    env = dict(os.environ)
    env.update(ONE_THREAD)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return float(out.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None


def cpu_baseline_record(value, dt):
    secs = run_c1_one_thread()
    return {"value": r4(value), "unit": "rows/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"numpy FP64 oracle, one product at n={CPU_SAMPLE_N} of the same workload, {dt:.1f} s",
            "cpu": cpu_model(),
            "n2048_one_thread": {"rows_s": r4(2048 / secs) if secs else None, "s": r4(secs)}}


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
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


KERNEL_OF = {0: "k_gemm<double>", 1: "k_gemm_f32<false>", 2: "k_qr<double>", 3: "k_qr<float>", 4: "k_pchol",
             5: "k_jacobi64", 6: "k_jacobi_pre", 7: "k_norm", 8: "k_copy", 9: "k_sumsq/k_finite", 10: "k_gemm_tc",
             11: "k_gemm_f32<true>"}


def family_sums(stats):
    out = {k: np.zeros(12) for k in ("ms", "fl", "by", "n")}
    for s in stats:
        out["ms"] += np.array(s["fam_ms"])
        out["fl"] += np.array(s["fam_flops"])
        out["by"] += np.array(s["fam_bytes"])
        out["n"] += np.array(s["fam_launches"])
    return out


def roofline(f, mode, peaks, lib_peaks):
    """Roofline of the dominant kernel family: achieved = algorithmic flops (or
    bytes) of its launches / their summed CUDA-event time, against the peak of
    the unit that bounds it."""
    top = int(np.argmax(f["ms"]))
    sec = f["ms"][top] / 1e3
    rate = f["fl"][top] / sec / 1e12
    tf32 = peaks.get("bf16_tflops", 1891.8) / 2.0
    if top in (0, 2, 4, 5, 7):  # FP64 pipe
        roof = {"bound": "alu", "achieved": rate, "peak": lib_peaks.get("fp64_tflops"), "unit": "TFLOP/s fp64",
                "peak_src": "cuBLAS DGEMM in this run"}
    elif top in (1, 3, 6):  # FP32 CUDA cores
        roof = {"bound": "alu", "achieved": rate, "peak": lib_peaks.get("fp32_tflops"), "unit": "TFLOP/s fp32",
                "peak_src": "cuBLAS SGEMM (no TF32) in this run"}
    elif top == 11:  # double-float: 6 FP32 lane operations per algorithmic flop
        f32 = lib_peaks.get("fp32_tflops")
        roof = {"bound": "alu", "achieved": 6.0 * rate, "peak": f32 / 2.0 if f32 else None,
                "unit": "T fp32 lane ops/s", "peak_src": "cuBLAS SGEMM in this run / 2"}
    elif top == 10:  # tensor cores: products issued per algorithmic flop by mode
        issued = {2: 3.0, 3: 1.0, 4: 3.0}.get(mode, 3.0)
        pk = tf32 if mode != 4 else 2.0 * tf32
        roof = {"bound": "tensor", "achieved": issued * rate, "peak": pk,
                "unit": "TFLOP/s issued on tcgen05 (%s)" % MODE_NAMES.get(mode),
                "peak_src": "MEASURED_PEAKS bf16 burst" + (" x 1/2 (TF32:BF16)" if mode != 4 else "")}
    else:
        rate = f["by"][top] / sec / 1e9
        roof = {"bound": "hbm", "achieved": rate, "peak": peaks.get("hbm_gbs", 6780.7), "unit": "GB/s",
                "peak_src": "MEASURED_PEAKS hbm_gbs"}
    roof["kernel"] = KERNEL_OF[top]
    roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("peak") else None
    roof["traffic"] = None
    n = max(1.0, f["n"][top])
    roof["avg_launch_ms"] = f["ms"][top] / n
    roof["share"] = float(f["ms"][top] / max(1e-9, f["ms"].sum()))
    for k in ("achieved", "peak", "frac", "avg_launch_ms", "share"):
        roof[k] = r4(roof[k])
    return roof


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
    fast = resolve_precision(P.H2_AUTO, w["eps"])
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    # each rank: its own independent product (seed offset by rank)
    pts = synth.make_points(w["geometry"], w["n"], rank_seed(w["seed"], rank))
    G = P.h2_build_interp(pts, w["kernel"], w["leaf"], w["eta"], w["order"], stream=sptr)

    def barrier():
        if world > 1:
            tdist.barrier()

    # the line runs the library's default schedules (h2_opts.autotune off); the
    # online tuner's result is reported beside it (forms_ms)
    P.set_autotune(False)

    def timed(G, c, precision, steps, warmup, eps2=True):
        """steps products (each on a fresh clone of G, made outside the timed
        region) timed back to back with CUDA events on the library's stream."""
        for _ in range(warmup):
            Zw = P.h2_clone(G, stream=sptr)
            P.h2_mul_add(Zw, G, G, c["eps"], precision, stream=sptr)
            Zw.free()
        Zs = [P.h2_clone(G, stream=sptr) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for Z in Zs:
            stats.append(P.h2_mul_add(Z, G, G, c["eps"], precision, stream=sptr))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, tdist, dev)
        # eps_2 of the last result (Sec. 7: relative spectral error, 20 power-iteration
        # steps through H^2 matrix-vector products), outside the timed region
        e2 = P.h2_product_error(Zs[-1], G, G, G, steps=20, stream=sptr)[0] if (eps2 and rank == 0) else None
        for Z in Zs:
            Z.free()
        return dt, stats, e2

    peaks = measured_peaks()
    sampler = ClockSampler(local)
    sampler.start()
    dtf, stf, e2f = timed(G, w, P.H2_AUTO, args.steps, args.warmup)
    clocks = sampler.stop()
    dt64, st64, e264 = timed(G, w, P.H2_FP64, args.steps, args.warmup)
    # the other precision modes on the same workload (context; fewer steps)
    forms = {}
    for p in (P.H2_MIXED, P.H2_TF32X3, P.H2_BF16X3):
        if p == fast:
            continue
        k = max(1, min(args.steps, 5))
        dtp, _, e2p = timed(G, w, p, k, 2)
        forms[MODE_NAMES[p]] = {"ms": r4(1e3 * dtp / k), "eps2": r4(e2p)}
    # the fast form with the online tuner (h2_opts.autotune): its warm-up products settle
    # the choice of kernel and split-K per batch shape
    P.set_autotune(True)
    k = max(1, min(args.steps, 5))
    dtp, _, e2p = timed(G, w, P.H2_AUTO, k, 6)
    P.set_autotune(False)
    forms[MODE_NAMES[fast] + "+tuner"] = {"ms": r4(1e3 * dtp / k), "eps2": r4(e2p)}
    # end to end through the public API with host buffers: points host->device,
    # build, product, result structure (permutation and ranks) device->host
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        X = P.h2_build_interp(pts, w["kernel"], w["leaf"], w["eta"], w["order"], stream=sptr)
        Z = P.h2_clone(X, stream=sptr)
        P.h2_mul_add(Z, X, X, w["eps"], P.H2_AUTO, stream=sptr)
        _ = Z.structure()
        Z.free()
        X.free()
    torch.cuda.synchronize(dev)
    e2e_dt = (time.perf_counter() - t0) / e2e_steps
    nclusters = G.info()["nclusters"]
    d2h = w["n"] * 8 + 3 * nclusters * 8 + 2 * nclusters * 4

    lib_peaks = library_peaks(torch, dev) if rank == 0 else {}
    ff = family_sums(stf)
    roof = roofline(ff, fast, peaks, lib_peaks)
    roof64 = roofline(family_sums(st64), P.H2_FP64, peaks, lib_peaks)

    # the other workloads: one warm-up and two timed products of the fast form,
    # one timed product of the FP64 form (after the fast form planned the structure)
    configs = {}
    if args.configs == "all" and world == 1:
        # the large workloads take the library's own device memory: its stream-ordered
        # pool reuses freed memory across the call's streams, while PyTorch's caching
        # allocator keeps one pool per stream, and the n = 131072 cube at eps 1e-6
        # needs over 250 GB at its peak
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        P.set_allocator("library")
        # without the tuner, as the line: its exploration (forced split-K slices) would
        # raise the peak memory
        for name, c in CONFIGS.items():
            pc = synth.make_points(c["geometry"], c["n"], c["seed"])
            Gc = P.h2_build_interp(pc, c["kernel"], c["leaf"], c["eta"], c["order"], stream=sptr)
            dfc, sfc, e2c = timed(Gc, c, P.H2_AUTO, 2, 1, eps2=(c["n"] <= 131072))
            d64c, _, _ = timed(Gc, c, P.H2_FP64, 1, 0, eps2=False)
            rf = roofline(family_sums(sfc), resolve_precision(P.H2_AUTO, c["eps"]), peaks, lib_peaks)
            configs[name] = {"mode": MODE_NAMES[resolve_precision(P.H2_AUTO, c["eps"])], "alloc": "library",
                             "ms": r4(1e3 * dfc / 2), "fp64_ms": r4(1e3 * d64c), "speedup": r4(d64c / (dfc / 2)),
                             "rows_s": r4(c["n"] * 2 / dfc), "eps2": r4(e2c),
                             "top": rf["kernel"], "frac": rf["frac"]}
            Gc.free()
        configs["batched64"] = batched_record(P, torch, dev, fp64=True)

    n_all = w["n"] * world
    value = n_all * args.steps / dtf
    line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dtf / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "%s products, f64 QR/SVD" % MODE_NAMES[fast],
            "data": "synthetic (seeded SplitMix64 points on the unit sphere)",
            "config": {"workload": w["name"], "n": w["n"], "leaf": w["leaf"], "eta": w["eta"],
                       "order": w["order"], "eps": w["eps"], "precision": "H2_AUTO -> " + MODE_NAMES[fast],
                       "autotune": False,
                       "X=Y=Z": True, "l2": "inputs larger than L2 (X: %.0f MB)" % (G.info()["device_bytes"] / 1e6),
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stf)),
            "roofline": roof,
            "clocks": clocks,
            "e2e": {"value": r4(n_all / e2e_dt), "unit": "rows/s", "h2d_bytes_per_step": int(pts.nbytes),
                    "d2h_bytes_per_step": int(d2h),
                    "note": "host points -> build + clone + h2_mul_add -> ranks and permutation back "
                            "(not the couplings: a lower bound on a full round trip)"}}
    if rank == 0 and not args.no_cpu_baseline:
        v, dt = run_cpu_sample()
        line["cpu_baseline"] = cpu_baseline_record(v, dt)
    # short records last, where a truncated tail still shows them
    line["fp64"] = {"value": r4(n_all * args.steps / dt64), "ms_per_step": r4(1e3 * dt64 / args.steps),
                    "top": roof64["kernel"], "frac": roof64["frac"]}
    line["speedup_vs_fp64"] = r4(dt64 / dtf)
    line["eps2"] = {"fast": r4(e2f), "fp64": r4(e264)}
    line["forms_ms"] = forms
    line["configs"] = configs
    G.free()
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


def batched_record(P, torch, dev, fp64=True, fast_reps=1):
    """The 64-product batch through h2_mul_add_batched: one warm-up and
    fast_reps timed calls of the fast form (H2_AUTO at eps 1e-5), one timed
    call of the FP64 form; CUDA events on the calling stream around each call
    (the call returns when its products are done)."""
    members = batch_members()
    Gs = [P.h2_build_interp(synth.make_points(g, n, seed), 0, BATCH["leaf"], BATCH["eta"], m)
          for g, n, m, seed in members]
    rows = sum(n for _, n, _, _ in members)
    stream = torch.cuda.current_stream(dev)
    out = {"products": len(members), "rows": rows}
    launches = 0
    for name, prec, warm, reps in (("fast", P.H2_AUTO, 1, fast_reps), ("fp64", P.H2_FP64, 0, 1 if fp64 else 0)):
        times = []
        for it in range(warm + reps):
            Zs = [P.h2_clone(G) for G in Gs]
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats, codes = P.h2_mul_add_batched(Zs, Gs, Gs, BATCH["eps"], prec, stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            assert codes == [0] * len(Zs), codes
            for Z in Zs:
                Z.free()
            if it >= warm:
                times.append(e0.elapsed_time(e1) / 1e3)
                if name == "fast":
                    launches = stats["kernel_launches"]
        if times:
            dt = sum(times) / len(times)
            out[name + "_ms"] = r4(1e3 * dt)
            out[name + "_rows_s"] = r4(rows / dt)
    out["mode"] = MODE_NAMES[resolve_precision(P.H2_AUTO, BATCH["eps"])]
    if "fp64_ms" in out:
        out["speedup"] = r4(out["fp64_ms"] / out["fast_ms"])
    out["launches"] = launches
    for G in Gs:
        G.free()
    return out


def batched_arm(args):
    import torch

    import paper_2309_09061_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.build()
    P.load()
    rec = batched_record(P, torch, dev, fp64=True, fast_reps=max(1, args.steps))
    line = {"metric": "H2 Z<-Z+XY rows/s, 64 independent products in one batched call",
            "value": rec["fast_rows_s"] * world, "unit": "rows/s", "n_gpus": world, "steps": max(1, args.steps),
            "warmup": 1, "ms_per_step": rec["fast_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "%s products, f64 QR/SVD" % rec["mode"], "data": "synthetic",
            "config": {"workload": "batched64", "products": rec["products"], "rows": rec["rows"],
                       "eps": BATCH["eps"]},
            "gpu_launches": rec["launches"], "batched": rec}
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
