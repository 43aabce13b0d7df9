"""Run products of the unit-sphere workload once, for profilers.

    python -m paper_2309_09061_gb300.profile_run [--n 8192] [--precision fp64|mixed|tf32x3|tf32|bf16x3|auto]
        [--eps 1e-6] [--order 4] [--reps 1] [--autotune]

Builds the Laplace H^2-matrix (leaf 64, eta 2, Chebyshev order 4) of n seeded
points on the unit sphere and computes Z <- Z + G G at eps (default 1e-6) on
cuda:0, reps times, printing the last call's statistics as JSON.  With
--autotune the library's online tuner is on (the first products settle it).
Under a profiler, pick the kernels with ncu's -k / -s / -c.
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2309_09061_gb300 as P  # noqa: E402
import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--precision", default="fp64", choices=sorted(P.PRECISIONS) + ["tc"])
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--autotune", action="store_true")
    a = ap.parse_args()
    P.build()
    P.load()
    pts = synth.sphere(a.n, 2309090611)
    G = P.h2_build_interp(pts, P.H2_K_LAPLACE, 64, 2.0, a.order)
    prec = P.H2_TC if a.precision == "tc" else P.PRECISIONS[a.precision]
    P.set_autotune(a.autotune)
    for _ in range(a.reps):
        Z = P.h2_clone(G)
        st = P.h2_mul_add(Z, G, G, a.eps, prec)
        Z.free()
    out = {k: st[k] for k in ("t_rows_a_ms", "t_cols_a_ms", "t_mat_a_ms", "t_rows_b_ms", "t_cols_b_ms",
                              "t_mat_b_ms", "kernel_launches", "max_rank_a", "max_rank_b")}
    # per kernel family: launches and algorithmic GFLOP of the last call
    out["families"] = {P.FAMILIES[i]: {"launches": st["fam_launches"][i], "gflop": st["fam_flops"][i] / 1e9}
                       for i in range(len(P.FAMILIES)) if st["fam_launches"][i]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
