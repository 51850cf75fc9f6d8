"""Timing of the dual-operator block apply Y = F X on one GPU.

Sets up and factorizes a synthetic modular problem (the 2D binary-module
layout or the 3D smoothed-field layout), then times ``feti_apply_dual`` on m
seeded random columns with CUDA events on the library's stream, writing a
buffer larger than L2 between launches.  Prints one JSON line: the time per
apply, and from the library's profile the time and algorithmic TFLOP/s of the
tensor-core local product (precision form) or of the FP64 GEMMs (FP64 form).

    python -m paper_2111_11728_gb300.applybench --dim 3 --tiles 8 --precision tf32x3 --m 512
"""
import argparse
import json
import os
import statistics
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3, choices=[2, 3])
    ap.add_argument("--tiles", type=int, default=8)
    ap.add_argument("--elems", type=int, default=None)
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "tf32x3", "bf16", "bf16x3"])
    ap.add_argument("--method", default="fetidp", choices=["fetidp", "tfeti"])
    ap.add_argument("--m", type=int, default=512)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)

    import torch

    import workloads
    import paper_2111_11728_gb300 as fg

    if a.dim == 3:
        p = workloads.config4(tiles=a.tiles, elems=a.elems or 8)
    else:
        p = workloads.config2(tiles=a.tiles, elems=a.elems or 32)
    prec = {"fp64": fg.FETI_FP64, "tf32": fg.FETI_TF32, "tf32x3": fg.FETI_TF32X3, "bf16": fg.FETI_BF16,
            "bf16x3": fg.FETI_BF16X3}[a.precision]
    method = {"fetidp": fg.FETI_FETIDP, "tfeti": fg.FETI_TFETI}[a.method]
    stream = torch.cuda.current_stream()
    s = fg.Solver(method, fg.FETI_SCALING_K, fg.FETI_RRS, stream=stream.cuda_stream, precision=prec)
    s.setup(p, rho=torch.from_numpy(p.rho).cuda(), f=torch.from_numpy(p.f).cuda(), on_device=True)
    fg.feti_factorize(s.ctx)
    n = s.query(fg.FETI_Q_N_LAMBDA)
    X = torch.from_numpy(np.random.default_rng(a.m).standard_normal((a.m, n))).cuda()
    Y = torch.zeros_like(X)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(a.warmup):
        fg.feti_apply_dual(s.ctx, X, n, a.m, Y, n)
        flush.zero_()
    torch.cuda.synchronize()
    times = []
    fg.feti_profile_begin(s.ctx)
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fg.feti_apply_dual(s.ctx, X, n, a.m, Y, n)
        e1.record(stream)
        flush.zero_()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    gf, gms, gn = fg.feti_profile_end(s.ctx)
    tf, tms, tn = fg.feti_profile_tensor(s.ctx)
    out = {"dim": a.dim, "tiles": a.tiles, "elems": a.elems or (8 if a.dim == 3 else 32), "method": a.method,
           "precision": a.precision, "m": a.m, "n_lambda": n, "n_sub": s.query(fg.FETI_Q_N_SUBDOMAINS),
           "max_nb": s.query(fg.FETI_Q_MAX_NB), "apply_ms_median": statistics.median(times),
           "apply_ms_min": min(times), "f_applies_per_s": a.m / (statistics.median(times) / 1e3)}
    if tn:
        out["tensor_product"] = {"launches": tn, "ms_per_launch": tms / tn, "alg_tflops": tf / (tms / 1e3) / 1e12}
        # the whole apply against the HBM roofline: the scaled local blocks read once,
        # the FP32 interface vectors in and out, the FP64 multiplier block in and out
        nbytes = (s.query(fg.FETI_Q_TC_BYTES_F) + 2.0 * 4 * s.query(fg.FETI_Q_N_B_TOTAL) * a.m
                  + 2.0 * 8 * n * a.m)
        out["apply_hbm"] = {"algorithmic_bytes": nbytes,
                            "achieved_gbs": nbytes / (statistics.median(times) / 1e3) / 1e9}
    if gn:
        out["fp64_gemm"] = {"launches": gn, "ms": gms / a.reps, "alg_tflops": gf / (gms / 1e3) / 1e12}
    s.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
