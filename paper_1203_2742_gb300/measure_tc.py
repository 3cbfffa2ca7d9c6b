"""Throughput of the FP64-accurate tensor-core product (chd_dgemm_tc)
against the FP64 GEMM of cuBLAS (torch.matmul in float64), and the rates of
the device's arithmetic units (chd_probe_units, chd_probe_tc_bf16_peak).

    python -m paper_1203_2742_gb300.measure_tc [--one M N K]

Each size runs twice as warm-up, then 5 times between CUDA events; the
chd_dgemm_tc time includes its stream-ordered scratch allocation and the
final synchronisation.  The maximum relative difference to cuBLAS FP64 is
printed beside.  --one M N K runs a single product of that shape once
(after one warm-up), for a profiler.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZES = [(1024, 1024, 1024), (2048, 2048, 1024), (4096, 4096, 1024), (896, 896, 512), (8192, 8192, 1024)]


def main(argv=None):
    import argparse
    import torch
    from paper_1203_2742_gb300 import build
    build.build()
    from paper_1203_2742_gb300 import binding as B
    ap = argparse.ArgumentParser()
    ap.add_argument("--one", type=int, nargs=3, default=None, metavar=("M", "N", "K"))
    a = ap.parse_args(argv)
    torch.manual_seed(0)
    if a.one:
        m, n, k = a.one
        x = torch.randn(k, m, dtype=torch.float64, device="cuda").T
        y = torch.randn(n, k, dtype=torch.float64, device="cuda").T
        B.chd_dgemm_tc(x, y)
        c = B.chd_dgemm_tc(x, y)
        torch.cuda.synchronize()
        print(f"{m}x{n}x{k}: max rel diff {(c - x @ y).abs().max().item() / (x @ y).abs().max().item():.2e}")
        return
    u = B.chd_probe_units()
    print(f"units: FP64 FMA {u['fp64_fma_tflops']:.3f} TFLOP/s, FP64 mma.sync {u['fp64_mma_tflops']:.3f} TFLOP/s, "
          f"FP32 FMA {u['fp32_fma_tflops']:.1f} TFLOP/s, dependent FP64 FMA {u['fp64_fma_latency_ns']:.1f} ns; "
          f"bf16 tcgen05.mma {B.chd_probe_tc_bf16_peak():.1f} TFLOP/s")
    for (m, n, k) in SIZES:
        a = torch.randn(k, m, dtype=torch.float64, device="cuda").T
        b = torch.randn(n, k, dtype=torch.float64, device="cuda").T
        c = torch.zeros(n, m, dtype=torch.float64, device="cuda").T
        for _ in range(2):
            B.chd_dgemm_tc(a, b, c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            B.chd_dgemm_tc(a, b, c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        ref = a @ b
        e0.record()
        for _ in range(reps):
            ref = a @ b
        e1.record()
        torch.cuda.synchronize()
        ms_ref = e0.elapsed_time(e1) / reps
        err = (c - ref).abs().max().item() / ref.abs().max().item()
        print(f"{m}x{n}x{k}: tensor cores {ms:.3f} ms = {2 * m * n * k / ms / 1e9:.1f} TFLOP/s FP64-equivalent; "
              f"cuBLAS FP64 {ms_ref:.3f} ms = {2 * m * n * k / ms_ref / 1e9:.2f} TFLOP/s; max rel diff {err:.2e}",
              flush=True)


if __name__ == "__main__":
    main()
