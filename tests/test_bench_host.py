"""bench.py on the host: the workload definitions have the sizes their
descriptions state, and the helpers of the JSON line compute what they claim."""
import time

import numpy as np

import bench


def test_workload_sizes():
    w = bench.make_workload("er5000")
    assert w["pattern"][0] == 5000 and w["m"] == 8 and w["opts"] == dict(ordering="mindeg", relax=16)
    assert w["gram"] == (50, 0.1)
    w = bench.make_workload("band200")
    n, cp, ri = w["pattern"]
    assert n == 200 and w["m"] == 1 and int(np.max(ri - np.repeat(np.arange(n), np.diff(cp)))) == 8
    assert w["gram"] == (20, 1.0)
    w = bench.make_workload("grid150")
    assert w["pattern"][0] == 22500 and w["m"] == 64
    w = bench.make_workload("batch256")
    assert len(w["batch"]) == 256 and w["m"] == 4
    w = bench.make_workload("serve")
    pool = w["pool"]
    assert len(pool) == 32 and w["rate"] == 2000.0 and w["m"] == 16
    assert pool[-1][0][0] == 64000  # the 40^3 grid
    assert all(1000 <= p[0][0] <= 61000 for p in pool[:-1])
    assert abs(sum(w["mix"].values()) - 1.0) < 1e-12 and w["mix"]["hessian"] == 0.5


def test_hbm_line_and_peak():
    peak, src = bench.hbm_peak_gbs()
    assert src in ("measured", "fallback") and peak > 1000.0
    h = bench.hbm_line(8e9, 1000.0)  # 8 GB in one second
    assert abs(h["achieved"] - 8.0) < 1e-12 and abs(h["frac"] - 8.0 / peak) < 1e-15 and h["unit"] == "GB/s"


def test_fp64_peak_from_unit_counts():
    assert abs(bench.FP64_PEAK_TFLOPS - 152 * 2.07e9 * 4 / 1e12) < 1e-12


def test_oracle_sample_repeats_to_its_budget():
    w = bench.make_workload("band200")
    n, cp, ri = w["pattern"]
    x, ys, _ = bench.workload_values(w, n, cp, ri)
    t0 = time.perf_counter()
    tz, te, reps = bench.oracle_hessian_repeated(w, n, cp, ri, x, ys, 1, budget_s=0.2)
    assert reps >= 1 and tz > 0 and te > 0
    assert time.perf_counter() - t0 >= 0.2 or reps == 1


def test_reference_arm_loads_no_library():
    """The CPU oracle's arm runs without the library: the analysed pattern
    comes from the oracle (for the Erdos-Renyi workload from the stored
    analysis, equal to the library's, see test_symbolic_host)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys, runpy; sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'band200', "
            "'--steps', '1', '--warmup', '3']\n"
            "runpy.run_path('bench.py', run_name='__main__')\n"
            "maps = open('/proc/self/maps').read()\n"
            "print('LOADED', 'libchordal_barrier' in maps, any('binding' in m for m in sys.modules))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().splitlines()
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["n"] == 200
    assert lines[-1] == "LOADED False False"


def test_reference_pattern_of_stored_analysis():
    """The reference arm's Erdos-Renyi pattern has the workload's size."""
    n, cp, ri = bench.reference_pattern(bench.make_workload("er5000"))
    assert n == 5000 and len(cp) == n + 1 and cp[-1] == len(ri) == 1114524
