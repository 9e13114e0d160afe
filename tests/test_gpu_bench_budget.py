"""The benchmark's default run fits well inside the time a benchmark run is given.

A short timed segment of the default workload (the precision workload, n = 2^20 - 1, M = 512, FP64,
64 levels per launch, autotuned plan) gives the cost of a level; the whole default run of
`bench.py --steps 20 --warmup 5` (5 warm-up marches, 20 timed marches, one end-to-end march, the
mixed-precision leg, the CPU oracle leg and both setups) is estimated from it and must stay under
900 s.
"""
import time

import pytest

import tsfcde_workloads as W
from gpu_common import solver_module

pytestmark = pytest.mark.gpu


def test_default_bench_run_fits_budget():
    import bench
    P = solver_module()
    prob = W.config_mixed()
    t0 = time.perf_counter()
    s = P.Solver.from_problem(prob, source="separable", autotune=True, levels_per_launch=64)
    setup_s = time.perf_counter() - t0
    seg = 16
    s.step(2)                                   # warm the plan
    st = s.step(seg)
    s.close()
    per_level_s = st["device_ms"] / 1e3 / seg
    # the history sum grows with j: 8 j n bytes at level j, at no less than 2 TB/s
    hist_s = sum(8.0 * j * prob.n / 2e12 for j in range(prob.M))
    march_s = prob.M * per_level_s + hist_s
    total = bench.estimate_total_s(march_s, setup_s, steps=20, warmup=5, cpu_budget=15.0,
                                   mixed_march_s=march_s)
    print(f"level {1e3 * per_level_s:.2f} ms, march {march_s:.1f} s, setup {setup_s:.1f} s, "
          f"estimated default run {total:.0f} s")
    assert total < 900.0, total
