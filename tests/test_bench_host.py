"""Host logic of bench.py that decides what its JSON line claims (no GPU):

* the DRAM traffic of the dominant kernel is taken from a committed ncu summary only while the
  CUDA sources hash to what that capture saw;
* the history's flop count with the fast history equals the direct count while no block
  boundary is crossed, and is below it after;
* the run-time estimate behind the default run's budget grows with every march it includes.
"""
import math
import os

import numpy as np
import pytest

import bench


def _fake_tree(tmp_path, body: str):
    csrc = tmp_path / "paper_1603_00279_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text(body)
    (csrc / "b.cuh").write_text("// header\n")
    (csrc / "notes.txt").write_text("not a source\n")
    (tmp_path / "profiles").mkdir()
    return csrc


def test_kernel_hash_follows_cuda_sources_only(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path, "__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_sha()
    assert h0 == bench.kernel_sources_sha()
    (csrc / "notes.txt").write_text("changed\n")
    assert bench.kernel_sources_sha() == h0
    (csrc / "b.cuh").write_text("// header, changed\n")
    assert bench.kernel_sources_sha() != h0


def test_captured_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_sources_sha()
    prof = tmp_path / "profiles" / "k.md"
    prof.write_text("# capture\n\n- traffic_bytes_per_launch: 123456789\n"
                    f"- kernel_sources_sha256: `{sha}`\n")
    traffic, src = bench.captured_traffic("k.md")
    assert traffic == 123456789.0 and "profiles/k.md" in src
    (tmp_path / "paper_1603_00279_gb300" / "csrc" / "a.cu").write_text("__global__ void k2() {}\n")
    traffic, src = bench.captured_traffic("k.md")
    assert traffic is None and "changed" in src
    assert bench.captured_traffic("missing.md")[0] is None
    (tmp_path / "profiles" / "bad.md").write_text("- kernel_sources_sha256: x\n")
    assert bench.captured_traffic("bad.md")[0] is None


def test_committed_traffic_profile_has_both_lines():
    """The profile the default line reads holds a traffic figure and a source hash."""
    path = os.path.join(bench.ROOT, "profiles", "level_kernel_precision_n1048575_dram.md")
    text = open(path).read()
    assert "traffic_bytes_per_launch:" in text and "kernel_sources_sha256:" in text


@pytest.mark.parametrize("M", [1, 2, 50, 127, 128])
def test_fast_history_flops_equal_direct_below_the_first_block(M):
    """With M <= B = 128 no level reaches a far block: level j sums its j direct terms (2 flops
    each), which is the direct count 2 n M (M - 1) / 2 of the history term of _alg_flops."""
    n = 1000
    hist_direct = 2.0 * n * (M * (M - 1) / 2.0)
    assert bench._fast_history_flops(n, M) == hist_direct
    assert bench._alg_flops(n, M, "none", np.zeros(M), 0) >= hist_direct


def test_fast_history_flops_below_direct_at_the_history_workload():
    n, M = (1 << 18) - 1, 8192
    fast = bench._fast_history_flops(n, M)
    direct = 2.0 * n * (M * (M - 1) / 2.0)
    # per point: about log2(2B)-scaled FFT work per block plus O(M^2 / B) accumulation
    assert 0.005 * direct < fast < 0.2 * direct, fast / direct


def test_alg_flops_counts_one_rhs_product_per_level_and_four_per_iteration():
    n, M = 127, 4
    L = 256
    conv = 5.0 * L * math.log2(L) + 3.0 * L
    its = np.array([7, 6, 6, 5])
    f = bench._alg_flops(n, M, "strang", its, 1)
    sym = 12.5 * L * math.log2(L) + 24.0 * n
    hist = 2.0 * n * (M * (M - 1) / 2.0)
    vec = 19.0 * n * its.sum() + 12.0 * n * M
    assert f == pytest.approx(conv * (M + 4 * its.sum()) + sym + hist + vec)
    # without a preconditioner: two products per iteration and no symbols
    f0 = bench._alg_flops(n, M, "none", its, 1)
    assert f0 == pytest.approx(conv * (M + 2 * its.sum()) + hist + vec)


def test_estimate_grows_with_every_march():
    base = bench.estimate_total_s(10.0, 1.0, steps=20, warmup=5, cpu_budget=15.0)
    assert bench.estimate_total_s(11.0, 1.0, steps=20, warmup=5, cpu_budget=15.0) - base == \
        pytest.approx(26.0)          # 5 warm-up + 20 timed + 1 end-to-end march
    assert bench.estimate_total_s(10.0, 1.0, steps=20, warmup=5, cpu_budget=15.0,
                                  mixed_march_s=10.0) > base
