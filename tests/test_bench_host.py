"""bench.py's host-side pieces: the committed ncu summaries it reads and its
per-ray work figures (no GPU)."""
import os
import re

import bench


def _kv(path):
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


def test_committed_profiles_carry_the_figures_bench_reads():
    for prec in ("fp32", "fp64"):
        kv = _kv(os.path.join(bench.ROOT, "profiles", f"k_ao_walk_{prec}_paper_1mp.txt"))
        assert re.fullmatch(r"[0-9a-f]{16}", kv["sources_hash"])
        assert float(kv["dram_bytes_per_launch"]) > 0
    kv = _kv(os.path.join(bench.ROOT, "profiles", "k_ao_walk_fp32_paper_1mp.txt"))
    assert 0 < float(kv["issue_active_pct"]) <= 100
    # the issue bound's count: warp instructions of one launch, with the launch
    # shape it was taken at
    assert float(kv["warp_instructions_per_launch"]) > 1e8
    assert {"grid_lambda", "refill", "block"} <= set(kv)


def test_profile_ignored_once_the_kernel_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "sources_hash", lambda: "0" * 16)
    assert bench.committed_profile("paper_1mp", "fp32") == {}
    assert bench.committed_traffic("paper_1mp", "fp32") is None


def test_sources_hash_ignores_comments():
    a = bench._code_only("int x; // one\n/* two */ int y;\n")
    b = bench._code_only("int x; // another\n/* three\n lines */ int y;\n")
    assert a == b


def test_per_ray_work_counts():
    c = {"ao_rays": 2, "ao_cells": 10, "ao_sphere_tests": 4, "ao_cylinder_tests": 2}
    flops, nbytes = bench.per_ray_work(c, "ao")
    assert flops == (10 * bench.FLOPS_CELL + 4 * bench.FLOPS_SPHERE + 2 * bench.FLOPS_CYLINDER) / 2
    assert nbytes == (10 * bench.BYTES_CELL + 6 * bench.BYTES_ITEM + 4 * bench.BYTES_SPHERE
                      + 2 * bench.BYTES_CYLINDER) / 2
    fd, _ = bench.per_ray_work(c, "ao", device_formulas=True)
    assert fd > flops
