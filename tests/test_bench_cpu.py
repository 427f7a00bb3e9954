"""Host logic of bench.py on the CPU: the launch counts it claims per step,
the staleness check of the committed ncu counters, and the workload table."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_counts_per_step():
    W = bench.WORKLOADS
    # mask 1, step size 2 + 156; tensor call: filters, counts, scan 3, pack,
    # A tiles, 2 per iteration (3 with an observation mask), unpack
    assert bench.launches_per_step(W["c3"], "bf16", 100, 64, False) == 1 + 158 + 8 + 200
    assert bench.launches_per_step(W["inpaint"], "bf16", 50, 10, False) == 1 + 158 + 8 + 150
    # plain path: apply-mask 1, synthesis and adjoint per iteration (per image)
    assert bench.launches_per_step(W["c3"], "fp32", 100, 64, False) == 1 + 158 + 1 + 200
    assert bench.launches_per_step(W["c5"], "fp32", 20, 512, True) == 1 + 158 + 1 + 20 * 1024
    # screening: 7 launches per test, a tensor call per chunk of 25 iterations
    assert bench.launches_per_step(W["screen"], "bf16", 100, 64, False) == \
        1 + 158 + 4 * (7 + 8 + 50)
    # ADMM: mask, init, A^T x, per iteration 1 + 3 + 1 + 2 + 7 per CG step + 1, final
    assert bench.launches_per_step(W["admm"], "fp32", 10, 10, False) == \
        1 + 2 + 10 * (8 + 7 * 20) + 1


def test_counter_staleness_follows_code_not_comments():
    src = "int f(int a) {\n  // one\n  return a + 1; /* two */\n}\n"
    same = "int f(int a) {   return a + 1;\n}  // three\n"
    other = "int f(int a) {\n  return a + 2;\n}\n"
    h = bench.source_code_sha1
    assert h(src) == h(same)
    assert h(src) != h(other)


def test_traffic_comes_from_the_counters_only_while_the_code_matches():
    with open(os.path.join(ROOT, "profiles", "tc_kernels_prof_workload_counters.json")) as f:
        c = json.load(f)
    with open(os.path.join(ROOT, c["source"])) as f:
        current = bench.source_code_sha1(f.read()) == c["source_code_sha1"]
    t = bench.measured_traffic("adj_tc", 2 * c["workload_pixels"])
    if current:
        assert t == 2 * c["kernels"]["adj2_kernel"]["dram_bytes_per_launch"]
    else:
        assert t is None


def test_workloads_name_their_configuration():
    for name, wl in bench.WORKLOADS.items():
        assert wl["K"] > 0 and wl["n_iters"] > 0 and wl["desc"]
        assert wl["p"][0] <= wl["p"][1]
    assert bench.WORKLOADS["c3"]["n"] == 64 and bench.WORKLOADS["c3"]["K"] == 100
