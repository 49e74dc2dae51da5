"""Host-side logic of the benchmark that decides what its JSON line says:
the measured break-even crossover of the gate leg, the clock summary that
accepts or rejects a run, the GPU-local core set the process binds to, the
parser's defaults against the timing rules, and the filter traffic constants
against the algorithmic bytes.  No GPU is touched."""
import math

import numpy as np
import pytest

import bench


# -- crossover of the measured gain (gate leg, Sec. V-D) ----------------------

def test_crossover_interpolates_in_log_n():
    ns = [1e3, 1e4, 1e5, 1e6]
    gain = [-3.0, -1.0, 1.0, 5.0]              # sign change between 1e4 and 1e5, halfway
    x = bench._crossover(ns, gain)
    assert math.isclose(x, math.sqrt(1e4 * 1e5), rel_tol=1e-12)


def test_crossover_exact_for_gain_linear_in_log_n():
    ns = np.geomspace(1e3, 1e8, 11)
    root = 3.7e5
    gain = [math.log(n / root) for n in ns]
    assert math.isclose(bench._crossover(ns, gain), root, rel_tol=1e-9)


def test_crossover_edge_cases():
    ns = [10.0, 100.0, 1000.0]
    assert bench._crossover(ns, [1.0, 2.0, 3.0]) == 10.0         # positive everywhere: the first point
    assert bench._crossover(ns, [-1.0, -2.0, -0.5]) == 0.0       # never positive: none
    # a zero gain is not positive; the interpolated root is that point itself
    assert bench._crossover(ns, [-1.0, 0.0, 1.0]) == pytest.approx(100.0)
    # positive, then negative again, then positive: the crossover that stays
    x = bench._crossover([1.0, 10.0, 100.0, 1000.0], [1.0, -1.0, -1.0, 1.0])
    assert 100.0 < x < 1000.0


# -- clock summary (rejection rules for a timed run) --------------------------

def _clk(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_median_and_reasons():
    rows = [f"{sm}, 2070, 900.5, 3996, Not Active, Not Active, Not Active, {cap}"
            for sm, cap in ((2070, "Not Active"), (1995, "Active"), (2070, "Not Active"))]
    s = _clk(rows + ["garbage", "1, 2, 3"])                     # malformed lines are skipped
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["mem_mhz"] == 3996.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_each_throttle_reason():
    row = "1500, 2070, 1300, 3996, Active, Active, Active, Not Active"
    assert _clk([row])["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = _clk([])
    assert s["sm_mhz"] is None and s["reasons"] == ["unavailable"] and s["samples"] == 0
    assert _clk(["[N/A], [N/A], [N/A], [N/A], a, b, c, d"])["samples"] == 0


# -- GPU-local cores from `nvidia-smi topo -m` --------------------------------

TOPO = ("\tGPU0\tGPU1\tNIC0\tCPU Affinity\tNUMA Affinity\tGPU NUMA ID\n"
        "GPU0\t X \tNV18\tSYS\t0-71\t0\t2\n"
        "GPU1\tNV18\t X \tSYS\t72-143,200\t1\t10\n"
        "NIC0\tSYS\tSYS\t X \t\t\t\n"
        "\nLegend:\n\n  X    = Self\n")


def test_topo_affinity_ranges_and_lists():
    assert bench._parse_topo_affinity(TOPO, 0) == set(range(0, 72))
    assert bench._parse_topo_affinity(TOPO, 1) == set(range(72, 144)) | {200}


def test_topo_affinity_missing_pieces():
    assert bench._parse_topo_affinity(TOPO, 5) is None                # no such GPU row
    assert bench._parse_topo_affinity("", 0) is None
    assert bench._parse_topo_affinity(TOPO.replace("CPU Affinity", "CPUs"), 0) is None
    assert bench._parse_topo_affinity(TOPO.replace("0-71", "N/A"), 0) is None


# -- parser defaults against the timing rules ----------------------------------

def test_parser_defaults_follow_the_timing_rules():
    a = bench.build_parser().parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.impl == "ours" and a.log2n == 28 and a.k == 1000 and a.key_type == "i64"
    assert a.dist == "uniform"
    legs = a.workload.split(",")
    assert legs[0] == "topk"
    assert set(legs) == {"topk", "single", "pair", "link", "join", "joincells", "topkcells", "batched", "fullrow",
                         "gate", "serving"}
    # the serving stream as configured: 100,000 requests
    assert a.serve_requests == 100_000
    # the keys at the default size exceed L2 (129 MB), so no flush is needed
    assert (1 << a.log2n) * 8 > 129 * 10**6


def test_filter_traffic_constants_cover_the_algorithmic_bytes():
    """DRAM bytes per key of the filter (from the ncu capture) can never be
    below the bytes it must read, and a pass that re-read keys would be near
    twice that."""
    for kt, width in (("i64", 8), ("f32", 4)):
        per_key = bench.FILTER_DRAM_BYTES_PER_KEY[kt]
        assert width <= per_key < 1.05 * width


# -- latency statistics, launch counts and host description ------------------

def test_median_p95():
    m, p = bench._median_p95(list(range(1, 101)))          # 1..100
    assert m == 50.5
    assert math.isclose(p, 95.05)                          # linear interpolation
    assert bench._median_p95([3.0]) == (3.0, 3.0)


def test_cpu_model_from_lscpu_then_cpuinfo():
    lscpu = "Architecture:  aarch64\nVendor ID:  ARM\nModel name:  Neoverse-V2\nCPU(s): 72\n"
    assert bench._parse_cpu_model(lscpu, "") == "Neoverse-V2"
    cpuinfo = "processor\t: 0\nmodel name\t: Intel(R) Xeon(R) Platinum\nflags\t: fpu\n"
    assert bench._parse_cpu_model("", cpuinfo) == "Intel(R) Xeon(R) Platinum"
    assert bench._parse_cpu_model("Model name: -\n", cpuinfo) == "Intel(R) Xeon(R) Platinum"
    assert bench._parse_cpu_model("", "CPU part\t: 0xd4f\n") is None


def test_host_info_here():
    h = bench._host_info()
    assert h["nproc"] >= 1 and h["machine"]
