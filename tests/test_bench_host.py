"""Host logic of bench.py: the algorithmic bytes of a rotation against the
closed form B(l) = 8N [2 ceil(l/alpha)(l+K) + 4l] (key read once, ciphertext
in and out), the roofline arithmetic, and the all-cores oracle timing
(spawned processes) on a small parameter set."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2510_03996_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("level", [4, 9, 16, 24])
def test_rotation_bytes_closed_form(level):
    N, L, K, alpha = 1 << 16, 24, 4, 4
    c = bench.algorithmic_costs(N, L, K, alpha, level)
    assert c["bytes"] == 8 * N * (2 * math.ceil(level / alpha) * (level + K) + 4 * level)
    # the inner product reads every key limb once, every raised digit once, writes two accumulators
    beta = math.ceil(level / alpha)
    ip = c["kernels"]["ks_inner"]["bytes"]
    assert ip == 8 * N * (2 * beta * (level + K) + beta * (level + K) + 2 * (level + K))
    # ModUp: new limbs = digits x (level + K) minus the digits' own limbs
    new = beta * (level + K) - level
    up = c["kernels"]["up_ntt_rows"]["mm"]
    assert sum(up.values()) == new * (N // 2) * 8
    # 50-bit Q primes take the lazy butterflies, 60-bit P primes Harvey's
    assert up.get("ct_lazy", 0) == (beta * level - level) * (N // 2) * 8 and up["ct_harvey"] == beta * K * (N // 2) * 8
    # ModUp's conversions: digit j of d_j limbs feeds the level + K - d_j other limbs
    digits = [min(alpha, level - j * alpha) for j in range(beta)]
    assert c["kernels"]["up_bconv_ntt_cols"]["mm"]["mac"] == N * sum(d * (level + K - d) for d in digits)
    assert c["kernels"]["dn_intt_rows"]["mm"] == {"gs_harvey": 2 * K * (N // 2) * 8}


def test_the_published_mean_bytes():
    """The mean over U{4..24} of B(l) at the rotation workload's sizes is 111.6 MB."""
    N = 1 << 16
    mean = sum(bench.algorithmic_costs(N, 24, 4, 4, lv)["bytes"] for lv in range(4, 25)) / 21
    assert abs(mean / 1e6 - 111.6) < 0.6


def test_roofline_arithmetic():
    costs = [bench.algorithmic_costs(1 << 16, 24, 4, 4, 12)]
    prof = {"ks_inner": (2, 1.0), "up_ntt_rows": (2, 2.0), "unknown": (1, 1.0)}
    rates = {"ct_lazy": 2e12, "gs_lazy": 2e12, "ct_harvey": 1e12, "gs_harvey": 1e12, "mac": 4e12}
    r = bench.rooflines(prof, costs, steps=2, hbm_peak=6784.5, alu_rates=rates)
    ip = costs[0]["kernels"]["ks_inner"]["bytes"] * 2 / 1e-3 / 1e9
    assert abs(r["ks_inner"]["achieved"] - ip) < 1e-6 and r["ks_inner"]["bound"] == "hbm"
    assert abs(r["ks_inner"]["frac"] - ip / 6784.5) < 1e-12
    up = r["up_ntt_rows"]
    assert up["bound"] == "alu" and up["avg_launch_ms"] == 1.0
    # frac = the shortest time at the measured rates over the measured time
    mm = costs[0]["kernels"]["up_ntt_rows"]["mm"]
    t_min = 2 * sum(v / rates[k] for k, v in mm.items())
    assert up["frac"] == pytest.approx(t_min / 2e-3)
    assert up["achieved"] == pytest.approx(2 * sum(mm.values()) / 2e-3 / 1e12)
    assert up["peak"] == pytest.approx(2 * sum(mm.values()) / t_min / 1e12)
    assert "unknown" not in r


def test_oracle_on_every_core():
    P = synth.params("tiny")
    rate, done, slowest, cores = bench.oracle_all_cores(P, 3, [2, 3, 4], per_core=2, cores=2)
    assert cores == 2 and done == 4 and slowest > 0 and rate == pytest.approx(done / slowest)


def test_reference_pool_steps_every_core():
    P = synth.params("tiny")
    pool = bench.OraclePool(P, 3, cores=2)
    try:
        t = pool.step([2, 4])
        assert t > 0
        assert pool.step([3, 3]) > 0
    finally:
        pool.close()
    assert all(p.exitcode == 0 for p in pool.procs)


def test_step_summary_and_clock_summary():
    s = bench.step_summary([37.5, 37.4, 150.2, 37.6])
    assert s == {"step_ms_median": 37.55, "step_ms_max": 150.2, "slowest_step": 3}
    assert bench.step_summary([]) == {}
    c = bench.ClockSampler(0)
    c.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1500", "2070", "1400", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2070", "2070", "950", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    out = c.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_min_mhz"] == 1500.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
