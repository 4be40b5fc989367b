"""Host-side arithmetic of bench.py's roofline object (no GPU)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def phases():
    ms = {"deposit": 50.0, "fft_fwd": 60.0, "poisson": 54.0, "fft_inv": 38.0, "fft_inv_x": 46.0,
          "gather": 58.0, "ics": 9.0, "power": 15.0}
    n = {k: 10 for k in ms}
    n["ics"] = n["power"] = 1
    return ms, n


def test_roofline_is_the_dominant_single_kernel_phase():
    ms, n = phases()
    r = bench.roofline(ms, n, 512, 1024, 6691.5)
    assert r["kernel"] == "gather"          # the forward passes take longer but are two kernels
    nbytes = 80 * 512 ** 3 + 12 * 1024 ** 3
    assert r["alg_bytes"] == nbytes
    assert abs(r["achieved"] - nbytes / 5.8e-3 / 1e9) <= 1e-9 * r["achieved"]
    assert r["frac"] == r["achieved"] / 6691.5 and r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert abs(r["traffic"] - 8 * bench.DRAM_512["gather"]) < 1.0   # 512^3 capture x cell ratio


def test_roofline_per_call_time_and_traffic_scope():
    ms, n = phases()
    ms["poisson"] = 90.0
    n["poisson"] = 15                        # mean call time, not the total
    r = bench.roofline(ms, n, 512, 1024, 6691.5)
    assert r["kernel"] == "poisson"
    assert abs(r["achieved"] - 12 * 1024 ** 3 / 6e-3 / 1e9) <= 1e-9 * r["achieved"]
    assert bench.roofline(ms, n, 512, 512, 6691.5)["traffic"] is None   # not N_m = 2 N_p


def test_roofline_traffic_of_a_kernel_that_runs_only_at_1024():
    """The force z pass at 1024^3 is another kernel (each task on a pair of lanes) than the one
    measured at 512^3: its traffic is its own 1024^3 measurement, not the scaled 512^3 one."""
    ms, n = phases()
    ms["poisson"] = 90.0
    r = bench.roofline(ms, n, 512, 1024, 6786.2)
    assert r["kernel"] == "poisson" and r["traffic"] == bench.DRAM_1024["poisson"]
    assert 1.0 <= r["traffic"] / r["alg_bytes"] < 1.1
    r = bench.roofline(ms, n, 256, 512, 6786.2)
    assert r["traffic"] == bench.DRAM_512["poisson"]
