"""The roofline arithmetic bench.py reports (host only)."""
import importlib.util
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bench():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")
    spec = importlib.util.spec_from_file_location("bench_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flop_per_unit(bench):
    from paper_2209_09848_gb300 import synth
    vx, _ = synth.velocity_grid(10, 10)
    assert bench.flop_per_unit(1, vx) == 50.0           # general 5 x 5: 25 FMAs
    assert bench.flop_per_unit(2, vx) == pytest.approx(11.0)   # 5 + 5 * 10 / 100 FMAs
    assert bench.flop_per_unit(2, vx, taps=1) == pytest.approx(2.2)
    vx2, _ = synth.velocity_grid(40, 25)
    assert bench.flop_per_unit(2, vx2) == pytest.approx(2 * (5 + 5 * 40 / 1000))
    assert bench.flop_per_unit(2, np.arange(7.0)) == pytest.approx(20.0)  # every v_x distinct


def test_peak_and_paper_rate(bench):
    assert bench._fp32_peak_tflops(2070.0, sms=152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.PAPER_RATE == pytest.approx(100 * 1000 * 2048 * 2048 / 300.0)
    assert bench.job_throughput(10.0, 4, 2.0) == 20.0


def test_traffic_comes_from_the_committed_summaries(bench):
    # the bench's roofline.traffic is the DRAM bytes per traj*pixel*frame
    # recorded in the ncu summary of the kernel the plan uses (a small case
    # of the same plan), times the step's units
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for kernel, name in ((2, "k_numerator_fac_paper_shaped.md"), (1, "k_numerator_paper_shaped.md")):
        text = open(os.path.join(root, "profiles", name)).read()
        m = re.search(r"^traffic_bytes_per_unit:\s*(\S+)", text, re.M)
        want = None if m is None or m.group(1) == "null" else float(m.group(1))
        assert bench._traffic_from_profiles(kernel) == want
    assert bench._traffic_from_profiles(2) == pytest.approx(0.1070)
