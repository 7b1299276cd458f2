"""The bench's roofline accounting on CPU: the per-kernel tables line up with
the six stages adr_time_kernels reports, and the whole-step HBM figure is the
DRAM bytes (or algorithmic bytes) of the stages that ran over their summed
time, against the measured copy peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_tables_cover_the_six_stages():
    import bench
    for table in (bench.KERNELS, bench.BYTES_PER_UNIT, bench.FLOPS_PER_UNIT, bench.NCU_TRAFFIC_SHEARED2048,
                  bench.KERNELS_DIRECT, bench.BYTES_PER_UNIT_DIRECT, bench.FLOPS_PER_UNIT_DIRECT,
                  bench.NCU_TRAFFIC_DIRECT_SHEARED2048):
        assert len(table) == 6
    # the direct transfer has no gather stages: nothing is counted for them
    assert bench.BYTES_PER_UNIT_DIRECT[0] == bench.BYTES_PER_UNIT_DIRECT[3] == 0.0


def test_step_hbm_sums_the_stages_that_ran():
    import bench
    hbm, _ = bench.peaks()
    ms = [0.05, 0.1, 0.08, 0.0, 0.1, 0.1]  # stage 3 did not run
    alg = [200e6, 300e6, 340e6, 999e6, 210e6, 370e6]
    traffic = [210e6, 350e6, 400e6, None, 260e6, 430e6]
    out = bench.step_hbm({"all_kernels_ms_list": ms, "algorithmic_bytes_list": alg}, traffic)
    t = sum(ms) * 1e-3
    assert out["ms"] == pytest.approx(sum(ms))
    assert out["dram_bytes"] == pytest.approx(1650e6)
    assert out["algorithmic_bytes"] == pytest.approx(1420e6)
    assert out["dram_frac"] == pytest.approx(1650e6 / t / 1e9 / hbm)
    assert out["algorithmic_frac"] == pytest.approx(1420e6 / t / 1e9 / hbm)
