"""Performance model (Sec. 5) against the worked example the paper prints."""
import os

import pytest

from paper_2204_02064_gb300 import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "perf_model_example.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_worked_example_reproduced():
    g = _golden()
    bw = g["bw_gbs"] * 1e9
    t_gm, t_halo, total = model.worked_example_time(g["d_cells"], g["d_cache_cells"],
                                                    int(g["n_steps"]), g["halo_cells"],
                                                    int(g["elem_bytes"]), bw)
    assert t_gm * 1e6 == pytest.approx(g["t_gm_us"], abs=0.01)
    assert t_halo * 1e6 == pytest.approx(g["t_halo_us"], abs=0.01)
    peak = model.projected_peak_cells_per_s(g["d_cells"], int(g["n_steps"]), total)
    assert peak / 1e9 == pytest.approx(g["peak_gcells"], abs=0.01)


def test_cached_fraction_limits():
    # nothing cached: every step reads and writes the whole domain
    assert model.global_cells_accessed(100, 0, 7) == 2 * 7 * 100
    # everything cached: one load and one store
    assert model.global_cells_accessed(100, 100, 7) == 200
    assert model.sm_cells_accessed(50, 1) == 0
    assert model.t_perks(3.0, 5.0) == 5.0


def test_littles_law_efficiency():
    c_hw = model.hardware_concurrency(throughput_per_cycle=64, latency_cycles=500)
    assert c_hw == 32000
    assert model.efficiency(model.sm_software_concurrency(20000, 2), c_hw) == 1.0
    assert model.efficiency(16000, c_hw) == 0.5
