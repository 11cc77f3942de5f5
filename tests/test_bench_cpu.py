"""Host logic of bench.py that needs no GPU: the recorded ncu traffic is
reported only while the profiled kernel source is unchanged."""
import copy

import bench


def test_measured_traffic_is_tied_to_the_kernel_source(monkeypatch):
    key = ("si8", "f16x3", "cgemm_tc")
    assert bench.measured_traffic(*key) == bench.MEASURED_TRAFFIC[key]["bytes_per_launch"]
    assert bench.measured_traffic("si64", "f16x3", "green_tc") is None
    changed = copy.deepcopy(bench.MEASURED_TRAFFIC)
    path = next(iter(changed[key]["sources"]))
    changed[key]["sources"][path] = "0" * 40
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", changed)
    assert bench.measured_traffic(*key) is None


def test_flop_model_at_the_bench_size():
    # G formation 2 * 8 N_r^2 N_b per tau, screening 4 N_chi^3 per omega (si8)
    fl = bench.flop_model(13824, 1024, 16, 13824, 8)
    assert abs(fl["green"] - 2 * 8 * 13824 ** 2 * 1024 * 16) < 1
    assert abs(fl["dyson"] - 4 * 13824 ** 3 * 16) < 1
