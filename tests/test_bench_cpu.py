"""Host-side pieces of bench.py that fix the reported workload and roofline inputs: the time
step of the Taylor-Green workload (CFL 0.5 with t = 9 on a step), the ncu traffic lookup keyed
by the kernel sources, and the peak fallback."""
import json
import math

import bench


def test_time_step_lands_on_t9():
    # max|u_x| = max|u_y| = 1, u_z = 0 at t = 0: dt = 0.5 dx / 2, rounded down to 9 / n
    for N, n in ((256, 1467), (384, 2201), (32, 184)):
        dt = bench.dt_for(N)
        assert abs(dt - 9.0 / n) < 1e-15
        assert dt <= 0.5 * (2 * math.pi / N) / 2 + 1e-15
        assert abs(9.0 / dt - round(9.0 / dt)) < 1e-9


def test_traffic_lookup_follows_the_kernel_sources(monkeypatch, tmp_path):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    d = {"kernel_source_hash": h, "kernels": {"slab_pass": {"dram_bytes_per_launch_full_size": 123}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.ncu_traffic("slab_pass") == 123
    assert bench.ncu_traffic("k_pencil") is None  # no entry
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("slab_pass") is None  # counters of other kernel sources


def test_peak_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6771.8}))
    assert bench.peaks() == (6771.8, "measured")
