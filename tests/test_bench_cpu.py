"""Host-side accounting of bench.py: algorithmic bytes, the traffic figure's source guard, the peak, the
clock record and the whole-job throughput. No GPU needed."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ST = {"vertices_light": 3, "vertices_heavy": 2, "arcs_light": 10, "arcs_heavy": 7, "far_scanned": 4}


def test_algorithmic_bytes_per_unit_figures():
    # 28 B per list entry, 16 B per relaxed arc, 20 B per re-binned overflow entry, 36 B per vertex
    assert bench.algorithmic_bytes(ST, 5) == 28 * 5 + 16 * 17 + 20 * 4 + 36 * 5
    assert bench.light_bytes(ST) == 28 * 3 + 16 * 10
    other = dict(ST, arcs_heavy=0, far_scanned=0)
    assert bench.batch_algorithmic_bytes([ST, other], [5, 7]) == \
        bench.algorithmic_bytes(ST, 5) + bench.algorithmic_bytes(other, 7)


def _source_hash():
    h = hashlib.sha256()
    for f in ("solve.cu", "dsssp_internal.cuh", "warp_util.cuh"):
        with open(os.path.join(ROOT, "paper_1911_06895_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_traffic_only_for_the_source_it_was_measured_on(monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_SOURCE_SHA256", _source_hash())
    assert bench.measured_traffic(22) == bench.TRAFFIC_BYTES_PER_LAUNCH
    assert bench.measured_traffic(20) is None                 # another workload
    monkeypatch.setattr(bench, "TRAFFIC_SOURCE_SHA256", "0" * 64)
    assert bench.measured_traffic(22) is None                 # the kernel changed since the capture


def test_peak_from_measured_file():
    peak, kind = bench.measured_peak_gbs()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000.0
    else:
        assert (peak, kind) == (6800.0, "fallback")


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_and_reasons():
    c = bench.ClockSampler(0)
    c.proc = _DoneProc()
    c.lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2010, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c2 = bench.ClockSampler(0)
    assert c2.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_job_gteps_counts_every_rank():
    # 1e6 arcs x 256 solves on each of 2 ranks in 0.5 s of the slowest rank
    assert abs(bench.job_gteps(1_000_000, 256, 2, 0.5) - 1.024) < 1e-12
