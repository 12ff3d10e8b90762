"""Host-side helpers of bench.py: figures read from an ncu summary only while the kernel
source hash recorded beside them matches, the clock record taken during the timed region
(median SM clock, throttle reasons), and the replay of a request stream against a server
(latency, per-size buckets, rates; a fake server here). CPU only."""
import os

import pytest

import bench


def _profile(tmp_path, text):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text(text)


def test_profiled_figure_is_gated_by_the_source_hash(tmp_path, monkeypatch):
    _profile(tmp_path, "# k\n\n- dram_bytes_per_launch: `1234` (a note)\n- issue_active_frac: `0.5`\n"
                       "- kernel_source_hash: `abc`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.profiled_traffic("k") == 1234.0
    assert bench.profiled_figure("k", "issue_active_frac") == 0.5
    assert bench.profiled_figure("k", "missing") is None
    assert bench.profiled_figure("absent", "issue_active_frac") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.profiled_traffic("k") is None          # counters of an older kernel are not used


def test_committed_profile_names_its_figures():
    """The headline kernel's summary carries the figures the benchmark reads."""
    text = open(os.path.join(bench.ROOT, "profiles", "k_trace16_surface1M_1080p.md")).read()
    for key in ("dram_bytes_per_launch", "issue_active_frac", "kernel_source_hash"):
        assert f"- {key}: `" in text
    assert len(bench.kernel_source_hash()) == 16


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, rows, gpu=0):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(r + "\n" for r in rows))
    s = bench.ClockSampler(gpu)
    s.proc, s.path = _Done(), str(path)
    return s


def test_clock_record_median_and_reasons(tmp_path):
    rows = ["0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1400, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active",
            "1, 900, 2070, 100, 0x8, Active, Not Active, Not Active, Not Active",   # another GPU
            "garbled line"]
    rec = _sampler(tmp_path, rows).stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


@pytest.mark.parametrize("reason_col,name", [(5, "hw_slowdown"), (6, "hw_thermal_slowdown"),
                                             (7, "sw_thermal_slowdown")])
def test_clock_record_reports_each_slowdown(tmp_path, reason_col, name):
    p = ["0", "1500", "2070", "1000", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    p[reason_col] = "Active"
    rec = _sampler(tmp_path, [", ".join(p)]).stop()
    assert rec["reasons"] == [name] and rec["sm_mhz"] == 1500.0


def test_clock_record_without_samples(tmp_path):
    assert _sampler(tmp_path, []).stop()["reasons"] == ["no samples"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


class _FakeServer:
    """Completes every request a fixed service time after its submission (CLOCK_MONOTONIC)."""

    def __init__(self, service_s):
        import time
        self.time = time
        self.service = service_s
        self.inflight = []

    def submit(self, batch):
        t = self.time.monotonic()
        for sid, cam, buf, tag in batch:
            assert buf.numel() >= cam["width"] * cam["height"] * 4
            self.inflight.append((t + self.service, tag))

    def poll(self, wait=False):
        now = self.time.monotonic()
        done = [dict(tag=tag, status=0, t_admit=t - self.service, t_done=t) for t, tag in self.inflight if t <= now]
        self.inflight = [(t, tag) for t, tag in self.inflight if t > now]
        return done


def test_request_stream_replay_latency_and_buckets():
    """The serving benchmark's replay: every request completes once, latency is completion -
    arrival (here the fake server's 3 ms service plus polling granularity), per-size buckets
    cover the sizes in the stream, and the rate is rays over the makespan."""
    import numpy as np
    reqs = []
    sizes = [(64, 64), (128, 96)]
    for j in range(60):
        w, h = sizes[j % 2]
        reqs.append(dict(scene=0, camera=dict(width=w, height=h), arrival=0.001 * j))
    res = bench.run_stream(_FakeServer(0.003), reqs, 1000.0, device="cpu")
    assert res["requests"] == 60
    assert 3.0 <= res["p50_ms"] <= 6.0 and res["p99_ms"] < 20.0
    assert sorted(res["latency_by_pixels"]) == sorted(str(w * h) for w, h in sizes)
    assert all(v["n"] == 30 for v in res["latency_by_pixels"].values())
    rays = sum(r["camera"]["width"] * r["camera"]["height"] for r in reqs)
    assert abs(res["Mrays_per_s"] - rays / res["makespan_s"] / 1e6) < 1e-9
    assert 0.059 <= res["makespan_s"] < 0.2
    assert np.isclose(res["offered_Mrays_per_s"], rays / 0.059 / 1e6)
