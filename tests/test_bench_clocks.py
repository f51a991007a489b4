"""The benchmark's clock record on CPU: nvidia-smi is replaced by a fake that
prints the query's CSV rows; the record must carry the median SM clock under
load, the largest maximum clock, and every throttle reason seen active."""
import io
import subprocess

import bench


class _FakeProc:
    def __init__(self, text):
        self.stdout = io.StringIO(text)
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sample(monkeypatch, text):
    procs = []

    def popen(cmd, **kw):
        assert cmd[0] == "nvidia-smi" and "--format=csv,noheader,nounits" in cmd
        assert any(a.startswith("--query-gpu=clocks.sm,clocks.max.sm") for a in cmd)
        procs.append(_FakeProc(text))
        return procs[-1]

    monkeypatch.setattr(subprocess, "Popen", popen)
    c = bench.ClockSampler(0)
    c.start()
    c.thread.join(timeout=5)
    rec = c.stop()
    assert procs[0].terminated
    return rec


def test_steady_clocks_have_no_reasons(monkeypatch):
    rows = "".join(f"{mhz}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   for mhz in (2070, 2055, 2070, 2040, 2070))
    rec = _sample(monkeypatch, rows)
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_active_reasons_are_reported(monkeypatch):
    rows = ("1800, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "1500, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active\n"
            "1900, 2070, 1000.0, 0x0, Not Active, Not Active, Active, Not Active\n"
            "garbage line\n")
    rec = _sample(monkeypatch, rows)
    assert rec["sm_mhz"] == 1800.0 and rec["samples"] == 3
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_missing_nvidia_smi_is_reported_as_unsampled(monkeypatch):
    def popen(cmd, **kw):
        raise FileNotFoundError("nvidia-smi")

    monkeypatch.setattr(subprocess, "Popen", popen)
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
