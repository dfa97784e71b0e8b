"""The benchmark's clock record keeps only the nvidia-smi samples taken inside
the timed region (each sample is stamped with the host clock when it is
read), falls back to the samples on either side when the region is shorter
than the sampling interval, and reports the throttle reasons of the kept
samples only. Host logic; no GPU and no nvidia-smi are needed."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _Joined:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    b = _bench()
    c = b.ClockSampler(0)
    c.proc, c.t, c.lines = _Done(), _Joined(), list(lines)
    return c


def _line(mhz, reasons=("Not Active",) * 4):
    return "%d, 2070, 900.0, 0x0, %s" % (mhz, ", ".join(reasons))


def test_only_samples_inside_the_window_are_kept():
    lines = [(0.0, _line(1200)), (1.0, _line(2070)), (1.5, _line(2060)), (2.0, _line(2070)),
             (3.0, _line(900, ("Not Active", "Active", "Not Active", "Not Active")))]
    c = _sampler(lines)
    c.window(0.9, 2.1)
    r = c.stop()
    assert r["samples_in_timed_region"] == 3 and r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == []          # the hw_thermal_slowdown sample lies after the window


def test_short_window_takes_its_neighbours():
    lines = [(0.0, _line(2000)), (1.0, _line(2070)), (2.0, _line(2050))]
    c = _sampler(lines)
    c.window(1.2, 1.3)
    r = c.stop()
    assert r["samples_in_timed_region"] == 0 and r["samples"] == 2
    assert r["sm_mhz"] == 2060.0


def test_reasons_inside_the_window_are_reported():
    lines = [(1.0, _line(1500, ("Not Active", "Not Active", "Not Active", "Active"))), (1.1, _line(1500))]
    c = _sampler(lines)
    c.window(0.5, 1.5)
    r = c.stop()
    assert r["reasons"] == ["sw_power_cap"]
