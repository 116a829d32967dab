"""The benchmark's host-side arithmetic on CPU: the algorithmic path-term count
behind the path-sum roofline, the OS-vs-MLEM iteration matching, the clock
summary, and the traffic figure's gating on the kernel source."""
import os
import sys
import threading
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2002_12471_gb300 import synthetic as S  # noqa: E402


def test_strip_terms_matches_event_by_pixel_enumeration():
    """strip_terms counts, per event, one primary strip over the support plus
    one per scatter pixel m whose collimator response reaches the event
    (|u_j - u_a(m)| <= k sigma_u(m), edges included).  Enumerate every
    (event, scatter pixel) pair instead of sorting and bisecting."""
    ph, g, _, _, _ = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 600, seed=11)
    k = 3.0
    got, n_nz = bench.strip_terms(ph, g, ev, k_sigma=k)
    ny, nx = ph.mu.shape
    iy, ix = np.nonzero(ph.mu > 0)
    assert n_nz == len(ix)
    x = (ix + 0.5 - 0.5 * nx) * ph.pixel_mm
    y = (iy + 0.5 - 0.5 * ny) * ph.pixel_mm
    fw = 2.0 * np.sqrt(2.0 * np.log(2.0))
    want = 0
    for a, u in zip(ev.angle, ev.u_mm.astype(np.float64)):
        th = g["angle0_rad"] + 2 * np.pi * a / g["n_angles"]
        depth = g["radius_mm"] - (x * np.cos(th) + y * np.sin(th))
        sig = (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * depth) / fw
        um = -x * np.sin(th) + y * np.cos(th)
        want += 1 + int(np.sum(np.abs(u - um) <= k * sig))
    assert got == want * n_nz


def test_os_vs_mlem_counts_iterations_to_the_same_likelihood(monkeypatch):
    """With OS curves that fall as 1/(N_s i), MLEM needs exactly N_s times
    the OS iterations; the paper's 4 subsets are always reported."""
    import torch

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, s):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 2.0

    class FakeLib:
        def lmosem_create(self, *a, **kw):
            return {}

        def lmosem_n_support(self, c):
            return 4

        def lmosem_sensitivity(self, c, n):
            c["ns"] = n

        def lmosem_build_model(self, c, *a):
            pass

        def lmosem_init_image(self, c, T, f):
            pass

        def lmosem_iterate(self, c, iters, T, f, ll=None):
            if ll is not None:
                ll.copy_(torch.tensor([-1.0 / (c["ns"] * (i + 1)) for i in range(iters)],
                                      dtype=torch.float64))

        def lmosem_destroy(self, c):
            pass

    monkeypatch.setattr(torch.cuda, "Event", Ev)
    ph = types.SimpleNamespace(mu=None, pixel_mm=1.0)
    res = bench.os_vs_mlem(FakeLib(), ph, {}, None, None, None, 8, 10, None, "cpu")
    assert [r["subsets"] for r in res] == [4, 8]
    assert [r["mlem_iters_to_match"] for r in res] == [40, 80]
    for r in res:
        assert r["os_s_per_iter"] == pytest.approx(2e-3 / 10)
        assert r["mlem_s_per_iter"] == pytest.approx(2e-3 / 80)
        want = r["mlem_iters_to_match"] * r["mlem_s_per_iter"] / (10 * r["os_s_per_iter"])
        assert r["speedup_to_same_loglik"] == pytest.approx(want)
    only4 = bench.os_vs_mlem(FakeLib(), ph, {}, None, None, None, 4, 10, None, "cpu")
    assert [r["subsets"] for r in only4] == [4]


def _sampled(lines, uuid="GPU-a"):
    cs = bench.ClockSampler(uuid)
    cs.lines = list(lines)
    cs.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0)
    cs.thread = threading.Thread(target=lambda: None)
    cs.thread.start()
    return cs.stop()


def test_clock_summary_takes_median_and_active_reasons():
    on = "GPU-a, %d, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, %s"
    lines = [on % (2070, "Not Active"), on % (1980, "Active"), on % (2040, "Not Active"),
             "GPU-b, 300, 2070, 100.0, 0x0, Active, Active, Active, Active",   # another GPU
             "GPU-a, [N/A], 2070, 0, 0x0, , , , ", "garbage"]
    c = _sampled(lines)
    assert c["sm_mhz"] == 2040.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert _sampled(["GPU-b, 300, 2070, 1, 0x0, a, b, c, d"]) is None


def test_traffic_figure_is_gated_on_the_path_sum_source():
    """The committed DRAM-bytes figure is used only while the path-sum
    kernel's source hash matches the one recorded beside it, and only for
    the workload it was taken on."""
    h = bench.kernel_source_sha1()
    assert len(h) == 12
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    rec = [dict(p.split("=", 1) for p in ln.split() if "=" in p) for ln in open(path)]
    mine = [r for r in rec if r.get("kernel") == "k_pathsum"]
    assert mine, "no k_pathsum traffic line"
    for wl in ("dat64_0.2M", "dat128_1M", "dat128_0.06M"):
        t = bench.read_traffic("k_pathsum", wl)
        match = [r for r in mine if r["source_sha1"] == h and r.get("workload", "") == wl]
        if match:
            assert t == float(match[0]["dram_bytes_per_launch"])
        else:
            assert t is None
    # the figure of the 1M-event benchmark is not reported for a smaller run
    assert bench.read_traffic("k_pathsum", "dat128_0.06M") is None
    assert "%s_%gM" % ("dat128", 1000000 / 1e6) == "dat128_1M"
    assert bench.read_traffic("no_such_kernel", "dat64") is None
    assert bench.read_traffic("k_pathsum", "no_such_workload") is None
