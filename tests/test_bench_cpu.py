"""Host logic of the benchmark (no GPU): the algorithmic bytes per lattice update
that the roofline divides by, the clock-record parser, and the concurrent
critical-pressure sweep's ordering and worker cap (device calls faked)."""
import threading
import time

import pytest

import bench


def test_bytes_per_lattice_update():
    # fused pass, moments pass.  D3Q19 FP32 populations: read and write f and g
    # (4 x 76 B) and read C1; moments pass reads g and writes C.
    assert bench.lu_bytes("D3Q19", "f32", False) == (308, 80)
    # g held as g_eq: f in and out (152 B), C1, A and u (4 + 4 + 12 B); the
    # moments pass reads A, u and the previous C and writes C (24 B)
    assert bench.lu_bytes("D3Q19", "f32", True) == (172, 24)
    assert bench.lu_bytes("D2Q9", "f32", True) == (88, 20)
    assert bench.lu_bytes("D2Q9", "f32", False) == (148, 40)
    # 16-bit populations with g_0 in FP32: 76 B of f each way, g 2 x (36 + 4) B, C1
    assert bench.lu_bytes("D3Q19", "bf16", False) == (160, 44)
    assert bench.lu_bytes("D3Q19", "f16", False) == bench.lu_bytes("D3Q19", "bf16", False)
    assert bench.lu_bytes("D2Q9", "f64", False) == (296, 80)


HDR = ("index, clocks.current.sm [MHz], clocks.max.sm [MHz], power.draw [W], "
       "clocks_event_reasons.active, clocks_event_reasons.hw_slowdown, "
       "clocks_event_reasons.hw_thermal_slowdown, clocks_event_reasons.sw_thermal_slowdown, "
       "clocks_event_reasons.sw_power_cap\n")


def _row(sm, cap="Not Active", thermal="Not Active"):
    return f"0, {sm} MHz, 2070 MHz, 900.00 W, 0x0, Not Active, {thermal}, Not Active, {cap}\n"


def test_clock_parser_median_and_reasons():
    lines = [HDR, _row(2070), _row(1980, cap="Active"), _row(2055), "garbage\n", "\n"]
    s = bench.parse_clocks(lines)
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.parse_clocks([HDR, _row(1500, thermal="Active")])
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500


def test_clock_parser_without_samples():
    assert bench.parse_clocks([HDR])["reasons"] == ["unsampled"]
    assert bench.parse_clocks([])["sm_mhz"] is None


def test_critical_sweep_order_and_worker_cap(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2504_19941_gb300 import critical as C
    active, peak, lock = [0], [0], threading.Lock()

    def fake(case, tol, dev, rms_tol, max_iter, stream):
        with lock:
            active[0] += 1
            peak[0] = max(peak[0], active[0])
        time.sleep(0.02 * (5 - case))   # later cases finish first
        with lock:
            active[0] -= 1
        return {"dP_c": case * 0.5, "stream": stream}

    monkeypatch.setattr(C, "critical_pressure", fake)
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: object())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    res, wall = C.critical_sweep(range(5), workers=2, device="cpu")
    assert [r["dP_c"] for r in res] == [0.0, 0.5, 1.0, 1.5, 2.0]
    assert len({id(r["stream"]) for r in res}) == 5      # one stream per case
    assert peak[0] == 2 and wall > 0
    res, _ = C.critical_sweep(range(4), device="cpu")
    assert peak[0] == 4                                   # default: all at once
    assert C.critical_sweep([], device="cpu") == ([], 0.0)


def test_meniscus_between_plates_recovers_height_and_angle():
    """A circular meniscus between two plates (gap 2w along y, rise along +x)
    with the liquid below it: the finder returns its height on the centre line
    and the angle it makes with the plates (cos theta = w / R)."""
    import math
    import numpy as np
    import synthetic as S
    nx, ny, nz = 160, 64, 4
    w, yc, theta = 14.0, 32, 45.0
    shape = (nx, ny, nz)
    # plates: y < yc - w and y >= yc + w (C1 = 1/2 planes at yc - w - 0.5, yc + w - 0.5)
    sd = S.union_sd(S.slab_sd(shape, 1, 0, int(yc - w)), S.slab_sd(shape, 1, int(yc + w), ny))
    c1 = (0.5 * (1 + np.tanh(sd / (2 * S.width_to_alpha(3.0))))).reshape(nz, ny, nx)
    w_eff = w                                  # between the C1 = 1/2 planes
    R = w_eff / math.cos(math.radians(theta))
    h0 = 90.0
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    yc_eff = yc - 0.5
    xc = h0 + R                                # centre above the meniscus (concave)
    r = np.sqrt((X - xc) ** 2 + (Y - yc_eff) ** 2)
    c2 = 0.5 * (1 + np.tanh((r - R) / 2.0))    # liquid outside the circle, below it
    c2[X > xc] = 0.0
    c2 = np.broadcast_to(c2, (nz, ny, nx)).copy()
    h, th = bench.meniscus_between_plates(c2, c1, yc, int(w), 20)
    # the centre line at y = yc is half a node off the circle's axis
    assert abs(h - (xc - math.sqrt(R * R - 0.25))) < 0.02, h
    assert abs(th - theta) < 1.0, th
