"""Host logic of the critical-pressure search (bisection and bracket widening),
driven by a fake collapse test on the CPU."""
import math

import pytest

torch = pytest.importorskip("torch")


def _bisect():
    # the module imports the package (which loads libdsm); the bisection itself
    # is host code
    import paper_2504_19941_gb300.critical as C
    return C.bisect_critical, C.critical_theory


@pytest.mark.parametrize("true,lo,hi", [(0.0123, 0.0, 0.05), (-0.02, -0.05, 0.0),
                                        (0.09, 0.0, 0.01), (-0.3, -0.01, 0.02)])
def test_bisection_finds_the_switch(true, lo, hi):
    bisect, _ = _bisect()
    calls = []

    def collapsed(dp):
        calls.append(dp)
        return dp > true
    dpc, a, b = bisect(collapsed, lo, hi, tol=1e-4)
    assert a <= true <= b and b - a <= 1e-4 and abs(dpc - true) <= 5e-5
    assert len(calls) < 40


def test_bisection_gives_up_without_a_switch():
    bisect, _ = _bisect()
    with pytest.raises(RuntimeError):
        bisect(lambda dp: False, 0.0, 1.0, max_widen=4)
    with pytest.raises(RuntimeError):
        bisect(lambda dp: True, 0.0, 1.0, max_widen=4)


def test_closed_form():
    _, theory = _bisect()
    assert theory(1.0, 90.0, 10.0) == pytest.approx(0.0, abs=1e-15)
    assert theory(0.5, 120.0, 20.0) == pytest.approx(-2 * 0.5 * math.cos(math.radians(120)) / 20)
