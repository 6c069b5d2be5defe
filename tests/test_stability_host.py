"""Host logic of the Sec. 6 stability sweeps: the threshold rule and the
speed-of-sound reading of the lid-speed study (no GPU)."""
import pytest

from paper_2103_02119_gb300 import stability as S


def test_largest_stable_stops_at_the_first_failure():
    assert S.largest_stable([(0.02, True), (0.04, True), (0.06, False), (0.08, True)]) == 0.04
    assert S.largest_stable([(0.08, True), (0.02, True), (0.04, True)]) == 0.08  # order-free
    assert S.largest_stable([(0.02, False), (0.04, True)]) == 0.0
    assert S.largest_stable([]) == 0.0


@pytest.mark.parametrize("a,factor,expected", [(1.0, 0.3, 0.3), (1.0, 0.6, 1.0 / 3.0),
                                               (0.5, 0.3, 0.075), (0.3, 0.15, 0.0135)])
def test_fig17_speed_of_sound(a, factor, expected):
    cs2 = S.fig17_cs2(a, factor)
    assert cs2 == pytest.approx(expected)
    assert cs2 < a * a  # rest weights stay positive


def test_default_reading():
    assert S.fig17_cs2(0.5) == pytest.approx(0.3 * 0.25)
