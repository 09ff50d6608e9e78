"""The FP64 oracle against facts fixed by the paper and by mathematics (CPU)."""
import pytest

import pins
from oracle import oracle as OR


@pytest.fixture(scope="module")
def O():
    return OR.default()


@pytest.mark.parametrize("pin", pins.FAST_PINS, ids=lambda p: p.__name__)
def test_pin(O, pin):
    pin(O)


def test_recover_roundtrip_bag(O):
    pins.pin_recover_roundtrip(O, eos=OR.EOS_BAG)


def test_riemann_values_consistent():
    """The exact solver itself: its star state satisfies the momentum jump
    condition across the shock and the Riemann invariant across the fan."""
    import math
    import riemann_exact as RE
    s = RE.solve()
    e, v, vs = s["e_star"], s["v_star"], s["v_shock"]
    g2 = 1.0 / (1.0 - v * v)
    p, pr = e / 3.0, s["e_r"] / 3.0
    M2 = (e + p) * g2 * v
    # v_s [M] = [M v + p] with the right state at rest
    assert abs(vs * M2 - (M2 * v + p - pr)) < 1e-12
    # Riemann invariant atanh v + sqrt(3)/4 ln e is constant across the fan
    assert abs(math.atanh(v) + math.sqrt(3) / 4 * math.log(e) - math.sqrt(3) / 4 * math.log(1.0)) < 1e-12
    # subluminal ordering of the waves
    assert -1 < s["xi_head"] < s["xi_tail"] < s["v_star"] < s["v_shock"] < 1
