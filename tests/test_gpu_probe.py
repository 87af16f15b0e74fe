"""The integer multiply-add pipe probe used for the blind rotation's roofline:
it runs on every SM and reports plausible lane rates (a 16-lane pipe per
scheduler: up to 64 lane operations per clock per SM for 32-bit multiply-adds;
the high-half and 64-bit forms at most that)."""
import pytest

from gpu_common import ce, ctx, keys  # noqa: F401

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible(ce, ctx):
    c, _ = ctx
    r = ce.ce_probe_int_pipes(c)
    assert 16 <= r["imad"] <= 130, r
    assert 8 <= r["imad_hi"] <= r["imad"] * 1.05, r
    assert 8 <= r["imad_wide"] <= r["imad"] * 1.05, r
