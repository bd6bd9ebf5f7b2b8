"""Pins of the oracle's ramp filters (no GPU): each spatial kernel applied to
a long sampled cosine reproduces its closed-form frequency response away
from the row ends (Ram-Lak |w|/2pi, Shepp-Logan |sin(w/2)|/pi, Hann
|w|/2pi (1 + cos w)/2), and all three have zero response to a constant."""
import math

import numpy as np
import pytest

RESPONSE = {
    "ramlak": lambda w: abs(w) / (2 * math.pi),
    "shepp-logan": lambda w: abs(math.sin(w / 2)) / math.pi,
    "hann": lambda w: abs(w) / (2 * math.pi) * (1 + math.cos(w)) / 2,
}


@pytest.mark.parametrize("kind", list(RESPONSE))
@pytest.mark.parametrize("w", [0.05, 0.4, 1.3, 2.6, math.pi])
def test_filter_frequency_response(orc, kind, w):
    n = 4096
    k = np.arange(n)
    p = np.cos(w * k + 0.3)[None]
    q = orc.filter_rows(p, kind)[0]
    mid = slice(n // 4, 3 * n // 4)
    # kernel tails beyond n/4 bins contribute at most ~ 2 / (pi^2 n/4) ~ 2e-4
    np.testing.assert_allclose(q[mid], RESPONSE[kind](w) * p[0, mid], atol=5e-4)


@pytest.mark.parametrize("kind", list(RESPONSE))
def test_filter_kills_constants(orc, kind):
    q = orc.filter_rows(np.ones((1, 4096)), kind)[0]
    assert np.abs(q[1024:3072]).max() < 5e-4


def test_ramlak_kind_is_the_ramlak_filter(orc):
    p = np.random.default_rng(0).standard_normal((3, 77))
    np.testing.assert_array_equal(orc.filter_rows(p, "ramlak"), orc.ramlak_filter(p))
