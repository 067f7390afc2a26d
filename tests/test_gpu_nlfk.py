"""GPU static-grid NLFK force (wec_nlfk_*) against the oracle, element for
element: same region, waves, body positions and times, both pressure modes."""
import math

import numpy as np
import pytest

from paper_2206_07732_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wec():
    from paper_2206_07732_gb300 import build, wec as W
    build.build()
    W.load()
    return W


@pytest.mark.parametrize("mode", [0, 1])
def test_nlfk_matches_oracle(wec, mode):
    from oracle import tank as O
    from oracle import waves as OW
    depth = 2.5
    # the large tank's sea state and the oracle's own wave numbers (the library
    # solves the dispersion relation itself from omega)
    ph = np.random.default_rng(4).uniform(0.0, 2.0 * math.pi, 64)
    amp, om, _ = OW.jonswap_components(0.15, 1.6, 3.3, 64, ph)
    kw = np.array([OW.dispersion_k(o, depth, 9.81) for o in om])
    region = (4.0, 1.5, 1.0 / 64.0, 192, 128)  # 3 m x 2 m around the body, large-tank spacing
    body = dict(xc=5.5, width=1.0, height=0.8)
    N = wec.Nlfk(region, depth, amp, om, ph, body)
    for t, yc in ((0.0, 2.5), (0.37, 2.47), (1.9, 2.56), (3.3, 2.5)):
        fx, fy = N.force(t, yc, mode)
        ox, oy = O.nlfk(region, depth, 1025.0, 9.81, amp, om, kw, ph, (5.5, 1.0, 0.8), t, yc, mode)
        scale = 1025.0 * 9.81 * 1.0 * 0.8
        assert abs(fy - oy) <= 1e-11 * scale
        assert abs(fx - ox) <= 1e-11 * scale
        again = N.force(t, yc, mode)
        assert again == (fx, fy)  # reproducible bit for bit
    N.close()
