"""The float <-> double conversions the FP32 and double-float stencils use
(integer operations, IEEE 754 round to nearest even) against this GPU's
conversion instructions, bit for bit: random values over the whole exponent
range, exact ties between neighbouring floats with even and odd significands,
the boundaries of the normal float range, zeros, subnormals, infinities, NaN."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return wec.load()


def _values():
    rng = np.random.default_rng(7)
    v = [rng.standard_normal(200000) * 10.0 ** rng.uniform(-50, 50, 200000)]
    # random bit patterns (every exponent, both signs)
    bits = rng.integers(0, 2**63, 200000, dtype=np.int64) * rng.choice([1, -1], 200000)
    v.append(bits.view(np.float64))
    # exact ties: a float plus half its ulp, and just either side of it
    f = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-30, 30, 100000)).astype(np.float32)
    f64 = f.astype(np.float64)
    up = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    tie = 0.5 * (f64 + up)
    v += [tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf), f64]
    fl = np.finfo(np.float32)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, float(fl.max), -float(fl.max), float(fl.tiny),
                      -float(fl.tiny), float(fl.tiny) / 2, float(fl.smallest_subnormal), 1e-45, 1e-46, 1e-300,
                      3.4028235677973366e38, 3.4028235677973362e38, 3.5e38, 1e39, 1.0, -1.0, 2.0 ** -126,
                      2.0 ** -126 * (1 - 2.0 ** -25), 2.0 ** 128 * (1 - 2.0 ** -25), 5e-324])
    v.append(edges)
    return np.concatenate(v)


def test_integer_conversions_equal_the_instructions(lib):
    vals = _values()
    t = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    assert wec.check_conversions(t) == 0


def test_small_and_empty_inputs(lib):
    t = torch.tensor([1.0, 0.1, -3.5e-20], dtype=torch.float64, device="cuda")
    assert wec.check_conversions(t) == 0
    assert wec.check_conversions(t[:0]) == 0
