"""The U-Net kernels (BF16 tensor cores, FP32 accumulation) against the network
oracle, which rounds its stored tensors to BF16 at the same points and sums in
FP64: forward outputs, the loss, and every layer's weight and bias gradient,
on grids whose levels span several tiles and a ragged last tile."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet as U  # noqa: E402
from paper_2206_07732_gb300 import build as B  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402
from paper_2206_07732_gb300 import wec  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    wec.load()


def _case(seed, n, h, w):
    rng = np.random.default_rng(seed)
    shapes = U.param_shapes(32)
    flat = synth.unet_weights(shapes, seed)
    k = 0
    for s in shapes:  # nonzero biases (ReLU kinks away from exact zeros)
        m = int(np.prod(s))
        if len(s) == 1:
            flat[k:k + m] = 0.05 * rng.standard_normal(m)
        k += m
    x = rng.standard_normal((n, h, w, 2)).astype(np.float32)
    t = rng.standard_normal((n, h, w)).astype(np.float32)
    return flat.astype(np.float32), x, t


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _dyadic_case(seed, n, h, w):
    # weights with one nonzero (+-1) per output channel and half-integer biases,
    # inputs and targets: every activation, gradient and weight-gradient sum is a
    # short sum of dyadic numbers, exact in BF16 and FP32, so both sides compute
    # the same numbers exactly (no rounding happens anywhere)
    return synth.unet_dyadic_case(U.param_shapes(32), seed, n, h, w)


@pytest.mark.parametrize("n,h,w", [(2, 32, 32), (1, 16, 64), (4, 8, 32)])
def test_exact_arithmetic_case_is_bit_exact(n, h, w):
    # every gather (3x3 with zero border, stride 2, nearest upsampling, skip
    # concatenation), the weight packing, the epilogues, the head, the input and
    # weight gradients and Adam's inputs: equal bit for bit (pixel counts are
    # powers of two, so 1/M is exact too)
    flat, x, t = _dyadic_case(7, n, h, w)
    net = wec.Net(h, w, max_batch=n)
    net.set_params(flat)
    out = torch.zeros((n, h, w), dtype=torch.float32, device="cuda")
    net.forward(_cuda(x), out)
    ref, A = U.forward(flat.astype(np.float64), x.astype(np.float64), 32, emulate_bf16=True)
    for li, (name, _, _, _) in enumerate(U.layers(32)[:-1]):
        assert np.array_equal(net.activation(li, n, A[name].shape).astype(np.float64), A[name]), name
    assert np.array_equal(out.cpu().numpy().astype(np.float64), ref)
    loss = net.loss_grad(_cuda(x), _cuda(t))
    lref, gref = U.loss_and_grads(flat.astype(np.float64), x.astype(np.float64), t.astype(np.float64), 32,
                                  emulate_bf16=True)
    assert loss == lref
    g = net.grads().astype(np.float64)
    k = 0
    for li, s in enumerate(U.param_shapes(32)):
        m = int(np.prod(s))
        assert np.array_equal(g[k:k + m], gref[k:k + m]), (U.layers(32)[li // 2][0], s)
        k += m
    net.close()


@pytest.mark.parametrize("n,h,w", [(2, 32, 32), (1, 16, 48), (3, 24, 40)])
def test_random_network_within_bf16_tolerance(n, h, w):
    # He-initialised weights: the two sides round the same stored tensors to
    # BF16, but FP32 (tensor-core) and FP64 sums differ in the last bits, so a
    # few values round to the neighbouring BF16 number (1 unit = 2^-8 relative);
    # those differences spread with depth.  Measured at the output: ~6e-3
    # relative (1.5 BF16 units); bound 1e-2.  Layer 0 sums 18 products plus the
    # bias: at most a rare single flip.
    flat, x, _ = _case(1, n, h, w)
    net = wec.Net(h, w, max_batch=n)
    net.set_params(flat)
    out = torch.zeros((n, h, w), dtype=torch.float32, device="cuda")
    net.forward(_cuda(x), out)
    ref, A = U.forward(flat.astype(np.float64), x.astype(np.float64), 32, emulate_bf16=True)
    a0 = net.activation(0, n, A["enc0a"].shape).astype(np.float64)
    assert np.linalg.norm(a0 - A["enc0a"]) <= 1e-3 * np.linalg.norm(A["enc0a"])
    g = out.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    print(f"forward {n}x{h}x{w}: relative error {err:.2e}")
    assert err < 1e-2
    net.close()


@pytest.mark.parametrize("n,h,w", [(2, 32, 32), (1, 16, 48)])
def test_random_network_gradients_within_bf16_tolerance(n, h, w):
    # With a random target the weight gradients are small residues of large,
    # cancelling sums over pixels, and the problem itself is that sensitive:
    # in the oracle, single-unit BF16 flips of 1 in 10^4 stored values move the
    # gradients by 7 % (global) and 13 % (median tensor).  The bounds are that
    # sensitivity: global relative error 0.15, cosine 0.98, loss 2e-3.  (The
    # exact-arithmetic case above is the equality check of the same kernels.)
    flat, x, t = _case(2, n, h, w)
    net = wec.Net(h, w, max_batch=n)
    net.set_params(flat)
    loss = net.loss_grad(_cuda(x), _cuda(t))
    g = net.grads().astype(np.float64)
    lref, gref = U.loss_and_grads(flat.astype(np.float64), x.astype(np.float64), t.astype(np.float64), 32,
                                  emulate_bf16=True)
    assert loss == pytest.approx(lref, rel=2e-3)
    k, errs = 0, []
    for li, s in enumerate(U.param_shapes(32)):
        m = int(np.prod(s))
        errs.append(np.linalg.norm(g[k:k + m] - gref[k:k + m]) / max(np.linalg.norm(gref[k:k + m]), 1e-30))
        k += m
    glob = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    print(f"gradients {n}x{h}x{w}: global relative error {glob:.2e}, cosine {cos:.4f}, "
          f"per-tensor median {np.median(errs):.2e}, max {max(errs):.2e}")
    assert glob < 0.15
    assert cos > 0.98
    net.close()


def test_results_are_reproducible_bit_for_bit():
    flat, x, t = _case(3, 2, 32, 32)
    out = []
    for _ in range(2):
        net = wec.Net(32, 32, max_batch=2)
        net.set_params(flat)
        net.loss_grad(_cuda(x), _cuda(t))
        out.append(net.grads())
        net.close()
    assert np.array_equal(out[0], out[1])


def test_adam_matches_its_definition():
    # one Adam step from zero moments: theta - lr * g / (|g| + eps) (bias-corrected)
    flat, x, t = _case(4, 1, 16, 16)
    net = wec.Net(16, 16, max_batch=1)
    net.set_params(flat)
    net.loss_grad(_cuda(x), _cuda(t))
    g = net.grads().astype(np.float64)
    net.adam(1e-3)
    th = net.params().astype(np.float64)
    ref = flat.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(th - ref)) < 1e-6
    net.close()


def test_training_lowers_the_loss():
    flat, x, t = _case(5, 2, 32, 32)
    t = (0.5 * x[..., 0] - 0.25 * x[..., 1]).astype(np.float32)  # a learnable map
    net = wec.Net(32, 32, max_batch=2)
    net.set_params(flat)
    xs, ts = _cuda(x), _cuda(t)
    l0 = net.train_step(xs, ts, [0, 1], 1e-3)
    for _ in range(60):
        l1 = net.train_step(xs, ts, [0, 1], 1e-3)
    assert l1 < 0.3 * l0
    net.close()
