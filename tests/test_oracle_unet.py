"""Pins of the network oracle (the learned warm start's U-Net) against things
that do not depend on it: brute-force loops for each layer, a library's BF16
conversion, finite differences of the FP64 loss, and the closed form of a
network with zero weights."""
import numpy as np
import pytest

from oracle import unet as U
from paper_2206_07732_gb300 import synth

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_library():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000).astype(np.float32) * np.exp(rng.uniform(-20, 20, 20000)).astype(np.float32)
    # exact ties: 8 significant bits plus a half unit in the last place
    ties = (np.arange(256, 512, dtype=np.float32) + 0.5) * np.float32(2.0 ** -8)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, 1.0, -3.0])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x.astype(np.float64)), ref)


def test_conv3_down2_up_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 4, 3))
    W = rng.standard_normal((3, 3, 3, 5))
    b = rng.standard_normal(5)
    y = U.conv3(x, W, b)
    for n in range(2):
        for i in range(6):
            for j in range(4):
                for o in range(5):
                    s = b[o]
                    for a in range(3):
                        for c in range(3):
                            ii, jj = i + a - 1, j + c - 1
                            if 0 <= ii < 6 and 0 <= jj < 4:
                                s += sum(x[n, ii, jj, k] * W[a, c, k, o] for k in range(3))
                    assert y[n, i, j, o] == pytest.approx(s, abs=1e-12)
    Wd = rng.standard_normal((2, 2, 3, 4))
    yd = U.down2(x, Wd, b[:4])
    for n in range(2):
        for i in range(3):
            for j in range(2):
                for o in range(4):
                    s = b[o] + sum(x[n, 2 * i + a, 2 * j + c, k] * Wd[a, c, k, o]
                                   for a in range(2) for c in range(2) for k in range(3))
                    assert yd[n, i, j, o] == pytest.approx(s, abs=1e-12)
    u = U.up(x)
    assert u.shape == (2, 12, 8, 3)
    assert all(u[n, i, j, k] == x[n, i // 2, j // 2, k]
               for n in range(2) for i in range(12) for j in range(8) for k in range(3))


def _small(seed, base=2, n=2, h=16, w=16):
    rng = np.random.default_rng(seed)
    flat = synth.unet_weights(U.param_shapes(base), seed).astype(np.float64)
    # nonzero biases: with zero ones, a dead region upstream leaves
    # pre-activations at exactly 0, the kink of ReLU, where central differences
    # see half a slope
    k = 0
    for s in U.param_shapes(base):
        n_ = int(np.prod(s))
        if len(s) == 1:
            flat[k:k + n_] = 0.1 * rng.standard_normal(n_)
        k += n_
    x = rng.standard_normal((n, h, w, 2))
    t = rng.standard_normal((n, h, w))
    return flat, x, t


def test_gradient_matches_finite_differences():
    # FP64 network: the analytic gradient's directional derivative along a
    # random direction, per layer, against central differences of the loss
    base = 2
    flat, x, t = _small(2, base)
    f = lambda p: U.loss_and_grads(p, x, t, base, emulate_bf16=False)[0]
    _, g = U.loss_and_grads(flat, x, t, base, emulate_bf16=False)
    rng = np.random.default_rng(3)
    k = 0
    for s in U.param_shapes(base):
        n = int(np.prod(s))
        d = np.zeros_like(flat)
        d[k:k + n] = rng.standard_normal(n)
        eps = 1e-6
        fd = (f(flat + eps * d) - f(flat - eps * d)) / (2 * eps)
        an = float(g @ d)
        assert fd == pytest.approx(an, rel=2e-5, abs=1e-10), (s, fd, an)
        k += n


def test_zero_weights_give_the_head_bias():
    # all weights and biases zero except the head bias: every ReLU output is 0,
    # the output is the head bias, and only the head bias gets a gradient
    base = 2
    shapes = U.param_shapes(base)
    flat = np.zeros(sum(int(np.prod(s)) for s in shapes))
    flat[-1] = 0.7
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 8, 8, 2))
    t = rng.standard_normal((1, 8, 8))
    out, _ = U.forward(flat, x, base, emulate_bf16=False)
    assert np.all(out == 0.7)
    loss, g = U.loss_and_grads(flat, x, t, base, emulate_bf16=False)
    assert loss == pytest.approx(np.mean((0.7 - t) ** 2), rel=1e-14)
    assert g[-1] == pytest.approx(2.0 * np.mean(0.7 - t), rel=1e-14)
    assert np.all(g[:-1] == 0.0)


def test_bf16_emulation_stays_near_fp64():
    # rounding the stored tensors to BF16 perturbs the loss and gradient by
    # about the BF16 unit (2^-8) times the depth, not more
    base = 4
    flat, x, t = _small(5, base, h=16, w=32)
    l64, g64 = U.loss_and_grads(flat, x, t, base, emulate_bf16=False)
    l16, g16 = U.loss_and_grads(flat, x, t, base, emulate_bf16=True)
    assert l16 == pytest.approx(l64, rel=0.05)
    assert np.linalg.norm(g16 - g64) <= 0.1 * np.linalg.norm(g64)
