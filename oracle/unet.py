"""FP64 CPU oracle of the learned warm start's network -- TEST INFRASTRUCTURE ONLY.

The network is the 4-level convolutional U-Net of the learned warm start
(BF16 tensors, FP32 accumulation on the GPU): two 3x3 convolutions per level
with base, 2, 4, 8 x base channels, a 2x2 stride-2 convolution down, nearest
upsampling followed by a 3x3 convolution up, the skip tensor concatenated after
the upsampled one, ReLU after every convolution, no normalisation layers, and a
1x1 FP32 head.  Tensors are NHWC.  Written in plain numpy FP64, one layer at a
time, with no fusion.

``emulate_bf16=True`` rounds every tensor to BF16 (round to nearest even) at the
points where the GPU stores one: the input, the 3x3 / 2x2 weights, every ReLU
output, and every gradient with respect to a stored activation.  Sums stay FP64,
so the two sides differ only by their accumulation order and precision.  With
``emulate_bf16=False`` the whole network is FP64 (used by the finite-difference
pins).

Layer table (name, kind, input channels, output channels) and parameter
layout: "conv3"/"up3" weights [3][3][cin][cout], "down2" [2][2][cin][cout],
"head" [cin][1]; each layer's weights are followed by its bias [cout]; the flat
parameter vector is the layers in table order.
"""
from __future__ import annotations

import numpy as np


def layers(base=32, cin=2):
    b = base
    return [("enc0a", "conv3", cin, b), ("enc0b", "conv3", b, b),
            ("down0", "down2", b, 2 * b), ("enc1a", "conv3", 2 * b, 2 * b), ("enc1b", "conv3", 2 * b, 2 * b),
            ("down1", "down2", 2 * b, 4 * b), ("enc2a", "conv3", 4 * b, 4 * b), ("enc2b", "conv3", 4 * b, 4 * b),
            ("down2", "down2", 4 * b, 8 * b), ("enc3a", "conv3", 8 * b, 8 * b), ("enc3b", "conv3", 8 * b, 8 * b),
            ("up2", "up3", 8 * b, 4 * b), ("cat2", "conv3", 8 * b, 4 * b), ("dec2", "conv3", 4 * b, 4 * b),
            ("up1", "up3", 4 * b, 2 * b), ("cat1", "conv3", 4 * b, 2 * b), ("dec1", "conv3", 2 * b, 2 * b),
            ("up0", "up3", 2 * b, b), ("cat0", "conv3", 2 * b, b), ("dec0", "conv3", b, b),
            ("head", "head", b, 1)]


def weight_shape(kind, ci, co):
    return {"conv3": (3, 3, ci, co), "up3": (3, 3, ci, co), "down2": (2, 2, ci, co), "head": (ci, co)}[kind]


def param_shapes(base=32, cin=2):
    out = []
    for _, kind, ci, co in layers(base, cin):
        out += [weight_shape(kind, ci, co), (co,)]
    return out


def unpack(flat, base=32, cin=2):
    ps, k = [], 0
    for s in param_shapes(base, cin):
        n = int(np.prod(s))
        ps.append(np.asarray(flat[k:k + n], dtype=np.float64).reshape(s))
        k += n
    assert k == len(flat)
    return ps


def pack(ps):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in ps])


def bf16(x):
    """Round to the nearest BF16 value (8 significant bits), ties to even."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


# ---------------------------------------------------------------- layers ----
def _pad(x):
    n, h, w, c = x.shape
    xp = np.zeros((n, h + 2, w + 2, c))
    xp[:, 1:-1, 1:-1] = x
    return xp


def conv3(x, W, b):
    """y[n,i,j,o] = b[o] + sum_{a,c,ci} x[n, i+a-1, j+c-1, ci] W[a,c,ci,o], zero outside."""
    n, h, w, _ = x.shape
    xp = _pad(x)
    y = np.zeros((n, h, w, W.shape[3])) + b
    for a in range(3):
        for c in range(3):
            y += xp[:, a:a + h, c:c + w, :] @ W[a, c]
    return y


def conv3_back(x, W, g):
    """Gradients of conv3 given g = dL/dy: (dL/dx, dL/dW, dL/db)."""
    n, h, w, ci = x.shape
    co = W.shape[3]
    xp = _pad(x)
    gxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    g2 = g.reshape(-1, co)
    for a in range(3):
        for c in range(3):
            dW[a, c] = xp[:, a:a + h, c:c + w, :].reshape(-1, ci).T @ g2
            gxp[:, a:a + h, c:c + w, :] += g @ W[a, c].T
    return gxp[:, 1:-1, 1:-1], dW, g2.sum(axis=0)


def down2(x, W, b):
    """y[n,i,j,o] = b[o] + sum_{a,c,ci} x[n, 2i+a, 2j+c, ci] W[a,c,ci,o]."""
    y = np.zeros((x.shape[0], x.shape[1] // 2, x.shape[2] // 2, W.shape[3])) + b
    for a in range(2):
        for c in range(2):
            y += x[:, a::2, c::2, :] @ W[a, c]
    return y


def down2_back(x, W, g):
    ci, co = W.shape[2], W.shape[3]
    gx = np.zeros_like(x)
    dW = np.zeros_like(W)
    g2 = g.reshape(-1, co)
    for a in range(2):
        for c in range(2):
            gx[:, a::2, c::2, :] = g @ W[a, c].T
            dW[a, c] = x[:, a::2, c::2, :].reshape(-1, ci).T @ g2
    return gx, dW, g2.sum(axis=0)


def up(x):
    """Nearest-neighbour upsampling by 2 in both directions."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_back(g):
    n, h, w, c = g.shape
    return g.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def relu(z):
    return np.maximum(z, 0.0)


# --------------------------------------------------------------- network ----
def forward(flat, x, base=32, emulate_bf16=True):
    """Network output (N,H,W) and the stored activations.  x: (N,H,W,cin)."""
    R = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    cin = x.shape[3]
    ps = unpack(flat, base, cin)
    L = {name: (kind, ps[2 * k], ps[2 * k + 1]) for k, (name, kind, _, _) in enumerate(layers(base, cin))}

    def wt(name):
        kind, W, b = L[name]
        return (W if kind == "head" else R(W)), b

    A = {"x": R(x)}

    def c3(name, inp):
        W, b = wt(name)
        A[name] = R(relu(conv3(inp, W, b)))
        return A[name]

    def d2(name, inp):
        W, b = wt(name)
        A[name] = R(relu(down2(inp, W, b)))
        return A[name]

    s = [None] * 4
    h = A["x"]
    for l in range(4):
        if l > 0:
            h = d2(f"down{l - 1}", s[l - 1])
        h = c3(f"enc{l}a", h)
        s[l] = c3(f"enc{l}b", h)
    h = s[3]
    for l in (2, 1, 0):
        u = c3(f"up{l}", up(h))
        h = c3(f"cat{l}", np.concatenate([u, s[l]], axis=3))
        h = c3(f"dec{l}", h)
    W, b = wt("head")
    out = (h @ W)[..., 0] + b[0]
    return out, A


def loss_and_grads(flat, x, target, base=32, emulate_bf16=True):
    """Mean squared error over all outputs, and its gradient as a flat vector."""
    R = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    cin = x.shape[3]
    ps = unpack(flat, base, cin)
    names = [n for n, _, _, _ in layers(base, cin)]
    L = {name: (ps[2 * k], ps[2 * k + 1]) for k, name in enumerate(names)}
    out, A = forward(flat, x, base, emulate_bf16)
    m = out.size
    dout = 2.0 * (out - target) / m
    loss = float(np.mean((out - target) ** 2))
    G = {}

    def Wq(name):
        return R(L[name][0])

    # head: out = dec0 . w + b
    w = L["head"][0]
    G["head"] = (A["dec0"].reshape(-1, w.shape[0]).T @ dout.reshape(-1, 1), np.array([dout.sum()]))
    g = R((dout[..., None] * w[:, 0]) * (A["dec0"] > 0))  # dL/d(pre-activation of dec0)

    skip = [None] * 4
    for l in (0, 1, 2):  # decoder, in reverse order of the forward pass
        gx, dW, db = conv3_back(A[f"cat{l}"], Wq(f"dec{l}"), g)
        G[f"dec{l}"] = (dW, db)
        g = R(gx * (A[f"cat{l}"] > 0))
        cat_in = np.concatenate([A[f"up{l}"], A[f"enc{l}b"]], axis=3)
        gx, dW, db = conv3_back(cat_in, Wq(f"cat{l}"), g)
        G[f"cat{l}"] = (dW, db)
        cu = A[f"up{l}"].shape[3]
        skip[l] = R(gx[..., cu:])
        g = R(gx[..., :cu] * (A[f"up{l}"] > 0))
        low = A["enc3b"] if l == 2 else A[f"dec{l + 1}"]
        gx, dW, db = conv3_back(up(low), Wq(f"up{l}"), g)
        G[f"up{l}"] = (dW, db)
        g = R(up_back(gx) * (low > 0))
    # g is now dL/d(pre-activation of enc3b) (enc3b's output feeds up2 only)
    for l in (3, 2, 1, 0):
        if l < 3:  # enc{l}b feeds down{l} and, through the skip, cat{l}
            gx, dW, db = down2_back(A[f"enc{l}b"], Wq(f"down{l}"), g)
            G[f"down{l}"] = (dW, db)
            g = R((gx + skip[l]) * (A[f"enc{l}b"] > 0))
        gx, dW, db = conv3_back(A[f"enc{l}a"], Wq(f"enc{l}b"), g)
        G[f"enc{l}b"] = (dW, db)
        g = R(gx * (A[f"enc{l}a"] > 0))
        inp = A["x"] if l == 0 else A[f"down{l - 1}"]
        gx, dW, db = conv3_back(inp, Wq(f"enc{l}a"), g)
        G[f"enc{l}a"] = (dW, db)
        if l > 0:
            g = R(gx * (inp > 0))
    return loss, pack([t for name in names for t in G[name]])
