"""FP64 reference of the warm-start surrogate network (TEST INFRASTRUCTURE ONLY:
the tests, the smoke check and the benchmark's CPU leg may use it; the CUDA
library never does).

The network ("WarmNet") maps per-cell inputs of a lid-driven cavity instance
(solid mask, aspect ratio a, log Reynolds number, lid speed) to an initial
guess of its steady fields (rho - 1, u_x / U, u_y / U).  It is an
encoder-decoder of 3x3 convolutions over L levels with channel counts
c[0] .. c[L-1]:

  encoder, level l = 0 .. L-1:
      x = relu(conv(x)); x = relu(conv(x)); skip[l] = x;
      x = avgpool2(x) unless l = L-1
  decoder, level l = L-2 .. 0:
      x = upsample2(x); x = relu(conv(x)) (c[l+1] -> c[l]);
      x = x + skip[l]; x = relu(conv(x))
  output: y = conv(x) (c[0] -> 3 channels, no activation)

Arrays are NHWC (n, h, w, c); a convolution has weights (3, 3, cin, cout)
(tap row, tap column, input channel, output channel) and a bias (cout,), and
computes out(y, x) = b + sum_{dy,dx} in(y + dy - 1, x + dx - 1) W[dy, dx]
with zeros outside the grid.  avgpool2 averages 2x2 blocks; upsample2
repeats each value into a 2x2 block.

With ``bf16_storage=True`` the weights, every stored activation and every
stored activation gradient are rounded to bfloat16 (round to nearest even)
where the CUDA kernels store them -- the inputs, each layer's output, the
loss gradient, each input gradient of a convolution, of an upsampling and
of a pooling (together with the skip gradient it joins) -- while sums stay
in FP64 and parameter gradients are not rounded.

Loss: L = sum_m fluid(m) sum_c (y - t)^2 / (3 sum_m fluid(m)), over all
cells m of the batch; solid cells do not count.

The backward pass is written out by hand (chain rule through each layer in
reverse); tests check it against central finite differences.
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b):
    n, h, wd, _ = x.shape
    xp = np.zeros((n, h + 2, wd + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, w.shape[3])) + b
    for dy in range(3):
        for dx in range(3):
            y += xp[:, dy:dy + h, dx:dx + wd, :] @ w[dy, dx]
    return y


def conv3x3_backward(x, w, gy):
    """Gradients (gx, gw, gb) of conv3x3 given the output gradient gy."""
    n, h, wd, _ = x.shape
    xp = np.zeros((n, h + 2, wd + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.einsum("nhwc,nhwo->co", xp[:, dy:dy + h, dx:dx + wd, :], gy)
            gxp[:, dy:dy + h, dx:dx + wd, :] += gy @ w[dy, dx].T
    return gxp[:, 1:-1, 1:-1], gw, gy.sum(axis=(0, 1, 2))


def avgpool2(x):
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])


def avgpool2_backward(gy):
    n, h, w, c = gy.shape
    gx = np.zeros((n, 2 * h, 2 * w, c))
    for a in (0, 1):
        for b in (0, 1):
            gx[:, a::2, b::2] = 0.25 * gy
    return gx


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_backward(gy):
    return gy[:, 0::2, 0::2] + gy[:, 1::2, 0::2] + gy[:, 0::2, 1::2] + gy[:, 1::2, 1::2]


def layer_shapes(channels, cin=4, cout=3):
    """(cin, cout) of the convolutions, in the order of the forward pass."""
    L = len(channels)
    shapes = []
    prev = cin
    for l in range(L):
        shapes += [(prev, channels[l]), (channels[l], channels[l])]
        prev = channels[l]
    for l in range(L - 2, -1, -1):
        shapes += [(channels[l + 1], channels[l]), (channels[l], channels[l])]
    shapes.append((channels[0], cout))
    return shapes


def init_params(channels, seed, cin=4, cout=3):
    """He-normal weights (std sqrt(2 / (9 cin))), zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for ci, co in layer_shapes(channels, cin, cout):
        w = rng.standard_normal((3, 3, ci, co)) * np.sqrt(2.0 / (9 * ci))
        params.append((w, np.zeros(co)))
    return params


class WarmNet:
    def __init__(self, channels, params, bf16_storage=False):
        self.channels = list(channels)
        self.L = len(channels)
        self.rnd = bf16 if bf16_storage else (lambda v: v)
        self.params = [(self.rnd(w), b.copy()) for w, b in params]

    def forward(self, x):
        """Returns the output and the tape of stored activations."""
        r = self.rnd
        P = self.params
        tape = []
        k = 0

        def conv(v, relu):
            nonlocal k
            w, b = P[k]
            pre = conv3x3(v, w, b)
            k += 1
            out = r(np.maximum(pre, 0.0) if relu else pre)
            tape.append(("conv", v, k - 1, relu, out))
            return out

        x = r(x)
        skips = []
        for l in range(self.L):
            x = conv(x, True)
            x = conv(x, True)
            skips.append(x)
            if l < self.L - 1:
                x = r(avgpool2(x))
                tape.append(("pool",))
        for l in range(self.L - 2, -1, -1):
            x = upsample2(x)
            tape.append(("up",))
            x = conv(x, True)
            x = r(x + skips[l])
            tape.append(("skip", l))
            x = conv(x, True)
        y = conv(x, False)
        return y, tape

    def loss(self, y, target, fluid):
        m = fluid[..., None].astype(np.float64)
        cnt = 3.0 * m.sum()
        d = (y - target) * m
        return float((d * d).sum() / cnt), 2.0 * d / cnt

    def backward(self, tape, gy):
        """Gradients [(gw, gb)] of every convolution from the output gradient.

        The encoder output e_l of level l (l < L-1) feeds both the pool into
        level l+1 and the skip addition of decoder level l, so its gradient is
        the sum of the two; the addition passes its gradient to both inputs."""
        r = self.rnd
        grads = [None] * len(self.params)
        skip_grads = {}
        pool_level = 0
        for item in tape:
            if item[0] == "pool":
                pool_level += 1
        g = r(gy)
        for item in reversed(tape):
            if item[0] == "conv":
                _, xin, k, relu, out = item
                if relu:
                    g = g * (out > 0.0)
                gx, gw, gb = conv3x3_backward(xin, self.params[k][0], g)
                grads[k] = (gw, gb)
                g = r(gx)
            elif item[0] == "skip":
                skip_grads[item[1]] = g
            elif item[0] == "up":
                g = r(upsample2_backward(g))
            elif item[0] == "pool":
                pool_level -= 1
                g = r(avgpool2_backward(g) + skip_grads.pop(pool_level))
        return grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected) of parameter p with gradient g."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
