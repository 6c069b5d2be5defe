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
  output: y = conv(x) (c[0] -> 3 channels, no activation), then the fixed
          output stage p = unstagger(smooth(y)) below

Arrays are NHWC (n, h, w, c); a convolution has weights (3, 3, cin, cout)
(tap row, tap column, input channel, output channel) and a bias (cout,), and
computes out(y, x) = b + sum_{dy,dx} in(y + dy - 1, x + dx - 1) W[dy, dx]
with zeros outside the grid.  avgpool2 averages 2x2 blocks; upsample2
repeats each value into a 2x2 block.

Output stage (fixed, no parameters; fluid = input channel 0 below 1/2):
smooth() applies [1, 2, 1] / 4 along x and then along y to each channel,
taking the values at solid cells and outside the grid as 0, and sets solid
cells to 0; unstagger() removes from channel 1 (u_x) its component along
(-1)^x and from channel 2 (u_y) its component along (-1)^y over the fluid
cells of each instance (an orthogonal projection).  The lattice Boltzmann
scheme keeps the staggered momenta sum (-1)^(x+n) rho u_x and
sum (-1)^(y+n) rho u_y exactly, so a start that carries them never reaches
the steady state of a start from rest; the smoothing removes the grid-scale
content that feeds them and the projection sets what is left to zero.  Both
maps are self-adjoint, so the backward pass applies them again (in reverse
order).

With ``bf16_storage=True`` the weights, every stored activation and every
stored activation gradient are rounded to bfloat16 (round to nearest even)
where the CUDA kernels store them -- the inputs, each layer's output, the
gradient of the last convolution's output (after the output stage's
backward pass), each input gradient of a convolution, of an upsampling and
of a pooling (together with the skip gradient it joins) -- while sums stay
in FP64, and the output stage, its result, the loss gradient and the
parameter gradients are not rounded (the kernels keep them in FP32).

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


def fluid_of_input(x):
    """Fluid flag per cell from the input planes (channel 0: solid flag)."""
    return np.asarray(x)[..., 0] < 0.5


def smooth(y, fluid):
    """[1, 2, 1] / 4 along x, then along y, of every channel; solid cells and
    cells outside the grid count as 0, and solid cells are set to 0."""
    m = fluid[..., None].astype(np.float64)
    g = y * m
    p = np.pad(g, ((0, 0), (0, 0), (1, 1), (0, 0)))
    g = 0.25 * p[:, :, :-2] + 0.5 * p[:, :, 1:-1] + 0.25 * p[:, :, 2:]
    p = np.pad(g, ((0, 0), (1, 1), (0, 0), (0, 0)))
    g = 0.25 * p[:, :-2] + 0.5 * p[:, 1:-1] + 0.25 * p[:, 2:]
    return g * m


def unstagger(y, fluid):
    """Channel 1 minus its projection on (-1)^x, channel 2 minus its
    projection on (-1)^y, over the fluid cells of each instance."""
    n, h, w, _ = y.shape
    yy, xx = np.mgrid[0:h, 0:w]
    out = np.array(y, dtype=np.float64, copy=True)
    for k in range(n):
        m = fluid[k].astype(np.float64)
        nf = m.sum()
        if nf == 0:
            continue
        for ch, sign in ((1, (-1.0) ** xx), (2, (-1.0) ** yy)):
            sm = sign * m
            out[k, :, :, ch] -= ((sm * y[k, :, :, ch]).sum() / nf) * sm
    return out


def output_stage(y, fluid):
    return unstagger(smooth(y, fluid), fluid)


def output_stage_backward(g, fluid):
    return smooth(unstagger(g, fluid), fluid)


def prolong(y, factor, fluid):
    """Bilinear interpolation of cell-centred fields y (n, h, w, c) onto a
    grid `factor` times finer: the centre of fine cell (Y, X) sits at coarse
    coordinates ((Y + 1/2) / factor - 1/2, (X + 1/2) / factor - 1/2), clamped
    to [0, h - 1] x [0, w - 1] (constant beyond the outermost coarse
    centres); fine cells where `fluid` (n, h factor, w factor) is false get
    0.  Written cell by cell from the definition."""
    y = np.asarray(y, dtype=np.float64)
    n, h, w, c = y.shape
    H, W = h * factor, w * factor
    out = np.zeros((n, H, W, c))
    for Y in range(H):
        yc = min(max((Y + 0.5) / factor - 0.5, 0.0), h - 1.0)
        y0 = int(np.floor(yc))
        y1 = min(y0 + 1, h - 1)
        ty = yc - y0
        for X in range(W):
            xc = min(max((X + 0.5) / factor - 0.5, 0.0), w - 1.0)
            x0 = int(np.floor(xc))
            x1 = min(x0 + 1, w - 1)
            tx = xc - x0
            out[:, Y, X] = ((1 - ty) * ((1 - tx) * y[:, y0, x0] + tx * y[:, y0, x1])
                            + ty * ((1 - tx) * y[:, y1, x0] + tx * y[:, y1, x1]))
    return out * np.asarray(fluid, dtype=np.float64)[..., None]


def prolong_stage(y, factor, fluid):
    """prolong() followed by the output stage on the fine grid."""
    return output_stage(prolong(y, factor, fluid), fluid)


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
    def __init__(self, channels, params, bf16_storage=False, sum_noise=None):
        """sum_noise: None, or a seed.  With a seed, every convolution sum
        (forward and input gradient) is multiplied by 1 + 2^-24 sqrt(K) xi,
        xi standard normal, K the number of terms: the size of the error of
        an FP32 accumulation.  Running the reference with and without it
        shows how far the rounding of stored bfloat16 values alone carries
        such an error through the network."""
        self.channels = list(channels)
        self.L = len(channels)
        self.rnd = bf16 if bf16_storage else (lambda v: v)
        self.params = [(self.rnd(w), b.copy()) for w, b in params]
        self.noise = None if sum_noise is None else np.random.default_rng(sum_noise)

    def _sum_error(self, v, terms):
        if self.noise is None:
            return v
        return v * (1.0 + 2.0 ** -24 * np.sqrt(terms) * self.noise.standard_normal(v.shape))

    def forward(self, x):
        """Returns the output and the tape of stored activations."""
        r = self.rnd
        P = self.params
        tape = []
        k = 0

        def conv(v, relu):
            nonlocal k
            w, b = P[k]
            pre = self._sum_error(conv3x3(v, w, b), 9 * v.shape[3])
            k += 1
            out = r(np.maximum(pre, 0.0) if relu else pre)
            tape.append(("conv", v, k - 1, relu, out))
            return out

        x = r(x)
        fluid = fluid_of_input(x)
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
        tape.append(("out", fluid))
        return output_stage(y, fluid), tape

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
        g = gy
        for item in reversed(tape):
            if item[0] == "out":
                g = r(output_stage_backward(g, item[1]))
            elif item[0] == "conv":
                _, xin, k, relu, out = item
                if relu:
                    g = g * (out > 0.0)
                gx, gw, gb = conv3x3_backward(xin, self.params[k][0], g)
                grads[k] = (gw, gb)
                g = r(self._sum_error(gx, 9 * g.shape[3]))
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
