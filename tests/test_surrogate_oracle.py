"""Pins of the FP64 reference of the warm-start surrogate network.

The hand-written backward pass against central finite differences, the
convolution against its definition evaluated cell by cell, the pooling and
upsampling against their adjoints, the bfloat16 rounding against PyTorch's
conversion, and the first Adam step against its closed form.
"""
import numpy as np
import pytest

from oracle import surrogate_oracle as S


def test_conv3x3_matches_its_definition_cell_by_cell():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 4, 3))
    w = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(2)
    y = S.conv3x3(x, w, b)
    for n in range(2):
        for i in range(5):
            for j in range(4):
                for o in range(2):
                    s = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            yy, xx = i + dy - 1, j + dx - 1
                            if 0 <= yy < 5 and 0 <= xx < 4:
                                s += sum(x[n, yy, xx, c] * w[dy, dx, c, o] for c in range(3))
                    assert abs(y[n, i, j, o] - s) < 1e-12


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 8, 3))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose((S.avgpool2(x) * y).sum(), (x * S.avgpool2_backward(y)).sum(), rtol=1e-13)
    z = rng.standard_normal((2, 6, 8, 3))
    assert np.isclose((S.upsample2(y) * z).sum(), (y * S.upsample2_backward(z)).sum(), rtol=1e-13)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 6, 3))
    w = rng.standard_normal((3, 3, 3, 5))
    gy = rng.standard_normal((1, 4, 6, 5))
    gx, gw, gb = S.conv3x3_backward(x, w, gy)
    # <conv(x, w, 0), gy> is linear in x and in w
    lin = (S.conv3x3(x, w, np.zeros(5)) * gy).sum()
    assert np.isclose((gx * x).sum(), lin, rtol=1e-12)
    assert np.isclose((gw * w).sum(), lin, rtol=1e-12)
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


@pytest.mark.parametrize("channels", [[4, 8], [3, 5, 6]])
def test_backward_matches_finite_differences(channels):
    params = S.init_params(channels, seed=3)
    net = S.WarmNet(channels, params)
    rng = np.random.default_rng(4)
    hw = 2 ** (len(channels) + 1)
    x = rng.standard_normal((2, hw, hw, 4))
    t = rng.standard_normal((2, hw, hw, 3))
    fluid = rng.random((2, hw, hw)) > 0.2
    y, tape = net.forward(x)
    _, gy = net.loss(y, t, fluid)
    grads = net.backward(tape, gy)
    eps = 1e-6
    for k, (w, b) in enumerate(net.params):
        for idx in [(0, 0, 0, 0), (1, 2, w.shape[2] - 1, w.shape[3] // 2), (2, 1, 0, w.shape[3] - 1)]:
            w[idx] += eps
            lp = net.loss(net.forward(x)[0], t, fluid)[0]
            w[idx] -= 2 * eps
            lm = net.loss(net.forward(x)[0], t, fluid)[0]
            w[idx] += eps
            fd = (lp - lm) / (2 * eps)
            assert abs(grads[k][0][idx] - fd) <= 1e-6 * max(1e-3, abs(fd)), (k, idx)
        j = b.shape[0] - 1
        b[j] += eps
        lp = net.loss(net.forward(x)[0], t, fluid)[0]
        b[j] -= 2 * eps
        lm = net.loss(net.forward(x)[0], t, fluid)[0]
        b[j] += eps
        fd = (lp - lm) / (2 * eps)
        assert abs(grads[k][1][j] - fd) <= 1e-6 * max(1e-3, abs(fd)), (k, "bias")


def test_solid_cells_do_not_count_in_the_loss():
    channels = [4, 8]
    net = S.WarmNet(channels, S.init_params(channels, seed=5))
    rng = np.random.default_rng(6)
    x = rng.standard_normal((1, 8, 8, 4))
    y, _ = net.forward(x)
    t = y.copy()
    fluid = np.ones((1, 8, 8), bool)
    fluid[0, 2, 3] = False
    t[0, 2, 3] += 5.0
    loss, g = net.loss(y, t, fluid)
    assert loss == 0.0 and np.all(g == 0.0)


def test_config_network_shapes():
    channels = [32, 64, 128, 256]
    shapes = S.layer_shapes(channels)
    assert len(shapes) == 15 and shapes[0] == (4, 32) and shapes[-1] == (32, 3)
    net = S.WarmNet(channels, S.init_params(channels, seed=7))
    y, _ = net.forward(np.zeros((1, 16, 16, 4)))
    assert y.shape == (1, 16, 16, 3)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0]])
    v32 = v.astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(v32), ref)
    assert S.bf16(1.0 + 2.0 ** -8) == 1.0          # tie to even
    assert S.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_first_adam_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    q, m, v = S.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)
    assert np.allclose(q, p - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_output_stage_maps_are_self_adjoint_and_remove_staggered_content():
    """The fixed output stage: smooth() and unstagger() are self-adjoint (so
    the backward pass is the same maps in reverse order), unstagger() is a
    projection whose result carries no staggered momentum over the fluid
    cells, and smooth() annihilates the grid-scale patterns (-1)^x and
    (-1)^y away from walls and solids."""
    rng = np.random.default_rng(7)
    a = rng.standard_normal((2, 12, 10, 3))
    b = rng.standard_normal((2, 12, 10, 3))
    fluid = rng.random((2, 12, 10)) > 0.2
    for f in (S.smooth, S.unstagger):
        assert np.isclose((f(a, fluid) * b).sum(), (a * f(b, fluid)).sum(), rtol=1e-13)
    p = S.unstagger(a, fluid)
    np.testing.assert_allclose(S.unstagger(p, fluid), p, atol=1e-13)
    yy, xx = np.mgrid[0:12, 0:10]
    for k in range(2):
        m = fluid[k]
        assert abs(((-1.0) ** xx * m * p[k, :, :, 1]).sum()) < 1e-12
        assert abs(((-1.0) ** yy * m * p[k, :, :, 2]).sum()) < 1e-12
    np.testing.assert_array_equal(p[..., 0], a[..., 0])
    allf = np.ones((1, 12, 10), bool)
    z = np.zeros((1, 12, 10, 3))
    z[0, :, :, 1] = (-1.0) ** xx
    z[0, :, :, 2] = (-1.0) ** yy
    s = S.smooth(z, allf)
    assert np.abs(s[0, 1:-1, 1:-1, 1:]).max() < 1e-15
    # a smooth field passes with an O(h^2) change
    sm = np.zeros((1, 12, 10, 3))
    sm[0, :, :, 0] = np.sin(2 * np.pi * xx / 10) * np.cos(np.pi * yy / 12)
    d = S.smooth(sm, allf) - sm
    assert np.abs(d[0, 1:-1, 1:-1, 0]).max() < 0.12


def test_output_stage_in_the_network_forward():
    channels = [4, 8]
    net = S.WarmNet(channels, S.init_params(channels, seed=5))
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, 8, 8, 4))
    x[..., 0] = rng.random((2, 8, 8)) > 0.8
    y, tape = net.forward(x)
    fluid = x[..., 0] < 0.5
    assert np.all(y[~fluid] == 0)
    yy, xx = np.mgrid[0:8, 0:8]
    for k in range(2):
        assert abs(((-1.0) ** xx * fluid[k] * y[k, :, :, 1]).sum()) < 1e-12
        assert abs(((-1.0) ** yy * fluid[k] * y[k, :, :, 2]).sum()) < 1e-12


# ---- prolongation of coarse predictions to a finer lattice ----

def test_prolong_identity_at_factor_one():
    rng = np.random.default_rng(21)
    y = rng.normal(size=(2, 5, 7, 3))
    fl = rng.random((2, 5, 7)) > 0.2
    assert np.array_equal(S.prolong(y, 1, fl), y * fl[..., None])


@pytest.mark.parametrize("factor", [2, 3, 4])
def test_prolong_reproduces_linear_fields_and_clamps(factor):
    """Bilinear interpolation between cell centres reproduces a field linear
    in the coarse centre coordinates; beyond the outermost centres it holds
    the value at the nearest one (coordinates clamped)."""
    h, w = 6, 9
    jj, ii = np.mgrid[0:h, 0:w]
    lin = lambda xc, yc: 0.3 + 1.7 * xc - 0.9 * yc
    y = np.stack([lin(ii, jj), 2 * lin(ii, jj), -lin(ii, jj)], axis=-1)[None]
    H, W = h * factor, w * factor
    out = S.prolong(y, factor, np.ones((1, H, W), bool))
    Y, X = np.mgrid[0:H, 0:W]
    xc = np.clip((X + 0.5) / factor - 0.5, 0, w - 1)
    yc = np.clip((Y + 0.5) / factor - 0.5, 0, h - 1)
    ref = lin(xc, yc)
    assert np.allclose(out[0, ..., 0], ref, atol=1e-12)
    assert np.allclose(out[0, ..., 1], 2 * ref, atol=1e-12)
    # the first fine rows lie before the first coarse centre
    edge = (Y + 0.5) / factor - 0.5 < 0
    assert np.allclose(out[0][edge][:, 0], lin(xc[edge], 0.0), atol=1e-12)


@pytest.mark.parametrize("factor", [2, 4])
def test_prolong_hat_sums_to_the_cell_count(factor):
    """A single interior coarse value of 1 spreads into the tensor-product
    hat of width 2 coarse cells: its fine samples are symmetric about the
    coarse centre and sum to factor^2 (the coarse cell's share of the
    partition of unity); a shifted or transposed index breaks both."""
    h, w = 7, 8
    y = np.zeros((1, h, w, 3))
    y[0, 3, 4, 0] = 1.0
    out = S.prolong(y, factor, np.ones((1, h * factor, w * factor), bool))[0, ..., 0]
    assert abs(out.sum() - factor ** 2) <= 1e-12
    rows = slice(3 * factor - factor + 1, 3 * factor + 2 * factor - 1)
    cols = slice(4 * factor - factor + 1, 4 * factor + 2 * factor - 1)
    block = out[rows, cols]
    assert abs(block.sum() - factor ** 2) <= 1e-12
    assert np.allclose(block, block[::-1, :]) and np.allclose(block, block[:, ::-1])


def test_prolong_stage_leaves_no_staggered_momentum():
    rng = np.random.default_rng(22)
    y = rng.normal(size=(2, 4, 5, 3))
    fl = rng.random((2, 12, 15)) > 0.15
    out = S.prolong_stage(y, 3, fl)
    Y, X = np.mgrid[0:12, 0:15]
    for k in range(2):
        assert abs((out[k, ..., 1] * (-1.0) ** X * fl[k]).sum()) <= 1e-12
        assert abs((out[k, ..., 2] * (-1.0) ** Y * fl[k]).sum()) <= 1e-12
        assert np.all(out[k][~fl[k]] == 0.0)
