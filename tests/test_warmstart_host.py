"""Host-side data preparation of the warm start on a coarser grid
(warmstart.coarsen): block means of the inputs, fluid-weighted block means
of the targets, the coarse fluid rule, and sizes that do not split."""
import numpy as np
import pytest

from paper_2103_02119_gb300 import warmstart as WS


def test_coarsen_block_means():
    rng = np.random.default_rng(5)
    n, H, W, f = 3, 12, 8, 4
    x = rng.random((n, H, W, 4)).astype(np.float32)
    x[..., 0] = rng.random((n, H, W)) < 0.4
    t = rng.normal(size=(n, H, W, 3)).astype(np.float32)
    fl = (x[..., 0] < 0.5).astype(np.uint8)
    xc, tc, flc = WS.coarsen(x, t, fl, f)
    assert xc.shape == (n, 3, 2, 4) and tc.shape == (n, 3, 2, 3) and flc.shape == (n, 3, 2)
    for k in range(n):
        for i in range(3):
            for j in range(2):
                blk = (k, slice(f * i, f * i + f), slice(f * j, f * j + f))
                assert np.allclose(xc[k, i, j], x[blk].reshape(-1, 4).mean(axis=0), atol=1e-6)
                solid = x[blk][..., 0].mean()
                assert flc[k, i, j] == (solid < 0.5)
                m = fl[blk].astype(bool)
                want = t[blk][m].mean(axis=0) if flc[k, i, j] else np.zeros(3)
                assert np.allclose(tc[k, i, j], want, atol=1e-6)


def test_coarsen_identity_and_bad_sizes():
    x = np.zeros((1, 6, 6, 4), np.float32)
    t = np.zeros((1, 6, 6, 3), np.float32)
    fl = np.ones((1, 6, 6), np.uint8)
    assert WS.coarsen(x, t, fl, 1)[0] is x
    with pytest.raises(ValueError):
        WS.coarsen(x, t, fl, 4)
