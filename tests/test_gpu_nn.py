"""The warm-start surrogate's CUDA kernels against the FP64 reference network.

The reference runs in its bfloat16 mode (weights, activations and
activation gradients rounded where the kernels store them), so the two
differ only by FP32 versus FP64 accumulation and the rare bfloat16 rounding
decision that flips because of it.
"""
import numpy as np
import pytest

from oracle import surrogate_oracle as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def setup(channels, n, hw, seed):
    from paper_2103_02119_gb300 import lbm as L
    params = S.init_params(channels, seed=seed)
    params = [(S.bf16(w), S.bf16(b)) for w, b in params]  # representable on both sides
    rng = np.random.default_rng(seed + 1)
    x = S.bf16(rng.standard_normal((n, hw, hw, 4)))
    t = rng.standard_normal((n, hw, hw, 3))
    fluid = rng.random((n, hw, hw)) > 0.15
    nn = L.lbm_nn_create(channels, n, hw, hw, seed=0)
    L.lbm_nn_set_params(nn, L.params_to_vec(params).astype(np.float32))
    ref = S.WarmNet(channels, params, bf16_storage=True)
    return L, nn, ref, x, t, fluid


@pytest.mark.parametrize("channels,n,hw", [([8, 16], 2, 16), ([8, 16, 24], 3, 24),
                                           ([32, 64, 128, 256], 2, 32)])
def test_forward_matches_reference(channels, n, hw):
    L, nn, ref, x, _, _ = setup(channels, n, hw, seed=1)
    y = L.lbm_nn_forward(nn, x)
    yr, _ = ref.forward(x)
    assert y.shape == yr.shape
    assert rel(y, yr) < 1e-2, rel(y, yr)
    L.lbm_nn_destroy(nn)


@pytest.mark.parametrize("channels,n,hw", [([8, 16], 2, 16), ([8, 16, 24], 3, 24),
                                           ([32, 64, 128, 256], 2, 32)])
def test_gradients_match_reference(channels, n, hw):
    L, nn, ref, x, t, fluid = setup(channels, n, hw, seed=2)
    loss, g = L.lbm_nn_gradients(nn, x, t, fluid)
    yr, tape = ref.forward(x)
    lr, gy = ref.loss(yr, t, fluid)
    gr = ref.backward(tape, gy)
    assert abs(loss - lr) <= 2e-3 * lr
    shapes = S.layer_shapes(channels)
    got = L.params_to_list(g, shapes)
    for k, ((gw, gb), (rw, rb)) in enumerate(zip(got, gr)):
        assert rel(gw, rw) < 3e-2, (k, rel(gw, rw))
        assert rel(gb, rb) < 3e-2, (k, rel(gb, rb))
    L.lbm_nn_destroy(nn)


def test_adam_step_matches_reference():
    L, nn, ref, x, t, fluid = setup([8, 16], 2, 16, seed=3)
    p0 = L.lbm_nn_get_params(nn).astype(np.float64)
    _, g = L.lbm_nn_gradients(nn, x, t, fluid)
    lr = 1e-3
    L.lbm_nn_train_step(nn, x, t, fluid, lr)
    p1 = L.lbm_nn_get_params(nn).astype(np.float64)
    q, _, _ = S.adam_step(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, lr)
    assert np.abs(p1 - q).max() <= 1e-6 + 1e-5 * np.abs(p0).max()
    L.lbm_nn_destroy(nn)


def test_training_reduces_the_loss():
    L, nn, _, x, _, fluid = setup([8, 16], 2, 16, seed=4)
    # a smooth target the network can fit
    yy, xx = np.meshgrid(np.linspace(0, 1, 16), np.linspace(0, 1, 16), indexing="ij")
    t = np.stack([np.sin(3 * xx) * yy, xx * yy, np.cos(2 * yy)], axis=-1)[None].repeat(2, 0)
    first = L.lbm_nn_train_step(nn, x, t, fluid, 3e-3)
    for _ in range(150):
        last = L.lbm_nn_train_step(nn, x, t, fluid, 3e-3)
    assert last < 0.2 * first, (first, last)
    L.lbm_nn_destroy(nn)


def test_batch_size_limits():
    from paper_2103_02119_gb300 import lbm as L
    nn = L.lbm_nn_create([8], 2, 8, 8)
    with pytest.raises(L.LbmError):
        L.lbm_nn_forward(nn, np.zeros((3, 8, 8, 4), np.float32))
    L.lbm_nn_destroy(nn)


def test_warm_start_against_rest_start(orc):
    """A network trained on solver-generated steady cavities starts new
    instances; the unmodified scheme finishes them to the same residual.  The
    warm-started final fields describe the same flow as the rest-started ones
    and stay steady under the FP64 oracle.  The steps either way are reported
    (the gain is not asserted: at the accuracy reached here the warm start
    needs more steps, see the design notes)."""
    from paper_2103_02119_gb300 import warmstart as WS
    n = 32
    wls, x, t, fl, _ = WS.build_dataset(128, seed=0, n=n, max_steps=200_000)
    assert len(wls) >= 120
    ws = WS.WarmStart([16, 32, 64, 128], n=n, max_batch=32, seed=0)
    hist = ws.train(x, t, fl, epochs=20, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    test = WS.cavity_set(8, seed=1, n=n)
    y = ws.predict(WS.inputs_of(test))
    assert np.isfinite(y).all()
    rest = WS.solve(test, max_steps=200_000)
    warm = WS.solve(test, inits=[WS.fields_of(w, y[k]) for k, w in enumerate(test)],
                    max_steps=400_000)
    for res in (rest, warm):
        assert np.all((res["residual"] >= 0) & (res["residual"] <= 1e-8))
    print("steps rest", rest["steps"].tolist(), "warm", warm["steps"].tolist())
    # Both runs meet the residual test, yet their final fields agree only to
    # a few per cent (relative L2): the start from the prediction excites
    # slowly decaying components that the residual test does not resolve
    # (these runs also take many more steps).  The bound checks the two
    # describe the same flow.
    for k, w in enumerate(test):
        fluid = w.mask == 0
        a = np.stack(rest["fields"][k][1:])[:, fluid]
        b = np.stack(warm["fields"][k][1:])[:, fluid]
        rel = np.linalg.norm(a - b) / np.linalg.norm(a)
        print("instance", k, "relative difference rest vs warm", rel)
        assert rel <= 0.25, (k, rel)
    # the warm-started steady state of one instance under the FP64 oracle
    from paper_2103_02119_gb300.lbm import Batch
    w = test[0]
    b = Batch([w])
    b.init_fields(0, *WS.fields_of(w, y[0]))
    b.run(1e-8, check_every=100, max_steps=400_000)
    f = b.get_f(0)
    _, ug, vg = b.moments(0)
    b.close()
    p = orc.OracleParams.make(w.nx, w.ny, w.a, w.cs2, w.omega, periodic_x=0, periodic_y=0,
                              wall_u=w.wall_u)
    o = orc.Oracle(p, w.mask)
    o.set_f(f)
    o.step(200)
    _, uo, vo = o.moments()
    fluid = o.solid() == 0
    assert np.abs(uo - ug)[fluid].max() < 1e-3 * w.info["U"]
    assert np.abs(vo - vg)[fluid].max() < 1e-3 * w.info["U"]
    ws.close()
