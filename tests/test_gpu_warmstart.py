"""Parity of the warm-start network kernels (lgnk_ws_*) with the oracle: the
forward pass, the loss and its gradient (every layer's W and b), one Adam step
and the bf16 weight copy it refreshes, on shapes that exercise ragged pixel
tiles, output-channel groups that do not fill a CTA, input-channel chunks, an
odd coarsest grid and batches of several images."""
import numpy as np
import pytest
import torch

from oracle import warmstart as W
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(4, 16, 2), (6, 40, 3), (8, 24, 1)]     # (c, m, B): m/8 = 2, 5, 3


def _inputs(c, m, B, seed=0):
    rng = np.random.default_rng(seed)
    T = rng.uniform(size=(B, m, m)).astype(np.float32)
    R = rng.uniform(size=(B, m, m)).astype(np.float32)
    vt = (0.05 * rng.normal(size=(B, 2, m // 2, m // 2))).astype(np.float32)
    p = synth.warmstart_init(c, seed)
    p = (p + 0.01 * rng.normal(size=p.shape)).astype(np.float32)      # nonzero biases
    return p, T, R, vt


def _net(c, m, B, scale, p):
    from paper_1703_04446_gb300 import lgnk
    net = lgnk.WarmStart(m, c, B, scale)
    net.set_params(torch.from_numpy(p))
    return net


def _cuda(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("c,m,B", SHAPES)
def test_forward_matches_oracle(c, m, B):
    scale = 0.05
    p, T, R, _ = _inputs(c, m, B)
    net = _net(c, m, B, scale, p)
    assert net.num_params == W.num_params(c)
    Tg, Rg = _cuda(T, R)
    v = net.predict(Tg, Rg).cpu().numpy()
    ref = W.forward(p.astype(np.float64), T.astype(np.float64), R.astype(np.float64), c, scale).numpy()
    assert v.shape == ref.shape
    assert _rel(v, ref) <= 1e-5
    assert np.max(np.abs(v - ref)) <= 1e-5 * np.max(np.abs(ref))
    # a smaller batch through the same buffers gives the same images
    if B > 1:
        v1 = net.predict(Tg[:1].contiguous(), Rg[:1].contiguous()).cpu().numpy()
        assert np.array_equal(v1, v[:1])


@pytest.mark.parametrize("c,m,B", SHAPES)
def test_loss_and_gradient_match_oracle(c, m, B):
    scale = 0.05
    p, T, R, vt = _inputs(c, m, B, seed=1)
    net = _net(c, m, B, scale, p)
    Tg, Rg, vg = _cuda(T, R, vt)
    loss = net.train_step(Tg, Rg, vg, lr=0.0)
    g = net.grads().cpu().numpy()
    lref, gref, _ = W.loss_and_grad(p.astype(np.float64), T, R, vt, c, scale)
    assert abs(loss - lref) <= 1e-5 * lref
    # every layer's W and b separately, so a wrong index in one layer shows
    o = 0
    for ci, co, _, _ in W.layer_shapes(c):
        for n in (co * ci * 9, co):
            assert _rel(g[o:o + n], gref[o:o + n]) <= 1e-4, (ci, co, n)
            o += n
    assert o == g.size


def test_adam_step_and_bf16_refresh():
    c, m, B, scale, lr = 6, 40, 3, 0.05, 1e-3
    p, T, R, vt = _inputs(c, m, B, seed=2)
    net = _net(c, m, B, scale, p)
    Tg, Rg, vg = _cuda(T, R, vt)
    net.train_step(Tg, Rg, vg, lr=lr)
    g = net.grads().cpu().numpy().astype(np.float64)
    p1 = net.params().cpu().numpy()
    zero = np.zeros_like(g)
    ref, m1, s1 = W.adam_step(p.astype(np.float64), g, zero, zero, 1, lr)
    assert np.max(np.abs(p1 - ref)) <= 1e-6 * lr + 1e-7 * np.max(np.abs(ref))
    # the second step uses the moments of the first
    net.train_step(Tg, Rg, vg, lr=lr)
    g2 = net.grads().cpu().numpy().astype(np.float64)
    ref2, _, _ = W.adam_step(p1.astype(np.float64), g2, m1, s1, 2, lr)
    assert np.max(np.abs(net.params().cpu().numpy() - ref2)) <= 1e-5 * lr + 1e-7 * np.max(np.abs(ref2))
    # predictions use the refreshed bf16 copy of the updated master weights
    p2 = net.params().cpu().numpy().astype(np.float64)
    v = net.predict(Tg, Rg).cpu().numpy()
    vref = W.forward(p2, T, R, c, scale).numpy()
    assert _rel(v, vref) <= 1e-5


def test_training_decreases_the_loss():
    c, m, B, scale = 4, 32, 4, 0.05
    p, T, R, vt = _inputs(c, m, B, seed=3)
    net = _net(c, m, B, scale, p)
    Tg, Rg, vg = _cuda(T, R, vt)
    losses = [net.train_step(Tg, Rg, vg, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def test_set_params_resets_adam():
    c, m, B, scale = 4, 16, 2, 0.05
    p, T, R, vt = _inputs(c, m, B, seed=4)
    net = _net(c, m, B, scale, p)
    Tg, Rg, vg = _cuda(T, R, vt)
    net.train_step(Tg, Rg, vg, lr=1e-3)
    a = net.params().cpu().numpy()
    net.set_params(torch.from_numpy(p))
    net.train_step(Tg, Rg, vg, lr=1e-3)
    assert np.array_equal(net.params().cpu().numpy(), a)


def test_rejects_batches_over_the_maximum():
    from paper_1703_04446_gb300 import lgnk
    c, m = 4, 16
    p, T, R, _ = _inputs(c, m, 3)
    net = _net(c, m, 2, 0.05, p)
    Tg, Rg = _cuda(T, R)
    with pytest.raises(ValueError):
        net.predict(Tg, Rg)
    with pytest.raises(lgnk.LgnkError):
        net._check(net.lib.lgnk_ws_predict(net.handle, 3, net._t(Tg, T.size, "T"), net._t(Rg, R.size, "R"),
                                           net._t(torch.empty(3 * 2 * 8 * 8, device="cuda"), 384, "v")))


def test_pipeline_end_to_end_small():
    """The whole learned-warm-start pipeline on a few pairs: solver-made
    targets, training, then warm-started solves that reach the zero-start
    solves' gradient norm (the solver has the last word on the prediction)."""
    from paper_1703_04446_gb300 import warmstart as WS
    out = WS.run(n_train=16, n_test=4, channels=4, epochs=2, batch=8)
    ev = out["eval"]
    assert out["train_steps"] == 4 and out["loss_last"] > 0.0
    assert ev["pairs"] == 4
    assert ev["zero"]["converged"] >= 3 and ev["warm"]["converged"] >= ev["zero"]["converged"] - 1
    assert ev["final_J_ratio_warm_over_zero"] == pytest.approx(1.0, rel=5e-2)
