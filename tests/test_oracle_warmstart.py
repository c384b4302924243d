"""Pins of the warm-start network oracle: its backward pass against central
differences of its loss, Adam's first step against its closed form, and the
shapes it produces."""
import numpy as np
import pytest
import torch

from oracle import warmstart as W
from paper_1703_04446_gb300 import synth


def _batch(c=4, m=16, B=2, seed=0):
    rng = np.random.default_rng(seed)
    T = rng.uniform(size=(B, m, m))
    R = rng.uniform(size=(B, m, m))
    vt = 0.05 * rng.normal(size=(B, 2, m // 2, m // 2))
    p = synth.warmstart_init(c, seed).astype(np.float64)
    p += 0.01 * rng.normal(size=p.shape)            # nonzero biases
    return p, T, R, vt


def test_shapes_and_parameter_count():
    c, m = 4, 16
    p, T, R, vt = _batch(c, m)
    assert p.size == W.num_params(c)
    assert W.forward(p, T, R, c, 0.05).shape == (2, 2, m // 2, m // 2)


def test_gradient_matches_central_differences():
    """The loss is piecewise smooth (ReLU); with the bf16 rounding held fixed it
    is piecewise quadratic in the biases of the last layer and smooth almost
    everywhere in the rest: central differences on random directions agree."""
    c, m, scale = 4, 16, 0.05
    p, T, R, vt = _batch(c, m)
    loss, g, _ = W.loss_and_grad(p, T, R, vt, c, scale)
    nb = W.num_params(c)
    # directions that move only the biases (no bf16 rounding involved)
    bias_mask = np.zeros(nb)
    o = 0
    for ci, co, _, _ in W.layer_shapes(c):
        o += co * ci * 9
        bias_mask[o:o + co] = 1.0
        o += co
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.normal(size=nb) * bias_mask
        eps = 1e-6
        lp = W.loss_and_grad(p + eps * d, T, R, vt, c, scale)[0]
        lm = W.loss_and_grad(p - eps * d, T, R, vt, c, scale)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))


def test_weight_gradient_against_differences_of_unrounded_network():
    """Weight gradients (straight-through rounding) equal the gradient of the
    same network evaluated without bf16 rounding, checked by differences."""
    c, m, scale = 4, 16, 0.05
    p, T, R, vt = _batch(c, m, seed=1)
    p = W.bf16_round(p).numpy()                     # rounding is exact at these weights
    _, g, _ = W.loss_and_grad(p, T, R, vt, c, scale)
    rng = np.random.default_rng(5)
    d = rng.normal(size=p.size)

    def plain_loss(q):
        q = torch.tensor(q)
        layers = W.unpack(q, c)
        x = torch.stack([torch.tensor(T), torch.tensor(R)], dim=1)
        conv = lambda z, k, s=1, up=False: torch.nn.functional.conv2d(
            torch.nn.functional.interpolate(z, scale_factor=2, mode="nearest") if up else z,
            layers[k][0], layers[k][1], stride=s, padding=1)
        e0 = torch.relu(conv(x, 0)); e1 = torch.relu(conv(e0, 1, 2)); e2 = torch.relu(conv(e1, 2, 2))
        e3 = torch.relu(conv(e2, 3, 2)); d2 = torch.relu(conv(e3, 4, up=True)) + e2
        d1 = torch.relu(conv(d2, 5, up=True)) + e1
        v = scale * conv(d1, 6)
        return float(0.5 * torch.mean((v - torch.tensor(vt)) ** 2) / scale ** 2)

    eps = 1e-7
    fd = (plain_loss(p + eps * d) - plain_loss(p - eps * d)) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-5 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    """After one step from zero moments, Adam moves each parameter by
    lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    p, g = rng.normal(size=50), rng.normal(size=50)
    new, m, s = W.adam_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    np.testing.assert_allclose(new, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_prior_velocity_is_windowed_and_scaled():
    g = synth.GridSpec((32, 32), (0.0, 0.0), (1.0, 1.0))
    v = synth.prior_velocity(g, 1e-2, 10 / 128, 3)
    assert v.shape == (1, 2, 32, 32)
    assert abs(np.sqrt((v[0] ** 2).sum(0)).max() - 10 / 128) < 1e-6


def test_forward_by_hand_on_single_tap_weights():
    """Architecture pin with c = 1 on 8 x 8 images, written out pixel by pixel
    without convolutions.  Layer e0 has only its top-left tap (output (i, j)
    reads input (i - 1, j - 1), zero padding), every other layer only its
    centre tap, so each layer is a channel mixing at the sampled pixel: stride
    2 reads pixel (2i, 2j), up2 reads (i // 2, j // 2).  This fixes the layer
    order, the skip connections, where the ReLUs sit, the strides, the
    upsampling, the padding and the output scale.  Weights are multiples of
    1/8 (exact in bfloat16) except one 1/3, which the network rounds to
    bfloat16: 0.333984375 (8 significant bits, to nearest)."""
    c, m, scale = 1, 8, 0.05
    rng = np.random.default_rng(11)
    shapes = W.layer_shapes(c)
    Ws, bs = [], []
    for k, (ci, co, _, _) in enumerate(shapes):
        Ws.append(rng.integers(-16, 17, size=(co, ci)) / 8.0)
        bs.append(rng.integers(-8, 9, size=co) / 8.0)
    Ws[3][5, 2] = 1.0 / 3.0
    params = []
    for k, (ci, co, _, _) in enumerate(shapes):
        w = np.zeros((co, ci, 3, 3))
        ky, kx = (0, 0) if k == 0 else (1, 1)
        w[:, :, ky, kx] = Ws[k]
        params += [w.ravel(), bs[k]]
    params = np.concatenate(params)
    T = rng.uniform(-1, 1, size=(m, m))
    R = rng.uniform(-1, 1, size=(m, m))
    Wr = [w.copy() for w in Ws]
    Wr[3][5, 2] = 0.333984375
    relu = lambda a: max(a, 0.0)
    e0 = np.zeros((1, m, m))
    for i in range(m):
        for j in range(m):
            t, r = (T[i - 1, j - 1], R[i - 1, j - 1]) if i >= 1 and j >= 1 else (0.0, 0.0)
            e0[0, i, j] = relu(bs[0][0] + Wr[0][0, 0] * t + Wr[0][0, 1] * r)

    def mix(k, src, co, i, j):
        return bs[k][co] + sum(Wr[k][co, q] * src[q] for q in range(len(src)))

    def down(k, x, n_out):
        co_n = Wr[k].shape[0]
        out = np.zeros((co_n, n_out, n_out))
        for o in range(co_n):
            for i in range(n_out):
                for j in range(n_out):
                    out[o, i, j] = relu(mix(k, x[:, 2 * i, 2 * j], o, i, j))
        return out

    e1 = down(1, e0, m // 2)
    e2 = down(2, e1, m // 4)
    e3 = down(3, e2, m // 8)

    def up(k, x, skip, n_out):
        co_n = Wr[k].shape[0]
        out = np.zeros((co_n, n_out, n_out))
        for o in range(co_n):
            for i in range(n_out):
                for j in range(n_out):
                    out[o, i, j] = relu(mix(k, x[:, i // 2, j // 2], o, i, j)) + skip[o, i, j]
        return out

    d2 = up(4, e3, e2, m // 4)
    d1 = up(5, d2, e1, m // 2)
    v = np.zeros((2, m // 2, m // 2))
    for o in range(2):
        for i in range(m // 2):
            for j in range(m // 2):
                v[o, i, j] = scale * mix(6, d1[:, i, j], o, i, j)
    got = W.forward(params, T[None], R[None], c, scale).numpy()[0]
    assert np.abs(v).max() > 0.01            # the chosen weights leave a nonzero output
    np.testing.assert_allclose(got, v, rtol=1e-12, atol=1e-14)
