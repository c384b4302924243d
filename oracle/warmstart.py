"""Oracle of the learned warm start: the encoder-decoder that maps an image pair
(T, R) to a starting velocity, and one Adam step of its training, in plain
PyTorch CPU FP64.  The paper has no such network (it is an addition that
feeds the Gauss-Newton solve of Eq. 11 a starting point); this file fixes the
architecture the CUDA kernels implement, so they can be checked layer by
layer.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network for m x m images (m divisible by 8), c base channels:
  e0 = relu(conv3(x, 2 -> c, stride 1))              m
  e1 = relu(conv3(e0, c -> 2c, stride 2))            m/2
  e2 = relu(conv3(e1, 2c -> 4c, stride 2))           m/4
  e3 = relu(conv3(e2, 4c -> 8c, stride 2))           m/8
  d2 = relu(conv3(up2(e3), 8c -> 4c)) + e2           m/4
  d1 = relu(conv3(up2(d2), 4c -> 2c)) + e1           m/2
  v  = scale * conv3(d1, 2c -> 2)                    m/2  (velocity, 2 components)
conv3: 3 x 3 kernel, zero padding 1; up2: nearest-neighbour doubling.  The
convolutions use the weights rounded to bfloat16 (round to nearest even);
the master weights, biases, accumulation and activations are wider.
Loss: 1/2 mean((v - v_target)^2) / scale^2.  Adam: beta1 0.9, beta2 0.999,
eps 1e-8, on the master weights.
Parameters are one flat vector: for each layer in the order above, W
[c_out][c_in][3][3] then b [c_out].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

LAYERS = ("e0", "e1", "e2", "e3", "d2", "d1", "out")


def layer_shapes(c: int):
    """(c_in, c_out, stride, upsample-input) of every layer."""
    return [(2, c, 1, False), (c, 2 * c, 2, False), (2 * c, 4 * c, 2, False), (4 * c, 8 * c, 2, False),
            (8 * c, 4 * c, 1, True), (4 * c, 2 * c, 1, True), (2 * c, 2, 1, False)]


def num_params(c: int) -> int:
    return sum(co * ci * 9 + co for ci, co, _, _ in layer_shapes(c))


def unpack(params, c: int):
    """Flat parameter vector -> list of (W, b) tensors."""
    out, o = [], 0
    p = torch.as_tensor(params)
    for ci, co, _, _ in layer_shapes(c):
        w = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned in float64."""
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64)


def forward(params, T, R, c: int, scale: float):
    """v [B][2][m/2][m/2] for images T, R [B][m][m] (float64 tensors)."""
    layers = unpack(torch.as_tensor(params, dtype=torch.float64), c)
    x = torch.stack([torch.as_tensor(T, dtype=torch.float64), torch.as_tensor(R, dtype=torch.float64)], dim=1)

    def conv(z, k, stride=1, up=False):
        w, b = layers[k]
        if up:
            z = F.interpolate(z, scale_factor=2, mode="nearest")
        return F.conv2d(z, bf16_round(w), b, stride=stride, padding=1)

    e0 = torch.relu(conv(x, 0))
    e1 = torch.relu(conv(e0, 1, 2))
    e2 = torch.relu(conv(e1, 2, 2))
    e3 = torch.relu(conv(e2, 3, 2))
    d2 = torch.relu(conv(e3, 4, up=True)) + e2
    d1 = torch.relu(conv(d2, 5, up=True)) + e1
    return scale * conv(d1, 6)


def loss_and_grad(params, T, R, v_target, c: int, scale: float):
    """Loss and its gradient with respect to the master parameters (the bf16
    rounding is treated as the identity in the backward pass)."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    layers = unpack(p, c)
    x = torch.stack([torch.as_tensor(T, dtype=torch.float64), torch.as_tensor(R, dtype=torch.float64)], dim=1)

    def conv(z, k, stride=1, up=False):
        w, b = layers[k]
        wq = w + (bf16_round(w.detach()) - w.detach())      # straight-through rounding
        if up:
            z = F.interpolate(z, scale_factor=2, mode="nearest")
        return F.conv2d(z, wq, b, stride=stride, padding=1)

    e0 = torch.relu(conv(x, 0))
    e1 = torch.relu(conv(e0, 1, 2))
    e2 = torch.relu(conv(e1, 2, 2))
    e3 = torch.relu(conv(e2, 3, 2))
    d2 = torch.relu(conv(e3, 4, up=True)) + e2
    d1 = torch.relu(conv(d2, 5, up=True)) + e1
    v = scale * conv(d1, 6)
    t = torch.as_tensor(v_target, dtype=torch.float64)
    loss = 0.5 * torch.mean((v - t) ** 2) / scale ** 2
    loss.backward()
    return float(loss.detach()), p.grad.detach().numpy(), v.detach().numpy()


def adam_step(params, grad, m, s, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected) of the master parameters."""
    m = b1 * m + (1 - b1) * grad
    s = b2 * s + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    sh = s / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(sh) + eps), m, s
