"""FP64 CPU oracle of the learned surrogate's network: forward pass, loss and
gradients, written plainly with numpy so that the GPU's BF16 tensor-core
kernels can be checked against it.

TEST INFRASTRUCTURE ONLY (tests/ and __graft_entry__.smoke() use it).

The network (a convolutional neural operator that advances the macroscopic
fields (rho, u_x, u_y, T) by K lattice steps; the paper has no such part, it
is the learned extension of the method this library builds):

    h_0     = conv_lift(x)                                   4 -> C channels
    h_{b+1} = h_b + conv_{b,2}(relu(conv_{b,1}(relu(h_b))))  b = 0 .. B-1
    y       = x + conv_proj(relu(h_B))                       C -> 4 channels

All convolutions are 3 x 3 with periodic padding (the lattice is periodic)
and a bias. Tensors are (N, H, W, C) arrays; weights are (9, Cout, Cin) with
tap t = 3 (dy + 1) + (dx + 1) reading input pixel (y + dy, x + dx).
The loss is the mean of the squared error over all pixels and the 4
channels.

With conserve_mass, a fixed output layer makes the network conserve mass
per sample: the density channel becomes y_rho - mean(y_rho - x_rho) (mean
over the image), so sum(y_rho) = sum(x_rho), as the LB update conserves
mass exactly on a periodic box (Eq. 6a). The layer is a linear projection
P, symmetric and idempotent, so the gradient passes back as P applied to
the gradient of the loss.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3x3(x, w, b):
    """out[n, y, x, o] = b[o] + sum_{t, i} x[n, y+dy_t, x+dx_t, i] w[t, o, i] (periodic)."""
    out = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, (dy, dx) in enumerate(TAPS):
        shifted = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
        out += np.einsum("nyxi,oi->nyxo", shifted, w[t])
    return out + b


def conv3x3_backward(x, w, dout):
    """Gradients of conv3x3 with respect to its input, weights and bias."""
    dx_ = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (dy, dx) in enumerate(TAPS):
        shifted = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
        dw[t] = np.einsum("nyxo,nyxi->oi", dout, shifted)
        contrib = np.einsum("nyxo,oi->nyxi", dout, w[t])
        dx_ += np.roll(contrib, shift=(dy, dx), axis=(1, 2))
    db = dout.sum(axis=(0, 1, 2))
    return dx_, dw, db


def relu(a):
    return np.maximum(a, 0.0)


def init_params(channels=64, blocks=6, cin=4, seed=0, scale=1.0):
    """Seeded He-style initial weights: {'lift': (w, b), 'blocks': [((w1, b1), (w2, b2)), ...],
    'proj': (w, b)}; the projection starts small so the initial network is
    close to the identity map."""
    rng = np.random.default_rng(seed)

    def conv(ci, co, s=1.0):
        std = s * np.sqrt(2.0 / (9 * ci))
        return rng.normal(0.0, std, size=(9, co, ci)), np.zeros(co)

    p = {"lift": conv(cin, channels, scale),
         "blocks": [(conv(channels, channels, scale), conv(channels, channels, 0.1 * scale)) for _ in range(blocks)],
         "proj": conv(channels, cin, 0.1 * scale)}
    return p


def forward(p, x, conserve_mass=False):
    """Returns the output and the cache of activations needed for backward."""
    h = conv3x3(x, *p["lift"])
    cache = {"x": x, "h": [h], "z1": []}
    for (w1, b1), (w2, b2) in p["blocks"]:
        z1 = conv3x3(relu(h), w1, b1)
        z2 = conv3x3(relu(z1), w2, b2)
        cache["z1"].append(z1)
        h = h + z2
        cache["h"].append(h)
    y = x + conv3x3(relu(h), *p["proj"])
    if conserve_mass:
        y = y.copy()
        y[..., 0] -= (y[..., 0] - x[..., 0]).mean(axis=(1, 2), keepdims=True)
    cache["conserve_mass"] = conserve_mass
    return y, cache


def loss(y, target):
    return float(np.mean((y - target) ** 2))


def backward(p, cache, y, target):
    """Gradients of the mean-squared loss with respect to every weight and bias."""
    g = {"blocks": [None] * len(p["blocks"])}
    dy = 2.0 * (y - target) / y.size
    if cache.get("conserve_mass"):
        dy[..., 0] -= dy[..., 0].mean(axis=(1, 2), keepdims=True)
    hB = cache["h"][-1]
    da, dw, db = conv3x3_backward(relu(hB), p["proj"][0], dy)
    g["proj"] = (dw, db)
    dh = da * (hB > 0)
    for k in range(len(p["blocks"]) - 1, -1, -1):
        (w1, b1), (w2, b2) = p["blocks"][k]
        h = cache["h"][k]
        z1 = cache["z1"][k]
        da2, dw2, db2 = conv3x3_backward(relu(z1), w2, dh)
        dz1 = da2 * (z1 > 0)
        da1, dw1, db1 = conv3x3_backward(relu(h), w1, dz1)
        g["blocks"][k] = ((dw1, db1), (dw2, db2))
        dh = dh + da1 * (h > 0)
    _, dw, db = conv3x3_backward(cache["x"], p["lift"][0], dh)
    g["lift"] = (dw, db)
    return g


def flatten(p):
    """All parameters in a fixed order: lift, blocks (w1, b1, w2, b2), proj."""
    out = [p["lift"][0], p["lift"][1]]
    for (w1, b1), (w2, b2) in p["blocks"]:
        out += [w1, b1, w2, b2]
    out += [p["proj"][0], p["proj"][1]]
    return out
