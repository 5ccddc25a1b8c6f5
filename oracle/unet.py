"""Plain FP64 CPU oracle of the learned warm start's network: a 3-D U-Net with
3x3x3 convolutions, its backward pass, a masked mean-squared loss and Adam.

TEST INFRASTRUCTURE ONLY: the test suite and the benchmark's CPU-baseline leg
are the only users. Nothing here is shared with the CUDA library: the layer
table below is written independently of the library's own, and both sides take
their seeded weights and inputs from ``paper_2606_05893_gb300.unet_inputs``
(random numbers only).

The network supplies the initial guess of the Krylov solve of Eq. (1). Its
shape is four resolution levels with 16/32/64/128 channels, two 3x3x3
convolutions with ReLU per level, 2x2x2 average pooling on the way down,
nearest-neighbour upsampling by 2 and channel concatenation [upsampled, skip]
on the way up, and a 1x1x1 convolution to one output channel. There are no
biases, so the network is positively homogeneous: f(a x) = a f(x) for a > 0,
which lets a caller normalise each input by a scalar and scale the output back.

Every operation is its textbook definition written out in numpy FP64: a
convolution is the sum over its 27 taps of a channel contraction of the
zero-padded input shifted by the tap; pooling is the mean of each 2x2x2 block;
upsampling copies each voxel to its 2x2x2 block; Adam follows Kingma and Ba
(2015, Algorithm 1) with bias correction. Tensors are (C, D, H, W), batch 1.
"""
from __future__ import annotations

import numpy as np

# (name, input channels, output channels) of the 3x3x3 convolutions, in
# forward order; "out" is the final 1x1x1 convolution.
CH = (16, 32, 64, 128)
IN_CHANNELS = 2
LAYERS = (
    ("e0a", IN_CHANNELS, 16), ("e0b", 16, 16),
    ("e1a", 16, 32), ("e1b", 32, 32),
    ("e2a", 32, 64), ("e2b", 64, 64),
    ("e3a", 64, 128), ("e3b", 128, 128),
    ("d2a", 128 + 64, 64), ("d2b", 64, 64),
    ("d1a", 64 + 32, 32), ("d1b", 32, 32),
    ("d0a", 32 + 16, 16), ("d0b", 16, 16),
)
OUT = ("out", 16, 1)


def weight_shapes():
    """Shapes of every weight, in the order of LAYERS then OUT."""
    return [(co, ci, 3, 3, 3) for _, ci, co in LAYERS] + [(OUT[2], OUT[1])]


# ----------------------------------------------------------------------------
# operations and their derivatives
# ----------------------------------------------------------------------------
TAPS = [(a, b, c) for a in range(3) for b in range(3) for c in range(3)]


def conv3x3(x, w):
    """y[o, z, y, x] = sum_{i, a, b, c} w[o, i, a, b, c] x[i, z+a-1, y+b-1, x+c-1],
    zero outside the volume."""
    ci, D, H, W = x.shape
    xp = np.zeros((ci, D + 2, H + 2, W + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], D, H, W))
    for a, b, c in TAPS:
        y += np.einsum("oi,idhw->odhw", w[:, :, a, b, c], xp[:, a:a + D, b:b + H, c:c + W], optimize=True)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of sum(dy * conv3x3(x, w)) with respect to x and w."""
    ci, D, H, W = x.shape
    xp = np.zeros((ci, D + 2, H + 2, W + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for a, b, c in TAPS:
        sl = (slice(None), slice(a, a + D), slice(b, b + H), slice(c, c + W))
        dxp[sl] += np.einsum("oi,odhw->idhw", w[:, :, a, b, c], dy, optimize=True)
        dw[:, :, a, b, c] = np.einsum("odhw,idhw->oi", dy, xp[sl], optimize=True)
    return dxp[:, 1:-1, 1:-1, 1:-1].copy(), dw


def conv1x1(x, w):
    return np.einsum("oi,idhw->odhw", w, x, optimize=True)


def conv1x1_backward(x, w, dy):
    return np.einsum("oi,odhw->idhw", w, dy, optimize=True), np.einsum("odhw,idhw->oi", dy, x, optimize=True)


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    c, D, H, W = x.shape
    return x.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample2_backward(dy):
    c, D, H, W = dy.shape
    return dy.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


# ----------------------------------------------------------------------------
# the network
# ----------------------------------------------------------------------------
def _keep(a):
    return a


def forward(params, x, rnd=None):
    """params: dict name -> weight (LAYERS and OUT); x: (IN_CHANNELS, D, H, W) with
    D, H, W multiples of 8. Returns (y of shape (1, D, H, W), cache).

    rnd (default: none) is applied to every stored activation (each ReLU output
    and each pooled tensor): a caller that stores activations in a narrower
    format passes its rounding here, so that both sides take the ReLU decisions
    on the same values. The arithmetic between those points stays FP64."""
    rnd = rnd or _keep
    cache = {"x": x}

    def block(name_a, name_b, inp):
        za = conv3x3(inp, params[name_a])
        ya = rnd(relu(za))
        zb = conv3x3(ya, params[name_b])
        yb = rnd(relu(zb))
        cache[name_a] = (inp, ya)
        cache[name_b] = (ya, yb)
        return yb

    e0 = block("e0a", "e0b", x)
    e1 = block("e1a", "e1b", rnd(avgpool2(e0)))
    e2 = block("e2a", "e2b", rnd(avgpool2(e1)))
    e3 = block("e3a", "e3b", rnd(avgpool2(e2)))
    d2 = block("d2a", "d2b", np.concatenate([upsample2(e3), e2]))
    d1 = block("d1a", "d1b", np.concatenate([upsample2(d2), e1]))
    d0 = block("d0a", "d0b", np.concatenate([upsample2(d1), e0]))
    cache["out"] = d0
    return conv1x1(d0, params["out"]), cache


def backward(params, cache, dy, rnd=None):
    """Gradients of sum(dy * forward(params, x)) for every weight, and for x.

    rnd (default: none) is applied to every stored activation gradient (the
    gradient at each convolution's output after its ReLU mask, at each
    convolution's input, and after each adjoint upsampling); weight gradients
    are never rounded."""
    rnd = rnd or _keep
    g = {}
    dd0, g["out"] = conv1x1_backward(cache["out"], params["out"], dy)

    def block_back(name_a, name_b, dout):
        ya, yb = cache[name_b]
        dzb = rnd(dout * (yb > 0))
        dya, g[name_b] = conv3x3_backward(ya, params[name_b], dzb)
        inp, ya2 = cache[name_a]
        dza = rnd(dya * (ya2 > 0))
        dinp, g[name_a] = conv3x3_backward(inp, params[name_a], dza)
        return rnd(dinp)

    c3, c2, c1 = CH[3], CH[2], CH[1]
    dcat0 = block_back("d0a", "d0b", dd0)
    dd1, de0 = rnd(upsample2_backward(dcat0[:c1])), dcat0[c1:]
    dcat1 = block_back("d1a", "d1b", dd1)
    dd2, de1 = rnd(upsample2_backward(dcat1[:c2])), dcat1[c2:]
    dcat2 = block_back("d2a", "d2b", dd2)
    de3, de2 = rnd(upsample2_backward(dcat2[:c3])), dcat2[c3:]
    dp3 = block_back("e3a", "e3b", de3)
    de2 = de2 + avgpool2_backward(dp3)
    dp2 = block_back("e2a", "e2b", de2)
    de1 = de1 + avgpool2_backward(dp2)
    dp1 = block_back("e1a", "e1b", de1)
    de0 = de0 + avgpool2_backward(dp1)
    dx = block_back("e0a", "e0b", de0)
    return g, dx


def mse_loss(y, t, mask=None):
    """L = mean over the masked voxels of (y - t)^2, and dL/dy."""
    if mask is None:
        mask = np.ones(y.shape, dtype=bool)
    n = int(mask.sum())
    d = np.where(mask, y - t, 0.0)
    return float((d * d).sum() / n), 2.0 * d / n


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba, Algorithm 1), in place."""
    for k in params:
        m[k] = beta1 * m[k] + (1.0 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * grads[k] * grads[k]
        mhat = m[k] / (1.0 - beta1 ** t)
        vhat = v[k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params, m, v


def names():
    return [n for n, _, _ in LAYERS] + [OUT[0]]


# ----------------------------------------------------------------------------
# the loss the warm start is trained on: the residual it leaves
# ----------------------------------------------------------------------------
def apply_A(y):
    """The scaled 7-point operator of Eq. (1) on a (1, D, H, W) network volume whose
    planes d = 0..D-2 are the unknown node planes k = d + 1 and whose last plane
    lies on the anode: periodic in x (W) and y (H), zero Dirichlet values on the
    cathode plane (d = -1) and the anode plane (d = D - 1). The last plane of the
    result is 0."""
    z = np.array(y, dtype=np.float64, copy=True)
    z[:, -1] = 0.0
    a = 6.0 * z - np.roll(z, 1, 3) - np.roll(z, -1, 3) - np.roll(z, 1, 2) - np.roll(z, -1, 2)
    a[:, 1:] -= z[:, :-1]
    a[:, :-1] -= z[:, 1:]
    a[:, -1] = 0.0
    return a


def residual_loss(y, r):
    """L = mean over the unknown planes of (r - A y)^2, the squared residual that
    the initial guess y leaves for the right-hand side r (both scaled by the same
    s), and dL/dy = -(2 / n) A (r - A y) (A is symmetric)."""
    e = np.array(r, dtype=np.float64, copy=True) - apply_A(y)
    e[:, -1] = 0.0
    n = e[:, :-1].size
    return float((e * e).sum() / n), -2.0 / n * apply_A(e)
