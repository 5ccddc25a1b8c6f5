"""Pins of the FP64 U-Net oracle (oracle/unet.py) against what does not come
from it: torch's FP64 CPU conv3d, pooling and interpolation (library routines)
and their autograd derivatives, an independently written torch network of the
same architecture, central finite differences, positive homogeneity of a
bias-free ReLU network, and torch's Adam."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet as U
from paper_2606_05893_gb300 import unet_inputs as I



def T(a):
    return torch.from_numpy(np.ascontiguousarray(a))


def test_conv3x3_forward_and_backward_match_torch():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 6, 5, 7))
    w = rng.standard_normal((5, 3, 3, 3, 3))
    dy = rng.standard_normal((5, 6, 5, 7))
    y = U.conv3x3(x, w)
    xt, wt = T(x).requires_grad_(), T(w).requires_grad_()
    yt = F.conv3d(xt[None], wt, padding=1)[0]
    assert np.abs(y - yt.detach().numpy()).max() <= 1e-12 * np.abs(y).max()
    (yt * T(dy)).sum().backward()
    dx, dw = U.conv3x3_backward(x, w, dy)
    assert np.abs(dx - xt.grad.numpy()).max() <= 1e-12 * np.abs(dx).max()
    assert np.abs(dw - wt.grad.numpy()).max() <= 1e-12 * np.abs(dw).max()


def test_conv1x1_pool_upsample_match_torch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 4, 8))
    w = rng.standard_normal((2, 4))
    dy = rng.standard_normal((2, 6, 4, 8))
    xt, wt = T(x).requires_grad_(), T(w).requires_grad_()
    yt = F.conv3d(xt[None], wt[:, :, None, None, None])[0]
    assert np.allclose(U.conv1x1(x, w), yt.detach().numpy(), rtol=0, atol=1e-13)
    (yt * T(dy)).sum().backward()
    dx, dw = U.conv1x1_backward(x, w, dy)
    assert np.allclose(dx, xt.grad.numpy(), rtol=0, atol=1e-13)
    assert np.allclose(dw, wt.grad.numpy(), rtol=0, atol=1e-12)
    # pooling and upsampling and their adjoints
    xt = T(x).requires_grad_()
    pt = F.avg_pool3d(xt[None], 2)[0]
    assert np.allclose(U.avgpool2(x), pt.detach().numpy(), rtol=0, atol=1e-14)
    dp = rng.standard_normal(pt.shape)
    (pt * T(dp)).sum().backward()
    assert np.allclose(U.avgpool2_backward(dp), xt.grad.numpy(), rtol=0, atol=1e-14)
    xt = T(x).requires_grad_()
    ut = F.interpolate(xt[None], scale_factor=2, mode="nearest")[0]
    assert np.array_equal(U.upsample2(x), ut.detach().numpy())
    du = rng.standard_normal(ut.shape)
    (ut * T(du)).sum().backward()
    assert np.allclose(U.upsample2_backward(du), xt.grad.numpy(), rtol=0, atol=1e-13)


def torch_unet(ws, x):
    """The architecture written again with torch ops: two 3x3x3 conv + ReLU per
    level, 16/32/64/128 channels, 2x2x2 average pooling down, nearest x2
    upsampling and concatenation [upsampled, skip] up, a 1x1x1 output conv."""
    def conv(t, w):
        return F.conv3d(t, w, padding=1)

    it = iter(ws)

    def block(t):
        return torch.relu(conv(torch.relu(conv(t, next(it))), next(it)))

    e0 = block(x[None])
    e1 = block(F.avg_pool3d(e0, 2))
    e2 = block(F.avg_pool3d(e1, 2))
    e3 = block(F.avg_pool3d(e2, 2))
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")  # noqa: E731
    d2 = block(torch.cat([up(e3), e2], 1))
    d1 = block(torch.cat([up(d2), e1], 1))
    d0 = block(torch.cat([up(d1), e0], 1))
    wo = next(it)
    return F.conv3d(d0, wo[:, :, None, None, None])[0]


def params_from(ws):
    return dict(zip(U.names(), ws))


def test_unet_forward_backward_match_torch_network():
    ws = I.init_weights(U.weight_shapes(), seed=3)
    x = I.random_volume(U.IN_CHANNELS, 16, 8, 8, seed=4, smooth=1)
    p = params_from(ws)
    y, cache = U.forward(p, x)
    wt = [T(w).requires_grad_() for w in ws]
    xt = T(x).requires_grad_()
    yt = torch_unet(wt, xt)
    assert y.shape == (1, 16, 8, 8)
    assert np.abs(y - yt.detach().numpy()).max() <= 1e-12 * np.abs(y).max()
    dy = np.random.default_rng(5).standard_normal(y.shape)
    (yt * T(dy)).sum().backward()
    g, dx = U.backward(p, cache, dy)
    for name, w in zip(U.names(), wt):
        ref = w.grad.numpy()
        assert np.abs(g[name] - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1e-300), name
    assert np.abs(dx - xt.grad.numpy()).max() <= 1e-11 * np.abs(dx).max()


def test_unet_gradients_by_central_differences():
    ws = I.init_weights(U.weight_shapes(), seed=6)
    x = I.random_volume(U.IN_CHANNELS, 8, 8, 8, seed=7)
    t = I.random_volume(1, 8, 8, 8, seed=8)
    mask = np.ones(t.shape, dtype=bool)
    mask[:, -1] = False  # the last plane is left out of the loss
    p = params_from(ws)

    def loss(pp, xx):
        return U.mse_loss(U.forward(pp, xx)[0], t, mask)[0]

    y, cache = U.forward(p, x)
    L, dy = U.mse_loss(y, t, mask)
    g, dx = U.backward(p, cache, dy)
    rng = np.random.default_rng(9)
    eps = 1e-5
    # central differences: truncation O(eps^2) plus rounding about ulp(L) / eps
    fd_round = 20.0 * np.finfo(float).eps * abs(L) / eps
    for name in ("e0a", "e1b", "e3b", "d2a", "d0a", "d0b", "out"):
        for _ in range(3):
            idx = tuple(int(rng.integers(0, s)) for s in p[name].shape)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += eps
            lp = loss(q, x)
            q[name][idx] -= 2 * eps
            lm = loss(q, x)
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name][idx]) <= 1e-6 * abs(fd) + fd_round, (name, idx, fd, g[name][idx])
    for _ in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (loss(p, xp) - loss(p, xm)) / (2 * eps)
        assert abs(fd - dx[idx]) <= 1e-6 * abs(fd) + fd_round, (idx, fd, dx[idx])


def test_unet_is_positively_homogeneous():
    ws = I.init_weights(U.weight_shapes(), seed=10)
    p = params_from(ws)
    x = I.random_volume(U.IN_CHANNELS, 8, 16, 8, seed=11)
    y1 = U.forward(p, x)[0]
    y2 = U.forward(p, 3.7 * x)[0]
    assert np.abs(y2 - 3.7 * y1).max() <= 1e-12 * np.abs(y2).max()


def test_adam_matches_torch():
    rng = np.random.default_rng(12)
    p = {"a": rng.standard_normal((3, 4)), "b": rng.standard_normal(5)}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    tp = {k: T(a.copy()).requires_grad_() for k, a in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 5):
        g = {k: rng.standard_normal(a.shape) for k, a in p.items()}
        p, m, v = U.adam_step(p, g, m, v, t, 1e-2)
        opt.zero_grad()
        for k in tp:
            tp[k].grad = T(g[k])
        opt.step()
        for k in p:
            assert np.abs(p[k] - tp[k].detach().numpy()).max() <= 1e-14
    # the first step moves every weight by lr against the sign of its gradient
    q = {"a": np.ones(3)}
    g = {"a": np.array([2.0, -0.5, 1e-3])}
    U.adam_step(q, g, {"a": np.zeros(3)}, {"a": np.zeros(3)}, 1, 0.1)
    assert np.allclose(q["a"], 1.0 - 0.1 * np.sign(g["a"]), rtol=0, atol=1e-6)


def test_mse_loss_gradient():
    rng = np.random.default_rng(13)
    y, t = rng.standard_normal((1, 4, 4, 4)), rng.standard_normal((1, 4, 4, 4))
    mask = rng.random(y.shape) > 0.3
    L, dy = U.mse_loss(y, t, mask)
    assert L == pytest.approx(((y - t)[mask] ** 2).mean(), rel=1e-14)
    eps = 1e-7
    for idx in [(0, 1, 2, 3), (0, 0, 0, 0), (0, 3, 1, 2)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += eps
        ym[idx] -= eps
        fd = (U.mse_loss(yp, t, mask)[0] - U.mse_loss(ym, t, mask)[0]) / (2 * eps)
        assert abs(fd - dy[idx]) <= 1e-7


def test_library_architecture_table_matches_the_oracle():
    """The library's layer table is written separately from the oracle's: same
    layers, same shapes, same flat weight count."""
    import paper_2606_05893_gb300 as pkg
    assert [n for n, _, _ in pkg.UNET_LAYERS] == [n for n, _, _ in U.LAYERS]
    assert [tuple(s) for s in pkg.UNET_WEIGHT_SHAPES] == [tuple(s) for s in U.weight_shapes()]


def test_operator_eigenfunction_and_residual_loss_gradient():
    """A sin(pi m (d+1) / D) cos(2 pi k x / W) cos(2 pi l y / H) = (6 - 2 cos(pi m / D)
    - 2 cos(2 pi k / W) - 2 cos(2 pi l / H)) times the same on the unknown planes
    (the discrete Dirichlet-periodic eigenfunctions); the residual loss's gradient
    by central differences."""
    D, H, W = 8, 6, 10
    d = np.arange(D)[:, None, None]
    yy = np.arange(H)[None, :, None]
    xx = np.arange(W)[None, None, :]
    for m, k, l in [(1, 0, 0), (3, 2, 1), (7, 5, 3)]:
        f = np.sin(np.pi * m * (d + 1) / D) * np.cos(2 * np.pi * k * xx / W) * np.cos(2 * np.pi * l * yy / H)
        lam = 6 - 2 * np.cos(np.pi * m / D) - 2 * np.cos(2 * np.pi * k / W) - 2 * np.cos(2 * np.pi * l / H)
        Af = U.apply_A(f[None])[0]
        assert np.abs(Af[:-1] - lam * f[:-1]).max() <= 1e-13 and not Af[-1].any()
    rng = np.random.default_rng(14)
    y, r = rng.standard_normal((1, D, H, W)), rng.standard_normal((1, D, H, W))
    L, dy = U.residual_loss(y, r)
    e = r - U.apply_A(y)
    assert L == pytest.approx((e[:, :-1] ** 2).mean(), rel=1e-14)
    assert not dy[:, -1].any()
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (0, 3, 2, 7), (0, 6, 5, 9), (0, 7, 1, 1)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += eps
        ym[idx] -= eps
        fd = (U.residual_loss(yp, r)[0] - U.residual_loss(ym, r)[0]) / (2 * eps)
        assert abs(fd - dy[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, dy[idx])
