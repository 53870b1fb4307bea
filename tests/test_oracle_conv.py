"""Pins of the oracle's convolution network: brute force, finite differences, Adam closed form."""
import numpy as np

import synth
from oracle import conv


def _brute_conv(x, W, b):
    ci, nz, ny, nx = x.shape
    co = W.shape[0]
    y = np.zeros((co, nz, ny, nx))
    for o in range(co):
        for z in range(nz):
            for yy in range(ny):
                for xx in range(nx):
                    s = b[o]
                    for c in range(ci):
                        for t, (dx, dy, dz) in enumerate(conv.OFFSETS):
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < nz and 0 <= y2 < ny and 0 <= x2 < nx:
                                s += W[o, c, t] * x[c, zz, y2, x2]
                    y[o, z, yy, xx] = s
    return y


def test_conv_matches_brute_force_and_special_kernels():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    assert np.abs(conv.conv(x, W, b) - _brute_conv(x, W, b)).max() < 1e-12
    # centre tap only, identity channel map -> identity
    Wi = np.zeros((3, 3, 27))
    for c in range(3):
        Wi[c, c, 13] = 1.0
    assert np.abs(conv.conv(x, Wi, np.zeros(3)) - x).max() == 0.0
    # single off-centre tap -> shift with zero padding
    Ws = np.zeros((1, 1, 27))
    Ws[0, 0, conv.OFFSETS.index((1, 0, -1))] = 1.0
    ys = conv.conv(x[:1], Ws, np.zeros(1))[0]
    assert np.allclose(ys[1:, :, :-1], x[0, :-1, :, 1:]) and np.all(ys[0] == 0) and np.all(ys[:, :, -1] == 0)


def test_network_gradients_match_central_differences():
    W, b = synth.conv_net_init((3, 4, 4, 2), seed=3, last_scale=1.0)
    b = [np.random.default_rng(7 + i).standard_normal(len(v)) * 0.1 for i, v in enumerate(b)]
    net = conv.Net(W, b)
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal((3, 4, 4, 5))
    target = rng.standard_normal((2, 4, 4, 5))
    mask = np.ones((4, 4, 5), bool)
    mask[0] = False
    loss, gW, gb = net.loss_and_grads(x0, target, mask)
    h = 1e-6
    for l in range(len(W)):
        for idx in [(0, 0, 13), (1, 2, 0), (W[l].shape[0] - 1, W[l].shape[1] - 1, 26)]:
            saved = net.W[l][idx]
            net.W[l][idx] = saved + h
            lp = net.loss_and_grads(x0, target, mask)[0]
            net.W[l][idx] = saved - h
            lm = net.loss_and_grads(x0, target, mask)[0]
            net.W[l][idx] = saved
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gW[l][idx]) < 1e-6 * max(1.0, abs(fd)), (l, idx, fd, gW[l][idx])
        saved = net.b[l][0]
        net.b[l][0] = saved + h
        lp = net.loss_and_grads(x0, target, mask)[0]
        net.b[l][0] = saved - h
        lm = net.loss_and_grads(x0, target, mask)[0]
        net.b[l][0] = saved
        assert abs((lp - lm) / (2 * h) - gb[l][0]) < 1e-6


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -4.0])]
    opt = conv.Adam(p, lr=0.1)
    out = opt.step(p, g)
    # first step: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (up to eps)
    assert np.allclose(out[0], p[0] - 0.1 * np.sign(g[0]), atol=1e-7)
