"""Direct 3D convolution network for the learned initial guess, FP64.

Test infrastructure (see oracle/__init__.py).  The paper has no learned component; this
is the plain definition of the network the GPU path trains (fields on the node grid):

  x_0 = input features, channels-first (C_0, nz, ny, nx)
  y_l = conv3x3x3(x_{l-1}, W_l) + b_l,   x_l = relu(y_l) for l < L,   output = y_L
  conv(x, W)[co, v] = sum_ci sum_{tap} W[co, ci, tap] x[ci, v + off(tap)],  zero padding,
  tap = (dx+1) + 3 (dy+1) + 9 (dz+1),  off(tap) = (dx, dy, dz) in {-1, 0, 1}^3
  loss = mean over unmasked voxels and output channels of (output - target)^2
  Adam (Kingma & Ba 2015) with bias correction.

Pins (tests/test_oracle_conv.py): identity and shift kernels against brute force, all
gradients against central finite differences, one Adam step against its closed form.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x: np.ndarray, off) -> np.ndarray:
    """s[..., z, y, x] = x[..., z+dz, y+dy, x+dx], zero outside the grid."""
    dx, dy, dz = off
    nz, ny, nx = x.shape[-3:]
    out = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), nz - max(0, dz)), slice(max(0, -dy), ny - max(0, dy)), slice(max(0, -dx), nx - max(0, dx))
    zt, yt, xt = slice(max(0, dz), nz - max(0, -dz)), slice(max(0, dy), ny - max(0, -dy)), slice(max(0, dx), nx - max(0, -dx))
    out[..., zs, ys, xs] = x[..., zt, yt, xt]
    return out


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (Ci, nz, ny, nx), W (Co, Ci, 27), b (Co,)."""
    y = np.zeros((W.shape[0],) + x.shape[1:])
    for t, off in enumerate(OFFSETS):
        y += np.einsum("oc,czyx->ozyx", W[:, :, t], shift(x, off))
    return y + b[:, None, None, None]


def conv_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of conv with respect to x, W and b, given dy = dL/dy."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for t, off in enumerate(OFFSETS):
        dW[:, :, t] = np.einsum("ozyx,czyx->oc", dy, shift(x, off))
        # y[v] uses x[v + off]  =>  dx[v] collects dy[v - off]
        dx += np.einsum("oc,ozyx->czyx", W[:, :, t], shift(dy, (-off[0], -off[1], -off[2])))
    db = dy.sum(axis=(1, 2, 3))
    return dx, dW, db


class Net:
    def __init__(self, weights, biases):
        self.W = [np.asarray(w, np.float64) for w in weights]
        self.b = [np.asarray(b, np.float64) for b in biases]

    def forward(self, x0):
        xs, ys = [x0], []
        x = x0
        for l, (W, b) in enumerate(zip(self.W, self.b)):
            y = conv(x, W, b)
            ys.append(y)
            x = np.maximum(y, 0.0) if l < len(self.W) - 1 else y
            xs.append(x)
        return xs[-1], (xs, ys)

    def loss_and_grads(self, x0, target, mask):
        """mask: (nz, ny, nx) bool of voxels that count; mean over mask x output channels."""
        out, (xs, ys) = self.forward(x0)
        count = mask.sum() * out.shape[0]
        diff = (out - target) * mask[None]
        loss = float((diff ** 2).sum() / count)
        dy = 2.0 * diff / count
        gW, gb = [None] * len(self.W), [None] * len(self.W)
        for l in reversed(range(len(self.W))):
            dx, gW[l], gb[l] = conv_backward(xs[l], self.W[l], dy)
            if l > 0:
                dy = dx * (ys[l - 1] > 0.0)
        return loss, gW, gb


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            out.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out
