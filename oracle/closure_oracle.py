"""FP64 CPU oracle of the learned coarse-grid closure network.

TEST INFRASTRUCTURE ONLY: used by tests/ to check the GPU training kernels.  It
restates the network from its definition with numpy in double precision: 1D
convolutions of kernel 5 (tap j reads position x + j - 2; beyond the ends,
periodic images or the end values repeated), ReLU between layers and none on
the output, mean squared error, and the gradients of that loss written out by
the chain rule.  Pinned (tests/test_closure_oracle.py): each tap against a
shift by hand under both paddings, the layer structure and the loss against an
identity network whose output is -ReLU of its input, and the gradient against
central finite differences of the loss.

Parameter vector layout (as ql_closure_params): for each layer W[cout][5][cin]
then bias[cout], channel counts padded to 16 (padding zero).
"""
from __future__ import annotations

import numpy as np

TAPS = 5


def layer_shapes(in_channels: int, out_channels: int, layers: int = 5, width: int = 64):
    """Padded (cin, cout) of each layer."""
    shapes = []
    for l in range(layers):
        cin = 16 if l == 0 else width
        cout = 16 if l == layers - 1 else width
        shapes.append((cin, cout))
    return shapes


def unpack(params: np.ndarray, shapes):
    out, off = [], 0
    for cin, cout in shapes:
        W = params[off:off + cout * TAPS * cin].reshape(cout, TAPS, cin)
        off += cout * TAPS * cin
        b = params[off:off + cout]
        off += cout
        out.append((W, b))
    assert off == len(params)
    return out


def _window(a: np.ndarray, periodic: bool) -> np.ndarray:
    """a [X][C] -> positions -2 .. X+1 (periodic images, else copies of the end values)."""
    X = a.shape[0]
    idx = np.arange(-2, X + 2)
    if periodic:
        return a[idx % X]
    return a[np.clip(idx, 0, X - 1)]


def conv(a: np.ndarray, W: np.ndarray, b: np.ndarray, periodic: bool) -> np.ndarray:
    """z[x][co] = b[co] + sum_j sum_ci W[co][j][ci] a[x + j - 2][ci]."""
    X = a.shape[0]
    w = _window(a, periodic)
    z = np.tile(b, (X, 1)).astype(np.float64)
    for j in range(TAPS):
        z += w[j:j + X] @ W[:, j, :].T
    return z


def forward(params, shapes, x: np.ndarray, periodic: bool):
    """x [X][cin_padded] (normalised inputs); returns pre-activations and activations per layer."""
    layers = unpack(params, shapes)
    acts, zs = [x], []
    a = x
    for l, (W, b) in enumerate(layers):
        z = conv(a, W, b, periodic)
        zs.append(z)
        a = np.maximum(z, 0.0) if l < len(layers) - 1 else z
        acts.append(a)
    return zs, acts


def loss_and_grad(params, shapes, xs, ys, periodic, out_channels: int):
    """Mean over samples, positions and the first out_channels outputs of (pred - y)^2,
    and its gradient with respect to params.  xs [B][X][cin_padded], ys [B][X][out_channels]."""
    layers = unpack(params, shapes)
    grad = np.zeros_like(params)
    gl = unpack(grad, shapes)  # views into grad
    B, X = xs.shape[0], xs.shape[1]
    nel = B * X * out_channels
    total = 0.0
    for s in range(B):
        zs, acts = forward(params, shapes, xs[s], bool(periodic[s]))
        pred = zs[-1]
        d = np.zeros_like(pred)
        d[:, :out_channels] = pred[:, :out_channels] - ys[s]
        total += float(np.sum(d[:, :out_channels] ** 2))
        dz = 2.0 * d / nel
        for l in range(len(layers) - 1, -1, -1):
            W, _ = layers[l]
            gW, gb = gl[l]
            a_in = acts[l]
            w = _window(a_in, bool(periodic[s]))
            for j in range(TAPS):
                gW[:, j, :] += dz.T @ w[j:j + X]
            gb += dz.sum(axis=0)
            if l == 0:
                break
            # gradient with respect to the window of the input, folded back onto positions
            dw = np.zeros((X + 4, W.shape[2]))
            for j in range(TAPS):
                dw[j:j + X] += dz @ W[:, j, :]
            da = dw[2:X + 2].copy()
            if periodic[s]:
                da[X - 2:] += dw[0:2]
                da[:2] += dw[X + 2:X + 4]
            else:
                da[0] += dw[0] + dw[1]
                da[X - 1] += dw[X + 2] + dw[X + 3]
            dz = da * (zs[l - 1] > 0.0)
    return total / nel, grad
