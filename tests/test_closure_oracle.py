"""Pins of the closure network oracle: its convolution against shifts by hand, and its
gradient against central finite differences of its loss."""
import numpy as np

from oracle import closure_oracle as C


def test_conv_taps_are_shifts_with_padding():
    X = 10
    a = np.arange(X * 3, dtype=float).reshape(X, 3) + 1.0
    for j in range(5):
        W = np.zeros((3, 5, 3))
        W[:, j, :] = np.eye(3)
        b = np.array([0.5, -1.0, 2.0])
        shift = j - 2
        zp = C.conv(a, W, b, periodic=True)
        np.testing.assert_array_equal(zp, a[(np.arange(X) + shift) % X] + b)
        zz = C.conv(a, W, b, periodic=False)
        ref = np.zeros_like(a)
        for x in range(X):
            ref[x] = a[min(max(x + shift, 0), X - 1)]
        np.testing.assert_array_equal(zz, ref + b)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shapes = C.layer_shapes(7, 5)
    n = sum(co * 5 * ci + co for ci, co in shapes)
    params = np.zeros(n)
    # real channels only: 7 inputs, 5 outputs
    layers = C.unpack(params, shapes)
    for l, (W, b) in enumerate(layers):
        cin = 7 if l == 0 else 64
        cout = 5 if l == len(layers) - 1 else 64
        W[:cout, :, :cin] = rng.normal(0, 0.15, (cout, 5, cin))
        b[:cout] = rng.normal(0, 0.05, cout)
    B, X = 2, 24
    xs = np.zeros((B, X, 16))
    xs[:, :, :7] = rng.normal(0, 1, (B, X, 7))
    ys = rng.normal(0, 0.3, (B, X, 5))
    per = [1, 0]
    loss, g = C.loss_and_grad(params, shapes, xs, ys, per, 5)
    idx = np.flatnonzero(params)
    pick = rng.choice(idx, 24, replace=False)
    # include biases of the first and last layers
    pick = np.concatenate([pick, [shapes[0][1] * 5 * 16 + 3, n - 16 + 2]])
    h = 1e-6
    for i in pick:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (C.loss_and_grad(p1, shapes, xs, ys, per, 5)[0] - C.loss_and_grad(p2, shapes, xs, ys, per, 5)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])
    # padded channels carry no gradient
    W0 = C.unpack(g, shapes)[0][0]
    assert np.all(W0[:, :, 7:] == 0)


def test_identity_network_pins_the_layer_structure_and_the_loss():
    """Centre taps set to the identity (the output layer to minus the identity), zero biases: the hidden ReLUs
    clear the negative inputs and the output layer has none, so the network gives -ReLU(x) on the real
    channels; with y = 0 the loss is the mean of ReLU(x)^2 over samples, positions and output channels."""
    shapes = C.layer_shapes(7, 5)
    n = sum(co * 5 * ci + co for ci, co in shapes)
    params = np.zeros(n)
    layers = C.unpack(params, shapes)
    for l, (W, b) in enumerate(layers):
        cout, cin = W.shape[0], W.shape[2]
        m = min(cout, cin)
        W[:m, 2, :m] = -np.eye(m) if l == len(layers) - 1 else np.eye(m)
    rng = np.random.default_rng(5)
    B, X = 3, 12
    xs = np.zeros((B, X, 16))
    xs[:, :, :7] = rng.normal(0, 1, (B, X, 7))
    for s in range(B):
        zs, acts = C.forward(params, shapes, xs[s], periodic=bool(s % 2))
        np.testing.assert_array_equal(zs[-1][:, :5], -np.maximum(xs[s, :, :5], 0.0))
        np.testing.assert_array_equal(acts[-1], zs[-1])
        assert (zs[-1][:, :5] < 0).any()
    loss, _ = C.loss_and_grad(params, shapes, xs, np.zeros((B, X, 5)), np.arange(B) % 2, 5)
    assert abs(loss - float(np.mean(np.maximum(xs[:, :, :5], 0.0) ** 2))) <= 1e-15
