"""Learned closure kernels: forward and gradients against the FP64 network oracle, training
progress, and the gain of the trained network over the coarse solve on held-out pairs."""
import numpy as np
import pytest

from oracle import closure_oracle as CO

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.tensor(a, dtype=torch.float32).bfloat16().float().numpy().astype(np.float64)


def _setup(q, B=3, X=64, seed=1):
    import torch
    rng = np.random.default_rng(seed)
    net = q.Closure(7, 5, X, B, seed=seed)
    shapes = CO.layer_shapes(7, 5)
    p = net.get_params().astype(np.float64)
    layers = CO.unpack(p, shapes)
    for l, (W, b) in enumerate(layers):
        cout = 5 if l == len(layers) - 1 else 64
        b[:cout] = rng.normal(0, 0.05, cout)
    net.set_params(p.astype(np.float32))
    x = rng.normal(0, 1, (B, X, 7)).astype(np.float32)
    y = rng.normal(0, 0.5, (B, X, 5)).astype(np.float32)
    per = np.array([1, 0, 1][:B], dtype=np.int32)
    dev = torch.device("cuda", 0)
    return net, shapes, p, x, y, per, [torch.tensor(a, device=dev) for a in (x, y, per)]


def _oracle_params(p, shapes):
    """The GPU multiplies bf16 weights and keeps f32 biases."""
    q_ = p.copy()
    for W, b in CO.unpack(q_, shapes):
        W[...] = _bf16(W)
    return q_


def test_forward_matches_oracle(gpu):
    import torch
    net, shapes, p, x, y, per, (xd, yd, pd) = _setup(gpu)
    out = torch.empty(x.shape[0], x.shape[1], 5, device=xd.device)
    net.forward(xd, pd, out)
    po = _oracle_params(p, shapes)
    got = out.cpu().numpy()
    for s in range(x.shape[0]):
        xin = np.zeros((x.shape[1], 16))
        xin[:, :7] = _bf16(x[s])
        zs, _ = CO.forward(po, shapes, xin, bool(per[s]))
        ref = zs[-1][:, :5]
        assert np.abs(got[s] - ref).max() <= 3e-2 * np.abs(ref).max() + 1e-4


def test_gradients_match_oracle(gpu):
    net, shapes, p, x, y, per, (xd, yd, pd) = _setup(gpu)
    loss, g = net.gradients(xd, yd, pd)
    po = _oracle_params(p, shapes)
    xin = np.zeros((x.shape[0], x.shape[1], 16))
    xin[:, :, :7] = _bf16(x)
    lo, go = CO.loss_and_grad(po, shapes, xin, y.astype(np.float64), per, 5)
    assert loss == pytest.approx(lo, rel=2e-2)
    g = g.astype(np.float64)
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert rel <= 5e-2 and cos >= 0.998, (rel, cos)
    # each layer separately
    for (Wg, bg), (Wo, bo) in zip(CO.unpack(g, shapes), CO.unpack(go, shapes)):
        assert np.linalg.norm(Wg - Wo) <= 8e-2 * np.linalg.norm(Wo) + 1e-9
        assert np.linalg.norm(bg - bo) <= 8e-2 * np.linalg.norm(bo) + 1e-9


@pytest.mark.parametrize("X", [100, 200])
def test_gradients_match_oracle_ragged_tiles(gpu, X):
    """Sample lengths that are not a multiple of the 64-position tile (one and several tiles)."""
    net, shapes, p, x, y, per, (xd, yd, pd) = _setup(gpu, B=3, X=X, seed=2)
    loss, g = net.gradients(xd, yd, pd)
    po = _oracle_params(p, shapes)
    xin = np.zeros((x.shape[0], X, 16))
    xin[:, :, :7] = _bf16(x)
    lo, go = CO.loss_and_grad(po, shapes, xin, y.astype(np.float64), per, 5)
    g = g.astype(np.float64)
    assert loss == pytest.approx(lo, rel=2e-2)
    assert np.linalg.norm(g - go) <= 5e-2 * np.linalg.norm(go)


def test_gradients_at_replicated_ends(gpu):
    """Loss concentrated on the two end positions at each side of a replicate-padded sample, so
    that the gradient is carried by the taps that reach past the ends."""
    import torch
    q = gpu
    rng = np.random.default_rng(4)
    X = 100
    net = q.Closure(7, 5, X, 1, seed=4)
    shapes = CO.layer_shapes(7, 5)
    p = net.get_params().astype(np.float64)
    po = _oracle_params(p, shapes)
    x = rng.normal(0, 1, (1, X, 7)).astype(np.float32)
    xin = np.zeros((1, X, 16))
    xin[:, :, :7] = _bf16(x)
    zs, _ = CO.forward(po, shapes, xin[0], False)
    y = zs[-1][:, :5].copy()
    y[[0, 1, X - 2, X - 1]] += rng.normal(0, 1.0, (4, 5))
    y = y[None].astype(np.float32)
    per = np.zeros(1, dtype=np.int32)
    dev = torch.device("cuda", 0)
    loss, g = net.gradients(*(torch.tensor(a, device=dev) for a in (x, y, per)))
    lo, go = CO.loss_and_grad(po, shapes, xin, y.astype(np.float64), per, 5)
    g = g.astype(np.float64)
    for (Wg, _), (Wo, _) in zip(CO.unpack(g, shapes), CO.unpack(go, shapes)):
        assert np.linalg.norm(Wg - Wo) <= 5e-2 * np.linalg.norm(Wo), np.linalg.norm(Wg - Wo) / np.linalg.norm(Wo)


def test_training_reduces_a_regression_loss(gpu):
    import torch
    q = gpu
    rng = np.random.default_rng(3)
    B, X = 64, 128
    xs = rng.normal(0, 1, (B, X, 7)).astype(np.float32)
    # target: a smooth local function of the inputs (a 3-point average of two channels)
    ys = np.zeros((B, X, 5), dtype=np.float32)
    sm = (np.roll(xs, 1, 1) + xs + np.roll(xs, -1, 1)) / 3.0
    ys[:, :, 0] = sm[:, :, 0] * sm[:, :, 1]
    ys[:, :, 1] = np.tanh(sm[:, :, 2])
    dev = torch.device("cuda", 0)
    xd, yd = torch.tensor(xs, device=dev), torch.tensor(ys, device=dev)
    pd = torch.ones(B, dtype=torch.int32, device=dev)
    net = q.Closure(7, 5, X, 16, seed=5)
    first = None
    for it in range(300):
        i = (it * 16) % B
        l = net.train_step(xd[i:i + 16].contiguous(), yd[i:i + 16].contiguous(), pd[i:i + 16].contiguous(), 2e-3,
                           want_loss=True)
        first = first if first is not None else l
    assert l < 0.2 * first, (first, l)


def test_device_training_loop_equals_single_steps(gpu):
    """ql_closure_train_steps (mini-batches gathered on the device from a permutation, one call for many
    steps) gives bitwise the parameters and losses of ql_closure_train_step on the same batches gathered by
    the caller, with a ragged data set (n not a multiple of B) and mixed padding kinds."""
    import torch
    q = gpu
    rng = np.random.default_rng(11)
    n, B, X, steps = 45, 8, 96, 5
    dev = torch.device("cuda", 0)
    xd = torch.tensor(rng.normal(0, 1, (n, X, 7)).astype(np.float32), device=dev)
    yd = torch.tensor(rng.normal(0, 0.5, (n, X, 5)).astype(np.float32), device=dev)
    pd = torch.tensor(rng.integers(0, 2, n).astype(np.int32), device=dev)
    perm = torch.tensor(rng.permutation(n)[:steps * B].astype(np.int32), device=dev)
    rates = np.linspace(2e-3, 1e-3, steps).astype(np.float32)
    a = q.Closure(7, 5, X, B, seed=9)
    b = q.Closure(7, 5, X, B, seed=9)
    losses = torch.zeros(steps, dtype=torch.float32, device=dev)
    a.train_steps(xd, yd, pd, perm, rates, losses)
    ref = []
    for s in range(steps):
        idx = perm[s * B:(s + 1) * B].long()
        ref.append(b.train_step(xd[idx].contiguous(), yd[idx].contiguous(), pd[idx].contiguous(), float(rates[s]),
                                want_loss=True))
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    np.testing.assert_allclose(losses.cpu().numpy(), np.array(ref, dtype=np.float32), rtol=1e-6)
    # an index outside the data set is reported, not read
    bad = perm.clone()
    bad[3] = n
    with pytest.raises(q.QLError) as e:
        a.train_steps(xd, yd, pd, bad[:B].contiguous(), rates[:1])
    assert e.value.status == q.QL_EINVAL


def test_device_training_loop_across_calls(gpu):
    """Repeated ql_closure_train_steps calls on the same buffers (the recorded step replayed, the Adam step
    count carried over), then a longer call without losses on new buffers, give bitwise the parameters of
    ql_closure_train_step on the same batches."""
    import torch
    q = gpu
    rng = np.random.default_rng(12)
    n, B, X = 40, 8, 64
    dev = torch.device("cuda", 0)
    xd = torch.tensor(rng.normal(0, 1, (n, X, 7)).astype(np.float32), device=dev)
    yd = torch.tensor(rng.normal(0, 0.5, (n, X, 5)).astype(np.float32), device=dev)
    pd = torch.tensor(rng.integers(0, 2, n).astype(np.int32), device=dev)
    a = q.Closure(7, 5, X, B, seed=4)
    b = q.Closure(7, 5, X, B, seed=4)
    perm = torch.tensor(rng.permutation(n)[:3 * B].astype(np.int32), device=dev)
    losses = torch.zeros(3, dtype=torch.float32, device=dev)
    longer = torch.tensor(rng.integers(0, n, 7 * B).astype(np.int32), device=dev)
    calls = [(perm, np.float32([3e-3, 2e-3, 1e-3]), losses), (perm, np.float32([1e-3, 5e-4, 2e-3]), losses),
             (longer, np.linspace(1e-3, 4e-3, 7).astype(np.float32), None)]
    for pm, rates, ls in calls:
        a.train_steps(xd, yd, pd, pm, rates, ls)
        for s in range(len(rates)):
            idx = pm[s * B:(s + 1) * B].long()
            b.train_step(xd[idx].contiguous(), yd[idx].contiguous(), pd[idx].contiguous(), float(rates[s]))
        np.testing.assert_array_equal(a.get_params(), b.get_params())


def test_trained_closure_improves_held_out_coarse_fields(gpu):
    """256 training pairs (2048 samples), 40 epochs; on 64 held-out pairs the corrected coarse fields are at
    least 2.5 times closer to the fine solve than the coarse fields alone, summed over rho, u, T, q, Pxx, and at
    least 1.8 times closer in every field (measured: 4.6 and 2.3 for q, the field the net helps least)."""
    from paper_2211_16933_gb300 import learned as L
    train_specs = L.pair_specs(256, 0)
    test_specs = L.pair_specs(64, 10 ** 6)
    x, y, per, _ = L.generate(train_specs, fine_steps=512)
    xt, yt, pt, ct = L.generate(test_specs, fine_steps=512)
    net, losses = L.train(x, y, per, epochs=40, batch=64, lr=2e-3, seed=0)
    pred = L.predict(net, xt, pt, 64)
    zero = yt * 0
    base = L.field_errors(zero, yt)      # coarse fields alone
    corr = L.field_errors(pred, yt)      # coarse fields plus the network
    rms_base = sum(v["l2"] for v in base.values())
    rms_corr = sum(v["l2"] for v in corr.values())
    assert losses[-1] < losses[0]
    assert rms_corr < rms_base / 2.5, (base, corr)
    for k in base:
        assert corr[k]["l2"] < base[k]["l2"] / 1.8, (k, base[k], corr[k])
