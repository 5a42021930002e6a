"""Pin of the reference network: its back-propagated gradient equals central finite
differences of its loss (FP64, no quantization), and the quantized forward pass differs
from the exact one only at the bfloat16 level; the network, its loss and gradient equal
torch's layers and autograd, and the bfloat16 rounding equals torch's conversion."""
import numpy as np
import pytest

from oracle import gauge_mlp as G


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = G.init_params(2)
    X = rng.standard_normal((37, G.IN))
    Y = rng.standard_normal((37, G.OUT))
    loss, g = G.loss_and_grad(p, X, Y, quantize=False)
    idx = np.concatenate([rng.choice(np.arange(G.O_W1, G.O_B1), 30), rng.choice(np.arange(G.O_B1, G.O_W2), 8),
                          rng.choice(np.arange(G.O_W2, G.O_B2), 30), rng.choice(np.arange(G.O_B2, G.O_W3), 8),
                          np.arange(G.O_W3, G.O_W3 + 3 * G.HID, 7), np.arange(G.O_B3, G.O_B3 + 3)])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (G.loss_and_grad(pp, X, Y, quantize=False)[0] - G.loss_and_grad(pm, X, Y, quantize=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # outputs 3..15 carry no loss: their weights get zero gradient
    assert np.all(g[G.O_W3 + 3 * G.HID:G.O_B3] == 0) and np.all(g[G.O_B3 + 3:] == 0)


def test_bf16_rounding():
    # bfloat16 keeps 7 fraction bits: the spacing at 1 is 2^-7
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.14159265, -2.5e-3, 0.0])
    r = G.bf16(a)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6  # halfway cases go to the even neighbour
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - a) <= np.abs(a) * 2 ** -8)
    p = G.init_params(3)
    X = np.random.default_rng(4).standard_normal((20, G.IN))
    oq, _ = G.forward(p, X, quantize=True)
    oe, _ = G.forward(p, X, quantize=False)
    assert np.abs(oq - oe).max() <= 0.05 * np.abs(oe).max()


def test_forward_loss_and_gradient_match_torch():
    """The plain network and its loss, written out in numpy, against torch's Linear/ReLU
    layers (y = x W^T + b, W stored [out][in]) and autograd, on the same FP64 parameters."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p = G.init_params(6)
    X = rng.standard_normal((29, G.IN))
    Y = rng.standard_normal((29, G.OUT))
    W1, b1, W2, b2, W3, b3 = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in G.unpack(p))
    x = torch.tensor(X, dtype=torch.float64)
    F = torch.nn.functional
    out = F.linear(F.relu(F.linear(F.relu(F.linear(x, W1, b1)), W2, b2)), W3, b3)
    loss = F.mse_loss(out[:, :G.OUT], torch.tensor(Y, dtype=torch.float64))
    loss.backward()
    ref_out, _ = G.forward(p, X, quantize=False)
    ref_loss, ref_g = G.loss_and_grad(p, X, Y, quantize=False)
    np.testing.assert_allclose(ref_out, out.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert ref_loss == pytest.approx(float(loss.detach()), rel=1e-13)
    tg = np.concatenate([t.grad.numpy().ravel() for t in (W1, b1, W2, b2, W3, b3)])
    np.testing.assert_allclose(ref_g, tg, rtol=1e-12, atol=1e-15)


def test_bf16_matches_torch_rounding():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(7).standard_normal(4096) * np.exp(np.random.default_rng(8).uniform(-20, 20, 4096))
    a = np.concatenate([a, [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, 65504.0]]).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(G.bf16(a), want)
