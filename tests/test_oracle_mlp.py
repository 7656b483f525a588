"""Pins of the FP64 surrogate reference (oracle/mlp.py).

- gradients against central finite differences of the loss (rel <= 1e-6),
  the prior's coefficients included;
- the forward pass against an independent float64 torch.nn implementation
  of the same network (Linear / SiLU) plus the prior written out;
- special cases: the embedding at the range ends (x = 0: sines 0, cosines 1;
  x = 1: sin(pi f) and cos(pi f)), zero first-layer weights make the output
  independent of energy up to the prior, zero network weights leave exactly
  the 1/v prior log(a + b / sqrt(E)), bf16 rounding against torch's
  bfloat16 cast.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as M


def _params(seed=1, scale=1.0):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    p = p * scale + 0.05 * rng.normal(size=p.shape)
    P = M.unpack(p)
    P["C"][:, 0] = rng.uniform(0.05, 5.0, M.OUT)   # a > 0
    P["C"][:, 1] = rng.uniform(0.0, 3.0, M.OUT)    # b >= 0
    return M.pack(P)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = _params(2)
    E = np.exp(rng.uniform(np.log(1e-5), np.log(2e7), 7))
    # targets near the outputs (residuals of order 1, as before the prior)
    T = np.log(M.prior(p, E)[0]) + rng.normal(size=(7, M.OUT))
    mask = rng.random((7, M.OUT)) < 0.8
    loss, g = M.loss_and_grad(p, E, T, mask, 1e-5, 2e7)
    idx = rng.choice(M.N_PARAMS, 300, replace=False)
    c0 = M.N_PARAMS - 2 * M.OUT  # the prior's coefficients
    idx = np.concatenate([idx, [0, M.N_PARAMS - 1, 64 * 128 + 5, 64 * 128 + 128 + 77],
                          np.arange(c0, M.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = M.loss_and_grad(p + e, E, T, mask, 1e-5, 2e7)
        lm, _ = M.loss_and_grad(p - e, E, T, mask, 1e-5, 2e7)
        fd = (lp - lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_forward_matches_torch_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    p = _params(3)
    E = np.exp(rng.uniform(np.log(1e-5), np.log(2e7), 50))
    y, _ = M.forward(p, E, 1e-5, 2e7)
    P = M.unpack(p)
    net = torch.nn.Sequential(torch.nn.Linear(M.EMB, M.HID), torch.nn.SiLU(),
                              torch.nn.Linear(M.HID, M.HID), torch.nn.SiLU(),
                              torch.nn.Linear(M.HID, M.OUT)).double()
    with torch.no_grad():
        for layer, (w, b) in zip([net[0], net[2], net[4]], [("W1", "b1"), ("W2", "b2"), ("W3", "b3")]):
            layer.weight.copy_(torch.from_numpy(P[w]))
            layer.bias.copy_(torch.from_numpy(P[b]))
        # embedding written independently: angle = pi * 2^(5k/31) * x
        x = (np.log10(E) + 5.0) / (np.log10(2e7) + 5.0)
        k = np.arange(32)
        ang = np.pi * np.exp2(5.0 * k / 31.0)[None, :] * x[:, None]
        emb = np.stack([np.sin(ang), np.cos(ang)], axis=2).reshape(len(E), 64)
        want = net(torch.from_numpy(emb)).numpy()
    # the 1/v prior, per material
    want = want + np.log(P["C"][:, 0][None, :] + P["C"][:, 1][None, :] / np.sqrt(E)[:, None])
    np.testing.assert_allclose(y, want, rtol=1e-12, atol=1e-12)


def test_embedding_end_values():
    e = M.embed(np.array([1e-5, 2e7]), 1e-5, 2e7)
    np.testing.assert_allclose(e[0, 0::2], 0.0, atol=1e-15)
    np.testing.assert_allclose(e[0, 1::2], 1.0, atol=1e-15)
    f = M.frequencies()
    assert f[0] == 1.0 and f[-1] == pytest.approx(32.0, rel=1e-14)
    np.testing.assert_allclose(e[1, 0::2], np.sin(np.pi * f), atol=1e-9)


def test_zero_first_layer_makes_output_constant():
    p = M.unpack(_params(4))
    p["W1"][:] = 0.0
    flat = M.pack(p)
    E = np.array([1e-3, 1.0, 1e6])
    y, _ = M.forward(flat, E, 1e-5, 2e7)
    y = y - np.log(p["C"][:, 0][None, :] + p["C"][:, 1][None, :] / np.sqrt(E)[:, None])
    np.testing.assert_allclose(y[0], y[1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(y[0], y[2], rtol=0, atol=1e-14)


def test_prior_alone_is_the_one_over_v_law():
    """With W3 = 0 and b3 = 0 the output is the prior: Sigma = a + b/sqrt(E),
    so at E = 1 eV it is a + b and at E = 1e-4 eV a + 100 b."""
    p = M.unpack(_params(6))
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    p["C"][:, 0] = 0.5
    p["C"][:, 1] = np.arange(M.OUT)
    y, _ = M.forward(M.pack(p), np.array([1.0, 1e-4]), 1e-5, 2e7)
    np.testing.assert_allclose(np.exp(y[0]), 0.5 + np.arange(M.OUT), rtol=1e-14)
    np.testing.assert_allclose(np.exp(y[1]), 0.5 + 100.0 * np.arange(M.OUT), rtol=1e-14)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    a = rng.normal(size=1000) * 10.0 ** rng.uniform(-5, 5, 1000)
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(M.bf16_round(a), want)
