"""FP64 reference of the learned cross-section surrogate (TEST INFRASTRUCTURE).

Only tests, smoke() and bench.py's CPU legs use this module; it shares no
code with the CUDA library.

The surrogate maps an energy to the natural log of the total cross section
of every material at once (energy is constant along a ray, so one
evaluation per ray serves every cell it crosses, Eq. 4):

    x      = (log10 E - log10 e_lo) / (log10 e_hi - log10 e_lo)
    emb(E) = [sin(pi f_0 x), cos(pi f_0 x), ..., sin(pi f_31 x), cos(pi f_31 x)],
             f_k = 2^(5 k / 31)  (32 frequencies, 1 to 32)
    h1 = silu(W1 emb + b1)   (64 -> 128)
    h2 = silu(W2 h1 + b2)    (128 -> 128)
    y  = W3 h2 + b3 + log(a + b E^(-1/2))   (128 -> 16), y_m = log Sigma_m(E)

silu(z) = z / (1 + exp(-z)).  The last term is a fixed prior per material,
the 1/v shape of a total cross section (a constant plus a term in
1/sqrt(E)), with a_m > 0 and b_m >= 0; the network learns the rest.
Parameters are one flat float vector in the order W1 [128][64], b1 [128],
W2 [128][128], b2 [128], W3 [16][128], b3 [16], C [16][2] (C[m] = a_m, b_m).
The training loss is the mean of (y_m - log Sigma_m)^2 over the unmasked
(row, material) pairs.
"""
from __future__ import annotations

import numpy as np

N_FREQ = 32
FREQ_MAX_LOG2 = 5  # highest frequency 2^5 = 32 periods over the energy range
EMB = 2 * N_FREQ
HID = 128
OUT = 16
SHAPES = (("W1", (HID, EMB)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,)), ("C", (OUT, 2)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def frequencies() -> np.ndarray:
    return 2.0 ** (FREQ_MAX_LOG2 * np.arange(N_FREQ) / (N_FREQ - 1))


def unpack(params):
    params = np.asarray(params, np.float64)
    assert params.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pack(tensors) -> np.ndarray:
    return np.concatenate([np.asarray(tensors[n], np.float64).reshape(-1) for n, _ in SHAPES])


def normalized_log_energy(E, e_lo: float, e_hi: float) -> np.ndarray:
    a, b = np.log10(e_lo), np.log10(e_hi)
    return (np.log10(np.asarray(E, np.float64)) - a) / (b - a)


def embed(E, e_lo: float, e_hi: float) -> np.ndarray:
    x = normalized_log_energy(E, e_lo, e_hi)[:, None]
    ph = np.pi * frequencies()[None, :] * x
    out = np.empty((x.shape[0], EMB))
    out[:, 0::2] = np.sin(ph)
    out[:, 1::2] = np.cos(ph)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def prior(params, E):
    """a_m + b_m E^(-1/2) per row and material, and E^(-1/2)."""
    P = unpack(params)
    r = 1.0 / np.sqrt(np.asarray(E, np.float64))
    return P["C"][None, :, 0] + P["C"][None, :, 1] * r[:, None], r


def forward(params, E, e_lo: float, e_hi: float):
    """Returns y [M][16] and the intermediate values the gradient needs."""
    P = unpack(params)
    x0 = embed(E, e_lo, e_hi)
    z1 = x0 @ P["W1"].T + P["b1"]
    h1 = silu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = silu(z2)
    q, r = prior(params, E)
    y = h2 @ P["W3"].T + P["b3"] + np.log(q)
    return y, dict(x0=x0, z1=z1, h1=h1, z2=z2, h2=h2, q=q, r=r)


def loss_and_grad(params, E, target, mask, e_lo: float, e_hi: float):
    """Mean squared error over mask (bool [M][16]) and its gradient (flat)."""
    P = unpack(params)
    y, c = forward(params, E, e_lo, e_hi)
    mask = np.asarray(mask, bool)
    count = max(int(mask.sum()), 1)
    r = np.where(mask, y - np.asarray(target, np.float64), 0.0)
    loss = float(np.sum(r * r) / count)
    dy = 2.0 * r / count
    g = {}
    g["W3"] = dy.T @ c["h2"]
    g["b3"] = dy.sum(0)
    g["C"] = np.stack([(dy / c["q"]).sum(0), (dy * c["r"][:, None] / c["q"]).sum(0)], axis=1)
    dz2 = (dy @ P["W3"]) * silu_grad(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * silu_grad(c["z1"])
    g["W1"] = dz1.T @ c["x0"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, and
    the prior a = 1, b = 0 (log q = 0)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            bound = 1.0 / np.sqrt(shape[1])
            P[name] = rng.uniform(-bound, bound, shape)
        elif name == "C":
            P[name] = np.stack([np.ones(OUT), np.zeros(OUT)], axis=1)
        else:
            P[name] = np.zeros(shape)
    return pack(P)


def bf16_round(a) -> np.ndarray:
    """Round float64 values to bfloat16 (nearest, ties to even) and back."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
