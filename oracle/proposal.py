"""Oracle of the learned density proposal (TEST INFRASTRUCTURE ONLY).

Plain numpy restatement of the proposal estimator's network, in the reading
this library takes of the paper's learned-proposal sampler (Table 1 "PDF
Approaches", Sec. 3.2: a small network predicts density, its transmittance
gives the PDF that inverse transform sampling, Eq. 1, resamples):

* encoding e(x) of a point x in R^3: [x, y, z] followed, for k = 0..7 and
  each axis a, by sin(2^k pi x_a), cos(2^k pi x_a) (51 values), zero-padded
  to 64;
* three layers of width 64: h1 = relu(W1 e + b1), h2 = relu(W2 h1 + b2),
  density = softplus(w3 . h2 + b3);
* BF16 operands (weights and each layer's input rounded to bfloat16,
  round-to-nearest-even), products summed in FP64 here (FP32 on the GPU),
  biases FP32;
* training: loss L = mean over the batch of (density - target)^2, the
  adjoint of the three layers, and Adam on FP32 master parameters.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import it; it shares no code with the CUDA library.  Pins in
``tests/test_oracle_pins.py``: closed-form encodings, a hand-built network,
finite differences of the loss, the closed-form first Adam step.
"""
from __future__ import annotations

import numpy as np

N_BANDS = 8
ENC = 3 + 6 * N_BANDS  # 51
IN = 64
WIDTH = 64


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32; returns float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def encode(xyz) -> np.ndarray:
    """[n][3] -> [n][64] in FP64 (before BF16 rounding)."""
    x = np.asarray(xyz, np.float64)
    n = x.shape[0]
    e = np.zeros((n, IN))
    e[:, 0:3] = x
    for k in range(N_BANDS):
        ang = (2.0 ** k) * np.pi * x
        for a in range(3):
            e[:, 3 + 6 * k + 2 * a] = np.sin(ang[:, a])
            e[:, 3 + 6 * k + 2 * a + 1] = np.cos(ang[:, a])
    return e


def init_params(seed: int = 7) -> dict:
    """Seeded initial parameters (uniform in +-1/sqrt(fan_in); the encoding's
    padding columns of W1 are zero), FP32 master copies."""
    g = np.random.default_rng(seed)
    W1 = g.uniform(-1, 1, (WIDTH, IN)) / np.sqrt(ENC)
    W1[:, ENC:] = 0.0
    return {
        "W1": W1.astype(np.float32), "b1": np.zeros(WIDTH, np.float32),
        "W2": (g.uniform(-1, 1, (WIDTH, WIDTH)) / np.sqrt(WIDTH)).astype(np.float32),
        "b2": np.zeros(WIDTH, np.float32),
        "w3": (g.uniform(-1, 1, WIDTH) / np.sqrt(WIDTH)).astype(np.float32),
        "b3": np.zeros(1, np.float32),
    }


def _softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def forward(params: dict, xyz, round_bf16: bool = True, enc=None) -> dict:
    """Density at the points; returns the intermediates too.  ``enc`` (n x 64)
    replaces the encoding when given (already in the operand precision)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    e = r(encode(xyz)) if enc is None else np.asarray(enc, np.float64)
    W1, W2, w3 = r(params["W1"]), r(params["W2"]), r(params["w3"])
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    z1 = e @ W1.T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + b2
    h2 = r(np.maximum(z2, 0.0))
    z3 = h2 @ w3 + b3[0]
    return {"e": e, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "sigma": _softplus(z3)}


def loss_and_grads(params: dict, xyz, target, round_bf16: bool = True, enc=None) -> tuple[float, dict]:
    """L = mean (sigma - target)^2 and dL/d(parameter) (FP64); ``enc`` as in
    :func:`forward`."""
    f = forward(params, xyz, round_bf16, enc=enc)
    t = np.asarray(target, np.float64)
    B = t.shape[0]
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    W2, w3 = r(params["W2"]), r(params["w3"])
    d = f["sigma"] - t
    L = float(np.mean(d * d))
    d3 = (2.0 / B) * d / (1.0 + np.exp(-f["z3"]))  # softplus' = logistic
    g = {"w3": f["h2"].T @ d3, "b3": np.array([d3.sum()])}
    d2 = np.outer(d3, w3) * (f["z2"] > 0)
    g["W2"], g["b2"] = d2.T @ f["h1"], d2.sum(0)
    d1 = (d2 @ W2) * (f["z1"] > 0)
    g["W1"], g["b1"] = d1.T @ f["e"], d1.sum(0)
    return L, g


def adam_step(params: dict, grads: dict, state: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """One Adam step on the FP32 master parameters (in place); ``state`` holds
    m, v per parameter and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k, gk in grads.items():
        gk = np.asarray(gk, np.float64)
        m = state.setdefault("m_" + k, np.zeros_like(gk))
        v = state.setdefault("v_" + k, np.zeros_like(gk))
        m[...] = b1 * m + (1 - b1) * gk
        v[...] = b2 * v + (1 - b2) * gk * gk
        mh, vh = m / (1 - b1 ** t), v / (1 - b2 ** t)
        params[k] = (params[k].astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)


def exact_optical_depth(rays_o, rays_d, t_near, t_far, mu, std, peak) -> np.ndarray:
    """Integral of the blob field's density along each ray over [t_near,
    t_far] (FP64).  Along x(t) = o + t d a blob's density is a 1-D Gaussian
    in t: peak exp(-p^2 / 2 s^2) exp(-(t - t*)^2 / 2 s_l^2) with t* the
    closest approach, p the distance there and s_l = s / |d|; its integral
    is the difference of two error functions (Eq. 2 with T = exp(-integral))."""
    from math import erf, pi, sqrt
    o, d = np.asarray(rays_o, np.float64), np.asarray(rays_d, np.float64)
    out = np.zeros(o.shape[0])
    for i in range(o.shape[0]):
        dd = d[i] @ d[i]
        if not (t_far[i] > t_near[i]) or dd == 0.0:
            continue
        acc = 0.0
        for b in range(len(peak)):
            m = np.asarray(mu[b], np.float64) - o[i]
            ts = (m @ d[i]) / dd
            p2 = max(m @ m - ts * ts * dd, 0.0)
            s = float(std[b])
            sl = s / sqrt(dd)
            acc += float(peak[b]) * np.exp(-p2 / (2 * s * s)) * sl * sqrt(pi / 2) * (
                erf((t_far[i] - ts) / (sl * sqrt(2))) - erf((t_near[i] - ts) / (sl * sqrt(2))))
        out[i] = acc
    return out
