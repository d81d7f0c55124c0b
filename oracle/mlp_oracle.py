"""CPU FP64 oracle for the learned step controller that stands beside the paper's plain
controller of Algorithm 2 (the paper itself has no learned part; the definitions below are the
library's, stated with the C declarations of the controller).

TEST INFRASTRUCTURE ONLY: imported by tests/ and nowhere on the product path.  Shares no code
with the CUDA library.

* The network: y = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4 with x in R^32,
  hidden widths 64, y in R^2; loss L = (1/n) sum_s ||y_s - t_s||^2.  Forward, hand-written
  backward (chain rule through the ReLUs) and Adam (Kingma & Ba 2015, bias-corrected), all in
  FP64.  Parameter vector layout: W1 (64x32 row-major), b1, W2, b2, W3, b3, W4 (2x64), b4.
* The featurisation of an accepted-step history and the training target of the next step.

The GPU keeps BF16 weights and activations with FP32 accumulation; comparisons round the
weights and inputs to BF16 (round to nearest even) before calling this oracle.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import numpy as np

NIN, NH, NOUT = 32, 64, 2
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NH)), ("b3", (NH,)), ("W4", (NOUT, NH)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
HISTORY = 8


def unpack(p: np.ndarray) -> Dict[str, np.ndarray]:
    """Split the flat parameter vector into the named tensors (views)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + k], np.float64).reshape(shp)
        o += k
    return out


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def forward(p: np.ndarray, X: np.ndarray):
    """Network output Y (n x 2) and the activations needed by backward."""
    P = unpack(p)
    X = np.asarray(X, np.float64)
    Z1 = X @ P["W1"].T + P["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(Z2, 0.0)
    Z3 = H2 @ P["W3"].T + P["b3"]
    H3 = np.maximum(Z3, 0.0)
    Y = H3 @ P["W4"].T + P["b4"]
    return Y, (X, Z1, H1, Z2, H2, Z3, H3)


def loss_and_grad(p: np.ndarray, X: np.ndarray, T: np.ndarray):
    """L = (1/n) sum ||Y - T||^2 and dL/dp (flat, FP64) by the chain rule."""
    P = unpack(p)
    Y, (X0, Z1, H1, Z2, H2, Z3, H3) = forward(p, X)
    n = X0.shape[0]
    R = Y - np.asarray(T, np.float64)
    L = float(np.sum(R * R) / n)
    D4 = 2.0 * R / n                          # dL/dY
    gW4 = D4.T @ H3
    gb4 = D4.sum(axis=0)
    D3 = (D4 @ P["W4"]) * (Z3 > 0)            # dL/dZ3
    gW3 = D3.T @ H2
    gb3 = D3.sum(axis=0)
    D2 = (D3 @ P["W3"]) * (Z2 > 0)
    gW2 = D2.T @ H1
    gb2 = D2.sum(axis=0)
    D1 = (D2 @ P["W2"]) * (Z1 > 0)
    gW1 = D1.T @ X0
    gb1 = D1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gW4.ravel(), gb4])
    return L, g


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------------------------
# featurisation and targets
# ---------------------------------------------------------------------------------------------
def _clamp(x, lo, hi):
    return min(hi, max(lo, x))


def _log10_floor(v, lo):
    return max(lo, math.log10(v)) if (v > 0 and math.isfinite(v)) else lo


def features(recs: Sequence[dict]) -> np.ndarray:
    """32 inputs from the last 8 accepted steps (latest first; missing steps repeat the oldest):
    log10(h/h_max)/3 in [-2, 0], m/m_max, log10(err/E)/3 in [-2, 1/3], (log10 dF + 6)/6."""
    out = np.zeros(4 * HISTORY)
    for j in range(HISTORY):
        r = recs[max(len(recs) - 1 - j, 0)]
        hr = r["h"] / r["h_max"] if r["h_max"] > 0 else 1.0
        out[4 * j + 0] = _clamp(_log10_floor(hr, -6.0), -6.0, 0.0) / 3.0
        out[4 * j + 1] = r["m"] / r["m_max"] if r["m_max"] > 0 else 0.0
        er = r["err"] / r["E"] if r["E"] > 0 else 0.0
        out[4 * j + 2] = _clamp(_log10_floor(er, -6.0), -6.0, 1.0) / 3.0
        out[4 * j + 3] = (_clamp(_log10_floor(r["dF"], -12.0), -12.0, 0.0) + 6.0) / 6.0
    return out


def target(recs: Sequence[dict], nxt: dict):
    """(log2 of the next accepted step over h_k widened by the error headroom, m_next/m_max),
    or None when the next step was cut to land on a corner."""
    if nxt["landed"] or not nxt["h"] > 0:
        return None
    head = 0.8 * math.sqrt(nxt["E"] / nxt["err"]) if nxt["err"] > 0 else 2.0
    head = _clamp(head, 1.0, 2.0)
    t0 = math.log2(nxt["h"] / recs[-1]["h"]) + math.log2(head)
    return np.array([_clamp(t0, -3.0, 2.0), nxt["m"] / nxt["m_max"] if nxt["m_max"] > 0 else 0.0])


def samples(traces: List[List[dict]]):
    """Training set from per-instance traces: one sample per accepted step with a usable
    successor."""
    X, T = [], []
    for R in traces:
        for k in range(len(R) - 1):
            t = target(R[:k + 1], R[k + 1])
            if t is None:
                continue
            X.append(features(R[:k + 1]))
            T.append(t)
    return np.array(X).reshape(-1, 4 * HISTORY), np.array(T).reshape(-1, 2)
