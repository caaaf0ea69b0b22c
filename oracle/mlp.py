"""Learned warm start: network, loss gradient, Adam, standardisation, and the
projection of a predicted point into the interior.

Oracle (test infrastructure only).  The paper's method has no learned part;
these are the plain definitions the warm-start kernels implement, in float64
numpy, each written from its textbook statement:

* network: two ReLU hidden layers,
      h1 = relu(W1 xn + b1),  h2 = relu(W2 h1 + b2),  yn = W3 h2 + b3,
  with xn = (x - in_mean) / in_std and y = yn out_std + out_mean;
* loss: L = sum_{b,o} (yn_bo - tn_bo)^2 / (B O), tn = (y* - out_mean) / out_std;
* gradient by the chain rule (reverse mode) through the three layers;
* Adam (Kingma and Ba 2015, Algorithm 1): m = b1 m + (1 - b1) g,
  v = b2 v + (1 - b2) g^2, w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
* starting point pushed inside its bounds by the rule of Wachter and Biegler
  (2006, Section 3.6) with kappa_1 = kappa_2 = push, every finite-bound
  multiplier at least mu0 / (its slack);
* training target: the solution's packed point and log of the barrier
  parameter at the first iteration whose KKT error E_0 <= a level.

With bf16=True the forward and backward passes round the GEMM operands to
bfloat16 (round to nearest, ties to even) at the points the tensor-core path
does: xn, W1, W2, W3, h1, h2, dL/dyn, dL/dz2, dL/dz1.  With bf16=False they are
the exact float64 definitions.

Pinned by tests/test_oracle_mlp.py: central finite differences of L against
the reverse-mode gradient, the linear regime against a direct matrix
product, the bfloat16 rounding against torch's conversion and hand-worked
ties, two Adam steps against their closed form, the standardisation against
numpy's mean/std, and the projection against its defining inequalities.
"""
from __future__ import annotations

import math
import numpy as np

BLOCKS = ("W1", "b1", "W2", "b2", "W3", "b3")


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), via float32; as float64."""
    x = np.asarray(a, dtype=np.float64).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    r = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(x), out, x.astype(np.float64))


def _r(a, on):
    return bf16_round(a) if on else np.asarray(a, dtype=np.float64)


def forward(params, X, in_mean, in_std, bf16=False):
    """Standardised output yn and the cached activations of a batch X (B x I)."""
    xn = _r((np.asarray(X, np.float64) - in_mean) / in_std, bf16)
    W1, W2, W3 = (_r(params[k], bf16) for k in ("W1", "W2", "W3"))
    h1 = _r(np.maximum(xn @ W1.T + params["b1"], 0.0), bf16)
    h2 = _r(np.maximum(h1 @ W2.T + params["b2"], 0.0), bf16)
    yn = h2 @ W3.T + params["b3"]
    return dict(xn=xn, h1=h1, h2=h2, yn=yn, W1=W1, W2=W2, W3=W3)


def predict(params, X, scaling, bf16=False):
    """Prediction y = yn out_std + out_mean."""
    c = forward(params, X, scaling["in_mean"], scaling["in_std"], bf16)
    return c["yn"] * scaling["out_std"] + scaling["out_mean"]


def loss_and_grad(params, X, Y, scaling, bf16=False):
    """L and dL/dparams (dict of the six blocks) for a batch (X, Y)."""
    c = forward(params, X, scaling["in_mean"], scaling["in_std"], bf16)
    B, O = c["yn"].shape
    tn = (np.asarray(Y, np.float64) - scaling["out_mean"]) / scaling["out_std"]
    diff = c["yn"] - tn
    L = float(np.sum(diff * diff) / (B * O))
    gy = _r(2.0 * diff / (B * O), bf16)                 # dL/dyn
    g = {"W3": gy.T @ c["h2"], "b3": gy.sum(axis=0)}
    dz2 = _r((gy @ c["W3"]) * (c["h2"] > 0), bf16)     # dL/dz2
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = _r((dz2 @ c["W2"]) * (c["h1"] > 0), bf16)    # dL/dz1
    g["W1"] = dz1.T @ c["xn"]
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t = index of this step, from 1); returns
    new (params, m, v)."""
    p2, m2, v2 = {}, {}, {}
    for k in params:
        g = np.asarray(grads[k], np.float64)
        m2[k] = beta1 * m[k] + (1.0 - beta1) * g
        v2[k] = beta2 * v[k] + (1.0 - beta2) * g * g
        mh = m2[k] / (1.0 - beta1 ** t)
        vh = v2[k] / (1.0 - beta2 ** t)
        p2[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def col_stats(Y):
    """Column mean and (population) standard deviation, the latter raised to
    1e-6 max(1, |mean|) where smaller."""
    Y = np.asarray(Y, np.float64)
    mu = Y.mean(axis=0)
    sd = np.sqrt(((Y - mu) ** 2).mean(axis=0))
    return mu, np.maximum(sd, 1e-6 * np.maximum(1.0, np.abs(mu)))


def push_inside(v, lo, hi, k1, k2):
    """Wachter-Biegler (2006) Section 3.6: move v at least
    min(k1 max(1, |bound|), k2 (hi - lo)) inside each finite bound."""
    v = np.array(v, dtype=np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    fl, fu = np.isfinite(lo), np.isfinite(hi)
    width = np.where(fl & fu, hi - lo, np.inf)
    with np.errstate(invalid="ignore"):
        pl = np.minimum(k1 * np.maximum(1.0, np.abs(lo)), k2 * width)
        pu = np.minimum(k1 * np.maximum(1.0, np.abs(hi)), k2 * width)
        v = np.where(fl, np.maximum(v, lo + pl), v)
        v = np.where(fu, np.minimum(v, hi - pu), v)
    return v


def clamp_mu0(log_mu0, tol, mu0_max):
    """mu0 = exp(log mu0) kept inside [tol / 10, mu0_max] (mu0_max if not finite)."""
    lo, hi = math.log(tol / 10.0), math.log(mu0_max)
    lm = float(log_mu0)
    lm = min(hi, max(lo, lm)) if math.isfinite(lm) else hi
    return math.exp(lm)


def project_start(pred, n, m_E, m_I, xl, xu, hl, hu, push, mu0):
    """Interior starting point from a predicted packed point
    [x | d | y_g | y_h | z_l | z_u | v_l | v_u] (float64 values)."""
    pred = np.asarray(pred, np.float64)
    off = np.cumsum([0, n, m_I, m_E, m_I, n, n, m_I, m_I])
    x, d, yg, yh, zl, zu, vl, vu = (pred[off[i]:off[i + 1]] for i in range(8))
    xp = push_inside(x, xl, xu, push, push)
    dp = push_inside(d, hl, hu, push, push)

    def mult(z, slack, finite):
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(finite, np.maximum(z, mu0 / slack), 0.0)

    xl, xu, hl, hu = (np.asarray(a, np.float64) for a in (xl, xu, hl, hu))
    out = [xp, dp, yg.copy(), yh.copy(),
           mult(zl, xp - xl, np.isfinite(xl)), mult(zu, xu - xp, np.isfinite(xu)),
           mult(vl, dp - hl, np.isfinite(hl)), mult(vu, hu - dp, np.isfinite(hu))]
    return np.concatenate(out)


def warmstart_log_mu(records, e0_level):
    """log of the barrier parameter of the first (E0, mu) record with
    E0 <= e0_level; of the last record if there is none."""
    for e0, mu in records:
        if e0 <= e0_level:
            return math.log(mu)
    return math.log(records[-1][1])
