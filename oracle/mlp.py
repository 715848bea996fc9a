"""Learned Kepler starting guess: plain FP64 reference (test infrastructure
only -- the tests, the smoke check and the benchmark's CPU baseline call it;
the library never does).

The universal Kepler equation F(x) = 0 (Appendix) is solved from a starting
guess; the standard one is x_std = sqrt(mu) dt / r0, exact for a circular
orbit. Its error is set by the ratio z = x* / x_std of the root x* to it. As
x* = sqrt(mu) * integral of dt'/r over the step, z - 1 = -u1 s / 2 + O(s^2)
with s = |dt| sqrt(mu / r0^3) the step over the local dynamical time, so the
network predicts the scaled deviation

  t = (z - 1) / sigma,   sigma = s / (1 + s),

which stays O(1) both for short steps (t -> -u1 / 2) and long ones; the guess
is x_guess = x_std (1 + sigma t). A 4 -> 64 -> 64 -> 1 perceptron maps four
dimensionless features of a body's state (q0, v0) and step dt about a star of
parameter mu to t:

  u1 = (q0 . v0) / sqrt(mu r0)          radial velocity over circular speed
  u2 = r0 |v0|^2 / mu                   2 - r0 / a
  u3 = ln s                             step over the local dynamical time
  u4 = dt / P = dt sqrt(mu alpha^3) / (2 pi) for alpha = 2/r0 - |v0|^2/mu > 0,
       else 0                           step over the orbital period

i.e. (r0, r0 . v0, |v0|^2, dt / P) made dimensionless. Each feature is
normalised, fn = (u - mean) / std; the network is

  h1 = gelu(W1 fn + b1),  h2 = gelu(W2 h1 + b2),  y = W3 . h2 + b3,
  t  = om + osd * y,

with the tanh form of GELU (Hendrycks & Gimpel):
  gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).

Weights are one flat float32 vector (NW = 4555 entries) in the order W1[64][4],
b1[64], W2[64][64], b2[64], W3[64], b3, mean[4], std[4], om, osd. The last ten
entries (normalisation) are fixed from data, never trained.

`emulate=True` evaluates the same arithmetic with the operands the GPU feeds
its BF16 tensor cores rounded as it does: the weight matrices W1, W2, W3 to
bf16, the features to float32, the hidden layer h1 (via float32) to bf16 before
W2, and in the backward pass the output gradient of the second layer (dp2) to
bf16 before its two products. Everything else, accumulation included, stays
FP64 here.

Training minimises the mean squared error of y against yt = (t - om) / osd
with Adam (Kingma & Ba), whose first-order bias-corrected form is used.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
NW = 4555
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 256, 320, 4416, 4480, 4544
OFF_MEAN, OFF_STD, OFF_OM, OFF_OSD = 4545, 4549, 4553, 4554
N_FROZEN = 10
K0 = math.sqrt(2.0 / math.pi)
K1 = 0.044715


# ---------------------------------------------------------------- helpers
def bf16(x):
    """Round to bfloat16 (8-bit significand) to nearest, ties to even, from
    float32; returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.shape == (NW,)
    return dict(W1=w[OFF_W1:OFF_B1].reshape(H, 4), b1=w[OFF_B1:OFF_W2],
                W2=w[OFF_W2:OFF_B2].reshape(H, H), b2=w[OFF_B2:OFF_W3],
                W3=w[OFF_W3:OFF_B3], b3=w[OFF_B3], mean=w[OFF_MEAN:OFF_STD],
                std=w[OFF_STD:OFF_OM], om=w[OFF_OM], osd=w[OFF_OSD])


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(K0 * (x + K1 * x ** 3)))


def dgelu(x):
    th = np.tanh(K0 * (x + K1 * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * K0 * (1.0 + 3.0 * K1 * x * x)


# ---------------------------------------------------------------- features
def features(q0, v0, dt, mu):
    """[n, 4] raw features u1..u4 of bodies q0, v0 ([n, 3]) for a step dt."""
    q0 = np.asarray(q0, dtype=np.float64).reshape(-1, 3)
    v0 = np.asarray(v0, dtype=np.float64).reshape(-1, 3)
    r0 = np.sqrt(np.sum(q0 * q0, axis=1))
    v2 = np.sum(v0 * v0, axis=1)
    rv = np.sum(q0 * v0, axis=1)
    alpha = 2.0 / r0 - v2 / mu
    u1 = rv / np.sqrt(mu * r0)
    u2 = r0 * v2 / mu
    u3 = np.log(abs(dt) * np.sqrt(mu / r0 ** 3))
    u4 = np.where(alpha > 0, dt * np.sqrt(mu * np.maximum(alpha, 0.0) ** 3) / (2.0 * math.pi), 0.0)
    return np.stack([u1, u2, u3, u4], axis=1)


def x_std(q0, dt, mu):
    """The standard starting guess sqrt(mu) dt / r0."""
    r0 = np.sqrt(np.sum(np.asarray(q0, dtype=np.float64).reshape(-1, 3) ** 2, axis=1))
    return math.sqrt(mu) * dt / r0


def sigma(q0, dt, mu):
    """sigma = s / (1 + s), s = |dt| sqrt(mu / r0^3)."""
    r0 = np.sqrt(np.sum(np.asarray(q0, dtype=np.float64).reshape(-1, 3) ** 2, axis=1))
    s = abs(dt) * np.sqrt(mu / r0 ** 3)
    return s / (1.0 + s)


def target(q0, dt, mu, xstar):
    """t = (x* / x_std - 1) / sigma for roots x* of the Kepler equation."""
    z = np.asarray(xstar, dtype=np.float64) / x_std(q0, dt, mu)
    return (z - 1.0) / sigma(q0, dt, mu)


def log_rows(q0, v0, dt, mu, xstar):
    """Training rows (u1, u2, u3, u4, t), float32 [n, 5] (meaningful for bound
    orbits, the ones the Kepler kernel logs)."""
    u = features(q0, v0, dt, mu)
    t = target(q0, dt, mu, xstar)
    return np.concatenate([u, t[:, None]], axis=1).astype(np.float32)


# ---------------------------------------------------------------- network
def forward(w, u, emulate=False):
    """y (normalised output) for raw features u [n, 4], and the
    intermediates (fn, p1, h1in, p2, h2)."""
    P = unpack(w)
    W1, W2, W3 = P["W1"], P["W2"], P["W3"]
    u = np.asarray(u, dtype=np.float64)
    if emulate:
        W1, W2, W3, u = bf16(W1), bf16(W2), bf16(W3), f32(u)
    fn = (u - P["mean"]) / P["std"]
    p1 = fn @ W1.T + P["b1"]
    h1 = gelu(p1)
    h1in = bf16(f32(h1)) if emulate else h1
    p2 = h1in @ W2.T + P["b2"]
    h2 = gelu(p2)
    y = h2 @ W3 + P["b3"]
    return y, (fn, p1, h1in, p2, h2)


def bound(q0, v0, mu):
    """alpha = 2/r0 - |v0|^2/mu > 0: the orbits the learned guess is used for
    (|u1| < sqrt 2 and u2 < 2 there); unbound bodies keep x_std."""
    q0 = np.asarray(q0, dtype=np.float64).reshape(-1, 3)
    v0 = np.asarray(v0, dtype=np.float64).reshape(-1, 3)
    return 2.0 / np.sqrt(np.sum(q0 * q0, axis=1)) - np.sum(v0 * v0, axis=1) / mu > 0


def guess(w, q0, v0, dt, mu, emulate=False):
    """The starting guess x for each body: learned on bound orbits, x_std
    elsewhere."""
    P = unpack(w)
    y, _ = forward(w, features(q0, v0, dt, mu), emulate)
    xs = x_std(q0, dt, mu)
    learned = xs * (1.0 + sigma(q0, dt, mu) * (P["om"] + P["osd"] * y))
    return np.where(bound(q0, v0, mu), learned, xs)


def y_tolerance(w, u, rel=1e-5, near=1e-5):
    """Bound on |y_gpu - y| against forward(w, u, emulate=True) for a float32
    evaluation: `rel` of the absolute-value sum of the terms (float32
    rounding, the float32 exponential and reciprocal inside GELU), plus for
    every hidden unit h1_k within `near` (relative) of a bf16 rounding midpoint
    the effect of landing in the other bf16 neighbour, |dy/dh1_k| ulp(h1_k)."""
    P = unpack(w)
    W1, W2, W3 = bf16(P["W1"]), bf16(P["W2"]), bf16(P["W3"])
    y, (fn, p1, h1in, p2, h2) = forward(w, u, emulate=True)
    a1 = np.abs(fn) @ np.abs(W1).T + np.abs(P["b1"])
    s2 = (np.abs(h1in) + np.abs(dgelu(p1)) * a1) @ np.abs(W2).T + np.abs(P["b2"])
    s = (np.abs(h2) + np.abs(dgelu(p2)) * s2) @ np.abs(W3) + abs(P["b3"])
    h1 = f32(gelu(p1))
    # bf16 neighbours of h1: spacing 2^(e - 7) for |h1| in [2^e, 2^(e+1))
    e = np.floor(np.log2(np.maximum(np.abs(h1), 1e-38)))
    ulp = 2.0 ** (e - 7)
    mid_off = np.abs(np.mod(np.abs(h1), ulp) - 0.5 * ulp)
    close = mid_off <= near * np.abs(h1) + 1e-30
    dydh1 = (W3 * dgelu(p2)) @ W2          # [n, 64]
    flip = np.sum(np.where(close, np.abs(dydh1) * ulp, 0.0), axis=1)
    return rel * s + flip


def loss_and_grad(w, u, t, emulate=False):
    """Mean squared error L of y against (t - om) / osd over the rows of
    (u, t), its gradient g with respect to every weight (zero for the ten
    normalisation entries), and gabs: the same sums taken over absolute values
    of their terms (the scale of each entry's rounding error)."""
    P = unpack(w)
    W2, W3 = P["W2"], P["W3"]
    if emulate:
        W2, W3 = bf16(W2), bf16(W3)
    y, (fn, p1, h1in, p2, h2) = forward(w, u, emulate)
    yt = (np.asarray(t, dtype=np.float64) - P["om"]) / P["osd"]
    n = len(y)
    r = y - yt
    L = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3, aW3 = h2.T @ dy, np.abs(h2).T @ np.abs(dy)
    gb3, ab3 = np.sum(dy), np.sum(np.abs(dy))
    dp2 = np.outer(dy, W3) * dgelu(p2)
    gb2, ab2 = dp2.sum(0), np.abs(dp2).sum(0)
    dp2in = bf16(f32(dp2)) if emulate else dp2
    gW2, aW2 = dp2in.T @ h1in, np.abs(dp2in).T @ np.abs(h1in)
    dh1 = dp2in @ W2
    adh1 = np.abs(dp2in) @ np.abs(W2)
    dp1 = dh1 * dgelu(p1)
    adp1 = adh1 * np.abs(dgelu(p1))
    gb1, ab1 = dp1.sum(0), adp1.sum(0)
    gW1, aW1 = dp1.T @ fn, adp1.T @ np.abs(fn)
    z10 = np.zeros(N_FROZEN)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3], z10])
    gabs = np.concatenate([aW1.ravel(), ab1, aW2.ravel(), ab2, aW3, [ab3], z10])
    return L, g, gabs


def loss(w, u, t):
    P = unpack(w)
    y, _ = forward(w, u)
    yt = (np.asarray(t, dtype=np.float64) - P["om"]) / P["osd"]
    return float(np.mean((y - yt) ** 2))


def adam(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam step t (1-based): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    w <- w - lr m_hat / (sqrt(v_hat) + eps) with m_hat = m / (1 - b1^t),
    v_hat = v / (1 - b2^t). The normalisation entries are not parameters of
    the fit: their w, m and v are left as they are. Returns (w, m, v) in
    float64."""
    w = np.array(w, dtype=np.float64)
    m0 = np.asarray(m, dtype=np.float64)
    v0 = np.asarray(v, dtype=np.float64)
    m = b1 * m0 + (1.0 - b1) * g
    v = b2 * v0 + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    upd = lr * mh / (np.sqrt(vh) + eps)
    fz = slice(NW - N_FROZEN, NW)
    upd[fz] = 0.0
    m[fz] = m0[fz]
    v[fz] = v0[fz]
    return w - upd, m, v


def lr_at(step, nsteps, lr, lr_final):
    """Cosine schedule from lr (step 0) towards lr_final."""
    return lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * step / nsteps))


def train(w, data, batch, epochs, lr, lr_final, emulate=False):
    """Minibatch Adam over data rows (u1..u4, t) in order, `epochs` passes,
    cosine learning rate; weights kept in float32 between steps as the GPU
    keeps them. Returns (w float32, per-step losses)."""
    data = np.asarray(data, dtype=np.float64)
    n = len(data)
    nb = (n + batch - 1) // batch
    S = nb * epochs
    w = np.asarray(w, dtype=np.float32)
    m = np.zeros(NW)
    v = np.zeros(NW)
    losses = []
    for s in range(S):
        b = s % nb
        rows = data[b * batch:min(n, (b + 1) * batch)]
        L, g, _ = loss_and_grad(w, rows[:, :4], rows[:, 4], emulate)
        losses.append(L)
        w64, m, v = adam(w, m, v, g, s + 1, lr_at(s, S, lr, lr_final))
        w = w64.astype(np.float32)
    return w, np.array(losses)
