"""Pins of the learned-guess reference (oracle.mlp) against what mathematics
and independent routines fix: the bf16 rounding against PyTorch's own
conversion, GELU's tanh form against the exact x Phi(x) and its derivative
against finite differences, the features and the target against closed forms
(circular orbit, short-step limit of the Kepler root), the analytic gradient
against central finite differences, Adam against its closed form, and a
training run that makes the learned guess cut Newton iterations in the
oracle's own Kepler solve (Appendix)."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as M
from paper_1007_3458_gb300 import workloads as W


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    f = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-6, 1000), rng.normal(0, 1e6, 1000)])
    f = f.astype(np.float32)
    # exact ties: bf16 value + half its spacing
    ties = (M.bf16(f[:500]) * (1 + 2.0 ** -8)).astype(np.float32)
    f = np.concatenate([f, ties])
    ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(f), ref)
    assert M.bf16(np.float32(1 + 2 ** -8)) == 1.0          # tie to even
    assert M.bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_gelu_tanh_form():
    x = np.linspace(-8, 8, 4001)
    exact = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    assert np.abs(M.gelu(x) - exact).max() < 5e-4             # the tanh form of x Phi(x)
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, rtol=0, atol=1e-15)
    assert M.gelu(np.array(0.0)) == 0.0
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.abs(M.dgelu(x) - fd).max() < 1e-8


def _circular(n, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.5, 40, n)
    th = rng.uniform(0, 2 * np.pi, n)
    q = np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n)], 1)
    vc = np.sqrt(1.0 / r)
    v = np.stack([-vc * np.sin(th), vc * np.cos(th), np.zeros(n)], 1)
    return q, v, r


def test_features_closed_forms():
    q, v, r = _circular(50, 1)
    dt = 0.37
    u = M.features(q, v, dt, 1.0)
    assert np.allclose(u[:, 0], 0, atol=1e-14)                # no radial velocity
    assert np.allclose(u[:, 1], 1, rtol=1e-14)                # r v^2 / mu = 1
    nmean = np.sqrt(1.0 / r ** 3)
    assert np.allclose(u[:, 2], np.log(dt * nmean), rtol=1e-13)
    assert np.allclose(u[:, 3], dt * nmean / (2 * np.pi), rtol=1e-13)  # dt / P
    # purely radial escape: u1 = v sqrt(r / mu), u4 = 0 for alpha < 0
    q2 = np.array([[2.0, 0, 0]])
    v2 = np.array([[1.5, 0, 0]])
    u2 = M.features(q2, v2, dt, 1.0)
    assert np.isclose(u2[0, 0], 1.5 * math.sqrt(2.0), rtol=1e-15)
    assert u2[0, 3] == 0.0
    # the learned guess is used on bound orbits only: x_std elsewhere
    assert M.bound(q, v, 1.0).all() and not M.bound(q2, v2, 1.0).any()
    w = W.mlp_init(0, u, np.zeros(len(u)))
    assert M.guess(w, q2, v2, dt, 1.0)[0] == M.x_std(q2, dt, 1.0)[0]


def test_target_circular_and_short_step_limit(oracle):
    # circular orbits: the standard guess is the root, t = 0
    q, v, r = _circular(40, 2)
    _, _, x, _, bad = oracle.kepler_drift(q, v, 1.0, 0.3, solver=1)
    assert bad == 0
    assert np.abs(M.target(q, 0.3, 1.0, x)).max() < 1e-10
    # eccentric orbits, short steps: t -> -u1 / 2 with an O(s) remainder
    qe, ve, _ = W.test_particles(200, seed=11)
    for dt in (1e-3, 1e-4):
        _, _, x, _, bad = oracle.kepler_drift(qe, ve, 1.0, dt, solver=1)
        assert bad == 0
        u = M.features(qe, ve, dt, 1.0)
        s = np.exp(u[:, 2])
        dev = np.abs(M.target(qe, dt, 1.0, x) + 0.5 * u[:, 0])
        assert np.all(dev <= 5 * s + 1e-7), float((dev / s).max())


def _weights(seed=0, n=512):
    rows = W.mlp_rows_synthetic(n, seed + 100)
    w = W.mlp_init(seed, rows[:, :4], rows[:, 4])
    # non-zero biases so that their gradients and uses are exercised
    rng = np.random.default_rng(seed + 7)
    w = w.astype(np.float64)
    for a, b in ((M.OFF_B1, M.OFF_W2), (M.OFF_B2, M.OFF_W3), (M.OFF_B3, M.OFF_MEAN)):
        w[a:b] = rng.normal(0, 0.2, b - a)
    return w.astype(np.float32), rows


def test_gradient_against_finite_differences():
    w, rows = _weights(1, 300)
    u, t = rows[:, :4], rows[:, 4]
    L, g, gabs = M.loss_and_grad(w, u, t)
    assert np.isclose(L, M.loss(w, u, t), rtol=1e-14)
    assert np.all(g[M.NW - M.N_FROZEN:] == 0)
    assert np.all(gabs >= np.abs(g) - 1e-15)
    w64 = w.astype(np.float64)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(np.arange(a, b), k, replace=False) for a, b, k in
                          ((M.OFF_W1, M.OFF_B1, 8), (M.OFF_B1, M.OFF_W2, 6), (M.OFF_W2, M.OFF_B2, 16),
                           (M.OFF_B2, M.OFF_W3, 6), (M.OFF_W3, M.OFF_B3, 8))] + [[M.OFF_B3]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(w64[i]))
        wp, wm = w64.copy(), w64.copy()
        wp[i] += h
        wm[i] -= h
        fd = (M.loss(wp, u, t) - M.loss(wm, u, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.abs(g).max()), (int(i), fd, g[i])


def test_emulated_bf16_within_its_envelope():
    """The bf16-operand evaluation differs from FP64 by no more than the bf16
    rounding of its operands allows, and does differ (the emulation is on)."""
    w, rows = _weights(2, 400)
    u, t = rows[:, :4], rows[:, 4]
    y, _ = M.forward(w, u)
    ye, _ = M.forward(w, u, emulate=True)
    assert 0 < np.abs(y - ye).max()
    tol = M.y_tolerance(w, u, rel=2.0 ** -6, near=1.0)
    assert np.all(np.abs(y - ye) <= tol)
    _, g, gabs = M.loss_and_grad(w, u, t)
    _, ge, _ = M.loss_and_grad(w, u, t, emulate=True)
    assert np.all(np.abs(g - ge) <= 2.0 ** -5 * gabs + 1e-12)
    assert np.linalg.norm(g - ge) <= 1e-2 * np.linalg.norm(g)


def test_adam_closed_form():
    rng = np.random.default_rng(4)
    w = rng.normal(size=M.NW)
    g = rng.normal(size=M.NW) * 1e-3
    m0 = np.zeros(M.NW)
    w1, m1, v1 = M.adam(w, m0, m0, g, 1, 1e-3)
    # step 1 from zero moments: w - lr g / (|g| + eps)
    exp = w - 1e-3 * g / (np.abs(g) + 1e-8)
    exp[M.NW - M.N_FROZEN:] = w[M.NW - M.N_FROZEN:]
    assert np.allclose(w1, exp, rtol=0, atol=1e-15)
    assert np.all(m1[M.NW - M.N_FROZEN:] == 0) and np.all(v1[M.NW - M.N_FROZEN:] == 0)
    # a constant gradient keeps the bias-corrected moments at g and g^2
    w2, _, _ = M.adam(w1, m1, v1, g, 2, 1e-3)
    assert np.allclose(w2 - w1, exp - w, rtol=0, atol=1e-15)
    assert M.lr_at(0, 10, 1.0, 0.1) == 1.0 and np.isclose(M.lr_at(10, 10, 1.0, 0.1), 0.1)


def test_training_cuts_newton_iterations(oracle):
    """Trained on the oracle's own solves for particles of seed 5 (a short
    FP64 run of the reference training loop), the learned guess needs fewer
    Newton iterations than the standard one on particles of seed 4, and both
    reach the 1e-14 residual."""
    q, v, dt = W.test_particles(6000, seed=5)
    _, _, x, _, bad = oracle.kepler_drift(q, v, 1.0, dt, solver=1)
    assert bad == 0
    rows = M.log_rows(q, v, dt, 1.0, x)
    w0 = W.mlp_init(1, rows[:, :4], rows[:, 4])
    w, L = M.train(w0, rows, 256, 6, 3e-3, 1e-4)
    assert L[-20:].mean() < 0.2 * L[:5].mean()
    qe, ve, _ = W.test_particles(3000, seed=4)
    xg = M.guess(w, qe, ve, dt, 1.0, emulate=True)
    _, _, x0, it0, b0 = oracle.kepler_drift(qe, ve, 1.0, dt, solver=1)
    _, _, x1, it1, b1 = oracle.kepler_drift(qe, ve, 1.0, dt, solver=1, guess=2, x_guess=xg)
    assert b0 == 0 and b1 == 0
    assert it1.mean() < 0.9 * it0.mean(), (it1.mean(), it0.mean())
    assert oracle.kepler_residuals(qe, ve, 1.0, dt, x1).max() <= 1e-14
    assert np.abs(x1 / x0 - 1).max() <= 1e-13
