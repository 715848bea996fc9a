"""GPU parity of the learned Kepler starting guess (the Appendix's universal
Kepler equation started from a predicted root) against the oracle: network
output, gradient, Adam step and a short training run against the FP64
reference evaluated with the same bf16 operands; the guess and the training
rows the Kepler kernel computes; logging from qym_step; and the gain of the
trained guess over the standard one on the 1,048,576 test particles."""
import math

import numpy as np
import pytest

import paper_1007_3458_gb300 as q
from paper_1007_3458_gb300 import workloads as W
from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return t


def _weights(seed, n=512):
    rows = W.mlp_rows_synthetic(n, seed + 100)
    w = W.mlp_init(seed, rows[:, :4], rows[:, 4]).astype(np.float64)
    rng = np.random.default_rng(seed + 7)
    for a, b in ((M.OFF_B1, M.OFF_W2), (M.OFF_B2, M.OFF_W3), (M.OFF_B3, M.OFF_MEAN)):
        w[a:b] = rng.normal(0, 0.2, b - a)
    return w.astype(np.float32)


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=dtype) if dtype else t.cuda()


def _soa(torch, x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float64).T)).cuda()


def _stumpff_np(y):
    """C(y), S(y) to a few digits (only for tolerances below)."""
    y = np.asarray(y, dtype=np.float64)
    C = np.full_like(y, 0.5)
    S = np.full_like(y, 1.0 / 6.0)
    big = np.abs(y) > 1e-3
    sp = np.sqrt(np.abs(y[big]))
    pos = y[big] > 0
    Cb = np.where(pos, (1 - np.cos(sp)) / np.abs(y[big]), (np.cosh(sp) - 1) / np.abs(y[big]))
    Sb = np.where(pos, (sp - np.sin(sp)) / sp ** 3, (np.sinh(sp) - sp) / sp ** 3)
    C[big], S[big] = Cb, Sb
    small = ~big
    C[small] = 0.5 - y[small] / 24
    S[small] = 1 / 6 - y[small] / 120
    return C, S


def _root_tolerance(qq, vv, dt, x, q1, res=1e-14 + 8 * 2.0 ** -53, mu=1.0):
    """How far apart two roots x that both meet the relative residual `res`
    can put the body: |dx| <= 2 res scale / F'(x) with F' = r1 (the distance
    at the end of the step) and scale the sum of |terms| of F, and
    |dq/dx| <= |U1| |q0| / r0 + |U2| |v0| / sqrt(mu) (U1 = x (1 - y S),
    U2 = x^2 C are the x-derivatives of x^2 C and x^3 S). Returns (dx, dq)."""
    r0 = np.linalg.norm(qq, axis=1)
    alpha = 2 / r0 - np.sum(vv * vv, axis=1) / mu
    sig = np.sum(qq * vv, axis=1) / np.sqrt(mu)
    y = alpha * x * x
    C, S = _stumpff_np(y)
    scale = (abs(np.sqrt(mu) * dt) + np.abs(sig * x * x * C) + np.abs((1 - r0 * alpha) * x ** 3 * S)
             + r0 * np.abs(x))
    dx = 2 * res * scale / np.linalg.norm(q1, axis=1)
    dq = (np.abs(x * (1 - y * S)) * r0 / r0 + np.abs(x * x * C) * np.linalg.norm(vv, axis=1)
          / np.sqrt(mu)) * dx
    return dx, dq


@pytest.mark.parametrize("n", [1, 31, 1000 + 37])
def test_forward_matches_oracle(torch, n):
    """Network output for raw features: within the float32 rounding envelope
    plus bf16 neighbour flips of hidden units near a rounding midpoint."""
    w = _weights(1)
    rows = W.mlp_rows_synthetic(n, 3)
    u = rows[:, :4].copy()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qym_mlp_forward_dev(n, _dev(torch, w), _dev(torch, u), y)
    torch.cuda.synchronize()
    yo, _ = M.forward(w, u, emulate=True)
    tol = M.y_tolerance(w, u, rel=2e-5, near=2e-5)
    err = np.abs(y.cpu().numpy() - yo)
    assert np.all(err <= tol), (float(err.max()), int(np.argmax(err - tol)))
    # and well inside the envelope for most rows
    assert np.median(err / tol) < 0.3


@pytest.mark.parametrize("n", [64, 3019, 40000 + 11])
def test_gradient_matches_oracle(torch, n):
    """dL/dw of all rows against the FP64 gradient with the same bf16
    operands: every entry within 2^-6 of its absolute term sum, the whole
    vector within 1e-3 relative; the loss within 1e-5."""
    w = _weights(2)
    rows = W.mlp_rows_synthetic(n, 4)
    work = torch.empty(q.qym_mlp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    g = torch.empty(q.QYM_MLP_NW, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    q.qym_mlp_grad_dev(n, _dev(torch, w), _dev(torch, rows), g, loss, work)
    torch.cuda.synchronize()
    L, go, gabs = M.loss_and_grad(w, rows[:, :4], rows[:, 4], emulate=True)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.all(gg[M.NW - M.N_FROZEN:] == 0)
    d = np.abs(gg - go)
    bad = np.nonzero(d > 2.0 ** -6 * gabs + 1e-7 * np.abs(go).max())[0]
    assert len(bad) == 0, [(int(i), gg[i], go[i], gabs[i]) for i in bad[:5]]
    assert np.linalg.norm(gg - go) <= 1e-3 * np.linalg.norm(go)
    assert abs(loss.item() - L) <= 1e-5 * L + 1e-7


def test_adam_matches_oracle(torch):
    rng = np.random.default_rng(5)
    w = rng.normal(size=M.NW).astype(np.float32)
    m = (rng.normal(size=M.NW) * 1e-3).astype(np.float32)
    v = (rng.uniform(0, 1e-6, M.NW)).astype(np.float32)
    g = (rng.normal(size=M.NW) * 1e-3).astype(np.float32)
    wd, md, vd = _dev(torch, w), _dev(torch, m), _dev(torch, v)
    q.qym_mlp_adam_dev(wd, md, vd, _dev(torch, g), 3, 1e-3)
    torch.cuda.synchronize()
    # the same float32 constants on both sides
    b1, b2, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-8))
    wo, mo, vo = M.adam(w, m, v, g.astype(np.float64), 3, float(np.float32(1e-3)), b1, b2, eps)
    upd = np.abs(wo - w)
    assert np.all(np.abs(wd.cpu().numpy() - wo) <= 2.0 ** -23 * np.abs(wo) + 1e-5 * upd + 1e-12)
    # float32 rounding of each moment update, relative to its terms
    assert np.all(np.abs(md.cpu().numpy() - mo) <= 2e-7 * (np.abs(m) + np.abs(g)))
    assert np.all(np.abs(vd.cpu().numpy() - vo) <= 2e-7 * (np.abs(v) + g.astype(np.float64) ** 2))
    assert np.array_equal(wd.cpu().numpy()[M.NW - M.N_FROZEN:], w[M.NW - M.N_FROZEN:])


def test_training_run_matches_oracle(torch):
    """24 Adam steps (3 epochs of 8 minibatches, the last ragged) on the GPU
    against the reference loop with the same bf16 operands: the same
    per-step losses to 1e-3, the same weight change to 1e-2."""
    rows = W.mlp_rows_synthetic(2000, 6)
    w0 = _weights(3)
    wd = _dev(torch, w0)
    md = torch.zeros(M.NW, dtype=torch.float32, device="cuda")
    vd = torch.zeros_like(md)
    steps = 3 * 8
    losses = torch.empty(steps, dtype=torch.float32, device="cuda")
    work = torch.empty(q.qym_mlp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    q.qym_mlp_train_dev(wd, md, vd, 0, _dev(torch, rows), len(rows), 256, 3, 3e-3, 1e-4, losses, work)
    torch.cuda.synchronize()
    wo, Lo = M.train(w0, rows, 256, 3, 3e-3, 1e-4, emulate=True)
    Lg = losses.cpu().numpy()
    assert len(Lo) == steps
    assert np.all(np.abs(Lg - Lo) <= 1e-3 * Lo), np.abs(Lg / Lo - 1).max()
    assert Lo[-1] < 0.5 * Lo[0]
    wg = wd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(wg - wo) <= 1e-2 * np.linalg.norm(wo - w0.astype(np.float64))


def test_kepler_learned_guess_and_log_rows(torch, oracle):
    """The Kepler kernel's fused guess equals the reference network's guess
    (bf16 operands) within the output envelope; the solve from it reaches the
    same root as the oracle from the standard guess; the training rows it
    logs equal the oracle's rows for the oracle's roots."""
    n = 4096 + 77
    qq, vv, dt = W.test_particles(n, seed=12)
    # 40 of them on unbound orbits (1.5 x the escape speed): outside the
    # network's domain
    qq, vv = qq.copy(), vv.copy()
    r = np.linalg.norm(qq[:40], axis=1)
    vv[:40] *= (1.5 * np.sqrt(2.0 / r) / np.linalg.norm(vv[:40], axis=1))[:, None]
    unb = ~M.bound(qq, vv, 1.0)
    assert unb[:40].all() and not unb[40:].any()
    w = _weights(4)
    q0, v0 = _soa(torch, qq), _soa(torch, vv)
    q1, v1 = torch.empty_like(q0), torch.empty_like(v0)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    x0 = torch.empty_like(x)
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    log = torch.full((n, 5), float("nan"), dtype=torch.float32, device="cuda")
    q.qym_kepler_drift_dev(n, q0, v0, q1, v1, 1.0, dt, q.QYM_SOLVER_NEWTON, q.QYM_GUESS_MLP,
                           _dev(torch, w), 50, x_out=x, x0_out=x0, iters=it, log_rows=log,
                           status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    # the guess
    u = M.features(qq, vv, dt, 1.0)
    tol_y = M.y_tolerance(w, u, rel=2e-5, near=2e-5)
    xs, sg = M.x_std(qq, dt, 1.0), M.sigma(qq, dt, 1.0)
    xg = M.guess(w, qq, vv, dt, 1.0, emulate=True)
    tol_x = np.abs(xs) * sg * float(w[M.OFF_OSD]) * tol_y + 1e-13 * np.abs(xg)
    x0g = x0.cpu().numpy()
    assert np.all(np.abs(x0g - xg) <= tol_x)
    assert np.all(np.abs(x0g[unb] - xs[unb]) <= 4e-16 * np.abs(xs[unb]))
    # the root and the state
    r1, s1, xr, _, bad = oracle.kepler_drift(qq, vv, 1.0, dt, solver=1)
    assert bad == 0
    xx = x.cpu().numpy()
    dxt, dqt = _root_tolerance(qq, vv, dt, xr, r1)
    assert np.all(np.abs(xx - xr) <= dxt + 2e-15 * np.abs(xr))
    qg = q1.cpu().numpy().T
    floor = 2e-15 * (np.linalg.norm(r1, axis=1) + np.linalg.norm(qq, axis=1))
    assert np.all(np.linalg.norm(qg - r1, axis=1) <= dqt + floor)
    # the training rows
    lo = M.log_rows(qq, vv, dt, 1.0, xr).astype(np.float64)
    lg = log.cpu().numpy().astype(np.float64)
    assert np.isnan(lg[unb]).all() and np.isfinite(lg[~unb]).all()
    lo, lg, sb = lo[~unb], lg[~unb], sg[~unb]
    assert np.all(np.abs(lg[:, :4] - lo[:, :4]) <= 2.0 ** -22 * np.abs(lo[:, :4]) + 1e-30)
    assert np.all(np.abs(lg[:, 4] - lo[:, 4]) <= 2.0 ** -21 * np.abs(lo[:, 4]) + 1e-9 / sb)


def test_step_with_learned_guess_and_log(torch):
    """qym_step with QYM_GUESS_MLP: refused without a network; with one, the
    plain step gives the positions of the standard guess (same Kepler roots)
    to 1e-12; the log holds one row per body and step across calls, stars
    left untouched, nothing past its capacity."""
    w = W.subsample(W.disk_260(), 100, seed=2)
    R = len(w.m)
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64, encounters=0,
                       guess=q.QYM_GUESS_MLP)
    with pytest.raises(q.QymError) as e:
        sim.step(w.tau, 2)
    assert e.value.status == q.QYM_EINVAL
    sim.set_mlp(_weights(5))
    cap = 4 * R + 7
    log = torch.full((cap + 50, 5), float("nan"), dtype=torch.float32, device="cuda")
    sim.set_kepler_log(log, cap)
    sim.step(w.tau, 3)
    sim.step(w.tau, 2)
    qa, va = sim.state()
    sim.close()
    ref = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64, encounters=0)
    ref.step(w.tau, 3)
    ref.step(w.tau, 2)
    qb, vb = ref.state()
    ref.close()
    nb = np.linalg.norm(qb, axis=1)
    assert np.all(np.linalg.norm(qa - qb, axis=1) <= 1e-12 * np.maximum(nb, 1e-300))
    lg = log.cpu().numpy()
    fin = np.isfinite(lg).all(axis=1)
    # steps 0..3 complete (4 R slots, star rows skipped), 7 rows of step 4
    expect = np.zeros(cap + 50, bool)
    for s in range(5):
        for k in range(1, R):
            if s * R + k < cap:
                expect[s * R + k] = True
    assert np.array_equal(fin, expect)
    assert np.all(lg[fin, 1] > 0)


def test_learned_guess_gain_on_test_particles(torch, oracle):
    """Trained on about 1e7 logged solves, the learned guess cuts the Newton
    iterations on the 1,048,576 test particles of seed 4; every solve still
    meets the 1e-14 residual (checked by the oracle on a sample) and both
    guesses reach the same state."""
    from paper_1007_3458_gb300 import guess as G
    wts, losses, nrows = G.train_default()
    assert nrows > 9_000_000
    assert losses[-100:].mean() < 0.05 * losses[:10].mean()
    qq, vv, dt = W.test_particles(1 << 20, seed=4)
    n = len(qq)
    q0, v0 = _soa(torch, qq), _soa(torch, vv)
    wd = torch.from_numpy(wts).cuda()
    res = {}
    # the last two arms take FP32 Newton steps before the FP64 ones
    arms = (("standard", q.QYM_GUESS_STANDARD, q.QYM_SOLVER_NEWTON),
            ("mlp", q.QYM_GUESS_MLP, q.QYM_SOLVER_NEWTON),
            ("standard32", q.QYM_GUESS_STANDARD, q.QYM_SOLVER_NEWTON32),
            ("mlp32", q.QYM_GUESS_MLP, q.QYM_SOLVER_NEWTON32))
    for name, guess, solver in arms:
        q1, v1 = torch.empty_like(q0), torch.empty_like(v0)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        q.qym_kepler_drift_dev(n, q0, v0, q1, v1, 1.0, dt, solver, guess,
                               wd if guess == q.QYM_GUESS_MLP else None, 50, x_out=x, iters=it,
                               status=st)
        torch.cuda.synchronize()
        assert st.item() == 0
        res[name] = (q1.cpu().numpy().T, x.cpu().numpy(), it.cpu().numpy())
    it_s, it_m = res["standard"][2].mean(), res["mlp"][2].mean()
    print(f"\nrows {nrows}, loss first {losses[:10].mean():.4g} last {losses[-100:].mean():.4g}; "
          f"Newton iterations: standard {it_s:.3f} (max {res['standard'][2].max()}), "
          f"learned {it_m:.3f} (max {res['mlp'][2].max()})")
    for name in res:
        print(f"  histogram {name:10s}", np.bincount(res[name][2])[:14])
    assert it_m < 0.85 * it_s
    # every root meets |F| <= 1e-14 (sum of |terms|), re-evaluated by the
    # oracle (whose F carries a few more ulp of that sum: eps), unless no
    # double next to it meets 1e-14 either: after a step at the rounding
    # level the solver evaluates once more and keeps the better of the two
    # points, which can sit above 1e-14 only where a step of one ulp in x
    # moves F by more than that (r1 >> r0)
    eps = 8 * 2.0 ** -53
    for name in res:
        x = res[name][1]
        r = oracle.kepler_residuals(qq, vv, 1.0, dt, x)
        over = np.nonzero(r > 1e-14 + eps)[0]
        print(f"  {name}: max residual {r.max():.3g}, {len(over)} roots above 1e-14")
        for d in (np.inf, -np.inf):
            rn = oracle.kepler_residuals(qq[over], vv[over], 1.0, dt, np.nextafter(x[over], d))
            assert np.all(rn > 1e-14 - eps), (name, over[rn <= 1e-14 - eps], rn[rn <= 1e-14 - eps])
    # every root meets the residual: the states agree within its conditioning
    qs = res["standard"][0]
    _, dqt = _root_tolerance(qq, vv, dt, res["standard"][1], qs)
    floor = 2e-15 * (np.linalg.norm(qs, axis=1) + np.linalg.norm(qq, axis=1))
    for name in ("mlp", "standard32", "mlp32"):
        assert np.all(np.linalg.norm(qs - res[name][0], axis=1) <= dqt + floor), name
