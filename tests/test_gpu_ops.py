"""GPU parity of the individual operators, each called through the C ABI on
device buffers and compared element by element with the oracle on the same
seeded inputs: E_Kep (Appendix), E_Int accelerations in FP64 and mixed
precision (Eq. 4), the rigorous encounter test (Sec. 2.4) and the energy
(Eqs. 2-4)."""
import math

import numpy as np
import pytest

import paper_1007_3458_gb300 as q
from paper_1007_3458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return t


def _soa(t, a):
    return t.tensor(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T), device="cuda")


def _aos(x):
    return x.cpu().numpy().T.copy()


# ------------------------------------------------------------------ E_Kep
def _orbits(n, seed, emax=0.95, amin=0.3, amax=50.0):
    rng = np.random.default_rng(seed)
    a = np.exp(rng.uniform(math.log(amin), math.log(amax), n))
    e = rng.uniform(0, emax, n)
    qq, vv = W.elements_to_cartesian(1.0, a, e, rng.uniform(0, math.pi, n),
                                     rng.uniform(0, 6.28, n), rng.uniform(0, 6.28, n),
                                     rng.uniform(0, 6.28, n))
    return qq, vv, a, e


def _kepler_gpu(torch, qq, vv, mu, dt, solver=0, guess=0, max_iter=50):
    n = len(qq)
    q0, v0 = _soa(torch, qq), _soa(torch, vv)
    q1, v1 = torch.empty_like(q0), torch.empty_like(v0)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    q.qym_kepler_drift_dev(n, q0, v0, q1, v1, mu, dt, solver, guess, None, max_iter, x_out=x,
                           iters=it, status=st)
    torch.cuda.synchronize()
    return _aos(q1), _aos(v1), x.cpu().numpy(), it.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("solver,guess", [(0, 0), (0, 1), (1, 0)])
@pytest.mark.parametrize("dt", [0.01, 1.756203, -0.7, 25.0])
def test_kepler_matches_oracle(torch, oracle, solver, guess, dt):
    qq, vv, a, e = _orbits(3000 + 37, seed=int(abs(dt) * 100) + solver)
    q1, v1, x, it, st = _kepler_gpu(torch, qq, vv, 1.0, dt, solver, guess)
    r1, u1, xr, itr, bad = oracle.kepler_drift(qq, vv, 1.0, dt, solver, guess)
    ok = np.ones(len(qq), bool)
    if solver == 1:
        # plain Newton is not globally convergent: where either side hit the
        # iteration cap there is no root to compare (the root is unique, so
        # wherever both converged they must agree)
        ok = (itr < 50) & (it < 50)
        assert ok.mean() > 0.5
    else:
        assert bad == 0 and st == 0
    # both sides stop at the same residual tolerance, whose phase error grows
    # with the number of orbits covered by dt, and near pericentre as 1/(1-e)
    scale = (1.0 + abs(dt) / (2 * math.pi * a ** 1.5)) / (1.0 - e)
    dq = np.linalg.norm(q1 - r1, axis=1) / np.linalg.norm(r1, axis=1)
    dv = np.linalg.norm(v1 - u1, axis=1) / np.linalg.norm(u1, axis=1)
    assert np.all(dq[ok] <= 1e-12 * scale[ok]), dq[ok].max()
    assert np.all(dv[ok] <= 1e-12 * scale[ok]), dv[ok].max()
    # same iteration counts except where a stopping test sits at rounding
    # level (more often for Newton far from the root)
    assert np.mean(it[ok] == itr[ok]) > (0.99 if solver == 0 else 0.95)


@pytest.mark.parametrize("dt", [0.01, 1.756203, -0.7, 25.0])
def test_kepler_newton32_matches_oracle(torch, oracle, dt):
    """QYM_SOLVER_NEWTON32 (FP32 Newton steps, then FP64 Laguerre under the same
    residual test and bracket) reaches the oracle's root: the states agree
    wherever both converged, within the tolerance of the FP64 solvers; 40
    hyperbolic rows among them."""
    qq, vv, a, e = _orbits(3000 + 37, seed=int(abs(dt) * 100) + 7)
    r = np.linalg.norm(qq[:40], axis=1)
    vv = vv.copy()
    vv[:40] *= (1.5 * np.sqrt(2.0 / r) / np.linalg.norm(vv[:40], axis=1))[:, None]
    q1, v1, x, it, st = _kepler_gpu(torch, qq, vv, 1.0, dt, q.QYM_SOLVER_NEWTON32, 0)
    r1, u1, xr, itr, bad = oracle.kepler_drift(qq, vv, 1.0, dt, 0, 0)
    assert bad == 0
    ok = it < 50
    assert ok.mean() > 0.5 and ok[:40].all()
    if abs(dt) < 2.0:
        assert ok.all() and st == 0
    # the bound rows as in the FP64 solvers' test; the hyperbolic rows by the
    # relative state error
    scale = (1.0 + abs(dt) / (2 * math.pi * a ** 1.5)) / (1.0 - e)
    scale[:40] = 1.0
    dq = np.linalg.norm(q1 - r1, axis=1) / np.linalg.norm(r1, axis=1)
    dv = np.linalg.norm(v1 - u1, axis=1) / np.linalg.norm(u1, axis=1)
    assert np.all(dq[ok] <= 1e-12 * scale[ok]), dq[ok].max()
    assert np.all(dv[ok] <= 1e-12 * scale[ok]), dv[ok].max()


def test_kepler_unbound_and_star_rows(torch, oracle):
    """Hyperbolic and near-parabolic orbits stay finite (Appendix: universal
    variables); a row at the origin (a star row) is left at zero."""
    qq = np.array([[1.0, 0.2, 0.0], [2.0, -1.0, 0.3], [0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    vv = np.array([[0.0, 1.8, 0.1], [-1.0, 0.2, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 1.6329931618]])
    q1, v1, x, it, st = _kepler_gpu(torch, qq, vv, 1.0, 3.0)
    r1, u1, *_ = oracle.kepler_drift(qq[[0, 1, 3]], vv[[0, 1, 3]], 1.0, 3.0)
    assert st == 0 and np.all(np.isfinite(q1))
    assert np.all(q1[2] == 0) and np.all(v1[2] == 0)
    assert np.allclose(q1[[0, 1, 3]], r1, rtol=1e-12, atol=0)


def test_kepler_full_size_test_particles_sampled(torch, oracle):
    """1,048,576 massless test particles (a log-uniform 0.5-50, e up to 0.9),
    dt = P(a=5)/40: sampled bodies against the oracle, all converged."""
    qq, vv, dt = W.test_particles()
    q1, v1, x, it, st = _kepler_gpu(torch, qq, vv, 1.0, dt)
    assert st == 0
    rng = np.random.default_rng(0)
    sel = rng.choice(len(qq), 4096, replace=False)
    r1, u1, *_ = oracle.kepler_drift(qq[sel], vv[sel], 1.0, dt)
    dq = np.linalg.norm(q1[sel] - r1, axis=1) / np.linalg.norm(r1, axis=1)
    assert dq.max() <= 1e-11


# ------------------------------------------------------------------ E_Int
def _accel_gpu(torch, m, qq, prec):
    rows = len(m)
    md = torch.tensor(m, dtype=torch.float64, device="cuda")
    qd = _soa(torch, qq)
    ad = torch.empty_like(qd)
    nb = q.qym_accel_workspace_bytes(rows, prec)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    q.qym_accel_dev(rows, md, qd, ad, 1.0, prec, work)
    torch.cuda.synchronize()
    return _aos(ad)


def _rel_err(a, ref):
    n = np.linalg.norm(ref, axis=1)
    return np.linalg.norm(a - ref, axis=1)[1:] / n[1:]


@pytest.mark.parametrize("nbody", [1, 2, 129, 257, 1000, 4099])
def test_accel_ragged_sizes(torch, oracle, nbody):
    """Sizes around the tile (256) and i-block (256 rows) edges, including a
    single body (zero acceleration)."""
    if nbody == 1:
        w = W.Workload("one", np.array([1.0, 1e-3]), np.array([[0, 0, 0], [5.0, 0, 0]]),
                       np.zeros((2, 3)), np.array([0, 2]), 1.0, 1)
    else:
        w = W.subsample(W.disk_16384(), nbody, seed=nbody)
    a64 = _accel_gpu(torch, w.m, w.q, q.QYM_KICK_FP64)
    amx = _accel_gpu(torch, w.m, w.q, q.QYM_KICK_MIXED)
    ref = oracle.accel_int(w.m, w.q)
    assert np.all(a64[0] == 0) and np.all(amx[0] == 0)
    if nbody == 1:
        assert np.all(a64 == 0) and np.all(amx == 0)
        return
    assert _rel_err(a64, ref).max() <= 1e-12
    assert _rel_err(amx, ref).max() <= 1e-6


@pytest.mark.parametrize("name", ["disk_260", "disk_16384"])
def test_accel_full_disks(torch, oracle, name):
    """The 260- and 16384-body disks: FP64 within 1e-12, mixed within 1e-6
    relative per body (the mixed-precision accuracy target)."""
    w = getattr(W, name)()
    ref = oracle.accel_int(w.m, w.q)
    assert _rel_err(_accel_gpu(torch, w.m, w.q, q.QYM_KICK_FP64), ref).max() <= 1e-12
    assert _rel_err(_accel_gpu(torch, w.m, w.q, q.QYM_KICK_MIXED), ref).max() <= 1e-6


def test_accel_dense_disk_sampled(torch, oracle):
    """The 262144-body embryo disk: sampled rows against the oracle."""
    w = W.disk_262144()
    amx = _accel_gpu(torch, w.m, w.q, q.QYM_KICK_MIXED)
    rng = np.random.default_rng(1)
    sel = np.concatenate([np.arange(1, 9), rng.choice(np.arange(65, len(w.m)), 56, replace=False)])
    ref = oracle.accel_rows(w.m, w.q, sel)
    err = np.linalg.norm(amx[sel] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-6


# ------------------------------------------------------------------ Sec. 2.4
def test_encounter_test_bit_exact(torch, oracle):
    """Same FP64 inputs on both sides: the interpolated minimum separation is
    bit-identical and so is every flag."""
    rng = np.random.default_rng(4)
    n = 400
    m = np.concatenate([[1.0], np.full(n, 1e-5)])
    qq, vv = W.elements_to_cartesian(1.0, rng.uniform(0.9, 1.1, n), rng.rayleigh(0.05, n),
                                     rng.rayleigh(0.02, n), rng.uniform(0, 6.28, n),
                                     rng.uniform(0, 6.28, n), rng.uniform(0, 6.28, n))
    q0 = np.concatenate([[[0, 0, 0]], qq])
    v0 = np.concatenate([[[0, 0, 0]], vv])
    tau = 0.2
    q1 = q0.copy()
    v1 = v0.copy()
    q1[1:], v1[1:], *_ = oracle.kepler_drift(q0[1:], v0[1:], 1.0, tau)
    rH = oracle.hill_radii(m, q0, v0)
    pairs = np.array([(i, j) for i in range(1, n + 1) for j in range(i + 1, n + 1)], np.int32)
    t = torch
    dq0, dv0, dq1, dv1 = (_soa(t, x) for x in (q0, v0, q1, v1))
    drH = t.tensor(rH, device="cuda")
    dp = t.tensor(pairs, device="cuda")
    d2 = t.empty(len(pairs), dtype=t.float64, device="cuda")
    fl = t.empty(len(pairs), dtype=t.int32, device="cuda")
    q.qym_encounter_test_dev(n + 1, dq0, dv0, dq1, dv1, drH, tau, 3.0, len(pairs), dp, d2, fl)
    t.cuda.synchronize()
    d2 = d2.cpu().numpy()
    ref = np.array([oracle.pair_dmin2(q0[i] - q0[j], v0[i] - v0[j], q1[i] - q1[j], v1[i] - v1[j],
                                      tau) for i, j in pairs])
    assert np.array_equal(d2, ref)
    ref_pairs, _, _ = oracle.encounters(q0, v0, q1, v1, rH, tau, 3.0)
    got = pairs[fl.cpu().numpy() == 1]
    assert len(ref_pairs) > 0
    assert np.array_equal(got, ref_pairs)


# ------------------------------------------------------------------ Sec. 2.1
def test_transition_matches_oracle(torch, oracle):
    """The transition function the Hermite sub-integrator evaluates (sin and
    cos of pi y / 2 by folded Taylor polynomials) against the oracle's libm
    sin/cos: K, K', K'' within a few ulp of their scales across the whole
    zone, the flat parts exact, and the zone's edges at y = 0 and y = 1."""
    rc = 0.37
    rng = np.random.default_rng(3)
    s = np.concatenate([np.linspace(0.0, 1.2 * rc, 20001), rng.uniform(0, rc, 20000),
                        [0.1 * rc / 1.1, rc, rc * (1 - 1e-15), 0.0]])
    n = len(s)
    sd = torch.from_numpy(s).cuda()
    K, Kp, Kpp = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    q.qym_transition_dev(n, sd, rc, K, Kp, Kpp)
    torch.cuda.synchronize()
    ref = np.array([oracle.transition(x, rc) for x in s])
    c = 0.5 * math.pi * 1.1 / rc
    K, Kp, Kpp = K.cpu().numpy(), Kp.cpu().numpy(), Kpp.cpu().numpy()
    # a few ulp: the polynomial's rounding plus one or two products by c
    assert np.all(np.abs(K - ref[:, 0]) <= 4e-16)
    assert np.all(np.abs(Kp - ref[:, 1]) <= 6e-16 * c)
    assert np.all(np.abs(Kpp - ref[:, 2]) <= 8e-16 * c * c)
    flat = (1.1 * s / rc - 0.1 <= 0) | (1.1 * s / rc - 0.1 >= 1)
    assert np.array_equal(K[flat], ref[flat, 0]) and np.all(Kp[flat] == 0) and np.all(Kpp[flat] == 0)


# ------------------------------------------------------------------ energy
@pytest.mark.parametrize("name", ["disk_260", "disk_16384"])
def test_energy_matches_oracle(torch, oracle, name):
    w = getattr(W, name)()
    vd = oracle.helio_to_dh(w.m, w.v)
    ref = oracle.energy(w.m, w.q, vd)
    t = torch
    rows = len(w.m)
    md = t.tensor(w.m, device="cuda")
    E = t.zeros(1, dtype=t.float64, device="cuda")
    work = t.empty(q.qym_energy_workspace_bytes(rows), dtype=t.uint8, device="cuda")
    q.qym_energy_dev(rows, md, _soa(t, w.q), _soa(t, vd), 1.0, E, work)
    assert abs(E.item() - ref) <= 1e-13 * abs(ref)


def test_kepler_unbound_parity(torch, oracle):
    """Near-parabolic and strongly hyperbolic orbits over long steps (the
    bracketed, safeguarded solve): all converge on both sides and agree."""
    rng = np.random.default_rng(1)
    n = 5000
    r = rng.uniform(0.3, 3, n)
    qq = np.zeros((n, 3))
    qq[:, 0] = r
    f = np.where(rng.random(n) < 0.5, 1 + rng.uniform(-1e-3, 1e-3, n), rng.uniform(1.0, 3.0, n))
    ang = rng.uniform(0, math.pi, n)
    vv = np.stack([np.cos(ang), np.sin(ang), np.zeros(n)], 1) * (f * np.sqrt(2 / r))[:, None]
    # orbits aimed at the star (periapsis below 1e-3) pass through the
    # singularity and are left out of the comparison
    h = np.linalg.norm(np.cross(qq, vv), axis=1)
    alpha = 2 / r - np.sum(vv * vv, 1)
    p = h * h
    rp = p / (1 + np.sqrt(np.maximum(0, 1 - p * alpha)))
    ok = rp > 1e-3
    for dt in (1.76, 20.0, -5.0):
        q1, v1, x, it, st = _kepler_gpu(torch, qq, vv, 1.0, dt)
        r1, u1, xr, itr, bad = oracle.kepler_drift(qq, vv, 1.0, dt)
        assert bad == 0 and np.all(np.isfinite(q1[ok]))
        dq = np.linalg.norm(q1 - r1, axis=1) / np.linalg.norm(r1, axis=1)
        dq[~ok] = 0.0
        k = int(np.argmax(dq))
        assert dq[k] <= 1e-11, (dt, k, dq[k], r[k], f[k], ang[k], rp[k], q1[k], r1[k], x[k], xr[k],
                                it[k], itr[k])
