"""Pins for the oracle's encounter machinery: the rigorous minimum-separation
test (Sec. 2.4), encounter sets and r_crit (Sec. 2.3 item 4, Eq. 9), the
transition function (Sec. 2.1), the K corrections (Sec. 2.3 items 5 and 7) and
the Hermite sub-integrator (Sec. 2.2).

References used: exact minima of polynomials, densely sampled true Kepler
trajectories, networkx connected components, finite-difference derivatives of
potentials written from Eqs. 6-7, conservation of H'_Kep, and the convergence
order of a 4th-order method."""
import math

import numpy as np
import pytest

from paper_1007_3458_gb300 import workloads as W


# ------------------------------------------------------------ rigorous test
def test_dmin_exact_for_linear_motion(oracle):
    """Straight-line relative motion makes d^2(t) quadratic, which the cubic
    interpolant reproduces exactly: the minimum is the textbook closest
    approach t* = clamp(-dq.dv/|dv|^2, 0, tau)."""
    rng = np.random.default_rng(0)
    for _ in range(500):
        dq0 = rng.normal(0, 1, 3)
        dv0 = rng.normal(0, 1, 3)
        tau = rng.uniform(0.05, 2.0)
        dq1 = dq0 + tau * dv0
        ts = np.clip(-(dq0 @ dv0) / (dv0 @ dv0), 0, tau)
        ref = np.sum((dq0 + ts * dv0) ** 2)
        got = oracle.pair_dmin2(dq0, dv0, dq1, dv0, tau)
        assert abs(got - ref) <= 1e-12 * (dq0 @ dq0 + tau ** 2 * (dv0 @ dv0))


def test_dmin_of_a_given_cubic(oracle):
    """End values and slopes taken from a known cubic g(t) > 0: the test
    returns its minimum over [0, tau] (dense sampling of g)."""
    rng = np.random.default_rng(1)
    for _ in range(300):
        tau = rng.uniform(0.1, 1.5)
        # g(t) = c0 + c1 t + c2 t^2 + c3 t^3, shifted to stay positive
        c = rng.normal(0, 1, 4)
        t = np.linspace(0, tau, 20001)
        g = c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3
        c[0] += 0.1 - g.min()
        g = c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3
        g0, g1 = g[0], g[-1]
        s0, s1 = c[1], c[1] + 2 * c[2] * tau + 3 * c[3] * tau ** 2
        dq0 = np.array([math.sqrt(g0), 0, 0])
        dv0 = np.array([s0 / (2 * math.sqrt(g0)), 0, 0])
        dq1 = np.array([0, math.sqrt(g1), 0])
        dv1 = np.array([0, s1 / (2 * math.sqrt(g1)), 0])
        got = oracle.pair_dmin2(dq0, dv0, dq1, dv1, tau)
        assert abs(got - g.min()) <= 1e-7 * (1 + abs(g).max())


def _crowded(n=15, seed=2, m=1e-4):
    rng = np.random.default_rng(seed)
    mass = np.concatenate([[1.0], np.full(n, m)])
    q, v = W.elements_to_cartesian(1.0 + m, rng.uniform(0.9, 1.1, n), rng.rayleigh(0.05, n),
                                   rng.rayleigh(0.02, n), rng.uniform(0, 6.28, n),
                                   rng.uniform(0, 6.28, n), rng.uniform(0, 6.28, n))
    return mass, np.concatenate([[[0, 0, 0]], q]), np.concatenate([[[0, 0, 0]], v])


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_encounter_list_brute_force_small_n(oracle, seed):
    """N <= 16: every pair whose true minimum separation over [0, tau]
    (Kepler trajectories sampled densely) is below 0.9 a_E (r_H,i + r_H,j)
    is flagged, none above 1.1 times it is, and the list is i < j sorted."""
    m, q0, v0 = _crowded(15, seed)
    tau, a_E = 0.3, 3.0
    q1 = q0.copy()
    v1 = v0.copy()
    q1[1:], v1[1:], *_ = oracle.kepler_drift(q0[1:], v0[1:], 1.0, tau)
    rH = oracle.hill_radii(m, q0, v0)
    pairs, d2, thr2 = oracle.encounters(q0, v0, q1, v1, rH, tau, a_E)
    ts = np.linspace(0, tau, 801)
    traj = np.stack([oracle.kepler_drift(q0[1:], v0[1:], 1.0, t)[0] for t in ts])  # [T, n, 3]
    flagged = {tuple(p) for p in pairs}
    n = len(m) - 1
    seen_close = 0
    for i in range(1, n + 1):
        for j in range(i + 1, n + 1):
            dmin = np.linalg.norm(traj[:, i - 1] - traj[:, j - 1], axis=1).min()
            R = a_E * (rH[i] + rH[j])
            if dmin < 0.9 * R:
                seen_close += 1
                assert (i, j) in flagged
            if dmin > 1.1 * R:
                assert (i, j) not in flagged
    assert seen_close > 0
    assert all(i < j for i, j in pairs)
    assert [tuple(p) for p in pairs] == sorted(flagged)
    # the selected-rows variant finds the same pairs for those rows
    # rows taken as the lower and as the upper index of a pair, so that
    # partners on both sides of a selected row count
    sel = np.unique(np.concatenate([pairs[:2, 0], pairs[-2:, 1]])) if len(pairs) else np.array([1])
    assert len(pairs) == 0 or any(p[1] in sel and p[0] not in sel for p in pairs)
    pr, _, _ = oracle.encounters_rows(q0, v0, q1, v1, rH, tau, a_E, sel)
    want = {tuple(p) for p in pairs if p[0] in sel or p[1] in sel}
    assert {tuple(p) for p in pr} == want


def test_hill_radius_definition(oracle):
    """r_H = |Q| (m / 3 m0)^(1/3): on a circular orbit this is the
    semi-major-axis form of Eq. 9's R_MH; it stays finite on a near-parabolic
    orbit (where 1/alpha diverges); massless bodies have zero radius."""
    m = np.array([1.0, 3e-3, 0.0, 3e-3])
    q = np.array([[0, 0, 0], [2.0, 0, 0], [0, 3.0, 0], [0, 0, 1.5]])
    v = np.array([[0, 0, 0], [0, math.sqrt(0.5), 0], [-math.sqrt(1 / 3), 0, 0],
                  [math.sqrt(2 / 1.5) * (1 - 1e-12), 0, 0]])
    rH = oracle.hill_radii(m, q, v)
    assert abs(rH[1] - 2.0 * 0.1) <= 1e-15
    assert abs(rH[3] - 1.5 * 0.1) <= 1e-15
    assert rH[2] == 0.0 and rH[0] == 0.0


def test_sets_are_connected_components(oracle):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(3)
    rows = 300
    pairs = np.unique(np.sort(rng.integers(1, rows, (120, 2)), axis=1), axis=0)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    rH = rng.uniform(0, 1, rows)
    set_of, start, members, rcrit = oracle.sets(rows, pairs, rH, 1.5)
    Gr = nx.Graph()
    Gr.add_edges_from(map(tuple, pairs))
    comps = sorted((sorted(c) for c in nx.connected_components(Gr)), key=lambda c: c[0])
    assert len(comps) == len(start) - 1
    for s, c in enumerate(comps):
        assert list(members[start[s]:start[s + 1]]) == c
        assert rcrit[s] == 1.5 * max(rH[c])
        assert np.all(set_of[c] == s)
    assert np.all(set_of[np.setdiff1d(np.arange(rows), pairs.ravel())] == -1)


# ------------------------------------------------------------ transition function
def test_transition_function_values_and_derivatives(oracle):
    """K = 0 for s <= r_crit/11, 1 for s >= r_crit, sin(pi y / 2) between
    (Sec. 2.1); K' and K'' are its derivatives in s (central differences)."""
    rc = 0.37
    assert oracle.transition(rc / 11 * 0.999, rc)[0] == 0.0
    assert oracle.transition(rc * 1.0001, rc)[0] == 1.0
    assert abs(oracle.transition(rc * 6 / 11, rc)[0] - math.sin(math.pi / 4)) < 1e-15
    h = 1e-7
    for s in np.linspace(rc / 11 * 1.01, rc * 0.99, 50):
        K, Kp, Kpp = oracle.transition(s, rc)
        Kn = (oracle.transition(s + h, rc)[0] - oracle.transition(s - h, rc)[0]) / (2 * h)
        Kpn = (oracle.transition(s + h, rc)[1] - oracle.transition(s - h, rc)[1]) / (2 * h)
        assert abs(Kn - Kp) <= 1e-6 * (abs(Kp) + 1)
        assert abs(Kpn - Kpp) <= 1e-5 * (abs(Kpp) + 1)


def _U_K(m, q, rc, weight, eps=0.0):
    """Pair potential of the set with weight(K) (Eqs. 6-7), via oracle.transition;
    with eps > 0 every pair distance is the softened sqrt(d^2 + eps^2)."""
    U = 0.0
    for i in range(len(m)):
        for j in range(i + 1, len(m)):
            d = math.sqrt(float(np.sum((q[i] - q[j]) ** 2)) + eps * eps)
            U -= m[i] * m[j] * weight(d) / d
    return U


def test_kcorr_turns_full_kick_into_K_weighted_kick(oracle):
    """Kick with the full pair force, then subtract (1-K) part: the net velocity
    change is dt times -grad(U_K)/m with U_K = -sum G m_i m_j K(q)/q (H'_Int,
    Eq. 7), here by central differences."""
    m = np.array([1.0, 2e-4, 5e-5, 1e-4, 0.0])
    q = np.array([[0, 0, 0], [1.0, 0, 0], [1.03, 0.02, 0], [0.98, -0.03, 0.01], [1.01, 0.01, -0.01]])
    v = np.zeros_like(q)
    rc, dt = 0.06, 0.1
    members = np.array([1, 2, 3, 4])
    vk = oracle.kick(m, q, v, dt)
    vc = oracle.kcorr(members, m, q, vk, rc, dt)
    Kw = lambda d: oracle.transition(d, rc)[0]
    h = 1e-7
    for i in members:
        if m[i] == 0:
            continue
        for k in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, k] += h
            qm[i, k] -= h
            g = (_U_K(m[1:], qp[1:], rc, Kw) - _U_K(m[1:], qm[1:], rc, Kw)) / (2 * h)
            assert abs(vc[i, k] - (-dt * g / m[i])) <= 1e-6 * (np.abs(vk[i]).max() + 1e-9)


# ------------------------------------------------------------ Hermite
def _phi_set(mm, x, rc, m0=1.0, eps=0.0):
    """H'_Kep potential of a set: star term + (1-K)-weighted pairs (Eq. 6),
    every distance softened to sqrt(d^2 + eps^2) when eps > 0 (the Hermite
    smoothing of Sec. 2.4, reading R16)."""
    U = -np.sum(m0 * mm / np.sqrt(np.sum(x * x, 1) + eps * eps))
    return U + _U_K(mm, x, rc, lambda d: 1.0 - oracle_transition(d, rc), eps)


def oracle_transition(d, rc):
    import oracle as O
    return O.transition(d, rc)[0]


@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_hermite_force_and_jerk(oracle, eps):
    """Hermite acceleration = -grad(Phi')/m (Sec. 2.2 with Eq. 6) by central
    differences, with the smoothing eps either 0 or comparable to the pair
    separations (the potential then softened the same way); jerk = d a / dt
    along the velocities, by central differences of the acceleration at
    x +- h u."""
    rng = np.random.default_rng(5)
    k = 5
    mm = np.array([3e-4, 1e-4, 2e-5, 1e-5, 0.0])
    x = np.array([1.0, 0.2, 0.0]) + rng.normal(0, 0.02, (k, 3))
    u = np.array([-0.2, 1.0, 0.0]) + rng.normal(0, 0.05, (k, 3))
    rc = 0.04
    a, j = oracle.hermite_force(mm, x, u, rc, eps=eps)
    h = 1e-7
    for i in range(k - 1):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            g = (_phi_set(mm, xp, rc, eps=eps) - _phi_set(mm, xm, rc, eps=eps)) / (2 * h)
            assert abs(-g / mm[i] - a[i, c]) <= 1e-6 * np.abs(a[i]).max()
    hh = 1e-6
    ap, _ = oracle.hermite_force(mm, x + hh * u, u, rc, eps=eps)
    am, _ = oracle.hermite_force(mm, x - hh * u, u, rc, eps=eps)
    jn = (ap - am) / (2 * hh)
    assert np.all(np.abs(jn - j) <= 1e-5 * (np.abs(j).max(1, keepdims=True) + 1e-12))


def test_hermite_reduces_to_kepler_with_fourth_order_convergence(oracle):
    """With r_crit -> 0 the set members feel only the star: the Hermite result
    approaches the universal-variable Kepler solution, with global error
    falling as eta^2 (dt ~ eta^(1/2), 4th order)."""
    m = np.array([1.0, 1e-3, 1e-3])
    q, v = W.elements_to_cartesian(1.0, np.array([1.0, 1.5]), np.array([0.1, 0.3]),
                                   np.array([0.1, 0.2]), np.array([0.0, 1.0]), np.array([1.0, 2.0]),
                                   np.array([0.5, 2.5]))
    q = np.concatenate([[[0, 0, 0]], q])
    v = np.concatenate([[[0, 0, 0]], v])
    tau = 2.0
    qk, vk, *_ = oracle.kepler_drift(q[1:], v[1:], 1.0, tau)
    errs = []
    for eta in (0.02, 0.005):
        qh, vh, steps, st = oracle.hermite_set([1, 2], m, q, v, 1e-30, tau, eta=eta, eta_s=eta / 2)
        assert st == 0
        errs.append(np.abs(qh[1:] - qk).max())
    assert errs[1] < 1e-5
    assert errs[0] / errs[1] > 8.0


def test_hermite_conserves_Hprime_kep_through_encounter(oracle):
    """Two bodies approach inside the transition zone (r_crit/11 < s < r_crit,
    0 < K < 1): the Hermite keeps H'_Kep (Eq. 6 restricted to the set) with a
    4th-order error, falling as eta^2."""
    m = np.array([1.0, 1e-4, 3e-5])
    q = np.array([[0, 0, 0], [1.0, 0.0, 0.0], [1.0, 0.04, 0.0]])
    v = np.array([[0, 0, 0], [0.0, 1.0, 0.0], [-0.06, 0.95, 0.0]])
    rc = 0.1

    def H(qq, vv):
        return 0.5 * np.sum(m[1:] * np.sum(vv[1:] ** 2, 1)) + _phi_set(m[1:], qq[1:], rc)

    E0 = H(q, v)
    errs = []
    # individual block steps are powers of two of tau, so eta values 16x apart
    # (steps 4x apart, two levels) are compared
    for eta in (0.005, 0.0003):
        qh, vh, steps, st = oracle.hermite_set([1, 2], m, q, v, rc, 1.0, eta=eta, eta_s=eta / 2)
        assert st == 0 and steps > 10
        s = np.linalg.norm(qh[1] - qh[2])
        assert rc / 11 < s < rc and 0 < oracle.transition(s, rc)[0] < 1
        errs.append(abs(H(qh, vh) - E0) / abs(E0))
    assert errs[0] < 1e-7 and errs[1] < 1e-9
    assert errs[0] / errs[1] > 64.0


def test_transition_kinks_are_the_papers(oracle):
    """The sine transition of Sec. 2.1 has K'(0+) = (pi/2)(1.1/r_crit) while
    K' = 0 for y <= 0, so the (1-K)-weighted force jumps at s = r_crit/11 (the
    bracket 1 - K + s K' goes from 1 to 1 + pi/20); at s = r_crit the force is
    continuous but K'' jumps. Hermite accuracy is lower for steps that cross
    these radii."""
    rc = 0.2
    s0 = rc / 11
    lo = oracle.transition(s0 * (1 - 1e-12), rc)
    hi = oracle.transition(s0 * (1 + 1e-12), rc)
    br = lambda K, s: 1 - K[0] + s * K[1]
    assert abs(br(lo, s0) - 1.0) < 1e-12
    assert abs(br(hi, s0) - (1 + math.pi / 20)) < 1e-9
    below = oracle.transition(rc * (1 - 1e-12), rc)
    assert abs(br(below, rc)) < 1e-9 and below[2] < 0


def test_hermite_step_cap_reports(oracle):
    m = np.array([1.0, 1e-4, 3e-5])
    q = np.array([[0, 0, 0], [1.0, 0.0, 0.0], [1.0, 0.05, 0.0]])
    v = np.array([[0, 0, 0], [0.0, 1.0, 0.0], [-0.06, 0.95, 0.0]])
    _, _, steps, st = oracle.hermite_set([1, 2], m, q, v, 0.05, 1.0, max_steps=3)
    assert st == 1 and steps == 3


def test_hermite_backward_returns_to_start(oracle):
    """A negative tau integrates backward: forward then backward over the same
    interval returns the set to its start within the 4th-order truncation."""
    m = np.array([1.0, 1e-4, 3e-5])
    q = np.array([[0, 0, 0], [1.0, 0.0, 0.0], [1.0, 0.04, 0.0]])
    v = np.array([[0, 0, 0], [0.0, 1.0, 0.0], [-0.06, 0.95, 0.0]])
    qf, vf, s1, st1 = oracle.hermite_set([1, 2], m, q, v, 0.1, 0.5, eta=0.002, eta_s=0.001)
    qb, vb, s2, st2 = oracle.hermite_set([1, 2], m, qf, vf, 0.1, -0.5, eta=0.002, eta_s=0.001)
    assert st1 == 0 and st2 == 0 and s1 > 5 and s2 > 5
    assert np.abs(qf - q).max() > 0.1
    assert np.abs(qb - q).max() < 1e-8 and np.abs(vb - v).max() < 1e-8


def test_escape_flyby_meets_inside_the_threshold_beyond_the_escape_reach(oracle):
    """The flyby of `workloads.escape_flyby` (a body at five times the escape
    speed aimed at a planetesimal) is an encounter by the rigorous all-pairs
    test of Sec. 2.4, while the pair starts farther apart than the escape
    rule of that section reaches (a_E Hill radii plus the distance covered at
    the escape velocity over the step, each body's own term, in the
    r^2 < 2 rho_i^2 + 2 rho_j^2 form): the case the paper says its crude
    sweep can miss. The straight-line construction is checked against the
    Kepler flow: the closest approach over the step is within 1e-3 AU of the
    aimed 0.005 AU."""
    w = W.escape_flyby()
    m, q = w.m, w.q
    v = oracle.helio_to_dh(m, w.v)
    r = oracle.step(m, q, v, w.offsets, w.tau, 1, oracle.params(eps_H=w.eps_H))
    assert [tuple(x) for x in r.encounters] == [(0, 1, 2)]
    rH = oracle.hill_radii(m, q, v)
    rr = np.linalg.norm(q[1:], axis=1)
    rho = w.a_E * rH[1:] + w.tau * np.sqrt(2.0 * m[0] / rr)
    sep = np.linalg.norm(q[1] - q[2])
    assert sep > 1.2 * np.sqrt(2 * rho[0] ** 2 + 2 * rho[1] ** 2)
    # closest approach along the two Kepler orbits, sampled over the step
    ts = np.linspace(0.0, w.tau, 2001)
    d = []
    for t in ts:
        q1 = oracle.kepler_drift(q[1:2], w.v[1:2], m[0] + m[1], t)[0] if t > 0 else q[1:2]
        q2 = oracle.kepler_drift(q[2:3], w.v[2:3], m[0] + m[2], t)[0] if t > 0 else q[2:3]
        d.append(np.linalg.norm(q1[0] - q2[0]))
    assert abs(min(d) - 0.005) < 1e-3, min(d)
