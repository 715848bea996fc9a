"""Pins for the oracle's E_Int acceleration, E_Dft drift, energy and the
heliocentric <-> DH velocity conversion (Section 2, Eqs. 1-4).

References used: finite-difference gradients of the energy, Newton's third
law, a closed-form symmetric configuration, and the textbook Newtonian energy
of the same bodies in the barycentric inertial frame."""
import math

import numpy as np

from paper_1007_3458_gb300 import workloads as W


def _system(n=12, seed=1):
    rng = np.random.default_rng(seed)
    m = np.concatenate([[1.0], rng.uniform(1e-6, 1e-3, n)])
    q = np.concatenate([[[0, 0, 0]], rng.normal(0, 2, (n, 3))])
    v = np.concatenate([[[0, 0, 0]], rng.normal(0, 0.5, (n, 3))])
    return m, q, v


def test_accel_is_minus_gradient_of_interaction_energy(oracle):
    """a_i = -(1/m_i) dH_Int/dQ_i (Eq. 4), by central differences of the
    oracle's total energy with v = 0 and a negligible star mass (so that the
    energy is H_Int alone; E_Int does not involve the star)."""
    m, q, _ = _system()
    v = np.zeros_like(q)
    a = oracle.accel_int(m, q)
    me = m.copy()
    me[0] = 1e-30
    h = 1e-6
    for i in range(1, len(m)):
        for k in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, k] += h
            qm[i, k] -= h
            g = (oracle.energy(me, qp, v) - oracle.energy(me, qm, v)) / (2 * h)
            assert abs(-g / m[i] - a[i, k]) <= 1e-7 * np.abs(a[i]).max()
    assert np.all(a[0] == 0.0)


def test_accel_conserves_momentum(oracle):
    """Newton's third law: sum_i m_i a_i = 0 (star excluded on both sides)."""
    m, q, _ = _system(40, 3)
    a = oracle.accel_int(m, q)
    tot = (m[:, None] * a).sum(0)
    assert np.all(np.abs(tot) <= 1e-15 * np.abs(m[:, None] * a).sum(0))


def test_accel_equilateral_triangle(oracle):
    """Three equal masses at the vertices of an equilateral triangle of side L:
    each is pulled toward the centroid with |a| = sqrt(3) G m / L^2."""
    L, mm = 0.7, 3e-4
    c = np.array([2.0, -1.0, 0.5])
    ang = np.array([0.0, 2 * math.pi / 3, 4 * math.pi / 3])
    R = L / math.sqrt(3)
    pts = c + R * np.stack([np.cos(ang), np.sin(ang), np.zeros(3)], 1)
    m = np.array([1.0, mm, mm, mm])
    q = np.concatenate([[[0, 0, 0]], pts])
    a = oracle.accel_int(m, q)
    for i in range(3):
        toward = (c - pts[i]) / R
        ref = math.sqrt(3) * mm / L ** 2 * toward
        assert np.linalg.norm(a[i + 1] - ref) <= 1e-13 * np.linalg.norm(ref)


def test_energy_equals_barycentric_newtonian_energy(oracle):
    """H_Dft + H_Kep + H_Int in (heliocentric Q, barycentric P) equals the
    plain Newtonian energy of the same bodies in the barycentric frame."""
    w = W.outer_disk(30, 1e-5, seed=4)
    m, q, vh = w.m, w.q, w.v
    vd = oracle.helio_to_dh(m, vh)
    E_dh = oracle.energy(m, q, vd)
    M = m.sum()
    X = q - (m[:, None] * q).sum(0) / M
    V = vh - (m[:, None] * vh).sum(0) / M
    T = 0.5 * np.sum(m * np.sum(V * V, 1))
    U = 0.0
    for i in range(len(m)):
        d = np.linalg.norm(X[i] - X[i + 1:], axis=1)
        U -= np.sum(m[i] * m[i + 1:] / d)
    assert abs(E_dh - (T + U)) <= 1e-13 * abs(T + U)


def test_dh_velocity_round_trip_and_barycentre(oracle):
    w = W.outer_disk(20, 1e-4, seed=5)
    vd = oracle.helio_to_dh(w.m, w.v)
    # barycentric velocities: the star moves with V0 = -S/m0 and the total
    # momentum vanishes; recomputing heliocentric velocities gives the input
    S = oracle.momentum(w.m, vd)
    V0 = -S / w.m[0]
    assert np.allclose(vd[1:] - V0, w.v[1:], rtol=0, atol=1e-15)
    back = oracle.dh_to_helio(w.m, vd)
    assert np.allclose(back[1:], w.v[1:], rtol=0, atol=1e-15)


def test_drift_is_uniform_and_commutes_with_kick(oracle):
    """E_Dft shifts every Q by the same vector (dt S / m0, Eq. 2) and commutes
    with E_Int: H_Int depends only on differences of Q and conserves sum P."""
    m, q, v = _system(15, 7)
    dt = 0.3
    qd = oracle.drift(m, q, v, dt)
    shift = qd[1:] - q[1:]
    assert np.allclose(shift, shift[0], rtol=0, atol=1e-15)
    assert np.allclose(shift[0] * m[0] / dt, (m[1:, None] * v[1:]).sum(0), rtol=1e-14)
    # drift then kick vs kick then drift
    v1 = oracle.kick(m, qd, v, dt)
    q1 = qd
    v2 = oracle.kick(m, q, v, dt)
    q2 = oracle.drift(m, q, v2, dt)
    assert np.allclose(q1, q2, rtol=0, atol=1e-14)
    assert np.allclose(v1, v2, rtol=0, atol=1e-14)


def test_selected_rows_match_full_accel(oracle):
    m, q, _ = _system(50, 9)
    a = oracle.accel_int(m, q)
    sel = np.array([1, 7, 50, 23])
    assert np.array_equal(oracle.accel_rows(m, q, sel), a[sel])


def test_energy_keeps_light_pair_terms(oracle):
    """A disk of 2000 light bodies around planets: the energy equals the
    correctly rounded sum (math.fsum) of every term of Eqs. 2-4, so pair
    terms far below an ulp of the total are not lost."""
    import math as _m
    w = W.outer_disk(1996, 1e-10, seed=3)
    m, q = w.m, w.q
    v = oracle.helio_to_dh(m, w.v)
    terms = []
    S = (m[1:, None] * v[1:]).sum(0)
    terms.append(S @ S / (2 * m[0]))
    for i in range(1, len(m)):
        terms.append(0.5 * m[i] * (v[i] @ v[i]))
        terms.append(-m[0] * m[i] / np.linalg.norm(q[i]))
        d = np.linalg.norm(q[i] - q[i + 1:], axis=1)
        terms.extend((-m[i] * m[i + 1:] / d).tolist())
    ref = _m.fsum(terms)
    # ordinary rounding over ~4000 large terms is ~1e-15; dropping the light
    # pair terms would show as ~2e-11 here
    assert abs(oracle.energy(m, q, v) - ref) <= 1e-13 * abs(ref)
