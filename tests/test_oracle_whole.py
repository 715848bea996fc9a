"""Pins for the oracle's whole-system Hermite step (Sec. 2.3, last paragraph):
when a step's encounter sets put two planets in one set, that step is done
for the whole system by the Hermite (with `whole_hermite`), from the
positions after the opening drift and the velocities entering the first
kick, with K = 0 for every pair, no K corrections and no second kick, and
the closing drift after it.

References: the composition drift(tau/2) o flow(tau) o drift(tau/2), with the
flow of H_Kep + H_Int (star fixed at the origin, the Hermite's smoothing)
integrated by scipy's DOP853 from the equations of motion written out here;
the switch left alone when no set holds two planets (bit-identical steps);
and the energy of a system with two planets in a close encounter, which the
paper says the switch protects."""
import numpy as np
import pytest

from paper_1007_3458_gb300 import workloads as W


def _dh(oracle, w):
    return w.m, w.q.copy(), oracle.helio_to_dh(w.m, w.v)


def _exact_composition(w, q, v, tau, G=1.0):
    """drift(tau/2), then the flow of H_Kep + H_Int over tau (every body; star
    at the origin; pair and star terms smoothed with eps_H as the Hermite's
    are) by DOP853 at rtol 1e-13, then drift(tau/2). DH state in and out."""
    from scipy.integrate import solve_ivp
    m = w.m
    eps2 = w.eps_H ** 2
    n = len(m) - 1
    q = q.copy()
    q[1:] += 0.5 * tau * (m[1:, None] * v[1:]).sum(0) / m[0]

    def rhs(t, y):
        x = y[:3 * n].reshape(n, 3)
        u = y[3 * n:].reshape(n, 3)
        s2 = (x * x).sum(1) + eps2
        a = -G * m[0] * x / (s2 * np.sqrt(s2))[:, None]
        d = x[:, None, :] - x[None, :, :]
        r2 = (d * d).sum(2) + eps2
        np.fill_diagonal(r2, 1.0)
        wgt = -G * m[1:][None, :] / (r2 * np.sqrt(r2))
        np.fill_diagonal(wgt, 0.0)
        a += (wgt[:, :, None] * d).sum(1)
        return np.concatenate([u.ravel(), a.ravel()])

    y0 = np.concatenate([q[1:].ravel(), v[1:].ravel()])
    sol = solve_ivp(rhs, (0.0, tau), y0, method="DOP853", rtol=1e-13, atol=1e-16)
    x = sol.y[:3 * n, -1].reshape(n, 3)
    u = sol.y[3 * n:, -1].reshape(n, 3)
    qo = np.zeros_like(q)
    vo = np.zeros_like(v)
    qo[1:] = x + 0.5 * tau * (m[1:, None] * u).sum(0) / m[0]
    vo[1:] = u
    return qo, vo


def _rel(a, b):
    return np.linalg.norm(a[1:] - b[1:], axis=1) / np.linalg.norm(b[1:], axis=1)


def test_whole_step_is_the_exact_flow_composition(oracle):
    """Two Jupiter-mass planets 0.78 AU apart: the first step switches to the
    whole-system Hermite, and with eta = 1e-4 (Hermite error ~ eta^2) it
    equals the composition with the DOP853 flow to 1e-10 in position and
    1e-9 in velocity; the hybrid step differs from it by ~3e-5 (the
    splitting the switch removes)."""
    w = W.planet_encounter()
    m, q, v = _dh(oracle, w)
    qe, ve = _exact_composition(w, q, v, w.tau)
    prm = oracle.params(eps_H=w.eps_H, whole_hermite=1, eta=1e-4, eta_s=5e-5)
    r = oracle.step(m, q, v, w.offsets, w.tau, 1, prm)
    assert r.status == 0 and r.stats[6] == 1
    dq, dv = _rel(r.q, qe).max(), _rel(r.v, ve).max()
    assert dq <= 1e-10 and dv <= 1e-9, (dq, dv)
    h = oracle.step(m, q, v, w.offsets, w.tau, 1, oracle.params(eps_H=w.eps_H, eta=1e-4,
                                                                    eta_s=5e-5))
    assert h.stats[6] == 0 and _rel(h.q, qe).max() > 1e-6


def test_whole_switch_needs_two_planets_in_a_set(oracle):
    """No set with two planets, no switch: the planet pair with a planet mass
    above both planets' (no body is a planet), and the stirred disk of
    crossers (sets of one planet and its crossers, 3 steps) step bit for bit
    as without the switch."""
    w = W.planet_encounter()
    m, q, v = _dh(oracle, w)
    off = oracle.step(m, q, v, w.offsets, w.tau, 2, oracle.params(eps_H=w.eps_H))
    on = oracle.step(m, q, v, w.offsets, w.tau, 2,
                     oracle.params(eps_H=w.eps_H, whole_hermite=1, planet_mass=0.01))
    assert off.stats[1] > 0 and on.stats[6] == 0
    assert np.array_equal(on.q, off.q) and np.array_equal(on.v, off.v)
    c = W.crossers()
    m, q, v = _dh(oracle, c)
    off = oracle.step(m, q, v, c.offsets, c.tau, 3, oracle.params(eps_H=c.eps_H))
    on = oracle.step(m, q, v, c.offsets, c.tau, 3, oracle.params(eps_H=c.eps_H, whole_hermite=1))
    assert off.stats[1] > 0 and on.stats[6] == 0
    assert np.array_equal(on.q, off.q) and np.array_equal(on.v, off.v)
    assert np.array_equal(on.encounters, off.encounters)


def test_whole_switch_holds_energy_in_planet_encounter(oracle):
    """40 steps of the two close planets: with the switch the relative energy
    error stays below 1e-4; the hybrid step alone loses more than 1e-2 (the
    paper: hybrid integrators deviate most in energy during planet/planet
    encounters, and the switch to a conventional N-body integrator there
    improves their accuracy)."""
    w = W.planet_encounter()
    m, q, v = _dh(oracle, w)
    E0 = oracle.energy(m, q, v)
    errs = {}
    for wh in (0, 1):
        r = oracle.step(m, q, v, w.offsets, w.tau, 40,
                        oracle.params(eps_H=w.eps_H, whole_hermite=wh))
        assert r.status == 0
        errs[wh] = abs(oracle.energy(m, r.q, r.v) / E0 - 1.0)
        if wh:
            assert r.stats[6] > 0
    assert errs[1] < 1e-4 and errs[0] > 1e-2, errs
