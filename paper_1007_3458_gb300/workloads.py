"""Seeded synthetic planetary-disk workloads (star + planets + planetesimals).

This module only draws initial conditions. It holds none of the integrator's
arithmetic: no DH coordinates, no universal-variable Kepler solve, no forces.
Orbital elements are converted to heliocentric Cartesian positions and
velocities with the classical elliptic relations (mean -> eccentric anomaly by
Newton's method on M = E - e sin E, then the perifocal-to-inertial rotation),
with mu_i = G (m0 + m_i) for each body about the star.

The disks follow the shapes of the paper's workloads: a few massive planets
inside a less massive planetesimal disk (Section 4, Tables 1-3), and the
massive-plus-massless disks used to stress the encounter search.

Arrays follow one convention everywhere in this project:
  * a system of N bodies plus its star has N+1 rows, the star at row 0 with
    q = v = 0 and mass m0;
  * positions and velocities are float64 arrays of shape [rows, 3];
  * a batch of systems is concatenated, with int64 offsets[nsys+1] giving the
    first row (the star) of each system.

Random draws use numpy's PCG64 (``numpy.random.default_rng(seed)``). Within a
population the element arrays are drawn in the order a, e, i, Omega, omega, M.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Workload:
    """One batch of planetary systems in heliocentric coordinates."""

    name: str
    m: np.ndarray          # [rows] masses, star first in each system
    q: np.ndarray          # [rows, 3] heliocentric positions
    v: np.ndarray          # [rows, 3] heliocentric velocities
    offsets: np.ndarray    # [nsys+1] int64 row offsets; star at offsets[s]
    tau: float             # time step
    nsteps: int            # steps in the paper-shaped run
    G: float = 1.0
    a_E: float = 3.0       # encounter factor in Hill radii
    a_H: float = 1.0       # transition radius factor in Hill radii
    eps_H: float = 1e-6    # Hermite smoothing: about the radius of the largest body

    @property
    def nsys(self) -> int:
        return int(len(self.offsets) - 1)

    @property
    def rows(self) -> int:
        return int(self.m.shape[0])

    @property
    def n_bodies(self) -> int:
        """Bodies other than the stars (the N of the N^2 kick)."""
        return self.rows - self.nsys

    def pairs_per_kick(self) -> int:
        """Ordered interacting pairs per kick, N_b (N_b - 1) summed over systems."""
        nb = np.diff(self.offsets) - 1
        return int(np.sum(nb * (nb - 1)))


def _solve_kepler_elliptic(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly from mean anomaly (elliptic), Newton on E - e sin E - M."""
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        fp = 1.0 - e * np.cos(E)
        dE = f / fp
        E = E - dE
        if np.all(np.abs(dE) < 1e-15):
            break
    return E


def elements_to_cartesian(mu, a, e, inc, Om, om, M):
    """Classical elliptic elements -> heliocentric (q, v), arrays of shape [n, 3]."""
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), np.shape(a))
    E = _solve_kepler_elliptic(np.mod(M, TWO_PI), e)
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    # perifocal frame
    xp = a * (cE - e)
    yp = a * b * sE
    n_mean = np.sqrt(mu / (a * a * a))
    edot = n_mean / (1.0 - e * cE)
    vxp = -a * sE * edot
    vyp = a * b * cE * edot
    cO, sO = np.cos(Om), np.sin(Om)
    co, so = np.cos(om), np.sin(om)
    ci, si = np.cos(inc), np.sin(inc)
    r11 = cO * co - sO * so * ci
    r12 = -cO * so - sO * co * ci
    r21 = sO * co + cO * so * ci
    r22 = -sO * so + cO * co * ci
    r31 = so * si
    r32 = co * si
    q = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp], axis=-1)
    v = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp], axis=-1)
    return q, v


def _population(rng, n, m, a_lo, a_hi, sig_e, sig_i, G, m0, log_a=False, e_uniform=None,
                i_uniform=False):
    """Draw n bodies of mass m; returns (m[n], q[n,3], v[n,3])."""
    if n == 0:
        z = np.zeros((0, 3))
        return np.zeros(0), z, z
    if log_a:
        a = np.exp(rng.uniform(math.log(a_lo), math.log(a_hi), n))
    else:
        a = rng.uniform(a_lo, a_hi, n)
    if e_uniform is not None:
        e = rng.uniform(e_uniform[0], e_uniform[1], n)
    else:
        e = rng.rayleigh(sig_e, n) if sig_e > 0 else np.zeros(n)
    if i_uniform:
        inc = rng.uniform(0.0, math.pi, n)
    else:
        inc = rng.rayleigh(sig_i, n) if sig_i > 0 else np.zeros(n)
    Om = rng.uniform(0.0, TWO_PI, n)
    om = rng.uniform(0.0, TWO_PI, n)
    M = rng.uniform(0.0, TWO_PI, n)
    e = np.minimum(e, 0.99)
    mass = np.full(n, float(m))
    q, v = elements_to_cartesian(G * (m0 + mass), a, e, inc, Om, om, M)
    return mass, q, v


def _planets(rng, masses, sma, G, m0):
    """Circular, coplanar planets with uniformly drawn orbital phases."""
    n = len(masses)
    mass = np.asarray(masses, dtype=np.float64)
    a = np.asarray(sma, dtype=np.float64)
    e = np.zeros(n)
    inc = np.zeros(n)
    Om = rng.uniform(0.0, TWO_PI, n)
    om = rng.uniform(0.0, TWO_PI, n)
    M = rng.uniform(0.0, TWO_PI, n)
    q, v = elements_to_cartesian(G * (m0 + mass), a, e, inc, Om, om, M)
    return mass, q, v


def _assemble(parts, m0=1.0):
    ms, qs, vs = [np.array([m0])], [np.zeros((1, 3))], [np.zeros((1, 3))]
    for m, q, v in parts:
        ms.append(m)
        qs.append(q)
        vs.append(v)
    return np.concatenate(ms), np.concatenate(qs), np.concatenate(vs)


OUTER_PLANETS_M = (1e-3, 3e-4, 5e-5, 5e-5)
OUTER_PLANETS_A = (5.0, 9.5, 19.0, 30.0)
TAU_A5 = TWO_PI * 5.0 ** 1.5 / 40.0      # P(a=5)/40 = 1.756203
TAU_A1 = TWO_PI / 40.0                   # P(a=1)/40 = 0.1570796


def outer_disk(n_planetesimals=256, m_pl=1e-9, seed=0, nsteps=1000, name=None,
               sig_e=0.01, sig_i=0.005, a_lo=10.0, a_hi=30.0):
    """Star + 4 giant planets (a = 5, 9.5, 19, 30; circular, coplanar) + a
    planetesimal disk with a uniform in [10, 30], Rayleigh e and i.

    Default: the 260-body disk (256 planetesimals of 1e-9, seed 0) with
    tau = P(a=5)/40. With n_planetesimals=16380, m_pl=1e-10, seed=1 it is the
    16384-body disk."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    pl = _planets(rng, OUTER_PLANETS_M, OUTER_PLANETS_A, G, m0)
    ps = _population(rng, n_planetesimals, m_pl, a_lo, a_hi, sig_e, sig_i, G, m0)
    m, q, v = _assemble([pl, ps], m0)
    # smoothing: Jupiter's radius in AU (lengths here are AU, G m0 = 1)
    return Workload(name or f"outer_disk_{4 + n_planetesimals}", m, q, v,
                    np.array([0, len(m)], dtype=np.int64), TAU_A5, nsteps, eps_H=4.7e-4)


def disk_260():
    """260 bodies: 4 planets + 256 planetesimals (m=1e-9), seed 0, 1000 steps."""
    return outer_disk(256, 1e-9, seed=0, nsteps=1000, name="disk_260")


def disk_16384():
    """16384 bodies: 4 planets + 16380 planetesimals (m=1e-10), seed 1, 100 steps."""
    return outer_disk(16380, 1e-10, seed=1, nsteps=100, name="disk_16384")


def embryo_disk(n_embryos=64, n_planetesimals=262080, seed=2, nsteps=10, name=None):
    """Dense-encounter disk: star + embryos (1e-6) + planetesimals (1e-11), all
    with a uniform in [1, 3] and Rayleigh(0.02) e and i; tau = P(a=1)/40."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    em = _population(rng, n_embryos, 1e-6, 1.0, 3.0, 0.02, 0.02, G, m0)
    ps = _population(rng, n_planetesimals, 1e-11, 1.0, 3.0, 0.02, 0.02, G, m0)
    m, q, v = _assemble([em, ps], m0)
    # smoothing: the radius of a 1e-6 solar-mass rocky embryo, ~2e-5 AU
    return Workload(name or f"embryo_disk_{n_embryos + n_planetesimals}", m, q, v,
                    np.array([0, len(m)], dtype=np.int64), TAU_A1, nsteps, eps_H=2e-5)


def disk_262144():
    """262144 bodies: 64 embryos + 262080 planetesimals, seed 2, 10 steps."""
    return embryo_disk(64, 262080, seed=2, nsteps=10, name="disk_262144")


def ensemble(nsys=512, n_lo=64, n_hi=4096, seed=3, nsteps=1000, name=None):
    """Batch of independent systems, N bodies per system uniform in [n_lo, n_hi]
    (2 planets of 1e-3 at a = 1 and 1.6, circular, + N-2 planetesimals of 1e-9,
    a uniform in [0.5, 3], Rayleigh(0.01) e and i); tau = P(a=1)/40."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    nper = rng.integers(n_lo, n_hi + 1, nsys)
    ms, qs, vs, offs = [], [], [], [0]
    for s in range(nsys):
        pl = _planets(rng, (1e-3, 1e-3), (1.0, 1.6), G, m0)
        ps = _population(rng, int(nper[s]) - 2, 1e-9, 0.5, 3.0, 0.01, 0.01, G, m0)
        m, q, v = _assemble([pl, ps], m0)
        ms.append(m)
        qs.append(q)
        vs.append(v)
        offs.append(offs[-1] + len(m))
    # smoothing: the radius of a Jupiter-mass planet at 1 AU
    return Workload(name or f"ensemble_{nsys}", np.concatenate(ms), np.concatenate(qs),
                    np.concatenate(vs), np.array(offs, dtype=np.int64), TAU_A1, nsteps,
                    eps_H=4.7e-4)


def crossers(seed=6, n_disk=500, n_ecc=150, n_retro=100, n_hill=40, n_hyper=30, nsteps=40,
             name=None):
    """A disk stirred up to test the close-encounter search where it is
    hardest: star + a Jupiter-mass planet at a = 1 (circular) + a 3e-4 planet
    at a = 1.6 (e = 0.05, i = 0.02) + a cold disk of planetesimals (1e-9, a
    uniform in [0.5, 3], Rayleigh(0.01) e and i), joined by
      * eccentric crossers: a uniform in [0.7, 2.5], e uniform in [0.5, 0.9],
        i uniform in [0, 90 deg];
      * retrograde bodies: a uniform in [0.6, 2.5], e uniform in [0, 0.6],
        i uniform in [90, 180 deg];
      * bodies within 1.5 Hill radii of the Jupiter-mass planet moving at
        0.05-1.5 times its orbital speed relative to it in random directions
        (many on hyperbolic orbits about the star);
      * hyperbolic flybys: r uniform in [1.5, 3], speed 1.1-2 times the local
        escape speed, aimed at a random point of the planet's orbit.
    All light bodies have m = 1e-9; tau = P(a=1)/40."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    mp = np.array([1e-3, 3e-4])
    qp, vp = elements_to_cartesian(G * (m0 + mp), np.array([1.0, 1.6]), np.array([0.0, 0.05]),
                                   np.array([0.0, 0.02]), rng.uniform(0, TWO_PI, 2),
                                   rng.uniform(0, TWO_PI, 2), rng.uniform(0, TWO_PI, 2))
    disk = _population(rng, n_disk, 1e-9, 0.5, 3.0, 0.01, 0.01, G, m0)

    def _elems(n, a_lo, a_hi, e_lo, e_hi, i_lo, i_hi):
        a = rng.uniform(a_lo, a_hi, n)
        e = rng.uniform(e_lo, e_hi, n)
        inc = rng.uniform(i_lo, i_hi, n)
        q, v = elements_to_cartesian(G * (m0 + 1e-9), a, e, inc, rng.uniform(0, TWO_PI, n),
                                     rng.uniform(0, TWO_PI, n), rng.uniform(0, TWO_PI, n))
        return np.full(n, 1e-9), q, v

    ecc = _elems(n_ecc, 0.7, 2.5, 0.5, 0.9, 0.0, 0.5 * math.pi)
    retro = _elems(n_retro, 0.6, 2.5, 0.0, 0.6, 0.5 * math.pi, math.pi)
    # inside the Jupiter-mass planet's Hill sphere, fast and slow
    rH = (mp[0] / 3.0) ** (1.0 / 3.0)
    d = rng.normal(size=(n_hill, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = rng.normal(size=(n_hill, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    vc = np.linalg.norm(vp[0])
    hq = qp[0] + d * (rng.uniform(0.3, 1.5, n_hill) * rH)[:, None]
    hv = vp[0] + u * (rng.uniform(0.05, 1.5, n_hill) * vc)[:, None]
    # flybys from outside, aimed at the planet's orbit
    r = rng.uniform(1.5, 3.0, n_hyper)
    ph = rng.uniform(0, TWO_PI, n_hyper)
    fq = np.stack([r * np.cos(ph), r * np.sin(ph), rng.normal(0, 0.05, n_hyper)], 1)
    tgt_ph = rng.uniform(0, TWO_PI, n_hyper)
    tgt = np.stack([np.cos(tgt_ph), np.sin(tgt_ph), np.zeros(n_hyper)], 1)
    aim = (tgt - fq) / np.linalg.norm(tgt - fq, axis=1, keepdims=True)
    fv = aim * (np.sqrt(2.0 * G * m0 / r) * rng.uniform(1.1, 2.0, n_hyper))[:, None]
    m, q, v = _assemble([(mp, qp, vp), disk, ecc, retro, (np.full(n_hill, 1e-9), hq, hv),
                         (np.full(n_hyper, 1e-9), fq, fv)], m0)
    return Workload(name or "crossers", m, q, v, np.array([0, len(m)], dtype=np.int64), TAU_A1,
                    nsteps, eps_H=4.7e-4)


def planet_encounter(n_planetesimals=60, seed=9, sep=0.6, phase=0.12, nsteps=20, name=None):
    """Two Jupiter-mass planets in a close encounter (the case of Sec. 2.3's
    last paragraph): star + planets of 1e-3 on circular coplanar orbits at
    a = 5 and 5 + sep, the second `phase` radians ahead (0.78 AU apart for
    the defaults, inside the 3 x 2 mutual Hill radii of the encounter test),
    + a cold disk of planetesimals (1e-9, a uniform in [8, 14], Rayleigh(0.01)
    e and i); tau = P(a=5)/40."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    mp = np.array([1e-3, 1e-3])
    M0 = rng.uniform(0.0, TWO_PI)
    qp, vp = elements_to_cartesian(G * (m0 + mp), np.array([5.0, 5.0 + sep]), np.zeros(2),
                                   np.zeros(2), np.zeros(2), np.zeros(2),
                                   np.array([M0, M0 + phase]))
    disk = _population(rng, n_planetesimals, 1e-9, 8.0, 14.0, 0.01, 0.01, G, m0)
    m, q, v = _assemble([(mp, qp, vp), disk], m0)
    return Workload(name or f"planet_encounter_{len(m)}", m, q, v,
                    np.array([0, len(m)], dtype=np.int64), TAU_A5, nsteps, eps_H=4.7e-4)


def escape_flyby(speed=2.3, miss=0.005, name="escape_flyby"):
    """The case Sec. 2.4 says its crude sweep can miss: star + a planetesimal
    (1e-9) on a circular orbit at 10 AU + a body of 1e-9 moving at `speed`
    (2.3: five times the escape speed at 10 AU) along -x on a straight line
    that passes `miss` AU from the planetesimal's position at mid-step (its
    circular motion written out); tau = P(a=5)/40. The pair starts 2.04 AU
    apart, farther than the two bodies' escape distances over the step
    (1.55 AU in the r^2 < 2 rho_i^2 + 2 rho_j^2 form), and meets well inside
    3 Hill radii."""
    G, m0, mp = 1.0, 1.0, 1e-9
    tau = TAU_A5
    om = math.sqrt(G * (m0 + mp) / 1000.0)  # circular at 10 AU
    th = 0.5 * tau * om
    tgt = np.array([10.0 * math.cos(th), 10.0 * math.sin(th) + miss, 0.0])
    q = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0], tgt + np.array([0.5 * tau * speed, 0.0, 0.0])])
    v = np.array([[0.0, 0.0, 0.0], [0.0, 10.0 * om, 0.0], [-speed, 0.0, 0.0]])
    return Workload(name, np.array([m0, mp, mp]), q, v, np.array([0, 3], dtype=np.int64), tau, 1)


def test_particles(n=1048576, seed=4):
    """Massless test particles about a unit-mass star: a log-uniform in
    [0.5, 50], e uniform in [0, 0.9], inclination and angles uniform.
    Returns (q[n,3], v[n,3], dt) with dt = P(a=5)/40 (no star row)."""
    G, m0 = 1.0, 1.0
    rng = np.random.default_rng(seed)
    _, q, v = _population(rng, n, 0.0, 0.5, 50.0, 0.0, 0.0, G, m0, log_a=True,
                          e_uniform=(0.0, 0.9), i_uniform=True)
    return q, v, TAU_A5


def subsample(w: Workload, n_bodies: int, seed: int = 0, name=None) -> Workload:
    """First system of ``w`` cut to its planets/embryos plus a random subset of
    the remaining bodies, keeping their shapes (for small parity cases)."""
    lo, hi = int(w.offsets[0]), int(w.offsets[1])
    m, q, v = w.m[lo:hi], w.q[lo:hi], w.v[lo:hi]
    heavy = np.nonzero(m[1:] > 10 * m[1:].min())[0] + 1 if len(m) > 1 else np.zeros(0, int)
    light = np.setdiff1d(np.arange(1, len(m)), heavy)
    rng = np.random.default_rng(seed)
    k = max(0, n_bodies - len(heavy))
    pick = np.sort(rng.choice(light, size=min(k, len(light)), replace=False))
    rows = np.concatenate([[0], heavy, pick]).astype(int)
    return Workload(name or f"{w.name}_sub{len(rows) - 1}", m[rows].copy(), q[rows].copy(),
                    v[rows].copy(), np.array([0, len(rows)], dtype=np.int64), w.tau, w.nsteps,
                    w.G, w.a_E, w.a_H, w.eps_H)


# ---------------------------------------------------------------- learned guess
MLP_NW = 4555   # 4*64 + 64 + 64*64 + 64 + 64 + 1 + 4 + 4 + 2


def mlp_init(seed, u, z, hidden=64):
    """Seeded initial weights of the 4 -> 64 -> 64 -> 1 guess network as one
    float32 vector (layout of qym_set_mlp): He-scaled normal matrices, zero
    biases, and the input/output normalisation taken from sample statistics
    of the training rows (u [n, 4] raw features, z [n] targets t)."""
    rng = np.random.default_rng(seed)
    H = hidden
    W1 = rng.normal(0.0, math.sqrt(2.0 / 4), (H, 4))
    W2 = rng.normal(0.0, math.sqrt(2.0 / H), (H, H))
    W3 = rng.normal(0.0, math.sqrt(1.0 / H), H)
    u = np.asarray(u, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    mean = u.mean(axis=0)
    std = u.std(axis=0) + 1e-6
    w = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0], mean, std,
                        [z.mean(), z.std() + 1e-6]])
    assert w.size == MLP_NW
    return w.astype(np.float32)


def mlp_rows_synthetic(n, seed):
    """Synthetic training rows (u1, u2, u3, u4, z) float32 [n, 5] spanning the
    ranges the features take on bound orbits with e < 0.9 and steps up to a
    period (u1 radial/circular speed, u2 = 2 - r0/a, u3 log step over the
    dynamical time, u4 step over period), with a smooth target z."""
    rng = np.random.default_rng(seed)
    u1 = rng.normal(0.0, 0.3, n)
    u2 = rng.uniform(0.1, 1.9, n)
    u3 = rng.uniform(-5.0, 1.6, n)
    u4 = rng.uniform(0.0, 0.8, n)
    z = 1.0 + 0.3 * np.tanh(u1 * u4 * 4.0) + 0.2 * (u2 - 1.0) * u4 + 0.05 * np.sin(u3)
    return np.stack([u1, u2, u3, u4, z], axis=1).astype(np.float32)
