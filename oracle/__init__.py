"""Python access to the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The CUDA product path never
imports this package. Functions here marshal numpy arrays into the C oracle and
add nothing to its arithmetic.

Parity status of each oracle function (what pins it) is stated in the tests
under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# a library built elsewhere from an edited copy of oracle.c (the tests that
# plant mistakes in the oracle load one in a child process); unset: this one
_LIB_OVERRIDE = os.environ.get("QYM_ORACLE_LIB")
_lib = None

D = C.POINTER(C.c_double)
I64 = C.POINTER(C.c_int64)
I32 = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, FP64, no FMA contraction)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-fopenmp", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("a_E", C.c_double), ("a_H", C.c_double),
                ("eps_H", C.c_double), ("eta", C.c_double), ("eta_s", C.c_double),
                ("solver", C.c_int32), ("guess", C.c_int32), ("encounters", C.c_int32),
                ("max_kepler_iter", C.c_int32), ("max_hermite_steps", C.c_int64),
                ("whole_hermite", C.c_int32), ("planet_mass", C.c_double)]


def params(G=1.0, a_E=3.0, a_H=1.0, eps_H=1e-6, eta=0.02, eta_s=0.01, solver=0, guess=0,
           encounters=1, max_kepler_iter=50, max_hermite_steps=100000, whole_hermite=0,
           planet_mass=1e-7) -> Params:
    return Params(G, a_E, a_H, eps_H, eta, eta_s, solver, guess, encounters, max_kepler_iter,
                  max_hermite_steps, whole_hermite, planet_mass)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_stumpff.argtypes = [C.c_double, D, D]
        L.or_kepler_F.argtypes = [C.c_double] * 6 + [D, D, D]
        L.or_kepler_solve.argtypes = [C.c_double] * 5 + [C.c_int, C.c_int, D, I32]
        L.or_kepler_solve.restype = C.c_int
        L.or_kepler_drift.argtypes = [C.c_int64, D, D, D, D, C.c_double, C.c_double, C.c_int32,
                                      C.c_int32, D, C.c_int32, D, I32]
        L.or_kepler_drift.restype = C.c_int64
        L.or_kepler_residuals.argtypes = [C.c_int64, D, D, C.c_double, C.c_double, D, D]
        L.or_momentum.argtypes = [C.c_int64, D, D, D]
        L.or_drift.argtypes = [C.c_int64, D, D, D, C.c_double]
        L.or_accel_int.argtypes = [C.c_int64, D, D, C.c_double, D]
        L.or_accel_rows.argtypes = [C.c_int64, D, D, C.c_double, C.c_int64, I64, D]
        L.or_kick.argtypes = [C.c_int64, D, D, D, C.c_double, C.c_double]
        L.or_energy.argtypes = [C.c_int64, D, D, D, C.c_double]
        L.or_energy.restype = C.c_double
        L.or_helio_to_dh.argtypes = [C.c_int64, D, D]
        L.or_dh_to_helio.argtypes = [C.c_int64, D, D]
        L.or_hill_radii.argtypes = [C.c_int64, D, D, D, C.c_double, D]
        L.or_pair_dmin2.argtypes = [D, D, D, D, C.c_double]
        L.or_pair_dmin2.restype = C.c_double
        L.or_encounters.argtypes = [C.c_int64, D, D, D, D, D, C.c_double, C.c_double, I64, D, D,
                                    C.c_int64]
        L.or_encounters.restype = C.c_int64
        L.or_encounters_rows.argtypes = [C.c_int64, D, D, D, D, D, C.c_double, C.c_double,
                                         C.c_int64, I64, I64, D, D, C.c_int64]
        L.or_encounters_rows.restype = C.c_int64
        L.or_sets.argtypes = [C.c_int64, C.c_int64, I64, D, C.c_double, I64, I64, I64, D]
        L.or_sets.restype = C.c_int64
        L.or_transition.argtypes = [C.c_double, C.c_double, D, D, D]
        L.or_kcorr.argtypes = [C.c_int64, I64, D, D, D, C.c_double, C.c_double, C.c_double]
        L.or_hermite_force.argtypes = [C.c_int64, D, D, D, C.c_double, C.c_double, C.c_double,
                                       C.c_double, D, D]
        L.or_hermite_set.argtypes = [C.c_int64, I64, D, C.c_double, D, D, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, I64]
        L.or_hermite_set.restype = C.c_int
        L.or_step.argtypes = [C.c_int64, D, D, D, C.POINTER(Params), C.c_double, C.c_int64,
                              C.c_int64, D, I64, D, C.c_int64, I64, I64, I64, D, C.c_int64, I64]
        L.or_step.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = None
        L.or_get_threads.argtypes = []
        L.or_get_threads.restype = C.c_int
    return _lib


def set_threads(n: int) -> None:
    """Threads for the loops over bodies (kick, Kepler drift, all-pairs
    encounter test); results are bit-identical for any count. 1 by default."""
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _d(a):
    return a.ctypes.data_as(D)


def _i64(a):
    return a.ctypes.data_as(I64)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- Appendix
def stumpff(y: float):
    c, s = C.c_double(), C.c_double()
    lib().or_stumpff(float(y), C.byref(c), C.byref(s))
    return c.value, s.value


def kepler_F(x, sqmu, dt, r0, sig, alpha):
    F, Fp, Fpp = C.c_double(), C.c_double(), C.c_double()
    lib().or_kepler_F(x, sqmu, dt, r0, sig, alpha, C.byref(F), C.byref(Fp), C.byref(Fpp))
    return F.value, Fp.value, Fpp.value


def kepler_drift(q0, v0, mu, dt, solver=0, guess=0, x_guess=None, max_iter=50):
    """E_Kep for bodies given as [n,3] arrays (no star row).
    Returns (q1, v1, x, iters, n_not_converged)."""
    q0 = _f64(q0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    n = q0.shape[0]
    q1 = np.empty_like(q0)
    v1 = np.empty_like(v0)
    x = np.empty(n)
    it = np.empty(n, dtype=np.int32)
    xg = None if x_guess is None else _f64(x_guess)
    bad = lib().or_kepler_drift(n, _d(q0), _d(v0), _d(q1), _d(v1), mu, dt, solver, guess,
                                None if xg is None else _d(xg), max_iter, _d(x),
                                it.ctypes.data_as(I32))
    return q1, v1, x, it, int(bad)


def kepler_residuals(q0, v0, mu, dt, x):
    """|F(x)| / (sum of |terms| of F) for each body (Appendix)."""
    q0 = _f64(q0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    x = _f64(x)
    res = np.empty(q0.shape[0])
    lib().or_kepler_residuals(q0.shape[0], _d(q0), _d(v0), float(mu), float(dt), _d(x), _d(res))
    return res


# ---------------------------------------------------------------- Sec. 2
def momentum(m, v):
    m = _f64(m)
    v = _f64(v, (-1, 3))
    S = np.zeros(3)
    lib().or_momentum(len(m), _d(m), _d(v), _d(S))
    return S


def drift(m, q, v, dt):
    m = _f64(m)
    q = _f64(q, (-1, 3)).copy()
    v = _f64(v, (-1, 3))
    lib().or_drift(len(m), _d(m), _d(q), _d(v), dt)
    return q


def accel_int(m, q, G=1.0):
    m = _f64(m)
    q = _f64(q, (-1, 3))
    a = np.zeros_like(q)
    lib().or_accel_int(len(m), _d(m), _d(q), G, _d(a))
    return a


def accel_rows(m, q, sel, G=1.0):
    m = _f64(m)
    q = _f64(q, (-1, 3))
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    a = np.zeros((len(sel), 3))
    lib().or_accel_rows(len(m), _d(m), _d(q), G, len(sel), _i64(sel), _d(a))
    return a


def kick(m, q, v, dt, G=1.0):
    m = _f64(m)
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3)).copy()
    lib().or_kick(len(m), _d(m), _d(q), _d(v), G, dt)
    return v


def energy(m, q, v, G=1.0) -> float:
    m = _f64(m)
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3))
    return float(lib().or_energy(len(m), _d(m), _d(q), _d(v), G))


def helio_to_dh(m, v):
    m = _f64(m)
    v = _f64(v, (-1, 3)).copy()
    lib().or_helio_to_dh(len(m), _d(m), _d(v))
    return v


def dh_to_helio(m, v):
    m = _f64(m)
    v = _f64(v, (-1, 3)).copy()
    lib().or_dh_to_helio(len(m), _d(m), _d(v))
    return v


# ---------------------------------------------------------------- Sec. 2.2-2.4
def hill_radii(m, q, v, G=1.0):
    m = _f64(m)
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3))
    rH = np.zeros(len(m))
    lib().or_hill_radii(len(m), _d(m), _d(q), _d(v), G, _d(rH))
    return rH


def pair_dmin2(dq0, dv0, dq1, dv1, tau) -> float:
    a = [_f64(x) for x in (dq0, dv0, dq1, dv1)]
    return float(lib().or_pair_dmin2(*[_d(x) for x in a], tau))


def encounters(q0, v0, q1, v1, rH, tau, a_E):
    """All pairs (i<j, both >= 1) flagged by the rigorous test.
    Returns (pairs[k,2] int64, d2min[k], thr2[k])."""
    q0, v0, q1, v1 = (_f64(x, (-1, 3)) for x in (q0, v0, q1, v1))
    rH = _f64(rH)
    rows = q0.shape[0]
    cap = 4096
    while True:
        pairs = np.zeros((cap, 2), dtype=np.int64)
        d2 = np.zeros(cap)
        t2 = np.zeros(cap)
        n = lib().or_encounters(rows, _d(q0), _d(v0), _d(q1), _d(v1), _d(rH), tau, a_E,
                                _i64(pairs), _d(d2), _d(t2), cap)
        if n <= cap:
            return pairs[:n].copy(), d2[:n].copy(), t2[:n].copy()
        cap = int(n)


def encounters_rows(q0, v0, q1, v1, rH, tau, a_E, sel):
    q0, v0, q1, v1 = (_f64(x, (-1, 3)) for x in (q0, v0, q1, v1))
    rH = _f64(rH)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    cap = 4096
    while True:
        pairs = np.zeros((cap, 2), dtype=np.int64)
        d2 = np.zeros(cap)
        t2 = np.zeros(cap)
        n = lib().or_encounters_rows(q0.shape[0], _d(q0), _d(v0), _d(q1), _d(v1), _d(rH), tau,
                                     a_E, len(sel), _i64(sel), _i64(pairs), _d(d2), _d(t2), cap)
        if n <= cap:
            return pairs[:n].copy(), d2[:n].copy(), t2[:n].copy()
        cap = int(n)


def sets(rows, pairs, rH, a_H):
    """Returns (set_of[rows], set_start[nsets+1], members[M], rcrit[nsets])."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    rH = _f64(rH)
    set_of = np.zeros(rows, dtype=np.int64)
    set_start = np.zeros(rows + 1, dtype=np.int64)
    members = np.zeros(rows, dtype=np.int64)
    rcrit = np.zeros(rows)
    ns = lib().or_sets(rows, len(pairs), _i64(pairs), _d(rH), a_H, _i64(set_of), _i64(set_start),
                       _i64(members), _d(rcrit))
    return set_of, set_start[:ns + 1].copy(), members[:set_start[ns]].copy(), rcrit[:ns].copy()


def transition(s, rcrit):
    K, Kp, Kpp = C.c_double(), C.c_double(), C.c_double()
    lib().or_transition(s, rcrit, C.byref(K), C.byref(Kp), C.byref(Kpp))
    return K.value, Kp.value, Kpp.value


def kcorr(members, m, q, v, rcrit, dt, G=1.0):
    mem = np.ascontiguousarray(members, dtype=np.int64)
    m = _f64(m)
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3)).copy()
    lib().or_kcorr(len(mem), _i64(mem), _d(m), _d(q), _d(v), G, rcrit, dt)
    return v


def hermite_force(mm, x, u, rcrit, m0=1.0, G=1.0, eps=0.0):
    mm = _f64(mm)
    x = _f64(x, (-1, 3))
    u = _f64(u, (-1, 3))
    a = np.zeros_like(x)
    j = np.zeros_like(x)
    lib().or_hermite_force(len(mm), _d(mm), _d(x), _d(u), G, m0, rcrit, eps, _d(a), _d(j))
    return a, j


def hermite_set(members, m, q, v, rcrit, tau, G=1.0, eps=0.0, eta=0.02, eta_s=0.01,
                max_steps=100000):
    """Integrate the members of one set; returns (q, v, steps, status)."""
    mem = np.ascontiguousarray(members, dtype=np.int64)
    m = _f64(m)
    q = _f64(q, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    steps = np.zeros(1, dtype=np.int64)
    st = lib().or_hermite_set(len(mem), _i64(mem), _d(m), float(m[0]), _d(q), _d(v), G, rcrit,
                              eps, eta, eta_s, tau, max_steps, _i64(steps))
    return q, v, int(steps[0]), int(st)


@dataclasses.dataclass
class StepResult:
    q: np.ndarray
    v: np.ndarray
    encounters: np.ndarray   # [k, 3] (step, i, j) with global row indices
    enc_d2: np.ndarray       # [k, 2] (d_min^2, threshold^2) of each record
    near: np.ndarray         # [k, 3] unflagged pairs within 2e-6 of the threshold (d^2)
    near_d2: np.ndarray      # [k, 2] their (d_min^2, threshold^2)
    stats: np.ndarray        # pairs, sets, largest set, Kepler iterations, Hermite steps, Kepler
                             # failures, steps integrated whole by the Hermite
    status: int


def step(m, q, v, offsets, tau, nsteps, prm: Params | None = None, step0=0,
         rH_fixed=None) -> StepResult:
    """Advance a batch of systems (DH state, star rows zero) by nsteps steps.
    rH_fixed: optional per-row Hill radii held fixed for the run (else the
    radii follow the orbit entering each Kepler step)."""
    prm = prm or params()
    m = _f64(m)
    q = _f64(q, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    offsets = np.asarray(offsets, dtype=np.int64)
    encs = []
    d2s = []
    nears, nd2s = [], []
    stats = np.zeros(7, dtype=np.int64)
    status = 0
    for s in range(len(offsets) - 1):
        lo, hi = int(offsets[s]), int(offsets[s + 1])
        ms = np.ascontiguousarray(m[lo:hi])
        qs = np.ascontiguousarray(q[lo:hi])
        vs = np.ascontiguousarray(v[lo:hi])
        rhs = None if rH_fixed is None else np.ascontiguousarray(rH_fixed[lo:hi], dtype=np.float64)
        cap = 1 << 14
        while True:
            enc = np.zeros((cap, 3), dtype=np.int64)
            ed2 = np.zeros((cap, 2))
            cnt = np.zeros(1, dtype=np.int64)
            ncap = 1 << 14
            nr = np.zeros((ncap, 3), dtype=np.int64)
            nd = np.zeros((ncap, 2))
            ncnt = np.zeros(1, dtype=np.int64)
            qt, vt = qs.copy(), vs.copy()
            st_s = np.zeros(7, dtype=np.int64)
            st = lib().or_step(hi - lo, _d(ms), _d(qt), _d(vt), C.byref(prm), tau, nsteps, step0,
                               None if rhs is None else _d(rhs), _i64(enc), _d(ed2), cap,
                               _i64(cnt), _i64(st_s), _i64(nr), _d(nd), ncap, _i64(ncnt))
            if cnt[0] <= cap:
                break
            cap = int(cnt[0])
        q[lo:hi] = qt
        v[lo:hi] = vt
        e = enc[:cnt[0]].copy()
        e[:, 1:] += lo
        encs.append(e)
        d2s.append(ed2[:cnt[0]].copy())
        k = min(int(ncnt[0]), ncap)
        nn = nr[:k].copy()
        nn[:, 1:] += lo
        nears.append(nn)
        nd2s.append(nd[:k].copy())
        stats[[0, 1, 3, 4, 5, 6]] += st_s[[0, 1, 3, 4, 5, 6]]
        stats[2] = max(stats[2], st_s[2])
        status = status or st
    return StepResult(q, v, np.concatenate(encs) if encs else np.zeros((0, 3), np.int64),
                      np.concatenate(d2s) if d2s else np.zeros((0, 2)),
                      np.concatenate(nears) if nears else np.zeros((0, 3), np.int64),
                      np.concatenate(nd2s) if nd2s else np.zeros((0, 2)), stats, status)


# an edited copy of mlp.py standing in for this package's (the tests that
# plant mistakes in the oracle load one in a child process); unset: mlp.py
_MLP_OVERRIDE = os.environ.get("QYM_ORACLE_MLP")
if _MLP_OVERRIDE:
    import importlib.util as _ilu
    import sys as _sys

    _spec = _ilu.spec_from_file_location(__name__ + ".mlp", _MLP_OVERRIDE)
    mlp = _ilu.module_from_spec(_spec)
    _sys.modules[__name__ + ".mlp"] = mlp
    _spec.loader.exec_module(mlp)
