"""GPU parity of the whole hybrid DH step (Sec. 2, Eq. 5; procedure of
Sec. 2.3) through the context API against the oracle's step on the same
seeded disks: positions, velocities, encounter lists, energy; batched systems;
error statuses."""
import numpy as np
import pytest

import paper_1007_3458_gb300 as q
from paper_1007_3458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return t


def _run_gpu(w, nsteps, **prm):
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, **prm)
    sim.step(w.tau, nsteps)
    qq, vv = sim.state()
    enc = sim.encounters()
    st = sim.stats()
    E = sim.energy()
    sim.close()
    return qq, vv, enc, st, E


def _run_oracle(oracle, w, nsteps, **prm):
    vd = np.concatenate([oracle.helio_to_dh(w.m[a:b], w.v[a:b])
                         for a, b in zip(w.offsets[:-1], w.offsets[1:])])
    r = oracle.step(w.m, w.q, vd, w.offsets, w.tau, nsteps, oracle.params(**prm))
    vh = np.concatenate([oracle.dh_to_helio(w.m[a:b], r.v[a:b])
                         for a, b in zip(w.offsets[:-1], w.offsets[1:])])
    return r, vh


def _energies(oracle, w, q, v):
    return np.array([oracle.energy(w.m[a:b], q[a:b], v[a:b])
                     for a, b in zip(w.offsets[:-1], w.offsets[1:])])


def _chaos_spread(oracle, w, nsteps, energy=False, **prm):
    """Per-body distance between the oracle's result and the oracle's results
    from initial positions moved by one ulp up and down (the larger of the
    two): how far rounding alone moves each body over the run (large for
    bodies in close encounters); with energy=True also the per-system energy
    difference of those runs."""
    r0, _ = _run_oracle(oracle, w, nsteps, **prm)
    dq = np.zeros(len(w.m))
    dE = np.zeros(w.nsys)
    for direction in (np.inf, -np.inf):
        pert = W.Workload(w.name, w.m, np.nextafter(w.q, direction), w.v, w.offsets, w.tau,
                          w.nsteps)
        r1, _ = _run_oracle(oracle, pert, nsteps, **prm)
        dq = np.maximum(dq, np.linalg.norm(r1.q - r0.q, axis=1))
        dE = np.maximum(dE, np.abs(_energies(oracle, w, r1.q, r1.v) - _energies(oracle, w, r0.q, r0.v)))
    return (dq, dE) if energy else dq


def _check_positions(qg, qo, spread, rel=1e-12):
    """FP64 parity: every body within max(rel |q|, 100 x its one-ulp chaos
    spread) of the oracle."""
    tol = np.maximum(rel * np.linalg.norm(qo, axis=1), 100.0 * spread)
    err = np.linalg.norm(qg - qo, axis=1)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, [(int(i), float(err[i]), float(tol[i])) for i in bad[:5]]
    return int((100.0 * spread > rel * np.linalg.norm(qo, axis=1)).sum())


def _relq(a, b):
    n = np.linalg.norm(b, axis=1)
    n[n == 0] = 1
    return np.linalg.norm(a - b, axis=1) / n


def test_fp64_plain_step_100_steps(gpu, oracle):
    """Plain DH step (no encounter search), FP64 kick, 100 steps of the
    260-body disk: positions within 1e-12 relative."""
    w = W.disk_260()
    qg, vg, enc, st, E = _run_gpu(w, 100, kick_prec=q.QYM_KICK_FP64, encounters=0)
    r, vh = _run_oracle(oracle, w, 100, encounters=0)
    assert _relq(qg, r.q).max() <= 1e-12
    assert _relq(vg, vh).max() <= 1e-11
    assert len(enc) == 0


def test_fp64_hybrid_step_with_encounters(gpu, oracle):
    """Hybrid step with encounters on the 260-body disk for 100 steps, FP64
    kick: same encounter records (step, i, j) as the oracle's all-pairs test,
    positions within 1e-12 relative."""
    w = W.disk_260()
    qg, vg, enc, st, E = _run_gpu(w, 100, kick_prec=q.QYM_KICK_FP64)
    r, vh = _run_oracle(oracle, w, 100)
    assert len(r.encounters) > 0
    assert np.array_equal(enc, r.encounters)
    assert st["encounters"] >= len(r.encounters) and st["hermite_steps"] > 0
    _check_positions(qg, r.q, _chaos_spread(oracle, w, 100))


def test_mixed_hybrid_step(gpu, oracle):
    """Mixed-precision kick: encounter records equal, positions within the
    drift that a 1e-6 relative acceleration error can cause over the run
    (|dq| <= 1e-6 max|a_int| T^2 / 2), and the energy error matching the
    oracle's to well below the step's own error."""
    w = W.disk_260()
    qg, vg, enc, st, E = _run_gpu(w, 100)
    r, vh = _run_oracle(oracle, w, 100)
    assert np.array_equal(enc, r.encounters)
    T = 100 * w.tau
    amax = np.linalg.norm(oracle.accel_int(w.m, w.q), axis=1).max()
    tol = 1e-6 * amax * T * T / 2
    assert np.linalg.norm(qg - r.q, axis=1).max() <= tol
    vd = oracle.helio_to_dh(w.m, w.v)
    E0 = oracle.energy(w.m, w.q, vd)
    Eo = oracle.energy(w.m, r.q, r.v)
    assert abs(E[0] - Eo) <= 1e-9 * abs(E0)


def test_mixed_energy_1000_steps(gpu, oracle):
    """The mixed-precision kick over the configured 1000 steps of the 260-body
    disk: the relative energy change matches the FP64 oracle's to within
    1e-9 (the mixed path's accuracy target per 1000 steps), and the records
    agree up to pairs at the threshold."""
    w = W.disk_260()
    qg, vg, enc, st, E = _run_gpu(w, 1000, eps_H=w.eps_H)
    r, vh = _run_oracle(oracle, w, 1000, eps_H=w.eps_H)
    assert st["status_bits"] == 0
    vd = oracle.helio_to_dh(w.m, w.v)
    E0 = oracle.energy(w.m, w.q, vd)
    Eo = oracle.energy(w.m, r.q, r.v)
    print(f"\n  dE/E oracle {(Eo - E0) / abs(E0):.6e}, GPU mixed {(E[0] - E0) / abs(E0):.6e}")
    assert abs(E[0] - Eo) <= 1e-9 * abs(E0)
    _compare_records(enc, r)


@pytest.mark.parametrize("a_E, a_H", [(1.0, 0.5), (6.0, 2.0)])
def test_hill_factor_parity(gpu, oracle, a_E, a_H):
    """The hybrid step at the ends of the Hill-factor sweep (a_E the encounter
    radius of Sec. 2.4, a_H the transition radius r_crit of Sec. 2.2), FP64
    kick, 300 steps of the 260-body disk (at a_E = 1 the first encounters come
    after step 100): records equal up to pairs at the threshold, positions
    within the chaos-aware tolerance."""
    w = W.disk_260()
    prm = dict(a_E=a_E, a_H=a_H, eps_H=w.eps_H)
    n = 300
    qg, vg, enc, st, E = _run_gpu(w, n, kick_prec=q.QYM_KICK_FP64, **prm)
    r, vh = _run_oracle(oracle, w, n, **prm)
    assert st["status_bits"] == 0 and len(r.encounters) > 0
    skip = _compare_records(enc, r)
    keep = np.array([i not in skip for i in range(len(w.m))])
    _check_positions(qg[keep], r.q[keep], _chaos_spread(oracle, w, n, **prm)[keep])


def _compare_records(enc, r, band=1e-9):
    """Encounter records equal, except pairs whose interpolated d_min lies
    within `band` (relative) of the 3-Hill-radius threshold on the oracle's
    side (flagged just below it, or missed just above it). Returns the
    bodies of such pairs: their integration legitimately differs afterwards."""
    A = {tuple(x) for x in enc}
    B = {tuple(x) for x in r.encounters}
    rel = lambda d2: abs(np.sqrt(d2[0] / d2[1]) - 1) if d2[1] > 0 else np.inf
    flagged = {tuple(x): rel(d) for x, d in zip(r.encounters, r.enc_d2)}
    missed = {tuple(x): rel(d) for x, d in zip(r.near, r.near_d2)}
    only_oracle = [x for x in B - A if flagged.get(x, np.inf) > band]
    only_gpu = [x for x in A - B if missed.get(x, np.inf) > band]
    assert not only_oracle, f"oracle-only records away from the threshold: {only_oracle[:10]}"
    assert not only_gpu, f"GPU-only records away from the threshold: {only_gpu[:10]}"
    return {i for rec in A ^ B for i in rec[1:]}


def test_batched_systems(gpu, oracle):
    """Several independent systems of uneven size in one context (ensemble
    shape, planets at a = 1 and 1.6): every system matches the oracle."""
    w = W.ensemble(nsys=6, n_lo=40, n_hi=300, seed=5, nsteps=30)
    qg, vg, enc, st, E = _run_gpu(w, 30, kick_prec=q.QYM_KICK_FP64)
    r, vh = _run_oracle(oracle, w, 30)
    skip = _compare_records(enc, r)
    keep = np.array([i not in skip for i in range(len(w.m))])
    spread, espread = _chaos_spread(oracle, w, 30, energy=True)
    n_chaotic = _check_positions(qg[keep], r.q[keep], spread[keep], rel=1e-11)
    assert n_chaotic < 0.10 * len(w.m)  # the check does not become vacuous
    Eo = _energies(oracle, w, r.q, r.v)
    if not skip:
        assert np.all(np.abs(E - Eo) <= 1e-12 * np.abs(Eo) + 100 * espread)


def _planet_swarm(k, seed):
    """Star, a Jupiter-mass planet at a = 1 and k light bodies inside its Hill
    sphere on near-circular orbits about it: one encounter set of k + 1
    members that the Hermite runs on a cluster of CTAs."""
    rng = np.random.default_rng(seed)
    mp = 1e-3
    rH = (mp / 3) ** (1 / 3)
    m = np.concatenate([[1.0, mp], np.full(k, 1e-12)])
    qp, vp = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    r = rng.uniform(0.3, 1.0, k) * rH
    th = rng.uniform(0, 2 * np.pi, k)
    off = np.stack([r * np.cos(th), r * np.sin(th), rng.normal(0, 0.05, k) * rH], 1)
    vc = np.sqrt(mp / r) * rng.uniform(0.7, 1.0, k)
    voff = np.stack([-vc * np.sin(th), vc * np.cos(th), np.zeros(k)], 1)
    q = np.concatenate([[[0.0, 0.0, 0.0]], [qp], qp + off])
    v = np.concatenate([[[0.0, 0.0, 0.0]], [vp], vp + voff])
    return W.Workload("swarm", m, q, v, np.array([0, k + 2]), 2 * np.pi / 40, 3)


@pytest.mark.parametrize("k, cluster", [(35, 8), (68, 8), (35, 4), (68, 2)])
def test_cluster_set_parity(gpu, oracle, k, cluster):
    """One large set on a cluster of 8, 4 or 2 CTAs, with k + 1 members such
    that the CTAs' member ranges straddle a power of two (36 over 8 CTAs -> 4
    or 5 per CTA, 69 -> 8 or 9; 36 over 4 -> 9; 69 over 2 -> 34 or 35): the
    records match the oracle and every body stays within the chaos-aware
    tolerance."""
    w = _planet_swarm(k, seed=k)
    qg, vg, enc, st, E = _run_gpu(w, 3, kick_prec=q.QYM_KICK_FP64, hermite_cluster=cluster)
    r, vh = _run_oracle(oracle, w, 3)
    assert st["status_bits"] == 0 and st["max_set"] == k + 1
    skip = _compare_records(enc, r)
    keep = np.array([i not in skip for i in range(len(w.m))])
    _check_positions(qg[keep], r.q[keep], _chaos_spread(oracle, w, 3)[keep], rel=1e-11)


@pytest.mark.parametrize("cluster", [8, 0])
def test_large_sets_one_cta_each_parity(gpu, oracle, cluster):
    """More large sets than clusters (120 systems, each a planet with a 68-body
    swarm): the clusters take as many sets as there are clusters (38 of 8 CTAs,
    or 76 of 2 with the automatic choice for a batch), every other set runs on
    one CTA, where with 69 members the CTA first rules out far partners in
    FP32 before the FP64 work. Sampled systems match the oracle stepping each
    alone, whichever path their sets took."""
    sw = [_planet_swarm(68, seed=100 + s) for s in range(120)]
    m = np.concatenate([w.m for w in sw])
    qq = np.concatenate([w.q for w in sw])
    vv = np.concatenate([w.v for w in sw])
    offs = np.concatenate([[0], np.cumsum([len(w.m) for w in sw])])
    w = W.Workload("swarms", m, qq, vv, offs, sw[0].tau, 3)
    qg, vg, enc, st, E = _run_gpu(w, 3, kick_prec=q.QYM_KICK_FP64, hermite_cluster=cluster)
    assert st["status_bits"] == 0 and st["max_set"] == 69
    for s in (0, 77, 119):
        a, b = int(offs[s]), int(offs[s + 1])
        r, _ = _run_oracle(oracle, sw[s], 3)
        mine = enc[(enc[:, 1] >= a) & (enc[:, 1] < b)].copy()
        mine[:, 1:] -= a
        skip = _compare_records(mine, r)
        keep = np.array([i not in skip for i in range(b - a)])
        _check_positions(qg[a:b][keep], r.q[keep], _chaos_spread(oracle, sw[s], 3)[keep],
                         rel=1e-11)


def _cut(w, rows, name):
    rows = np.asarray(rows)
    return W.Workload(name, w.m[rows].copy(), w.q[rows].copy(), w.v[rows].copy(),
                      np.array([0, len(rows)], dtype=np.int64), w.tau, w.nsteps, w.G, w.a_E,
                      w.a_H, w.eps_H)


def test_ragged_batch_with_massless_bodies(gpu, oracle):
    """One context holding systems of 1, 2, 4, 32, 256 and 999 bodies, the
    32-body one with 14 massless bodies (zero Hill radius, no pull): the
    hybrid step over 20 steps matches the oracle system by system."""
    d = W.disk_260()
    mixed = W.subsample(d, 32, seed=11, name="massless")
    mixed.m[-14:] = 0.0
    systems = [_cut(d, [0, 1], "one"), _cut(d, [0, 1, 2], "two"), W.subsample(d, 4, seed=1),
               mixed, W.subsample(d, 256, seed=2), W.subsample(W.disk_16384(), 999, seed=3)]
    m = np.concatenate([w.m for w in systems])
    qq = np.concatenate([w.q for w in systems])
    vv = np.concatenate([w.v for w in systems])
    offs = np.concatenate([[0], np.cumsum([len(w.m) for w in systems])])
    w = W.Workload("ragged", m, qq, vv, offs, d.tau, 20)
    qg, vg, enc, st, E = _run_gpu(w, 20, kick_prec=q.QYM_KICK_FP64)
    assert st["status_bits"] == 0
    for s, ws in enumerate(systems):
        a, b = int(offs[s]), int(offs[s + 1])
        r, _ = _run_oracle(oracle, ws, 20)
        mine = enc[(enc[:, 1] >= a) & (enc[:, 1] < b)].copy()
        mine[:, 1:] -= a
        skip = _compare_records(mine, r)
        keep = np.array([i not in skip for i in range(b - a)])
        _check_positions(qg[a:b][keep], r.q[keep], _chaos_spread(oracle, ws, 20)[keep])


def test_16384_disk_steps(gpu, oracle):
    """The 16384-body disk, 3 steps, FP64 kick: positions within 1e-12."""
    w = W.disk_16384()
    qg, vg, enc, st, E = _run_gpu(w, 3, kick_prec=q.QYM_KICK_FP64)
    r, vh = _run_oracle(oracle, w, 3)
    assert np.array_equal(enc, r.encounters)
    assert _relq(qg, r.q).max() <= 1e-12


def test_state_round_trip_and_resume(gpu, oracle):
    """get_state / set_state resume: 20 steps in one call equal 10 + 10 steps
    with a host round trip of the state in between."""
    w = W.subsample(W.disk_260(), 60, seed=3)
    a = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64)
    a.step(w.tau, 20)
    qa, va = a.state()
    b = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64)
    b.step(w.tau, 10)
    qm, vm = b.state()
    b.set_state(qm, vm)
    b.step(w.tau, 10)
    qb, vb = b.state()
    a.close()
    b.close()
    assert _relq(qb, qa).max() <= 1e-13


def test_set_state_of_the_held_positions_keeps_the_fused_search(gpu):
    """A state read back and set again (positions bit for bit) leaves the
    next step on the fused search (the last kick's |a| still bounds it): the
    same encounter records and state as a run without the round trip, and
    two launches fewer than after a state with one position moved, which
    searches after its kick (the stirred disk of crossers: encounters from
    the first step on)."""
    w = W.crossers()

    def run(edit):
        s = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
        s.step(w.tau, 2)
        if edit is not None:
            qs, vs = s.state()
            edit(qs)
            s.set_state(qs, vs)
        s.step(w.tau, 3)
        out = s.state(), s.encounters(), s.stats()
        s.close()
        return out

    (qa, va), ea, _ = run(None)
    (qb, vb), eb, sb = run(lambda x: None)
    (qc, vc), ec, sc = run(lambda x: x.__setitem__((7, 0), x[7, 0] * (1 + 1e-15)))
    assert sb["status_bits"] == 0 and sc["status_bits"] == 0
    assert np.array_equal(eb, ea) and _relq(qb, qa).max() <= 1e-13
    assert sc["launches"] == sb["launches"] + 2 and sc["rescans"] == 0
    assert sb["encounters"] > 0


def test_step_graphs_follow_tau(gpu):
    """A call's steps are replayed from graphs captured for its tau: after
    calls with tau, a call with tau / 2 on the same context gives the bits of
    a fresh context started from the same state (no encounters, so the first
    call's search makes no difference), and steps with -tau retrace the
    plain DH step (time reversal to rounding)."""
    w = W.disk_16384()
    # democratic-heliocentric coordinates in and out: the state read back
    # starts the fresh context bit for bit
    a = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, encounters=0, coords=1)
    a.step(w.tau, 3)
    a.step(w.tau, 3)
    qm, vm = a.state()
    b = q.Simulation(w.m, qm, vm, w.offsets, eps_H=w.eps_H, encounters=0, coords=1)
    for sim in (a, b):
        sim.step(0.5 * w.tau, 4)
    (qa, va), (qb, vb) = a.state(), b.state()
    b.close()
    assert np.array_equal(qa, qb) and np.array_equal(va, vb), (_relq(qa, qb).max(),
                                                              _relq(va, vb).max())
    a.step(-0.5 * w.tau, 4)
    a.step(-w.tau, 6)
    qr, vr = a.state()
    a.close()
    assert _relq(qr, w.q).max() <= 1e-11


def test_step_graphs_follow_the_kick_shape(gpu):
    """A launch shape set after steps were replayed from graphs is the one
    the next call runs: the same bits as a fresh context started from the same
    state with that shape."""
    w = W.disk_16384()
    a = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, encounters=0, coords=1)
    a.step(w.tau, 3)
    qm, vm = a.state()
    b = q.Simulation(w.m, qm, vm, w.offsets, eps_H=w.eps_H, encounters=0, coords=1)
    for sim in (a, b):
        q.qym_set_kick_shape(sim.ctx, 256, 1, 16)
        sim.step(w.tau, 3)
    (qa, va), (qb, vb) = a.state(), b.state()
    assert a.stats()["kick_tile_splits"] == 16
    a.close()
    b.close()
    assert np.array_equal(qa, qb) and np.array_equal(va, vb)


def test_time_drift_leaves_the_state(gpu):
    """qym_time_drift (E_Dft timed alone) puts the state back bit for bit, and
    the steps after it equal those without it; batches and single systems."""
    for w in (W.disk_260(), W.ensemble(nsys=4, n_lo=64, n_hi=300)):
        runs = []
        for timed in (False, True):
            s = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
            s.step(w.tau, 2)
            q0, v0 = s.state()
            if timed:
                mom, drift = q.qym_time_drift(s.ctx, w.tau, 3)
                assert mom > 0 and drift > 0
                q1, v1 = s.state()
                assert np.array_equal(q1, q0) and np.array_equal(v1, v0)
            s.step(w.tau, 2)
            runs.append((s.state(), s.encounters()))
            s.close()
        (qa, va), ea = runs[0]
        (qb, vb), eb = runs[1]
        assert np.array_equal(qa, qb) and np.array_equal(va, vb) and np.array_equal(ea, eb)


def test_error_statuses(gpu):
    """Capacities and caps report statuses; the context stays usable."""
    w = W.disk_260()
    wc = W.crossers()
    for search in (q.QYM_SEARCH_FUSED, q.QYM_SEARCH_BINNED):
        sim = q.Simulation(wc.m, wc.q, wc.v, wc.offsets, max_candidates=1, search=search,
                           eps_H=wc.eps_H)
        with pytest.raises(q.QymError) as e:
            sim.step(wc.tau, 5)
        assert e.value.status == q.QYM_EOVERFLOW
        sim.close()
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, max_kepler_iter=1, encounters=0)
    with pytest.raises(q.QymError) as e:
        sim.step(w.tau, 2)
    assert e.value.status == q.QYM_ENOCONV
    qq, vv = sim.state()
    assert np.all(np.isfinite(qq))
    sim.close()
    bad = w.q.copy()
    bad[5, 0] = np.nan
    with pytest.raises(q.QymError) as e:
        q.Simulation(w.m, bad, w.v, w.offsets)
    assert e.value.status == q.QYM_EINVAL


def test_ensemble_full_size_sampled(gpu, oracle):
    """The 512-system ensemble (about 1.06e6 rows, the bench's batched
    workload) stepped as one batch: sampled systems match the oracle stepping
    each alone (records equal, positions within the chaos-aware tolerance),
    no status bits, and no set larger than the oracle's."""
    w = W.ensemble()
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64)
    sim.step(w.tau, 3)
    qg, vg = sim.state()
    enc = sim.encounters()
    st = sim.stats()
    sim.close()
    assert st["status_bits"] == 0
    rng = np.random.default_rng(7)
    pick = np.concatenate([[int(np.argmax(np.diff(w.offsets)))], rng.choice(w.nsys, 5, replace=False)])
    max_set = 0
    for s in pick:
        a, b = int(w.offsets[s]), int(w.offsets[s + 1])
        ws = W.Workload("sys", w.m[a:b], w.q[a:b], w.v[a:b], np.array([0, b - a]), w.tau, 3)
        r, _ = _run_oracle(oracle, ws, 3)
        max_set = max(max_set, int(r.stats[2]))
        mine = enc[(enc[:, 1] >= a) & (enc[:, 1] < b)].copy()
        mine[:, 1:] -= a
        skip = _compare_records(mine, r)
        spread = _chaos_spread(oracle, ws, 3)
        keep = np.array([i not in skip for i in range(b - a)])
        _check_positions(qg[a:b][keep], r.q[keep], spread[keep], rel=1e-11)
    assert max_set < 320 and st["max_set"] < 320


def test_merged_kicks_equal_two_kicks(gpu, oracle):
    """merge_kicks = 1 (one kick of tau between steps inside a call, exact
    since E_Dft is a uniform shift and E_Int conserves the momentum): the
    plain DH step gives the two-kick result to rounding over 50 steps, in two
    calls (the state is synchronised at the end of each)."""
    w = W.subsample(W.disk_260(), 120, seed=4)
    a = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64, encounters=0)
    b = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=q.QYM_KICK_FP64, encounters=0,
                     merge_kicks=1)
    for sim in (a, b):
        sim.step(w.tau, 30)
        sim.step(w.tau, 20)
    qa, va = a.state()
    qb, vb = b.state()
    la, lb = a.stats()["launches"], b.stats()["launches"]
    a.close()
    b.close()
    assert _relq(qb, qa).max() <= 1e-12 and _relq(vb, va).max() <= 1e-11
    r, vh = _run_oracle(oracle, w, 50, encounters=0)
    assert _relq(qb, r.q).max() <= 1e-12
    assert lb < la   # fewer kernels: one kick and finish less per interior step


def test_merged_kicks_hybrid_step(gpu, oracle):
    """The hybrid step with merged kicks on the 260-body disk, FP64: the same
    encounter records as the oracle's two-kick step (up to pairs at the
    threshold), positions within the chaos-aware tolerance."""
    w = W.disk_260()
    qg, vg, enc, st, E = _run_gpu(w, 100, kick_prec=q.QYM_KICK_FP64, merge_kicks=1)
    r, vh = _run_oracle(oracle, w, 100)
    skip = _compare_records(enc, r)
    keep = np.array([i not in skip for i in range(len(w.m))])
    _check_positions(qg[keep], r.q[keep], _chaos_spread(oracle, w, 100)[keep])


@pytest.mark.parametrize("case", ["batch", "swarm"])
def test_repeat_runs_bit_identical(gpu, case):
    """The same calls on two fresh contexts give the same bits: every sum has
    a fixed order, and the Hermite's schedule (which large sets take
    clusters, the queue order) follows only the context's own past. A batch
    of 80 planet swarms (more large sets than the 76 two-CTA clusters, so the
    plan and the queue both matter) and one swarm on an eight-CTA cluster."""
    if case == "batch":
        sw = [_planet_swarm(30, seed=300 + s) for s in range(80)]
        w = W.Workload("swarms", np.concatenate([x.m for x in sw]),
                       np.concatenate([x.q for x in sw]), np.concatenate([x.v for x in sw]),
                       np.concatenate([[0], np.cumsum([len(x.m) for x in sw])]), sw[0].tau, 4)
    else:
        w = _planet_swarm(68, seed=7)
    runs = []
    for _ in range(2):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets)
        sim.step(w.tau, 2)
        sim.step(w.tau, 2)
        qq, vv = sim.state()
        runs.append((qq, vv, sim.encounters(), sim.stats()))
        sim.close()
    (q0, v0, e0, s0), (q1, v1, e1, s1) = runs
    assert s0["status_bits"] == 0 and s0["max_set"] >= 24
    assert np.array_equal(q0, q1) and np.array_equal(v0, v1)
    assert np.array_equal(e0, e1)
    assert s0["hermite_steps"] == s1["hermite_steps"] and s0["sets"] == s1["sets"]


def test_newton32_step_matches_laguerre(gpu, oracle):
    """The hybrid step with E_Kep by FP32 Newton steps finished in FP64
    (QYM_SOLVER_NEWTON32) against the paper's Laguerre: both stop at the same
    1e-14 residual, so 100 steps of the 260-body disk (FP64 kick) end with
    the same records and positions within the chaos-aware tolerance of the
    oracle's Laguerre run."""
    w = W.disk_260()
    n = 100
    qg, vg, enc, st, E = _run_gpu(w, n, kick_prec=q.QYM_KICK_FP64, eps_H=w.eps_H,
                                  solver=q.QYM_SOLVER_NEWTON32)
    assert st["status_bits"] == 0
    r, vh = _run_oracle(oracle, w, n, eps_H=w.eps_H)
    skip = _compare_records(enc, r)
    keep = np.array([i not in skip for i in range(len(w.m))])
    _check_positions(qg[keep], r.q[keep], _chaos_spread(oracle, w, n, eps_H=w.eps_H)[keep])
