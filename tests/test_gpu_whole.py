"""GPU parity of the whole-system Hermite (Sec. 2.3, last paragraph;
qym_params.whole_hermite): when a step's encounter sets put two planets in
one set, that system's step is integrated whole by the Hermite (whole.cu).
Compared with the oracle's step in the same mode on the same seeded
systems: records equal, the number of steps switched equal, positions within
the chaos-aware tolerance (two Jupiter-mass planets 0.8 AU apart are
strongly chaotic); the energy held in the encounter that the hybrid step
alone loses; the modes it refuses."""
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


def _oracle_run(oracle, w, n, **prm):
    vd = np.concatenate([oracle.helio_to_dh(w.m[a:b], w.v[a:b])
                         for a, b in zip(w.offsets[:-1], w.offsets[1:])])
    r = oracle.step(w.m, w.q, vd, w.offsets, w.tau, n, oracle.params(**prm))
    return r, vd


def _spread(oracle, w, n, **prm):
    """How far one ulp in the initial positions moves each body in the
    oracle's own run (the larger of up and down)."""
    r0, _ = _oracle_run(oracle, w, n, **prm)
    dq = np.zeros(len(w.m))
    for d in (np.inf, -np.inf):
        p = W.Workload(w.name, w.m, np.nextafter(w.q, d), w.v, w.offsets, w.tau, w.nsteps)
        r1, _ = _oracle_run(oracle, p, n, **prm)
        dq = np.maximum(dq, np.linalg.norm(r1.q - r0.q, axis=1))
    return dq


def _gpu_run(w, n, **prm):
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, **prm)
    sim.step(w.tau, n)
    qq, vv = sim.state()
    out = (qq, vv, sim.encounters(), sim.stats(), sim.energy())
    sim.close()
    return out


def test_whole_hermite_matches_oracle(gpu, oracle):
    """Two close Jupiter-mass planets and 60 planetesimals, FP64 kick, 6
    steps with the switch: every step switched on both sides, the records
    equal, every body within max(1e-11 |q|, 100 x its one-ulp spread) of the
    oracle."""
    w = W.planet_encounter()
    n = 6
    prm = dict(eps_H=w.eps_H, whole_hermite=1)
    r, vd = _oracle_run(oracle, w, n, **prm)
    wd = W.Workload(w.name, w.m, w.q, vd, w.offsets, w.tau, w.nsteps)
    qg, vg, enc, st, E = _gpu_run(wd, n, kick_prec=q.QYM_KICK_FP64, coords=1, **prm)
    assert st["status_bits"] == 0, st
    assert r.stats[6] == n and st["whole_steps"] == n, (r.stats, st)
    assert np.array_equal(enc, r.encounters)
    spread = _spread(oracle, w, n, **prm)
    tol = np.maximum(1e-11 * np.linalg.norm(r.q, axis=1), 100.0 * spread)
    err = np.linalg.norm(qg - r.q, axis=1)
    print(f"\n  max err {err.max():.3g}, max spread {spread.max():.3g}")
    assert np.all(err <= tol), np.nonzero(err > tol)[0][:5]


def test_whole_hermite_batch_and_energy(gpu, oracle):
    """A batch of the close planet pair (switches) and the 260-body disk (no
    set with two planets: steps as without the switch), FP64 kick, 20 steps:
    the pair switches as often as in the oracle's run, the disk's positions
    match the same batch stepped without the switch to 1e-13, and the pair's
    energy error stays below 1e-5 (the oracle's: 1.7e-7) where without the
    switch it exceeds 1e-2 (the oracle's: 4.6e-2)."""
    a, b = W.planet_encounter(), W.disk_260()
    w = W.Workload("batch", np.concatenate([a.m, b.m]), np.concatenate([a.q, b.q]),
                   np.concatenate([a.v, b.v]), np.array([0, len(a.m), len(a.m) + len(b.m)]),
                   a.tau, 20)
    n = 20
    on = _gpu_run(w, n, eps_H=a.eps_H, whole_hermite=1, kick_prec=q.QYM_KICK_FP64)
    off = _gpu_run(w, n, eps_H=a.eps_H, kick_prec=q.QYM_KICK_FP64)
    assert on[3]["status_bits"] == 0 and off[3]["status_bits"] == 0
    ro, _ = _oracle_run(oracle, a, n, eps_H=a.eps_H, whole_hermite=1)
    assert on[3]["whole_steps"] == ro.stats[6] > 0, (on[3], ro.stats)
    k = len(a.m)
    rel = np.linalg.norm(on[0][k + 1:] - off[0][k + 1:], axis=1) / np.linalg.norm(off[0][k + 1:], axis=1)
    assert rel.max() <= 1e-13, rel.max()
    sim = q.Simulation(w.m, w.q, w.v, w.offsets)
    E0 = sim.energy()
    sim.close()
    e_on = abs(on[4][0] / E0[0] - 1.0)
    e_off = abs(off[4][0] / E0[0] - 1.0)
    print(f"\n  energy error of the planet pair: {e_on:.3g} with the switch, {e_off:.3g} without")
    assert e_on < 1e-5 and e_off > 1e-2


def test_whole_hermite_refusals(gpu):
    """The switch needs the paper's two kicks per step and one GPU per
    system."""
    w = W.planet_encounter()
    with pytest.raises(q.QymError) as e:
        q.Simulation(w.m, w.q, w.v, w.offsets, whole_hermite=1, merge_kicks=1)
    assert e.value.status == q.QYM_EINVAL
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, whole_hermite=1)
    assert q.lib().qym_split_init(sim.ctx, 0, 2) == q.QYM_EINVAL
    sim.close()
