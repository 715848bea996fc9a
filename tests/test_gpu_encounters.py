"""GPU parity of the close-encounter search (Sec. 2.3 item 4, Sec. 2.4): the
encounter records of a step are the pairs the rigorous test flags among ALL
pairs of a system, so whatever the search does first to cut the pairs down
must keep every one of them. Each test records, through
qym_set_encounter_snapshot, the exact inputs of the last step's rigorous test
(the GPU's own opening drift, first kick and Kepler drift) and requires the
GPU's records of that step to equal the oracle's all-pairs (or selected-rows)
test on those inputs, bit for bit: both sides evaluate the same FP64
expression sequence on equal inputs, so no threshold band is needed."""
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


class Snapshot:
    """Device arrays receiving the rigorous test's inputs of the last step."""

    def __init__(self, torch, sim, rows):
        self.b = [torch.empty((3, rows), dtype=torch.float64, device="cuda") for _ in range(4)]
        self.b.append(torch.empty(rows, dtype=torch.float64, device="cuda"))
        sim.set_encounter_snapshot(*self.b)

    def host(self):
        q0, v0, q1, v1 = (x.cpu().numpy().T.copy() for x in self.b[:4])
        return q0, v0, q1, v1, self.b[4].cpu().numpy()


def _last_step_records(sim, nsteps):
    enc = sim.encounters()
    return enc[enc[:, 0] == nsteps - 1][:, 1:]


def _check_hill(oracle, w, q0, v0, rH):
    """The Hill radii of the step (reading R6: at |Q| of the state entering the
    Kepler drift) agree with the oracle's to a few ulp (the device forms |Q|
    with fused multiply-adds); the records are compared with the oracle run
    on the device's radii, so they stay comparable bit for bit."""
    ref = oracle.hill_radii(w.m, q0, v0)
    body = np.ones(len(w.m), bool)
    body[w.offsets[:-1]] = False
    rel = np.abs(rH[body] - ref[body]) / np.where(ref[body] > 0, ref[body], 1.0)
    assert rel.max() <= 2e-15, rel.max()


@pytest.mark.parametrize("search", [q.QYM_SEARCH_BINNED, q.QYM_SEARCH_FUSED])
def test_dense_disk_records_sampled(torch, oracle, search):
    """The 262144-body embryo disk (64 embryos of 1e-6 among 262080
    planetesimals of 1e-11, the dense-encounter configuration), mixed kick,
    binned and fused searches: for every embryo and 64 random planetesimals,
    the step's encounter records involving them equal the oracle's test of
    those rows against all 262143 partners, on the first step of a call and on
    the last step of a three-step call (with the fused search: a search after
    a fresh kick, then one inside the kick with the |a| of the previous kick
    as allowance). The Kepler output of the step matches the oracle's drift of
    the same state on a sample of bodies, and the first kick's accelerations
    (the velocity change it made, over tau/2) match the oracle's on a sample
    within the mixed kick's 1e-6: on this disk the kick adds its 64 partial
    slots per row inside the kick (each i-block's last CTA) instead of in the
    finisher."""
    w = W.disk_262144()
    R = len(w.m)
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, search=search)
    snap = Snapshot(torch, sim, R)
    rng = np.random.default_rng(12)
    sel = np.concatenate([np.arange(1, 65), rng.choice(np.arange(65, R), 64, replace=False)])
    in_sel = np.zeros(R, bool)
    in_sel[sel] = True
    total = 0
    for nsteps in (1, 3):
        sim.step(w.tau, nsteps)
        st = sim.stats()
        assert st["status_bits"] == 0, st
        mine = _last_step_records(sim, nsteps)
        q0, v0, q1, v1, rH = snap.host()
        _check_hill(oracle, w, q0, v0, rH)
        k = rng.choice(np.arange(1, R), 2000, replace=False)
        r1, u1, *_ = oracle.kepler_drift(q0[k], v0[k], 1.0, w.tau)
        assert np.max(np.linalg.norm(q1[k] - r1, axis=1) / np.linalg.norm(r1, axis=1)) <= 1e-12
        if nsteps == 1:
            # first step of a fresh context: v0 = DH velocity + (tau/2) a(q0)
            a_gpu = (v0[k] - oracle.helio_to_dh(w.m, w.v)[k]) / (0.5 * w.tau)
            a_ref = oracle.accel_rows(w.m, q0, k)
            err = np.linalg.norm(a_gpu - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
            assert err.max() <= 1e-6, err.max()
        pairs, d2, t2 = oracle.encounters_rows(q0, v0, q1, v1, rH, w.tau, w.a_E, sel)
        ref = {tuple(p) for p in pairs.tolist()}
        got = {tuple(p) for p in mine.tolist() if in_sel[p[0]] or in_sel[p[1]]}
        assert got == ref, (sorted(ref - got)[:10], sorted(got - ref)[:10])
        total += len(ref)
    print(f"\n  {total} records checked on the sampled rows")
    assert total > 100
    sim.close()


@pytest.mark.parametrize("search", [q.QYM_SEARCH_BINNED, q.QYM_SEARCH_FUSED])
@pytest.mark.parametrize("prec, merge", [(q.QYM_KICK_MIXED, 0), (q.QYM_KICK_FP64, 0),
                                         (q.QYM_KICK_MIXED, 1)])
def test_search_superset_adversarial(torch, oracle, prec, merge, search):
    """A stirred disk (workloads.crossers: eccentric crossers up to e = 0.9,
    inclinations up to 90 deg, retrograde bodies, bodies inside a Jupiter-mass
    planet's Hill sphere at up to 1.5 times its orbital speed, hyperbolic
    flybys): on one-step calls and on the last step of four-step calls (the
    step graph, and with merged kicks the allowance of a kick a whole step
    earlier), the GPU's records equal the oracle's all-pairs rigorous test on
    the step's own inputs; for the binned search (its candidate set a superset
    by construction) and the fused one (a reach per body, audited)."""
    w = W.crossers()
    R = len(w.m)
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, kick_prec=prec, merge_kicks=merge,
                       search=search)
    snap = Snapshot(torch, sim, R)
    calls = [1] * 12 + [4, 4, 4]
    checked = 0
    for nsteps in calls:
        sim.step(w.tau, nsteps)
        st = sim.stats()
        assert st["status_bits"] == 0, st
        mine = _last_step_records(sim, nsteps)
        q0, v0, q1, v1, rH = snap.host()
        _check_hill(oracle, w, q0, v0, rH)
        pairs, d2, t2 = oracle.encounters(q0, v0, q1, v1, rH, w.tau, w.a_E)
        assert np.array_equal(mine, pairs), (len(mine), len(pairs))
        checked += len(pairs)
    print(f"\n  {checked} records over {len(calls)} checked steps")
    assert checked > 50
    sim.close()


def test_auto_search_choice(torch):
    """QYM_SEARCH_AUTO (the default) takes the binned search for one system of
    at least 65536 bodies and the fused one otherwise; qym_get_params reports
    the choice."""
    for w, want in ((W.disk_262144(), q.QYM_SEARCH_BINNED), (W.disk_16384(), q.QYM_SEARCH_FUSED),
                     (W.ensemble(nsys=4, n_lo=64, n_hi=200), q.QYM_SEARCH_FUSED)):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
        assert sim.params.search == q.QYM_SEARCH_AUTO
        assert sim.effective_params().search == want, w.name
        sim.close()


@pytest.mark.parametrize("prec, merge", [(q.QYM_KICK_MIXED, 0), (q.QYM_KICK_FP64, 0),
                                         (q.QYM_KICK_MIXED, 1)])
def test_escape_velocity_search(torch, oracle, prec, merge):
    """QYM_SEARCH_ESCAPE, the paper's own crude sweep (Sec. 2.4: a_E Hill
    radii plus the distance covered at the escape velocity over the step):
    on the 260-body disk and the stirred disk of crossers its records equal
    the oracle's all-pairs rigorous test on each step's inputs (one-step
    calls and the last step of four-step calls), with no audit or re-search
    (on the cold disk with six times the fused reach's candidates, on the
    crossers, whose fast bodies widen the fused reach, with a sixth); on a
    body at five
    times the escape speed aimed at a planetesimal (workloads.escape_flyby)
    it misses the encounter the oracle and the fused search find, as the
    paper says it can. With the mixed and the FP64 kick, and with merged kicks."""
    for w, calls in ((W.disk_260(), [1] * 6 + [4, 4]), (W.crossers(), [1] * 8 + [4, 4])):
        R = len(w.m)
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, search=q.QYM_SEARCH_ESCAPE,
                           kick_prec=prec, merge_kicks=merge)
        assert sim.effective_params().search == q.QYM_SEARCH_ESCAPE
        snap = Snapshot(torch, sim, R)
        cand = 0
        for nsteps in calls:
            sim.step(w.tau, nsteps)
            st = sim.stats()
            assert st["status_bits"] == 0 and st["rescans"] == 0, st
            cand += st["candidates"]
            mine = _last_step_records(sim, nsteps)
            q0, v0, q1, v1, rH = snap.host()
            pairs, _, _ = oracle.encounters(q0, v0, q1, v1, rH, w.tau, w.a_E)
            assert np.array_equal(mine, pairs), (w.name, len(mine), len(pairs))
        sim.close()
        fused = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, search=q.QYM_SEARCH_FUSED,
                             kick_prec=prec, merge_kicks=merge)
        fc = 0
        for nsteps in calls:
            fused.step(w.tau, nsteps)
            fc += fused.stats()["candidates"]
        fused.close()
        print(f"\n  {w.name}: candidates escape {cand}, fused {fc}")
        if w.name == "disk_260":
            assert cand > fc
    w = W.escape_flyby()
    vd = oracle.helio_to_dh(w.m, w.v)
    ref = oracle.step(w.m, w.q, vd, w.offsets, w.tau, 1, oracle.params(eps_H=w.eps_H))
    assert [tuple(x) for x in ref.encounters] == [(0, 1, 2)]
    got = {}
    for name, search in (("escape", q.QYM_SEARCH_ESCAPE), ("fused", q.QYM_SEARCH_FUSED)):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, search=search,
                           kick_prec=prec, merge_kicks=merge)
        sim.step(w.tau, 1)
        got[name] = [tuple(x) for x in sim.encounters()]
        sim.close()
    assert got["fused"] == [(0, 1, 2)] and got["escape"] == [], got


def test_snapshot_set_after_steps(torch, oracle):
    """Snapshot arrays given to a context that has already replayed its step
    graphs (captured without the snapshot copies) are filled from the next
    call on: the graphs are captured again, and the records of that call's
    last step equal the oracle's all-pairs test on the arrays' contents."""
    w = W.crossers()
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
    sim.step(w.tau, 4)
    sim.step(w.tau, 1)
    snap = Snapshot(torch, sim, len(w.m))
    for b in snap.b:
        b.fill_(float("nan"))
    sim.step(w.tau, 4)
    q0, v0, q1, v1, rH = snap.host()
    assert np.isfinite(q1).all() and np.isfinite(rH).all()
    pairs, _, _ = oracle.encounters(q0, v0, q1, v1, rH, w.tau, w.a_E)
    assert len(pairs) > 0 and np.array_equal(_last_step_records(sim, 4), pairs)
    sim.close()
