"""The split step on the GPU: one system's hybrid step driven phase by phase
through qym_split_phase (paper_1007_3458_gb300.split), as one rank and as two
ranks. This run has one GPU, so the two ranks are two contexts on it, each
driven by its own host thread; their exchanges are host-side all-gathers
between the phases (no kernel waits on another context's). Results equal the
unsplit qym_step to rounding: a row's kick sums the same partial slots in the
same order whatever the block of rows it is in."""
import threading

import numpy as np
import pytest

import paper_1007_3458_gb300 as q
from paper_1007_3458_gb300 import split as SP
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


class ThreadComm:
    """All-gather between host threads of one process (one per context)."""

    def __init__(self, shared, rank, world):
        self.shared, self.rank, self.world = shared, rank, world

    def allgather(self, t):
        sh = self.shared
        sh["slots"][self.rank] = t.clone()
        sh["barrier"].wait()
        out = [sh["slots"][r].clone() for r in range(self.world)]
        sh["barrier"].wait()
        return out


class LocalComm:
    rank, world = 0, 1

    def allgather(self, t):
        return [t.clone()]


def _state(sim):
    qq, vv = sim.state()
    return qq, vv, sim.encounters(), sim.stats()


def _split_run(w, world, nsteps, **prm):
    sims = [q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, **prm) for _ in range(world)]
    engines = [SP.GpuEngine(s, r, world) for r, s in enumerate(sims)]
    if world == 1:
        SP.SplitRun(engines[0], LocalComm()).step(w.tau, nsteps)
    else:
        shared = {"slots": [None] * world, "barrier": threading.Barrier(world)}
        errs = []

        def body(r):
            try:
                SP.SplitRun(engines[r], ThreadComm(shared, r, world)).step(w.tau, nsteps)
            except BaseException as ex:  # noqa: BLE001 - reported below
                errs.append(ex)
                shared["barrier"].abort()
        th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errs, errs
    out = [_state(s) for s in sims]
    for s in sims:
        s.close()
    return out


def _relq(a, b):
    n = np.linalg.norm(b, axis=1)
    n[n == 0] = 1
    return np.linalg.norm(a - b, axis=1) / n


@pytest.mark.parametrize("prec", [q.QYM_KICK_MIXED, q.QYM_KICK_FP64])
def test_split_matches_unsplit_step(torch, prec):
    """The 16384-body disk, 4 hybrid steps: one rank and two ranks through the
    phases give the unsplit qym_step's encounter records exactly, and its
    positions and velocities to rounding (FP64 kick: 1e-13 relative,
    bit-identical unless a large set took a thread-block cluster in one run
    and not the other; mixed kick: the FP32 sums grouped in another order,
    whose rounding is the mixed kick's (up to 1e-6 of a body's
    acceleration): 1e-8 for the bodies in no encounter record of the run,
    1e-5 for those in one, where close encounters amplify it)."""
    w = W.disk_16384()
    n = 4
    ref = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, kick_prec=prec)
    ref.step(w.tau, n)
    qr, vr, er, sr = _state(ref)
    ref.close()
    assert len(er) > 0
    for world in (1, 2):
        for rank, (qq, vv, enc, st) in enumerate(_split_run(w, world, n, kick_prec=prec)):
            assert st["status_bits"] == 0, (world, rank, st)
            assert np.array_equal(enc, er), (world, rank, len(enc), len(er))
            rq, rv = _relq(qq, qr), _relq(vv, vr)
            dq, dv = rq.max(), rv.max()
            print(f"\n  world {world} rank {rank}: max rel dq {dq:.3g} dv {dv:.3g}")
            if prec == q.QYM_KICK_FP64:
                assert dq <= 1e-13 and dv <= 1e-13, (world, rank, dq, dv)
            else:
                # the unsplit step holds the bodies in Morton order (sort.cu)
                # and the split in row order, which groups the FP32 tile sums
                # differently
                inenc = np.zeros(len(w.m), bool)
                inenc[er[:, 1:].ravel()] = True
                far = ~inenc
                assert rq[far].max() <= 1e-8 and rv[far].max() <= 1e-8, (world, rank, rq[far].max(),
                                                                          rv[far].max())
                assert dq <= 1e-5 and dv <= 1e-5, (world, rank, dq, dv)


def test_split_three_ranks_uneven_blocks(torch):
    """Three ranks over a 1001-body cut of the disk (blocks of 334, 334 and
    332 bodies) and over the stirred crossers disk (823 rows: eccentric,
    inclined, retrograde and hyperbolic bodies, sets in most steps), mixed
    kick, 20 steps: every rank ends with the same bits, and they match the
    unsplit qym_step (records exactly, positions to rounding)."""
    for w in (W.subsample(W.disk_16384(), 1000, seed=21), W.crossers()):
        outs = _split_run(w, 3, 20)
        q0, v0, e0, _ = outs[0]
        for qq, vv, enc, st in outs:
            assert st["status_bits"] == 0
            assert np.array_equal(qq, q0) and np.array_equal(vv, v0) and np.array_equal(enc, e0)
        ref = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
        ref.step(w.tau, 20)
        qr, vr, er, _ = _state(ref)
        ref.close()
        assert np.array_equal(e0, er), (w.name, len(e0), len(er))
        assert _relq(q0, qr).max() <= 1e-13, (w.name, _relq(q0, qr).max())
