"""One system's step split over several ranks (paper_1007_3458_gb300.split):
the orchestration (row blocks, the exchanges after each phase, the encounter
pairs gathered into one list, the Hermite of each set on the rank of its
lowest row and its members sent to the others) run as two gloo processes on
the CPU. Each rank's compute is a stand-in engine made of the oracle's own
functions applied to that rank's rows in the order of the oracle's step, so a
correct split reproduces the oracle's single-process step bit for bit: the
positions, velocities and encounter records of two ranks equal those of one
rank and of oracle.step. The same orchestration drives the GPU engine (one
libqym context per GPU) in tests/test_gpu_split.py."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1007_3458_gb300 import split as SP  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleEngine:
    """A rank's compute from the oracle's functions, on torch CPU tensors in
    the layout of the GPU engine (SoA [3][rows], barycentric velocities)."""

    def __init__(self, O, w, rank, world, prm):
        import torch
        self.O, self.w, self.prm = O, w, prm
        self.torch = torch
        self.rows = len(w.m)
        self.own = SP.split_rows(self.rows, rank, world)
        vd = O.helio_to_dh(w.m, w.v)
        R = self.rows
        t = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a).T))
        self.a = {"q": t(w.q), "v": t(vd), "q1": torch.zeros(3, R, dtype=torch.float64),
                  "v1": torch.zeros(3, R, dtype=torch.float64),
                  "rH": torch.zeros(R, dtype=torch.float64),
                  "amag": torch.zeros(R, dtype=torch.float32),
                  "hcost": torch.zeros(R, dtype=torch.int32)}
        self.enc = np.zeros((0, 2), np.int64)
        self.records = []
        self.step_no = 0
        self.members = np.zeros(0, np.int64)

    def array(self, name):
        return self.a[name]

    def sync(self):
        pass

    def sync_torch(self):
        pass

    def _get(self, name):
        return self.a[name].numpy().T.copy()

    def _put(self, name, aos, rows=None):
        x = self.a[name].numpy()
        if rows is None:
            x[:] = aos.T
        else:
            x[:, rows] = aos[rows].T

    def phase(self, ph, tau, last=0):
        O, w, prm = self.O, self.w, self.prm
        m = w.m
        lo, hi = self.own
        own = np.arange(lo, hi)
        if ph == SP.QYM_PHASE_OPEN:
            self._put("q", O.drift(m, self._get("q"), self._get("v"), 0.5 * tau))
        elif ph in (SP.QYM_PHASE_KICK1, SP.QYM_PHASE_KICK2):
            if ph == SP.QYM_PHASE_KICK2:
                self._put("q", self._get("q1"))
                self._put("v", self._get("v1"))
            q, v = self._get("q"), self._get("v")
            if len(own):
                acc = O.accel_rows(m, q, own, prm.G)
                v[own] += 0.5 * tau * acc
                self.a["amag"][lo:hi] = self.torch.from_numpy(
                    np.linalg.norm(acc, axis=1).astype(np.float32))
            self._put("v", v, own)
            if ph == SP.QYM_PHASE_KICK1:
                self.a["rH"][lo:hi] = self.torch.from_numpy(O.hill_radii(m, q, v, prm.G)[lo:hi])
        elif ph == SP.QYM_PHASE_SEARCH:
            pass
        elif ph == SP.QYM_PHASE_KEPLER:
            q, v = self._get("q"), self._get("v")
            q1, v1 = self._get("q1"), self._get("v1")
            if len(own):
                q1[own], v1[own], _, _, bad = O.kepler_drift(q[own], v[own], prm.G * m[0], tau,
                                                             prm.solver, prm.guess,
                                                             max_iter=prm.max_kepler_iter)
                assert bad == 0
            self._put("q1", q1, own)
            self._put("v1", v1, own)
        elif ph == SP.QYM_PHASE_REFINE:
            args = [self._get(n) for n in ("q", "v", "q1", "v1")]
            p, _, _ = O.encounters_rows(*args, self.a["rH"].numpy(), tau, prm.a_E, own)
            p = p[(p[:, 0] >= lo) & (p[:, 0] < hi)] if len(p) else p
            self.enc = np.unique(p, axis=0) if len(p) else np.zeros((0, 2), np.int64)
        elif ph == SP.QYM_PHASE_HERMITE:
            self.members = np.zeros(0, np.int64)
            pairs = self.all_pairs
            if len(pairs):
                rH = self.a["rH"].numpy()
                set_of, start, mem, rcrit = O.sets(self.rows, pairs, rH, prm.a_H)
                q, v = self._get("q"), self._get("v")
                q1, v1 = self._get("q1"), self._get("v1")
                hc = self.a["hcost"].numpy()
                hc[:] = 0
                mine = []
                for s in range(len(rcrit)):
                    ms = mem[start[s]:start[s + 1]]
                    if not (lo <= ms.min() < hi):
                        continue
                    mine.append(ms)
                    vc = O.kcorr(ms, m, q, v, rcrit[s], 0.5 * tau, prm.G)
                    q1[ms], v1[ms] = q[ms], vc[ms]
                    qh, vh, steps, st = O.hermite_set(ms, m, q1, v1, rcrit[s], tau, prm.G,
                                                      prm.eps_H, prm.eta, prm.eta_s,
                                                      prm.max_hermite_steps)
                    assert st == 0
                    q1[ms], v1[ms] = qh[ms], vh[ms]
                    v1 = O.kcorr(ms, m, q1, v1, rcrit[s], 0.5 * tau, prm.G)
                    hc[ms] = steps
                self._put("q1", q1)
                self._put("v1", v1)
                if mine:
                    self.members = np.concatenate(mine)
        elif ph == SP.QYM_PHASE_CLOSE:
            q = O.drift(m, self._get("q"), self._get("v"), 0.5 * tau)
            if not last:
                q = O.drift(m, q, self._get("v"), 0.5 * tau)
            self._put("q", q)
            self.step_no += 1

    def own_encounters(self):
        return self.torch.from_numpy(self.enc.astype(np.int32).reshape(-1, 2))

    def import_encounters(self, pairs):
        p = pairs.numpy().astype(np.int64).reshape(-1, 2)
        self.all_pairs = p
        self.records += [(self.step_no, int(i), int(j)) for i, j in p]

    def own_members(self):
        return self.torch.from_numpy(self.members.astype(np.int64))


class LocalComm:
    def __init__(self):
        self.rank, self.world = 0, 1

    def allgather(self, t):
        return [t.clone()]


def _workload():
    from paper_1007_3458_gb300 import workloads as W
    return W.disk_16384()


def _run(O, rank, world, comm, nsteps=3):
    w = _workload()
    prm = O.params(eps_H=w.eps_H)
    eng = OracleEngine(O, w, rank, world, prm)
    run = SP.SplitRun(eng, comm)
    run.step(w.tau, nsteps)
    q = eng.a["q"].numpy().T.copy()
    v = eng.a["v"].numpy().T.copy()
    return q, v, np.array(sorted(eng.records), np.int64).reshape(-1, 3)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    O.build()
    O.set_threads(max(1, (os.cpu_count() or 2) // world))  # results do not depend on it
    q, v, rec = _run(O, rank, world, SP.TorchComm())
    out.put((rank, q, v, rec))
    dist.barrier()
    dist.destroy_process_group()


def test_split_rows_blocks():
    """Contiguous blocks of bodies covering rows 1 .. rows-1 once, equal but
    for the last, empty past the end; the same as the library's blocks."""
    from paper_1007_3458_gb300 import lib
    lib()
    for rows, world in ((2, 1), (2, 3), (16384, 2), (16384, 3), (262145, 8), (100, 7)):
        bl = [SP.split_rows(rows, r, world) for r in range(world)]
        cover = np.concatenate([np.arange(lo, hi) for lo, hi in bl])
        assert np.array_equal(cover, np.arange(1, rows))
        sizes = [hi - lo for lo, hi in bl]
        assert len(set(s for s in sizes[:-1] if s)) <= 1
        for r in range(world):
            assert SP.split_rows_library(rows, r, world) == bl[r]


def test_split_two_gloo_ranks_equal_one_rank(oracle):
    """The 16384-body disk, 3 hybrid steps with encounters: two gloo ranks
    (each kicking, drifting and testing half of the bodies, each integrating
    the sets rooted in its half) give the same bits as one rank and as the
    oracle's own step, records included."""
    mp = pytest.importorskip("torch.multiprocessing")
    w = _workload()
    vd = oracle.helio_to_dh(w.m, w.v)
    oracle.set_threads(os.cpu_count() or 1)  # the oracle's results do not depend on it
    try:
        ref = oracle.step(w.m, w.q, vd, w.offsets, w.tau, 3, oracle.params(eps_H=w.eps_H))
        q1, v1, rec1 = _run(oracle, 0, 1, LocalComm())
    finally:
        oracle.set_threads(1)
    assert len(ref.encounters) > 0
    assert np.array_equal(q1, ref.q) and np.array_equal(v1, ref.v)
    assert np.array_equal(rec1, ref.encounters)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=600) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, q, v, rec in res:
        assert np.array_equal(q, ref.q), rank
        assert np.array_equal(v, ref.v), rank
        assert np.array_equal(rec, ref.encounters), rank
