"""The kick's body order (sort.cu) read back through qym_get_order: bodies
ordered by (Morton code, row), the code from the positions scaled into the
cube over the system's bounding box (10 bits per axis, FP32), recomputed here
with numpy's IEEE FP32 arithmetic, at sizes of one and of several sort
blocks (2048 keys each) with ragged ends."""
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


def _spread10(b):
    x = b.astype(np.uint32) & np.uint32(0x3FF)
    x = (x | (x << np.uint32(16))) & np.uint32(0x030000FF)
    x = (x | (x << np.uint32(8))) & np.uint32(0x0300F00F)
    x = (x | (x << np.uint32(4))) & np.uint32(0x030C30C3)
    x = (x | (x << np.uint32(2))) & np.uint32(0x09249249)
    return x


def _host_order(qpos):
    x = qpos[1:].astype(np.float32)
    lo = x.min(axis=0)
    hi = -((-x).min(axis=0))
    span = np.float32(0.0)
    for c in range(3):
        span = max(span, np.float32(hi[c] - lo[c]))
    code = np.zeros(len(x), dtype=np.uint32)
    for c in range(3):
        u = (x[:, c] - lo[c]) / span if span > 0 else np.zeros(len(x), np.float32)
        u = np.clip(u.astype(np.float32), np.float32(0), np.float32(1))
        b = np.minimum((u * np.float32(1024.0)).astype(np.uint32), np.uint32(1023))
        code |= _spread10(b) << np.uint32(c)
    rows = np.arange(1, len(qpos), dtype=np.int64)
    key = (code.astype(np.uint64) << np.uint64(32)) | rows.astype(np.uint64)
    return np.concatenate([[0], (np.sort(key) & np.uint64(0xFFFFFFFF)).astype(np.int64)])


@pytest.mark.parametrize("make", [lambda: W.outer_disk(3000, 1e-9, seed=5), W.disk_16384,
                                  lambda: W.outer_disk(20479, 1e-10, seed=5)],
                         ids=["3005", "16384", "20484"])
def test_kick_order_is_the_morton_order(gpu, make):
    """After qym_set_state and after steps: the order equals the host's
    (code, row) order of the positions it was taken from."""
    w = make()
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H)
    qs, vs = sim.state()
    sim.set_state(qs, vs)
    got = sim.order()
    assert np.array_equal(np.sort(got), np.arange(len(w.m)))
    assert np.array_equal(got, _host_order(qs))
    # every qym_step call takes the order from the positions it starts from
    sim.step(w.tau, 2)
    q2, _ = sim.state()
    sim.step(w.tau, 1)
    assert np.array_equal(sim.order(), _host_order(q2))
    sim.close()


def test_order_is_the_identity_without_the_sort(gpu):
    """A batch of systems, a system below 2048 bodies, and the FP64 kick
    keep row order."""
    for w, prm in ((W.ensemble(nsys=4, n_lo=64, n_hi=256), {}), (W.disk_260(), {}),
                   (W.outer_disk(3000, 1e-9, seed=5), {"kick_prec": q.QYM_KICK_FP64})):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, **prm)
        sim.step(w.tau, 1)
        assert np.array_equal(sim.order(), np.arange(len(w.m)))
        sim.close()
