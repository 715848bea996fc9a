"""qym_accel_dev_static: the acceleration call for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
Called through the C ABI, twice in a row, it must give the same result as
qym_accel_dev with a caller workspace, within the tolerances the other tests
use (FP64: 1e-12, mixed: 1e-6 relative per body)."""
import numpy as np
import pytest

import paper_1007_3458_gb300 as q
from paper_1007_3458_gb300 import workloads as W


def test_static_scratch_fits_every_allowed_size():
    q.build()
    cap = q.qym_static_scratch_bytes()
    for rows in list(range(2, 600, 7)) + list(range(600, 32769, 97)) + [32768]:
        for prec in (q.QYM_KICK_FP64, q.QYM_KICK_MIXED):
            assert q.qym_accel_workspace_bytes(rows, prec) <= cap, (rows, prec)


@pytest.mark.gpu
def test_static_scratch_accel_matches_workspace_accel():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    w = W.subsample(W.disk_16384(), 3000, seed=11)
    rows = len(w.m)
    m = torch.tensor(w.m, device="cuda")
    qd = torch.tensor(np.ascontiguousarray(w.q.T), device="cuda")
    for prec, tol in ((q.QYM_KICK_FP64, 1e-12), (q.QYM_KICK_MIXED, 1e-6)):
        ref = torch.empty_like(qd)
        work = torch.empty(q.qym_accel_workspace_bytes(rows, prec), dtype=torch.uint8, device="cuda")
        q.qym_accel_dev(rows, m, qd, ref, 1.0, prec, work)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy().T
        n = np.linalg.norm(ref, axis=1)
        for _ in range(2):  # two calls in a row share the one array
            got = torch.full_like(qd, float("nan"))
            q.qym_accel_dev_static(rows, m, qd, got, 1.0, prec)
            torch.cuda.synchronize()
            got = got.cpu().numpy().T
            assert np.all(got[0] == 0)
            err = np.linalg.norm(got - ref, axis=1)[1:] / n[1:]
            assert err.max() <= tol, (prec, err.max())
    # beyond the fixed limit: a clear error, nothing launched
    big = q.QYM_STATIC_MAX_ROWS + 1 if hasattr(q, "QYM_STATIC_MAX_ROWS") else 32769
    with pytest.raises(q.QymError) as e:
        q.qym_accel_dev_static(big, m, qd, qd, 1.0, q.QYM_KICK_MIXED)
    assert e.value.status == q.QYM_EINVAL and "limit" in str(e.value)
