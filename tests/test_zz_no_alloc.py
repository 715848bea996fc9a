"""qym_accel_dev_static: the acceleration call for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
Called through the C ABI, twice in a row after a larger system, it must give
the same bits as qym_accel_dev with a caller workspace (the same kernels with
the same layout), and allocate nothing."""
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
    """Two calls in a row after a larger one (so that the shared array holds a
    bigger system's leftovers): bit-identical to the workspace call (same
    kernels, same layout, partial sums in a fixed order), and free device
    memory unchanged by the calls that follow the first."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    big = W.subsample(W.disk_16384(), 16000, seed=12)
    w = W.subsample(W.disk_16384(), 3000, seed=11)

    def dev(wl):
        return (len(wl.m), torch.tensor(wl.m, device="cuda"),
                torch.tensor(np.ascontiguousarray(wl.q.T), device="cuda"))

    for prec in (q.QYM_KICK_FP64, q.QYM_KICK_MIXED):
        rb, mb, qb = dev(big)
        ab = torch.empty_like(qb)
        q.qym_accel_dev_static(rb, mb, qb, ab, 1.0, prec)
        rows, m, qd = dev(w)
        ref = torch.empty_like(qd)
        work = torch.empty(q.qym_accel_workspace_bytes(rows, prec), dtype=torch.uint8, device="cuda")
        q.qym_accel_dev(rows, m, qd, ref, 1.0, prec, work)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        outs = [torch.full_like(qd, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for got in outs:  # two calls in a row share the one array
            q.qym_accel_dev_static(rows, m, qd, got, 1.0, prec)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for got in outs:
            assert np.array_equal(got.cpu().numpy(), ref), prec
    # beyond the fixed limit: a clear error, nothing launched, and the same
    # message from the library's context-free error getter
    with pytest.raises(q.QymError) as e:
        q.qym_accel_dev_static(q.QYM_STATIC_MAX_ROWS + 1, m, qd, qd, 1.0, q.QYM_KICK_MIXED)
    assert e.value.status == q.QYM_EINVAL and "limit" in str(e.value)
    assert "limit" in q.qym_last_error(None)
