"""The C-ABI library loads without a GPU and exports every function that
include/qym.h declares; its parameter defaults and argument checks behave as
documented there (no GPU computation is run)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1007_3458_gb300 as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "qym.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qym_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    q.build()
    return q.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        ctypes.cast(getattr(lib, n), ctypes.c_void_p)


def test_header_struct_layout_matches_binding():
    # qym_params: 7 doubles, 11 int32, 5 int64 = 56 + 44 + 40 bytes, padded to 8
    assert ctypes.sizeof(q.qym_params) == 152
    assert ctypes.sizeof(q.qym_stats) == 10 * 8 + 4 * 4
    # the same fields in the same order and of the same types as the header
    txt = open(os.path.join(ROOT, "include", "qym.h")).read()
    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64}
    for struct, binding in (("qym_params", q.qym_params), ("qym_stats", q.qym_stats)):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, struct), txt, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for t, names in re.findall(r"\b(double|int32_t|int64_t)\s+([^;]+);", body):
            fields += [(n.strip(), ctype[t]) for n in names.split(",")]
        assert fields == list(binding._fields_), struct


def test_defaults(lib):
    p = q.qym_default_params()
    assert (p.G, p.a_E, p.a_H, p.eps_H, p.eta, p.eta_s) == (1.0, 3.0, 1.0, 1e-6, 0.02, 0.01)
    assert p.kick_prec == q.QYM_KICK_MIXED and p.encounters == 1 and p.max_kepler_iter == 50


def test_argument_checks_without_gpu(lib):
    p = q.qym_default_params()
    with pytest.raises(q.QymError) as e:
        q.qym_init(p, [0, 1], [1.0], np.zeros((1, 3)), np.zeros((1, 3)))
    assert e.value.status == q.QYM_EINVAL  # a system without bodies
    p.eta = -1
    with pytest.raises(q.QymError) as e:
        q.qym_init(p, [0, 2], [1.0, 1e-3], np.zeros((2, 3)), np.zeros((2, 3)))
    assert e.value.status == q.QYM_EINVAL
    p = q.qym_default_params(hermite_cluster=3)  # clusters are 2, 4 or 8 CTAs (0: automatic)
    with pytest.raises(q.QymError) as e:
        q.qym_init(p, [0, 2], [1.0, 1e-3], np.zeros((2, 3)), np.zeros((2, 3)))
    assert e.value.status == q.QYM_EINVAL
    assert lib.qym_kepler_drift_dev(-1, None, None, None, None, 1.0, 1.0, 0, 0, None, 50, None,
                                    None, None, None, None, None) == q.QYM_EINVAL
    # the learned guess needs its weights; an unknown guess or solver is refused
    assert lib.qym_kepler_drift_dev(4, None, None, None, None, 1.0, 1.0, 0, q.QYM_GUESS_MLP, None,
                                    50, None, None, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_kepler_drift_dev(4, None, None, None, None, 1.0, 1.0, 0, 7, None, 50, None,
                                    None, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_kepler_drift_dev(4, None, None, None, None, 1.0, 1.0, 3, 0, None, 50, None,
                                    None, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_mlp_workspace_bytes() >= 256 * q.QYM_MLP_NW * 4
    assert lib.qym_mlp_forward_dev(-1, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_mlp_grad_dev(0, None, None, None, None, None, 0, None) == q.QYM_EINVAL
    assert lib.qym_mlp_adam_dev(None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, None) == q.QYM_EINVAL
    assert lib.qym_mlp_train_dev(None, None, None, 0, None, 10, 4, 1, 1e-3, 1e-4, None, None, 0,
                                 None) == q.QYM_EINVAL
    assert lib.qym_set_mlp(None, None, q.QYM_MLP_NW) == q.QYM_EINVAL
    assert lib.qym_set_kepler_log(None, None, 0) == q.QYM_EINVAL
    assert lib.qym_set_encounter_snapshot(None, None, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_probe_fma(3, 10, 4, None, None, None) == q.QYM_EINVAL
    assert lib.qym_transition_dev(4, None, 0.0, None, None, None, None) == q.QYM_EINVAL
    assert lib.qym_transition_dev(0, None, 1.0, None, None, None, None) == q.QYM_OK
    assert lib.qym_accel_workspace_bytes(1, 1) == 0
    assert lib.qym_accel_workspace_bytes(16385, 1) > 16385 * 3 * 8
    # context calls refuse a NULL context or NULL outputs before any CUDA work
    d = ctypes.c_double()
    assert lib.qym_get_order(None, None) == q.QYM_EINVAL
    assert lib.qym_time_drift(None, 1.0, 3, ctypes.byref(d), ctypes.byref(d)) == q.QYM_EINVAL
    assert lib.qym_time_kick(None, 0, 3, ctypes.byref(d), None) == q.QYM_EINVAL
    # the escape-velocity search is a valid mode; other values are refused
    p = q.qym_default_params(search=7)
    with pytest.raises(q.QymError) as e:
        q.qym_init(p, [0, 2], [1.0, 1e-3], np.zeros((2, 3)), np.zeros((2, 3)))
    assert e.value.status == q.QYM_EINVAL and "QYM_SEARCH_ESCAPE" in str(e.value)


def test_mlp_layout_constants_agree():
    """The guess network's weight count is the same in the header, the
    binding, the oracle and the input generators."""
    import re
    from oracle import mlp as M
    from paper_1007_3458_gb300 import workloads as W
    hdr = open(q.HEADER).read()
    nw = int(re.search(r"#define QYM_MLP_NW (\d+)", hdr).group(1))
    assert nw == q.QYM_MLP_NW == M.NW == W.MLP_NW == 4 * 64 + 64 + 64 * 64 + 64 + 64 + 1 + 10
