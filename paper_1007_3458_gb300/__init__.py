"""Python binding of libqym (include/qym.h): the democratic-heliocentric hybrid
symplectic step of Moore & Quillen on GB300 (sm_103a) CUDA kernels.

The names mirror the C ABI one for one; this module only marshals arguments
(numpy arrays for host buffers, torch CUDA tensors for device buffers) and turns
nonzero statuses into QymError. Every step of the integrator runs in the CUDA
library: when libqym.so is missing the import of a function fails loudly; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqym.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "qym.h")

QYM_OK, QYM_EINVAL, QYM_ENOMEM, QYM_ECUDA, QYM_ENAN, QYM_ENOCONV, QYM_EOVERFLOW, QYM_ENODEV = range(8)
STATUS_NAMES = ["QYM_OK", "QYM_EINVAL", "QYM_ENOMEM", "QYM_ECUDA", "QYM_ENAN", "QYM_ENOCONV",
                "QYM_EOVERFLOW", "QYM_ENODEV"]
QYM_ST_KEPLER_NOCONV, QYM_ST_HERMITE_CAP, QYM_ST_CAND_OVERFLOW, QYM_ST_ENC_OVERFLOW = 1, 2, 4, 8
QYM_ST_SET_OVERFLOW, QYM_ST_NAN, QYM_ST_UF_CAP, QYM_ST_LOG_OVERFLOW = 16, 32, 64, 128
QYM_KICK_FP64, QYM_KICK_MIXED = 0, 1
QYM_SEARCH_FUSED, QYM_SEARCH_BINNED, QYM_SEARCH_AUTO, QYM_SEARCH_ESCAPE = 0, 1, 2, 3
QYM_SOLVER_LAGUERRE, QYM_SOLVER_NEWTON, QYM_SOLVER_NEWTON32 = 0, 1, 2
QYM_GUESS_STANDARD, QYM_GUESS_R0, QYM_GUESS_MLP = 0, 1, 2
QYM_STATIC_MAX_ROWS = 32768
QYM_MLP_NW = 4555
(QYM_PHASE_OPEN, QYM_PHASE_KICK1, QYM_PHASE_SEARCH, QYM_PHASE_KEPLER, QYM_PHASE_REFINE,
 QYM_PHASE_HERMITE, QYM_PHASE_KICK2, QYM_PHASE_CLOSE) = range(8)


class QymError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


class qym_params(C.Structure):
    _fields_ = [("G", C.c_double), ("a_E", C.c_double), ("a_H", C.c_double),
                ("eps_H", C.c_double), ("eta", C.c_double), ("eta_s", C.c_double),
                ("kick_prec", C.c_int32), ("solver", C.c_int32), ("guess", C.c_int32),
                ("encounters", C.c_int32), ("coords", C.c_int32), ("hill_fixed", C.c_int32),
                ("max_kepler_iter", C.c_int32), ("device", C.c_int32),
                ("max_hermite_steps", C.c_int64), ("max_candidates", C.c_int64),
                ("max_encounters", C.c_int64), ("max_log", C.c_int64),
                ("l2_flush_bytes", C.c_int64), ("heavy_mass", C.c_double),
                ("merge_kicks", C.c_int32), ("hermite_cluster", C.c_int32),
                ("search", C.c_int32), ("whole_hermite", C.c_int32),
                ("planet_mass", C.c_double)]


class qym_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("candidates", C.c_int64), ("encounters", C.c_int64),
                ("sets", C.c_int64), ("max_set", C.c_int64), ("kepler_iters", C.c_int64),
                ("hermite_steps", C.c_int64), ("rescans", C.c_int64), ("launches", C.c_int64),
                ("hermite_steps_max", C.c_int64),
                ("status_bits", C.c_int32), ("kick_tile_i", C.c_int32),
                ("kick_tile_splits", C.c_int32), ("whole_steps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qym_split_view(C.Structure):
    _fields_ = [("rows", C.c_int64), ("own_lo", C.c_int64), ("own_hi", C.c_int64),
                ("q", C.c_void_p), ("v", C.c_void_p), ("q1", C.c_void_p), ("v1", C.c_void_p),
                ("rH", C.c_void_p), ("amag", C.c_void_p), ("hcost", C.c_void_p),
                ("enc", C.c_void_p), ("max_enc", C.c_int64), ("set_mem", C.c_void_p),
                ("stream", C.c_void_p)]


_lib = None
P = C.c_void_p
D = C.POINTER(C.c_double)
I64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """The loaded libqym.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqym.so is not built ({LIB_PATH}); run paper_1007_3458_gb300.build()")
    L = C.CDLL(LIB_PATH)
    S = C.c_int
    L.qym_default_params.argtypes = [C.POINTER(qym_params)]
    L.qym_init.argtypes = [C.POINTER(qym_params), C.c_int32, I64, D, D, D, C.POINTER(P)]
    L.qym_step.argtypes = [P, C.c_double, C.c_int64]
    L.qym_get_state.argtypes = [P, D, D]
    L.qym_set_state.argtypes = [P, D, D]
    L.qym_get_encounters.argtypes = [P, I64, C.c_int64, I64]
    L.qym_energy.argtypes = [P, D]
    L.qym_get_order.argtypes = [P, C.POINTER(C.c_int32)]
    L.qym_get_stats.argtypes = [P, C.POINTER(qym_stats)]
    L.qym_get_params.argtypes = [P, C.POINTER(qym_params)]
    L.qym_set_mlp.argtypes = [P, C.POINTER(C.c_float), C.c_int64]
    L.qym_last_error.argtypes = [P]
    L.qym_last_error.restype = C.c_char_p
    L.qym_destroy.argtypes = [P]
    L.qym_destroy.restype = None
    L.qym_shape.argtypes = [P, I64, C.POINTER(C.c_int32)]
    L.qym_get_stream.argtypes = [P, C.POINTER(P)]
    L.qym_time_kick.argtypes = [P, C.c_int32, C.c_int32, D, I64]
    L.qym_time_drift.argtypes = [P, C.c_double, C.c_int32, D, D]
    L.qym_autotune.argtypes = [P]
    L.qym_set_kick_shape.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
    L.qym_kepler_drift_dev.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_int32,
                                       C.c_int32, P, C.c_int32, P, P, P, P, P, P]
    L.qym_set_kepler_log.argtypes = [P, P, C.c_int64]
    L.qym_set_encounter_snapshot.argtypes = [P, P, P, P, P, P]
    L.qym_probe_fma.argtypes = [C.c_int32, C.c_int64, C.c_int32, D, D, P]
    L.qym_split_rows.argtypes = [C.c_int64, C.c_int32, C.c_int32, I64, I64]
    L.qym_split_rows.restype = None
    L.qym_split_init.argtypes = [P, C.c_int32, C.c_int32]
    L.qym_split_phase.argtypes = [P, C.c_int32, C.c_double, C.c_int32]
    L.qym_split_arrays.argtypes = [P, C.POINTER(qym_split_view)]
    L.qym_split_encounter_count.argtypes = [P, I64]
    L.qym_split_import_encounters.argtypes = [P, P, C.c_int64]
    L.qym_split_owned_members.argtypes = [P, I64, I64]
    L.qym_transition_dev.argtypes = [C.c_int64, P, C.c_double, P, P, P, P]
    L.qym_mlp_workspace_bytes.argtypes = []
    L.qym_mlp_workspace_bytes.restype = C.c_size_t
    L.qym_mlp_forward_dev.argtypes = [C.c_int64, P, P, P, P]
    L.qym_mlp_grad_dev.argtypes = [C.c_int64, P, P, P, P, P, C.c_size_t, P]
    L.qym_mlp_adam_dev.argtypes = [P, P, P, P, C.c_int64, C.c_float, C.c_float, C.c_float,
                                   C.c_float, P]
    L.qym_mlp_train_dev.argtypes = [P, P, P, C.c_int64, P, C.c_int64, C.c_int64, C.c_int32,
                                    C.c_float, C.c_float, P, P, C.c_size_t, P]
    L.qym_accel_workspace_bytes.argtypes = [C.c_int64, C.c_int32]
    L.qym_accel_workspace_bytes.restype = C.c_size_t
    L.qym_accel_dev.argtypes = [C.c_int64, P, P, P, C.c_double, C.c_int32, C.c_double, P,
                                C.c_size_t, P]
    L.qym_accel_dev_static.argtypes = [C.c_int64, P, P, P, C.c_double, C.c_int32, C.c_double, P]
    L.qym_accel_dev_static.restype = C.c_int
    L.qym_static_scratch_bytes.argtypes = []
    L.qym_static_scratch_bytes.restype = C.c_size_t
    L.qym_static_last_error.argtypes = []
    L.qym_static_last_error.restype = C.c_char_p
    L.qym_encounter_test_dev.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, C.c_double,
                                         C.c_int64, P, P, P, P]
    L.qym_energy_workspace_bytes.argtypes = [C.c_int64]
    L.qym_energy_workspace_bytes.restype = C.c_size_t
    L.qym_energy_dev.argtypes = [C.c_int64, P, P, P, C.c_double, P, P, C.c_size_t, P]
    for name in ("qym_default_params", "qym_init", "qym_step", "qym_get_state", "qym_set_state",
                 "qym_get_encounters", "qym_get_order", "qym_energy", "qym_get_stats", "qym_get_params",
                 "qym_set_mlp", "qym_shape",
                 "qym_get_stream", "qym_time_kick", "qym_time_drift", "qym_autotune", "qym_set_kick_shape",
                 "qym_kepler_drift_dev", "qym_accel_dev", "qym_encounter_test_dev",
                 "qym_energy_dev", "qym_set_kepler_log", "qym_mlp_forward_dev",
                 "qym_mlp_grad_dev", "qym_mlp_adam_dev", "qym_mlp_train_dev",
                 "qym_transition_dev", "qym_set_encounter_snapshot", "qym_probe_fma",
                 "qym_split_init", "qym_split_phase", "qym_split_arrays",
                 "qym_split_encounter_count", "qym_split_import_encounters",
                 "qym_split_owned_members"):
        getattr(L, name).restype = S
    _lib = L
    return L


def _check(st, ctx=None):
    if st != QYM_OK:
        msg = lib().qym_last_error(ctx)
        raise QymError(st, msg.decode() if msg else "")


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _d(a):
    return a.ctypes.data_as(D)


# ---------------------------------------------------------------- context API
def qym_default_params(**kw) -> qym_params:
    p = qym_params()
    _check(lib().qym_default_params(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def qym_init(params: qym_params, offsets, m, q, v):
    """Create a context; returns an opaque handle (int)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    m = _f64(m)
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3))
    if not (len(m) == q.shape[0] == v.shape[0] == offsets[-1]):
        raise ValueError("m, q, v must have offsets[-1] rows")
    h = P()
    _check(lib().qym_init(C.byref(params), len(offsets) - 1, offsets.ctypes.data_as(I64), _d(m),
                          _d(q), _d(v), C.byref(h)))
    return h.value


def qym_step(ctx, tau: float, nsteps: int):
    _check(lib().qym_step(ctx, tau, nsteps), ctx)


def qym_shape(ctx):
    r = C.c_int64()
    n = C.c_int32()
    _check(lib().qym_shape(ctx, C.byref(r), C.byref(n)), ctx)
    return r.value, n.value


def qym_get_stream(ctx) -> int:
    h = P()
    _check(lib().qym_get_stream(ctx, C.byref(h)), ctx)
    return h.value or 0


def qym_time_drift(ctx, tau, reps=10):
    """(ms per momentum reduction, ms per drift + pack), state unchanged."""
    a, b = C.c_double(), C.c_double()
    _check(lib().qym_time_drift(ctx, tau, reps, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def qym_time_kick(ctx, with_search=0, reps=10):
    """(mean ms per launch of the kick kernel, ordered pairs per launch)"""
    ms = C.c_double()
    pairs = C.c_int64()
    _check(lib().qym_time_kick(ctx, with_search, reps, C.byref(ms), C.byref(pairs)), ctx)
    return ms.value, pairs.value


def qym_autotune(ctx):
    _check(lib().qym_autotune(ctx), ctx)


def qym_set_kick_shape(ctx, threads, ipt, splits):
    _check(lib().qym_set_kick_shape(ctx, threads, ipt, splits), ctx)


def qym_get_state(ctx, q=None, v=None):
    """Positions and velocities [rows, 3]; q and v, when given, are filled in
    place (C-contiguous float64 [rows, 3], e.g. views of pinned memory)."""
    rows, _ = qym_shape(ctx)
    q = np.empty((rows, 3)) if q is None else q
    v = np.empty((rows, 3)) if v is None else v
    for a in (q, v):
        if a.dtype != np.float64 or a.shape != (rows, 3) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("qym_get_state: buffers must be C-contiguous float64 [rows, 3]")
    _check(lib().qym_get_state(ctx, _d(q), _d(v)), ctx)
    return q, v


def qym_set_state(ctx, q, v):
    q = _f64(q, (-1, 3))
    v = _f64(v, (-1, 3))
    _check(lib().qym_set_state(ctx, _d(q), _d(v)), ctx)


def qym_get_encounters(ctx):
    """(step, i, j) records of the last qym_step call, sorted, int64 [k, 3]."""
    cnt = C.c_int64()
    _check(lib().qym_get_encounters(ctx, None, 0, C.byref(cnt)), ctx)
    out = np.zeros((max(cnt.value, 1), 3), dtype=np.int64)
    _check(lib().qym_get_encounters(ctx, out.ctypes.data_as(I64), cnt.value, C.byref(cnt)), ctx)
    return out[:cnt.value]


def qym_get_order(ctx):
    """The kick's body order, int32 [rows]: position p holds row order[p]."""
    rows, _ = qym_shape(ctx)
    out = np.zeros(rows, dtype=np.int32)
    _check(lib().qym_get_order(ctx, out.ctypes.data_as(C.POINTER(C.c_int32))), ctx)
    return out


def qym_energy(ctx):
    _, nsys = qym_shape(ctx)
    E = np.zeros(nsys)
    _check(lib().qym_energy(ctx, _d(E)), ctx)
    return E


def qym_get_stats(ctx) -> qym_stats:
    s = qym_stats()
    _check(lib().qym_get_stats(ctx, C.byref(s)), ctx)
    return s


def qym_get_params(ctx) -> qym_params:
    """The parameters the context runs with (the library's choices filled in)."""
    p = qym_params()
    _check(lib().qym_get_params(ctx, C.byref(p)), ctx)
    return p


def qym_set_mlp(ctx, weights):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(lib().qym_set_mlp(ctx, w.ctypes.data_as(C.POINTER(C.c_float)), len(w)), ctx)


def qym_set_kepler_log(ctx, rows, cap=None):
    """rows: CUDA float32 tensor [cap, 5] (None stops logging)."""
    if rows is None:
        _check(lib().qym_set_kepler_log(ctx, None, 0), ctx)
    else:
        cap = rows.shape[0] if cap is None else cap
        _check(lib().qym_set_kepler_log(ctx, _ptr(rows), cap), ctx)


def qym_set_encounter_snapshot(ctx, q0=None, v0=None, q1=None, v1=None, rH=None):
    """CUDA float64 tensors [3, rows] (q0, v0, q1, v1) and [rows] (rH) that
    receive the rigorous encounter test's inputs of the last step of each
    following qym_step call; all None stops recording."""
    _check(lib().qym_set_encounter_snapshot(ctx, _ptr(q0), _ptr(v0), _ptr(q1), _ptr(v1),
                                            _ptr(rH)), ctx)


def qym_probe_fma(kind, iters=1 << 16, blocks_per_sm=4, stream=None):
    """Measured FMA throughput of the device (kind 0: FP32 FFMA, 1: FP32x2
    FFMA2, 2: FP64 DFMA): (TFLOP/s, ms)."""
    tf = C.c_double()
    ms = C.c_double()
    _check(lib().qym_probe_fma(kind, iters, blocks_per_sm, C.byref(tf), C.byref(ms),
                               _stream(stream)))
    return tf.value, ms.value


def qym_last_error(ctx=None) -> str:
    s = lib().qym_last_error(ctx)
    return s.decode() if s else ""


def qym_destroy(ctx):
    lib().qym_destroy(ctx)


# ---------------------------------------------------------------- device-level calls
def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def qym_kepler_drift_dev(n, q0, v0, q1, v1, mu, dt, solver=0, guess=0, mlp_w=None,
                         max_iter=50, x_out=None, x0_out=None, iters=None, log_rows=None,
                         status=None, stream=None):
    """Tensors are CUDA float64 [3, n] (mlp_w float32 [QYM_MLP_NW], x_out and
    x0_out float64 [n], iters / status int32, log_rows float32 [n, 5])."""
    _check(lib().qym_kepler_drift_dev(n, _ptr(q0), _ptr(v0), _ptr(q1), _ptr(v1), mu, dt, solver,
                                      guess, _ptr(mlp_w), max_iter, _ptr(x_out), _ptr(x0_out),
                                      _ptr(iters), _ptr(log_rows), _ptr(status), _stream(stream)))


def qym_transition_dev(n, s, r_crit, K, Kp, Kpp, stream=None):
    """CUDA float64 tensors [n]: K(s), K'(s), K''(s) of the transition function."""
    _check(lib().qym_transition_dev(n, _ptr(s), r_crit, _ptr(K), _ptr(Kp), _ptr(Kpp),
                                    _stream(stream)))


def qym_mlp_workspace_bytes() -> int:
    return int(lib().qym_mlp_workspace_bytes())


def qym_mlp_forward_dev(n, w, u, y, stream=None):
    """w float32 [QYM_MLP_NW], u float32 [n, 4], y float32 [n] (CUDA)."""
    _check(lib().qym_mlp_forward_dev(n, _ptr(w), _ptr(u), _ptr(y), _stream(stream)))


def qym_mlp_grad_dev(n, w, rows, grad, loss, work, work_bytes=None, stream=None):
    wb = work.numel() * work.element_size() if work_bytes is None else work_bytes
    _check(lib().qym_mlp_grad_dev(n, _ptr(w), _ptr(rows), _ptr(grad), _ptr(loss), _ptr(work), wb,
                                  _stream(stream)))


def qym_mlp_adam_dev(w, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().qym_mlp_adam_dev(_ptr(w), _ptr(m), _ptr(v), _ptr(grad), t, lr, beta1, beta2, eps,
                                  _stream(stream)))


def qym_mlp_train_dev(w, m, v, t0, rows, n, batch, epochs, lr, lr_final, losses, work,
                      work_bytes=None, stream=None):
    wb = work.numel() * work.element_size() if work_bytes is None else work_bytes
    _check(lib().qym_mlp_train_dev(_ptr(w), _ptr(m), _ptr(v), t0, _ptr(rows), n, batch, epochs, lr,
                                   lr_final, _ptr(losses), _ptr(work), wb, _stream(stream)))


def qym_accel_workspace_bytes(rows, prec) -> int:
    return int(lib().qym_accel_workspace_bytes(rows, prec))


def qym_accel_dev(rows, m, q, a, G, prec, work, work_bytes=None, stream=None, heavy_mass=1e-7):
    wb = work.numel() * work.element_size() if work_bytes is None else work_bytes
    _check(lib().qym_accel_dev(rows, _ptr(m), _ptr(q), _ptr(a), G, prec, heavy_mass, _ptr(work),
                               wb, _stream(stream)))


def qym_accel_dev_static(rows, m, q, a, G, prec, heavy_mass=1e-7, stream=None):
    """qym_accel_dev with the library's fixed scratch array (allocates nothing)."""
    st = lib().qym_accel_dev_static(rows, _ptr(m), _ptr(q), _ptr(a), G, prec, heavy_mass,
                                    _stream(stream))
    if st != QYM_OK:
        msg = lib().qym_static_last_error()
        raise QymError(st, msg.decode() if msg else "")


def qym_static_scratch_bytes() -> int:
    return int(lib().qym_static_scratch_bytes())


def qym_encounter_test_dev(rows, q0, v0, q1, v1, rH, tau, a_E, npairs, pairs, d2, flag,
                           stream=None):
    _check(lib().qym_encounter_test_dev(rows, _ptr(q0), _ptr(v0), _ptr(q1), _ptr(v1), _ptr(rH),
                                        tau, a_E, npairs, _ptr(pairs), _ptr(d2), _ptr(flag),
                                        _stream(stream)))


def qym_energy_workspace_bytes(rows) -> int:
    return int(lib().qym_energy_workspace_bytes(rows))


def qym_energy_dev(rows, m, q, v, G, E, work, work_bytes=None, stream=None):
    wb = work.numel() * work.element_size() if work_bytes is None else work_bytes
    _check(lib().qym_energy_dev(rows, _ptr(m), _ptr(q), _ptr(v), G, _ptr(E), _ptr(work), wb,
                                _stream(stream)))


# ---------------------------------------------------------------- convenience
class Simulation:
    """Owns one context: a batch of planetary systems resident on the GPU."""

    def __init__(self, m, q, v, offsets=None, **params):
        m = np.asarray(m)
        offsets = np.array([0, len(m)]) if offsets is None else offsets
        self.params = qym_default_params(**params)
        self.ctx = qym_init(self.params, offsets, m, q, v)

    def step(self, tau, nsteps=1):
        qym_step(self.ctx, tau, nsteps)

    def state(self):
        return qym_get_state(self.ctx)

    def set_state(self, q, v):
        qym_set_state(self.ctx, q, v)

    def encounters(self):
        return qym_get_encounters(self.ctx)

    def energy(self):
        return qym_energy(self.ctx)

    def order(self):
        return qym_get_order(self.ctx)

    def stats(self):
        return qym_get_stats(self.ctx).as_dict()

    def effective_params(self):
        return qym_get_params(self.ctx)

    def set_mlp(self, weights):
        qym_set_mlp(self.ctx, weights)

    def set_kepler_log(self, rows, cap=None):
        qym_set_kepler_log(self.ctx, rows, cap)

    def set_encounter_snapshot(self, q0=None, v0=None, q1=None, v1=None, rH=None):
        qym_set_encounter_snapshot(self.ctx, q0, v0, q1, v1, rH)

    def close(self):
        if self.ctx:
            qym_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
