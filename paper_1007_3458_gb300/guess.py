"""The learned Kepler starting guess: the method's own Kepler solves are
logged as training rows and the guess network is fitted to them on the GPU.

Rows (u1, u2, u3, u4, t) come from the Kepler kernel itself, either from
qym_step with qym_set_kepler_log (planetary systems) or from
qym_kepler_drift_dev with log_rows (test particles); the fit is
qym_mlp_train_dev (forward and backward on BF16 tensor cores, Adam on float32
master weights). PyTorch only provides device memory; every arithmetic step
runs in libqym. The network, its features and its target are described in
include/qym.h (QYM_MLP_NW).
"""
from __future__ import annotations

import numpy as np

from . import (QYM_GUESS_STANDARD, QYM_SOLVER_LAGUERRE, Simulation, qym_kepler_drift_dev,
               qym_mlp_train_dev, qym_mlp_workspace_bytes)
from . import workloads as W


def _torch():
    import torch
    return torch


def log_system_rows(w, nsteps, **params):
    """Rows of every Kepler solve of `nsteps` qym_step calls on workload w
    (bound orbits only), as a CUDA float32 tensor [rows, 5]."""
    torch = _torch()
    R = len(w.m)
    sim = Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, **params)
    log = torch.full((R * nsteps, 5), float("nan"), dtype=torch.float32, device="cuda")
    sim.set_kepler_log(log)
    sim.step(w.tau, nsteps)
    sim.close()
    return log[torch.isfinite(log).all(dim=1)].contiguous()


def log_particle_rows(qq, vv, dt, nsteps, mu=1.0, solver=QYM_SOLVER_LAGUERRE):
    """Rows of the Kepler solves of test particles (host [n, 3] states) over
    `nsteps` consecutive drifts of dt about a star of parameter mu (bound
    orbits only), as a CUDA float32 tensor."""
    torch = _torch()
    n = len(qq)
    q0 = torch.from_numpy(np.ascontiguousarray(np.asarray(qq, dtype=np.float64).T)).cuda()
    v0 = torch.from_numpy(np.ascontiguousarray(np.asarray(vv, dtype=np.float64).T)).cuda()
    q1, v1 = torch.empty_like(q0), torch.empty_like(v0)
    out = []
    for _ in range(nsteps):
        log = torch.full((n, 5), float("nan"), dtype=torch.float32, device="cuda")
        qym_kepler_drift_dev(n, q0, v0, q1, v1, mu, dt, solver, QYM_GUESS_STANDARD, None, 50,
                             log_rows=log)
        out.append(log)
        q0, q1 = q1, q0
        v0, v1 = v1, v0
    rows = torch.cat(out)
    return rows[torch.isfinite(rows).all(dim=1)].contiguous()


def fit(rows, seed=0, batch=16384, epochs=8, lr=2e-3, lr_final=2e-5):
    """Fit the guess network to CUDA rows [n, 5]: seeded shuffle, seeded
    initial weights with the normalisation of the first 200000 shuffled rows,
    Adam over `epochs` passes. Returns (weights float32 numpy, per-step
    losses numpy)."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(rows.shape[0], generator=g).to(rows.device)
    rows = rows[perm].contiguous()
    head = rows[:200000].cpu().numpy()
    w0 = W.mlp_init(seed, head[:, :4], head[:, 4])
    wd = torch.from_numpy(w0).cuda()
    md = torch.zeros_like(wd)
    vd = torch.zeros_like(wd)
    n = rows.shape[0]
    steps = ((n + batch - 1) // batch) * epochs
    losses = torch.empty(steps, dtype=torch.float32, device="cuda")
    work = torch.empty(qym_mlp_workspace_bytes(), dtype=torch.uint8, device="cuda")
    qym_mlp_train_dev(wd, md, vd, 0, rows, n, batch, epochs, lr, lr_final, losses, work)
    torch.cuda.synchronize()
    return wd.cpu().numpy(), losses.cpu().numpy()


def train_default(seed=0, disk_steps=300, particle_steps=5, **fit_kw):
    """The network used for the test-particle workload: about 1e7 rows, from
    300 steps of the 16384-body disk and 5 drifts of 1,048,576 test particles
    of seed 5 (disjoint from the seed-4 particles it is evaluated on).
    Returns (weights, losses, number of rows)."""
    torch = _torch()
    qq, vv, dt = W.test_particles(1 << 20, seed=5)
    rows = torch.cat([log_system_rows(W.disk_16384(), disk_steps),
                      log_particle_rows(qq, vv, dt, particle_steps)])
    wts, losses = fit(rows, seed=seed, **fit_kw)
    return wts, losses, int(rows.shape[0])


def train_disk_only(seed=0, disk_steps=600, **fit_kw):
    """The network fitted to planetary-system logs alone (no test particles):
    the Kepler solves of `disk_steps` steps of the 16384-body disk (seed 1).
    Its domain is the disk's (dt / P below about 0.03); on the test
    particles, which reach dt / P = 0.79, it extrapolates. Returns (weights,
    losses, number of rows)."""
    rows = log_system_rows(W.disk_16384(), disk_steps)
    wts, losses = fit(rows, seed=seed, **fit_kw)
    return wts, losses, int(rows.shape[0])


def heldout_disk(seed=8):
    """A disk drawn like the 16384-body disk from another seed, its
    planetesimals' heliocentric states and the step tau: solves the
    disk-only network has not seen."""
    w = W.outer_disk(n_planetesimals=16380, m_pl=1e-10, seed=seed, name="disk_16384_heldout")
    return w.q[5:], w.v[5:], w.tau
