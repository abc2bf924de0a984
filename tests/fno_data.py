"""Training data for the surrogate tests: exit-plane fields of seeded ellipsoid
phantoms computed by the FP64 oracle (coupled-wave solve, then the field just
below the sample, Eq. 9), in a pool of spawned worker processes.

The phantoms are those of the surrogate workload (32x32x8 voxels of 0.25 um,
1-8 ellipsoids with semi-axes of 2-8 voxels, x-polarised unit plane wave,
lambda = 1 um); the order count is a parameter so that a test can trade
fidelity for solve time.
"""
from __future__ import annotations

import dataclasses
import multiprocessing as mp
import os
import time

import numpy as np


def _one(args):
    seed, U = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import workloads as wl
    from oracle import cw, synth
    p = dataclasses.replace(wl.config_surrogate_sample(seed), U=U, V=U)
    t0 = time.perf_counter()
    sol = cw.solve_problem(p)
    E = synth.synthesize_direct(sol, p.Fx, p.Fy, p.z_planes)[:, 0]  # [3][64][64]
    dt = time.perf_counter() - t0
    n = p.n_volume.astype(np.complex64)                              # [8][32][32]
    return n, E.astype(np.complex64), dt


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def exit_fields(seeds, U=7, workers=None):
    """(n [S][8][32][32] complex64, E [S][3][64][64] complex64, seconds per solve [S]).

    One single-threaded worker per core: the BLAS thread limits are put in the
    environment before the workers start, so that their numpy honours them."""
    workers = workers or max(1, min(len(seeds), os.cpu_count() or 1))
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_limit_threads) as pool:
            out = pool.map(_one, [(int(s), U) for s in seeds], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    n = np.stack([o[0] for o in out])
    E = np.stack([o[1] for o in out])
    return n, E, np.array([o[2] for o in out])


def _limit_threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass
