"""Training data for the surrogate tests: exit-plane fields of seeded ellipsoid
phantoms, computed either by the FP64 oracle (coupled-wave solve, then the field
just below the sample, Eq. 9) in a pool of spawned worker processes, or by the
library's plain method on the GPU (scw_solve, then the recomposition of the
transmitted spectrum p_trn on the 64x64 exit plane) in a few host threads.

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


def exit_fields_gpu(seeds, U=15, workers=4, device="cuda"):
    """(n [S][8][32][32] complex64, E [S][3][64][64] complex64, seconds per sample [S]) from the
    library's plain method on the GPU: per sample one scw_solve (FP64) of the phantom, then the
    field just below the sample, E = sum_m p_trn,m exp(2 pi i (u x / X + v y / Y)) (Eq. 9 at
    z = z_L, Eq. 10), recomposed by scw_recompose. `workers` host threads each own a solver, a
    recompose plan and a CUDA stream (the library calls release the GIL), so that the solves of
    different samples overlap on the device. Seconds per sample are each solve's own wall time."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import paper_2404_07293_gb300 as scw
    import workloads as wl

    probs = [dataclasses.replace(wl.config_surrogate_sample(int(s)), U=U, V=U) for s in seeds]
    p0 = probs[0]
    L = p0.L
    ny, nx = p0.n_volume.shape[1:]
    n_out = np.stack([p.n_volume.astype(np.complex64) for p in probs])
    E_out = np.empty((len(seeds), 3, p0.Fy, p0.Fx), dtype=np.complex64)
    secs = np.empty(len(seeds))
    local = threading.local()
    made = []
    lock = threading.Lock()

    def ctx():
        if not hasattr(local, "solver"):
            dev = torch.device(device)
            torch.cuda.set_device(dev if dev.index is not None else torch.device("cuda", 0))
            st = torch.cuda.Stream()
            solver = scw.Solver(U, U, L, p0.lam, p0.X, p0.Y, p0.z_bounds, nx, ny)
            with torch.cuda.stream(st):
                img = torch.from_numpy(p0.incident_image.astype(np.complex128)).to(device)
                p_inc = solver.incident(img, stream=st)
            plan = scw.Plan(U, U, 1, p0.lam, p0.X, p0.Y, [0.0, 1.0], p0.Fx, p0.Fy, [0.5], precision="fp32",
                            stream=st)
            local.solver, local.stream, local.p_inc, local.plan = solver, st, p_inc, plan
            with lock:
                made.append((solver, plan))
        return local

    def one(i):
        c = ctx()
        with torch.cuda.stream(c.stream):
            nv = torch.from_numpy(probs[i].n_volume.astype(np.complex128)).to(device, non_blocking=False)
            t0 = time.perf_counter()
            _, _, _, _, pt = c.solver.solve(nv, c.p_inc, stream=c.stream)
            S = pt.to(torch.complex64).reshape(1, 3, -1).contiguous()
            E = c.plan.recompose(S, stream=c.stream)
            c.stream.synchronize()
            secs[i] = time.perf_counter() - t0
            E_out[i] = E[:, 0].cpu().numpy()

    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(one, range(len(seeds))))
    torch.cuda.synchronize()
    for solver, plan in made:
        solver.close()
        plan.close()
    return n_out, E_out, secs
