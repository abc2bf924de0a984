"""scw_recompose_noalloc against the plan-based scw_recompose, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory (a host framework's own pool, loops that must not pay cudaMalloc's
implicit synchronisation, processes that forbid allocation after start-up).
It must give the same field as the plan path and as the FP64 oracle's direct
sum of Eq. 10; two calls in a row with different sizes also check that the
shared fixed scratch, which keeps the previous call's contents, never leaks
into a result. This file is collected
last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 recompose tolerance used by the other GPU tests


def _rel(a, b):
    return [float(np.linalg.norm(a[c] - b[c]) / np.linalg.norm(b[c])) for c in range(3)]


def test_noalloc_matches_plan_recompose_two_calls(cuda_device):
    import torch

    import paper_2404_07293_gb300 as scw
    from paper_2404_07293_gb300 import _lib

    lib = _lib.load()
    cases = [(21, 21, 16.0, 16.0, 256, 256, 6, 0.0, 0.0),
             (9, 5, 2.7, 3.1, 40, 24, 5, 0.2, -0.3)]
    for call, (U, V, X, Y, Fx, Fy, Fz, x0, y0) in enumerate(cases):
        rng = np.random.default_rng(100 + call)
        S = (rng.standard_normal((Fz, 3, U * V)) + 1j * rng.standard_normal((Fz, 3, U * V))).astype(np.complex64)
        Sd = torch.from_numpy(S).to(cuda_device)
        plan = scw.Plan(U, V, 1, 1.0, X, Y, [0.0, 1.0], Fx, Fy, np.linspace(0.1, 0.9, Fz), x0=x0, y0=y0,
                        precision="fp32")
        ref = plan.recompose(Sd).cpu().numpy()
        plan.check()
        out = torch.empty((3, Fz, Fy, Fx), dtype=torch.complex64, device=cuda_device)
        st = lib.scw_recompose_noalloc(U, V, X, Y, Fx, Fy, Fz, x0, y0, ctypes.c_void_p(Sd.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, lib.scw_last_error()
        torch.cuda.synchronize()
        err = _rel(out.cpu().numpy(), ref)
        print("no-alloc call", call, "rel-L2 vs plan recompose", err)
        assert max(err) <= TOL
        ls = cw.LayerSet(lam=1.0, X=X, Y=Y, U=U, V=V, z_bounds=np.array([0.0, 1.0]), W=None, gamma=None,
                         alpha=None, p_inc=None, p_ref=None, p_trn=None)
        xs, ys = synth.pixel_coords(ls, Fx, Fy, x0, y0)
        got = out.cpu().numpy()
        for f in range(Fz):
            ora = synth.field_direct(ls, S[f].astype(np.complex128), xs, ys)
            assert max(_rel(got[:, f], ora)) <= TOL, (call, f)
        plan.close()

