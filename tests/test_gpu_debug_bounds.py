"""The index-check path (SCW_FLAG_DEBUG_BOUNDS) on the GPU.

A plan with the flag runs the same kernels with every global index compared
against its buffer's extent. These tests check that
  - it gives bit-identical fields to the plan without the flag (tensor-core and
    FP32 contractions, exterior planes, a batch of uneven items), and
  - a violation is caught and reported: the test lowers the extent the checks
    use for one buffer at a time (scw_plan_debug_set_extent), so that accesses
    that lie inside the real buffer count as outside. The kernels then skip
    them and scw_plan_check returns SCW_ERR_BOUNDS; no access ever leaves an
    allocation. Restoring the extent restores the exact field.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, to_device
from oracle import cw

pytestmark = pytest.mark.gpu

BOUNDS = 8  # SCW_ERR_BOUNDS


def _case(exterior):
    if not exterior:
        p = wl.config_tiny()
        sol = cw.solve_problem(p)
        return sol, p.Fx, p.Fy, p.z_planes
    W, g, a, pi, pr, pt = wl.random_layer_set(3, 9, 9, 3)
    ls = layerset_from_arrays(1.0, 2.7, 3.1, 9, 9, [0.0, 0.3, 0.31, 0.9], W, g, a, pi, pr, pt, n_top=1.0,
                              n_bot=1.3 + 0.02j, z_inc=-0.05)
    return ls, 40, 24, np.array([-0.4, -0.01, 0.0, 0.05, 0.17, 0.3, 0.31, 0.5, 0.77, 0.9, 0.95, 1.6])


def _plan(ls, Fx, Fy, zp, precision, exterior, debug):
    import paper_2404_07293_gb300 as scw
    plan = scw.Plan(ls.U, ls.V, ls.L, ls.lam, ls.X, ls.Y, ls.z_bounds, Fx, Fy, zp, precision=precision,
                    n_top=ls.n_top, n_bot=ls.n_bot, z_inc=ls.z_inc, exterior=exterior, debug_bounds=debug)
    W, g, a, ps = to_device(ls)
    plan.set_layers(W, g, a, *(ps if exterior else ()))
    return plan, (W, g, a, ps)


@pytest.mark.parametrize("precision", ["split_bf16", "fp16", "fp32"])
@pytest.mark.parametrize("exterior", [False, True])
def test_checked_plan_is_bit_identical_and_reports_lowered_extents(precision, exterior, cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    ls, Fx, Fy, zp = _case(exterior)
    ref_plan, keep = _plan(ls, Fx, Fy, zp, precision, exterior, False)
    ref = ref_plan.synthesize()
    ref_plan.check()
    plan, keep2 = _plan(ls, Fx, Fy, zp, precision, exterior, True)
    out = plan.synthesize()
    plan.check()
    assert torch.equal(out, ref)
    buffers = ["s_part", "t", "twx", "twy", "gamma", "alpha", "field"]
    buffers += ["c", "wt"] if precision == "fp32" else ["b"]
    for name in buffers:
        plan.debug_set_extent(name, 1)  # every access but the first element of the buffer counts as outside
        plan.synthesize(out)
        with pytest.raises(scw.ScwError) as e:
            plan.check()
        assert e.value.status == BOUNDS, (name, str(e.value))
        plan.debug_set_extent(name, 0)
    plan.synthesize(out)
    plan.check()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()
    ref_plan.close()


def test_checked_batch_is_bit_identical(cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    items, dev = [], []
    for k, (U, V, L, lam, X, Fx, Fy) in enumerate([(9, 9, 4, 10.0, 64.0, 32, 32), (5, 7, 2, 1.0, 3.0, 24, 16)]):
        W, g, a, pi, pr, pt = wl.random_layer_set(40 + k, U, V, L)
        zb = np.cumsum(np.concatenate([[0.0], 0.2 + 0.1 * np.arange(L)])) * lam / 4
        zp = wl.cell_centred_planes(zb[0], zb[-1], 4 * L)
        items.append(dict(U=U, V=V, L=L, lam=lam, X=X, Y=X * 1.1, z_bounds=zb, Fx=Fx, Fy=Fy, z_planes=zp))
        dev.append(tuple(torch.from_numpy(x).cuda() for x in (W, g, a)))
    outs = []
    for debug in (False, True):
        bp = scw.BatchedPlan([dict(kw, debug_bounds=debug) for kw in items], precision="split_bf16")
        for i, d in enumerate(dev):
            bp.set_layers(i, *d)
        outs.append(bp.synthesize())
        bp.check()
        bp.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
