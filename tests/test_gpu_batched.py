"""Batched sweep (scw_plan_batched / scw_synthesize_batched) on the GPU.

Item i of a batched run must equal the single-plan scw_synthesize of item i
(rel-L2 <= 1e-6: only the order of FP32 partial sums may differ) and the FP64
oracle within the precision's tolerance. Items have uneven order counts,
layer counts, grids and wavelengths, like the wavenumbers of a sweep.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2, to_device
from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-3, "fp16": 1e-3}


def _items(seed=5):
    """Four uneven items: (U, V, L, lam, X, Fx, Fy, planes per layer)."""
    shapes = [(9, 9, 4, 10.0, 64.0, 32, 32, 4), (11, 11, 3, 8.7, 64.0, 40, 32, 4),
              (5, 7, 2, 1.0, 3.0, 24, 16, 3), (13, 13, 5, 6.0, 64.0, 64, 64, 4)]
    out = []
    for k, (U, V, L, lam, X, Fx, Fy, ppl) in enumerate(shapes):
        W, g, a, pi, pr, pt = wl.random_layer_set(seed + k, U, V, L)
        zb = np.cumsum(np.concatenate([[0.0], 0.2 + 0.1 * np.arange(L)])) * lam / 4
        ls = layerset_from_arrays(lam, X, X * 1.1, U, V, zb, W, g, a, pi, pr, pt)
        zp = wl.cell_centred_planes(zb[0], zb[-1], ppl * L)
        out.append((ls, dict(U=U, V=V, L=L, lam=lam, X=X, Y=X * 1.1, z_bounds=zb, Fx=Fx, Fy=Fy, z_planes=zp)))
    return out


@pytest.mark.parametrize("precision", ["split_bf16", "fp16", "fp32"])
def test_batched_equals_single_and_oracle(precision, cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    items = _items()
    bp = scw.BatchedPlan([kw for _, kw in items], precision=precision)
    dev = []
    for i, (ls, _) in enumerate(items):
        W, g, a, _ = to_device(ls)
        dev.append((W, g, a))
        bp.set_layers(i, W, g, a)
    outs = bp.synthesize()
    torch.cuda.synchronize()
    bp.check()
    info = bp.info()
    assert info["items"] == len(items)
    for i, (ls, kw) in enumerate(items):
        single = scw.Plan(precision=precision, **kw)
        single.set_layers(*dev[i])
        ref_gpu = single.synthesize().cpu().numpy()
        single.check()
        got = outs[i].cpu().numpy()
        assert max(rel_l2(got, ref_gpu)) <= 1e-6, i
        ref = synth.synthesize_direct(ls, kw["Fx"], kw["Fy"], kw["z_planes"])
        err = rel_l2(got, ref)
        print(precision, "item", i, "rel-L2 vs oracle", err)
        assert max(err) <= TOL[precision]
    # graph replay into the same and into new buffers
    again = bp.synthesize(outs)
    other = bp.synthesize()
    torch.cuda.synchronize()
    for i in range(len(items)):
        assert torch.equal(again[i], other[i])
    bp.check()
    # the DEVICE item table form, created on a side stream (scw_plan_batched with a stream), twice
    side = torch.cuda.Stream()
    bp2 = scw.BatchedPlan([kw for _, kw in items], precision=precision, stream=side)
    for i in range(len(items)):
        bp2.set_layers(i, *dev[i], stream=side)
    for rep in range(2):
        tab_outs = [torch.full_like(o, float("nan")) for o in outs]
        table = bp2.item_table(tab_outs)
        bp2.synthesize_table(table, stream=side)
        side.synchronize()
        bp2.check(stream=side)
        for i in range(len(items)):
            assert torch.equal(tab_outs[i], other[i]), (rep, i)
    bp2.close()


def test_sweep_items_from_real_solves(cuda_device):
    """Two wavenumbers of the mid-IR sweep (64x64x16 voxels of 1 um, sphere with a
    Lorentzian absorber), solved by the oracle, synthesised in one batch."""
    import torch
    import paper_2404_07293_gb300 as scw
    picks = [0, 40]
    sols, kws = [], []
    for i in picks:
        p = wl.config_sweep_item(i)
        sol = cw.solve_problem(p)
        sols.append(sol)
        kws.append(dict(U=p.U, V=p.V, L=p.L, lam=p.lam, X=p.X, Y=p.Y, z_bounds=p.z_bounds, Fx=p.Fx, Fy=p.Fy,
                        z_planes=p.z_planes))
    bp = scw.BatchedPlan(kws, precision="split_bf16", autotune=True)
    keep = []
    for i, sol in enumerate(sols):
        W, g, a, _ = to_device(sol)
        keep.append((W, g, a))
        bp.set_layers(i, W, g, a)
    outs = bp.synthesize()
    torch.cuda.synchronize()
    bp.check()
    assert bp.tune_report()
    for i, sol in enumerate(sols):
        zp = kws[i]["z_planes"][::7]  # every 7th plane keeps the oracle quick
        ref = synth.synthesize_direct(sol, kws[i]["Fx"], kws[i]["Fy"], zp)
        got = outs[i].cpu().numpy()[:, ::7]
        err = rel_l2(got, ref)
        print("sweep item", picks[i], "U", kws[i]["U"], "rel-L2", err)
        assert max(err) <= TOL["split_bf16"]


def test_single_plan_graph_replay_is_stable(cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    ls, kw = _items()[3]
    plan = scw.Plan(precision="split_bf16", **kw)
    W, g, a, _ = to_device(ls)
    plan.set_layers(W, g, a)
    out = torch.empty(plan.out_shape(), dtype=torch.complex64, device="cuda")
    first = plan.synthesize(out).clone()   # direct launches, then captured
    second = plan.synthesize(out).clone()  # graph replay
    third = plan.synthesize(out)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(first, second) and torch.equal(second, third)
    assert plan.info()["kernels_per_synthesis"] == 4  # phases, contraction, x-pass, y-pass


@pytest.mark.parametrize("groups", [2, 3, 5])
def test_pipelined_plan_equals_serial(groups, cuda_device):
    """Layer-group pipelining only reorders independent work: bit-identical field."""
    import torch
    import paper_2404_07293_gb300 as scw
    W, g, a, pi, pr, pt = wl.random_layer_set(21, 9, 9, 7)
    zb = np.linspace(0.0, 1.4, 8)
    ls = layerset_from_arrays(1.0, 3.0, 3.0, 9, 9, zb, W, g, a, pi, pr, pt)
    zp = np.concatenate([[-0.2], wl.cell_centred_planes(0.0, 1.4, 35), [1.6]])
    kw = dict(U=9, V=9, L=7, lam=1.0, X=3.0, Y=3.0, z_bounds=zb, Fx=32, Fy=24, z_planes=zp, exterior=True)
    dev = to_device(ls)
    serial = scw.Plan(precision="split_bf16", **kw)
    serial.set_layers(dev[0], dev[1], dev[2], *dev[3])
    ref = serial.synthesize()
    piped = scw.Plan(precision="split_bf16", **kw)
    piped.set_pipeline(groups)
    piped.set_layers(dev[0], dev[1], dev[2], *dev[3])
    out = torch.empty_like(ref)
    for _ in range(3):  # direct launch, capture, replay
        piped.synthesize(out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    piped.check()
    serial.check()
