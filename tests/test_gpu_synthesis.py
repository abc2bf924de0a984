"""GPU parity: libscw (through the C ABI) against the FP64 oracle.

Tolerances (per-component relative L2, ||E_gpu - E_oracle|| / ||E_oracle||):
  FP32 path 1e-5, split-BF16 and FP16 paths 1e-3 (the targets of the method's
  GPU synthesis). The recompose step alone is FP32 everywhere: 1e-5.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2, to_device
from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-3, "fp16": 1e-3}


def _plan(ls, Fx, Fy, zp, precision, **kw):
    import paper_2404_07293_gb300 as scw
    return scw.Plan(ls.U, ls.V, ls.L, ls.lam, ls.X, ls.Y, ls.z_bounds, Fx, Fy, zp, precision=precision,
                    n_top=ls.n_top, n_bot=ls.n_bot, z_inc=ls.z_inc, **kw)


def _run(ls, Fx, Fy, zp, precision, x0=0.0, y0=0.0, exterior=False, k_split=0):
    import torch
    plan = _plan(ls, Fx, Fy, zp, precision, x0=x0, y0=y0, exterior=exterior, k_split=k_split)
    W, g, a, ps = to_device(ls)
    if exterior:
        plan.set_layers(W, g, a, *ps)
    else:
        plan.set_layers(W, g, a)
    out = plan.synthesize()
    S = plan.spectrum()
    torch.cuda.synchronize()
    plan.check()
    return plan, out.cpu().numpy(), S.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    ref = synth.synthesize_direct(sol, p.Fx, p.Fy, p.z_planes)
    return p, sol, ref


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "fp16"])
def test_tiny_volume(tiny, precision, cuda_device):
    p, sol, ref = tiny
    _, E, S = _run(sol, p.Fx, p.Fy, p.z_planes, precision)
    err = rel_l2(E, ref)
    print(precision, "rel-L2 per component", err)
    assert max(err) <= TOL[precision]
    Sref = synth.spectra(sol, p.z_planes)
    serr = np.linalg.norm(S - Sref) / np.linalg.norm(Sref)
    assert serr <= TOL[precision]


@pytest.mark.parametrize("U,V,Fx,Fy,x0,y0", [
    (7, 7, 64, 64, 0.0, 0.0), (9, 5, 24, 40, 0.3, -1.1), (11, 3, 8, 16, 0.5, 0.2), (21, 21, 256, 256, 0.0, 0.0),
    (25, 25, 128, 128, 1.7, 0.4), (1, 1, 16, 8, 0.0, 0.0)])
def test_recompose_matches_direct_sum(U, V, Fx, Fy, x0, y0, cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    rng = np.random.default_rng(U * 100 + Fx)
    M, Fz, X, Y = U * V, 3, 4.0, 3.0
    S = (rng.standard_normal((Fz, 3, M)) + 1j * rng.standard_normal((Fz, 3, M))).astype(np.complex64)
    plan = scw.Plan(U, V, 1, 1.0, X, Y, [0.0, 1.0], Fx, Fy, np.linspace(0.1, 0.9, Fz), x0=x0, y0=y0,
                    precision="fp32")
    E = plan.recompose(torch.from_numpy(S).cuda()).cpu().numpy()
    plan.check()
    ls = cw.LayerSet(lam=1.0, X=X, Y=Y, U=U, V=V, z_bounds=np.array([0.0, 1.0]), W=None, gamma=None,
                     alpha=None, p_inc=None, p_ref=None, p_trn=None)
    xs, ys = synth.pixel_coords(ls, Fx, Fy, x0, y0)
    for f in range(Fz):
        ref = synth.field_direct(ls, S[f].astype(np.complex128), xs, ys)
        assert max(rel_l2(E[:, f], ref)) <= 1e-5


def _edge_problem(seed=3, U=9, V=9):
    W, g, a, pi, pr, pt = wl.random_layer_set(seed, U, V, 3)
    zb = np.array([0.0, 0.3, 0.31, 0.9])
    ls = layerset_from_arrays(1.0, 2.7, 3.1, U, V, zb, W, g, a, pi, pr, pt, n_top=1.0, n_bot=1.3 + 0.02j,
                              z_inc=-0.05)
    # above, on z0, inside layer 1, on both interfaces, layer 3 (layer 2 gets only its boundary), on zL, below
    zp = np.array([-0.4, -0.01, 0.0, 0.05, 0.17, 0.3, 0.31, 0.5, 0.77, 0.9, 0.95, 1.6])
    return ls, zp


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "fp16"])
@pytest.mark.parametrize("k_split", [0, 1, 3])
def test_edges_exterior_boundaries_ragged(precision, k_split, cuda_device):
    ls, zp = _edge_problem()
    Fx, Fy = 40, 24
    _, E, S = _run(ls, Fx, Fy, zp, precision, x0=0.2, y0=-0.3, exterior=True, k_split=k_split)
    Sref = synth.spectra(ls, zp)
    ref = np.stack([synth.field_direct(ls, Sref[i], *synth.pixel_coords(ls, Fx, Fy, 0.2, -0.3))
                    for i in range(len(zp))], axis=1)
    err = rel_l2(E, ref)
    print(precision, k_split, err)
    assert max(err) <= TOL[precision]
    for i in range(len(zp)):  # every plane on its own, exterior and interface planes included
        e = np.linalg.norm(S[i] - Sref[i]) / np.linalg.norm(Sref[i])
        assert e <= TOL[precision], (i, zp[i], e)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_many_planes_in_one_layer(precision, cuda_device):
    """200 planes in one layer: two work units (128 + 72), N = 256 on the tensor path."""
    W, g, a, pi, pr, pt = wl.random_layer_set(11, 3, 3, 1)
    ls = layerset_from_arrays(1.0, 1.9, 1.9, 3, 3, [0.0, 2.0], W, g, a, pi, pr, pt)
    zp = np.linspace(0.0, 2.0, 200)
    _, E, _ = _run(ls, 16, 16, zp, precision)
    ref = synth.synthesize_direct(ls, 16, 16, zp)
    assert max(rel_l2(E, ref)) <= TOL[precision]


def test_host_io_matches_device_path(tiny, cuda_device):
    p, sol, ref = tiny
    plan = _plan(sol, p.Fx, p.Fy, p.z_planes, "split_bf16", host_io=True, exterior=True)
    args = [np.ascontiguousarray(sol.W, dtype=np.complex64), np.ascontiguousarray(sol.gamma),
            np.ascontiguousarray(sol.alpha), sol.p_inc, sol.p_ref, sol.p_trn]
    E = plan.synthesize_host(*args)
    plan.check()
    assert max(rel_l2(E, ref)) <= TOL["split_bf16"]
    E2 = plan.synthesize_host(*args)
    assert np.array_equal(E, E2)


@pytest.mark.parametrize("precision", ["split_bf16", "fp32"])
def test_full_size_sampled_voxels(precision, cuda_device):
    """21x21 orders, 32 layers, 256^3 output (the benchmark's launch configuration):
    sampled voxels against the oracle's per-point direct sum."""
    import torch
    U, L = 21, 32
    W, g, a, pi, pr, pt = wl.random_layer_set(0, U, U, L)
    zb = np.arange(L + 1) * 0.25
    zp = wl.cell_centred_planes(zb[0], zb[-1], 256)
    ls = layerset_from_arrays(1.0, 16.0, 16.0, U, U, zb, W, g, a, pi, pr, pt)
    plan = _plan(ls, 256, 256, zp, precision)
    Wd = torch.from_numpy(W).cuda()
    plan.set_layers(Wd, torch.from_numpy(g).cuda(), torch.from_numpy(a).cuda())
    out = plan.synthesize()
    torch.cuda.synchronize()
    plan.check()
    rng = np.random.default_rng(7)
    idx = np.stack([rng.integers(0, 256, 96), rng.integers(0, 256, 96), rng.integers(0, 256, 96)], axis=1)
    idx[:8, 2] = [0, 7, 8, 127, 128, 248, 254, 255]  # first/last plane, layer edges
    got = out[:, torch.from_numpy(idx[:, 2]), torch.from_numpy(idx[:, 1]), torch.from_numpy(idx[:, 0])]
    got = got.cpu().numpy()
    xs = idx[:, 0] * 16.0 / 256
    ys = idx[:, 1] * 16.0 / 256
    pts = np.stack([xs, ys, zp[idx[:, 2]]], axis=1)
    ref = synth.field_points(ls, pts)
    err = rel_l2(got, ref)
    print(precision, "sampled rel-L2", err)
    assert max(err) <= TOL[precision]
    del Wd
