"""GPU parity of periodic tiling and patch composition.

Periodic tiling: the field of a periodic sample repeats with the lateral
period (Eq. 10 is a sum of plane waves with u/X, v/Y orders), so a plan with
tiles (tx, ty) computes one unit cell and stores it to every tile. The oracle
evaluates the direct sum at every pixel of the tiled grid (no copying).

Patch composition: a large sample split into lateral patches, each solved as
its own periodic cell, with every patch's field written into its place in one
mosaic (Sec. 1). Each batched item gets a strided view of the mosaic
(out_ld, out_plane_stride); the result equals each patch's own field.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2
from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-3}


def _c(a, dt=np.complex128):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


@pytest.fixture(scope="module")
def sphere():
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    zp = np.concatenate([[-0.3], p.z_planes[::4], [p.z_bounds[-1] + 0.5]])
    return p, sol, zp


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_periodic_tiling_against_the_direct_sum(sphere, precision, cuda_device):
    import paper_2404_07293_gb300 as scw
    p, sol, zp = sphere
    Fx, Fy, tx, ty, x0, y0 = 32, 16, 3, 2, 0.4, -1.2
    plan = scw.Plan(sol.U, sol.V, sol.L, sol.lam, sol.X, sol.Y, sol.z_bounds, Fx, Fy, zp, x0=x0, y0=y0,
                    precision=precision, exterior=True, tiles=(tx, ty), n_bot=sol.n_bot)
    plan.set_layers(_c(sol.W, np.complex64), _c(sol.gamma), _c(sol.alpha), _c(sol.p_inc), _c(sol.p_ref),
                    _c(sol.p_trn))
    E = plan.synthesize().cpu().numpy()
    plan.check()
    assert E.shape == (3, len(zp), ty * Fy, tx * Fx)
    xs = x0 + np.arange(tx * Fx) * (sol.X / Fx)
    ys = y0 + np.arange(ty * Fy) * (sol.Y / Fy)
    ref = np.stack([synth.field_direct(sol, synth.spectrum_at(sol, float(z)), xs, ys) for z in zp], axis=1)
    assert max(rel_l2(E, ref)) <= TOL[precision]
    cell = E[:, :, :Fy, :Fx]
    for b in range(ty):
        for a in range(tx):
            assert np.array_equal(E[:, :, b * Fy:(b + 1) * Fy, a * Fx:(a + 1) * Fx], cell)
    # the fused recompose entry point stores the same tiles
    again = plan.recompose(plan.spectrum()).cpu().numpy()
    assert np.array_equal(again, E)
    plan.close()


def test_tiled_host_io_matches_device(sphere, cuda_device):
    import paper_2404_07293_gb300 as scw
    p, sol, zp = sphere
    kw = dict(precision="split_bf16", exterior=True, tiles=(2, 3), n_bot=sol.n_bot)
    args = [np.ascontiguousarray(sol.W, dtype=np.complex64), np.ascontiguousarray(sol.gamma),
            np.ascontiguousarray(sol.alpha), sol.p_inc, sol.p_ref, sol.p_trn]
    host = scw.Plan(sol.U, sol.V, sol.L, sol.lam, sol.X, sol.Y, sol.z_bounds, 16, 24, zp, host_io=True, **kw)
    E = host.synthesize_host(*args)
    host.check()
    dev = scw.Plan(sol.U, sol.V, sol.L, sol.lam, sol.X, sol.Y, sol.z_bounds, 16, 24, zp, **kw)
    dev.set_layers(*[_c(x, np.complex64 if j == 0 else np.complex128) for j, x in enumerate(args)])
    assert np.array_equal(E, dev.synthesize().cpu().numpy())
    host.close()
    dev.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_patch_mosaic_from_a_batched_plan(precision, cuda_device):
    """3 x 2 patches of different samples (and order counts) written into one
    mosaic with a border column of padding that nothing may touch."""
    import torch
    import paper_2404_07293_gb300 as scw
    Fx, Fy, nx, ny = 24, 16, 3, 2
    H, W = ny * Fy, nx * Fx + 8                      # 8 padding columns on the right
    zb = np.array([0.0, 0.4, 0.9])
    zp = np.array([-0.2, 0.1, 0.5, 0.85, 1.3])
    items, layers = [], []
    for k in range(nx * ny):
        U = 5 + 2 * (k % 3)
        items.append(dict(U=U, V=U, L=2, lam=1.0, X=2.0, Y=1.5, z_bounds=zb, Fx=Fx, Fy=Fy, z_planes=zp,
                          exterior=True, out_ld=W, out_plane_stride=H * W, n_bot=1.1))
        layers.append(wl.random_layer_set(40 + k, U, U, 2))
    bp = scw.BatchedPlan(items, precision=precision)
    for k, (Wm, g, a, pi, pr, pt) in enumerate(layers):
        bp.set_layers(k, _c(Wm, np.complex64), _c(g), _c(a), _c(pi), _c(pr), _c(pt))
    mosaic = torch.full((3, len(zp), H, W), float("nan"), dtype=torch.complex64, device="cuda")
    views = [mosaic[:, :, (k // nx) * Fy:(k // nx + 1) * Fy, (k % nx) * Fx:(k % nx + 1) * Fx] for k in range(nx * ny)]
    bp.synthesize(views)
    bp.check()
    got = mosaic.cpu().numpy()
    assert np.isnan(got[:, :, :, nx * Fx:].real).all()  # padding untouched
    for k, (Wm, g, a, pi, pr, pt) in enumerate(layers):
        kw = items[k]
        ls = layerset_from_arrays(1.0, 2.0, 1.5, kw["U"], kw["V"], zb, Wm, g, a, pi, pr, pt, n_bot=1.1)
        ref = synth.synthesize_direct(ls, Fx, Fy, zp)
        blk = got[:, :, (k // nx) * Fy:(k // nx + 1) * Fy, (k % nx) * Fx:(k % nx + 1) * Fx]
        assert max(rel_l2(blk, ref)) <= TOL[precision], k
    bp.close()


def test_patch_view_with_wrong_strides_is_rejected(cuda_device):
    import torch
    import paper_2404_07293_gb300 as scw
    zb = np.array([0.0, 1.0])
    plan = scw.Plan(3, 3, 1, 1.0, 1.0, 1.0, zb, 16, 16, [0.5], out_ld=40, out_plane_stride=40 * 16)
    with pytest.raises(ValueError):
        plan.synthesize(torch.empty((3, 1, 16, 16), dtype=torch.complex64, device="cuda"))
    plan.close()
