"""GPU parity of the point-set recomposition (x-z / y-z planes, scattered points).

Eq. 10 evaluated at given lateral points on every z plane of a plan, as a
dense product over the orders (split-BF16 tcgen05 GEMM on tensor-core plans,
FP32 SIMT GEMM on FP32 plans), against the FP64 oracle's per-point sum; and
scattered 3-D points, each evaluated on its own plane only.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2
from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-3, "fp16": 1e-3}


def _c(a, dt=np.complex128):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _plan(ls, Fx, Fy, zp, precision, **kw):
    import paper_2404_07293_gb300 as scw
    return scw.Plan(ls.U, ls.V, ls.L, ls.lam, ls.X, ls.Y, ls.z_bounds, Fx, Fy, zp, precision=precision,
                    n_top=ls.n_top, n_bot=ls.n_bot, z_inc=ls.z_inc, **kw)


def _oracle_points(ls, xy, zp):
    """E[3][Fz][P] from the oracle's per-point sum."""
    P = len(xy)
    pts = np.concatenate([np.column_stack([xy, np.full(P, z)]) for z in zp])
    return synth.field_points(ls, pts).reshape(3, len(zp), P)


def _err(E, ref, precision):
    if precision == "fp16":  # FP16 eigenvectors: every component's error scales with the whole field
        n = np.linalg.norm(ref)
        return [float(np.linalg.norm(E[c] - ref[c]) / n) for c in range(3)]
    return rel_l2(E, ref)


@pytest.fixture(scope="module")
def sphere():
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    zp = np.concatenate([[-0.5], p.z_planes[::3], [p.z_bounds[-1] + 0.3]])
    return p, sol, zp


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "fp16"])
def test_xz_yz_planes_and_scattered_points(sphere, precision, cuda_device):
    p, sol, zp = sphere
    rng = np.random.default_rng(7)
    plan = _plan(sol, p.Fx, p.Fy, zp, precision, exterior=True)
    plan.set_layers(_c(sol.W, np.complex64), _c(sol.gamma), _c(sol.alpha), _c(sol.p_inc), _c(sol.p_ref),
                    _c(sol.p_trn))
    cases = {
        "xz": np.column_stack([np.linspace(0, sol.X, 96, endpoint=False), np.full(96, 1.3)]),
        "yz": np.column_stack([np.full(40, 2.9), np.linspace(-1.0, 3.0, 40)]),
        # ragged count, points outside one period and at negative coordinates
        "scattered": rng.uniform(-2.0 * sol.X, 3.0 * sol.X, size=(1001, 2)),
        "one": np.array([[0.7, -0.4]]),
    }
    for name, xy in cases.items():
        plan.set_points(xy)
        E = plan.synthesize_points().cpu().numpy()
        plan.check()
        assert E.shape == (3, len(zp), len(xy))
        ref = _oracle_points(sol, xy, zp)
        err = _err(E, ref, precision)
        print(precision, name, err)
        assert max(err) <= TOL[precision], name
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_grid_points_equal_the_volume(sphere, precision, cuda_device):
    """Points on the pixel grid reproduce the FFT path's volume (same spectra)."""
    p, sol, zp = sphere
    plan = _plan(sol, 32, 16, zp, precision, exterior=True, x0=0.25, y0=-0.5)
    plan.set_layers(_c(sol.W, np.complex64), _c(sol.gamma), _c(sol.alpha), _c(sol.p_inc), _c(sol.p_ref),
                    _c(sol.p_trn))
    vol = plan.synthesize().cpu().numpy()                      # [3][Fz][16][32]
    xs, ys = synth.pixel_coords(sol, 32, 16, 0.25, -0.5)
    gx, gy = np.meshgrid(xs, ys)
    plan.set_points(np.column_stack([gx.ravel(), gy.ravel()]))
    E = plan.synthesize_points().cpu().numpy().reshape(3, len(zp), 16, 32)
    plan.check()
    tol = 1e-5 if precision == "fp32" else 1e-4
    assert max(rel_l2(E, vol)) <= tol
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_points_many_planes_and_illuminations(precision, cuda_device):
    """3 illuminations x 130 planes: 2340 product columns (several column tiles,
    a partial last one) and 300 points (a partial last row tile); each
    illumination equals a one-illumination plan, and one is checked against the oracle."""
    U, V, L, I = 7, 9, 2, 3
    W, g, _, *_ = wl.random_layer_set(21, U, V, L)
    amps = [wl.random_layer_set(300 + i, U, V, L)[2:] for i in range(I)]
    zb = np.array([0.0, 0.7, 1.5])
    zp = np.linspace(-0.2, 1.8, 130)
    ls = layerset_from_arrays(1.0, 2.2, 3.4, U, V, zb, W, g, *amps[0], n_bot=1.2 + 0.01j, z_inc=-0.1)
    xy = np.random.default_rng(3).uniform(-1.0, 4.0, size=(300, 2))
    multi = _plan(ls, 16, 16, zp, precision, exterior=True, illuminations=I)
    multi.set_layers(_c(W, np.complex64), _c(g), *[_c(np.stack([a[j] for a in amps])) for j in range(4)])
    multi.set_points(xy)
    E = multi.synthesize_points().cpu().numpy()
    multi.check()
    assert E.shape == (I, 3, len(zp), len(xy))
    single = _plan(ls, 16, 16, zp, precision, exterior=True)
    single.set_points(xy)
    for i in range(I):
        single.set_layers(_c(W, np.complex64), _c(g), *[_c(x) for x in amps[i]])
        Ei = single.synthesize_points().cpu().numpy()
        single.check()
        assert np.linalg.norm(E[i] - Ei) / np.linalg.norm(Ei) <= 1e-6
    ls1 = layerset_from_arrays(1.0, 2.2, 3.4, U, V, zb, W, g, *amps[1], n_bot=1.2 + 0.01j, z_inc=-0.1)
    assert max(rel_l2(E[1], _oracle_points(ls1, xy, zp))) <= TOL[precision]
    multi.close()
    single.close()


def test_point_errors(sphere, cuda_device):
    import paper_2404_07293_gb300 as scw
    p, sol, zp = sphere
    plan = _plan(sol, 16, 16, zp, "split_bf16", exterior=True)
    with pytest.raises(scw.ScwError):
        plan.set_points(np.array([[0.0, np.nan]]))
    plan.set_layers(_c(sol.W, np.complex64), _c(sol.gamma), _c(sol.alpha), _c(sol.p_inc), _c(sol.p_ref),
                    _c(sol.p_trn))
    plan.n_points = 4
    with pytest.raises(scw.ScwError) as e:
        plan.synthesize_points()   # no point set yet
    assert e.value.status == 7
    plan.set_points(np.zeros((4, 2)))
    plan.set_points(np.zeros((0, 2)))  # released
    with pytest.raises(scw.ScwError):
        plan.synthesize_points()
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_scattered_3d_points(sphere, precision, cuda_device):
    """Each point on its own plane: (x_p, y_p, z_planes[plane_p]) against the oracle, and against
    the same points evaluated on every plane by the GEMM path."""
    p, sol, zp = sphere
    rng = np.random.default_rng(11)
    P = 777
    xy = rng.uniform(-sol.X, 2 * sol.X, size=(P, 2))
    plane = rng.integers(0, len(zp), size=P)
    plan = _plan(sol, p.Fx, p.Fy, zp, precision, exterior=True)
    plan.set_layers(_c(sol.W, np.complex64), _c(sol.gamma), _c(sol.alpha), _c(sol.p_inc), _c(sol.p_ref),
                    _c(sol.p_trn))
    plan.set_points(xy)
    full = plan.synthesize_points().cpu().numpy()          # [3][Fz][P]
    plan.set_points(xy, plane=plane)
    E = plan.synthesize_points().cpu().numpy()             # [3][P]
    plan.check()
    assert E.shape == (3, P)
    ref = synth.field_points(sol, np.column_stack([xy, zp[plane]]))
    err = _err(E, ref, precision)
    print(precision, "scattered", err)
    assert max(err) <= TOL[precision]
    picked = full[:, plane, np.arange(P)]
    assert np.linalg.norm(E - picked) / np.linalg.norm(picked) <= (1e-6 if precision == "fp32" else 1e-4)
    with pytest.raises(Exception):
        plan.set_points(xy, plane=np.full(P, len(zp)))      # index out of range
    plan.close()
