"""GPU parity: libscw (through the C ABI) against the FP64 oracle.

Tolerances (per-component relative L2, ||E_gpu - E_oracle|| / ||E_oracle||):
  FP32 path 1e-5, split-BF16 and FP16 paths 1e-3 (the targets of the method's
  GPU synthesis). The recompose step alone is FP32 everywhere: 1e-5. The large
  cases also bound the per-component max-abs error by the same tolerance times
  the component's largest magnitude, so a few bad voxels cannot hide in the norm.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, max_abs, rel_l2, to_device
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


def _check(tag, E, ref, tol):
    err = rel_l2(E, ref)
    ab, abn = max_abs(E, ref)
    print(tag, "rel-L2 per component", err, "max-abs", ab, "max-abs / max|E|", abn)
    assert max(err) <= tol, (tag, err)
    assert max(abn) <= tol, (tag, abn)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_thick_layer_hundreds_of_phase_cycles(precision, cuda_device):
    """One heterogeneous layer 200 wavelengths thick (n in [1.25, 1.6]): forward
    modes reach ~290 cycles of phase at its bottom. The phase builder reduces the cycle
    count before its FP32 sine (Eq. 7 / Eq. 30 with the FP64 argument range-
    reduced); an unreduced FP32 argument would lose ~1e-4 there."""
    rng = np.random.default_rng(21)
    N, X, U = 16, 4.0, 5
    n = 1.25 + 0.35 * rng.random((1, N, N)) + 0.0005j * rng.random((1, N, N))
    zb = np.array([0.0, 200.0])
    sol = cw.solve(n, zb, 1.0, X, X, U, U, wl.gaussian_beam_image(N, X, 1.0, 0.4))
    assert sol.gamma[0].real.max() > 1.4
    zp = np.concatenate([np.linspace(0.0, 199.9, 40), [190.37, 199.2, 199.99, 200.0]])
    zp.sort()
    _, E, _ = _run(sol, 32, 32, zp, precision)
    ref = synth.synthesize_direct(sol, 32, 32, zp)
    _check(f"thick {precision}", E, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_strongly_evanescent_orders(precision, cuda_device):
    """A period of 1.2 wavelengths with 11x11 orders: the outer orders have
    |s| up to ~5.9 and modes with Im(gamma) up to ~5.8, decaying by e^-11 across
    a 0.3-wavelength layer. Forward modes are referenced to the layer top and
    backward ones to its bottom, so no factor exceeds 1 (Sec. 2.6.2). (Much
    thicker layers would make the connection-equation solve itself ill-conditioned:
    T_l's backward columns carry e^(-k Im(gamma) d).)"""
    rng = np.random.default_rng(5)
    N, X, U = 24, 1.2, 11
    n = 1.3 + 0.3 * rng.random((2, N, N)) + 0.02j * rng.random((2, N, N))
    zb = np.array([0.0, 0.3, 0.55])
    sol = cw.solve(n, zb, 1.0, X, X, U, U, wl.gaussian_beam_image(N, X, 1.0, 0.5))
    assert np.abs(sol.gamma.imag).max() > 5.0
    zp = np.concatenate([[0.0, 1e-3, 0.02], np.linspace(0.05, 0.52, 28), [0.299, 0.3, 0.549, 0.55]])
    zp.sort()
    _, E, _ = _run(sol, 48, 48, zp, precision)
    ref = synth.synthesize_direct(sol, 48, 48, zp)
    _check(f"evanescent {precision}", E, ref, TOL[precision])


def _whole_volume(ls, W_dev, g_dev, a_dev, zp, tag):
    """Both contraction precisions against the oracle's direct sum of every voxel."""
    import torch
    ref = synth.synthesize_direct(ls, 256, 256, zp)
    for precision in ("split_bf16", "fp32"):
        plan = _plan(ls, 256, 256, zp, precision)
        plan.set_layers(W_dev, g_dev, a_dev)
        out = plan.synthesize()
        torch.cuda.synchronize()
        plan.check()
        E = out.cpu().numpy()
        del out
        plan.close()
        _check(f"{tag} {precision}", E, ref, TOL[precision])
        del E


def test_full_size_whole_volume_random_layers(cuda_device):
    """21x21 orders, 32 layers, 256^3 output (the benchmark's launch configuration)
    on synthetic layer sets with 5 % evanescent modes: every voxel of both
    precisions against the oracle."""
    import torch
    U, L = 21, 32
    W, g, a, pi, pr, pt = wl.random_layer_set(0, U, U, L)
    zb = np.arange(L + 1) * 0.25
    zp = wl.cell_centred_planes(zb[0], zb[-1], 256)
    ls = layerset_from_arrays(1.0, 16.0, 16.0, U, U, zb, W, g, a, pi, pr, pt)
    _whole_volume(ls, torch.from_numpy(W).cuda(), torch.from_numpy(g).cuda(), torch.from_numpy(a).cuda(), zp,
                  "random layers 256^3")


def test_full_size_whole_volume_gpu_solved_sample(cuda_device):
    """The single-wavelength sample itself: 64x64x32 voxels of seeded ellipsoids lit
    by a focused Gaussian beam (NA 0.5), solved on the GPU (scw_solve), then
    synthesised at 256^3 in both precisions. The oracle synthesises the same
    (W, gamma, alpha) in FP64, every voxel."""
    import torch
    import paper_2404_07293_gb300 as scw
    p = wl.config_single_wavelength(0)
    dev = cuda_device
    s = scw.Solver(p.U, p.V, p.L, p.lam, p.X, p.Y, p.z_bounds, p.n_volume.shape[2], p.n_volume.shape[1])
    p_inc = s.incident(torch.from_numpy(p.incident_image.astype(np.complex128)).to(dev))
    W, g, a, pr, pt = s.solve(torch.from_numpy(p.n_volume.astype(np.complex128)).to(dev), p_inc)
    torch.cuda.synchronize()
    s.close()
    ls = cw.LayerSet(lam=p.lam, X=p.X, Y=p.Y, U=p.U, V=p.V, z_bounds=p.z_bounds,
                     W=W.cpu().numpy().astype(np.complex128), gamma=g.cpu().numpy(), alpha=a.cpu().numpy(),
                     p_inc=None, p_ref=None, p_trn=None)
    assert np.abs(ls.alpha).max() > 1e-3  # the beam reaches every layer
    _whole_volume(ls, W, g, a, p.z_planes, "gpu-solved sample 256^3")
