"""GPU parity of the coupled-wave solve stage (scw_solver_*) against the FP64 oracle.

The eigenvector basis is not unique (scale, order, and any basis of a repeated
eigenvalue's eigenspace), so W and alpha are compared through what they
determine: the synthesised field and spectra. p_ref, p_trn and the eigenvalues
(as sets) are unique and compared directly. Both sides run in FP64; they use
different eigen-algorithms (the GPU solves the half-size problem A B, the
oracle the full D), so agreement is to FP64 rounding times the conditioning
of the connection equations.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2
from oracle import cw, synth

pytestmark = pytest.mark.gpu


def _c(a, dt=np.complex128):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _gpu_solve(n_vol, zb, lam, X, Y, U, V, img, pol="x", n_top=1.0, n_bot=1.0, z_inc=None):
    import paper_2404_07293_gb300 as scw
    L, Ny, Nx = n_vol.shape
    s = scw.Solver(U, V, L, lam, X, Y, zb, Nx, Ny, n_top=n_top, n_bot=n_bot, z_inc=z_inc)
    p_inc = s.incident(_c(img), pol)
    out = s.solve(_c(n_vol), p_inc)
    times = s.times()
    s.close()
    return p_inc, out, times


def _same_set(a, b, tol):
    """Every eigenvalue of a has one of b within tol, and the other way round."""
    d = np.abs(np.asarray(a)[:, None] - np.asarray(b)[None, :])
    return max(d.min(axis=1).max(), d.min(axis=0).max()) <= tol


def _compare(sol, p_inc, out, Fx, Fy, zp, tol_p=1e-8):
    import paper_2404_07293_gb300 as scw
    W, g, a, pr, pt = out
    assert np.abs(p_inc.cpu().numpy() - sol.p_inc).max() <= 1e-12 * max(1.0, np.abs(sol.p_inc).max())
    scale = max(np.abs(sol.p_ref).max(), np.abs(sol.p_trn).max())
    assert np.abs(pr.cpu().numpy() - sol.p_ref).max() <= tol_p * scale
    assert np.abs(pt.cpu().numpy() - sol.p_trn).max() <= tol_p * scale
    gg = g.cpu().numpy()
    for l in range(sol.L):
        assert _same_set(gg[l], sol.gamma[l], 1e-9 * np.abs(sol.gamma[l]).max())
    # the field from the GPU's (W, gamma, alpha) against the oracle's own solve, both ways of synthesis
    plan = scw.Plan(sol.U, sol.V, sol.L, sol.lam, sol.X, sol.Y, sol.z_bounds, Fx, Fy, zp, precision="fp32",
                    exterior=True, n_top=sol.n_top, n_bot=sol.n_bot, z_inc=sol.z_inc)
    plan.set_layers(W, g, a, p_inc, pr, pt)
    E = plan.synthesize().cpu().numpy()
    plan.check()
    plan.close()
    ref = synth.synthesize_direct(sol, Fx, Fy, zp)
    err = rel_l2(E, ref)
    # FP64 (W, gamma, alpha) of the GPU solve through the oracle's FP64 synthesis: no FP32 step at all
    gpu_ls = layerset_from_arrays(sol.lam, sol.X, sol.Y, sol.U, sol.V, sol.z_bounds, W.cpu().numpy(), gg,
                                  a.cpu().numpy(), p_inc.cpu().numpy(), pr.cpu().numpy(), pt.cpu().numpy(),
                                  n_top=sol.n_top, n_bot=sol.n_bot, z_inc=sol.z_inc)
    S_gpu = synth.spectra(gpu_ls, zp)
    S_ref = synth.spectra(sol, zp)
    return err, float(np.linalg.norm(S_gpu - S_ref) / np.linalg.norm(S_ref))


def test_sphere_tiny_config(cuda_device):
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    p_inc, out, t = _gpu_solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, p.incident_image)
    zp = np.concatenate([[-0.4], p.z_planes[::2], [p.z_bounds[-1] + 0.6]])
    err, serr = _compare(sol, p_inc, out, p.Fx, p.Fy, zp)
    print("field rel-L2", err, "spectrum (W in complex64)", serr, t)
    assert max(err) <= 1e-5
    assert serr <= 1e-6  # W is delivered in complex64 (the synthesis input type)


@pytest.mark.parametrize("pol", ["x", "y"])
def test_heterogeneous_oblique_substrate(pol, cuda_device):
    """Ellipsoids in 3 layers, U != V, X != Y, a tilted Gaussian beam, an absorbing
    substrate and an incident plane above the sample."""
    U, V, L = 5, 7, 3
    vol = wl.ellipsoid_volume(11, 16, 20, L, semi_axes=(2, 6), kappa=(0.0, 0.05))
    zb = np.array([0.0, 0.2, 0.45, 0.6])
    X, Y = 3.0, 3.5
    img = wl.gaussian_beam_image(16, X, 1.0, 0.4)
    img = np.repeat(img, 2, axis=0)[:20] * np.exp(2j * np.pi * np.arange(16)[None, :] / 16)
    kw = dict(pol=pol, n_top=1.0, n_bot=1.4 + 0.02j, z_inc=-0.15)
    sol = cw.solve(vol, zb, 1.0, X, Y, U, V, img, **kw)
    p_inc, out, _ = _gpu_solve(vol, zb, 1.0, X, Y, U, V, img, **kw)
    zp = np.array([-0.5, -0.01, 0.1, 0.2, 0.3, 0.5, 0.6, 0.9])
    err, serr = _compare(sol, p_inc, out, 24, 32, zp)
    print(pol, err, serr)
    assert max(err) <= 1e-5
    assert serr <= 1e-6


def test_homogeneous_slab_repeated_eigenvalues(cuda_device):
    """A laterally uniform slab: every s_z appears twice (TE and TM), so each
    eigenspace is two-dimensional; the GPU's basis differs from the oracle's and
    the field must still agree (and match the Airy closed form the oracle is pinned to)."""
    U = V = 5
    vol = np.full((2, 12, 12), 1.5 + 0.01j)
    zb = np.array([0.0, 0.3, 0.7])
    img = wl.plane_wave_image(12)
    sol = cw.solve(vol, zb, 1.0, 2.0, 2.0, U, V, img)
    p_inc, out, _ = _gpu_solve(vol, zb, 1.0, 2.0, 2.0, U, V, img)
    zp = np.array([-0.2, 0.15, 0.5, 0.69, 1.1])
    err, serr = _compare(sol, p_inc, out, 16, 16, zp)
    # normal incidence, x-polarised: E_y and E_z vanish, so their per-component ratios are noise over
    # noise; the error is measured against the whole field
    assert err[0] <= 1e-5
    assert serr <= 1e-6


def test_gpu_solve_then_split_bf16_synthesis_end_to_end(cuda_device):
    """The whole method on the GPU: sample -> solve -> split-BF16 synthesis, against
    the oracle's solve + direct sum."""
    import paper_2404_07293_gb300 as scw
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    p_inc, (W, g, a, pr, pt), _ = _gpu_solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, p.incident_image)
    plan = scw.Plan(p.U, p.V, len(p.z_bounds) - 1, p.lam, p.X, p.Y, p.z_bounds, p.Fx, p.Fy, p.z_planes,
                    precision="split_bf16")
    plan.set_layers(W, g, a)
    E = plan.synthesize().cpu().numpy()
    plan.check()
    ref = synth.synthesize_direct(sol, p.Fx, p.Fy, p.z_planes)
    assert max(rel_l2(E, ref)) <= 1e-3
    plan.close()


def test_grazing_incidence_is_reported(cuda_device):
    import paper_2404_07293_gb300 as scw
    # X = 2 lambda: the order u = 2 has s_x = 1 = n_top, s_z = 0; an image with that order
    s = scw.Solver(5, 1, 1, 1.0, 2.0, 2.0, [0.0, 0.3], 12, 4)
    img = np.exp(2j * np.pi * 2 * np.arange(12)[None, :] / 12) * np.ones((4, 1))
    with pytest.raises(scw.ScwError) as e:
        s.incident(_c(img), "y")  # y-polarised: s_x p_x + s_y p_y = 0 -> no error
        s.incident(_c(img), "x")  # x-polarised: p_x nonzero at s_z = 0
    assert e.value.status == 6
    s.close()


def test_medium_sample_eleven_orders(cuda_device):
    """A larger case (11 x 11 orders, 4M = 484 modes per layer, 5 layers of
    ellipsoids on a 32 x 32 grid, focused beam): several eigen-workers and
    longer connection products."""
    U, L = 11, 5
    vol = wl.ellipsoid_volume(21, 32, 32, L)
    zb = np.arange(L + 1) * 0.25
    img = wl.gaussian_beam_image(32, 8.0, 1.0, 0.5)
    sol = cw.solve(vol, zb, 1.0, 8.0, 8.0, U, U, img)
    p_inc, out, t = _gpu_solve(vol, zb, 1.0, 8.0, 8.0, U, U, img)
    zp = np.array([-0.3, 0.1, 0.6, 1.1, 1.5])
    err, serr = _compare(sol, p_inc, out, 64, 64, zp, tol_p=1e-7)
    print("medium", err, serr, t)
    assert max(err) <= 1e-5
    assert serr <= 1e-6
