"""GPU parity of multi-illumination plans and of the objective pupil.

One coupled-wave solve serves every incident field that is expanded in the
same orders: the layer eigenvectors W and eigenvalues gamma depend on the
sample and the wavelength only, and each illumination brings its own mode
amplitudes alpha and exterior amplitudes p (Sec. 2.3-2.5). A plan with I
illuminations contracts all I of them against one read of W.

Below the sample an imaging system only collects the plane waves inside its
numerical aperture; a plan with pupil_na > 0 drops the other orders there
(Sec. 1, Sec. 4.1: imaging needs only the external field).
"""
import numpy as np
import pytest

import workloads as wl
from helpers import layerset_from_arrays, rel_l2
from oracle import cw, synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-3, "fp16": 1e-3}


def _err(E, ref, precision):
    """Per-component rel-L2. With FP16 eigenvectors (11 significant bits) the
    absolute error of every component scales with the whole field, so a weak
    cross-polarised component is measured against the norm of all three."""
    if precision == "fp16":
        n = np.linalg.norm(ref)
        return [float(np.linalg.norm(E[c] - ref[c]) / n) for c in range(3)]
    return rel_l2(E, ref)


def _c(a, dt=np.complex128):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _plan(ls, Fx, Fy, zp, precision, **kw):
    import paper_2404_07293_gb300 as scw
    return scw.Plan(ls.U, ls.V, ls.L, ls.lam, ls.X, ls.Y, ls.z_bounds, Fx, Fy, zp, precision=precision,
                    n_top=ls.n_top, n_bot=ls.n_bot, z_inc=ls.z_inc, **kw)


@pytest.fixture(scope="module")
def two_beams():
    """One sphere sample lit by an x-polarised plane wave and by a tilted,
    y-polarised Gaussian beam: one set of modes, two sets of amplitudes."""
    p = wl.config_tiny()
    a = cw.solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, p.incident_image, pol="x")
    img = wl.gaussian_beam_image(16, p.X, 1.0, 0.4) * np.exp(2j * np.pi * np.arange(16)[None, :] / 16)
    b = cw.solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, img, pol="y")
    assert np.array_equal(a.W, b.W) and np.array_equal(a.gamma, b.gamma)
    zp = np.concatenate([[-0.6, -0.1], p.z_planes[::2], [p.z_bounds[-1] + 0.2, p.z_bounds[-1] + 0.9]])
    return p, (a, b), zp


@pytest.mark.parametrize("precision", ["fp32", "split_bf16", "fp16"])
def test_two_illuminations_against_the_oracle(two_beams, precision, cuda_device):
    p, sols, zp = two_beams
    a = sols[0]
    plan = _plan(a, p.Fx, p.Fy, zp, precision, exterior=True, illuminations=2)
    stack = lambda name: np.stack([getattr(s, name) for s in sols])
    plan.set_layers(_c(a.W, np.complex64), _c(a.gamma), _c(stack("alpha")), _c(stack("p_inc")),
                    _c(stack("p_ref")), _c(stack("p_trn")))
    E = plan.synthesize().cpu().numpy()
    plan.check()
    assert E.shape == (2, 3, len(zp), p.Fy, p.Fx)
    for i, s in enumerate(sols):
        ref = synth.synthesize_direct(s, p.Fx, p.Fy, zp)
        err = _err(E[i], ref, precision)
        print(precision, i, err, rel_l2(E[i], ref))
        assert max(err) <= TOL[precision]
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
@pytest.mark.parametrize("I", [3, 16])
def test_illumination_slots_equal_single_plans(precision, I, cuda_device):
    """Illumination i of an I-illumination plan equals a one-illumination plan fed
    alpha_i and p_i (random amplitudes, interfaces, exterior planes, ragged sizes)."""
    U, V, L = 9, 7, 3
    W, g, _, *_ = wl.random_layer_set(5, U, V, L)
    amps = [wl.random_layer_set(100 + i, U, V, L)[2:] for i in range(I)]
    zb = np.array([0.0, 0.3, 0.31, 0.9])
    zp = np.array([-0.4, 0.0, 0.05, 0.3, 0.31, 0.5, 0.9, 0.95, 1.6])
    ls = layerset_from_arrays(1.0, 2.7, 3.1, U, V, zb, W, g, *amps[0], n_bot=1.3 + 0.02j, z_inc=-0.05)
    Fx, Fy = 24, 40
    multi = _plan(ls, Fx, Fy, zp, precision, exterior=True, illuminations=I, x0=0.1)
    multi.set_layers(_c(W, np.complex64), _c(g), *[_c(np.stack([a[j] for a in amps])) for j in range(4)])
    E = multi.synthesize().cpu().numpy()
    multi.check()
    single = _plan(ls, Fx, Fy, zp, precision, exterior=True, x0=0.1)
    for i in range(I):
        single.set_layers(_c(W, np.complex64), _c(g), *[_c(x) for x in amps[i]])
        Ei = single.synthesize().cpu().numpy()
        single.check()
        d = np.linalg.norm(E[i] - Ei) / np.linalg.norm(Ei)
        assert d <= 1e-6, (i, d)
    # and one illumination against the oracle
    ls_last = layerset_from_arrays(1.0, 2.7, 3.1, U, V, zb, W, g, *amps[-1], n_bot=1.3 + 0.02j, z_inc=-0.05)
    ref = synth.synthesize_direct(ls_last, Fx, Fy, zp, x0=0.1)
    assert max(rel_l2(E[-1], ref)) <= TOL[precision]
    multi.close()
    single.close()


def test_multi_illumination_host_io(two_beams, cuda_device):
    p, sols, zp = two_beams
    a = sols[0]
    stack = lambda name: np.stack([getattr(s, name) for s in sols])
    args = [np.ascontiguousarray(a.W, dtype=np.complex64), np.ascontiguousarray(a.gamma),
            stack("alpha"), stack("p_inc"), stack("p_ref"), stack("p_trn")]
    host = _plan(a, p.Fx, p.Fy, zp, "split_bf16", exterior=True, illuminations=2, host_io=True)
    E = host.synthesize_host(*args)
    host.check()
    dev = _plan(a, p.Fx, p.Fy, zp, "split_bf16", exterior=True, illuminations=2)
    dev.set_layers(*[_c(x, np.complex64 if j == 0 else np.complex128) for j, x in enumerate(args)])
    assert np.array_equal(E, dev.synthesize().cpu().numpy())
    host.close()
    dev.close()


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
@pytest.mark.parametrize("na", [0.3, 0.55, 0.9])
def test_pupil_below_the_sample(two_beams, precision, na, cuda_device):
    p, sols, zp = two_beams
    s = sols[1]
    plan = _plan(s, p.Fx, p.Fy, zp, precision, exterior=True, pupil_na=na)
    plan.set_layers(_c(s.W, np.complex64), _c(s.gamma), _c(s.alpha), _c(s.p_inc), _c(s.p_ref), _c(s.p_trn))
    E = plan.synthesize().cpu().numpy()
    S = plan.spectrum().cpu().numpy()
    plan.check()
    ref = synth.synthesize_direct(s, p.Fx, p.Fy, zp, pupil_na=na)
    assert max(rel_l2(E, ref)) <= TOL[precision]
    Sref = synth.spectra(s, zp, pupil_na=na)
    below = zp > s.z_bounds[-1]
    outside = synth.pupil_mask(s, na) == 0
    assert np.all(S[np.ix_(below, np.arange(3), outside)] == 0)  # blocked orders are exactly zero
    assert np.linalg.norm(S - Sref) / np.linalg.norm(Sref) <= TOL[precision]
    plan.close()


def test_host_io_pipeline_with_split_layers(cuda_device):
    """Host-IO synthesis runs in layer groups (copies overlapping the kernels); a layer
    with more plane slots than one work unit (3 illuminations x 50 planes) must stay in
    one group. The result equals the device path bit for bit."""
    U, V, L, I = 5, 5, 4, 3
    W, g, _, *_ = wl.random_layer_set(8, U, V, L)
    amps = [wl.random_layer_set(60 + i, U, V, L)[2:] for i in range(I)]
    zb = np.array([0.0, 0.2, 1.2, 1.3, 1.5])
    zp = np.concatenate([[-0.3], np.linspace(0.01, 0.19, 5), np.linspace(0.2, 1.19, 50), [1.25, 1.4], [1.9]])
    ls = layerset_from_arrays(1.0, 2.0, 2.0, U, V, zb, W, g, *amps[0])
    args = [np.ascontiguousarray(W, dtype=np.complex64), np.ascontiguousarray(g)] + \
        [np.ascontiguousarray(np.stack([a[j] for a in amps])) for j in range(4)]
    host = _plan(ls, 16, 16, zp, "split_bf16", exterior=True, illuminations=I, host_io=True)
    E = host.synthesize_host(*args)
    E2 = host.synthesize_host(*args)
    host.check()
    dev = _plan(ls, 16, 16, zp, "split_bf16", exterior=True, illuminations=I)
    dev.set_layers(*[_c(x, np.complex64 if j == 0 else np.complex128) for j, x in enumerate(args)])
    Ed = dev.synthesize().cpu().numpy()
    assert np.array_equal(E, Ed)
    assert np.array_equal(E, E2)
    host.close()
    dev.close()
