"""Pins of the FP64 surrogate oracle (oracle/fno.py) against things other than itself.

- the kept-mode DFT against a brute-force double loop over pixels and modes;
- the spectral convolution with identity mixing against a brute-force low-pass sum;
- translation equivariance of the whole network (periodic shifts of the input
  shift the field and leave the error head unchanged) -- a wrong sign or a
  swapped axis in either DFT breaks it;
- GELU at a textbook value, its odd part GELU(z) - GELU(-z) = z, and its
  derivative by finite differences;
- every parameter group's gradient against central finite differences of the
  loss (the hand-derived backward);
- the first Adam step, which moves each parameter by lr g/(|g| + eps);
- the conformal offset on a set whose residual quantile is known.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import fno_init_groups
from oracle import fno

TINY = fno.FnoShape(width=4, grid=8, modes=4, layers=2, slices=2, in_grid=4)


def _setup(sh, seed=0, B=2):
    flat = wl.random_flat(seed, fno_init_groups(sh))
    n = wl.phantom_batch(100 + seed, B, nx=sh.in_grid, ny=sh.in_grid, nz=sh.slices, semi_axes=(1.0, 3.0))
    rng = np.random.default_rng(seed + 7)
    T = rng.standard_normal((B, fno.OUT_CH, sh.grid, sh.grid))
    return flat, n, T


def test_truncated_dft_brute_force():
    sh = TINY
    rng = np.random.default_rng(1)
    v = rng.standard_normal((3, sh.grid, sh.grid))
    got = fno.truncated_dft(v, sh)
    ky, kx = fno.kept_frequencies(sh)
    ref = np.zeros((3, sh.n_modes), dtype=complex)
    for k in range(sh.n_modes):
        for y in range(sh.grid):
            for x in range(sh.grid):
                ref[:, k] += v[:, y, x] * np.exp(-2j * np.pi * (kx[k] * x + ky[k] * y) / sh.grid)
    assert np.abs(got - ref).max() < 1e-12
    # mode index convention: (ky + m/2) m + (kx + m/2)
    assert ky[0] == -sh.modes // 2 and kx[1] == -sh.modes // 2 + 1 and ky[sh.modes] == -sh.modes // 2 + 1


def test_identity_mixing_is_brute_force_lowpass():
    sh = TINY
    rng = np.random.default_rng(2)
    v = rng.standard_normal((2, sh.width, sh.grid, sh.grid))
    R = np.broadcast_to(np.eye(sh.width), (sh.n_modes, sh.width, sh.width)).astype(complex)
    U, _ = fno.spectral_conv(v, R, sh)
    ky, kx = fno.kept_frequencies(sh)
    N = sh.grid
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ref = np.zeros_like(v)
    for k in range(sh.n_modes):
        ph = np.exp(-2j * np.pi * (kx[k] * xx + ky[k] * yy) / N)
        coef = (v * ph).sum(axis=(2, 3))
        ref += (coef[:, :, None, None] * np.conj(ph)).real / N ** 2
    assert np.abs(U - ref).max() < 1e-12


def test_translation_equivariance():
    sh = TINY
    flat, n, _ = _setup(sh, seed=3)
    F, h, _ = fno.forward(flat, n, sh)
    r = sh.grid // sh.in_grid
    dy, dx = 1, 3
    Fs, hs, _ = fno.forward(flat, np.roll(n, (dy, dx), axis=(2, 3)), sh)
    assert np.abs(Fs - np.roll(F, (dy * r, dx * r), axis=(2, 3))).max() < 1e-11
    assert np.abs(hs - h).max() < 1e-11


def test_gelu_values_and_derivative():
    assert fno.gelu(1.0) == pytest.approx(0.8413447460685429, abs=1e-15)  # Phi(1)
    z = np.linspace(-6, 6, 101)
    assert np.abs(fno.gelu(z) - fno.gelu(-z) - z).max() < 1e-14
    eps = 1e-6
    fd = (fno.gelu(z + eps) - fno.gelu(z - eps)) / (2 * eps)
    assert np.abs(fd - fno.gelu_grad(z)).max() < 1e-8


@pytest.mark.parametrize("group", ["P", "p", "R0", "W0", "c0", "R1", "W1", "c1", "Q", "q", "e", "e0"])
def test_gradient_finite_differences(group):
    sh = TINY
    flat, n, T = _setup(sh, seed=4)
    L, _, _, g = fno.loss_and_grads(flat, n, T, sh)
    assert L == pytest.approx(fno.loss(flat, n, T, sh)[0], rel=1e-14)
    off = 0
    for name, s, cplx in fno.param_layout(sh):
        size = int(np.prod(s)) * (2 if cplx else 1)
        if name == group:
            break
        off += size
    rng = np.random.default_rng(5)
    idx = off + rng.choice(size, size=min(size, 12), replace=False)
    # the trunk is trained by L_field alone (the head sees it as constant); the
    # head parameters do not enter L_field, so their derivative is that of L
    part = 0 if group in ("e", "e0") else 1
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        fd = (fno.loss(fp, n, T, sh)[part] - fno.loss(fm, n, T, sh)[part]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (group, i, fd, g[i])


def test_head_does_not_train_trunk():
    """Changing only the head leaves every trunk gradient bit-identical."""
    sh = TINY
    flat, n, T = _setup(sh, seed=6)
    _, _, _, g = fno.loss_and_grads(flat, n, T, sh)
    P = fno.unpack(flat, sh)
    P["e"] = np.zeros_like(P["e"])  # change only the head: trunk gradients unchanged
    P["e0"] = np.array([3.0])
    _, _, _, g2 = fno.loss_and_grads(fno.pack(P, sh), n, T, sh)
    nh = sh.width + 1
    assert np.array_equal(g[:-nh], g2[:-nh])


def test_first_adam_step():
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(50)
    grad = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    new, m, v = fno.adam_step(theta, grad, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    assert np.abs(new - (theta - lr * grad / (np.abs(grad) + eps))).max() < 1e-15
    assert np.abs(m - 0.1 * grad).max() < 1e-15 and np.abs(v - 0.001 * grad ** 2).max() < 1e-15


def test_conformal_offset_quantile():
    h = np.zeros(99)
    true_rel = np.exp(np.arange(99) / 10.0)        # residuals 0.0, 0.1, ..., 9.8
    q = fno.conformal_offset(h, true_rel, miss=0.1)
    assert q == pytest.approx(8.9)                  # ceil(0.9 * 100) = 90th smallest
    assert np.mean(np.log(true_rel) <= q) >= 0.9


def test_kernel_gelu_erf_approximation_error_bound():
    """The surrogate kernels evaluate the normal CDF through Abramowitz & Stegun's formula 7.1.26
    for erf (stated |error| <= 1.5e-7). Check that bound, and the GELU / GELU' it gives, against
    the exact erf on a dense grid (the kernels' other rounding is FP32)."""
    import math
    z = np.linspace(-12.0, 12.0, 200001)
    x = np.abs(z) / math.sqrt(2.0)
    t = 1.0 / (1.0 + 0.3275911 * x)
    poly = t * (0.254829592 + t * (-0.284496736 + t * (1.421413741 + t * (-1.453152027 + t * 1.061405429))))
    E = np.exp(-0.5 * z * z)
    erf_abs = 1.0 - poly * E
    exact = np.array([math.erf(v) for v in x])
    assert np.abs(erf_abs - exact).max() <= 1.5e-7
    Phi = 0.5 + np.sign(z) * 0.5 * erf_abs
    Phi_exact = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    assert np.abs(z * Phi - z * Phi_exact).max() <= 1.5e-7 * 12
    grad = Phi + z * E / math.sqrt(2.0 * math.pi)
    grad_exact = Phi_exact + z * E / math.sqrt(2.0 * math.pi)
    assert np.abs(grad - grad_exact).max() <= 1e-7
