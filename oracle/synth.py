"""Field synthesis in FP64 (TEST INFRASTRUCTURE; see oracle/__init__.py).

The synthesis is a plain definition, so the oracle writes it out:

  region(z):  z < z0 -> above the sample; z_{l-1} <= z < z_l -> layer l
              (the last layer also takes z = z_L); z > z_L -> below (Sec. 2.6,
              a plane exactly on an interface belongs to the layer below it).
  spectrum:   above:  p_inc exp(i k s_z(n_top)(z - z_bar)) + p_ref exp(-i k s_z(n_top)(z - z0))
              below:  p_trn exp(i k s_z(n_bot)(z - z_L))                       (Eq. 9)
              inside: S(z) = W_l (alpha_l o g(z)), g_j = exp(i k gamma_j (z - z_ref,j)),
                      z_ref = z_{l-1} for forward modes, z_l for backward modes
                      (Eq. 30-31 with the precompute of Sec. 4.1, Eq. 34).
  field:      E_c(x, y, z) = sum_m S_c[m](z) exp(2 pi i (u_m x / X + v_m y / Y))   (Eq. 10)
              on pixels x_i = x0 + i X/Fx, y_j = y0 + j Y/Fy, summed directly.

``field_fft`` evaluates the same sum through numpy's inverse FFT; it exists
only to pin the direct sum (the two must agree to rounding).
"""
from __future__ import annotations

import numpy as np

from .cw import LayerSet, orders, directions, s_z


def region(z: float, z_bounds) -> int:
    """-1 above the sample, l (0-based) inside layer l+1, L below (Sec. 2.6)."""
    zb = np.asarray(z_bounds)
    L = len(zb) - 1
    if z < zb[0]:
        return -1
    if z > zb[-1]:
        return L
    l = int(np.searchsorted(zb, z, side="right")) - 1
    return min(l, L - 1)


def propagators(gamma_l: np.ndarray, z: float, z_top: float, z_bot: float, k: float) -> np.ndarray:
    """g(z) of one layer: exp(i k gamma (z - z_ref)), forward modes referenced
    to the top z_{l-1}, backward modes to the bottom z_l (Eq. 7, Eq. 30)."""
    h = len(gamma_l) // 2
    zref = np.concatenate([np.full(h, z_top), np.full(h, z_bot)])
    return np.exp(1j * k * gamma_l * (z - zref))


def pupil_mask(ls: LayerSet, na: float) -> np.ndarray:
    """1 for the orders a collecting objective of numerical aperture `na` passes
    (|s_bar| <= na, s_bar = lambda (u/X, v/Y), Eq. 6), 0 for the rest; all ones for
    na <= 0. An imaging system sees the external field below the sample (Sec. 1:
    objectives of a given NA; Sec. 4.1: only the external field is needed to model
    an imaging system); the mask is applied there."""
    sx, sy = directions(ls.U, ls.V, ls.lam, ls.X, ls.Y)
    if na <= 0:
        return np.ones(ls.M)
    return (sx * sx + sy * sy <= na * na * (1.0 + 1e-12)).astype(np.float64)


def spectrum_at(ls: LayerSet, z: float, pupil_na: float = 0.0) -> np.ndarray:
    """Per-plane Fourier-domain field S[c][m] at height z (Eq. 9 / Eq. 34); below the
    sample the orders outside the pupil (pupil_mask) are dropped when pupil_na > 0."""
    k = 2 * np.pi / ls.lam
    zb = np.asarray(ls.z_bounds)
    r = region(z, zb)
    if r == -1 or r == ls.L:
        sx, sy = directions(ls.U, ls.V, ls.lam, ls.X, ls.Y)
        if r == -1:
            st = s_z(ls.n_top, sx, sy)
            return (ls.p_inc * np.exp(1j * k * st * (z - ls.zbar))
                    + ls.p_ref * np.exp(-1j * k * st * (z - zb[0])))
        sb = s_z(ls.n_bot, sx, sy)
        return ls.p_trn * np.exp(1j * k * sb * (z - zb[-1])) * pupil_mask(ls, pupil_na)
    g = propagators(ls.gamma[r], z, zb[r], zb[r + 1], k)
    return (ls.W[r] @ (ls.alpha[r] * g)).reshape(3, ls.M)


def pixel_coords(ls: LayerSet, Fx: int, Fy: int, x0: float = 0.0, y0: float = 0.0):
    return x0 + np.arange(Fx) * (ls.X / Fx), y0 + np.arange(Fy) * (ls.Y / Fy)


def field_direct(ls: LayerSet, S: np.ndarray, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """Eq. 10 by direct summation over the M orders: returns E[3][len(ys)][len(xs)]."""
    u, v = orders(ls.U, ls.V)
    ex = np.exp(2j * np.pi * np.outer(u, xs) / ls.X)   # [M][Fx]
    ey = np.exp(2j * np.pi * np.outer(v, ys) / ls.Y)   # [M][Fy]
    out = np.empty((3, len(ys), len(xs)), dtype=np.complex128)
    for c in range(3):
        out[c] = (S[c][:, None] * ey).T @ ex            # sum_m S_m ey[m,j] ex[m,i]
    return out


def field_points(ls: LayerSet, pts: np.ndarray) -> np.ndarray:
    """Eq. 9/10/34 at arbitrary points pts[n] = (x, y, z): returns E[3][n].

    Each point is summed on its own (spectrum at its z, then the M-term sum)."""
    u, v = orders(ls.U, ls.V)
    out = np.empty((3, len(pts)), dtype=np.complex128)
    cache = {}
    for i, (x, y, z) in enumerate(pts):
        if z not in cache:
            cache[z] = spectrum_at(ls, float(z))
        ph = np.exp(2j * np.pi * (u * x / ls.X + v * y / ls.Y))
        out[:, i] = cache[z] @ ph
    return out


def synthesize_direct(ls: LayerSet, Fx: int, Fy: int, z_planes, x0: float = 0.0,
                      y0: float = 0.0, pupil_na: float = 0.0) -> np.ndarray:
    """The whole volume E[3][Fz][Fy][Fx] by direct summation."""
    xs, ys = pixel_coords(ls, Fx, Fy, x0, y0)
    zs = np.asarray(z_planes, dtype=np.float64)
    out = np.empty((3, len(zs), Fy, Fx), dtype=np.complex128)
    for iz, z in enumerate(zs):
        out[:, iz] = field_direct(ls, spectrum_at(ls, float(z), pupil_na), xs, ys)
    return out


def spectra(ls: LayerSet, z_planes, pupil_na: float = 0.0) -> np.ndarray:
    """S[Fz][3][M] for every plane."""
    return np.stack([spectrum_at(ls, float(z), pupil_na) for z in np.asarray(z_planes)])


def field_fft(ls: LayerSet, S: np.ndarray, Fx: int, Fy: int, x0: float = 0.0,
              y0: float = 0.0) -> np.ndarray:
    """Eq. 10 through numpy's inverse FFT (cross-check only).

    Orders are folded into bins (u mod Fx, v mod Fy) after multiplying by the
    origin phase exp(2 pi i (u x0/X + v y0/Y)); numpy's 1/N is undone."""
    u, v = orders(ls.U, ls.V)
    ph = np.exp(2j * np.pi * (u * x0 / ls.X + v * y0 / ls.Y))
    out = np.empty((3, Fy, Fx), dtype=np.complex128)
    for c in range(3):
        grid = np.zeros((Fy, Fx), dtype=np.complex128)
        np.add.at(grid, (v % Fy, u % Fx), S[c] * ph)
        out[c] = np.fft.ifft2(grid) * (Fx * Fy)
    return out
