"""Seeded synthetic inputs shaped like the sCWatter paper's workloads.

This module is shared by the FP64 oracle, the tests and the benchmark. It only
draws random numbers and lays out geometry; it holds none of the coupled-wave
arithmetic (no orders, no s_z, no propagators, no Fourier sums).

Shapes follow the paper's samples: a refractive-index volume on a uniform
grid, filled with spheres or ellipsoids (Sec. 4.4-4.6), and an incident field
given as a 2D image orthogonal to the optical axis (abstract, Sec. 2.3).

Conventions (shared by both sides as *data*, not code):
  * volumes are complex128 arrays ``n[L][Ny][Nx]`` (x fastest); voxel (p,q,r)
    has its centre at ((p+1/2)dx, (q+1/2)dy, (r+1/2)dz) for the geometry test;
  * images are complex128 ``E[Ny][Nx]``; pixel (p,q) sits at (p X/N, q Y/N);
  * every generator takes an explicit seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "sphere_volume", "ellipsoid_volume", "gaussian_beam_image", "plane_wave_image",
    "random_layer_set", "Problem", "config_tiny", "config_single_wavelength",
    "config_sweep_item", "config_surrogate_sample", "cell_centred_planes",
    "phantom_batch", "random_flat",
]


def _centres(n: int, d: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * d


def sphere_volume(nx: int, ny: int, nz: int, centre_vox, radius_vox: float,
                  n_inside: complex, n_background: complex = 1.0) -> np.ndarray:
    """Volume with one sphere; a voxel is inside when its centre is.

    ``centre_vox`` and ``radius_vox`` are in voxel units (all axes share one
    voxel size, as in the paper's cubic-voxel samples).
    """
    z, y, x = np.meshgrid(_centres(nz, 1.0), _centres(ny, 1.0), _centres(nx, 1.0), indexing="ij")
    cx, cy, cz = centre_vox
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius_vox ** 2
    vol = np.full((nz, ny, nx), complex(n_background), dtype=np.complex128)
    vol[inside] = complex(n_inside)
    return vol


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    # Uniform rotation from a normalised Gaussian quaternion.
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def ellipsoid_volume(seed: int, nx: int, ny: int, nz: int, count=(1, 8),
                     semi_axes=(4.0, 16.0), n_re=(1.33, 1.6), kappa=(0.0, 0.05),
                     n_background: complex = 1.0) -> np.ndarray:
    """1..8 random ellipsoids (later ones overwrite earlier ones).

    Semi-axes uniform in ``semi_axes`` voxels, uniform random orientation,
    centre uniform in the grid, n = n_re + i*kappa with both uniform.
    """
    rng = np.random.default_rng(seed)
    k = int(rng.integers(count[0], count[1] + 1))
    z, y, x = np.meshgrid(_centres(nz, 1.0), _centres(ny, 1.0), _centres(nx, 1.0), indexing="ij")
    pts = np.stack([x, y, z], axis=-1)
    vol = np.full((nz, ny, nx), complex(n_background), dtype=np.complex128)
    for _ in range(k):
        ax = rng.uniform(semi_axes[0], semi_axes[1], size=3)
        rot = _random_rotation(rng)
        c = rng.uniform([0, 0, 0], [nx, ny, nz])
        nval = complex(rng.uniform(*n_re), rng.uniform(*kappa))
        local = (pts - c) @ rot  # coordinates in the ellipsoid frame
        inside = np.sum((local / ax) ** 2, axis=-1) <= 1.0
        vol[inside] = nval
    return vol


def gaussian_beam_image(n: int, X: float, lam: float, NA: float = 0.5) -> np.ndarray:
    """Complex image of a Gaussian beam waist, E = exp(-r^2/w0^2), w0 = lam/(pi NA).

    Centred in the image; pixel (p,q) at (p X/n, q X/n). This is the x-component
    of the incident field on the plane z = z_bar.
    """
    w0 = lam / (math.pi * NA)
    c = np.arange(n) * (X / n) - X / 2
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.exp(-(xx ** 2 + yy ** 2) / w0 ** 2).astype(np.complex128)


def plane_wave_image(n: int) -> np.ndarray:
    """Unit normally incident plane wave sampled on an n x n image."""
    return np.ones((n, n), dtype=np.complex128)


def cell_centred_planes(z0: float, zL: float, fz: int) -> np.ndarray:
    """fz output planes at the cell centres of [z0, zL]."""
    return z0 + (np.arange(fz) + 0.5) * ((zL - z0) / fz)


def random_layer_set(seed: int, U: int, V: int, L: int, evanescent_frac: float = 0.05,
                     backward_scale: float = 0.1, dtype=np.complex64):
    """Synthetic per-layer modes with the structure of a solved sample.

    Returns ``(W, gamma, alpha, p_inc, p_ref, p_trn)``:
      * W      [L][3M][4M] (``dtype``): E-field rows of unit-ish eigenvector columns,
               entries complex normal / sqrt(3M);
      * gamma  [L][4M] complex128: modes [0,2M) forward with Re in [0.3,1.6] and
               small Im >= 0 (a fraction ``evanescent_frac`` nearly evanescent,
               Re ~ 0, Im in [0.1,1]); modes [2M,4M) are the negated forward set;
      * alpha  [L][4M] complex128: forward amplitudes complex normal / sqrt(2M),
               backward ones ``backward_scale`` times smaller;
      * p_inc, p_ref, p_trn [3][M] complex128 exterior amplitudes.
    These values are random draws, not a physical solve; they carry the sizes,
    the mode split and the magnitude ranges the synthesis path sees.
    """
    M = U * V
    rng = np.random.default_rng(seed)
    re = rng.uniform(0.3, 1.6, size=(L, 2 * M))
    im = rng.exponential(0.01, size=(L, 2 * M))
    ev = rng.random((L, 2 * M)) < evanescent_frac
    re[ev] = rng.uniform(0.0, 0.05, size=int(ev.sum()))
    im[ev] = rng.uniform(0.1, 1.0, size=int(ev.sum()))
    gf = re + 1j * im
    gamma = np.concatenate([gf, -gf], axis=1)
    scale_w = 1.0 / math.sqrt(2 * 3 * M)
    W = np.empty((L, 3 * M, 4 * M), dtype=dtype)
    for l in range(L):  # per layer keeps the peak host memory at one layer of float64 draws
        W[l].real = rng.standard_normal((3 * M, 4 * M)) * scale_w
        W[l].imag = rng.standard_normal((3 * M, 4 * M)) * scale_w
    sa = 1.0 / math.sqrt(2 * 2 * M)
    af = (rng.standard_normal((L, 2 * M)) + 1j * rng.standard_normal((L, 2 * M))) * sa
    ab = (rng.standard_normal((L, 2 * M)) + 1j * rng.standard_normal((L, 2 * M))) * sa * backward_scale
    alpha = np.concatenate([af, ab], axis=1)
    sp = 1.0 / math.sqrt(2 * M)
    ext = [(rng.standard_normal((3, M)) + 1j * rng.standard_normal((3, M))) * sp for _ in range(3)]
    return W, gamma, alpha, ext[0], ext[1], ext[2]


def random_illuminations(seed: int, I: int, U: int, V: int, L: int, backward_scale: float = 0.1):
    """Amplitudes of I incident fields on one solved sample (same draws as the
    alpha and p of random_layer_set, one set per illumination).

    Returns ``(alpha, p_inc, p_ref, p_trn)``: alpha [I][L][4M], p_* [I][3][M], complex128.
    """
    M = U * V
    rng = np.random.default_rng(seed)
    sa = 1.0 / math.sqrt(2 * 2 * M)
    af = (rng.standard_normal((I, L, 2 * M)) + 1j * rng.standard_normal((I, L, 2 * M))) * sa
    ab = (rng.standard_normal((I, L, 2 * M)) + 1j * rng.standard_normal((I, L, 2 * M))) * sa * backward_scale
    sp = 1.0 / math.sqrt(2 * M)
    ext = [(rng.standard_normal((I, 3, M)) + 1j * rng.standard_normal((I, 3, M))) * sp for _ in range(3)]
    return np.concatenate([af, ab], axis=2), ext[0], ext[1], ext[2]


@dataclass
class Problem:
    """Everything that defines one forward simulation plus its output grid."""
    name: str
    lam: float
    X: float
    Y: float
    U: int
    V: int
    n_volume: np.ndarray          # [L][Ny][Nx] complex
    z_bounds: np.ndarray          # [L+1] ascending
    incident_image: np.ndarray    # [Ny][Nx] complex, x-component unless pol='y'
    pol: str = "x"
    n_top: float = 1.0
    n_bot: complex = 1.0
    z_inc: float | None = None    # defaults to z_bounds[0]
    Fx: int = 64
    Fy: int = 64
    z_planes: np.ndarray = field(default_factory=lambda: np.zeros(0))
    x0: float = 0.0
    y0: float = 0.0

    @property
    def M(self) -> int:
        return self.U * self.V

    @property
    def L(self) -> int:
        return int(self.n_volume.shape[0])


def config_tiny() -> Problem:
    """16x16x4 voxels of 0.25 um, one sphere r=5 voxels n=1.5+0.01i, 7x7 orders,
    normal x-polarised unit plane wave at lambda=1 um; output 64x64x32."""
    d = 0.25
    vol = sphere_volume(16, 16, 4, (8.0, 8.0, 2.0), 5.0, 1.5 + 0.01j, 1.0)
    zb = np.arange(5) * d
    return Problem("tiny", 1.0, 16 * d, 16 * d, 7, 7, vol, zb, plane_wave_image(16),
                   Fx=64, Fy=64, z_planes=cell_centred_planes(zb[0], zb[-1], 32))


def config_single_wavelength(seed: int = 0, U: int = 21, L: int = 32) -> Problem:
    """64x64xL voxels of 0.25 um with 1-8 random ellipsoids in n=1, 21x21 orders,
    x-polarised focused Gaussian beam (NA 0.5) image, output 256x256x(8L)."""
    d = 0.25
    vol = ellipsoid_volume(seed, 64, 64, L)
    zb = np.arange(L + 1) * d
    return Problem("single_wavelength", 1.0, 64 * d, 64 * d, U, U, vol, zb,
                   gaussian_beam_image(64, 64 * d, 1.0, 0.5), Fx=256, Fy=256,
                   z_planes=cell_centred_planes(zb[0], zb[-1], 8 * L))


def config_sweep_item(i: int, n_items: int = 128) -> Problem:
    """Item i of the mid-IR sweep: nu evenly in [1000,1800] cm^-1, 64x64x16 voxels
    of 1 um, centred sphere r=6 voxels, n = 1.5 + i*kappa(nu) with a Lorentzian
    kappa (peak 0.1 at 1650 cm^-1, half-width 10 cm^-1), orders 9+2*floor(9i/128)."""
    nu = 1000.0 + 800.0 * i / (n_items - 1)
    lam = 1e4 / nu  # um
    g = 10.0
    kap = 0.1 * g * g / ((nu - 1650.0) ** 2 + g * g)
    vol = sphere_volume(64, 64, 16, (32.0, 32.0, 8.0), 6.0, 1.5 + 1j * kap, 1.0)
    zb = np.arange(17) * 1.0
    U = 9 + 2 * ((9 * i) // n_items)
    return Problem(f"sweep_{i}", lam, 64.0, 64.0, U, U, vol, zb, plane_wave_image(64),
                   Fx=128, Fy=128, z_planes=cell_centred_planes(zb[0], zb[-1], 64))


def config_surrogate_sample(seed: int) -> Problem:
    """32x32x8 voxels of 0.25 um, ellipsoids with semi-axes in [2,8] voxels,
    15x15 orders, normal x-polarised plane wave; the target is the exit plane."""
    d = 0.25
    vol = ellipsoid_volume(seed, 32, 32, 8, semi_axes=(2.0, 8.0))
    zb = np.arange(9) * d
    return Problem(f"surrogate_{seed}", 1.0, 32 * d, 32 * d, 15, 15, vol, zb,
                   plane_wave_image(32), Fx=64, Fy=64, z_planes=np.array([zb[-1] + 1e-9]))


def random_layer_set_torch(seed: int, U: int, V: int, L: int, device="cuda", evanescent_frac: float = 0.05,
                           backward_scale: float = 0.1):
    """random_layer_set drawn with a seeded torch generator on ``device``.

    Same distributions (and the same returned shapes and dtypes, as tensors);
    used where the host draw would be too slow, e.g. the 25 GB of W of a
    128-wavenumber sweep. The values differ from random_layer_set's.
    """
    import torch
    M = U * V
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device, generator=g)
    re = torch.rand((L, 2 * M), **f64) * 1.3 + 0.3
    im = torch.empty((L, 2 * M), dtype=torch.float64, device=device).exponential_(1.0 / 0.01, generator=g)
    ev = torch.rand((L, 2 * M), **f64) < evanescent_frac
    re = torch.where(ev, torch.rand((L, 2 * M), **f64) * 0.05, re)
    im = torch.where(ev, torch.rand((L, 2 * M), **f64) * 0.9 + 0.1, im)
    gf = torch.complex(re, im)
    gamma = torch.cat([gf, -gf], dim=1)
    scale_w = 1.0 / math.sqrt(2 * 3 * M)
    W = torch.randn((L, 3 * M, 4 * M), dtype=torch.complex64, device=device, generator=g) * (scale_w * math.sqrt(2))
    sa = 1.0 / math.sqrt(2 * 2 * M)
    af = torch.randn((L, 2 * M), dtype=torch.complex128, device=device, generator=g) * (sa * math.sqrt(2))
    ab = torch.randn((L, 2 * M), dtype=torch.complex128, device=device, generator=g) * (sa * math.sqrt(2) * backward_scale)
    alpha = torch.cat([af, ab], dim=1)
    sp = 1.0 / math.sqrt(2 * M)
    ext = [torch.randn((3, M), dtype=torch.complex128, device=device, generator=g) * (sp * math.sqrt(2))
           for _ in range(3)]
    return W, gamma, alpha, ext[0], ext[1], ext[2]


def sweep_geometry(i: int, n_items: int = 128):
    """Sizes of item i of the mid-IR sweep without building its sample volume:
    (lam [um], U, X [um], z_bounds, z_planes, Fx, Fy) -- see config_sweep_item."""
    nu = 1000.0 + 800.0 * i / (n_items - 1)
    zb = np.arange(17) * 1.0
    U = 9 + 2 * ((9 * i) // n_items)
    return 1e4 / nu, U, 64.0, zb, cell_centred_planes(zb[0], zb[-1], 64), 128, 128


def phantom_batch(seed: int, B: int, nx: int = 32, ny: int = 32, nz: int = 8,
                  semi_axes=(2.0, 8.0)) -> np.ndarray:
    """B refractive-index phantoms n[B][nz][ny][nx] (complex128), sample b drawn
    by ellipsoid_volume with seed ``seed + b`` (1..8 ellipsoids, semi-axes in
    ``semi_axes`` voxels, n_re in [1.33, 1.6], kappa in [0, 0.05], background 1)."""
    return np.stack([ellipsoid_volume(seed + b, nx, ny, nz, semi_axes=semi_axes) for b in range(B)])


def random_flat(seed: int, groups) -> np.ndarray:
    """Concatenated seeded draws: for each (size, scale) in ``groups``, ``size``
    values uniform in [-scale, scale] (float64)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-sc, sc, size=int(n)) for n, sc in groups])
