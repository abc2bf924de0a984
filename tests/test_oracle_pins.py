"""Pins of the FP64 oracle against what the physics and mathematics fix.

None of these re-types the oracle's own formulas: each compares it with a
closed form (Fresnel/Airy, characteristic-matrix thin film, homogeneous
spectrum), an invariant (energy, Gauss, continuity, layer splitting,
translation) or a brute force (full block system, FFT vs direct sum).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import cw, synth

K0 = 2 * np.pi  # lambda = 1


def _slab(n_s, d, U=3, V=3, X=2.0, img=None, pol="x", n_bot=1.0, split=1, N=8):
    vol = np.full((split, N, N), complex(n_s))
    zb = np.linspace(0.0, d, split + 1)
    img = wl.plane_wave_image(N) if img is None else img
    return cw.solve(vol, zb, 1.0, X, X, U, V, img, pol=pol, n_bot=n_bot)


def _airy(y1, y2, y3, beta):
    r12, r23 = (y1 - y2) / (y1 + y2), (y2 - y3) / (y2 + y3)
    t12, t23 = 2 * y1 / (y1 + y2), 2 * y2 / (y2 + y3)
    e = np.exp(2j * beta)
    return (r12 + r23 * e) / (1 + r12 * r23 * e), t12 * t23 * np.exp(1j * beta) / (1 + r12 * r23 * e)


# P1 -------------------------------------------------------------------------
@pytest.mark.parametrize("n_s,d,n_bot", [(1.5, 0.37, 1.0), (2.2 + 0.1j, 0.61, 1.33), (1.1 + 0.3j, 1.3, 1.0)])
def test_airy_normal_incidence(n_s, d, n_bot):
    sol = _slab(n_s, d, n_bot=n_bot)
    r, t = _airy(1.0, n_s, n_bot, K0 * n_s * d)
    m0 = 4  # (u, v) = (0, 0) for U = V = 3
    assert abs(sol.p_ref[0, m0] - r) < 1e-12
    assert abs(sol.p_trn[0, m0] - t) < 1e-12
    others = np.delete(np.abs(sol.p_ref[0]), m0)
    assert others.max() < 1e-13


@pytest.mark.parametrize("pol", ["x", "y"])
def test_fresnel_oblique_te_tm(pol):
    """Plane wave in order (u,v) = (1,0): TM for x-polarisation, TE for y."""
    N, X, n_s, d, n_bot = 8, 2.0, 1.7 + 0.05j, 0.45, 1.2
    xs = np.arange(N) * X / N
    img = np.tile(np.exp(2j * np.pi * xs / X), (N, 1))
    sol = _slab(n_s, d, img=img, pol=pol, n_bot=n_bot)
    sx = 0.5  # lambda * u / X
    sz = [np.sqrt(n ** 2 - sx ** 2 + 0j) for n in (1.0, n_s, n_bot)]
    if pol == "x":
        Y = [n ** 2 / s for n, s in zip((1.0, n_s, n_bot), sz)]
        comp = 0
    else:
        Y = sz
        comp = 1
    r, t = _airy(Y[0], Y[1], Y[2], K0 * sz[1] * d)
    m = 5  # (u, v) = (1, 0)
    pin = sol.p_inc[comp, m]
    assert abs(sol.p_ref[comp, m] / pin - r) < 1e-12
    assert abs(sol.p_trn[comp, m] / pin - t) < 1e-12


def test_slab_interior_field_closed_form_tm():
    """Inside a homogeneous slab the field is two plane waves whose amplitudes
    follow from E_x and H_y continuity at z0; E_z = -(s_x/s_z) per wave."""
    N, X, n_s, d = 8, 2.0, 1.45 + 0.02j, 0.8
    xs = np.arange(N) * X / N
    img = np.tile(np.exp(2j * np.pi * xs / X), (N, 1))
    sol = _slab(n_s, d, img=img, pol="x", split=3)
    sx = 0.5
    s1 = np.sqrt(1 - sx ** 2 + 0j)
    s2 = np.sqrt(n_s ** 2 - sx ** 2 + 0j)
    m = 5
    pin, pr = sol.p_inc[0, m], sol.p_ref[0, m]
    Y1, Y2 = 1 / s1, n_s ** 2 / s2
    a = 0.5 * ((pin + pr) + Y1 * (pin - pr) / Y2)
    b = 0.5 * ((pin + pr) - Y1 * (pin - pr) / Y2)
    for z in [0.0, 0.13, 0.4, 0.55, 0.79, 0.8]:
        S = synth.spectrum_at(sol, z)
        f, g = a * np.exp(1j * K0 * s2 * z), b * np.exp(-1j * K0 * s2 * z)
        assert abs(S[0, m] - (f + g)) < 1e-11
        assert abs(S[2, m] - (-(sx / s2) * (f - g))) < 1e-11
        assert np.abs(np.delete(S[0], m)).max() < 1e-12


def test_airy_interior_volume_normal():
    n_s, d = 1.5 + 0.01j, 0.5
    sol = _slab(n_s, d, split=2)
    r, _ = _airy(1.0, n_s, 1.0, K0 * n_s * d)
    a = 0.5 * ((1 + r) + (1 - r) / n_s)
    b = 0.5 * ((1 + r) - (1 - r) / n_s)
    zs = np.linspace(-0.3, 0.8, 12)
    E = synth.synthesize_direct(sol, 16, 16, zs)
    for iz, z in enumerate(zs):
        if z < 0:
            ex = np.exp(1j * K0 * z) + r * np.exp(-1j * K0 * z)
        elif z <= d:
            ex = a * np.exp(1j * K0 * n_s * z) + b * np.exp(-1j * K0 * n_s * z)
        else:
            ex = _airy(1.0, n_s, 1.0, K0 * n_s * d)[1] * np.exp(1j * K0 * (z - d))
        assert np.abs(E[0, iz] - ex).max() < 1e-11
        assert np.abs(E[1:, iz]).max() < 1e-11


# P2 -------------------------------------------------------------------------
def test_homogeneous_spectrum():
    U, V, lam, X, Y = 5, 3, 1.0, 2.3, 1.7
    sx, sy = cw.directions(U, V, lam, X, Y)
    u, v = cw.orders(U, V)
    n = 1.6 + 0.03j
    _, _, D = cw.layer_operators(np.full((12, 12), n), sx, sy, u, v)
    g, _ = cw.layer_modes(D)
    sz = np.sqrt(n ** 2 - sx ** 2 - sy ** 2)
    expect = np.sort_complex(np.concatenate([sz, sz, -sz, -sz]))
    assert np.abs(np.sort_complex(g) - expect).max() < 1e-12


# P3 -------------------------------------------------------------------------
def test_energy_lossless_heterogeneous():
    vol = wl.ellipsoid_volume(3, 16, 16, 3, semi_axes=(2, 6), kappa=(0.0, 0.0))
    img = wl.gaussian_beam_image(16, 4.0, 1.0, 0.3)
    sol = cw.solve(vol, np.arange(4) * 0.3, 1.0, 4.0, 4.0, 5, 5, img, n_bot=1.33)
    st = cw.s_z(1.0, sol.sx, sol.sy)
    sb = cw.s_z(1.33, sol.sx, sol.sy)
    prop_t, prop_b = np.abs(st.imag) < 1e-14, np.abs(sb.imag) < 1e-14
    pin = np.sum(st.real[prop_t] * np.sum(np.abs(sol.p_inc[:, prop_t]) ** 2, axis=0))
    pr = np.sum(st.real[prop_t] * np.sum(np.abs(sol.p_ref[:, prop_t]) ** 2, axis=0))
    pt = np.sum(sb.real[prop_b] * np.sum(np.abs(sol.p_trn[:, prop_b]) ** 2, axis=0))
    assert abs(pin - pr - pt) / pin < 1e-10
    assert pr > 1e-4 and pt > 0.5 * pin  # the sample scatters, energy is not trivially 0 = 0


# P4 -------------------------------------------------------------------------
def test_gauss_law_exterior_and_modes():
    sol = cw.solve_problem(wl.config_tiny())
    st = cw.s_z(1.0, sol.sx, sol.sy)
    assert np.abs(sol.sx * sol.p_ref[0] + sol.sy * sol.p_ref[1] - st * sol.p_ref[2]).max() < 1e-12
    assert np.abs(sol.sx * sol.p_trn[0] + sol.sy * sol.p_trn[1] + st * sol.p_trn[2]).max() < 1e-12
    # inside a homogeneous layer every mode's (Px, Py, Pz) satisfies s . p = 0
    hs = _slab(1.3 + 0.02j, 0.3, U=5, V=5, X=2.3, N=12)
    M = 25
    W, g = hs.W[0], hs.gamma[0]
    div = hs.sx[:, None] * W[:M] + hs.sy[:, None] * W[M:2 * M] + g[None, :] * W[2 * M:]
    assert np.abs(div).max() < 1e-12


# P5 -------------------------------------------------------------------------
def test_interface_continuity():
    sol = cw.solve_problem(wl.config_tiny())
    k = 2 * np.pi / sol.lam
    zb = sol.z_bounds
    M = sol.M

    def from_layer(l, z):
        g = synth.propagators(sol.gamma[l], z, zb[l], zb[l + 1], k)
        return (sol.W[l] @ (sol.alpha[l] * g)).reshape(3, M)

    for l in range(sol.L - 1):
        assert np.abs(sol.Bm[l] @ sol.alpha[l] - sol.T[l + 1] @ sol.alpha[l + 1]).max() < 1e-10
        a, b = from_layer(l, zb[l + 1]), from_layer(l + 1, zb[l + 1])
        assert np.abs(a[:2] - b[:2]).max() < 1e-10
    above = sol.p_inc + sol.p_ref  # exterior spectrum at z0 (z_bar = z0)
    assert np.abs(above[:2] - from_layer(0, zb[0])[:2]).max() < 1e-10
    assert np.abs(sol.p_trn[:2] - from_layer(sol.L - 1, zb[-1])[:2]).max() < 1e-10


# P6 -------------------------------------------------------------------------
def test_layer_split_invariance():
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    vol2 = np.repeat(p.n_volume, 2, axis=0)
    zb2 = np.linspace(p.z_bounds[0], p.z_bounds[-1], 2 * p.L + 1)
    sol2 = cw.solve(vol2, zb2, p.lam, p.X, p.Y, p.U, p.V, p.incident_image)
    assert np.abs(sol.p_ref - sol2.p_ref).max() < 1e-10
    assert np.abs(sol.p_trn - sol2.p_trn).max() < 1e-10
    zs = [0.05, 0.3, 0.62, 0.99, -0.2, 1.3]
    for z in zs:
        assert np.abs(synth.spectrum_at(sol, z) - synth.spectrum_at(sol2, z)).max() < 1e-10


# P7 -------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_block_system_brute_force(seed):
    vol = wl.ellipsoid_volume(seed, 12, 12, 3, semi_axes=(2, 5))
    img = wl.gaussian_beam_image(12, 3.0, 1.0, 0.4)
    sol = cw.solve(vol, np.array([0.0, 0.2, 0.45, 0.6]), 1.0, 3.0, 3.0, 5, 5, img, n_bot=1.2 + 0.01j)
    pr, pt, al = cw.solve_block_system(sol)
    assert np.abs(pr - sol.p_ref).max() < 1e-9
    assert np.abs(pt - sol.p_trn).max() < 1e-9
    assert np.abs(al - sol.alpha).max() < 1e-9 * max(1.0, np.abs(al).max())


# P8 -------------------------------------------------------------------------
@pytest.mark.parametrize("Fx,Fy,x0,y0", [(16, 16, 0.0, 0.0), (32, 16, 0.3, -1.1), (4, 8, 0.7, 0.2)])
def test_direct_sum_equals_fft(Fx, Fy, x0, y0):
    sol = cw.solve_problem(wl.config_tiny())
    S = synth.spectrum_at(sol, 0.41)
    xs, ys = synth.pixel_coords(sol, Fx, Fy, x0, y0)
    a = synth.field_direct(sol, S, xs, ys)
    b = synth.field_fft(sol, S, Fx, Fy, x0, y0)  # Fx = 4 < U = 7 folds orders
    assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(a).max())


# P9 -------------------------------------------------------------------------
def test_convolution_matrix_is_the_product_rule():
    rng = np.random.default_rng(5)
    U, V, N = 5, 4, 10
    u, v = cw.orders(U, V)
    eps = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    fhat = rng.standard_normal(U * V) + 1j * rng.standard_normal(U * V)
    p = np.arange(N)
    # band-limited f on the grid, then the product and its spectrum at the orders
    f = np.zeros((N, N), dtype=complex)
    for m in range(U * V):
        f += fhat[m] * np.exp(2j * np.pi * (u[m] * p[None, :] + v[m] * p[:, None]) / N)
    prod = eps * f
    ghat = np.array([np.sum(prod * np.exp(-2j * np.pi * (u[m] * p[None, :] + v[m] * p[:, None]) / N))
                     for m in range(U * V)]) / N ** 2
    Phi = cw.convolution_matrix(cw.fourier_table(eps), u, v)
    assert np.abs(Phi @ fhat - ghat).max() < 1e-12


def _ez_from_curl(Q, n_grid, U, V, X, Y, lam):
    """E_z spectrum of each column of Q (rows [Px, Py, Bx, By]) from Maxwell on
    the sample grid: B_x, B_y as band-limited fields, (curl B)_z by exact spectral
    derivatives of those trigonometric polynomials, then E_z = (curl B)_z /
    (-i k n^2) pointwise (curl B = -i k n^2 E in the oracle's units), and its
    spectrum at the orders."""
    M = U * V
    k = 2 * np.pi / lam
    ny, nx = n_grid.shape
    u, v = cw.orders(U, V)
    out = np.empty((M, Q.shape[1]), dtype=complex)
    fx = np.fft.fftfreq(nx, d=X / nx)  # cycles per unit length of each FFT bin
    fy = np.fft.fftfreq(ny, d=Y / ny)
    for j in range(Q.shape[1]):
        grids = []
        for blk in (2, 3):  # B_x, B_y
            spec = np.zeros((ny, nx), dtype=complex)
            spec[v % ny, u % nx] = Q[blk * M:(blk + 1) * M, j] * nx * ny
            grids.append(spec)
        dBy_dx = np.fft.ifft2(grids[1] * (2j * np.pi * fx[None, :]))
        dBx_dy = np.fft.ifft2(grids[0] * (2j * np.pi * fy[:, None]))
        ez = (dBy_dx - dBx_dy) / (-1j * k * n_grid.astype(complex) ** 2)
        out[:, j] = (np.fft.fft2(ez) / (nx * ny))[v % ny, u % nx]
    return out


@pytest.mark.parametrize("kind", ["random", "ellipsoids"])
def test_ez_rows_follow_maxwell_in_a_heterogeneous_layer(kind):
    """The E_z rows of W (Eq. 33, reading R5) inside a heterogeneous complex-n
    layer equal the truncated spectrum of (curl B)_z / (-i k n^2) on the sample
    grid. Exact (no aliasing) because the grid holds every order difference
    (N >= 2U-1). The sample has no inversion symmetry, so Psi^T differs from Psi
    and an index reversal inside e_rows would fail here."""
    U, V, nx, ny, X, Y, lam = 5, 4, 12, 10, 2.3, 1.9, 1.0
    rng = np.random.default_rng(17)
    if kind == "random":
        n = 1.2 + 0.4 * rng.random((ny, nx)) + 0.08j * rng.random((ny, nx))
    else:
        n = wl.ellipsoid_volume(4, nx, ny, 3, semi_axes=(2, 5), kappa=(0.01, 0.05))[1]
        assert np.ptp(n.real) > 0.2  # the slice cuts an ellipsoid
    sx, sy = cw.directions(U, V, lam, X, Y)
    u, v = cw.orders(U, V)
    _, Psi, _ = cw.layer_operators(n, sx, sy, u, v)
    M = U * V
    Q = rng.standard_normal((4 * M, 6)) + 1j * rng.standard_normal((4 * M, 6))
    W = cw.e_rows(Q, Psi, sx, sy)
    ez = _ez_from_curl(Q, n, U, V, X, Y, lam)
    scale = np.abs(ez).max()
    assert np.abs(W[2 * M:] - ez).max() < 1e-12 * scale
    assert np.array_equal(W[:2 * M], Q[:2 * M])  # E_x, E_y rows are the P rows themselves
    # the test tells the two convolution orientations apart on this sample
    h = sy[:, None] * Q[2 * M:3 * M] - sx[:, None] * Q[3 * M:]
    assert np.abs(Psi.T @ h - ez).max() > 1e-3 * scale


# P10 ------------------------------------------------------------------------
def test_translation_covariance():
    p = wl.config_tiny()
    sol = cw.solve_problem(p)
    dlt = 3
    vol = np.roll(p.n_volume, dlt, axis=2)
    img = np.roll(wl.gaussian_beam_image(16, p.X, 1.0, 0.4), dlt, axis=1)
    sol_a = cw.solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, np.roll(img, -dlt, axis=1))
    sol_b = cw.solve(vol, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, img)
    u, _ = cw.orders(p.U, p.V)
    ph = np.exp(-2j * np.pi * u * dlt / 16)
    assert np.abs(sol_a.p_ref * ph - sol_b.p_ref).max() < 1e-12
    assert np.abs(sol_a.p_trn * ph - sol_b.p_trn).max() < 1e-12
    del sol


# P11 ------------------------------------------------------------------------
def test_single_order_is_thin_film_transfer_matrix():
    ns = [1.4 + 0.01j, 2.1, 1.7 + 0.2j, 1.2]
    ds = [0.13, 0.29, 0.07, 0.41]
    n_sub = 1.52
    vol = np.stack([np.full((1, 1), n) for n in ns])
    zb = np.concatenate([[0.0], np.cumsum(ds)])
    sol = cw.solve(vol, zb, 1.0, 1.0, 1.0, 1, 1, np.ones((1, 1)), n_bot=n_sub)
    # Born & Wolf characteristic matrix, normal incidence, exp(-i w t)
    Mt = np.eye(2, dtype=complex)
    for n, d in zip(ns, ds):
        b = K0 * n * d
        Mt = Mt @ np.array([[np.cos(b), -1j * np.sin(b) / n], [-1j * n * np.sin(b), np.cos(b)]])
    A = (Mt[0, 0] + Mt[0, 1] * n_sub) * 1.0
    B = Mt[1, 0] + Mt[1, 1] * n_sub
    r, t = (A - B) / (A + B), 2.0 / (A + B)
    assert abs(sol.p_ref[0, 0] - r) < 1e-12
    assert abs(sol.p_trn[0, 0] - t) < 1e-12


# P12 ------------------------------------------------------------------------
def test_convergence_in_orders():
    p = wl.config_tiny()
    xs = np.arange(16) * p.X / 16
    fields = []
    for U in (3, 5, 7):
        sol = cw.solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, U, U, p.incident_image)
        S = synth.spectrum_at(sol, p.z_bounds[-1] + 0.25)
        fields.append(synth.field_direct(sol, S, xs, xs)[0])
    d1 = np.linalg.norm(fields[1] - fields[0]) / np.linalg.norm(fields[1])
    d2 = np.linalg.norm(fields[2] - fields[1]) / np.linalg.norm(fields[2])
    assert d2 < d1


# region convention ----------------------------------------------------------
def test_region_half_open():
    zb = [0.0, 1.0, 2.0]
    assert synth.region(-1e-12, zb) == -1
    assert synth.region(0.0, zb) == 0
    assert synth.region(1.0, zb) == 1
    assert synth.region(2.0, zb) == 1
    assert synth.region(2.0 + 1e-12, zb) == 2


# objective pupil below the sample -------------------------------------------
@pytest.mark.parametrize("na,passed", [(0.3, 5), (0.55, 13), (5.0, 49)])
def test_pupil_is_an_ideal_low_pass_of_the_transmitted_field(na, passed):
    """Below the sample the pupil keeps exactly the plane waves a lens of the
    given NA collects: filtering the unfiltered field's own FFT with the disk
    |lambda f| <= NA (f the FFT's spatial frequencies) gives the pupil field, and
    the number of passed orders is the lattice-point count of that disk."""
    sol = cw.solve_problem(wl.config_tiny())
    Fx = Fy = 32
    zs = [sol.z_bounds[-1] + 0.3, sol.z_bounds[-1] + 1.7]
    full = synth.synthesize_direct(sol, Fx, Fy, zs)
    cut = synth.synthesize_direct(sol, Fx, Fy, zs, pupil_na=na)
    fx = np.fft.fftfreq(Fx, d=sol.X / Fx)
    fy = np.fft.fftfreq(Fy, d=sol.Y / Fy)
    disk = (sol.lam * fx[None, :]) ** 2 + (sol.lam * fy[:, None]) ** 2 <= na * na * (1 + 1e-9)
    spec = np.fft.fft2(full, axes=(-2, -1))
    lowpass = np.fft.ifft2(spec * disk, axes=(-2, -1))
    assert np.abs(cut - lowpass).max() < 1e-12 * np.abs(full).max()
    assert int(synth.pupil_mask(sol, na).sum()) == passed
    if passed < sol.U * sol.V:
        assert np.abs(cut - full).max() > 1e-3 * np.abs(full).max()  # the pupil removes something
    # above the sample and inside it the pupil changes nothing
    zin = [sol.z_bounds[0] - 0.4, 0.5 * (sol.z_bounds[0] + sol.z_bounds[-1])]
    assert np.array_equal(synth.synthesize_direct(sol, 8, 8, zin, pupil_na=na),
                          synth.synthesize_direct(sol, 8, 8, zin))


# field at arbitrary points ----------------------------------------------------
def test_point_sums_match_the_fft_on_the_grid_and_are_periodic():
    """The per-point sum (x-z / y-z planes and point sets) agrees with numpy's
    inverse FFT at grid points and repeats with the lateral period."""
    sol = cw.solve_problem(wl.config_tiny())
    z = 0.41
    Fx, Fy, x0, y0 = 16, 8, 0.3, -0.2
    grid = synth.field_fft(sol, synth.spectrum_at(sol, z), Fx, Fy, x0, y0)
    xs, ys = synth.pixel_coords(sol, Fx, Fy, x0, y0)
    gx, gy = np.meshgrid(xs, ys)
    pts = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, z)], axis=1)
    E = synth.field_points(sol, pts).reshape(3, Fy, Fx)
    assert np.abs(E - grid).max() < 1e-12 * np.abs(grid).max()
    far = pts + np.array([3 * sol.X, -2 * sol.Y, 0.0])
    assert np.abs(synth.field_points(sol, far).reshape(3, Fy, Fx) - E).max() < 1e-10 * np.abs(E).max()
