"""Coupled-wave solve in FP64 (TEST INFRASTRUCTURE; see oracle/__init__.py).

Units: lengths in the same unit as the vacuum wavelength lambda; k = 2 pi / lambda.
The magnetic amplitudes B are H with the impedance factors of Eq. 15-16 dropped,
so that curl E = i k B and curl B = -i k n^2 E.

Readings of the paper taken here (each is pinned by a CPU test):
  R1  Eq. 11-12 carry no normalisation; we divide by Nx*Ny so that a homogeneous
      layer gives Phi = n^2 I (pinned: homogeneous spectrum, Airy slab).
  R2  The circulant printed for Psi (Sec. 2.5.2) is read as the 2-D convolution
      matrix Phi[m,m'] = phi at (u_m-u_m', v_m-v_m') (pinned: convolution test).
  R3  Eq. 21 as printed gives exponentially growing fields in a homogeneous
      medium; re-deriving it from Eq. 15-16 negates its lower two block rows and
      makes their s s^T products diagonal (pinned: homogeneous spectrum, Airy).
  R4  The B_x row of C (Eq. 28) is -s_z P_y + s_y P_z (from B = s x p), and s_z
      is taken per wave: +s_z(n_top) incident, -s_z(n_top) reflected,
      +s_z(n_bot) transmitted (pinned: oblique TE/TM Fresnel slab).
  R5  E_z = Psi (s_y B_x - s_x B_y) (Eq. 33 with B = +H) (pinned: Gauss law per
      mode in a homogeneous layer, interface continuity).
  R6  The accents of the two per-layer matrices (Sec. 2.5.4) are used as in the
      boundary equations 24-26: T_l = field at the top of layer l,
      B_l = field at its bottom (pinned: full block system).
  R7  The reflected wave of Eq. 9 travels towards -z: p_ref exp(-i k s_z (z-z0)).
  R8  "gamma >= 0" (Sec. 2.5.3) is read as: forward = Im gamma > tau|gamma|, or
      |Im gamma| <= tau|gamma| and Re gamma > 0 (tau = 1e-10); forward modes
      are referenced to z_{l-1}, backward ones to z_l, so |exp| <= 1 inside.
  R9  s_z branch (Eq. 2): principal root, negated when Im < 0 (or Im = 0, Re < 0).
  R10 G_bar (Sec. 2.5.4) repeats the M-vector exp(i k s_z (z0 - z_bar)) over the
      four blocks of R.
  R11 The incident image is projected with 1/N_pix (Eq. 4 on the pixel grid);
      x-polarised by default, p_z from Gauss' law (Eq. 14).
  R12 The Psi of Eq. 12 (Fourier series of 1/n^2) is used as printed, not the
      inverse of Phi.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TAU = 1e-10


# ---------------------------------------------------------------- Sec. 2.2 ---
def orders(U: int, V: int):
    """Signed integer orders in the flat order of Sec. 2.2.

    u in [-floor(U/2), floor((U-1)/2)], v likewise; m = (v+floor(V/2))U + u+floor(U/2).
    Returns (u[m], v[m]) as int arrays of length M = U V.
    """
    u = np.arange(U) - U // 2
    v = np.arange(V) - V // 2
    return np.tile(u, V), np.repeat(v, U)


def directions(U: int, V: int, lam: float, X: float, Y: float):
    """Eq. 6: s_bar = (2 pi / k)[u/X, v/Y] = lambda [u/X, v/Y]."""
    u, v = orders(U, V)
    return lam * u / X, lam * v / Y


def s_z(n, sx, sy):
    """Eq. 2, s_z = sqrt(n^2 - sx^2 - sy^2), on the decaying branch (reading R9)."""
    w = np.sqrt(np.asarray(n, dtype=np.complex128) ** 2 - np.asarray(sx) ** 2 - np.asarray(sy) ** 2 + 0j)
    flip = (w.imag < 0) | ((w.imag == 0) & (w.real < 0))
    return np.where(flip, -w, w)


# ---------------------------------------------------------------- Sec. 2.4 ---
def fourier_table(values: np.ndarray) -> np.ndarray:
    """Eq. 11 / Eq. 12 on the sample grid, divided by Nx*Ny (reading R1).

    ``values[q, p]`` is the layer's n^2 (or 1/n^2) at (p X/Nx, q Y/Ny). Returns
    F[dv mod Ny, du mod Nx] = (1/(Nx Ny)) sum_{p,q} values[q,p]
    exp(-2 pi i (du p/Nx + dv q/Ny)).
    """
    ny, nx = values.shape
    return np.fft.fft2(values) / (nx * ny)


def convolution_matrix(table: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Phi[m, m'] = phi_(u_m - u_m', v_m - v_m') (Sec. 2.5.2, reading R2)."""
    ny, nx = table.shape
    # order differences reach +-(U-1); fewer samples than 2U-1 would alias them
    if nx < 2 * (u.max() - u.min()) + 1 or ny < 2 * (v.max() - v.min()) + 1:
        raise ValueError("sample grid too coarse for the requested orders")
    du = (u[:, None] - u[None, :]) % nx
    dv = (v[:, None] - v[None, :]) % ny
    return table[dv, du]


# ------------------------------------------------------------- Sec. 2.5.2 ---
def property_matrix(sx, sy, Phi, Psi) -> np.ndarray:
    """D of Eq. 21 with d R / dz = i k D R, R = [Px, Py, Bx, By] (reading R3).

    Top-right block (d[Px,Py]/dz from [Bx,By]):
        [[ diag(sx) Psi diag(sy),      I - diag(sx) Psi diag(sx)],
         [ diag(sy) Psi diag(sy) - I,  -diag(sy) Psi diag(sx)   ]]
    Bottom-left block (d[Bx,By]/dz from [Px,Py]):
        [[ -diag(sx sy),       diag(sx^2) - Phi ],
         [ Phi - diag(sy^2),   diag(sx sy)      ]]
    """
    M = len(sx)
    I = np.eye(M)
    Sx = np.diag(sx).astype(np.complex128)
    Sy = np.diag(sy).astype(np.complex128)
    A = np.block([[Sx @ Psi @ Sy, I - Sx @ Psi @ Sx],
                  [Sy @ Psi @ Sy - I, -Sy @ Psi @ Sx]])
    B = np.block([[-Sx @ Sy, Sx @ Sx - Phi],
                   [Phi - Sy @ Sy, Sy @ Sx]])
    Z = np.zeros((2 * M, 2 * M), dtype=np.complex128)
    return np.block([[Z, A], [B, Z]])


# ------------------------------------------------------------- Sec. 2.5.3 ---
def layer_modes(D: np.ndarray):
    """Eigendecomposition D = Q Gamma Q^-1 (LAPACK geev, Sec. 3.2), split into
    2M forward then 2M backward modes (reading R8).

    Forward modes are ordered by descending Re(gamma), backward ones by
    descending Re(-gamma). Columns of Q have unit 2-norm.
    """
    g, Q = np.linalg.eig(D)
    a = np.abs(g)
    fwd = (g.imag > TAU * a) | ((np.abs(g.imag) <= TAU * a) & (g.real > 0))
    n = D.shape[0]
    if int(fwd.sum()) != n // 2:
        raise ValueError(f"expected {n // 2} forward modes, found {int(fwd.sum())}")
    fi = np.where(fwd)[0]
    bi = np.where(~fwd)[0]
    fi = fi[np.argsort(-g[fi].real, kind="stable")]
    bi = bi[np.argsort(g[bi].real, kind="stable")]
    order = np.concatenate([fi, bi])
    return g[order], Q[:, order]


# ------------------------------------------------------------- Sec. 2.5.4 ---
def top_bottom(gamma, Q, d: float, k: float):
    """Per-layer matrices of Eq. 24-26 (reading R6).

    With the forward modes referenced to the layer top and the backward modes
    to its bottom:
      T = [Q_f, Q_b diag(exp(-i k gamma_b d))]  (field at z_{l-1})
      B = [Q_f diag(exp(i k gamma_f d)), Q_b]   (field at z_l)
    """
    h = Q.shape[1] // 2
    ef = np.exp(1j * k * gamma[:h] * d)
    eb = np.exp(-1j * k * gamma[h:] * d)
    T = np.concatenate([Q[:, :h], Q[:, h:] * eb[None, :]], axis=1)
    B = np.concatenate([Q[:, :h] * ef[None, :], Q[:, h:]], axis=1)
    return T, B


def p_to_r(sx, sy, sz) -> np.ndarray:
    """C of Eq. 28 (reading R4): R = [Px, Py, Bx, By] of waves with amplitude P.

    Rows: [I,0,0], [0,I,0], [0,-diag(sz),diag(sy)], [diag(sz),0,-diag(sx)].
    """
    M = len(sx)
    I = np.eye(M, dtype=np.complex128)
    Z = np.zeros((M, M), dtype=np.complex128)
    dz = np.diag(np.asarray(sz, dtype=np.complex128))
    return np.block([[I, Z, Z], [Z, I, Z], [Z, -dz, np.diag(sy).astype(complex)],
                     [dz, Z, -np.diag(sx).astype(complex)]])


def project_image(img: np.ndarray, u, v) -> np.ndarray:
    """Plane-wave amplitudes of a sampled image (Eq. 4 on the pixel grid,
    reading R11): p_m = (1/N_pix) sum E(p,q) exp(-2 pi i (u_m p/Nx + v_m q/Ny))."""
    ny, nx = img.shape
    F = np.fft.fft2(img) / (nx * ny)
    return F[v % ny, u % nx]


# ------------------------------------------------------------------ results ---
@dataclass
class LayerSet:
    """Everything the synthesis path consumes (the solve's output).

    W[l] is [3M][4M] (rows c*M + m, c = x,y,z), gamma/alpha[l] are [4M] with
    modes [0,2M) forward and [2M,4M) backward; p_* are [3][M].
    """
    lam: float
    X: float
    Y: float
    U: int
    V: int
    z_bounds: np.ndarray
    W: np.ndarray
    gamma: np.ndarray
    alpha: np.ndarray
    p_inc: np.ndarray
    p_ref: np.ndarray
    p_trn: np.ndarray
    n_top: float = 1.0
    n_bot: complex = 1.0
    z_inc: float | None = None

    @property
    def M(self) -> int:
        return self.U * self.V

    @property
    def L(self) -> int:
        return len(self.z_bounds) - 1

    @property
    def zbar(self) -> float:
        return float(self.z_bounds[0]) if self.z_inc is None else float(self.z_inc)


@dataclass
class Solution(LayerSet):
    """LayerSet plus the intermediate matrices used by the pins."""
    sx: np.ndarray = field(default=None)
    sy: np.ndarray = field(default=None)
    Q: list = field(default_factory=list)
    T: list = field(default_factory=list)
    Bm: list = field(default_factory=list)
    Psi: list = field(default_factory=list)
    Phi: list = field(default_factory=list)
    K: np.ndarray = field(default=None)
    system_residual: float = 0.0


def incident_amplitudes(img, pol, sx, sy, sz_top, u, v):
    """p_bar [3][M] from the incident image (reading R11): the image is one
    transverse component, the other is zero, p_z follows from Gauss (Eq. 14)."""
    M = len(sx)
    p = np.zeros((3, M), dtype=np.complex128)
    proj = project_image(img, u, v)
    if pol == "x":
        p[0] = proj
    elif pol == "y":
        p[1] = proj
    else:
        raise ValueError(pol)
    num = sx * p[0] + sy * p[1]
    grazing = sz_top == 0
    if np.any(np.abs(num[grazing]) > 0):
        raise ValueError("incident light in a grazing order (s_z = 0) has no p_z")
    p[2] = np.where(grazing, 0.0, -num / np.where(grazing, 1.0, sz_top))
    return p


def layer_operators(n_layer: np.ndarray, sx, sy, u, v):
    """Phi, Psi (Sec. 2.4-2.5.2) and D (Eq. 21) of one layer."""
    eps = n_layer.astype(np.complex128) ** 2
    Phi = convolution_matrix(fourier_table(eps), u, v)
    Psi = convolution_matrix(fourier_table(1.0 / eps), u, v)
    return Phi, Psi, property_matrix(sx, sy, Phi, Psi)


def e_rows(Q, Psi, sx, sy) -> np.ndarray:
    """W = [Q_Px; Q_Py; Psi (diag(sy) Q_Bx - diag(sx) Q_By)] (Eq. 33, reading R5),
    the E-field rows precomputed per layer (Sec. 4.1)."""
    M = len(sx)
    qpz = Psi @ (sy[:, None] * Q[2 * M:3 * M] - sx[:, None] * Q[3 * M:4 * M])
    return np.concatenate([Q[:M], Q[M:2 * M], qpz], axis=0)


def solve(n_volume: np.ndarray, z_bounds, lam: float, X: float, Y: float, U: int, V: int,
          incident_image: np.ndarray, pol: str = "x", n_top: float = 1.0, n_bot: complex = 1.0,
          z_inc: float | None = None) -> Solution:
    """Forward simulation by the connection equations (Sec. 2.5.1 steps 1-4).

    1. D per layer (Eq. 21) and its eigenmodes (Sec. 2.5.3);
    2. K = B_L T_L^-1 ... B_1 T_1^-1 (Eq. 27, reading R6), via LU solves;
    3. the 6M system (Fig. 2, Eq. 29 plus Gauss Eq. 14) for P_ref, P_trn;
    4. alpha_1 = T_1^-1 (G_bar R_bar + R_ref), alpha_l = T_l^-1 B_{l-1} alpha_{l-1}
       (Sec. 2.5.4, Sec. 2.6.2);
    5. the E-field rows W per layer (Eq. 33).
    """
    z_bounds = np.asarray(z_bounds, dtype=np.float64)
    L = len(z_bounds) - 1
    assert n_volume.shape[0] == L
    M = U * V
    k = 2 * np.pi / lam
    u, v = orders(U, V)
    sx, sy = directions(U, V, lam, X, Y)
    sz_t = s_z(n_top, sx, sy)
    sz_b = s_z(n_bot, sx, sy)
    zbar = float(z_bounds[0]) if z_inc is None else float(z_inc)

    gam, Qs, Ts, Bs, Psis, Phis, Ws = [], [], [], [], [], [], []
    K = np.eye(4 * M, dtype=np.complex128)
    for l in range(L):
        Phi, Psi, D = layer_operators(n_volume[l], sx, sy, u, v)
        g, Q = layer_modes(D)
        T, B = top_bottom(g, Q, z_bounds[l + 1] - z_bounds[l], k)
        K = B @ np.linalg.solve(T, K)
        gam.append(g); Qs.append(Q); Ts.append(T); Bs.append(B)
        Psis.append(Psi); Phis.append(Phi); Ws.append(e_rows(Q, Psi, sx, sy))

    p_inc = incident_amplitudes(incident_image, pol, sx, sy, sz_t, u, v)
    Gbar = np.tile(np.exp(1j * k * sz_t * (z_bounds[0] - zbar)), 4)
    Rbar = Gbar * (p_to_r(sx, sy, sz_t) @ p_inc.ravel())
    Cref = p_to_r(sx, sy, -sz_t)
    Ctrn = p_to_r(sx, sy, sz_b)

    A = np.zeros((6 * M, 6 * M), dtype=np.complex128)
    rhs = np.zeros(6 * M, dtype=np.complex128)
    A[:4 * M, :3 * M] = -K @ Cref
    A[:4 * M, 3 * M:] = Ctrn
    rhs[:4 * M] = K @ Rbar
    r = 4 * M
    A[r:r + M, 0:M] = np.diag(sx)
    A[r:r + M, M:2 * M] = np.diag(sy)
    A[r:r + M, 2 * M:3 * M] = np.diag(-sz_t)
    r = 5 * M
    A[r:r + M, 3 * M:4 * M] = np.diag(sx)
    A[r:r + M, 4 * M:5 * M] = np.diag(sy)
    A[r:r + M, 5 * M:6 * M] = np.diag(sz_b)
    x = np.linalg.solve(A, rhs)
    res = np.linalg.norm(A @ x - rhs) / max(np.linalg.norm(rhs), 1e-300)
    p_ref = x[:3 * M].reshape(3, M)
    p_trn = x[3 * M:].reshape(3, M)

    alphas = []
    a = np.linalg.solve(Ts[0], Rbar + Cref @ p_ref.ravel())
    alphas.append(a)
    for l in range(1, L):
        a = np.linalg.solve(Ts[l], Bs[l - 1] @ a)
        alphas.append(a)

    return Solution(lam=lam, X=X, Y=Y, U=U, V=V, z_bounds=z_bounds,
                    W=np.stack(Ws), gamma=np.stack(gam), alpha=np.stack(alphas),
                    p_inc=p_inc, p_ref=p_ref, p_trn=p_trn, n_top=n_top, n_bot=n_bot,
                    z_inc=z_inc, sx=sx, sy=sy, Q=Qs, T=Ts, Bm=Bs, Psi=Psis, Phi=Phis,
                    K=K, system_residual=float(res))


def solve_problem(p) -> Solution:
    """solve() on a workloads.Problem."""
    return solve(p.n_volume, p.z_bounds, p.lam, p.X, p.Y, p.U, p.V, p.incident_image,
                 p.pol, p.n_top, p.n_bot, p.z_inc)


def solve_block_system(sol: Solution):
    """Brute force: the full banded system the connection equations reduce
    (Sec. 5, 'reduce the dimensionality ... by a factor of L').

    Unknowns [P_ref (3M), P_trn (3M), alpha_1 .. alpha_L (4M each)]; equations
    Eq. 24 (top), Eq. 25 (each interface), Eq. 26 (bottom) and Gauss (Eq. 14)
    for the two exterior waves. Returns (p_ref, p_trn, alphas).
    """
    M, L = sol.M, sol.L
    k = 2 * np.pi / sol.lam
    sx, sy = sol.sx, sol.sy
    sz_t = s_z(sol.n_top, sx, sy)
    sz_b = s_z(sol.n_bot, sx, sy)
    Gbar = np.tile(np.exp(1j * k * sz_t * (sol.z_bounds[0] - sol.zbar)), 4)
    Rbar = Gbar * (p_to_r(sx, sy, sz_t) @ sol.p_inc.ravel())
    n = 6 * M + 4 * M * L
    A = np.zeros((n, n), dtype=np.complex128)
    b = np.zeros(n, dtype=np.complex128)
    ai = lambda l: 6 * M + 4 * M * l  # column offset of alpha_l (0-based l)
    r = 0
    A[r:r + 4 * M, ai(0):ai(0) + 4 * M] = sol.T[0]
    A[r:r + 4 * M, 0:3 * M] = -p_to_r(sx, sy, -sz_t)
    b[r:r + 4 * M] = Rbar
    r += 4 * M
    for l in range(L - 1):
        A[r:r + 4 * M, ai(l):ai(l) + 4 * M] = sol.Bm[l]
        A[r:r + 4 * M, ai(l + 1):ai(l + 1) + 4 * M] = -sol.T[l + 1]
        r += 4 * M
    A[r:r + 4 * M, ai(L - 1):ai(L - 1) + 4 * M] = sol.Bm[L - 1]
    A[r:r + 4 * M, 3 * M:6 * M] = -p_to_r(sx, sy, sz_b)
    r += 4 * M
    A[r:r + M, 0:M] = np.diag(sx)
    A[r:r + M, M:2 * M] = np.diag(sy)
    A[r:r + M, 2 * M:3 * M] = np.diag(-sz_t)
    r += M
    A[r:r + M, 3 * M:4 * M] = np.diag(sx)
    A[r:r + M, 4 * M:5 * M] = np.diag(sy)
    A[r:r + M, 5 * M:6 * M] = np.diag(sz_b)
    x = np.linalg.solve(A, b)
    alphas = np.stack([x[ai(l):ai(l) + 4 * M] for l in range(L)])
    return x[:3 * M].reshape(3, M), x[3 * M:6 * M].reshape(3, M), alphas
