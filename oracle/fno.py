"""Fourier-neural-operator surrogate in FP64 (TEST INFRASTRUCTURE; see oracle/__init__.py).

The surrogate is not part of the coupled-wave paper: it is the learned
shortcut that maps refractive-index slices to the exit-plane field, with the
coupled-wave solve as its fallback and its reference. Its network is the Fourier
neural operator of Li et al. (ICLR 2021), written out here from that
definition with numpy FFTs (the GPU side uses truncated DFT matrices; the two
share nothing).

Definition (all sums unnormalised unless stated; pixel (x, y) of an N x N
grid, x fastest; kept frequencies kx, ky in [-m/2, m/2), m = ``modes``):

  features   a[b, 2s]   = Re n[b, s] - 1,  a[b, 2s+1] = Im n[b, s]   (s < slices),
             nearest-upsampled from in_grid^2 to N^2 (factor N / in_grid).
  lift       V0 = P a + p                                   (1x1 convolution)
  layer l    Vh[b,i,k] = sum_x V_l[b,i,x] exp(-2 pi i k.x / N)          (k kept)
             Wh[b,o,k] = sum_i R_l[k,o,i] Vh[b,i,k]                      (complex)
             U[b,o,x]  = (1/N^2) Re sum_k Wh[b,o,k] exp(+2 pi i k.x / N)
             Z_l       = U + W_l V_l + c_l
             V_{l+1}   = GELU(Z_l) for l < layers-1, V_layers = Z_{layers-1}
  projection F = Q V_L + q            (6 channels: Re/Im of E_x, E_y, E_z)
  error head h[b] = e . mean_x V_L[b, :, x] + e0     (predicts log rel-L2)
  loss       rel2[b] = ||F_b - T_b||^2 / ||T_b||^2,  L_field = mean_b rel2[b]
             L_head  = mean_b (h[b] - log(rel2[b] + 1e-12) / 2)^2, with rel2
             and V_L held constant (the head does not train the trunk)
             L = L_field + L_head
  GELU(z) = z Phi(z) (exact, erf form).
  Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
             theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Flat parameter vector (float64 here, float32 on the GPU), in this order:
  P [width][2 slices], p [width], then per layer: R [m^2][width][width] as
  (re, im) pairs, W [width][width] (row = output channel), c [width]; then
  Q [6][width], q [6], e [width], e0 [1].

Parity status: pinned by tests/test_fno_oracle_pins.py (finite differences of
every parameter group, brute-force truncated DFT, low-pass special case,
translation equivariance, GELU values and symmetry, first Adam step).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import erf

OUT_CH = 6


@dataclass(frozen=True)
class FnoShape:
    width: int = 32
    grid: int = 64
    modes: int = 16
    layers: int = 4
    slices: int = 8
    in_grid: int = 32

    @property
    def in_ch(self) -> int:
        return 2 * self.slices

    @property
    def n_modes(self) -> int:
        return self.modes * self.modes


def param_layout(sh: FnoShape):
    """[(name, shape, complex?)] in flat order."""
    w = sh.width
    out = [("P", (w, sh.in_ch), False), ("p", (w,), False)]
    for l in range(sh.layers):
        out += [(f"R{l}", (sh.n_modes, w, w), True), (f"W{l}", (w, w), False), (f"c{l}", (w,), False)]
    out += [("Q", (OUT_CH, w), False), ("q", (OUT_CH,), False), ("e", (w,), False), ("e0", (1,), False)]
    return out


def param_count(sh: FnoShape) -> int:
    return sum(int(np.prod(s)) * (2 if c else 1) for _, s, c in param_layout(sh))


def unpack(flat, sh: FnoShape) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == param_count(sh)
    d, o = {}, 0
    for name, s, cplx in param_layout(sh):
        n = int(np.prod(s)) * (2 if cplx else 1)
        x = flat[o:o + n]
        o += n
        d[name] = (x[0::2] + 1j * x[1::2]).reshape(s) if cplx else x.reshape(s).copy()
    return d


def pack(d: dict, sh: FnoShape) -> np.ndarray:
    parts = []
    for name, s, cplx in param_layout(sh):
        x = np.asarray(d[name]).reshape(-1)
        if cplx:
            y = np.empty(2 * x.size)
            y[0::2], y[1::2] = x.real, x.imag
            x = y
        parts.append(np.asarray(x, dtype=np.float64))
    return np.concatenate(parts)


def kept_frequencies(sh: FnoShape):
    """(ky, kx) of the m^2 kept modes, mode index = (ky + m/2) m + (kx + m/2)."""
    k = np.arange(sh.modes) - sh.modes // 2
    return np.repeat(k, sh.modes), np.tile(k, sh.modes)


def features(n: np.ndarray, sh: FnoShape) -> np.ndarray:
    """a[B][2 slices][N][N] from n[B][slices][in_grid][in_grid] (complex)."""
    n = np.asarray(n, dtype=np.complex128)
    B = n.shape[0]
    f = np.empty((B, sh.in_ch, sh.in_grid, sh.in_grid))
    f[:, 0::2] = n.real - 1.0
    f[:, 1::2] = n.imag
    r = sh.grid // sh.in_grid
    return np.repeat(np.repeat(f, r, axis=2), r, axis=3)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def _gather(spec: np.ndarray, sh: FnoShape) -> np.ndarray:
    """Kept modes of an unshifted N x N spectrum (last two axes y, x) -> [..., m^2]."""
    ky, kx = kept_frequencies(sh)
    return spec[..., ky % sh.grid, kx % sh.grid]


def _scatter(coef: np.ndarray, sh: FnoShape) -> np.ndarray:
    """[..., m^2] -> full N x N spectrum with only the kept modes non-zero."""
    ky, kx = kept_frequencies(sh)
    full = np.zeros(coef.shape[:-1] + (sh.grid, sh.grid), dtype=np.complex128)
    full[..., ky % sh.grid, kx % sh.grid] = coef
    return full


def truncated_dft(v: np.ndarray, sh: FnoShape) -> np.ndarray:
    """Vh[..., k] = sum_x v[..., y, x] exp(-2 pi i (kx x + ky y)/N) on the kept modes."""
    return _gather(np.fft.fft2(v), sh)


def truncated_idft_re(coef: np.ndarray, sh: FnoShape) -> np.ndarray:
    """(1/N^2) Re sum_k coef[..., k] exp(+2 pi i (kx x + ky y)/N)."""
    return np.fft.ifft2(_scatter(coef, sh)).real


def spectral_conv(v: np.ndarray, R: np.ndarray, sh: FnoShape):
    """U = (1/N^2) Re IDFT(R Vh); returns (U, Vh)."""
    vh = truncated_dft(v, sh)                      # [B][i][k]
    wh = np.einsum("koi,bik->bok", R, vh)
    return truncated_idft_re(wh, sh), vh


def forward(flat, n, sh: FnoShape):
    """Field channels F[B][6][N][N], head h[B] and the values backward needs."""
    P = unpack(flat, sh)
    a = features(n, sh)
    V = np.einsum("oc,bcyx->boyx", P["P"], a) + P["p"][None, :, None, None]
    cache = {"a": a, "V": [V], "Z": [], "Vh": []}
    for l in range(sh.layers):
        U, vh = spectral_conv(V, P[f"R{l}"], sh)
        Z = U + np.einsum("oi,biyx->boyx", P[f"W{l}"], V) + P[f"c{l}"][None, :, None, None]
        V = gelu(Z) if l < sh.layers - 1 else Z
        cache["Z"].append(Z)
        cache["Vh"].append(vh)
        cache["V"].append(V)
    F = np.einsum("jo,boyx->bjyx", P["Q"], V) + P["q"][None, :, None, None]
    pool = V.mean(axis=(2, 3))
    h = pool @ P["e"] + P["e0"][0]
    cache["pool"] = pool
    return F, h, cache


def field_from_channels(F: np.ndarray) -> np.ndarray:
    """complex field [B][3][N][N] from the 6 real channels."""
    return F[:, 0::2] + 1j * F[:, 1::2]


def channels_from_field(E: np.ndarray) -> np.ndarray:
    E = np.asarray(E)
    F = np.empty((E.shape[0], OUT_CH) + E.shape[2:])
    F[:, 0::2], F[:, 1::2] = E.real, E.imag
    return F


def loss(flat, n, target_F, sh: FnoShape):
    """(L, L_field, L_head, rel2[B], h[B])."""
    F, h, _ = forward(flat, n, sh)
    T = np.asarray(target_F, dtype=np.float64)
    rel2 = ((F - T) ** 2).sum(axis=(1, 2, 3)) / (T ** 2).sum(axis=(1, 2, 3))
    Lf = rel2.mean()
    Lh = ((h - 0.5 * np.log(rel2 + 1e-12)) ** 2).mean()
    return Lf + Lh, Lf, Lh, rel2, h


def loss_and_grads(flat, n, target_F, sh: FnoShape):
    """Loss and its gradient w.r.t. the flat parameter vector (hand-derived backward)."""
    P = unpack(flat, sh)
    F, h, c = forward(flat, n, sh)
    T = np.asarray(target_F, dtype=np.float64)
    B = F.shape[0]
    tn = (T ** 2).sum(axis=(1, 2, 3))
    rel2 = ((F - T) ** 2).sum(axis=(1, 2, 3)) / tn
    Lf = rel2.mean()
    tgt = 0.5 * np.log(rel2 + 1e-12)
    Lh = ((h - tgt) ** 2).mean()
    g = {}
    # head (trunk held constant)
    dh = 2.0 * (h - tgt) / B
    g["e"] = c["pool"].T @ dh
    g["e0"] = np.array([dh.sum()])
    # projection
    dF = 2.0 * (F - T) / (B * tn[:, None, None, None])
    VL = c["V"][-1]
    g["Q"] = np.einsum("bjyx,boyx->jo", dF, VL)
    g["q"] = dF.sum(axis=(0, 2, 3))
    dV = np.einsum("jo,bjyx->boyx", P["Q"], dF)
    N2 = sh.grid * sh.grid
    for l in reversed(range(sh.layers)):
        Z, V, vh = c["Z"][l], c["V"][l], c["Vh"][l]
        dZ = dV * gelu_grad(Z) if l < sh.layers - 1 else dV
        g[f"c{l}"] = dZ.sum(axis=(0, 2, 3))
        g[f"W{l}"] = np.einsum("boyx,biyx->oi", dZ, V)
        # U = (1/N^2) Re sum Wh e^{+i theta}: dL/dRe Wh + i dL/dIm Wh = (1/N^2) sum_x dZ e^{-i theta}
        gWh = truncated_dft(dZ, sh) / N2
        R = P[f"R{l}"]
        # Wh = R Vh (complex-linear): G_R = G_Wh conj(Vh), G_Vh = conj(R)^T G_Wh
        gR = np.einsum("bok,bik->koi", gWh, np.conj(vh))
        g[f"R{l}"] = gR
        gVh = np.einsum("koi,bok->bik", np.conj(R), gWh)
        # Vh = sum_x V e^{-i theta} with V real: dL/dV = Re sum_k G_Vh e^{+i theta}
        dV = N2 * truncated_idft_re(gVh, sh) + np.einsum("oi,boyx->biyx", P[f"W{l}"], dZ)
    g["P"] = np.einsum("boyx,bcyx->oc", dV, c["a"])
    g["p"] = dV.sum(axis=(0, 2, 3))
    return Lf + Lh, Lf, Lh, pack(g, sh)


def adam_step(flat, grad, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def infer(flat, n, sh: FnoShape, q_cal: float = 0.0, threshold: float = 5e-2):
    """(complex field [B][3][N][N], estimated rel-L2 [B], fallback flags [B])."""
    F, h, _ = forward(flat, n, sh)
    est = np.exp(h + q_cal)
    return field_from_channels(F), est, est > threshold


def conformal_offset(h: np.ndarray, true_rel: np.ndarray, miss: float) -> float:
    """Split-conformal offset q: the ceil((1-miss)(n+1))-th smallest residual
    log(true_rel) - h over the calibration set, so that exp(h + q) bounds the
    true error with probability >= 1 - miss on exchangeable samples."""
    r = np.sort(np.log(np.asarray(true_rel)) - np.asarray(h))
    k = int(np.ceil((1.0 - miss) * (len(r) + 1))) - 1
    return float(r[min(max(k, 0), len(r) - 1)])
