"""Shared test helpers: oracle LayerSets <-> device tensors, error metrics."""
import numpy as np

from oracle import cw


def layerset_from_arrays(lam, X, Y, U, V, z_bounds, W, gamma, alpha, p_inc, p_ref, p_trn,
                         n_top=1.0, n_bot=1.0, z_inc=None):
    return cw.LayerSet(lam=lam, X=X, Y=Y, U=U, V=V, z_bounds=np.asarray(z_bounds, float),
                       W=np.asarray(W).astype(np.complex128), gamma=np.asarray(gamma),
                       alpha=np.asarray(alpha), p_inc=np.asarray(p_inc), p_ref=np.asarray(p_ref),
                       p_trn=np.asarray(p_trn), n_top=n_top, n_bot=n_bot, z_inc=z_inc)


def to_device(ls, device="cuda"):
    import torch
    W = torch.from_numpy(np.ascontiguousarray(ls.W, dtype=np.complex64)).to(device)
    g = torch.from_numpy(np.ascontiguousarray(ls.gamma, dtype=np.complex128)).to(device)
    a = torch.from_numpy(np.ascontiguousarray(ls.alpha, dtype=np.complex128)).to(device)
    ps = [torch.from_numpy(np.ascontiguousarray(p, dtype=np.complex128)).to(device)
          for p in (ls.p_inc, ls.p_ref, ls.p_trn)]
    return W, g, a, ps


def rel_l2(a, b, axis_c=True):
    """Per-component relative L2 ||a_c - b_c|| / ||b_c|| for arrays [3][...]."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return [float(np.linalg.norm(a[c] - b[c]) / max(np.linalg.norm(b[c]), 1e-300)) for c in range(a.shape[0])]


def fno_init_groups(sh):
    """(size, scale) per flat parameter group of the surrogate, in flat order."""
    from oracle import fno
    out = []
    for name, shape, cplx in fno.param_layout(sh):
        n = int(np.prod(shape)) * (2 if cplx else 1)
        if name == "P":
            sc = 1.0 / np.sqrt(sh.in_ch)
        elif name.startswith("R"):
            sc = 1.0 / sh.width
        elif name.startswith("W") or name in ("Q", "e"):
            sc = 1.0 / np.sqrt(sh.width)
        else:
            sc = 0.1
        out.append((n, sc))
    return out


def max_abs(a, b):
    """Per-component max |a_c - b_c| over all voxels, and the same over max |b_c|."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ab = [float(np.abs(a[c] - b[c]).max()) for c in range(a.shape[0])]
    return ab, [x / max(float(np.abs(b[c]).max()), 1e-300) for c, x in enumerate(ab)]
