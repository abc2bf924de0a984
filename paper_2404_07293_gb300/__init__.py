"""GB300-native volumetric field synthesis for the coupled-wave method of
arXiv 2404.07293 (sCWatter): thin Python binding over libscw (include/scw.h,
include/scw_fno.h for the learned surrogate).

Every step of the hot path runs in the library's CUDA kernels; this module
only checks tensor shapes/dtypes and passes pointers and the current torch
stream. PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (FLAG_AUTOTUNE, FLAG_DEBUG_BOUNDS, FLAG_EXTERIOR, FLAG_HOST_IO, FNO_PRECISION, PRECISION, ScwDesc, ScwError,
                   ScwFnoDesc, ScwFnoTimes, ScwKernelTimes, ScwPlanInfo, ScwSolveDesc, ScwSolveTimes, check, load)

__all__ = ["Plan", "BatchedPlan", "Solver", "Surrogate", "ScwError", "load", "PRECISION"]


def _make_desc(U, V, L, lam, X, Y, z_bounds, Fx, Fy, z_planes, x0=0.0, y0=0.0, n_top=1.0, n_bot=1.0,
               z_inc=None, precision="split_bf16", exterior=False, host_io=False, k_split=0, autotune=False,
               illuminations=1, pupil_na=0.0, tiles=(1, 1), out_ld=0, out_plane_stride=0, debug_bounds=False):
    """scw_desc for one item plus the host arrays it points to (keep them alive)."""
    zb = np.ascontiguousarray(z_bounds, dtype=np.float64)
    zp = np.ascontiguousarray(z_planes, dtype=np.float64)
    if len(zb) != int(L) + 1:
        raise ValueError("z_bounds must have L+1 entries")
    nb = complex(n_bot)
    flags = (FLAG_EXTERIOR if exterior else 0) | (FLAG_HOST_IO if host_io else 0) | (FLAG_AUTOTUNE if autotune else 0) \
        | (FLAG_DEBUG_BOUNDS if debug_bounds else 0)
    d = ScwDesc(U=int(U), V=int(V), L=int(L), lam=float(lam), X=float(X), Y=float(Y),
                z_bounds=zb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                Fx=int(Fx), Fy=int(Fy), Fz=len(zp),
                z_planes=zp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                x0=float(x0), y0=float(y0), n_top=float(n_top), n_bot_re=nb.real, n_bot_im=nb.imag,
                z_inc=float(zb[0] if z_inc is None else z_inc),
                precision=PRECISION[precision], flags=flags, k_split=int(k_split),
                illuminations=int(illuminations), pupil_na=float(pupil_na),
                tiles_x=int(tiles[0]), tiles_y=int(tiles[1]), out_ld=int(out_ld),
                out_plane_stride=int(out_plane_stride))
    return d, (zb, zp)


def _field_layout(I, Fz, Fy, Fx, tiles=(1, 1), out_ld=0, out_plane_stride=0):
    """Shape and element strides of a field [I][3][Fz][ty Fy][tx Fx] (I == 1: no leading axis)."""
    H, W = int(tiles[1]) * int(Fy), int(tiles[0]) * int(Fx)
    ld = int(out_ld) or W
    ps = int(out_plane_stride) or H * ld
    shape, strides = (3, Fz, H, W), (Fz * ps, ps, ld, 1)
    if I > 1:
        shape, strides = (I,) + shape, (3 * Fz * ps,) + strides
    return shape, strides


def _field_ptr(t, shape, strides, name):
    """Pointer of a complex64 CUDA field tensor, possibly a strided view (a patch of a mosaic)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64:
        raise TypeError(f"{name} must be a complex64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if any(n > 1 and a != b for n, a, b in zip(shape, t.stride(), strides)):
        raise ValueError(f"{name} must have element strides {tuple(strides)}, got {tuple(t.stride())}")
    return ctypes.c_void_p(t.data_ptr())


def _empty_field(shape, strides):
    import torch
    n = 1 + sum((s - 1) * st for s, st in zip(shape, strides))
    return torch.empty(n, dtype=torch.complex64, device="cuda").as_strided(shape, strides)


def _per_illum(I, shape):
    """Shape of an input given once per illumination (I > 1) or once (I == 1)."""
    return tuple(shape) if I == 1 else (I,) + tuple(shape)


TRACE_SLOTS = ("phases", "exterior", "contraction", "xpass", "ypass")
DEBUG_BUFFERS = ("s_part", "t", "twx", "twy", "b", "gamma", "alpha", "field", "c", "wt")


def _stream_handle(stream):
    import torch
    if stream is None and not torch.cuda.is_available():
        return ctypes.c_void_p(0)  # no device: the library call itself reports it (no CPU fallback)
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype, shape, name):
    a = np.asarray(a)
    if a.dtype != dtype or tuple(a.shape) != tuple(shape) or not a.flags.c_contiguous:
        raise ValueError(f"{name} must be a C-contiguous {np.dtype(dtype).name} array of shape {tuple(shape)}")
    return ctypes.c_void_p(a.ctypes.data)


class Plan:
    """One synthesis configuration (scw_plan) and its workspace."""

    def __init__(self, U, V, L, lam, X, Y, z_bounds, Fx, Fy, z_planes, x0=0.0, y0=0.0, n_top=1.0,
                 n_bot=1.0, z_inc=None, precision="split_bf16", exterior=False, host_io=False, k_split=0,
                 autotune=False, illuminations=1, pupil_na=0.0, tiles=(1, 1), out_ld=0, out_plane_stride=0,
                 stream=None, debug_bounds=False):
        """``illuminations`` incident fields share this solve: alpha becomes [I][L][4M], p_* [I][3][M]
        and the field [I][3][Fz][Fy][Fx]. ``pupil_na`` > 0 keeps only the orders inside that NA below
        the sample."""
        self._lib = load()
        self.U, self.V, self.L = int(U), int(V), int(L)
        self.M = self.U * self.V
        self.Fx, self.Fy = int(Fx), int(Fy)
        self.X, self.Y, self.x0, self.y0 = float(X), float(Y), float(x0), float(y0)
        self.n_points = 0
        self.I = max(1, int(illuminations))
        self.exterior = bool(exterior)
        d, (self._zb, self._zp) = _make_desc(U, V, L, lam, X, Y, z_bounds, Fx, Fy, z_planes, x0, y0, n_top, n_bot,
                                             z_inc, precision, exterior, host_io, k_split, autotune,
                                             illuminations, pupil_na, tiles, out_ld, out_plane_stride, debug_bounds)
        self.Fz = len(self._zp)
        self._layout = _field_layout(self.I, self.Fz, self.Fy, self.Fx, tiles, out_ld, out_plane_stride)
        h = ctypes.c_void_p()
        check(self._lib.scw_plan(ctypes.byref(d), _stream_handle(stream), ctypes.byref(h)), "scw_plan")
        self._h = h
        self._keep = ()

    # ------------------------------------------------------------------ inputs
    def set_layers(self, W, gamma, alpha, p_inc=None, p_ref=None, p_trn=None, stream=None):
        """W complex64 [L][3M][4M]; gamma complex128 [L][4M]; alpha complex128 [L][4M] ([I][L][4M]
        with I illuminations); p_* complex128 [3][M] ([I][3][M])."""
        import torch
        L, M, I = self.L, self.M, self.I
        args = [_dev_ptr(W, torch.complex64, (L, 3 * M, 4 * M), "W"),
                _dev_ptr(gamma, torch.complex128, (L, 4 * M), "gamma"),
                _dev_ptr(alpha, torch.complex128, _per_illum(I, (L, 4 * M)), "alpha")]
        for p, n in ((p_inc, "p_inc"), (p_ref, "p_ref"), (p_trn, "p_trn")):
            args.append(ctypes.c_void_p(0) if p is None else _dev_ptr(p, torch.complex128, _per_illum(I, (3, M)), n))
        check(self._lib.scw_plan_set_layers(self._h, *args, _stream_handle(stream)), "scw_plan_set_layers")
        self._keep = (W, gamma, alpha, p_inc, p_ref, p_trn)  # W until its conversion has run

    # ------------------------------------------------------------------ compute
    def out_shape(self):
        """[3][Fz][tiles_y Fy][tiles_x Fx] ([I][3]... with I illuminations)."""
        return self._layout[0]

    def out_strides(self):
        """Element strides the field must have (a custom out_ld / out_plane_stride makes it a strided view)."""
        return self._layout[1]

    def synthesize(self, out=None, stream=None):
        if out is None:
            out = _empty_field(*self._layout)
        check(self._lib.scw_synthesize(self._h, _field_ptr(out, *self._layout, "out"), _stream_handle(stream)),
              "scw_synthesize")
        return out

    def spectrum(self, S=None, stream=None):
        import torch
        shape = (self.I * self.Fz, 3, self.M)  # plane slot f I + illumination i
        if S is None:
            S = torch.empty(shape, dtype=torch.complex64, device="cuda")
        check(self._lib.scw_spectrum(self._h, _dev_ptr(S, torch.complex64, shape, "S"), _stream_handle(stream)),
              "scw_spectrum")
        return S

    def recompose(self, S, out=None, stream=None):
        import torch
        if out is None:
            out = _empty_field(*self._layout)
        check(self._lib.scw_recompose(self._h, _dev_ptr(S, torch.complex64, (self.I * self.Fz, 3, self.M), "S"),
                                      _field_ptr(out, *self._layout, "out"), _stream_handle(stream)),
              "scw_recompose")
        return out

    # ------------------------------------------------------------- point sets
    def set_points(self, xy, plane=None):
        """Lateral points (x, y) [P][2] at which synthesize_points evaluates the field on every z plane,
        or, with ``plane`` (int [P], indices into z_planes), scattered 3-D points: point p only at
        z_planes[plane[p]]."""
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
        check(self._lib.scw_plan_set_points(self._h, xy.ctypes.data_as(ctypes.c_void_p), int(xy.shape[0])),
              "scw_plan_set_points")
        self.n_points = int(xy.shape[0])
        self.point_planes = None
        if plane is not None:
            pl = np.ascontiguousarray(np.asarray(plane, dtype=np.int32).reshape(-1))
            if pl.shape[0] != self.n_points:
                raise ValueError("plane must have one entry per point")
            check(self._lib.scw_plan_set_point_planes(self._h, pl.ctypes.data_as(ctypes.c_void_p)),
                  "scw_plan_set_point_planes")
            self.point_planes = pl

    def set_xz_plane(self, y, n=None):
        """Points of the x-z plane at height y: x_i = x0 + i X / n (n = Fx by default)."""
        n = self.Fx if n is None else int(n)
        self.set_points(np.stack([self.x0 + np.arange(n) * self.X / n, np.full(n, float(y))], axis=1))

    def set_yz_plane(self, x, n=None):
        """Points of the y-z plane at x: y_j = y0 + j Y / n (n = Fy by default)."""
        n = self.Fy if n is None else int(n)
        self.set_points(np.stack([np.full(n, float(x)), self.y0 + np.arange(n) * self.Y / n], axis=1))

    def points_shape(self):
        if getattr(self, "point_planes", None) is not None:
            return _per_illum(self.I, (3, self.n_points))
        return _per_illum(self.I, (3, self.Fz, self.n_points))

    def synthesize_points(self, out=None, stream=None):
        """Field at the points of set_points on every z plane: [3][Fz][P] ([I][3][Fz][P])."""
        import torch
        if out is None:
            out = torch.empty(self.points_shape(), dtype=torch.complex64, device="cuda")
        check(self._lib.scw_synthesize_points(self._h, _dev_ptr(out, torch.complex64, self.points_shape(), "out"),
                                              _stream_handle(stream)), "scw_synthesize_points")
        return out

    def synthesize_host(self, W, gamma, alpha, p_inc=None, p_ref=None, p_trn=None, out=None, stream=None):
        """End to end through host memory (plan created with host_io=True)."""
        L, M, I = self.L, self.M, self.I
        if out is None:
            out = np.empty(self.out_shape(), dtype=np.complex64)
        args = [_host_ptr(W, np.complex64, (L, 3 * M, 4 * M), "W"),
                _host_ptr(gamma, np.complex128, (L, 4 * M), "gamma"),
                _host_ptr(alpha, np.complex128, _per_illum(I, (L, 4 * M)), "alpha")]
        for p, n in ((p_inc, "p_inc"), (p_ref, "p_ref"), (p_trn, "p_trn")):
            args.append(ctypes.c_void_p(0) if p is None else _host_ptr(p, np.complex128, _per_illum(I, (3, M)), n))
        args.append(_host_ptr(out, np.complex64, self.out_shape(), "out"))
        check(self._lib.scw_synthesize_host(self._h, *args, _stream_handle(stream)), "scw_synthesize_host")
        return out

    def check(self, stream=None):
        check(self._lib.scw_plan_check(self._h, _stream_handle(stream)), "scw_plan_check")

    def set_timeout_ns(self, ns):
        check(self._lib.scw_plan_set_timeout_ns(self._h, int(ns)), "scw_plan_set_timeout_ns")

    def inject_stall(self, on=True):
        """Failure injection: the next synthesis's contraction waits run out (see scw_plan_inject_stall)."""
        check(self._lib.scw_plan_inject_stall(self._h, 1 if on else 0), "scw_plan_inject_stall")

    def enable_timing(self, on=True):
        check(self._lib.scw_plan_enable_timing(self._h, 1 if on else 0), "scw_plan_enable_timing")

    def timings(self) -> dict:
        t = ScwKernelTimes()
        check(self._lib.scw_plan_get_timings(self._h, ctypes.byref(t)), "scw_plan_get_timings")
        return {f: getattr(t, f) for f, _ in ScwKernelTimes._fields_}

    def info(self) -> dict:
        i = ScwPlanInfo()
        check(self._lib.scw_plan_get_info(self._h, ctypes.byref(i)), "scw_plan_get_info")
        return {f: getattr(i, f) for f, _ in ScwPlanInfo._fields_}

    def debug_set_extent(self, buffer, elements=0):
        """SCW_FLAG_DEBUG_BOUNDS plans: lower the extent the index checks use for `buffer` (a name of
        DEBUG_BUFFERS or its index); 0 restores the real extent."""
        b = DEBUG_BUFFERS.index(buffer) if isinstance(buffer, str) else int(buffer)
        check(self._lib.scw_plan_debug_set_extent(self._h, b, int(elements)), "scw_plan_debug_set_extent")

    def enable_trace(self, on=True):
        check(self._lib.scw_plan_enable_trace(self._h, 1 if on else 0), "scw_plan_enable_trace")

    def trace(self) -> dict:
        """Kernel begin/end (us from the earliest begin) since the previous read, per step."""
        buf = (ctypes.c_double * (2 * len(TRACE_SLOTS)))()
        check(self._lib.scw_plan_get_trace(self._h, buf, len(TRACE_SLOTS)), "scw_plan_get_trace")
        return {name: (buf[2 * i], buf[2 * i + 1]) for i, name in enumerate(TRACE_SLOTS) if buf[2 * i + 1] >= 0}

    def tune_report(self) -> str:
        r = self._lib.scw_plan_tune_report(self._h)
        return r.decode() if r else ""

    def set_pipeline(self, groups: int):
        check(self._lib.scw_plan_set_pipeline(self._h, int(groups)), "scw_plan_set_pipeline")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.scw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """Many independent items (e.g. the wavenumbers of a sweep) synthesised by
    one set of kernels and replayed as one CUDA graph (scw_plan_batched).

    ``items`` is a list of keyword dicts with the arguments of ``Plan`` (without
    ``precision``/``host_io``)."""

    def __init__(self, items, precision="split_bf16", autotune=False, stream=None):
        self._lib = load()
        n = len(items)
        descs = (ScwDesc * n)()
        self._keep_desc = []
        self.shapes = []
        self.layouts = []
        self.sizes = []
        for i, kw in enumerate(items):
            kw = dict(kw)
            d, keep = _make_desc(precision=precision, autotune=autotune, **kw)
            descs[i] = d
            self._keep_desc.append(keep)
            M = int(kw["U"]) * int(kw["V"])
            I = max(1, int(kw.get("illuminations", 1)))
            self.sizes.append((int(kw["L"]), M, I))
            lay = _field_layout(I, len(keep[1]), kw["Fy"], kw["Fx"], kw.get("tiles", (1, 1)), kw.get("out_ld", 0),
                                kw.get("out_plane_stride", 0))
            self.shapes.append(lay[0])
            self.layouts.append(lay)
        h = ctypes.c_void_p()
        check(self._lib.scw_plan_batched(descs, n, _stream_handle(stream), ctypes.byref(h)), "scw_plan_batched")
        self._h = h
        self._keep = [()] * n

    def __len__(self):
        return len(self.shapes)

    def set_layers(self, i, W, gamma, alpha, p_inc=None, p_ref=None, p_trn=None, stream=None):
        import torch
        L, M, I = self.sizes[i]
        args = [_dev_ptr(W, torch.complex64, (L, 3 * M, 4 * M), "W"),
                _dev_ptr(gamma, torch.complex128, (L, 4 * M), "gamma"),
                _dev_ptr(alpha, torch.complex128, _per_illum(I, (L, 4 * M)), "alpha")]
        for p, nme in ((p_inc, "p_inc"), (p_ref, "p_ref"), (p_trn, "p_trn")):
            args.append(ctypes.c_void_p(0) if p is None else _dev_ptr(p, torch.complex128, _per_illum(I, (3, M)), nme))
        check(self._lib.scw_plan_batched_set_layers(self._h, int(i), *args, _stream_handle(stream)),
              "scw_plan_batched_set_layers")
        self._keep[i] = (W, gamma, alpha, p_inc, p_ref, p_trn)

    def synthesize(self, outs=None, stream=None):
        import torch
        if outs is None:
            outs = [_empty_field(*lay) for lay in self.layouts]
        if len(outs) != len(self.layouts):
            raise ValueError("one output per item")
        ptrs = (ctypes.c_void_p * len(outs))(*[_field_ptr(o, *lay, "out").value
                                              for o, lay in zip(outs, self.layouts)])
        check(self._lib.scw_synthesize_batched(self._h, None, ptrs, _stream_handle(stream)), "scw_synthesize_batched")
        return outs

    def item_table(self, outs):
        """DEVICE int64 [n] table of the outputs' addresses (validated here), for synthesize_table."""
        import torch
        if len(outs) != len(self.layouts):
            raise ValueError("one output per item")
        ptrs = [_field_ptr(o, *lay, "out").value for o, lay in zip(outs, self.layouts)]
        return torch.tensor(ptrs, dtype=torch.int64).to(outs[0].device)

    def synthesize_table(self, table, stream=None):
        """scw_synthesize_batched with a DEVICE item table (int64 [n] of field addresses)."""
        import torch
        if not (table.is_cuda and table.dtype == torch.int64 and table.is_contiguous() and
                table.numel() == len(self.layouts)):
            raise ValueError("table must be a contiguous CUDA int64 tensor with one address per item")
        check(self._lib.scw_synthesize_batched(self._h, ctypes.c_void_p(table.data_ptr()), None,
                                               _stream_handle(stream)), "scw_synthesize_batched")

    def check(self, stream=None):
        check(self._lib.scw_plan_check(self._h, _stream_handle(stream)), "scw_plan_check")

    def enable_timing(self, on=True):
        check(self._lib.scw_plan_enable_timing(self._h, 1 if on else 0), "scw_plan_enable_timing")

    def timings(self) -> dict:
        t = ScwKernelTimes()
        check(self._lib.scw_plan_get_timings(self._h, ctypes.byref(t)), "scw_plan_get_timings")
        return {f: getattr(t, f) for f, _ in ScwKernelTimes._fields_}

    def info(self) -> dict:
        i = ScwPlanInfo()
        check(self._lib.scw_plan_get_info(self._h, ctypes.byref(i)), "scw_plan_get_info")
        return {f: getattr(i, f) for f, _ in ScwPlanInfo._fields_}

    def tune_report(self) -> str:
        r = self._lib.scw_plan_tune_report(self._h)
        return r.decode() if r else ""

    def close(self):
        if getattr(self, "_h", None):
            self._lib.scw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """The coupled-wave solve stage on the GPU (scw_solver_*): a layered sample n [L][Ny][Nx]
    (complex128) and an incident field give W, gamma, alpha, p_ref, p_trn, the inputs of
    ``Plan.set_layers``."""

    def __init__(self, U, V, L, lam, X, Y, z_bounds, Nx, Ny, n_top=1.0, n_bot=1.0, z_inc=None):
        self._lib = load()
        self.U, self.V, self.L, self.M = int(U), int(V), int(L), int(U) * int(V)
        self.Nx, self.Ny = int(Nx), int(Ny)
        self._zb = np.ascontiguousarray(z_bounds, dtype=np.float64)
        if len(self._zb) != self.L + 1:
            raise ValueError("z_bounds must have L+1 entries")
        nb = complex(n_bot)
        d = ScwSolveDesc(U=self.U, V=self.V, L=self.L, lam=float(lam), X=float(X), Y=float(Y),
                         z_bounds=self._zb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), Nx=self.Nx, Ny=self.Ny,
                         n_top=float(n_top), n_bot_re=nb.real, n_bot_im=nb.imag,
                         z_inc=float(self._zb[0] if z_inc is None else z_inc))
        h = ctypes.c_void_p()
        check(self._lib.scw_solver_create(ctypes.byref(d), ctypes.byref(h)), "scw_solver_create")
        self._h = h

    def incident(self, image, pol="x", stream=None):
        """p_inc [3][M] (complex128, device) from a [Ny][Nx] complex128 image of the x or y component."""
        import torch
        p = torch.empty((3, self.M), dtype=torch.complex128, device="cuda")
        check(self._lib.scw_solver_incident(self._h, _dev_ptr(image, torch.complex128, (self.Ny, self.Nx), "image"),
                                            {"x": 0, "y": 1}[pol], _dev_ptr(p, torch.complex128, (3, self.M), "p_inc"),
                                            _stream_handle(stream)), "scw_solver_incident")
        return p

    def solve(self, n, p_inc, stream=None):
        """Returns (W [L][3M][4M] c64, gamma [L][4M] c128, alpha [L][4M] c128, p_ref, p_trn [3][M] c128)."""
        import torch
        L, M = self.L, self.M
        W = torch.empty((L, 3 * M, 4 * M), dtype=torch.complex64, device="cuda")
        g = torch.empty((L, 4 * M), dtype=torch.complex128, device="cuda")
        a = torch.empty((L, 4 * M), dtype=torch.complex128, device="cuda")
        pr = torch.empty((3, M), dtype=torch.complex128, device="cuda")
        pt = torch.empty((3, M), dtype=torch.complex128, device="cuda")
        check(self._lib.scw_solve(self._h, _dev_ptr(n, torch.complex128, (L, self.Ny, self.Nx), "n"),
                                  _dev_ptr(p_inc, torch.complex128, (3, M), "p_inc"), ctypes.c_void_p(W.data_ptr()),
                                  ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                  ctypes.c_void_p(pr.data_ptr()), ctypes.c_void_p(pt.data_ptr()),
                                  _stream_handle(stream)), "scw_solve")
        return W, g, a, pr, pt

    def times(self) -> dict:
        t = ScwSolveTimes()
        check(self._lib.scw_solver_get_times(self._h, ctypes.byref(t)), "scw_solver_get_times")
        return {f: getattr(t, f) for f, _ in ScwSolveTimes._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.scw_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The learned surrogate (scw_surrogate_*): a Fourier neural operator from
    refractive-index slices n [B][S][in][in] (complex64) to the exit-plane field
    [B][3][N][N] (complex64), trained and evaluated by the library's kernels."""

    def __init__(self, grid=64, modes=16, layers=4, slices=8, in_grid=32, batch_max=256, precision="bf16", seed=0,
                 width=32):
        self._lib = load()
        self.grid, self.modes, self.layers, self.slices, self.in_grid = grid, modes, layers, slices, in_grid
        self.batch_max = batch_max
        d = ScwFnoDesc(width=int(width), grid=int(grid), modes=int(modes), layers=int(layers), slices=int(slices),
                       in_grid=int(in_grid), batch_max=int(batch_max), precision=FNO_PRECISION[precision],
                       seed=int(seed))
        h = ctypes.c_void_p()
        check(self._lib.scw_surrogate_create(ctypes.byref(d), ctypes.byref(h)), "scw_surrogate_create")
        self._h = h
        n = ctypes.c_size_t()
        check(self._lib.scw_surrogate_param_count(self._h, ctypes.byref(n)), "scw_surrogate_param_count")
        self.n_params = n.value

    def _n_ptr(self, n, B):
        import torch
        return _dev_ptr(n, torch.complex64, (B, self.slices, self.in_grid, self.in_grid), "n")

    def _f_ptr(self, t, B, name):
        import torch
        return _dev_ptr(t, torch.complex64, (B, 3, self.grid, self.grid), name)

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        check(self._lib.scw_surrogate_set_params(self._h, _host_ptr(a, np.float32, (self.n_params,), "flat"),
                                                            self.n_params), "scw_surrogate_set_params")

    def params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        check(self._lib.scw_surrogate_get_params(self._h, ctypes.c_void_p(a.ctypes.data), self.n_params),
              "scw_surrogate_get_params")
        return a

    def grads(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        check(self._lib.scw_surrogate_get_grads(self._h, ctypes.c_void_p(a.ctypes.data), self.n_params),
              "scw_surrogate_get_grads")
        return a

    def forward_backward(self, n, target, read_loss=True, stream=None):
        B = n.shape[0]
        loss = np.zeros(3, dtype=np.float32)
        check(self._lib.scw_surrogate_forward_backward(
            self._h, self._n_ptr(n, B), self._f_ptr(target, B, "target"), B,
            ctypes.c_void_p(loss.ctypes.data) if read_loss else None, _stream_handle(stream)),
            "scw_surrogate_forward_backward")
        return loss if read_loss else None

    def train_step(self, n, target, lr=1e-3, read_loss=True, stream=None):
        B = n.shape[0]
        loss = np.zeros(3, dtype=np.float32)
        check(self._lib.scw_surrogate_train_step(
            self._h, self._n_ptr(n, B), self._f_ptr(target, B, "target"), B, float(lr),
            ctypes.c_void_p(loss.ctypes.data) if read_loss else None, _stream_handle(stream)),
            "scw_surrogate_train_step")
        return loss if read_loss else None

    def infer(self, n, threshold=5e-2, field=None, stream=None):
        """(field, est_err, need_fallback) as device tensors."""
        import torch
        B = n.shape[0]
        if field is None:
            field = torch.empty((B, 3, self.grid, self.grid), dtype=torch.complex64, device=n.device)
        est = torch.empty(B, dtype=torch.float32, device=n.device)
        flag = torch.empty(B, dtype=torch.uint8, device=n.device)
        check(self._lib.scw_surrogate_infer(
            self._h, self._n_ptr(n, B), B, self._f_ptr(field, B, "field"), ctypes.c_void_p(est.data_ptr()),
            ctypes.c_void_p(flag.data_ptr()), float(threshold), _stream_handle(stream)), "scw_surrogate_infer")
        return field, est, flag

    def calibrate(self, est, true_err, miss=0.01) -> float:
        e = np.ascontiguousarray(est, dtype=np.float32)
        t = np.ascontiguousarray(true_err, dtype=np.float32)
        if e.shape != t.shape or e.ndim != 1:
            raise ValueError("est and true_err must be 1-D arrays of one length")
        q = ctypes.c_float()
        check(self._lib.scw_surrogate_calibrate(self._h, ctypes.c_void_p(e.ctypes.data),
                                                           ctypes.c_void_p(t.ctypes.data), len(e), float(miss),
                                                           ctypes.byref(q)), "scw_surrogate_calibrate")
        return q.value

    def set_offset(self, q: float):
        check(self._lib.scw_surrogate_set_offset(self._h, float(q)), "scw_surrogate_set_offset")

    def state(self) -> np.ndarray:
        """The whole training state (parameters, Adam moments, step, calibration) as host bytes."""
        n = ctypes.c_size_t()
        check(self._lib.scw_surrogate_state_bytes(self._h, ctypes.byref(n)), "scw_surrogate_state_bytes")
        buf = np.empty(n.value, dtype=np.uint8)
        check(self._lib.scw_surrogate_save_state(self._h, ctypes.c_void_p(buf.ctypes.data), n.value),
              "scw_surrogate_save_state")
        return buf

    def load_state(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        check(self._lib.scw_surrogate_load_state(self._h, ctypes.c_void_p(b.ctypes.data), b.size),
              "scw_surrogate_load_state")

    def save(self, path):
        """torch.save of the training state as a host tensor."""
        import torch
        torch.save({"scw_surrogate_state": torch.from_numpy(self.state())}, path)

    def load(self, path):
        import torch
        self.load_state(torch.load(path)["scw_surrogate_state"].numpy())

    def enable_timing(self, on=True):
        check(self._lib.scw_surrogate_enable_timing(self._h, 1 if on else 0), "scw_surrogate_enable_timing")

    def timings(self) -> dict:
        t = ScwFnoTimes()
        check(self._lib.scw_surrogate_get_timings(self._h, ctypes.byref(t)), "scw_surrogate_get_timings")
        return {k: getattr(t, k) for k, _ in ScwFnoTimes._fields_}

    def launches(self) -> dict:
        a, b = ctypes.c_int(), ctypes.c_int()
        check(self._lib.scw_surrogate_launches(self._h, ctypes.byref(a), ctypes.byref(b)),
              "scw_surrogate_launches")
        return {"train_step": a.value, "infer": b.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.scw_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
