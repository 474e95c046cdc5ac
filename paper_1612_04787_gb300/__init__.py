"""GB300-native SWiFT-IR block matching ("swim", Sec. III of Wetzel et al.).

Thin Python binding over the C ABI in ``include/swift.h``: it only marshals
torch tensors' device pointers, sizes and the current CUDA stream into the
library's structs.  Every step of the matching runs in the library's CUDA
kernels; there is no CPU path, and importing this package fails if the built
library is missing.

    plan = Plan([Level(256, whiten_exponent=0.65)], dtype="u8")
    res = plan.match(ref_section, mov_section, ref_origin, mov_origin)  # [B, 8] int32 on device
    fields = decode(res)  # dy, dx, sy, sx, snr, peak, status as numpy arrays
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (APOD, DTYPE, PRECISION, SwiftBatch, SwiftImage, SwiftLevel, SwiftMesh, SwiftError,  # noqa: F401
                   FIT_DEGENERATE, FIT_FALLBACK, FIT_OK, WIN_FLAT, WIN_NONFINITE, WIN_OK, WIN_OUT_OF_BOUNDS, WIN_TIMEOUT,
                   check,
                   lib)

__all__ = ["Level", "Plan", "decode", "SwiftError", "version", "match_warped", "WIN_OK", "WIN_OUT_OF_BOUNDS",
           "WIN_FLAT", "WIN_NONFINITE", "WIN_TIMEOUT", "Mesh", "correspondences", "fit_affine", "mesh_fit", "render", "render_records", "downsample", "zmodel",
           "FIT_OK", "FIT_FALLBACK", "FIT_DEGENERATE"]


def version() -> str:
    return lib.swift_version().decode()


@dataclass
class Level:
    """One matching configuration (Sec. III): window side, whitening exponent
    (0 = correlation, 1 = phase-only), cosine taper, SNR exclusion radius."""
    n: int
    whiten_exponent: float = 0.65
    apod: str = "hann"
    tukey_alpha: float = 1.0
    snr_exclusion_radius: float = 3.0

    def c(self) -> SwiftLevel:
        return SwiftLevel(int(self.n), float(self.whiten_exponent), APOD[self.apod],
                          float(self.tukey_alpha), float(self.snr_exclusion_radius))


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _image(t: torch.Tensor, want: torch.dtype, patch: bool) -> SwiftImage:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("images must be CUDA tensors")
    if t.dtype != want:
        raise TypeError(f"image dtype {t.dtype} does not match the plan's {want}")
    if t.stride(-1) != 1:
        raise ValueError("image rows must be contiguous")
    if patch:
        if t.dim() != 3:
            raise ValueError("patch mode takes [B, n, n] tensors")
        if not t.is_contiguous():
            raise ValueError("patch stacks must be contiguous")
        return SwiftImage(t.data_ptr(), t.shape[2], t.stride(0), t.shape[1], t.shape[2], 1)
    if t.dim() == 2:
        return SwiftImage(t.data_ptr(), t.stride(0), 0, t.shape[0], t.shape[1], 1)
    if t.dim() == 3:  # a stack of K sections averaged into one model image
        return SwiftImage(t.data_ptr(), t.stride(1), t.stride(0), t.shape[1], t.shape[2], t.shape[0])
    raise ValueError("section mode takes [H, W] or [K, H, W] tensors")


class Plan:
    """A matching plan: per-level tables on the current device."""

    def __init__(self, levels, dtype: str = "u8", precision: str = "fp32", max_windows: int = 1 << 22):
        if isinstance(levels, Level):
            levels = [levels]
        self.levels = list(levels)
        self.dtype = dtype
        self.torch_dtype = torch.uint8 if dtype == "u8" else torch.float32
        arr = (SwiftLevel * len(self.levels))(*[lv.c() for lv in self.levels])
        self._h = C.c_void_p()
        check(lib.swift_plan_create(arr, len(self.levels), DTYPE[dtype], PRECISION[precision],
                                    int(max_windows), C.byref(self._h)), "swift_plan_create")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.swift_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    def set_whitening(self, level: int, w: float):
        """Whitening exponent of one level for later calls."""
        check(lib.swift_plan_set_whitening(self._h, int(level), float(w)), "swift_plan_set_whitening")
        self.levels[level].whiten_exponent = float(w)

    def _batch(self, ref, mov, ref_origin, mov_origin, level, affine, level_offsets=None):
        patch = ref_origin is None and mov_origin is None
        refs = ref if isinstance(ref, (list, tuple)) else [ref]
        movs = mov if isinstance(mov, (list, tuple)) else [mov]
        if len(refs) != len(movs):
            raise ValueError("ref and mov need one image per level")
        nlv = len(self.levels)
        if len(refs) == 1 and nlv > 1:
            refs, movs = list(refs) * nlv, list(movs) * nlv  # one image serves every level
        if len(refs) != nlv:
            raise ValueError(f"the plan has {nlv} levels: give one image per level (or one for all)")
        if patch:
            B = refs[0].shape[0]
        else:
            for o in (ref_origin, mov_origin):
                if o.dtype != torch.int32 or not o.is_cuda or not o.is_contiguous() or o.dim() != 2 or o.shape[1] != 2:
                    raise ValueError("origins must be contiguous int32 [B, 2] CUDA tensors")
            B = ref_origin.shape[0]
            if mov_origin.shape[0] != B:
                raise ValueError("origin counts differ")
        if level is not None:
            if level.dtype != torch.int32 or not level.is_cuda or not level.is_contiguous() or level.numel() != B:
                raise ValueError("level must be a contiguous int32 [B] CUDA tensor")
        if affine is not None:
            if patch:
                raise ValueError("affine warps need section mode (origins)")
            if affine.dtype != torch.float32 or not affine.is_cuda or not affine.is_contiguous() \
                    or tuple(affine.shape) != (B, 6):
                raise ValueError("affine must be a contiguous float32 [B, 6] CUDA tensor")
        offs = None
        if level_offsets is not None:
            lo = [int(v) for v in level_offsets]
            if len(lo) != nlv + 1 or lo[0] != 0 or lo[-1] != B or any(b < a for a, b in zip(lo, lo[1:])):
                raise ValueError("level_offsets must be n_levels + 1 non-decreasing counts from 0 to B")
            offs = (C.c_int64 * len(lo))(*lo)
        nl = len(refs)
        ri = (SwiftImage * nl)(*[_image(t, self.torch_dtype, patch) for t in refs])
        mi = (SwiftImage * nl)(*[_image(t, self.torch_dtype, patch) for t in movs])
        bt = SwiftBatch(ri, mi,
                        None if patch else ref_origin.data_ptr(),
                        None if patch else mov_origin.data_ptr(),
                        None if level is None else level.data_ptr(),
                        int(B), 1 if patch else 0,
                        None if affine is None else affine.data_ptr(),
                        offs)
        return bt, (ri, mi, offs), B, refs[0].device

    def set_schedule(self, level: int, schedule: str):
        """Forward schedule of one level: "fused", "stream" or "default"."""
        check(lib.swift_plan_set_schedule(self._h, int(level), _lib.SCHEDULE[schedule]), "swift_plan_set_schedule")

    def autotune(self, ref, mov, ref_origin=None, mov_origin=None, level=None, out=None, stream=None,
                 level_offsets=None):
        """Time every schedule of every level on this batch, keep the fastest;
        returns the chosen schedule names per level."""
        bt, keep, B, dev = self._batch(ref, mov, ref_origin, mov_origin, level, None, level_offsets)
        if out is None:
            out = torch.empty((B, 8), dtype=torch.int32, device=dev)
        chosen = (C.c_int32 * len(self.levels))()
        check(lib.swift_plan_autotune(self._h, C.byref(bt), out.data_ptr(), _stream_ptr(stream), chosen),
              "swift_plan_autotune")
        names = {v: k for k, v in _lib.SCHEDULE.items()}
        return [names[int(c)] for c in chosen], out

    def capture(self, ref, mov, ref_origin=None, mov_origin=None, level=None, out=None, stream=None,
                level_offsets=None):
        """Capture one forward call into a CUDA graph (see replay)."""
        bt, keep, B, dev = self._batch(ref, mov, ref_origin, mov_origin, level, None, level_offsets)
        if out is None:
            out = torch.empty((B, 8), dtype=torch.int32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream()
        check(lib.swift_plan_capture(self._h, C.byref(bt), out.data_ptr(), _stream_ptr(stream)),
              "swift_plan_capture")
        return out

    KERNEL_SLOTS = ("stats", "rows", "cols", "irows", "final", "fused", "persistent")

    def set_test_stall(self, enable: bool):
        """Test hook: the row staging by asynchronous copies (aligned float32
        rows, uint8 tensor-map tiles) waits for bytes that never arrive, so its
        bounded wait runs out and those windows report status 4 (timeout)."""
        check(lib.swift_plan_set_test_stall(self._h, 1 if enable else 0), "swift_plan_set_test_stall")

    def set_skew(self, skew: int):
        """Skew (1..16) of the persistent schedule's work order."""
        check(lib.swift_plan_set_skew(self._h, int(skew)), "swift_plan_set_skew")

    def set_lanes(self, lanes: int):
        """Lanes (1 or 2) that the plan's forward calls spread their
        launches over: the call's stream and one auxiliary stream."""
        check(lib.swift_plan_set_lanes(self._h, int(lanes)), "swift_plan_set_lanes")

    @property
    def lanes(self) -> int:
        v = C.c_int32(0)
        check(lib.swift_plan_get_lanes(self._h, C.byref(v)), "swift_plan_get_lanes")
        return int(v.value)

    def set_row_tma(self, mode: int):
        """How the streaming row kernel loads uint8 section windows: 0 plain
        loads only, 1 (default) tensor-map tile copies for windows whose rows
        start off a 16-byte boundary, 2 tensor-map copies for every window."""
        check(lib.swift_plan_set_row_tma(self._h, int(mode)), "swift_plan_set_row_tma")

    @property
    def row_tma(self) -> int:
        v = C.c_int32(0)
        check(lib.swift_plan_get_row_tma(self._h, C.byref(v)), "swift_plan_get_row_tma")
        return int(v.value)

    def set_test_hold(self, window: int):
        """Test hook: the row items of ``window`` (its position in the
        persistent launch's window sequence) never report completion and the
        launch's waits give up after about 10 ms; -1 turns it off."""
        check(lib.swift_plan_set_test_hold(self._h, int(window)), "swift_plan_set_test_hold")

    def set_test_stale_status(self, enable: bool):
        """Test hook: the statistics kernel reports windows of other levels as
        OK without reading them; the row kernels' own guard must skip them."""
        check(lib.swift_plan_set_test_stale_status(self._h, 1 if enable else 0),
              "swift_plan_set_test_stale_status")

    def set_timing(self, enable: bool):
        """Record CUDA events around every kernel of later forward calls."""
        check(lib.swift_plan_set_timing(self._h, 1 if enable else 0), "swift_plan_set_timing")

    def timings(self) -> dict:
        """{kernel: (total ms, launches)} since the last read (synchronises)."""
        ms = (C.c_float * 8)()
        n = (C.c_int32 * 8)()
        check(lib.swift_plan_timings(self._h, ms, n), "swift_plan_timings")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNEL_SLOTS) if n[i] > 0}

    def replay(self, stream=None):
        """Re-run the captured forward call with one graph launch."""
        check(lib.swift_plan_replay(self._h, _stream_ptr(stream)), "swift_plan_replay")

    def backward(self, ref, mov, ref_origin, mov_origin, grad_peak, grad_snr, affine=None, level=None,
                 stream=None):
        """Gradients of sum(grad_peak * peak + grad_snr * snr) with respect to
        the affine warps ([B, 6]) and the levels' whitening exponents
        ([n_levels]); the peak positions are held fixed."""
        bt, keep, B, dev = self._batch(ref, mov, ref_origin, mov_origin, level, affine)
        gp = grad_peak.to(device=dev, dtype=torch.float32).contiguous()
        gs = grad_snr.to(device=dev, dtype=torch.float32).contiguous()
        if gp.numel() != B or gs.numel() != B:
            raise ValueError("grad_peak and grad_snr need one value per window")
        g_aff = torch.zeros((B, 6), dtype=torch.float32, device=dev)
        g_w = torch.zeros((len(self.levels),), dtype=torch.float32, device=dev)
        check(lib.swift_match_backward(self._h, C.byref(bt), gp.data_ptr(), gs.data_ptr(), g_aff.data_ptr(),
                                       g_w.data_ptr(), _stream_ptr(stream)), "swift_match_backward")
        return g_aff, g_w

    def match(self, ref, mov, ref_origin=None, mov_origin=None, level=None, out=None, stream=None, affine=None,
              level_offsets=None):
        """Forward match; returns ``out`` ([B, 8] int32 device tensor of results).

        Section mode: ``ref`` / ``mov`` are [H, W] uint8/float32 images (``ref``
        may be [K, H, W]: the reference window is then the mean of K
        sections) or lists with one image per level, and the origins are
        int32 [B, 2] (y, x) device tensors.  Patch mode (no origins): ``ref``
        and ``mov`` are [B, n, n] stacks.  ``affine`` ([B, 6] float32, section
        mode) resamples each moving window bilinearly under its warp.
        ``level_offsets`` (n_levels + 1 ints): the windows are sorted by
        level, level l's being [level_offsets[l], level_offsets[l + 1]); each
        level's launches then cover only its own windows.
        """
        bt, keep, B, dev = self._batch(ref, mov, ref_origin, mov_origin, level, affine, level_offsets)
        if out is None:
            out = torch.empty((B, 8), dtype=torch.int32, device=dev)
        elif out.dtype != torch.int32 or out.shape != (B, 8) or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 [B, 8] tensor")
        check(lib.swift_match_batch(self._h, C.byref(bt), out.data_ptr(), _stream_ptr(stream)),
              "swift_match_batch")
        return out


class _MatchFn(torch.autograd.Function):
    """(affine [B, 6], w [n_levels]) -> (peak [B], snr [B]); backward through
    the library's adjoint kernels (peak positions held fixed)."""

    @staticmethod
    def forward(ctx, affine, w, plan, ref, mov, ref_origin, mov_origin, level):
        for l, wl in enumerate(w.detach().cpu().tolist()):
            plan.set_whitening(l, wl)
        res = plan.match(ref, mov, ref_origin, mov_origin, level=level, affine=affine.detach().contiguous())
        f = res.view(torch.float32)
        peak = f[:, 5].clone()
        snr = f[:, 4].clone()
        ctx.plan = plan
        ctx.w_device = w.device
        ctx.args = (ref, mov, ref_origin, mov_origin, level)
        ctx.save_for_backward(affine)
        ctx.mark_non_differentiable(res)
        return peak, snr, res

    @staticmethod
    def backward(ctx, grad_peak, grad_snr, _grad_res):
        (affine,) = ctx.saved_tensors
        ref, mov, ro, mo, level = ctx.args
        B = affine.shape[0]
        gp = grad_peak if grad_peak is not None else torch.zeros(B, device=affine.device)
        gs = grad_snr if grad_snr is not None else torch.zeros(B, device=affine.device)
        g_aff, g_w = ctx.plan.backward(ref, mov, ro, mo, gp, gs, affine=affine.detach().contiguous(), level=level)
        return g_aff, g_w.to(ctx.w_device), None, None, None, None, None, None


def match_warped(plan: Plan, ref, mov, ref_origin, mov_origin, affine, w, level=None):
    """Differentiable match of affinely warped moving windows.

    ``affine``: [B, 6] float32 CUDA tensor (a_yy, a_yx, t_y, a_xy, a_xx, t_x);
    ``w``: [n_levels] float32 tensor of whitening exponents.  Returns
    (peak [B], snr [B], results [B, 8]); gradients flow to ``affine`` and
    ``w`` through the library's backward kernels.
    """
    return _MatchFn.apply(affine, w, plan, ref, mov, ref_origin, mov_origin, level)


def window_check(n: int, level: int, want_level: int, ref_origin, mov_origin, ref_shape, mov_shape) -> int:
    """The kernels' window guard on the host: 0 (readable), 1 (out of bounds)
    or -1 (a window of another level)."""
    ro = (C.c_int32 * 2)(*[int(v) for v in ref_origin])
    mo = (C.c_int32 * 2)(*[int(v) for v in mov_origin])
    return int(lib.swift_window_check(int(n), int(level), int(want_level), ro, mo, int(ref_shape[0]),
                                      int(ref_shape[1]), int(mov_shape[0]), int(mov_shape[1])))


def whitening_sweep(ref, mov, n: int, exponents, apod: str = "hann", tukey_alpha: float = 1.0,
                    snr_exclusion_radius: float = 3.0, stream=None):
    """Match every patch pair at every whitening exponent in one call.

    ``ref`` / ``mov``: [P, n, n] uint8 or float32 CUDA stacks.  One plan level
    per exponent (same window size), a batch of P * E windows whose level index
    selects the exponent (the pairs repeated E times on the device).  Returns
    a [E, P, 8] int32 result tensor (row e holds exponent ``exponents[e]``).
    """
    ws = [float(w) for w in exponents]
    P, E = int(ref.shape[0]), len(ws)
    dtype = "u8" if ref.dtype == torch.uint8 else "f32"
    plan = Plan([Level(n, w, apod, tukey_alpha, snr_exclusion_radius) for w in ws], dtype=dtype,
                max_windows=max(1, P * E))
    rr = ref.unsqueeze(0).expand(E, P, n, n).reshape(E * P, n, n).contiguous()
    mm = mov.unsqueeze(0).expand(E, P, n, n).reshape(E * P, n, n).contiguous()
    lvl = torch.arange(E, dtype=torch.int32, device=ref.device).repeat_interleave(P)
    out = plan.match([rr] * E, [mm] * E, level=lvl, stream=stream, level_offsets=[P * e for e in range(E + 1)])
    return out.view(E, P, 8)


def decode(res) -> dict:
    """Split a [B, 8] int32 result tensor into named numpy arrays."""
    a = res.detach().cpu().numpy() if isinstance(res, torch.Tensor) else np.asarray(res)
    a = np.ascontiguousarray(a, dtype=np.int32)
    f = a.view(np.float32)
    return {"dy": a[:, 0].copy(), "dx": a[:, 1].copy(), "sy": f[:, 2].copy(), "sx": f[:, 3].copy(),
            "snr": f[:, 4].copy(), "peak": f[:, 5].copy(), "status": a[:, 6].copy()}


# --------------------------------------------------------------------------- #
# rendering step (mir): least-squares affines, triangle mesh, texture mapping
# --------------------------------------------------------------------------- #
@dataclass
class Mesh:
    """ny x nx square cells of side ``cell`` (>= 8) from the output-frame
    corner (origin_y, origin_x); two triangles per cell (Sec. IV)."""
    origin_y: int
    origin_x: int
    cell: int
    ny: int
    nx: int

    @property
    def n_triangles(self) -> int:
        return 2 * self.ny * self.nx

    def c(self) -> SwiftMesh:
        return SwiftMesh(int(self.origin_y), int(self.origin_x), int(self.cell), int(self.ny), int(self.nx))


def _dev(t: torch.Tensor, dtype: torch.dtype, shape_tail, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [N, {', '.join(map(str, shape_tail))}]")
    return t


def correspondences(res, ref_origin, mov_origin, n: int, min_snr: float = 0.0, stream=None):
    """(q, p, w) from forward-match results: reference window centres, the
    matching moving-section points, and SNR weights (0 for failed windows)."""
    B = int(res.shape[0])
    dev = res.device
    q = torch.empty((B, 2), dtype=torch.float32, device=dev)
    p = torch.empty((B, 2), dtype=torch.float32, device=dev)
    w = torch.empty((B,), dtype=torch.float32, device=dev)
    check(lib.swift_correspondences(res.data_ptr(), ref_origin.data_ptr(), mov_origin.data_ptr(), B, int(n),
                                    float(min_snr), q.data_ptr(), p.data_ptr(), w.data_ptr(), _stream_ptr(stream)),
          "swift_correspondences")
    return q, p, w


def fit_affine(q, p, w, offsets=None, stream=None, update=None, status=None):
    """Weighted least-squares affines p ~ A q + t, one per group of points
    (``offsets`` int64 [G + 1], default one group).  Returns (theta [G, 6]
    float64, status [G] int32) on the device.  ``update``: a contiguous
    float64 [G, 6] device tensor of previous affines, overwritten in place
    where a group's fit is OK and kept where it is degenerate (returned as
    theta); ``status``: an int32 [G] device tensor to write into."""
    _dev(q, torch.float32, (2,), "q")
    _dev(p, torch.float32, (2,), "p")
    if w.shape[0] != q.shape[0] or p.shape[0] != q.shape[0]:
        raise ValueError("q, p and w must have the same length")
    if offsets is None:
        offsets = torch.tensor([0, q.shape[0]], dtype=torch.int64, device=q.device)
    G = int(offsets.shape[0]) - 1
    if update is not None:
        if update.dtype != torch.float64 or tuple(update.shape) != (G, 6) or not update.is_contiguous():
            raise ValueError("update must be a contiguous float64 [G, 6] tensor")
        theta = update
    else:
        theta = torch.empty((G, 6), dtype=torch.float64, device=q.device)
    if status is None:
        status = torch.empty((G,), dtype=torch.int32, device=q.device)
    elif status.dtype != torch.int32 or tuple(status.shape) != (G,) or not status.is_contiguous():
        raise ValueError("status must be a contiguous int32 [G] tensor")
    fn, name = ((lib.swift_fit_affine_update, "swift_fit_affine_update") if update is not None
                else (lib.swift_fit_affine, "swift_fit_affine"))
    check(fn(q.data_ptr(), p.data_ptr(), w.data_ptr(), offsets.data_ptr(), G, theta.data_ptr(), status.data_ptr(),
             _stream_ptr(stream)), name)
    return theta, status


def mesh_fit(q, p, w, mesh: Mesh, band: int, stream=None):
    """Per-triangle affines [2 ny nx, 6] (float64) and statuses, each fitted
    to the points within Chebyshev distance ``band`` of its triangle."""
    _dev(q, torch.float32, (2,), "q")
    _dev(p, torch.float32, (2,), "p")
    if w.shape[0] != q.shape[0] or p.shape[0] != q.shape[0]:
        raise ValueError("q, p and w must have the same length")
    theta = torch.empty((mesh.n_triangles, 6), dtype=torch.float64, device=q.device)
    status = torch.empty((mesh.n_triangles,), dtype=torch.int32, device=q.device)
    mc = mesh.c()
    check(lib.swift_mesh_fit(q.data_ptr(), p.data_ptr(), w.data_ptr(), q.shape[0], C.byref(mc), int(band),
                             theta.data_ptr(), status.data_ptr(), _stream_ptr(stream)), "swift_mesh_fit")
    return theta, status


def render_records(theta, mesh: Mesh, records=None, stream=None):
    """Per-triangle render records (FP64 work done once per mesh)."""
    if theta.dtype != torch.float64 or tuple(theta.shape) != (mesh.n_triangles, 6) or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous float64 [2 ny nx, 6] tensor")
    if records is None:
        records = torch.empty((mesh.n_triangles, 8), dtype=torch.float32, device=theta.device)
    mc = mesh.c()
    check(lib.swift_render_prepare(theta.data_ptr(), C.byref(mc), records.data_ptr(), _stream_ptr(stream)),
          "swift_render_prepare")
    return records


def render(src, theta, mesh: Mesh, out_h: int, out_w: int, fill: float = 0.0, out=None, records=None,
           stream=None):
    """Texture-map ``src`` ([H, W] uint8 / float32 CUDA tensor) through the
    mesh's triangle affines into a float32 [out_h, out_w] image (or into
    ``out``: float32, or uint8 for values rounded half to even and clamped).
    ``records`` (from ``render_records``) skips the per-mesh preparation."""
    if src.dtype not in (torch.uint8, torch.float32) or src.dim() != 2:
        raise TypeError("src must be a [H, W] uint8 or float32 CUDA tensor")
    img = _image(src, src.dtype, False)
    if records is None:
        records = render_records(theta, mesh, stream=stream)
    if out is None:
        out = torch.empty((out_h, out_w), dtype=torch.float32, device=src.device)
    elif out.dtype not in (torch.float32, torch.uint8) or out.dim() != 2 or out.shape[0] < out_h or \
            out.shape[1] < out_w or out.stride(1) != 1:
        raise ValueError("out must be a float32 or uint8 [>= out_h, >= out_w] tensor with contiguous rows")
    mc = mesh.c()
    check(lib.swift_render(C.byref(img), DTYPE["u8" if src.dtype == torch.uint8 else "f32"], records.data_ptr(),
                           C.byref(mc), out.data_ptr(), DTYPE["u8" if out.dtype == torch.uint8 else "f32"],
                           int(out_h), int(out_w), out.stride(0), float(fill), _stream_ptr(stream)), "swift_render")
    return out


# --------------------------------------------------------------------------- #
# pyramid (iscale) and Z-model (remod)
# --------------------------------------------------------------------------- #
def downsample(img, factor: int, out=None, stream=None):
    """f x f box-mean downsampling of a [H, W] (or a batch [N, H, W]) uint8 /
    float32 CUDA image (uint8: exact mean rounded half to even).  Returns
    [H // f, W // f] (or [N, H // f, W // f])."""
    if img.dtype not in (torch.uint8, torch.float32) or img.dim() not in (2, 3) or not img.is_cuda:
        raise TypeError("img must be a [H, W] or [N, H, W] uint8 or float32 CUDA tensor")
    if img.stride(-1) != 1:
        raise ValueError("image rows must be contiguous")
    batch = img.dim() == 3
    N = img.shape[0] if batch else 1
    H, W = img.shape[-2] // factor, img.shape[-1] // factor
    shape = (N, H, W) if batch else (H, W)
    if out is None:
        out = torch.empty(shape, dtype=img.dtype, device=img.device)
    elif out.dtype != img.dtype or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError("out must be a contiguous tensor of the downsampled size and type")
    im = SwiftImage(img.data_ptr(), img.stride(-2), img.stride(0) if batch else 0, img.shape[-2], img.shape[-1], N)
    check(lib.swift_downsample(C.byref(im), DTYPE["u8" if img.dtype == torch.uint8 else "f32"], int(factor),
                               out.data_ptr(), W, _stream_ptr(stream)), "swift_downsample")
    return out


def zmodel(stack, k: int, valid=None, out=None, dtype=torch.float32, stream=None):
    """Z-averaged models ([Z, H, W], float32 or uint8) of a uint8 [Z, H, W]
    CUDA stack: the mean of the valid sections within +-k, the section itself
    excluded (uint8: the exact mean rounded half to even)."""
    if stack.dtype != torch.uint8 or stack.dim() != 3 or not stack.is_cuda or stack.stride(2) != 1:
        raise TypeError("stack must be a [Z, H, W] uint8 CUDA tensor with contiguous rows")
    Z, H, W = stack.shape
    if out is None:
        out = torch.empty((Z, H, W), dtype=dtype, device=stack.device)
    elif out.dtype not in (torch.float32, torch.uint8) or tuple(out.shape) != (Z, H, W) or out.stride(2) != 1:
        raise ValueError("out must be a float32 or uint8 [Z, H, W] tensor with contiguous rows")
    vptr = None
    if valid is not None:
        valid = valid.to(device=stack.device, dtype=torch.uint8).contiguous()
        if valid.numel() != Z:
            raise ValueError("valid must have one flag per section")
        vptr = valid.data_ptr()
    check(lib.swift_zmodel(stack.data_ptr(), stack.stride(0), Z, H, W, stack.stride(1), int(k), vptr,
                           out.data_ptr(), DTYPE["u8" if out.dtype == torch.uint8 else "f32"], out.stride(0),
                           out.stride(1), _stream_ptr(stream)), "swift_zmodel")
    return out
