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
from ._lib import (APOD, DTYPE, PRECISION, SwiftBatch, SwiftImage, SwiftLevel, SwiftError,  # noqa: F401
                   WIN_FLAT, WIN_NONFINITE, WIN_OK, WIN_OUT_OF_BOUNDS, check, lib)

__all__ = ["Level", "Plan", "decode", "SwiftError", "version", "WIN_OK", "WIN_OUT_OF_BOUNDS",
           "WIN_FLAT", "WIN_NONFINITE"]


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

    def match(self, ref, mov, ref_origin=None, mov_origin=None, level=None, out=None, stream=None):
        """Forward match; returns ``out`` ([B, 8] int32 device tensor of results).

        Section mode: ``ref`` / ``mov`` are [H, W] uint8/float32 images (``ref``
        may be [K, H, W]: the reference window is then the mean of K
        sections) or lists with one image per level, and the origins are
        int32 [B, 2] (y, x) device tensors.  Patch mode (no origins): ``ref``
        and ``mov`` are [B, n, n] stacks.
        """
        patch = ref_origin is None and mov_origin is None
        refs = ref if isinstance(ref, (list, tuple)) else [ref]
        movs = mov if isinstance(mov, (list, tuple)) else [mov]
        if len(refs) != len(movs):
            raise ValueError("ref and mov need one image per level")
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
        if out is None:
            out = torch.empty((B, 8), dtype=torch.int32, device=refs[0].device)
        elif out.dtype != torch.int32 or out.shape != (B, 8) or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 [B, 8] tensor")
        nl = len(refs)
        ri = (SwiftImage * nl)(*[_image(t, self.torch_dtype, patch) for t in refs])
        mi = (SwiftImage * nl)(*[_image(t, self.torch_dtype, patch) for t in movs])
        bt = SwiftBatch(ri, mi,
                        None if patch else ref_origin.data_ptr(),
                        None if patch else mov_origin.data_ptr(),
                        None if level is None else level.data_ptr(),
                        int(B), 1 if patch else 0)
        check(lib.swift_match_batch(self._h, C.byref(bt), out.data_ptr(), _stream_ptr(stream)),
              "swift_match_batch")
        return out


def decode(res) -> dict:
    """Split a [B, 8] int32 result tensor into named numpy arrays."""
    a = res.detach().cpu().numpy() if isinstance(res, torch.Tensor) else np.asarray(res)
    a = np.ascontiguousarray(a, dtype=np.int32)
    f = a.view(np.float32)
    return {"dy": a[:, 0].copy(), "dx": a[:, 1].copy(), "sy": f[:, 2].copy(), "sx": f[:, 3].copy(),
            "snr": f[:, 4].copy(), "peak": f[:, 5].copy(), "status": a[:, 6].copy()}
