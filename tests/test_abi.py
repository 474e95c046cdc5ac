"""The C-ABI library loads and exports every entry point include/swift.h
declares; argument errors come back as status codes before any CUDA work
(so these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "swift.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(swift_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ("swift_plan_create", "swift_plan_destroy", "swift_match_batch", "swift_status_string"):
        assert name in fns


def test_library_exports_every_declared_symbol():
    from paper_1612_04787_gb300 import _lib
    lib = C.CDLL(_lib.LIB_PATH)
    for name in header_functions():
        assert hasattr(lib, name), f"{name} declared in swift.h but not exported"
    assert set(_lib.EXPORTS) == set(header_functions())


def test_status_strings_and_version():
    from paper_1612_04787_gb300 import _lib
    for code in range(7):
        assert _lib.lib.swift_status_string(code).decode().startswith("SWIFT_")
    assert b"sm_103a" in _lib.lib.swift_version()


def test_argument_errors_are_reported_before_any_launch():
    from paper_1612_04787_gb300 import _lib
    lib = _lib.lib
    h = C.c_void_p(1234)
    assert lib.swift_plan_create(None, 1, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    assert h.value is None  # *out cleared on failure
    lv = (_lib.SwiftLevel * 1)(_lib.SwiftLevel(100, 0.5, 1, 1.0, 3.0))  # not a power of two
    assert lib.swift_plan_create(lv, 1, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    lv = (_lib.SwiftLevel * 1)(_lib.SwiftLevel(64, 1.5, 1, 1.0, 3.0))  # exponent outside [0, 1]
    assert lib.swift_plan_create(lv, 1, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    lv = (_lib.SwiftLevel * 1)(_lib.SwiftLevel(64, 0.5, 2, 0.0, 3.0))  # tukey alpha 0
    assert lib.swift_plan_create(lv, 1, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    lv = (_lib.SwiftLevel * 1)(_lib.SwiftLevel(1024, 0.5, 1, 1.0, 3.0))  # size not built
    assert lib.swift_plan_create(lv, 1, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_UNSUPPORTED
    lv = (_lib.SwiftLevel * 1)(_lib.SwiftLevel(64, 0.5, 1, 1.0, 3.0))
    assert lib.swift_plan_create(lv, 0, 0, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_plan_create(lv, 1, 7, 0, 10, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_plan_create(lv, 1, 0, 0, 0, C.byref(h)) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_match_batch(None, None, None, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_plan_destroy(None) == _lib.SWIFT_OK


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_1612_04787_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).replace("the oracle", ""), f


def test_mir_argument_errors_before_any_launch():
    """Invalid meshes, sizes and pointers are rejected on the host."""
    import ctypes as C
    from paper_1612_04787_gb300 import _lib
    lib = _lib.lib
    bad = _lib.SwiftMesh(0, 0, 4, 2, 2)  # cell below 8
    good = _lib.SwiftMesh(0, 0, 16, 2, 2)
    dummy = C.c_void_p(16)
    assert lib.swift_mesh_fit(dummy, dummy, dummy, 1, C.byref(bad), 0, dummy, dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_mesh_fit(dummy, dummy, dummy, 1, C.byref(good), -1, dummy, dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_mesh_fit(None, None, None, 1, C.byref(good), 0, dummy, dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_render_prepare(dummy, C.byref(bad), dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_render_prepare(dummy, C.byref(good), C.c_void_p(8), None) == _lib.SWIFT_ERR_INVALID_ARG
    img = _lib.SwiftImage(None, 8, 0, 8, 8, 1)
    assert lib.swift_render(C.byref(img), 0, dummy, C.byref(good), dummy, 1, 8, 8, 8, 0.0, None) == _lib.SWIFT_ERR_INVALID_ARG
    img = _lib.SwiftImage(16, 8, 0, 8, 8, 1)
    assert lib.swift_render(C.byref(img), 0, dummy, C.byref(good), dummy, 1, 8, 8, 4, 0.0, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_render(C.byref(img), 0, dummy, C.byref(good), dummy, 7, 8, 8, 8, 0.0, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_fit_affine(dummy, dummy, dummy, dummy, -1, dummy, dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_fit_affine(None, None, None, None, 0, None, None, None) == _lib.SWIFT_OK
    assert lib.swift_fit_affine_update(dummy, dummy, dummy, dummy, -1, dummy, dummy, None) == _lib.SWIFT_ERR_INVALID_ARG
    assert lib.swift_fit_affine_update(None, None, None, None, 0, None, None, None) == _lib.SWIFT_OK
    assert lib.swift_correspondences(None, None, None, 4, 64, 0.0, None, None, None, None) == _lib.SWIFT_ERR_INVALID_ARG


def test_window_guard_rule():
    """The guard every origin-reading kernel applies (swift_window_check):
    hand-picked edges of the bounds, negative and huge origins, images
    smaller than the window, and level mismatches (which win over bounds)."""
    import paper_1612_04787_gb300 as swift
    wc = swift.window_check
    n, H, W = 256, 1024, 768
    ok, oob, other = 0, 1, -1
    cases = [
        ((0, 0), (0, 0), ok),
        ((H - n, W - n), (H - n, W - n), ok),          # last fitting origin
        ((H - n + 1, 0), (0, 0), oob),                 # one row too far (reference)
        ((0, W - n + 1), (0, 0), oob),
        ((0, 0), (H - n + 1, 0), oob),                 # moving window
        ((0, 0), (0, W - n + 1), oob),
        ((-1, 0), (0, 0), oob),                        # negative origins
        ((0, -1), (0, 0), oob),
        ((0, 0), (-1, 5), oob),
        ((0, 0), (5, -2147483648), oob),
        ((2147483647, 0), (0, 0), oob),                # no overflow into "inside"
        ((0, 2147483647), (0, 0), oob),
    ]
    for ro, mo, want in cases:
        assert wc(n, 2, 2, ro, mo, (H, W), (H, W)) == want, (ro, mo)
    # moving image smaller than the reference image
    assert wc(n, 0, 0, (H - n, 0), (H - n, 0), (H, W), (H - 1, W)) == oob
    # an image smaller than the window holds no window
    assert wc(n, 0, 0, (0, 0), (0, 0), (n - 1, W), (H, W)) == oob
    assert wc(n, 0, 0, (0, 0), (0, 0), (H, W), (H, n - 1)) == oob
    # another level: skipped whatever its origins
    for ro, mo, _ in cases:
        assert wc(n, 1, 2, ro, mo, (H, W), (H, W)) == other
        assert wc(n, 3, 2, ro, mo, (H, W), (H, W)) == other
    assert wc(n, -5, 0, (0, 0), (0, 0), (H, W), (H, W)) == other
