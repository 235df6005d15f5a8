"""The C-ABI library loads and exports every function that include/spdhss.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "spdhss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:spdhss_status|const char\*|int64_t|void)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_declared_symbols():
    from paper_2011_07632_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    lib.spdhss_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.spdhss_version()


def test_binding_signatures_cover_header():
    from paper_2011_07632_gb300 import native
    assert set(_declared()) <= set(native.exported_symbols())


def test_invalid_arguments_rejected_before_device_work():
    """Argument checks run on the host before any CUDA call: each bad argument returns
    EINVAL with a message (no GPU needed)."""
    import numpy as np
    from paper_2011_07632_gb300 import build, native
    build.build()
    L = native.lib()
    pts = np.zeros((4, 3))
    P = pts.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()

    def h2(points, n, dim, kind, ell, shift, leaf, tol):
        kd = native.KernelDesc(kind, ell, shift)
        return L.h2_build(points, n, dim, kd, leaf, tol, None, ctypes.byref(h))

    cases = [
        ((None, 4, 3, 0, 1.0, 0.0, 8, 1e-8), b"points is NULL"),
        ((P, 0, 3, 0, 1.0, 0.0, 8, 1e-8), b"n out of range"),
        ((P, 4, 4, 0, 1.0, 0.0, 8, 1e-8), b"dim must be 2 or 3"),
        ((P, 4, 3, 0, 1.0, 0.0, 0, 1e-8), b"leaf_size"),
        ((P, 4, 3, 0, 1.0, 0.0, 8, 1.0), b"tol"),
        ((P, 4, 3, 5, 1.0, 0.0, 8, 1e-8), b"unknown kernel kind"),
        ((P, 4, 2, native.KERNELS["rpy"], 0.3, 0.0, 8, 1e-8), b"RPY kernel needs dim 3"),
        ((P, 4, 3, 0, 0.0, 0.0, 8, 1e-8), b"length scale"),
        ((P, 4, 3, 0, 1.0, -1.0, 8, 1e-8), b"shift"),
    ]
    for args, msg in cases:
        assert h2(*args) == native.EINVAL, args
        assert msg in L.spdhss_last_error(), (args, L.spdhss_last_error())
    # products and solves with NULL handles
    assert L.h2_matmul(None, None, None, 1, 4, None) == native.EINVAL
    assert L.pcg_solve(None, None, None, None, 1, 4, 1e-6, 10, None, None, None) == native.EINVAL
    assert L.ulv_solve_noalloc(None, None, None, 1, 4, None) == native.EINVAL
