"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point declared in include/*.h."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(feast_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("feast_setup", "feast_iterate", "feast_eigs", "feast_destroy", "feast_strerror"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1404_1768_gb300 import build, EXPORTS
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert names == set(EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_without_gpu():
    from paper_1404_1768_gb300 import load
    lib = load()
    lib.feast_strerror.restype = ctypes.c_char_p
    assert lib.feast_strerror(0) == b"ok"
    assert b"pivot" in lib.feast_strerror(-4)


def test_workspace_size_validation_without_gpu():
    import paper_1404_1768_gb300 as fg
    lib = fg.load()
    p = fg.Pencil(0, 200, 1, 1, 200, 0, 0, 0)
    c = fg.Contour(0, 0.0, 0.0, 1.0, 1.0, 16, 0)
    o = fg.Options(64, 1, 1e-12, 1e-3, 50, 0, 5, 1e-14, None, 0, 0)
    nb = ctypes.c_size_t(0)
    assert lib.feast_workspace_size(ctypes.byref(p), ctypes.byref(c), ctypes.byref(o), ctypes.byref(nb)) == 0
    # factors alone: 16 * 200 * 200 complex128
    assert nb.value > 16 * 200 * 200 * 16
    bad = fg.Options(300, 1, 1e-12, 1e-3, 50, 0, 5, 1e-14, None, 0, 0)  # m0 > n
    assert lib.feast_workspace_size(ctypes.byref(p), ctypes.byref(c), ctypes.byref(bad), ctypes.byref(nb)) == -1


def test_last_cuda_error_without_gpu():
    """The error-detail accessor is host-only: an empty string while no CUDA
    call of this thread has failed."""
    from paper_1404_1768_gb300 import load
    lib = load()
    assert lib.feast_last_cuda_error() == b""


def test_band_width_bounded_by_the_solve_staging():
    """The band solves keep a circular window of kl + ku + 1 + jc right-hand-
    side rows and jc staged factor columns in shared memory (jc >= 1 staged
    steps, fewer right-hand sides per CTA for wide bands): in FP64 (16-byte
    elements) the narrowest staging, 2 (kl + ku) + 3 elements, fits up to
    kl = ku = 3615 and not 3616; in the precision form (8-byte elements)
    every band up to the kl, ku <= 4096 limit fits.  Wider bands are refused
    at set-up (FEAST_EINVAL) rather than failing to launch."""
    import paper_1404_1768_gb300 as fg
    lib = fg.load()
    c = fg.Contour(1, 0.0, 0.0, 2.0, 1.0, 8, 1)
    nb = ctypes.c_size_t(0)
    for prec, ok_w, bad_w in ((0, 3615, 3616), (1, 4096, 4097)):
        o = fg.Options(8, 1, 1e-12, 1e-3, 50, prec, 5, 1e-14, None, 0, 0)
        for w, expect in ((ok_w, 0), (bad_w, -1)):
            p = fg.Pencil(1, 9000, 1, 1, 2 * w + 1, w, w, 0)
            assert lib.feast_workspace_size(ctypes.byref(p), ctypes.byref(c), ctypes.byref(o),
                                            ctypes.byref(nb)) == expect, (prec, w)
