"""The C ABI library builds, loads and exports every call include/fatiguefft.h
declares; argument checks that need no GPU return FFT_ERR_ARG.  No compute
call runs here (there may be no GPU)."""
import ctypes as C
import os
import re

import numpy as np

from paper_2304_01125_gb300 import build as B
from paper_2304_01125_gb300 import fatiguefft as FF
from paper_2304_01125_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fatiguefft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return", "sizeof")))


def test_library_builds_and_exports_every_declared_call():
    path = B.build()
    L = C.CDLL(path)
    decl = _declared()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert set(FF.SYMBOLS) <= set(decl)


def test_init_rejects_bad_arguments_without_touching_the_gpu():
    L = FF.load(B.build())
    g = FF.Grid()
    g.n[:] = (0, 4, 4)
    g.h = I.VOXEL_MM
    m = FF._material(I.material("baseline"))
    o = FF._options(I.solver_options("paper"), "fp64", None)
    gid = np.zeros(16, dtype=np.int32)
    eul = np.zeros(3)
    h = C.c_void_p()
    assert L.init_rve(C.byref(h), C.byref(g), gid.ctypes.data, 1, eul.ctypes.data, C.byref(m),
                      C.byref(o), None, None) == FF.FFT_ERR_ARG
    g.n[:] = (4, 2, 2)
    g.h = -1.0
    assert L.init_rve(C.byref(h), C.byref(g), gid.ctypes.data, 1, eul.ctypes.data, C.byref(m),
                      C.byref(o), None, None) == FF.FFT_ERR_ARG
    g.h = I.VOXEL_MM
    bad = np.full(16, 3, dtype=np.int32)  # grain id out of range
    assert L.init_rve(C.byref(h), C.byref(g), bad.ctypes.data, 1, eul.ctypes.data, C.byref(m),
                      C.byref(o), None, None) == FF.FFT_ERR_ARG
    assert L.init_rve(None, C.byref(g), gid.ctypes.data, 1, eul.ctypes.data, C.byref(m),
                      C.byref(o), None, None) == FF.FFT_ERR_ARG
    o.max_cutbacks = 11  # beyond the documented depth
    g.n[:] = (4, 2, 2)
    assert L.init_rve(C.byref(h), C.byref(g), gid.ctypes.data, 1, eul.ctypes.data, C.byref(m),
                      C.byref(o), None, None) == FF.FFT_ERR_ARG
    o.max_cutbacks = 0
    # beyond 32-bit spectral indexing, and an extent above 4096: rejected
    # before the grain ids are read
    for n in ((4096, 4096, 64), (8192, 1, 1)):
        g.n[:] = n
        assert L.init_rve(C.byref(h), C.byref(g), gid.ctypes.data, 1, eul.ctypes.data,
                          C.byref(m), C.byref(o), None, None) == FF.FFT_ERR_ARG
    assert L.apply_increment(None, None, 1.0) == FF.FFT_ERR_ARG
    b = C.c_void_p()
    assert L.batch_create(C.byref(b), None, 2, 1) == FF.FFT_ERR_ARG
    arr = (C.c_void_p * 1)(None)
    assert L.batch_create(C.byref(b), arr, 1, 1) == FF.FFT_ERR_ARG
    assert L.batch_create(C.byref(b), arr, 0, 1) == FF.FFT_ERR_ARG
    assert L.batch_size(None) == 0
    assert L.batch_create_ex(C.byref(b), arr, 1, 1, 4) == FF.FFT_ERR_ARG  # unknown flag
    assert L.batch_create_ex(C.byref(b), None, 2, 1, 1) == FF.FFT_ERR_ARG
    assert L.batch_classes(None, -1, None, None, None, None) == 0
    one = (C.c_double * 9)(*np.eye(3).reshape(9))
    assert L.batch_run_increment_mixed(None, one, None, None, one, None, None) == FF.FFT_ERR_ARG
    F9 = (C.c_double * 9)(*np.eye(3).reshape(9))
    m9 = (C.c_int32 * 9)(*([1] * 9))
    assert L.run_increment_mixed(None, F9, None, m9, 1.0, None) == FF.FFT_ERR_ARG
    assert L.apply_increment_mixed(None, F9, None, None, 1.0) == FF.FFT_ERR_ARG
    assert L.rve_device_bytes(None) == 0
    nb = C.c_size_t(0)
    assert L.state_save(None, None, C.byref(nb)) == FF.FFT_ERR_ARG
    assert L.state_load(None, b"x" * 16, 16) == FF.FFT_ERR_ARG


def test_derivative_scheme_option():
    """The derivative scheme reaches the C ABI as an integer (0 spectral,
    1 Willot's rotated scheme); an unknown name fails before any handle is
    made."""
    import pytest
    from paper_2304_01125_gb300 import fatiguefft as FF
    from paper_2304_01125_gb300 import inputs as I
    assert FF._options(I.solver_options("paper"), "mixed", None).derivative == 0
    assert FF._options(I.solver_options("paper", derivative="willot"), "mixed",
                       None).derivative == 1
    with pytest.raises(ValueError):
        FF._options(I.solver_options("paper", derivative="central"), "mixed", None)


def test_kernel_variant_option():
    """The kernel-variant bits reach the C ABI unchanged; the default is 0
    (bulk-copy update pass, unfused x pass)."""
    from paper_2304_01125_gb300 import fatiguefft as FF
    from paper_2304_01125_gb300 import inputs as I
    assert FF._options(I.solver_options("paper"), "mixed", None).kernel_variant == 0
    for v in range(4):
        assert FF._options(I.solver_options("paper", kernel_variant=v), "fp64",
                           None).kernel_variant == v


def test_header_is_plain_c():
    """The boundary header compiles as C99 (no C++ in the C ABI)."""
    import os
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "fatiguefft.h")
    subprocess.run([cc, "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-x", "c", hdr],
                   check=True)
