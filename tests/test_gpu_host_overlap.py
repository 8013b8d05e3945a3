"""The host inside the GMRES cycle (Sec. 3.2, the Newton-Krylov solve of
Eq. newton): the solver enqueues Arnoldi column j before it reads the
coefficients of column j - 1, so the device should never wait for the host
within a restart cycle.  A probe built against the library's internal header
(tests/native/hostgap_probe.cu) times 10 and 30 columns of the 64^3 / 50-grain
workload after eight increments, once with the solver's read pattern and once
enqueued back to back: the per-column times agree within 5 %."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2304_01125_gb300 import build as B
from paper_2304_01125_gb300 import fatiguefft as FF
from paper_2304_01125_gb300 import inputs as I

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _probe(tmp_path):
    B.build()
    FF.load()
    so = str(tmp_path / "hostgap_probe.so")
    nvcc = shutil.which("nvcc") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"),
                                                "bin", "nvcc")
    libdir = os.path.dirname(B.LIB)
    subprocess.check_call([nvcc, *B.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", B.CSRC,
                           os.path.join(HERE, "native", "hostgap_probe.cu"), "-o", so,
                           "-L", libdir, "-lfatiguefft", "-lcufft",
                           "-Xlinker", "-rpath=" + libdir])
    L = C.CDLL(so)
    L.hostgap.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double)]
    L.hostgap.restype = C.c_int
    return L


def test_host_reads_are_off_the_critical_path(tmp_path):
    import torch
    L = _probe(tmp_path)
    cfg = I.build_config("poly64")
    r = FF.RVE(cfg["n"], I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], I.material("baseline"),
               I.solver_options("paper"), prec="mixed", stream=torch.cuda.Stream())
    for Fb, dt in cfg["program"][:8]:
        r.run_increment(Fb, dt)
    out = (C.c_double * 2)()
    for ncols in (10, 30):
        assert L.hostgap(r._h, ncols, 5, out) == 0
        back_to_back, with_reads = out[0], out[1]
        assert 0 < back_to_back < 1.0  # ms per column at 64^3
        assert with_reads < 1.05 * back_to_back, (ncols, back_to_back, with_reads)
    r.close()
