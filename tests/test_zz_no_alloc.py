"""The allocation-free reduction (degraded_average_noalloc) agrees with the
mean stress the library reports through update_damage/run_increment.

It is meant for callers that may not allocate device memory themselves, so
it keeps its scratch in a fixed array inside the library; here it is called
twice in a row through the C ABI on device buffers owned by the test and
compared with the handle's own result each time.  This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2304_01125_gb300 import build as B
from paper_2304_01125_gb300 import fatiguefft as FF
from paper_2304_01125_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_average_matches_reported_mean_stress_twice():
    torch = pytest.importorskip("torch")
    B.build()
    L = FF.load()
    n = (12, 10, 8)
    N = int(np.prod(n))
    mat = I.material("baseline", tau_c0=250.0)
    gid, eul = I.voronoi(n, 5, 21)
    r = FF.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("parity64"), prec="fp64")
    P = torch.empty(9 * N, dtype=torch.float64, device="cuda")
    phi = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    prog = I.uniaxial_cycle_program(0.006, 24, 1)
    for Fb, dt in prog[4:6]:  # two calls in a row, on two different states
        s, st = r.run_increment(Fb, dt)
        r.field_to_device("Pu", P.data_ptr(), P.numel() * 8)
        r.field_to_device("phi", phi.data_ptr(), phi.numel() * 8)
        status = L.degraded_average_noalloc(P.data_ptr(), 9, phi.data_ptr(), N, mat["k_res"],
                                            out.data_ptr(), stream.cuda_stream)
        assert status == FF.FFT_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = np.array(st["Pbar"])
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
    # a component count beyond the fixed scratch is refused, nothing launched
    assert L.degraded_average_noalloc(P.data_ptr(), 82, phi.data_ptr(), N, 0.0,
                                      out.data_ptr(), stream.cuda_stream) == FF.FFT_ERR_ARG
    r.close()
