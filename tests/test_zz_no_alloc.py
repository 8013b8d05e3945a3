"""The allocation-free reduction (degraded_average_noalloc) against the mean
stress the library reports through run_increment (the allocating path) and
against a NumPy mean of the same device buffers copied to the host.

It serves callers that may not allocate device memory themselves (a host
framework that owns all device memory, a pre-sized pool, code that must not
allocate once a run has started), so it keeps its scratch in a fixed array
inside the library; here it is called twice in a row through the C ABI on
device buffers owned by the test, on two different states.  This file is
collected last so that a failure here comes after every other test has run.
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
    K = torch.empty(81 * N, dtype=torch.float64, device="cuda")
    phi = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.full((81,), float("nan"), dtype=torch.float64, device="cuda")
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
        got = out.cpu().numpy()[:9]
        # the allocating path: the mean stress run_increment reports
        want = np.array(st["Pbar"])
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
        # an independent host mean of the same buffers
        g = (1.0 - phi.cpu().numpy()) ** 2 + mat["k_res"]
        host = np.mean(g * P.cpu().numpy().reshape(9, N), axis=1)
        assert np.linalg.norm(got - host) <= 1e-12 * np.linalg.norm(host)
    # all 81 components (the largest count the scratch holds): the averaged
    # tangent of the last state
    r.field_to_device("K", K.data_ptr(), K.numel() * 8)
    assert L.degraded_average_noalloc(K.data_ptr(), 81, phi.data_ptr(), N, mat["k_res"],
                                      out.data_ptr(), stream.cuda_stream) == FF.FFT_OK
    torch.cuda.synchronize()
    g = (1.0 - phi.cpu().numpy()) ** 2 + mat["k_res"]
    host = np.mean(g * K.cpu().numpy().reshape(81, N), axis=1)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - host) <= 1e-12 * np.linalg.norm(host)
    # a component count beyond the fixed scratch is refused, nothing launched
    assert L.degraded_average_noalloc(P.data_ptr(), 82, phi.data_ptr(), N, 0.0,
                                      out.data_ptr(), stream.cuda_stream) == FF.FFT_ERR_ARG
    r.close()
