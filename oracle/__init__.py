"""ctypes binding of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the package smoke
check and by the CPU-baseline leg of ``bench.py``; never by the product path.
The oracle restates the paper's equations plainly (own FFT, own slip tables,
own solvers) and shares no code with the GPU library.
"""
import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None


class Material(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "C11", "C12", "C44", "tau_c0", "b", "nu_D", "k_B", "T", "dF", "rho_m", "lambda_h",
        "dV", "mu", "xi_store", "rho_ssd0", "G_crit", "ell", "ell_Fp", "k_res")]


class Options(C.Structure):
    _fields_ = [("tol_stag", C.c_double), ("tol_newton", C.c_double), ("tol_lin", C.c_double),
                ("tol_pf", C.c_double), ("tol_local", C.c_double),
                ("max_stag", C.c_int), ("max_newton", C.c_int), ("max_lin", C.c_int),
                ("max_pf", C.c_int), ("max_local", C.c_int), ("restart", C.c_int),
                ("use_naive_dft", C.c_int), ("n_threads", C.c_int), ("max_cutbacks", C.c_int),
                ("derivative", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("stag_it", C.c_int), ("newton_it", C.c_int), ("lin_it_total", C.c_int),
                ("pf_it_total", C.c_int), ("local_fail", C.c_int), ("converged", C.c_int),
                ("skipped_equilibrium", C.c_int), ("res_F", C.c_double),
                ("res_phi", C.c_double), ("Pbar", C.c_double * 9), ("cracked", C.c_long),
                ("mixed_it", C.c_int), ("Fbar", C.c_double * 9), ("cutbacks", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["Pbar"] = list(self.Pbar)
        d["Fbar"] = list(self.Fbar)
        return d


class CPResult(C.Structure):
    _fields_ = [("P", C.c_double * 9), ("K", C.c_double * 81), ("S_L", C.c_double * 6),
                ("Fp_L", C.c_double * 9), ("dgamma", C.c_double * 12), ("tau", C.c_double * 12),
                ("tau_c", C.c_double), ("dWp", C.c_double), ("drho_ssd", C.c_double),
                ("We_plus", C.c_double), ("iters", C.c_int), ("fail", C.c_int)]


FIELDS = {"F": (0, 9), "P": (1, 9), "phi": (2, 1), "Fp": (3, 9), "rho_ssd": (4, 1),
          "rho_gnd": (5, 1), "Wp": (6, 1), "Gs": (7, 1), "Hmax": (8, 1), "Wcrit": (9, 1),
          "drive": (10, 1), "gamma": (11, 12), "Ft": (12, 9), "phi_t": (13, 1), "We": (14, 1)}

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _declare(L):
    L.orc_fft3d.argtypes = [C.c_int * 3, _dp, C.c_int, C.c_int]
    L.orc_material_paper.argtypes = [C.POINTER(Material)]
    L.orc_euler_to_Q.argtypes = [_dp, _dp]
    L.orc_fcc_systems.argtypes = [_dp, _dp]
    L.orc_gnd_basis.argtypes = [_dp, _dp]
    L.orc_cp_point.argtypes = [C.POINTER(Material), _dp, _dp, _dp, C.c_double, C.c_double,
                               C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                               C.POINTER(CPResult)]
    L.orc_we_plus.argtypes = [C.POINTER(Material), _dp]
    L.orc_we_plus.restype = C.c_double
    L.orc_sym_eig3.argtypes = [_dp, _dp, _dp]
    L.orc_green_precond.argtypes = [_dp, _dp, _dp]
    L.orc_gnd_field.argtypes = [C.c_int * 3, C.c_double, C.POINTER(Material), _dp, _dp,
                                C.c_int, _dp, _dp]
    L.orc_phase_field.argtypes = [C.c_int * 3, C.c_double, C.c_double, _dp, _dp, _dp,
                                  C.c_double, C.c_int, C.c_int, _dp, C.POINTER(C.c_int)]
    L.orc_rve_create.argtypes = [C.c_int * 3, C.c_double, _ip, C.c_int, _dp,
                                 C.POINTER(Material), C.POINTER(Options), C.c_void_p,
                                 C.c_void_p]
    L.orc_rve_create.restype = C.c_void_p
    L.orc_rve_destroy.argtypes = [C.c_void_p]
    L.orc_apply_increment.argtypes = [C.c_void_p, _dp, C.c_double]
    for fn in ("orc_solve_equilibrium", "orc_update_damage"):
        getattr(L, fn).argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.orc_commit.argtypes = [C.c_void_p]
    L.orc_run_increment.argtypes = [C.c_void_p, _dp, C.c_double, C.POINTER(Stats)]
    L.orc_run_increment_mixed.argtypes = [C.c_void_p, _dp, _dp, C.POINTER(C.c_int),
                                          C.c_double, C.POINTER(Stats)]
    L.orc_fields_out.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_fields_in.argtypes = [C.c_void_p, C.c_int, _dp]
    return L


def lib():
    global _LIB
    if _LIB is None:
        _LIB = _declare(C.CDLL(_build.build()))
    return _LIB


@contextlib.contextmanager
def library(path):
    """Route every call of this module through another build of the oracle
    (the mutation tests load builds with a planted mistake) until the block
    ends.  Handles created inside the block must be closed inside it."""
    global _LIB
    prev = lib()
    _LIB = _declare(C.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        _LIB = prev


def _n3(n):
    return (C.c_int * 3)(*[int(x) for x in n])


def material(params):
    m = Material()
    for k, _ in Material._fields_:
        setattr(m, k, float(params[k]))
    return m


def options(opts, naive=False, threads=0):
    o = Options()
    for k in ("tol_stag", "tol_newton", "tol_lin", "tol_pf", "tol_local"):
        setattr(o, k, float(opts[k]))
    for k in ("max_stag", "max_newton", "max_lin", "max_pf", "max_local", "restart"):
        setattr(o, k, int(opts[k]))
    o.use_naive_dft = 1 if naive else 0
    o.n_threads = int(threads)
    o.max_cutbacks = int(opts.get("max_cutbacks", 0))
    o.derivative = {"spectral": 0, "willot": 1}[opts.get("derivative", "spectral")]
    return o


def fft3d(a, sign=-1, naive=False):
    """3-D transform of a complex array of shape (n2, n1, n0) (x fastest)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    n = (a.shape[2], a.shape[1], a.shape[0])
    buf = a.view(np.float64).reshape(-1).copy()
    lib().orc_fft3d(_n3(n), buf, int(sign), 1 if naive else 0)
    return buf.view(np.complex128).reshape(a.shape)


def euler_to_Q(e):
    Q = np.zeros(9)
    lib().orc_euler_to_Q(np.ascontiguousarray(e, dtype=np.float64), Q)
    return Q.reshape(3, 3)


def fcc_systems():
    s = np.zeros(36)
    n = np.zeros(36)
    lib().orc_fcc_systems(s, n)
    return s.reshape(12, 3), n.reshape(12, 3)


def gnd_basis():
    A = np.zeros(162)
    Ap = np.zeros(162)
    lib().orc_gnd_basis(A, Ap)
    return A.reshape(9, 18), Ap.reshape(18, 9)


def cp_point(params, Q, F, Fp_L, rho_ssd, rho_gnd, dt, elastic_only=False, tol_local=1e-10,
             max_local=100, tangent=True):
    m = material(params)
    r = CPResult()
    lib().orc_cp_point(C.byref(m), np.ascontiguousarray(Q, dtype=np.float64).reshape(9),
                       np.ascontiguousarray(F, dtype=np.float64).reshape(9),
                       np.ascontiguousarray(Fp_L, dtype=np.float64).reshape(9),
                       float(rho_ssd), float(rho_gnd), float(dt), int(bool(elastic_only)),
                       float(tol_local), int(max_local), int(bool(tangent)), C.byref(r))
    return {"P": np.array(r.P).reshape(3, 3), "K": np.array(r.K).reshape(9, 9),
            "S_L": np.array(r.S_L), "Fp_L": np.array(r.Fp_L).reshape(3, 3),
            "dgamma": np.array(r.dgamma), "tau": np.array(r.tau), "tau_c": r.tau_c,
            "dWp": r.dWp, "drho_ssd": r.drho_ssd, "We_plus": r.We_plus, "iters": r.iters,
            "fail": r.fail}


def we_plus(params, Fe_L):
    m = material(params)
    return lib().orc_we_plus(C.byref(m), np.ascontiguousarray(Fe_L, dtype=np.float64).reshape(9))


def sym_eig3(A):
    w = np.zeros(3)
    V = np.zeros(9)
    lib().orc_sym_eig3(np.ascontiguousarray(A, dtype=np.float64).reshape(9), w, V)
    return w, V.reshape(3, 3)


def green_precond(Kbar, xi):
    M = np.zeros(9)
    lib().orc_green_precond(np.ascontiguousarray(Kbar, dtype=np.float64).reshape(81),
                            np.ascontiguousarray(xi, dtype=np.float64), M)
    return M.reshape(3, 3)


def gnd_field(n, h, params, Q_per_voxel, Fp, naive=False):
    N = int(np.prod(n))
    m = material(params)
    Lam = np.zeros(9 * N)
    rho = np.zeros(N)
    lib().orc_gnd_field(_n3(n), float(h), C.byref(m),
                        np.ascontiguousarray(Q_per_voxel, dtype=np.float64).reshape(-1),
                        np.ascontiguousarray(Fp, dtype=np.float64).reshape(-1), int(naive),
                        Lam, rho)
    return Lam.reshape(9, N), rho


def phase_field(n, h, ell, S, phi_prev, phi_t, tol=1e-12, max_it=1000, naive=False):
    N = int(np.prod(n))
    out = np.zeros(N)
    it = C.c_int(0)
    st = lib().orc_phase_field(_n3(n), float(h), float(ell),
                               np.ascontiguousarray(S, dtype=np.float64).reshape(-1),
                               np.ascontiguousarray(phi_prev, dtype=np.float64).reshape(-1),
                               np.ascontiguousarray(phi_t, dtype=np.float64).reshape(-1),
                               float(tol), int(max_it), int(naive), out, C.byref(it))
    return out, it.value, st


class RVE:
    """The oracle's Algorithm 1 solver on one periodic voxel RVE."""

    def __init__(self, n, h, grain_ids, euler, params, opts, phi0=None, elastic_only=None,
                 naive=False, threads=0):
        self.n = tuple(int(x) for x in n)
        self.N = int(np.prod(self.n))
        if not threads:
            # the oracle starts its threads for every parallel loop, which
            # outweighs the work of a loop over fewer than ~32k voxels
            threads = 1 if self.N < 32768 else (os.cpu_count() or 1)
        self._m = material(params)
        self._o = options(opts, naive, threads)
        g = np.ascontiguousarray(grain_ids, dtype=np.int32).reshape(-1)
        e = np.ascontiguousarray(euler, dtype=np.float64).reshape(-1)
        self._keep = []
        p0 = None
        if phi0 is not None:
            a = np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
            self._keep.append(a)
            p0 = a.ctypes.data
        eo = None
        if elastic_only is not None:
            a = np.ascontiguousarray(elastic_only, dtype=np.uint8).reshape(-1)
            self._keep.append(a)
            eo = a.ctypes.data
        self._h = lib().orc_rve_create(_n3(self.n), float(h), g, int(e.size // 3), e,
                                       C.byref(self._m), C.byref(self._o), p0, eo)

    def close(self):
        if self._h:
            lib().orc_rve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_increment(self, Fbar, dt):
        return lib().orc_apply_increment(self._h, np.ascontiguousarray(Fbar, dtype=np.float64)
                                         .reshape(9), float(dt))

    def solve_equilibrium(self, st=None):
        st = st or Stats()
        return lib().orc_solve_equilibrium(self._h, C.byref(st)), st

    def update_damage(self, st=None):
        st = st or Stats()
        return lib().orc_update_damage(self._h, C.byref(st)), st

    def commit(self):
        return lib().orc_commit(self._h)

    def run_increment(self, Fbar, dt, Pbar=None, stress_mask=None):
        """One increment; with stress_mask (9 flags), the flagged components
        of the macroscopic first Piola stress are prescribed (Pbar, default 0)
        and the matching components of Fbar are solved for (mixed control)."""
        st = Stats()
        F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
        if stress_mask is None:
            s = lib().orc_run_increment(self._h, F, float(dt), C.byref(st))
        else:
            P = np.ascontiguousarray(np.zeros(9) if Pbar is None else Pbar,
                                     dtype=np.float64).reshape(9)
            m = (C.c_int * 9)(*[int(bool(x)) for x in np.asarray(stress_mask).reshape(9)])
            s = lib().orc_run_increment_mixed(self._h, F, P, m, float(dt), C.byref(st))
        return s, st.as_dict()

    def field(self, name):
        fid, nc = FIELDS[name]
        out = np.zeros(nc * self.N)
        s = lib().orc_fields_out(self._h, fid, out)
        if s:
            raise ValueError(f"oracle field {name}: status {s}")
        return out.reshape(nc, self.N) if nc > 1 else out

    def set_field(self, name, values):
        fid, nc = FIELDS[name]
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        assert a.size == nc * self.N
        s = lib().orc_fields_in(self._h, fid, a)
        if s:
            raise ValueError(f"oracle set_field {name}: status {s}")
