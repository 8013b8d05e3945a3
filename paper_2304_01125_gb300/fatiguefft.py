"""ctypes binding of ``libfatiguefft.so`` (declared in ``include/fatiguefft.h``).

Argument marshalling only: every stage of the solve runs in the library's
CUDA kernels.  Importing works without a GPU; creating a handle needs the
built library and a CUDA device and raises otherwise (there is no CPU path).
PyTorch, when given, supplies the CUDA stream and device buffers.
"""
import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfatiguefft.so")

FFT_OK, FFT_ERR_ARG, FFT_ERR_OOM, FFT_ERR_CUDA = 0, -1, -2, -3
FFT_ERR_CUFFT, FFT_ERR_NOT_CONVERGED, FFT_ERR_NONFINITE, FFT_ERR_STATE = -4, -5, -6, -7
FFT_PREC_FP64, FFT_PREC_MIXED = 0, 1
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_CUFFT",
          -5: "ERR_NOT_CONVERGED", -6: "ERR_NONFINITE", -7: "ERR_STATE"}

# field name -> (id, components)
FIELDS = {"F": (0, 9), "P": (1, 9), "phi": (2, 1), "Fp": (3, 9), "rho_ssd": (4, 1),
          "rho_gnd": (5, 1), "Wp": (6, 1), "Gs": (7, 1), "Hmax": (8, 1), "Wcrit": (9, 1),
          "drive": (10, 1), "gamma": (11, 12), "Ft": (12, 9), "phi_t": (13, 1), "We": (14, 1),
          "K": (15, 81), "Pu": (16, 9)}
SYMBOLS = ["init_rve", "apply_increment", "solve_equilibrium", "update_damage",
           "commit_increment", "run_increment", "fields_out", "fields_in", "eval_constitutive",
           "eval_gnd", "solve_phase_field", "rve_device_bytes", "rve_destroy", "fft_last_error",
           "rve_kernel_launches", "rve_profile", "rve_profile_read",
           "degraded_average_noalloc", "batch_create", "batch_run_increment", "batch_size",
           "batch_destroy", "fft_selftest_bounded_wait", "apply_increment_mixed",
           "run_increment_mixed", "state_save", "state_load", "batch_run_increment_mixed",
           "batch_create_ex", "batch_classes"]
KERNEL_FAMILIES = ["constitutive", "tangent_apply", "precond_grad", "contract", "gmres_dot",
                   "gs_update", "gmres_xupdate", "kbar", "residual", "f_update", "phase_field",
                   "gnd", "cufft_9field", "cufft_scalar", "reductions", "other"]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double)]


class Material(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "C11", "C12", "C44", "tau_c0", "b", "nu_D", "k_B", "T", "dF", "rho_m", "lambda_h",
        "dV", "mu", "xi_store", "rho_ssd0", "G_crit", "ell", "ell_Fp", "k_res")]


class Options(C.Structure):
    _fields_ = [("tol_stag", C.c_double), ("tol_newton", C.c_double), ("tol_lin", C.c_double),
                ("tol_pf", C.c_double), ("tol_local", C.c_double),
                ("max_stag", C.c_int), ("max_newton", C.c_int), ("max_lin", C.c_int),
                ("max_pf", C.c_int), ("max_local", C.c_int), ("restart", C.c_int),
                ("prec", C.c_int), ("cuda_stream", C.c_void_p), ("max_cutbacks", C.c_int),
                ("derivative", C.c_int), ("kernel_variant", C.c_int)]

DERIVATIVES = {"spectral": 0, "willot": 1}


class Stats(C.Structure):
    _fields_ = [("stag_it", C.c_int), ("newton_it", C.c_int), ("lin_it_total", C.c_int),
                ("pf_it_total", C.c_int), ("local_fail", C.c_int), ("converged", C.c_int),
                ("skipped_equilibrium", C.c_int), ("res_F", C.c_double),
                ("res_phi", C.c_double), ("Pbar", C.c_double * 9), ("cracked", C.c_long),
                ("cutbacks", C.c_int), ("mixed_it", C.c_int), ("Fbar", C.c_double * 9)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["Pbar"] = list(self.Pbar)
        d["Fbar"] = list(self.Fbar)
        return d


_lib = None


def load(path=LIB_PATH):
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2304_01125_gb300.build")
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.init_rve.argtypes = [C.POINTER(vp), C.POINTER(Grid), C.c_void_p, C.c_int, C.c_void_p,
                           C.POINTER(Material), C.POINTER(Options), C.c_void_p, C.c_void_p]
    L.apply_increment.argtypes = [vp, dp, C.c_double]
    L.solve_equilibrium.argtypes = [vp, C.POINTER(Stats)]
    L.update_damage.argtypes = [vp, C.POINTER(Stats)]
    L.commit_increment.argtypes = [vp]
    L.run_increment.argtypes = [vp, dp, C.c_double, C.POINTER(Stats)]
    L.apply_increment_mixed.argtypes = [vp, dp, dp, C.POINTER(C.c_int32), C.c_double]
    L.run_increment_mixed.argtypes = [vp, dp, dp, C.POINTER(C.c_int32), C.c_double,
                                      C.POINTER(Stats)]
    L.fields_out.argtypes = [vp, C.c_int, C.c_void_p, C.c_size_t, C.c_int]
    L.fields_in.argtypes = [vp, C.c_int, C.c_void_p, C.c_size_t]
    L.state_save.argtypes = [vp, C.c_void_p, C.POINTER(C.c_size_t)]
    L.state_load.argtypes = [vp, C.c_void_p, C.c_size_t]
    L.eval_constitutive.argtypes = [vp, C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.eval_gnd.argtypes = [vp]
    L.solve_phase_field.argtypes = [vp, C.POINTER(C.c_int)]
    L.rve_device_bytes.argtypes = [vp]
    L.rve_device_bytes.restype = C.c_size_t
    L.rve_kernel_launches.argtypes = [vp]
    L.rve_kernel_launches.restype = C.c_longlong
    L.rve_profile.argtypes = [vp, C.c_uint]
    L.rve_profile.restype = C.c_int
    L.rve_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_double), C.c_int]
    L.rve_profile_read.restype = C.c_int
    L.degraded_average_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t,
                                           C.c_double, C.c_void_p, C.c_void_p]
    L.degraded_average_noalloc.restype = C.c_int
    L.rve_destroy.argtypes = [vp]
    L.rve_destroy.restype = None
    L.batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_int]
    L.batch_create.restype = C.c_int
    L.batch_run_increment.argtypes = [vp, dp, dp, C.POINTER(Stats), C.POINTER(C.c_int)]
    L.batch_run_increment.restype = C.c_int
    L.batch_run_increment_mixed.argtypes = [vp, dp, dp, C.POINTER(C.c_int32), dp,
                                            C.POINTER(Stats), C.POINTER(C.c_int)]
    L.batch_run_increment_mixed.restype = C.c_int
    L.batch_create_ex.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_int, C.c_int]
    L.batch_create_ex.restype = C.c_int
    L.batch_classes.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                dp, dp]
    L.batch_classes.restype = C.c_int
    L.batch_size.argtypes = [vp]
    L.batch_size.restype = C.c_int
    L.batch_destroy.argtypes = [vp]
    L.batch_destroy.restype = None
    L.fft_selftest_bounded_wait.argtypes = [C.c_uint]
    L.fft_selftest_bounded_wait.restype = C.c_int
    L.fft_last_error.argtypes = [vp]
    L.fft_last_error.restype = C.c_char_p
    for t in ("init_rve", "apply_increment", "solve_equilibrium", "update_damage",
              "commit_increment", "run_increment", "fields_out", "fields_in",
              "eval_constitutive", "eval_gnd", "solve_phase_field", "apply_increment_mixed",
              "run_increment_mixed", "state_save", "state_load"):
        getattr(L, t).restype = C.c_int
    _lib = L
    return L


def degraded_average_noalloc(X_ptr, ncomp, phi_ptr, N, k_res, out_ptr, stream=0):
    """(1/N) sum_v g(phi_v) X[c][v] into out (device pointers), allocating
    nothing; see include/fatiguefft.h.  Returns the status code."""
    return load().degraded_average_noalloc(int(X_ptr), int(ncomp), int(phi_ptr), int(N),
                                           float(k_res), int(out_ptr), int(stream) or None)


class FFTError(RuntimeError):
    def __init__(self, call, status, msg):
        super().__init__(f"{call}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _material(params):
    m = Material()
    for k, _ in Material._fields_:
        setattr(m, k, float(params[k]))
    return m


def _options(opts, prec, stream):
    d = opts.get("derivative", "spectral")
    if d not in DERIVATIVES:
        raise ValueError(f"derivative scheme {d!r}: one of {sorted(DERIVATIVES)}")
    o = Options()
    for k in ("tol_stag", "tol_newton", "tol_lin", "tol_pf", "tol_local"):
        setattr(o, k, float(opts[k]))
    for k in ("max_stag", "max_newton", "max_lin", "max_pf", "max_local", "restart"):
        setattr(o, k, int(opts[k]))
    o.prec = FFT_PREC_FP64 if prec in ("fp64", FFT_PREC_FP64) else FFT_PREC_MIXED
    o.cuda_stream = stream or None
    o.max_cutbacks = int(opts.get("max_cutbacks", 0))
    o.derivative = DERIVATIVES[d]
    o.kernel_variant = int(opts.get("kernel_variant", 0))
    return o


class RVE:
    """One RVE handle of the library.  ``prec``: "fp64" or "mixed".
    ``stream``: a ``torch.cuda.Stream`` or raw ``cudaStream_t`` (int)."""

    def __init__(self, n, h, grain_ids, euler, params, opts, prec="fp64", phi0=None,
                 elastic_only=None, stream=None):
        L = load()
        self.n = tuple(int(x) for x in n)
        self._batches = weakref.WeakSet()  # live batches holding this handle
        self.N = int(np.prod(self.n))
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._stream = stream
        g = Grid()
        g.n[:] = self.n
        g.h = float(h)
        gid = np.ascontiguousarray(grain_ids, dtype=np.int32).reshape(-1)
        eul = np.ascontiguousarray(euler, dtype=np.float64).reshape(-1)
        assert gid.size == self.N
        p0 = None if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64).reshape(-1)
        eo = None if elastic_only is None else np.ascontiguousarray(elastic_only,
                                                                    dtype=np.uint8).reshape(-1)
        self._m = _material(params)
        self._o = _options(opts, prec, stream)
        h_ = C.c_void_p()
        s = L.init_rve(C.byref(h_), C.byref(g), gid.ctypes.data, int(eul.size // 3),
                       eul.ctypes.data, C.byref(self._m), C.byref(self._o),
                       None if p0 is None else p0.ctypes.data,
                       None if eo is None else eo.ctypes.data)
        if s != FFT_OK:
            raise FFTError("init_rve", s, "")
        self._h = h_

    # -- helpers
    def _check(self, call, s):
        if s != FFT_OK:
            raise FFTError(call, s, load().fft_last_error(self._h).decode())
        return s

    def close(self):
        if getattr(self, "_h", None):
            # a batch holding the handle is destroyed first (a lockstep class
            # keeps part of the handle's buffers in its arenas)
            for b in list(getattr(self, "_batches", ())):
                b.close()
            load().rve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the C calls
    def apply_increment(self, Fbar, dt):
        F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
        return self._check("apply_increment", load().apply_increment(
            self._h, F.ctypes.data_as(C.POINTER(C.c_double)), float(dt)))

    def solve_equilibrium(self, st=None, check=True):
        st = st or Stats()
        s = load().solve_equilibrium(self._h, C.byref(st))
        if check:
            self._check("solve_equilibrium", s)
        return s, st

    def update_damage(self, st=None, check=True):
        st = st or Stats()
        s = load().update_damage(self._h, C.byref(st))
        if check:
            self._check("update_damage", s)
        return s, st

    def commit_increment(self):
        return self._check("commit_increment", load().commit_increment(self._h))

    def run_increment(self, Fbar, dt, check=True, Pbar=None, stress_mask=None):
        """One increment (run_increment).  With stress_mask (9 flags) the
        flagged components of the mean degraded first Piola stress are
        prescribed (Pbar, default 0) and the matching components of Fbar
        (initial guesses) are solved for (run_increment_mixed)."""
        F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(9)
        st = Stats()
        fp = F.ctypes.data_as(C.POINTER(C.c_double))
        if stress_mask is None:
            s = load().run_increment(self._h, fp, float(dt), C.byref(st))
            call = "run_increment"
        else:
            P = np.ascontiguousarray(np.zeros(9) if Pbar is None else Pbar,
                                     dtype=np.float64).reshape(9)
            m = (C.c_int32 * 9)(*[int(bool(x)) for x in np.asarray(stress_mask).reshape(9)])
            s = load().run_increment_mixed(self._h, fp, P.ctypes.data_as(C.POINTER(C.c_double)),
                                           m, float(dt), C.byref(st))
            call = "run_increment_mixed"
        if check:
            self._check(call, s)
        return s, st.as_dict()

    def state_save(self):
        """Checkpoint of the committed state (state_save), as bytes."""
        n = C.c_size_t(0)
        self._check("state_save", load().state_save(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check("state_save", load().state_save(self._h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def state_load(self, data):
        """Restore a checkpoint from state_save (state_load)."""
        b = bytes(data)
        self._check("state_load", load().state_load(self._h, b, len(b)))

    def field(self, name):
        fid, nc = FIELDS[name]
        out = np.empty(nc * self.N, dtype=np.float64)
        self._check("fields_out", load().fields_out(self._h, fid, out.ctypes.data, out.nbytes, 0))
        return out.reshape(nc, self.N) if nc > 1 else out

    def field_to_device(self, name, dst_ptr, nbytes):
        fid, _ = FIELDS[name]
        return self._check("fields_out", load().fields_out(self._h, fid, int(dst_ptr),
                                                           int(nbytes), 1))

    def set_field(self, name, values):
        fid, nc = FIELDS[name]
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        assert a.size == nc * self.N
        return self._check("fields_in", load().fields_in(self._h, fid, a.ctypes.data, a.nbytes))

    def eval_constitutive(self, dt, with_history=False):
        nf = C.c_int(0)
        self._check("eval_constitutive", load().eval_constitutive(self._h, float(dt),
                                                                  int(with_history),
                                                                  C.byref(nf)))
        return nf.value

    def eval_gnd(self):
        return self._check("eval_gnd", load().eval_gnd(self._h))

    def solve_phase_field(self):
        it = C.c_int(0)
        self._check("solve_phase_field", load().solve_phase_field(self._h, C.byref(it)))
        return it.value

    def profile(self, families):
        """Time the given kernel families (names from KERNEL_FAMILIES)."""
        mask = 0
        for f in families:
            mask |= 1 << KERNEL_FAMILIES.index(f)
        return self._check("rve_profile", load().rve_profile(self._h, mask))

    def profile_read(self, reset=True):
        ms = (C.c_double * 16)()
        cnt = (C.c_longlong * 16)()
        by = (C.c_double * 16)()
        self._check("rve_profile_read", load().rve_profile_read(self._h, ms, cnt, by,
                                                                int(reset)))
        return {f: (ms[i], cnt[i], by[i]) for i, f in enumerate(KERNEL_FAMILIES) if cnt[i]}

    @property
    def device_bytes(self):
        return load().rve_device_bytes(self._h)

    @property
    def kernel_launches(self):
        return load().rve_kernel_launches(self._h)


class Batch:
    """Many independent RVE handles advanced together (batch_run_increment):
    each handle needs its own stream; a native thread pool of ``threads``
    host threads (None: the hardware concurrency) drives them concurrently.
    With ``classes`` (default True), handles of one size class (grid,
    precision, options) of at most 2^16 voxels run in lockstep under strain
    control, each Krylov column of a class one graph launch
    (batch_create_ex); ``classes="all"`` forms classes at any grid size,
    False none.  The handles stay owned by the caller."""

    def __init__(self, rves, threads=None, classes=True):
        self.rves = list(rves)
        arr = (C.c_void_p * len(self.rves))(*[r._h for r in self.rves])
        h = C.c_void_p()
        flags = 3 if classes == "all" else (1 if classes else 0)
        s = load().batch_create_ex(C.byref(h), arr, len(self.rves), int(threads or 0), flags)
        if s != FFT_OK:
            raise FFTError("batch_create", s, "distinct handles, each with its own stream "
                                              "and in no other live batch")
        self._h = h
        for r in self.rves:
            r._batches.add(self)

    def classes(self, timing=None):
        """[(members, column graphs launched, graph ms, algorithmic bytes)]
        per lockstep class; timing True/False switches the event timing of
        the column graphs on/off (the sums are read, then zeroed)."""
        n = len(self.rves)
        sz = (C.c_int * n)()
        gl = (C.c_longlong * n)()
        ms = (C.c_double * n)()
        by = (C.c_double * n)()
        t = -1 if timing is None else int(bool(timing))
        k = load().batch_classes(self._h, t, sz, gl, ms, by)
        return [(int(sz[i]), int(gl[i]), float(ms[i]), float(by[i])) for i in range(k)]

    def run_increment(self, Fbars, dts, check=True, Pbars=None, stress_masks=None):
        """Fbars: (n, 9) absolute macroscopic F per handle; dts: (n,).  With
        stress_masks (n, 9) flags, mixed control per handle
        (batch_run_increment_mixed, Pbars (n, 9) or None for zero targets).
        Returns (status, per-handle statuses, per-handle stats dicts)."""
        n = len(self.rves)
        dp = C.POINTER(C.c_double)
        F = np.ascontiguousarray(np.asarray(Fbars, dtype=np.float64).reshape(n, 9))
        dt = np.ascontiguousarray(np.asarray(dts, dtype=np.float64).reshape(n))
        stats = (Stats * n)()
        st = (C.c_int * n)()
        if stress_masks is None:
            call = "batch_run_increment"
            s = load().batch_run_increment(self._h, F.ctypes.data_as(dp), dt.ctypes.data_as(dp),
                                           stats, st)
        else:
            call = "batch_run_increment_mixed"
            m = np.ascontiguousarray((np.asarray(stress_masks).reshape(n, 9) != 0)
                                     .astype(np.int32))
            P = np.ascontiguousarray(np.zeros((n, 9)) if Pbars is None else
                                     np.asarray(Pbars, dtype=np.float64).reshape(n, 9))
            s = load().batch_run_increment_mixed(
                self._h, F.ctypes.data_as(dp), P.ctypes.data_as(dp),
                m.ctypes.data_as(C.POINTER(C.c_int32)), dt.ctypes.data_as(dp), stats, st)
        per = list(st)
        if check and s != FFT_OK:
            bad = [i for i, x in enumerate(per) if x != FFT_OK]
            msg = load().fft_last_error(self.rves[bad[0]]._h).decode() if bad else ""
            raise FFTError(call, s, f"handles {bad}: {msg}")
        return s, per, [x.as_dict() for x in stats]

    def close(self):
        if getattr(self, "_h", None):
            load().batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
