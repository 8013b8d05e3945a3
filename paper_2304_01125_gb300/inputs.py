"""Seeded synthetic inputs: material presets, solver presets, periodic Voronoi
polycrystals, orientations, pre-crack masks and cyclic loading programs.

This module holds none of the method's arithmetic.  It only produces the data
a run starts from, so the GPU library and the CPU oracle can be fed exactly
the same inputs.  Units are MPa, mm, s.

The paper's own microstructures are not available (they appear only as
figures), so seeded periodic Voronoi tessellations with orientations uniform
on SO(3) stand in for them, with the voxel size of Sec. 4 (0.78 um).
"""
import math

import numpy as np

VOXEL_MM = 0.78e-3  # Sec. 4: characteristic voxel length 0.78 um

# Table 1 (CMSX-4) as printed, plus the constants the paper uses without a
# value: activation volume dV (20 b^3), shear modulus mu (= C44), stored-energy
# fraction xi_store, initial SSD density (= rho_m).  G_crit = 4 J/m^2 and
# ell = 2.34 um, ell_Fp = 1.56 um are from Sec. 4.
_B = 3.5e-7
PAPER_TABLE1 = {
    "C11": 250e3, "C12": 161e3, "C44": 129e3, "tau_c0": 350.0, "b": _B, "nu_D": 1e11,
    "k_B": 1.4e-23, "T": 295.0, "dF": 4.9e-20, "rho_m": 5.0e6, "lambda_h": 150e6,
    "dV": 20.0 * _B ** 3, "mu": 129e3, "xi_store": 0.05, "rho_ssd0": 5.0e6,
    "G_crit": 4e-3, "ell": 2.34e-3, "ell_Fp": 1.56e-3, "k_res": 1e-5,
}


def material(preset="baseline", **overrides):
    """Material dictionary.

    ``paper``: Table 1 exactly.  ``baseline``: Table 1 with the cubic constants
    C11/C12/C44 = 246.5/147.3/124.7 GPa and ell = ell_Fp = 2 voxels.
    """
    m = dict(PAPER_TABLE1)
    if preset == "baseline":
        m.update(C11=246.5e3, C12=147.3e3, C44=124.7e3, mu=124.7e3,
                 ell=2 * VOXEL_MM, ell_Fp=2 * VOXEL_MM)
    elif preset != "paper":
        raise ValueError(preset)
    m.update(overrides)
    return m


def solver_options(preset="paper", **overrides):
    """Tolerance presets.

    ``paper``: Newton and staggered 5e-3, Krylov 1e-5 (Sec. 3.1-3.2).
    ``parity64``: tight tolerances for FP64 parity.  ``parity32``: the
    tightest the FP32-bulk path reaches reliably.
    """
    base = {"max_stag": 300, "max_newton": 25, "max_lin": 2000, "max_pf": 500, "max_local": 100,
            "restart": 30, "max_cutbacks": 0}
    if preset == "paper":
        o = dict(tol_stag=5e-3, tol_newton=5e-3, tol_lin=1e-5, tol_pf=1e-5, tol_local=1e-9)
    elif preset == "parity64":
        o = dict(tol_stag=1e-9, tol_newton=1e-9, tol_lin=1e-10, tol_pf=1e-11,
                 tol_local=1e-10)
    elif preset == "parity32":
        o = dict(tol_stag=1e-4, tol_newton=1e-4, tol_lin=1e-6, tol_pf=1e-6, tol_local=3e-4)
    else:
        raise ValueError(preset)
    base.update(o)
    base.update(overrides)
    return base


def random_orientations(rng, n):
    """Bunge Euler angles uniform on SO(3): phi1, phi2 uniform, cos(Phi) uniform."""
    phi1 = 2.0 * math.pi * rng.random(n)
    Phi = np.arccos(np.clip(2.0 * rng.random(n) - 1.0, -1.0, 1.0))
    phi2 = 2.0 * math.pi * rng.random(n)
    return np.stack([phi1, Phi, phi2], axis=1)


def voronoi(n, n_grains, seed, h=VOXEL_MM):
    """Periodic Voronoi polycrystal.

    Centres uniform in the periodic box, voxel centres at (i + 1/2) h, grain
    id = nearest centre under the minimum-image distance.  Returns grain ids
    as int32 of length n0*n1*n2 (x fastest) and Euler angles (n_grains, 3)
    drawn from the same seeded stream.
    """
    n = tuple(int(x) for x in n)
    rng = np.random.default_rng(seed)
    L = np.array(n, dtype=np.float64) * h
    centres = rng.random((n_grains, 3)) * L
    euler = random_orientations(rng, n_grains)
    x = (np.arange(n[0]) + 0.5) * h
    y = (np.arange(n[1]) + 0.5) * h
    z = (np.arange(n[2]) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    try:
        from scipy.spatial import cKDTree
        tree = cKDTree(centres, boxsize=L)
        _, idx = tree.query(pts, k=1)
    except ImportError:  # pragma: no cover - scipy is present on both hosts
        idx = np.empty(len(pts), dtype=np.int64)
        for s in range(0, len(pts), 65536):
            d = pts[s:s + 65536, None, :] - centres[None, :, :]
            d -= L * np.round(d / L)
            idx[s:s + 65536] = np.argmin((d * d).sum(-1), axis=1)
    return idx.astype(np.int32), euler


def _power_assign(n, h, centres, w):
    """Grain id per voxel: argmin_i |x - c_i|^2 - w_i under the minimum image
    (separable over the axes), x fastest."""
    L = np.array(n, dtype=np.float64) * h
    d2 = []
    for a in range(3):
        x = (np.arange(n[a]) + 0.5) * h
        dx = x[:, None] - centres[None, :, a]
        dx -= L[a] * np.round(dx / L[a])
        d2.append(dx * dx)
    out = np.empty((n[2], n[1], n[0]), dtype=np.int32)
    base = d2[1][:, None, :] + d2[0][None, :, :] - w[None, None, :]  # (n1, n0, G)
    for k in range(n[2]):
        out[k] = np.argmin(base + d2[2][k][None, None, :], axis=2)
    return out.reshape(-1)


def lognormal_polycrystal(n, n_grains, sigma, seed, h=VOXEL_MM, iters=400):
    """Periodic polycrystal with log-normal grain sizes (Sec. 4.3 and 4.4:
    equivalent diameters log-normal, 0.1 standard deviation of the log).

    Target equivalent diameters d_i = exp(sigma Z_i), scaled so that the
    discs (n2 = 1, a plate) or balls they define fill the box; a periodic
    Laguerre (power) tessellation, voxel -> argmin_i |x - c_i|^2 - w_i under
    the minimum image with centres uniform in the box, whose weights are
    moved towards the targets (w_i += eta (R_target^2 - R_cell^2) with R the
    equivalent radius, eta 0.3 for the first half of ``iters`` rounds and 0.1
    after) until every cell is within 2 % (or half a voxel) of its target.  Returns grain ids (int32, x
    fastest), Euler angles (n_grains, 3) uniform on SO(3), and the target
    diameters in mm."""
    n = tuple(int(x) for x in n)
    rng = np.random.default_rng(seed)
    D = 2 if n[2] == 1 else 3
    L = np.array(n, dtype=np.float64) * h
    centres = rng.random((n_grains, 3)) * L
    if D == 2:
        centres[:, 2] = 0.5 * h
    euler = random_orientations(rng, n_grains)
    d = np.exp(sigma * rng.standard_normal(n_grains))
    unit = math.pi / 4 if D == 2 else math.pi / 6  # measure of a unit-diameter disc / ball
    d *= (np.prod(L[:D]) / (unit * np.sum(d ** D))) ** (1.0 / D)
    vox = h ** D
    r_t2 = (d / 2) ** 2
    target = unit * d ** D / vox
    w = np.zeros(n_grains)
    for it in range(iters):
        gid = _power_assign(n, h, centres, w)
        cnt = np.bincount(gid, minlength=n_grains).astype(np.float64)
        if np.all(np.abs(cnt - target) <= 0.02 * target + 0.5):
            return gid, euler, d
        r_c2 = (cnt * vox / unit) ** (2.0 / D) / 4
        w += (0.3 if it < iters // 2 else 0.1) * (r_t2 - r_c2)
    gid = _power_assign(n, h, centres, w)
    return gid, euler, d


def single_crystal(n, euler=(0.0, 0.0, 0.0)):
    N = int(np.prod(n))
    return np.zeros(N, dtype=np.int32), np.array([euler], dtype=np.float64)


def precrack_plane(n, x_range, y, value=1.0):
    """Pre-crack: phase field 1 and plasticity off on a one-voxel-thick plane
    y = const spanning x in x_range and every z (the paper's soft pre-crack
    region of Sec. 4.1 with stiffness g(1) = k)."""
    n0, n1, n2 = n
    phi = np.zeros((n2, n1, n0))
    phi[:, y, x_range[0]:x_range[1] + 1] = value
    mask = (phi > 0).astype(np.uint8)
    return phi.reshape(-1), mask.reshape(-1)


def soft_region(n, x_range, y_range, phi=None, mask=None):
    """Soft elastic region: phase field 1 and plasticity off on x in x_range,
    y in y_range (inclusive) and every z, added to ``phi`` / ``mask`` when
    given.  Its stiffness is g(1) = k (Sec. 4.1's pre-crack, Sec. 4.5's
    free-surface buffer)."""
    n0, n1, n2 = n
    ph = np.zeros((n2, n1, n0)) if phi is None else phi.reshape(n2, n1, n0).copy()
    ph[:, y_range[0]:y_range[1] + 1, x_range[0]:x_range[1] + 1] = 1.0
    m = (ph > 0).astype(np.uint8)
    if mask is not None:
        m |= mask.reshape(n2, n1, n0).astype(np.uint8)
    return ph.reshape(-1), m.reshape(-1)


def plate_precrack(n, length, thickness=2):
    """Central pre-crack of a plate: a soft region ``length`` voxels along x
    and ``thickness`` voxels along y, centred in the cell (Sec. 4.1: a
    central crack normal to the loading axis y)."""
    n0, n1, _ = n
    x0 = (n0 - length) // 2
    y0 = n1 // 2 - thickness // 2
    return soft_region(n, (x0, x0 + length - 1), (y0, y0 + thickness - 1))


def free_surface_buffer(n, thickness, phi=None, mask=None):
    """Free surfaces normal to y in the periodic cell: soft layers at
    y < thickness and y >= n1 - thickness (Sec. 4.5's buffer layers)."""
    n0, n1, _ = n
    phi, mask = soft_region(n, (0, n0 - 1), (0, thickness - 1), phi, mask)
    return soft_region(n, (0, n0 - 1), (n1 - thickness, n1 - 1), phi, mask)


def edge_notch(n, depth, width=2, thickness=0, phi=None, mask=None):
    """A notch from the lower free surface (inside a buffer of ``thickness``
    layers) into the sample at x = n0 / 2: ``width`` voxels along x, reaching
    ``depth`` voxels past the buffer along y."""
    n0 = n[0]
    x0 = n0 // 2 - width // 2
    return soft_region(n, (x0, x0 + width - 1), (thickness, thickness + depth - 1), phi, mask)


def bicrystal(n, boundary, euler_a, euler_b):
    """Periodic bicrystal plate: grain 1 is the band between two parallel
    grain boundaries, grain 0 the rest.  ``boundary`` = "perpendicular"
    (boundaries y = n1/4 and 3 n1/4, normal to the loading axis y) or
    "45" (boundaries x + y = n/4 and 3n/4 mod n, at 45 degrees to y; needs
    n0 = n1).  Returns grain ids (int32, x fastest) and Euler angles (2, 3)."""
    n0, n1, n2 = n
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    if boundary == "perpendicular":
        g = (y >= n1 // 4) & (y < n1 // 4 + n1 // 2)
    elif boundary == "45":
        if n0 != n1:
            raise ValueError("a periodic 45 degree boundary needs n0 = n1")
        s = (x + y) % n0
        g = (s >= n0 // 4) & (s < n0 // 4 + n0 // 2)
    else:
        raise ValueError(boundary)
    return g.astype(np.int32).reshape(-1), np.array([euler_a, euler_b], dtype=np.float64)


# Bunge angles (Q = Rz(phi1) Rx(Phi) Rz(phi2), lattice -> sample) that put a
# lattice direction along the sample y axis: [010] (the cube orientation) and
# [1 1 -1] (a <111> direction: Q^T e_y = (sin phi2 cos Phi, cos phi2 cos Phi,
# -sin Phi) with phi2 = 45 deg, sin Phi = 1 / sqrt 3).
EULER_Y100 = (0.0, 0.0, 0.0)
EULER_Y111 = (0.0, math.asin(1.0 / math.sqrt(3.0)), math.pi / 4)


def uniaxial_cycle_program(amplitude, inc_per_cycle, cycles, axis=1, eps_rate=1e-3):
    """Fully reversed (R = -1) triangle wave 0 -> +a -> 0 -> -a -> 0 per cycle,
    equal strain steps, dt = |d eps| / eps_rate.  Returns a list of
    (Fbar_target (9,), dt) with Fbar = I + eps e_axis (x) e_axis.
    inc_per_cycle = 4q samples the wave at t = i / inc_per_cycle; 4q + 2
    samples it at t = (i - 1/2) / inc_per_cycle, which puts both peaks on
    samples and keeps every step at 4a / inc_per_cycle (the first is half
    that), so no increment holds the strain (Delta Fbar = 0 leaves the
    relative Newton test with nothing but round-off to compare against).
    Other counts are rejected."""
    assert cycles >= 1
    eps = [0.0]
    if inc_per_cycle >= 4 and inc_per_cycle % 4 == 0:
        q = inc_per_cycle // 4
        de = amplitude / q
        for _ in range(cycles):
            for k in range(1, q + 1):
                eps.append(k * de)
            for k in range(q - 1, -q - 1, -1):
                eps.append(k * de)
            for k in range(-q + 1, 1):
                eps.append(k * de)
    elif inc_per_cycle >= 2 and inc_per_cycle % 4 == 2:
        for i in range(1, inc_per_cycle * cycles + 1):
            t = ((i - 0.5) % inc_per_cycle) / inc_per_cycle
            tri = 4 * t if t <= 0.25 else (2 - 4 * t if t <= 0.75 else 4 * t - 4)
            eps.append(amplitude * tri)
    else:
        raise ValueError("increments per cycle must be 4q or 4q + 2")
    prog = []
    for i in range(1, len(eps)):
        F = np.eye(3)
        F[axis, axis] += eps[i]
        prog.append((F.reshape(9).copy(), abs(eps[i] - eps[i - 1]) / eps_rate))
    return prog


def pulsating_cycle_program(eps_max, inc_per_cycle, cycles, axis=1, eps_rate=1e-3):
    """Strain ratio R = 0 triangle wave 0 -> eps_max -> 0 per cycle (Sec. 4's
    loading), equal strain steps of 2 eps_max / inc_per_cycle sampled at
    t = i / inc_per_cycle (the peak and the zero are samples, no increment
    holds the strain), dt = |d eps| / eps_rate.  inc_per_cycle must be even.
    Returns a list of (Fbar_target (9,), dt) with Fbar_target =
    I + eps e_axis (x) e_axis; under uniaxial stress only the axial component
    is a target, the lateral ones are solved for."""
    assert cycles >= 1
    if inc_per_cycle < 2 or inc_per_cycle % 2:
        raise ValueError("increments per cycle must be even")
    q = inc_per_cycle // 2
    de = eps_max / q
    eps = [0.0]
    for _ in range(cycles):
        eps += [k * de for k in range(1, q + 1)] + [k * de for k in range(q - 1, -1, -1)]
    prog = []
    for i in range(1, len(eps)):
        F = np.eye(3)
        F[axis, axis] += eps[i]
        prog.append((F.reshape(9).copy(), abs(eps[i] - eps[i - 1]) / eps_rate))
    return prog


def uniaxial_stress_mask(axis=1):
    """Stress mask (9,) for uniaxial stress along ``axis``: the two lateral
    normal stresses prescribed (zero), the axial stretch and the off-diagonal
    F prescribed (no shear, no rigid rotation)."""
    m = np.zeros(9, dtype=np.int32)
    for c in range(3):
        if c != axis:
            m[4 * c] = 1
    return m


def increment_args(cfg, k, Fbar_prev=None):
    """(args, kwargs) of ``run_increment`` for increment k of a config's
    loading.  Strain control: ((Fbar, dt), {}).  Under a stress mask the
    stress-controlled components of Fbar start from the previous increment's
    solved values (``Fbar_prev``, the stats' Fbar; the target's at the first
    increment) and Pbar / stress_mask are passed."""
    Fb, dt = cfg["program"][k]
    m = cfg.get("stress_mask")
    if m is None:
        return (Fb, dt), {}
    guess = Fb.copy() if Fbar_prev is None else np.where(m == 1, Fbar_prev, Fb)
    return (guess, dt), {"Pbar": np.array(cfg["Pbar"], dtype=np.float64), "stress_mask": m}


# The workloads: grids, grain counts, loading (Sec. 4 shapes).
CONFIGS = {
    "sx16": dict(n=(16, 16, 16), grains=1, amplitude=0.005, inc_per_cycle=20, cycles=1,
                 precrack=True, seed=1001),
    "poly64": dict(n=(64, 64, 64), grains=50, amplitude=0.006, inc_per_cycle=40, cycles=3,
                   precrack=False, seed=1002),
    "poly128": dict(n=(128, 128, 128), grains=200, amplitude=0.007, inc_per_cycle=40,
                    cycles=10, precrack=False, seed=1003, probe=(3, 6)),
    "batch32": dict(sizes=(32, 48, 64, 96), count=32, grains=(20, 150), amplitude=0.006,
                    inc_per_cycle=30, cycles=2, seed=2000),
    # the same loading on 32 small cells of one size (one lockstep class)
    "batch32x32": dict(sizes=(32,), count=32, grains=(20, 150), amplitude=0.006,
                       inc_per_cycle=30, cycles=2, seed=3000),
    "poly64_r0": dict(n=(64, 64, 64), grains=50, amplitude=0.02, inc_per_cycle=40, cycles=2,
                      precrack=False, seed=1002, ratio=0, control="uniaxial_stress"),
    # 2-D plates (one voxel thick, plane stress through mixed control)
    "plate256_sx100": dict(n=(256, 256, 1), plate="single", euler=EULER_Y100, crack=64,
                           amplitude=0.02, inc_per_cycle=40, cycles=2, ratio=0, seed=0),
    "plate256_sx111": dict(n=(256, 256, 1), plate="single", euler=EULER_Y111, crack=64,
                           amplitude=0.02, inc_per_cycle=40, cycles=2, ratio=0, seed=0),
    "plate256_bx90": dict(n=(256, 256, 1), plate="bicrystal", boundary="perpendicular",
                          amplitude=0.02, inc_per_cycle=40, cycles=2, ratio=0,
                          seed=1006),
    "plate256_bx45": dict(n=(256, 256, 1), plate="bicrystal", boundary="45",
                          amplitude=0.02, inc_per_cycle=40, cycles=2, ratio=0,
                          seed=1006),
    "plate256_poly62": dict(n=(256, 256, 1), plate="lognormal", grains=62, sigma=0.1,
                            amplitude=0.02, inc_per_cycle=40, cycles=2, ratio=0, seed=1008),
    "poly128_ln64": dict(n=(128, 128, 128), grains=64, sigma=0.1, amplitude=0.02,
                         inc_per_cycle=40, cycles=2, precrack=False, seed=1009, ratio=0,
                         control="uniaxial_stress"),
    "plate256x128_notch": dict(n=(256, 128, 1), plate="notched", grains=40, buffer=8,
                               notch=16, amplitude=0.01, inc_per_cycle=40, cycles=2, ratio=0,
                               seed=1007),
    # (the benchmark's kernel probe runs increments 4-6 here: the plastic
    # peak increments take thousands of Krylov iterations at this size)
    "poly256": dict(n=(256, 256, 256), grains=1000, amplitude=0.007, inc_per_cycle=40,
                    cycles=5, precrack=False, seed=1005, probe=(3, 6)),
    # the timed workload with damage switched on early (softer slip,
    # full storage of the plastic work, G_crit reached at the first tensile
    # peak): the drive turns positive in the second cycle
    "poly64_damage": dict(n=(64, 64, 64), grains=50, amplitude=0.006, inc_per_cycle=40,
                          cycles=3, precrack=False, seed=1002,
                          material=dict(tau_c0=250.0, xi_store=1.0, G_crit=7e-4),
                          options=dict(max_cutbacks=4)),
    # the 128^3 / 200-grain polycrystal with the stored-energy fraction
    # calibrated (reading A4) so that W_crit is reached in its second cycle;
    # cut-back at the load peaks (their Krylov solves stall at full steps)
    "poly128_damage": dict(n=(128, 128, 128), grains=200, amplitude=0.007, inc_per_cycle=40,
                           cycles=10, precrack=False, seed=1003,
                           material=dict(xi_store=0.25),
                           options=dict(max_cutbacks=4)),
}


def build_config(name, n_override=None, cycles=None):
    """Grain ids, Euler angles, phi0, elastic mask and loading for one config.

    ``sx16``'s pre-crack is the plane y = 8, x = 6..9, all z (a 4 x 16 plane
    at mid-height, one voxel thick), scaled with the grid when ``n_override``
    is given."""
    c = CONFIGS[name]
    n = tuple(n_override) if n_override else c["n"]
    if "plate" in c:
        return _plate_config(c, n, cycles)
    if c["grains"] == 1:
        gid, eul = single_crystal(n)
    elif "sigma" in c:
        gid, eul, _ = lognormal_polycrystal(n, c["grains"], c["sigma"], c["seed"])
    else:
        gid, eul = voronoi(n, c["grains"], c["seed"])
    phi0 = mask = None
    if c.get("precrack"):
        s = n[0] / 16.0
        x0, x1 = int(round(6 * s)), int(round(10 * s)) - 1
        phi0, mask = precrack_plane(n, (x0, x1), n[1] // 2)
    ncyc = int(cycles) if cycles else c["cycles"]
    if c.get("ratio", -1) == 0:
        prog = pulsating_cycle_program(c["amplitude"], c["inc_per_cycle"], ncyc)
    else:
        prog = uniaxial_cycle_program(c["amplitude"], c["inc_per_cycle"], ncyc)
    out = dict(n=n, h=VOXEL_MM, grain_ids=gid, euler=eul, phi0=phi0, elastic_only=mask,
               program=prog, stress_mask=None, Pbar=None, material=dict(c.get("material", {})),
               options=dict(c.get("options", {})))
    if "probe" in c:
        out["probe"] = tuple(c["probe"])
    if c.get("control") == "uniaxial_stress":
        out["stress_mask"] = uniaxial_stress_mask(1)
        out["Pbar"] = np.zeros(9)
    return out


def _plate_config(c, n, cycles=None):
    """Plates of Sec. 4 (2-D, one voxel thick): single crystal with a central
    soft pre-crack (length scaled with n0), periodic bicrystal, polycrystal
    with log-normal grain sizes (Sec. 4.3), notched
    polycrystal between free-surface buffer layers (loaded along x).  Plane
    stress: the lateral in-plane and the out-of-plane normal mean stresses
    are held at zero."""
    phi0 = mask = None
    axis = 1
    if c["plate"] == "single":
        gid, eul = single_crystal(n, c["euler"])
        phi0, mask = plate_precrack(n, max(2, c["crack"] * n[0] // 256))
    elif c["plate"] == "lognormal":
        gid, eul, _ = lognormal_polycrystal(n, c["grains"], c["sigma"], c["seed"])
    elif c["plate"] == "bicrystal":
        rng = np.random.default_rng(c["seed"])
        ea, eb = random_orientations(rng, 2)
        gid, eul = bicrystal(n, c["boundary"], ea, eb)
    else:
        gid, eul = voronoi(n, c["grains"], c["seed"])
        b = max(1, c["buffer"] * n[1] // 128)
        phi0, mask = free_surface_buffer(n, b)
        phi0, mask = edge_notch(n, max(1, c["notch"] * n[1] // 128), 2, b, phi0, mask)
        axis = 0
    if c.get("ratio", -1) == 0:
        prog = pulsating_cycle_program(c["amplitude"], c["inc_per_cycle"],
                                       int(cycles) if cycles else c["cycles"], axis)
    else:
        prog = uniaxial_cycle_program(c["amplitude"], c["inc_per_cycle"],
                                      int(cycles) if cycles else c["cycles"], axis)
    return dict(n=n, h=VOXEL_MM, grain_ids=gid, euler=eul, phi0=phi0, elastic_only=mask,
                program=prog, stress_mask=uniaxial_stress_mask(axis), Pbar=np.zeros(9),
                material={}, options={})


def batch_configs(seed=2000, count=32, sizes=(32, 48, 64, 96), grains=(20, 150)):
    """The batched-RVE workload: ``count`` polycrystals with grids drawn from
    ``sizes`` (cubes) and grain counts uniform in ``grains``, seed + r each."""
    out = []
    for r in range(count):
        rng = np.random.default_rng(seed + r)
        s = int(sizes[rng.integers(len(sizes))])
        g = int(rng.integers(grains[0], grains[1] + 1))
        gid, eul = voronoi((s, s, s), g, seed + 10000 + r)
        out.append(dict(n=(s, s, s), h=VOXEL_MM, grain_ids=gid, euler=eul, phi0=None,
                        elastic_only=None))
    return out
