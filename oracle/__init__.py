"""FP64 CPU oracle of the particle-deposition hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The CUDA library never does, and this
package never imports the library: the two share no code.  The particle step is
plain C++ (``pdq_oracle.cpp``) loaded through ctypes; the multi-fidelity
estimators are plain numpy (``oracle.mfmc``).
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdq_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libpdq_oracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with the host C++ compiler (plain -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class Phys(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "nu", "radius", "re_tau", "u_bulk", "rho_p", "rho_f", "eps0", "qmax_coef",
        "hamaker0", "delta_min", "young", "delta_c", "sigma_y0", "g",
        "restitution", "tau_col_steps", "neg_charge_frac", "contact_scale")]


class Field(C.Structure):
    _fields_ = [("r_plus", C.c_double), ("l_plus", C.c_double),
                ("n_r", C.c_int32), ("n_th", C.c_int32), ("n_z", C.c_int32), ("n_modes", C.c_int32),
                ("u_rms", C.c_double), ("beta", C.c_double), ("kappa", C.c_double),
                ("b_log", C.c_double), ("k_min", C.c_double), ("k_max", C.c_double)]


class Cfg(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("mode", C.c_int32),
                ("forces", C.c_int32), ("window_start", C.c_int64), ("smooth_eps", C.c_double),
                ("stick_eps", C.c_double)]


F_DRAG, F_GRAV, F_COUL, F_IMAGE, F_VDW = 1, 2, 4, 8, 16
F_ALL = 31
F_COLLIDE, F_VDWPP = 32, 64          # particle-particle contact (soft-sphere collisions, Eq. vdw)
F_CONTACT = F_COLLIDE | F_VDWPP
STICK, REBOUND = 0, 1

_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P, Fp, Cp = C.POINTER(Phys), C.POINTER(Field), C.POINTER(Cfg)
        sig = {
            "orc_phys_default": (None, [P]),
            "orc_class_table": (None, [P, C.c_int, _D, _D]),
            "orc_vdw_pp": (C.c_double, [C.c_double] * 3),
            "orc_coulomb_pp": (C.c_double, [C.c_double] * 4),
            "orc_wall_average": (C.c_double, [C.c_int] + [C.c_double] * 6),
            "orc_ycross": (C.c_double, [C.c_double, C.c_double]),
            "orc_mean_profile": (C.c_double, [C.c_double] * 4),
            "orc_field_modes": (None, [Fp, C.c_uint64, _D]),
            "orc_field_velocity": (None, [Fp, _D, C.c_int, _D, _D]),
            "orc_field_grid": (None, [Fp, _D, _D]),
            "orc_interp": (None, [Fp, _D, C.c_int, _D, _D]),
            "orc_seed": (C.c_int, [P, Fp, C.c_int, _D, C.c_double, C.c_uint64, C.c_int, _I64, _D,
                                   _D, _D, _D, _D, _D, _D, _D, _I32, _I32, _I32, C.c_int]),
            "orc_run": (C.c_int, [P, Fp, _D, Cp, C.c_int, _D, C.c_int, _I64, _D, C.c_int64, C.c_int64,
                                  _D, _D, _D, _D, _D, _D, _D, _I32, _I32, _I64, _I64]),
            "orc_vdep": (None, [C.c_int, _I64, _I64, C.c_double, C.c_double, _D]),
            "orc_smooth_run": (C.c_int, [P, Fp, _D, Cp, C.c_int, _D, C.c_int, _I64, _D, C.c_int64,
                                         _D, _D, _D, _D, _I32, C.c_void_p, C.c_void_p, C.c_int, _D, _D]),
            "orc_coulomb_accel": (None, [P, Fp, C.c_int, _D, C.c_int, _D, _D, _D, _D, _I32, _I32, _D]),
            "orc_wall_accel": (None, [P, Fp, Cp, C.c_int, _D, C.c_int, _D, _D, _D, _I32, C.c_double, _D]),
            "orc_cor": (C.c_double, [P, C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_philox": (None, [_U32, _U32, _U32]),
            "orc_boot_indices": (None, [C.c_uint64, C.c_uint32, C.c_int, _I64, _I64]),
            "orc_num_threads": (C.c_int, []),
            "orc_capture_factor": (C.c_double, [P, Fp]),
            "orc_coulomb_periodic": (None, [C.c_int, _D, _D, _D, _D, _I32, C.c_double, C.c_double, C.c_int, _D]),
            "orc_run_ext": (C.c_int, [P, Fp, _D, Cp, C.c_int, _D, C.c_int, _I64, _D, C.c_int64, _D,
                                      _D, _D, _D, _D, _D, _D, _D, _I32, _I32, _I64, _I64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# Descriptors
# ---------------------------------------------------------------------------
def phys():
    p = Phys()
    lib().orc_phys_default(C.byref(p))
    return p


def field_desc(n_r=64, n_th=32, n_z=64, n_modes=64, r_plus=180.0, l_over_r=4.0, u_rms=1.0,
               beta=2.0, kappa=0.41, b_log=5.2, lam_min=20.0, lam_max=400.0):
    """Synthetic-field descriptor; the wavenumber shell spans wavelengths lam_min..lam_max (wall units)."""
    return Field(r_plus, l_over_r * r_plus, n_r, n_th, n_z, n_modes, u_rms, beta, kappa, b_log,
                 2 * np.pi / lam_max, 2 * np.pi / lam_min)


def cfg(dt, forces=F_ALL, mode=STICK, gravity=(0.0, 0.0, 1.0), window_start=0, smooth_eps=0.0, stick_eps=0.0):
    c = Cfg()
    c.dt = dt
    for k in range(3):
        c.gravity[k] = gravity[k]
    c.mode, c.forces, c.window_start, c.smooth_eps, c.stick_eps = mode, forces, window_start, smooth_eps, stick_eps
    return c


def class_table(st_plus, p=None):
    """Rows [tau+, d+, d (m), mass (kg), (d/1um)^2] per class."""
    p = p or phys()
    st = np.ascontiguousarray(st_plus, np.float64)
    out = np.zeros((len(st), 5))
    lib().orc_class_table(C.byref(p), len(st), st, out)
    return out


# ---------------------------------------------------------------------------
# Field
# ---------------------------------------------------------------------------
def field_modes(f, seed):
    m = np.zeros((f.n_modes, 7))
    lib().orc_field_modes(C.byref(f), seed, m)
    return m


def field_velocity(f, modes, xyz):
    xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
    out = np.zeros_like(xyz)
    lib().orc_field_velocity(C.byref(f), np.ascontiguousarray(modes), len(xyz), xyz, out)
    return out


def field_grid(f, modes):
    g = np.zeros((f.n_z, f.n_th, f.n_r, 3))
    lib().orc_field_grid(C.byref(f), np.ascontiguousarray(modes), g)
    return g


def interp(f, grid, xyz):
    xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
    out = np.zeros_like(xyz)
    lib().orc_interp(C.byref(f), np.ascontiguousarray(grid), len(xyz), xyz, out)
    return out


# ---------------------------------------------------------------------------
# Particles
# ---------------------------------------------------------------------------
class State:
    """Plain per-particle arrays of all samples (sample s = [offset[s], offset[s+1]))."""

    def __init__(self, n):
        self.x, self.y, self.z = (np.zeros(n) for _ in range(3))
        self.vx, self.vy, self.vz = (np.zeros(n) for _ in range(3))
        self.q = np.zeros(n)
        self.alive = np.ones(n, np.int32)
        self.cls = np.zeros(n, np.int32)
        self.id = np.zeros(n, np.int32)

    def copy(self):
        s = State(0)
        for k, v in self.__dict__.items():
            setattr(s, k, v.copy())
        return s


def seed(f, st_plus, counts, params, seed_value, charge_sigma=0.0, p=None, independent=False):
    """Initial state of S samples with counts[s] particles; params [S,3] = (xi, zeta, theta).
    independent: a Philox stream per sample (counter word 3 = s + 1) instead of common random numbers."""
    p = p or phys()
    counts = np.asarray(counts, np.int64)
    offset = np.zeros(len(counts) + 1, np.int64)
    offset[1:] = np.cumsum(counts)
    st = State(int(offset[-1]))
    prm = np.ascontiguousarray(params, np.float64).reshape(-1, 3)
    stp = np.ascontiguousarray(st_plus, np.float64)
    rc = lib().orc_seed(C.byref(p), C.byref(f), len(stp), stp, charge_sigma, seed_value, len(counts),
                        offset, prm, st.x, st.y, st.z, st.vx, st.vy, st.vz, st.q, st.alive, st.cls, st.id,
                        int(independent))
    assert rc == 0
    return st, offset


def run(f, grid, c, st_plus, offset, params, state, n_steps, step0=0, tallies=None, p=None):
    """Advance ``state`` in place; returns (ndep, nalive) tallies [S, C] (accumulated)."""
    p = p or phys()
    S, nc = len(offset) - 1, len(st_plus)
    if tallies is None:
        tallies = (np.zeros((S, nc), np.int64), np.zeros((S, nc), np.int64))
    ndep, nal = tallies
    rc = lib().orc_run(C.byref(p), C.byref(f), np.ascontiguousarray(grid), C.byref(c), nc,
                       np.ascontiguousarray(st_plus, np.float64), S, np.ascontiguousarray(offset, np.int64),
                       np.ascontiguousarray(params, np.float64).reshape(-1, 3), step0, n_steps,
                       state.x, state.y, state.z, state.vx, state.vy, state.vz, state.q, state.alive,
                       state.cls, ndep, nal)
    assert rc == 0
    return ndep, nal


def run_ext(f, grid, c, st_plus, offset, params, state, ext, step0=0, tallies=None, p=None):
    """One step with given Coulomb sums ext [N, 3] instead of the all-pairs loop."""
    p = p or phys()
    S, nc = len(offset) - 1, len(st_plus)
    if tallies is None:
        tallies = (np.zeros((S, nc), np.int64), np.zeros((S, nc), np.int64))
    ndep, nal = tallies
    rc = lib().orc_run_ext(C.byref(p), C.byref(f), np.ascontiguousarray(grid), C.byref(c), nc,
                           np.ascontiguousarray(st_plus, np.float64), S, np.ascontiguousarray(offset, np.int64),
                           np.ascontiguousarray(params, np.float64).reshape(-1, 3), step0,
                           np.ascontiguousarray(ext, np.float64).reshape(-1, 3),
                           state.x, state.y, state.z, state.vx, state.vy, state.vz, state.q, state.alive,
                           state.cls, ndep, nal)
    assert rc == 0
    return ndep, nal


def coulomb_periodic(x, y, z, q, L, contact, n_img=2000, alive=None):
    """Coulomb sums over all periodic images along z (exact electrostatics of the periodic pipe)."""
    n = len(x)
    alive = np.ones(n, np.int32) if alive is None else np.ascontiguousarray(alive, np.int32)
    s = np.zeros((n, 3))
    lib().orc_coulomb_periodic(n, *(np.ascontiguousarray(v, np.float64) for v in (x, y, z, q)), alive, L, contact,
                               n_img, s)
    return s


def vdep(ndep, nalive, dt, r_plus=180.0):
    ndep = np.ascontiguousarray(ndep, np.int64)
    out = np.zeros(ndep.shape)
    lib().orc_vdep(ndep.size, ndep, np.ascontiguousarray(nalive, np.int64), dt, r_plus, out)
    return out


def smooth_run(f, grid, c, st_plus, offset, params, x0, y0, z0, qhat, cls, n_steps, want_grad=True, p=None,
               v0=None, w0=None):
    """Smoothed functional J [S, C] and (if want_grad) dJ/d(xi, zeta, theta) [S, C, 3].

    The particles start at (x0, y0, z0) with velocities v0 [N, 3] (None: at rest) and weights
    w0 [N] (None: 1); charge xi * qhat.
    """
    p = p or phys()
    S, nc = len(offset) - 1, len(st_plus)
    J = np.zeros((S, nc))
    dJ = np.zeros((S, nc, 3))
    v0 = None if v0 is None else np.ascontiguousarray(v0, np.float64).reshape(-1, 3)
    w0 = None if w0 is None else np.ascontiguousarray(w0, np.float64)
    rc = lib().orc_smooth_run(C.byref(p), C.byref(f), np.ascontiguousarray(grid), C.byref(c), nc,
                              np.ascontiguousarray(st_plus, np.float64), S, np.ascontiguousarray(offset, np.int64),
                              np.ascontiguousarray(params, np.float64).reshape(-1, 3), n_steps,
                              *(np.ascontiguousarray(a, np.float64) for a in (x0, y0, z0, qhat)),
                              np.ascontiguousarray(cls, np.int32),
                              None if v0 is None else v0.ctypes.data, None if w0 is None else w0.ctypes.data,
                              int(want_grad), J, dJ)
    assert rc == 0
    return J, dJ


def coulomb_accel(f, st_plus, x, y, z, q, cls, alive=None, p=None):
    p = p or phys()
    n = len(x)
    alive = np.ones(n, np.int32) if alive is None else np.ascontiguousarray(alive, np.int32)
    a = np.zeros((n, 3))
    lib().orc_coulomb_accel(C.byref(p), C.byref(f), len(st_plus), np.ascontiguousarray(st_plus, np.float64), n,
                            *(np.ascontiguousarray(v, np.float64) for v in (x, y, z, q)),
                            np.ascontiguousarray(cls, np.int32), alive, a)
    return a


def wall_accel(f, c, st_plus, x, y, q, cls, zeta, p=None):
    p = p or phys()
    n = len(x)
    a = np.zeros((n, 3))
    lib().orc_wall_accel(C.byref(p), C.byref(f), C.byref(c), len(st_plus),
                         np.ascontiguousarray(st_plus, np.float64), n,
                         *(np.ascontiguousarray(v, np.float64) for v in (x, y, q)),
                         np.ascontiguousarray(cls, np.int32), zeta, a)
    return a


def cor(st_plus, zeta, theta, vn1, p=None):
    p = p or phys()
    return lib().orc_cor(C.byref(p), st_plus, zeta, theta, vn1)


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def boot_indices(seed, b, m):
    """Group indices of bootstrap replicate b for nested counts m (resampled within each nesting block)."""
    m = np.ascontiguousarray(m, np.int64)
    out = np.zeros(int(m[-1]), np.int64)
    lib().orc_boot_indices(seed, b, len(m), m, out)
    return out


def vdw_pp(A, d, delta):
    return lib().orc_vdw_pp(A, d, delta)


def coulomb_pp(q1, q2, r, eps0=8.854e-12):
    return lib().orc_coulomb_pp(q1, q2, r, eps0)


def wall_average(kind, d, q, A, D=0.02, eps0=8.854e-12, delta_min=1e-9):
    return lib().orc_wall_average(kind, D, d, q, A, eps0, delta_min)


def ycross(kappa=0.41, b_log=5.2):
    return lib().orc_ycross(kappa, b_log)


def mean_profile(yplus, kappa=0.41, b_log=5.2):
    yc = ycross(kappa, b_log)
    return lib().orc_mean_profile(yplus, kappa, b_log, yc)


def num_threads():
    return lib().orc_num_threads()


def capture_factor(f, p=None):
    p = p or phys()
    return lib().orc_capture_factor(C.byref(p), C.byref(f))
