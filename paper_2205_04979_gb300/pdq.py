"""Thin ctypes binding of libpdq (include/pdq.h).

Argument marshalling only: torch provides device memory and streams, every
step of the particle path runs in libpdq's kernels.  Importing this module
fails loudly when libpdq.so has not been built; there is no CPU fallback.
"""
import ctypes as C
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdq.so")

PDQ_OK = 0
FP64, MIXED = 0, 1
STICK, REBOUND = 0, 1
F_DRAG, F_GRAVITY, F_COULOMB, F_IMAGE, F_VDW, F_ALL = 1, 2, 4, 8, 16, 31
F_COLLIDE, F_VDW_PP = 32, 64        # particle-particle contact (collisions, Eq. vdw between particles)
F_CONTACT = F_COLLIDE | F_VDW_PP
MAX_CLASSES = 16


class PdqError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s failed: %s (%d)" % (where, lib().pdq_strerror(status).decode(), status))
        self.status = status


class Phys(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "nu", "radius", "re_tau", "u_bulk", "rho_p", "rho_f", "eps0", "q_unit", "hamaker0", "delta_min",
        "young", "delta_c", "sigma_y0", "g", "restitution", "tau_col_steps", "neg_charge_frac", "contact_scale")]


class FieldDesc(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_th", C.c_int32), ("n_z", C.c_int32), ("n_modes", C.c_int32),
                ("r_plus", C.c_double), ("l_plus", C.c_double), ("u_rms", C.c_double), ("beta", C.c_double),
                ("kappa", C.c_double), ("b_log", C.c_double), ("k_min", C.c_double), ("k_max", C.c_double)]


class StateStruct(C.Structure):
    _fields_ = [("precision", C.c_int32), ("cur", C.c_int32), ("n_samples", C.c_int32), ("n_classes", C.c_int32),
                ("st_plus", C.c_double * MAX_CLASSES), ("capacity", C.c_int64), ("step", C.c_int64),
                ("offset", C.c_void_p), ("count", C.c_void_p), ("pos", C.c_void_p * 2), ("vel", C.c_void_p * 2),
                ("xy", C.c_void_p * 2), ("tag", C.c_void_p), ("ctl", C.c_void_p)]


class StepCfg(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("mode", C.c_int32), ("forces", C.c_int32),
                ("window_start", C.c_int64), ("compact_every", C.c_int32), ("block", C.c_int32),
                ("use_graph", C.c_int32), ("variant", C.c_int32)]


class P3MDesc(C.Structure):
    _fields_ = [("M", C.c_int32), ("Nz", C.c_int32), ("alpha", C.c_double), ("r_cut", C.c_double),
                ("n_img", C.c_int32), ("pad", C.c_int32)]


class BatchStruct(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_samples", C.c_int32), ("n_classes", C.c_int32), ("pad", C.c_int32),
                ("st_plus", C.c_double * MAX_CLASSES), ("capacity", C.c_int64), ("offset", C.c_void_p)]


class LfDesc(C.Structure):
    _fields_ = [("n_y", C.c_int32), ("precision", C.c_int32), ("stretch", C.c_double), ("t_lagr", C.c_double),
                ("temperature", C.c_double), ("vdw_cutoff", C.c_double)]


class TallyStruct(C.Structure):
    _fields_ = [("n_dep", C.c_void_p), ("n_alive", C.c_void_p)]


_lib = None


def lib():
    """Load libpdq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpdq.so is not built (%s); run __graft_entry__.build() on a machine with nvcc"
                              % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "pdq_strerror": (C.c_char_p, [C.c_int]),
            "pdq_version": (C.c_int, []),
            "pdq_phys_default": (None, [C.POINTER(Phys)]),
            "pdq_create_pipe_field": (C.c_int, [C.POINTER(FieldDesc), C.c_uint64, P, C.POINTER(P)]),
            "pdq_destroy_pipe_field": (C.c_int, [P]),
            "pdq_field_views": (C.c_int, [P, C.POINTER(FieldDesc), P, P, P]),
            "pdq_field_copy": (C.c_int, [P, P, P, P, P]),
            "pdq_seed_particles": (C.c_int, [P, C.POINTER(Phys), C.c_double, C.c_uint64, P,
                                             C.POINTER(StateStruct), P]),
            "pdq_seed_particles_independent": (C.c_int, [P, C.POINTER(Phys), C.c_double, C.c_uint64, P,
                                                         C.POINTER(StateStruct), P]),
            "pdq_step_workspace_size": (C.c_int, [C.POINTER(StateStruct), C.POINTER(StepCfg),
                                                  C.POINTER(C.c_size_t)]),
            "pdq_step_particles": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P, C.POINTER(StepCfg),
                                             C.c_int64, C.POINTER(TallyStruct), P, C.c_size_t, P]),
            "pdq_step_particles_noalloc": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P,
                                                     C.POINTER(StepCfg), C.c_int64, C.POINTER(TallyStruct), P]),
            "pdq_compact": (C.c_int, [C.POINTER(StateStruct), P]),
            "pdq_release_graphs": (C.c_int, []),
            "pdq_autotune_workspace_size": (C.c_int, [C.POINTER(StateStruct), C.POINTER(C.c_size_t)]),
            "pdq_autotune": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P, C.POINTER(StepCfg), P,
                                       C.c_size_t, P]),
            "pdq_check_state": (C.c_int, [C.POINTER(StateStruct), P]),
            "pdq_deposition_tally": (C.c_int, [C.POINTER(TallyStruct), C.c_int32, C.c_int32, C.c_double,
                                               C.c_double, P, P, P, P]),
            "pdq_mfmc_allocate": (C.c_int, [C.c_int32, P, P, P, C.c_double, C.c_int32, P, P, P, P]),
            "pdq_adjoint_workspace_size": (C.c_int, [C.POINTER(BatchStruct), C.c_int64, C.c_int32,
                                                     C.POINTER(C.c_size_t)]),
            "pdq_adjoint_state_workspace_size": (C.c_int, [C.POINTER(StateStruct), C.c_int64, C.c_int32,
                                                           C.POINTER(C.c_size_t)]),
            "pdq_adjoint_stored_sums_size": (C.c_int, [C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]),
            "pdq_adjoint_run": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P, C.POINTER(StepCfg),
                                          C.c_int64, C.c_int32, C.c_double, C.c_double, C.c_int32, P, P, P, P,
                                          C.c_size_t, P]),
            "pdq_adjoint_run_seeded": (C.c_int, [P, C.POINTER(Phys), C.POINTER(BatchStruct), P, C.c_double,
                                                 C.c_uint64, C.POINTER(StepCfg), C.c_int64, C.c_int32, C.c_double,
                                                 C.c_double, C.c_int32, P, P, P, P, C.c_size_t, P]),
            "pdq_adjoint_reverse": (C.c_int, [P, C.POINTER(Phys), C.POINTER(BatchStruct), P, C.POINTER(StepCfg),
                                              C.c_int64, C.c_int32, C.c_double, C.c_double, C.c_int32, P, P, P,
                                              C.c_size_t, P]),
            "pdq_dgsm_workspace_size": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
            "pdq_dgsm_bounds": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P, C.c_size_t, P]),
            "pdq_capture_efficiency": (C.c_int, [P, C.POINTER(Phys), P, C.c_int64, P, P]),
            "pdq_p3m_create": (C.c_int, [P, C.POINTER(P3MDesc), C.c_int64, P, C.POINTER(C.c_void_p)]),
            "pdq_p3m_destroy": (C.c_int, [P]),
            "pdq_p3m_params": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int32)]),
            "pdq_p3m_coulomb": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P, P]),
            "pdq_step_particles_p3m": (C.c_int, [P, C.POINTER(Phys), C.POINTER(StateStruct), P, C.POINTER(StepCfg),
                                                 C.c_int64, C.POINTER(TallyStruct), P, P, C.c_size_t, P]),
            "pdq_lf_desc_default": (None, [C.POINTER(LfDesc)]),
            "pdq_lf_fluid_variance": (C.c_int, [P, P, P]),
            "pdq_lf_vdep": (C.c_int, [P, C.POINTER(Phys), C.POINTER(LfDesc), P, C.c_int32, P, C.c_int64, P, P, P]),
            "pdq_mfmc_workspace_size": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                                  C.POINTER(C.c_size_t)]),
            "pdq_mfmc_sobol": (C.c_int, [C.c_int32, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                         P, P, P, P, P, P, P, C.c_size_t, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


def _check(rc, where):
    if rc != PDQ_OK:
        raise PdqError(rc, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def phys_default():
    p = Phys()
    lib().pdq_phys_default(C.byref(p))
    return p


def field_desc(n_r=64, n_th=32, n_z=64, n_modes=64, r_plus=180.0, l_over_r=4.0, u_rms=1.0, beta=2.0,
               kappa=0.41, b_log=5.2, lam_min=20.0, lam_max=400.0):
    """Field descriptor; the mode shell spans wavelengths lam_min..lam_max (wall units)."""
    return FieldDesc(n_r, n_th, n_z, n_modes, r_plus, l_over_r * r_plus, u_rms, beta, kappa, b_log,
                     2 * math.pi / lam_max, 2 * math.pi / lam_min)


class Field:
    """Owning wrapper of a pdq_field handle."""

    def __init__(self, desc, seed, stream=None):
        self.desc = desc
        h = C.c_void_p()
        _check(lib().pdq_create_pipe_field(C.byref(desc), seed, _stream(stream), C.byref(h)), "create_pipe_field")
        self.handle = h

    def grids(self, stream=None):
        d = self.desc
        g64 = torch.empty((d.n_z, d.n_th, d.n_r, 4), dtype=torch.float64, device="cuda")
        g32 = torch.empty((d.n_z, d.n_th, d.n_r, 4), dtype=torch.float32, device="cuda")
        modes = torch.empty((max(d.n_modes, 1), 7), dtype=torch.float64, device="cuda")
        _check(lib().pdq_field_copy(self.handle, _ptr(g64), _ptr(g32), _ptr(modes), _stream(stream)), "field_copy")
        return g64, g32, modes[: d.n_modes]

    def close(self):
        if self.handle:
            lib().pdq_destroy_pipe_field(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class P3M:
    """Owning wrapper of a pdq_p3m plan (P3M electrostatics of the periodic pipe)."""

    def __init__(self, field, M=123, Nz=256, alpha=0.0, r_cut=0.0, n_img=0, max_particles=1, stream=None):
        d = P3MDesc()
        d.M, d.Nz, d.alpha, d.r_cut, d.n_img = M, Nz, alpha, r_cut, n_img
        h = C.c_void_p()
        _check(lib().pdq_p3m_create(field.handle, C.byref(d), int(max_particles), _stream(stream), C.byref(h)),
               "p3m_create")
        self.handle = h
        a, rc, ni, nx = C.c_double(), C.c_double(), C.c_int32(), C.c_int32()
        _check(lib().pdq_p3m_params(h, C.byref(a), C.byref(rc), C.byref(ni), C.byref(nx)), "p3m_params")
        self.alpha, self.r_cut, self.n_img, self.nx = a.value, rc.value, ni.value, nx.value

    def coulomb(self, phys, state, stream=None):
        """P3M Coulomb sums [capacity, 3] (float64) of the current state."""
        out = torch.empty((max(state.st.capacity, 1), 3), dtype=torch.float64, device="cuda")
        _check(lib().pdq_p3m_coulomb(self.handle, C.byref(phys), C.byref(state.st), _ptr(out), _stream(stream)),
               "p3m_coulomb")
        return out[: state.st.capacity]

    def close(self):
        if self.handle:
            lib().pdq_p3m_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Caller-owned particle state (torch tensors) plus its pdq_state struct."""

    def __init__(self, precision, counts, st_plus, device="cuda"):
        counts = [int(c) for c in counts]
        S = len(counts)
        if not 1 <= len(st_plus) <= MAX_CLASSES:
            raise ValueError("1..16 size classes")
        off = [0]
        for c in counts:
            off.append(off[-1] + c)
        n = max(off[-1], 1)
        dev = torch.device(device)
        self.precision = precision
        self.counts0 = counts
        self.offset = torch.tensor(off, dtype=torch.int64, device=dev)
        self.count = torch.tensor(counts, dtype=torch.int32, device=dev)
        fdt = torch.float64 if precision == FP64 else torch.float32
        self.pos = [torch.zeros((n, 4), dtype=fdt, device=dev) for _ in range(2)]
        self.vel = [torch.zeros((n, 4), dtype=fdt, device=dev) for _ in range(2)]
        self.xy = [torch.zeros((n, 2), dtype=torch.float64, device=dev) for _ in range(2)] if precision == MIXED else None
        self.tag = torch.zeros((n, 2), dtype=torch.int32, device=dev)
        self.ctl = torch.zeros(8, dtype=torch.int64, device=dev)
        s = StateStruct()
        s.precision, s.cur, s.n_samples, s.n_classes = precision, 0, S, len(st_plus)
        for k, v in enumerate(st_plus):
            s.st_plus[k] = float(v)
        s.capacity, s.step = off[-1], 0
        s.offset, s.count = self.offset.data_ptr(), self.count.data_ptr()
        for h in range(2):
            s.pos[h] = self.pos[h].data_ptr()
            s.vel[h] = self.vel[h].data_ptr()
            s.xy[h] = self.xy[h].data_ptr() if self.xy else None
        s.tag, s.ctl = self.tag.data_ptr(), self.ctl.data_ptr()
        self.st = s
        self.n_samples, self.n_classes, self.st_plus = S, len(st_plus), list(st_plus)

    @property
    def cur(self):
        return self.st.cur

    @property
    def step_index(self):
        return self.st.step

    def current(self):
        """(pos, vel, xy or None) tensors of the current half."""
        h = self.st.cur
        return self.pos[h], self.vel[h], (self.xy[h] if self.xy else None)

    def positions64(self):
        """[N, 3] float64 positions of the current half (x, y from the FP64 copy in MIXED)."""
        pos, _, xy = self.current()
        out = pos[:, :3].double().clone()
        if xy is not None:
            out[:, :2] = xy
        return out


class Tally:
    def __init__(self, n_samples, n_classes, device="cuda"):
        self.n_dep = torch.zeros((n_samples, n_classes), dtype=torch.int64, device=device)
        self.n_alive = torch.zeros((n_samples, n_classes), dtype=torch.int64, device=device)
        self.t = TallyStruct(self.n_dep.data_ptr(), self.n_alive.data_ptr())

    def zero_(self):
        self.n_dep.zero_()
        self.n_alive.zero_()


def step_cfg(dt, forces=F_ALL, mode=STICK, gravity=(0.0, 0.0, 1.0), window_start=0, compact_every=0, block=0,
             use_graph=False, variant=0):
    c = StepCfg()
    c.dt = dt
    for k in range(3):
        c.gravity[k] = gravity[k]
    c.mode, c.forces, c.window_start = mode, forces, window_start
    # use_graph: False/0 direct, True/1 captured graph (replayed on later calls), 2 capture only
    c.compact_every, c.block, c.use_graph, c.variant = compact_every, block, int(use_graph), variant
    return c


def lf_desc(n_y=None, stretch=None, t_lagr=None, temperature=None, vdw_cutoff=None, precision=None):
    """Parameters of the 1-D Eulerian low-fidelity model (library defaults where None)."""
    d = LfDesc()
    lib().pdq_lf_desc_default(C.byref(d))
    for k, v in dict(n_y=n_y, stretch=stretch, t_lagr=t_lagr, temperature=temperature,
                     vdw_cutoff=vdw_cutoff, precision=precision).items():
        if v is not None:
            setattr(d, k, v)
    return d


def lf_fluid_variance(field, stream=None):
    """v_f'^2 [n_r] (float64, device) of the field's radial velocity at its radial nodes."""
    out = torch.empty(field.desc.n_r, dtype=torch.float64, device="cuda")
    _check(lib().pdq_lf_fluid_variance(field.handle, _ptr(out), _stream(stream)), "lf_fluid_variance")
    return out


def lf_vdep(field, phys, desc, var, st_plus, params_dev, out=None, stream=None):
    """V_dep+ [S, C] (float64, device) of the 1-D Eulerian model for params_dev (pdq_sample_params[S])."""
    S, Cn = int(params_dev.shape[0]), len(st_plus)
    out = out if out is not None else torch.empty((S, Cn), dtype=torch.float64, device="cuda")
    st = (C.c_double * Cn)(*[float(x) for x in st_plus])
    _check(lib().pdq_lf_vdep(field.handle, C.byref(phys), C.byref(desc), _ptr(var), Cn, C.cast(st, C.c_void_p), S,
                             _ptr(params_dev), _ptr(out), _stream(stream)), "lf_vdep")
    return out


def params_tensor(params, device="cuda"):
    """[S, 3] (xi, zeta, theta) -> device pdq_sample_params[S] (float64 [S, 4])."""
    p = torch.as_tensor(params, dtype=torch.float64).reshape(-1, 3)
    out = torch.zeros((p.shape[0], 4), dtype=torch.float64)
    out[:, :3] = p
    return out.to(device)


def seed_particles(field, phys, state, params_dev, seed, charge_sigma=0.0, stream=None):
    _check(lib().pdq_seed_particles(field.handle, C.byref(phys), charge_sigma, seed, _ptr(params_dev),
                                    C.byref(state.st), _stream(stream)), "seed_particles")


def seed_particles_independent(field, phys, state, params_dev, seed, charge_sigma=0.0, stream=None):
    _check(lib().pdq_seed_particles_independent(field.handle, C.byref(phys), charge_sigma, seed, _ptr(params_dev),
                                                C.byref(state.st), _stream(stream)), "seed_particles_independent")


def workspace(state, cfg):
    n = C.c_size_t()
    _check(lib().pdq_step_workspace_size(C.byref(state.st), C.byref(cfg), C.byref(n)), "step_workspace_size")
    return torch.empty(max(int(n.value), 256), dtype=torch.uint8, device="cuda")


def step_particles(field, phys, state, params_dev, cfg, n_steps, tally, ws, stream=None):
    _check(lib().pdq_step_particles(field.handle, C.byref(phys), C.byref(state.st), _ptr(params_dev), C.byref(cfg),
                                    int(n_steps), C.byref(tally.t), _ptr(ws), ws.numel(), _stream(stream)),
           "step_particles")


def step_particles_p3m(field, phys, state, params_dev, cfg, n_steps, tally, plan, ws, stream=None):
    """The step with the Coulomb acceleration from a P3M plan (periodic-pipe electrostatics)."""
    _check(lib().pdq_step_particles_p3m(field.handle, C.byref(phys), C.byref(state.st), _ptr(params_dev),
                                        C.byref(cfg), int(n_steps), C.byref(tally.t), plan.handle, _ptr(ws),
                                        ws.numel(), _stream(stream)), "step_particles_p3m")


def step_particles_noalloc(field, phys, state, params_dev, cfg, n_steps, tally, stream=None):
    """The step without a caller workspace (uses libpdq's built-in 1 MiB scratch)."""
    _check(lib().pdq_step_particles_noalloc(field.handle, C.byref(phys), C.byref(state.st), _ptr(params_dev),
                                            C.byref(cfg), int(n_steps), C.byref(tally.t), _stream(stream)),
           "step_particles_noalloc")


def autotune(field, phys, state, params_dev, cfg, stream=None):
    """Pick cfg.block / cfg.variant by timing one step of each candidate (cached per size bucket)."""
    n = C.c_size_t()
    _check(lib().pdq_autotune_workspace_size(C.byref(state.st), C.byref(n)), "autotune_workspace_size")
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    _check(lib().pdq_autotune(field.handle, C.byref(phys), C.byref(state.st), _ptr(params_dev), C.byref(cfg),
                              _ptr(ws), ws.numel(), _stream(stream)), "autotune")
    return cfg


def release_graphs():
    _check(lib().pdq_release_graphs(), "release_graphs")


def compact(state, stream=None):
    _check(lib().pdq_compact(C.byref(state.st), _stream(stream)), "compact")


def check_state(state, stream=None):
    return lib().pdq_check_state(C.byref(state.st), _stream(stream))


def capture_efficiency(field, phys, vdep, stream=None):
    """CE = (4 L / D)(u*/U_b) V_dep+ (Sec. 4.3) of a device float64 tensor."""
    v = vdep.contiguous()
    ce = torch.empty_like(v)
    _check(lib().pdq_capture_efficiency(field.handle, C.byref(phys), _ptr(v), v.numel(), _ptr(ce), _stream(stream)),
           "capture_efficiency")
    return ce


def deposition_tally(tally, dt, r_plus=180.0, stream=None):
    """(vdep [S, C], mean [C], se [C]) device float64 tensors."""
    S, Cn = tally.n_dep.shape
    vdep = torch.empty((S, Cn), dtype=torch.float64, device="cuda")
    mean = torch.empty(Cn, dtype=torch.float64, device="cuda")
    se = torch.empty(Cn, dtype=torch.float64, device="cuda")
    _check(lib().pdq_deposition_tally(C.byref(tally.t), S, Cn, dt, r_plus, _ptr(vdep), _ptr(mean), _ptr(se),
                                      _stream(stream)), "deposition_tally")
    return vdep, mean, se


# ---------------------------------------------------------------------------
# Multi-fidelity Monte Carlo (host arrays via numpy)
# ---------------------------------------------------------------------------
def _np_ptr(a):
    return C.c_void_p(a.ctypes.data)


def mfmc_allocate(rho, sigma, w, budget, d_inputs=0):
    """(m [k] int64, alpha [k], m_real [k], gamma) of the optimal MFMC allocation."""
    import numpy as np
    rho, sigma, w = (np.ascontiguousarray(v, np.float64) for v in (rho, sigma, w))
    k = len(rho)
    m = np.zeros(k, np.int64)
    alpha, m_real = np.zeros(k), np.zeros(k)
    gamma = C.c_double()
    _check(lib().pdq_mfmc_allocate(k, _np_ptr(rho), _np_ptr(sigma), _np_ptr(w), float(budget), int(d_inputs),
                                   _np_ptr(m), _np_ptr(alpha), _np_ptr(m_real), C.byref(gamma)), "mfmc_allocate")
    return m, alpha, m_real, gamma.value


def mfmc_sobol(ys, m, alpha, n_boot=0, seed=0, stream=None):
    """MFMC Sobol' analysis of device tensors ys[i] [n_i, d+2, C] (float64).

    Returns dict(mean [C], var [C], s_main [d, C], s_total [d, C], s_main_ci, s_total_ci [d, C, 2]).
    """
    import numpy as np
    k = len(ys)
    d = ys[0].shape[1] - 2
    Cn = ys[0].shape[2]
    ys = [t.contiguous() for t in ys]
    yp = (C.c_void_p * k)(*[t.data_ptr() for t in ys])
    m = np.ascontiguousarray(m, np.int64)
    alpha = np.ascontiguousarray(alpha, np.float64)
    n = C.c_size_t()
    _check(lib().pdq_mfmc_workspace_size(k, d, Cn, n_boot, C.byref(n)), "mfmc_workspace_size")
    ws = torch.empty(max(n.value, 8), dtype=torch.uint8, device=ys[0].device)
    out = {"mean": np.zeros(Cn), "var": np.zeros(Cn), "s_main": np.zeros((d, Cn)), "s_total": np.zeros((d, Cn)),
           "s_main_ci": np.zeros((d, Cn, 2)), "s_total_ci": np.zeros((d, Cn, 2))}
    _check(lib().pdq_mfmc_sobol(k, C.cast(yp, C.c_void_p), _np_ptr(m), _np_ptr(alpha), d, Cn, n_boot, seed,
                                *(_np_ptr(out[q]) for q in ("mean", "var", "s_main", "s_total", "s_main_ci",
                                                            "s_total_ci")),
                                _ptr(ws), ws.numel(), _stream(stream)), "mfmc_sobol")
    if n_boot == 0:
        del out["s_main_ci"], out["s_total_ci"]
    return out


# ---------------------------------------------------------------------------
# Adjoint of the smoothed deposition functional
# ---------------------------------------------------------------------------
class Batch:
    """Sample layout for the adjoint (it seeds its own particles)."""

    def __init__(self, precision, counts, st_plus, device="cuda"):
        off = [0]
        for c in counts:
            off.append(off[-1] + int(c))
        self.offset = torch.tensor(off, dtype=torch.int64, device=device)
        b = BatchStruct()
        b.precision, b.n_samples, b.n_classes = precision, len(counts), len(st_plus)
        for k, v in enumerate(st_plus):
            b.st_plus[k] = float(v)
        b.capacity, b.offset = off[-1], self.offset.data_ptr()
        self.b = b
        self.n_samples, self.n_classes = len(counts), len(st_plus)


def batch_of_state(state):
    """The pdq_batch (workspace layout) of a state's adjoint."""
    b = BatchStruct()
    st = state.st
    b.precision, b.n_samples, b.n_classes = st.precision, st.n_samples, st.n_classes
    for k in range(st.n_classes):
        b.st_plus[k] = st.st_plus[k]
    b.capacity, b.offset = st.capacity, st.offset
    return b


def _adjoint_outputs(S, Cn, gbar):
    J = torch.empty((S, Cn), dtype=torch.float64, device="cuda")
    nv = 0 if gbar is None else gbar.shape[0]
    pbar = torch.zeros((max(nv, 1), S, 3), dtype=torch.float64, device="cuda")
    g = gbar.contiguous().to(torch.float64) if gbar is not None else None
    return J, nv, pbar, g


def _stored_sums_bytes(capacity, n_steps, store_sums):
    if not store_sums:
        return 0
    n = C.c_size_t()
    _check(lib().pdq_adjoint_stored_sums_size(int(capacity), int(n_steps), C.byref(n)), "adjoint_stored_sums_size")
    return n.value


def adjoint_workspace_bytes(batch_struct, n_steps, K, store_sums=False):
    """Bytes of the adjoint's workspace; store_sums adds room for every step's Newton-pair sums (MIXED
    with Coulomb forces: the reverse sweep's recompute then skips the pair sums)."""
    n = C.c_size_t()
    _check(lib().pdq_adjoint_workspace_size(C.byref(batch_struct), int(n_steps), int(K), C.byref(n)),
           "adjoint_workspace_size")
    return n.value + _stored_sums_bytes(batch_struct.capacity, n_steps, store_sums)


def adjoint_workspace(batch_struct, n_steps, K, store_sums=False):
    """The adjoint's workspace (device bytes), see adjoint_workspace_bytes."""
    return torch.empty(adjoint_workspace_bytes(batch_struct, n_steps, K, store_sums), dtype=torch.uint8,
                       device="cuda")


def adjoint_run(field, phys, state, params_dev, cfg, n_steps, K, eps, gbar=None, stream=None, eps_stick=10.0,
                ws=None, store_sums=False):
    """pdq_adjoint_run from the current half of `state`: J [S, C] and, for cotangents gbar [V, S, C],
    pbar [V, S, 3] = gbar . dJ/d(xi, zeta, theta).  Returns (J, pbar or None, workspace)."""
    if ws is None:
        n = C.c_size_t()
        _check(lib().pdq_adjoint_state_workspace_size(C.byref(state.st), int(n_steps), int(K), C.byref(n)),
               "adjoint_state_workspace_size")
        extra = _stored_sums_bytes(state.st.capacity, n_steps, store_sums)
        ws = torch.empty(n.value + extra, dtype=torch.uint8, device="cuda")
    J, nv, pbar, g = _adjoint_outputs(state.n_samples, state.n_classes, gbar)
    _check(lib().pdq_adjoint_run(field.handle, C.byref(phys), C.byref(state.st), _ptr(params_dev), C.byref(cfg),
                                 int(n_steps), int(K), float(eps), float(eps_stick), nv, _ptr(g), _ptr(J),
                                 _ptr(pbar), _ptr(ws), ws.numel(), _stream(stream)), "adjoint_run")
    return J, (pbar[:nv] if nv else None), ws


def adjoint_run_seeded(field, phys, batch, params_dev, cfg, n_steps, K, eps, seed, charge_sigma=0.0, gbar=None,
                       stream=None, eps_stick=10.0, ws=None, store_sums=False):
    """pdq_adjoint_run_seeded: J [S, C] and, for cotangents gbar [V, S, C], pbar [V, S, 3]."""
    if ws is None:
        ws = adjoint_workspace(batch.b, n_steps, K, store_sums)
    J, nv, pbar, g = _adjoint_outputs(batch.n_samples, batch.n_classes, gbar)
    _check(lib().pdq_adjoint_run_seeded(field.handle, C.byref(phys), C.byref(batch.b), _ptr(params_dev),
                                        charge_sigma, seed, C.byref(cfg), int(n_steps), int(K), float(eps),
                                        float(eps_stick), nv, _ptr(g), _ptr(J), _ptr(pbar), _ptr(ws), ws.numel(),
                                        _stream(stream)), "adjoint_run_seeded")
    return J, (pbar[:nv] if nv else None)


def adjoint_reverse(field, phys, batch_struct, params_dev, cfg, n_steps, K, eps, gbar, ws, stream=None,
                    eps_stick=10.0):
    """pdq_adjoint_reverse: pbar [V, S, 3] from the forward sweep an earlier call left in `ws`."""
    nv = gbar.shape[0]
    pbar = torch.zeros((nv, batch_struct.n_samples, 3), dtype=torch.float64, device="cuda")
    g = gbar.contiguous().to(torch.float64)
    _check(lib().pdq_adjoint_reverse(field.handle, C.byref(phys), C.byref(batch_struct), _ptr(params_dev),
                                     C.byref(cfg), int(n_steps), int(K), float(eps), float(eps_stick), nv, _ptr(g),
                                     _ptr(pbar), _ptr(ws), ws.numel(), _stream(stream)), "adjoint_reverse")
    return pbar


class PdqDeposition(torch.autograd.Function):
    """J = smoothed V_dep+ [S, C] of the particle model as a function of params [S, 3] = (xi, zeta, theta).

    forward runs the smoothed forward sweep (pdq_adjoint_run_seeded with no cotangent) and keeps
    its workspace, checkpoints included (and with store_sums every step's pair sums), until
    backward; backward runs only the reverse sweep (pdq_adjoint_reverse) with the incoming
    gradient as cotangent.
    """

    @staticmethod
    def forward(ctx, params, field, phys, batch, cfg, n_steps, K, eps, seed, charge_sigma, store_sums=False):
        prm = params_tensor(params.detach())
        ws = adjoint_workspace(batch.b, n_steps, K, store_sums)
        J, _ = adjoint_run_seeded(field, phys, batch, prm, cfg, n_steps, K, eps, seed, charge_sigma, ws=ws)
        ctx.save_for_backward(params.detach())
        ctx.args = (field, phys, batch, cfg, n_steps, K, eps, prm, ws)
        return J

    @staticmethod
    def backward(ctx, grad_out):
        (params,) = ctx.saved_tensors
        field, phys, batch, cfg, n_steps, K, eps, prm, ws = ctx.args
        pbar = adjoint_reverse(field, phys, batch.b, prm, cfg, n_steps, K, eps,
                               grad_out.detach().to(torch.float64).unsqueeze(0), ws)
        ctx.args = None
        return (pbar[0].to(device=params.device, dtype=params.dtype),) + (None,) * 10


def dgsm_bounds(grad, y, width, stream=None):
    """(nu [d, C], bound [d, C]) from device grad [S, C, d] and y [S, C] (float64)."""
    import numpy as np
    S, Cn, d = grad.shape
    w = np.ascontiguousarray(width, np.float64)
    nu, bound = np.zeros((d, Cn)), np.zeros((d, Cn))
    g, yy = grad.contiguous().to(torch.float64), y.contiguous().to(torch.float64)
    n = C.c_size_t()
    _check(lib().pdq_dgsm_workspace_size(Cn, d, C.byref(n)), "dgsm_workspace_size")
    ws = torch.empty(n.value, dtype=torch.uint8, device=grad.device)
    _check(lib().pdq_dgsm_bounds(S, Cn, d, _ptr(g), _ptr(yy), _np_ptr(w), _np_ptr(nu), _np_ptr(bound), _ptr(ws),
                                 ws.numel(), _stream(stream)), "dgsm_bounds")
    return nu, bound
