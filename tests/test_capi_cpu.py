"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/pdq.h declares, and rejects invalid arguments before touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pdq():
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    p.lib()
    return p


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pdq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdq_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_function(pdq):
    names = declared_functions()
    assert len(names) >= 12
    L = pdq.lib()
    for n in names:
        assert hasattr(L, n), n


def test_status_strings_and_defaults(pdq):
    L = pdq.lib()
    assert L.pdq_strerror(0) == b"ok"
    assert b"invalid" in L.pdq_strerror(-1)
    assert L.pdq_version() >= 100
    p = pdq.phys_default()
    assert p.re_tau == 180.0 and p.rho_p == 2650.0 and p.delta_min == 1e-9


def test_invalid_arguments_rejected_on_host(pdq):
    L = pdq.lib()
    P = C.c_void_p
    # NULL descriptor / handle
    assert L.pdq_create_pipe_field(None, 0, None, None) == -1
    d = pdq.field_desc(n_r=1)
    h = C.c_void_p()
    assert L.pdq_create_pipe_field(C.byref(d), 0, None, C.byref(h)) == -1
    d = pdq.field_desc(n_modes=5000)
    assert L.pdq_create_pipe_field(C.byref(d), 0, None, C.byref(h)) == -1
    assert L.pdq_destroy_pipe_field(None) == -1
    # state with bad precision / class count
    s = pdq.StateStruct()
    s.precision, s.n_samples, s.n_classes = 7, 1, 1
    n = C.c_size_t()
    assert L.pdq_step_workspace_size(C.byref(s), None, C.byref(n)) == -1
    s.precision, s.n_classes = 0, 0
    assert L.pdq_step_workspace_size(C.byref(s), None, C.byref(n)) == -1
    t = pdq.TallyStruct()
    assert L.pdq_deposition_tally(C.byref(t), 1, 1, 0.1, 180.0, None, None, None, None) == -1
    assert L.pdq_step_particles(None, None, None, None, None, 1, None, None, 0, None) == -1


def test_mfmc_allocate_host_logic(pdq):
    # host-only entry point: matches the oracle's allocation and the paper's Table 3 / gamma values
    import json
    import numpy as np
    from oracle import mfmc
    tab = json.load(open(os.path.join(ROOT, "tests", "golden", "mfmc_tables.json")))
    for case in tab["cases"]:
        rho = [1.0, case["rho12"]]
        sig = [case["sigma1"], case["sigma2"]]
        w = [1.0, tab["w2"]]
        for p, key in ((36, "p36"), (72, "p72")):
            m, alpha, m_real, gamma = pdq.mfmc_allocate(rho, sig, w, p, d_inputs=2)
            a_ref, _, m_ref = mfmc.mfmc_allocation(rho, sig, w, p / 4)
            assert np.allclose(alpha, a_ref, rtol=1e-14) and np.allclose(m_real, m_ref, rtol=1e-13)
            assert m[0] == case[key]["m1"]
            assert round(gamma, 3) == case["gamma"]
            assert abs(gamma - mfmc.gamma_two_model(rho[1], w[1])) < 1e-12
    # three models: gamma from the general MSE formula is below the two-model value
    m, alpha, m_real, g3 = pdq.mfmc_allocate([1.0, 0.99, 0.9], [1.0, 1.0, 1.0], [1.0, 1e-2, 1e-4], 100.0)
    assert m[0] <= m[1] <= m[2] and 0 < g3 < mfmc.gamma_two_model(0.99, 1e-2)
    # precondition violated / unsorted correlations
    L = pdq.lib()
    import ctypes as C
    for rho, w in (([1.0, 0.3], [1.0, 0.5]), ([1.0, 0.5, 0.9], [1.0, 0.1, 0.01])):
        rho, sig, w = (np.ascontiguousarray(v, np.float64) for v in (rho, np.ones(len(rho)), w))
        mo, ao = np.zeros(len(rho), np.int64), np.zeros(len(rho))
        rc = L.pdq_mfmc_allocate(len(rho), C.c_void_p(rho.ctypes.data), C.c_void_p(sig.ctypes.data),
                                 C.c_void_p(w.ctypes.data), 10.0, 0, C.c_void_p(mo.ctypes.data),
                                 C.c_void_p(ao.ctypes.data), None, None)
        assert rc == -6


def test_contact_and_p3m_arguments_rejected_on_host(pdq):
    L = pdq.lib()
    p = pdq.phys_default()
    assert p.restitution == 0.9 and p.tau_col_steps == 15.0 and p.neg_charge_frac == 0.0
    # capture efficiency, P3M plan and solve: NULL / out-of-range arguments fail before any CUDA call
    assert L.pdq_capture_efficiency(None, C.byref(p), None, 1, None, None) == -1
    d = pdq.P3MDesc()
    d.M, d.Nz = 2, 64
    h = C.c_void_p()
    assert L.pdq_p3m_create(None, C.byref(d), 100, None, C.byref(h)) == -1
    assert L.pdq_p3m_coulomb(None, C.byref(p), None, None, None) == -1
    assert L.pdq_p3m_params(None, None, None, None, None) == -1
    assert L.pdq_p3m_destroy(None) == 0
    # the P3M step refuses graph mode and contact forces before touching the plan or the GPU
    cfg = pdq.step_cfg(0.05, use_graph=True)
    s = pdq.StateStruct()
    t = pdq.TallyStruct()
    fake = C.c_void_p(1)
    assert L.pdq_step_particles_p3m(None, C.byref(p), C.byref(s), None, C.byref(cfg), 1, C.byref(t), fake, None, 0,
                                    None) == -1
    cfg = pdq.step_cfg(0.05, forces=pdq.F_ALL | pdq.F_CONTACT)
    assert L.pdq_step_particles_p3m(None, C.byref(p), C.byref(s), None, C.byref(cfg), 1, C.byref(t), fake, None, 0,
                                    None) == -1


def _fake_mixed_state(pdq, capacity):
    s = pdq.StateStruct()
    s.precision, s.n_samples, s.n_classes, s.capacity = 1, 2, 1, capacity
    s.st_plus[0] = 1.0
    s.offset = s.count = s.tag = s.ctl = 16
    for h in range(2):
        s.pos[h] = s.vel[h] = s.xy[h] = 16
    return s


def test_newton_pair_variant_host_logic(pdq):
    # pair variant 3 keeps FP32 sums float4 [capacity] in the workspace; it runs at 64 or 128
    # threads (its update step uses twice as many), and variants above 3 are rejected
    L = pdq.lib()
    s = _fake_mixed_state(pdq, 100_000)
    sizes = {}
    for v in (2, 3):
        cfg = pdq.step_cfg(0.05, block=128, variant=v)
        n = C.c_size_t()
        assert L.pdq_step_workspace_size(C.byref(s), C.byref(cfg), C.byref(n)) == 0
        sizes[v] = n.value
    assert sizes[3] - sizes[2] >= 16 * 100_000
    t = pdq.TallyStruct()
    t.n_dep = t.n_alive = 16
    fake = C.c_void_p(16)
    for block, variant in ((256, 3), (128, 4)):
        cfg = pdq.step_cfg(0.05, block=block, variant=variant)
        rc = L.pdq_step_particles(fake, C.byref(pdq.phys_default()), C.byref(s), fake, C.byref(cfg), 1, C.byref(t),
                                  C.c_void_p(256), 1 << 40, None)
        assert rc == -1, (block, variant)


def test_newton_pair_workspace_by_precision_and_forces(pdq):
    # FP64 variant 3 keeps double sums [capacity][3] (24 B each, no one-sided chunk partials);
    # MIXED contact runs under variant 3 take the float sums too; FP64 contact runs ignore it
    L = pdq.lib()
    cap = 50_000

    def size(precision, variant, forces=pdq.F_ALL, block=128):
        s = _fake_mixed_state(pdq, cap)
        s.precision = precision
        cfg = pdq.step_cfg(0.05, block=block, variant=variant, forces=forces)
        n = C.c_size_t()
        assert L.pdq_step_workspace_size(C.byref(s), C.byref(cfg), C.byref(n)) == 0
        return n.value

    assert size(0, 3) >= 24 * cap
    assert size(1, 3, pdq.F_ALL | pdq.F_CONTACT) - size(1, 0, pdq.F_ALL | pdq.F_CONTACT) >= 16 * cap
    assert size(0, 3, pdq.F_ALL | pdq.F_CONTACT) == size(0, 0, pdq.F_ALL | pdq.F_CONTACT)


def test_adjoint_workspace_holds_the_newton_pair_sums(pdq):
    # per particle: 8 FP64 + 2 int32 arrays per checkpoint, 10 per segment level, 19 more, and
    # 16 B of float sums
    L = pdq.lib()
    b = pdq.BatchStruct()
    b.precision, b.n_samples, b.n_classes, b.capacity = 1, 4, 3, 4096
    n = C.c_size_t()
    assert L.pdq_adjoint_workspace_size(C.byref(b), 100, 10, C.byref(n)) == 0
    per = 10 * (8 * 8 + 2 * 4) + 11 * 10 * 8 + 19 * 8 + 16
    assert n.value >= per * 4096
    assert L.pdq_adjoint_workspace_size(C.byref(b), 0, 10, C.byref(n)) == -1


def test_adjoint_stored_sums_size(pdq):
    # a 256-byte marker, then one float4 [capacity] array (256-byte aligned) per step
    L = pdq.lib()
    n = C.c_size_t()
    for cap, steps in ((4096, 100), (1000, 7), (0, 1)):
        assert L.pdq_adjoint_stored_sums_size(cap, steps, C.byref(n)) == 0
        stride = -(-16 * max(cap, 1) // 256) * 256
        assert n.value == 256 + stride * steps
    assert L.pdq_adjoint_stored_sums_size(-1, 10, C.byref(n)) == -1
    assert L.pdq_adjoint_stored_sums_size(4096, 0, C.byref(n)) == -1
    assert L.pdq_adjoint_stored_sums_size(4096, 10, None) == -1


def test_low_fidelity_defaults_and_arguments_rejected_on_host(pdq):
    L = pdq.lib()
    d = pdq.lf_desc()
    assert (d.n_y, d.precision, d.stretch, d.t_lagr, d.temperature, d.vdw_cutoff) == (2048, 0, 8.0, 10.0, 293.15,
                                                                                     1e-12)
    p = pdq.phys_default()
    st = (C.c_double * 1)(1.0)
    # NULL field / variance / descriptor fail before any CUDA call
    assert L.pdq_lf_fluid_variance(None, None, None) == -1
    assert L.pdq_lf_vdep(None, C.byref(p), C.byref(d), None, 1, C.cast(st, C.c_void_p), 1, None, None, None) == -1
    assert L.pdq_lf_vdep(None, C.byref(p), None, None, 1, C.cast(st, C.c_void_p), 0, None, None, None) == -1
