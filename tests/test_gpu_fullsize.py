"""Parity at the full size of the batched workload: 1,024 samples of 4,107..32,737
particles (18,659,370 in all), 5 classes, 128 x 64 x 128 field, dt+ = 0.05,
compaction every 100 steps, MIXED, in the launch configuration the benchmark
times (the autotuner's tile and pair variant, z-binned at the start of the call).

One GPU step of the whole batch; then the oracle (FP64) rebuilds six samples from
the same seeds (a particle's seed depends only on the key and its index within
its sample), steps each whole sample once and the GPU particles of those samples
are compared by id, with the MIXED bars of the small-size parity tests.  The
largest and smallest samples are among the six.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


def test_full_batched_workload_one_step_sampled(pdq):
    w = workloads.WORKLOADS["batched_mixed"]
    params, counts = workloads.workload_inputs("batched_mixed")
    assert len(counts) == 1024 and int(counts.sum()) == 18_659_370
    phys = pdq.phys_default()
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    field = pdq.Field(desc, w["field_seed"])
    st = pdq.State(pdq.MIXED, counts, w["st_plus"])
    prm = pdq.params_tensor(params)
    pdq.seed_particles(field, phys, st, prm, w["particle_seed"], w.get("charge_sigma", 0.0))
    cfg = pdq.step_cfg(w["dt"], window_start=0, compact_every=w["compact_every"], forces=pdq.F_ALL)
    pdq.autotune(field, phys, st, prm, cfg)
    assert cfg.block in (64, 128, 256) and cfg.variant in (0, 1, 2, 3)
    tally = pdq.Tally(len(counts), len(w["st_plus"]))
    pdq.step_particles(field, phys, st, prm, cfg, 1, tally, pdq.workspace(st, cfg))
    assert pdq.check_state(st) == 0
    assert st.step_index == 1

    of = oracle.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    grid = oracle.field_grid(of, oracle.field_modes(of, w["field_seed"]))
    rng = np.random.default_rng(5)
    picks = [int(counts.argmax()), int(counts.argmin())] + [int(s) for s in rng.choice(1024, 4, replace=False)]
    offs = st.offset.cpu().numpy()
    cnt = st.count.cpu().numpy()
    n_alive = tally.n_alive.cpu().numpy()
    n_dep = tally.n_dep.cpu().numpy()
    checked = 0
    for s in picks:
        ost, off = oracle.seed(of, w["st_plus"], [counts[s]], params[s:s + 1], w["particle_seed"],
                               w.get("charge_sigma", 0.0))
        nd, na = oracle.run(of, grid, oracle.cfg(w["dt"], window_start=0), w["st_plus"], off, params[s:s + 1],
                            ost, 1)
        # tallies of the sample: every particle alive at the start of the step, deposits exact
        assert np.array_equal(n_alive[s], na[0]) and np.array_equal(n_dep[s], nd[0])
        sl = slice(int(offs[s]), int(offs[s] + cnt[s]))
        assert cnt[s] == counts[s]                     # compaction removes nothing before its first pass
        pos = st.positions64()[sl].cpu().numpy()
        vel = st.current()[1][sl].double().cpu().numpy()
        ids = st.tag[sl, 0].cpu().numpy()
        assert np.array_equal(np.sort(ids), np.arange(counts[s]))
        alive = vel[:, 3] > 0.5
        assert np.array_equal(alive, ost.alive[ids] == 1)
        ref_x = np.stack([ost.x, ost.y, ost.z], 1)[ids]
        ref_v = np.stack([ost.vx, ost.vy, ost.vz], 1)[ids]
        dx = np.abs(pos - ref_x)
        dx[:, 2] = np.minimum(dx[:, 2], 720.0 - dx[:, 2])      # periodic z, measured against L = 720
        scale = 1 + np.abs(ref_x)
        scale[:, 2] = 720.0
        assert np.all(dx[alive] <= 2e-6 * scale[alive]), np.max(dx[alive] / scale[alive])
        dv = np.abs(vel[:, :3] - ref_v)
        assert np.all(dv[alive] <= 2e-5 * (1 + np.abs(ref_v[alive]))), np.max(dv[alive])
        checked += int(alive.sum())
    assert checked > 6 * 4000
