"""Autotuner and cached CUDA-graph replay of the step (through the C ABI).

A tuned run, an untuned run (another tile shape) and a graph-replayed run of
FP64 must agree bit for bit per particle (the Coulomb sums' regrouping between
tile shapes stays far below the last place of positions and velocities); the
autotuner must leave the state unchanged apart from binning it by z.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04979_gb300 import build
    build.build()
    import paper_2205_04979_gb300.pdq as p
    return p


def _setup(pdq, precision, counts, st_plus=(0.1, 1.0, 10.0)):
    field = pdq.Field(pdq.field_desc(n_r=33, n_th=16, n_z=32), 0)
    phys = pdq.phys_default()
    st = pdq.State(precision, counts, list(st_plus))
    prm = pdq.params_tensor(np.tile([0.08, 0.5, 0.5], (len(counts), 1)))
    pdq.seed_particles(field, phys, st, prm, 3)
    return field, phys, st, prm


def _by_id(st):
    """State arrays with each sample's rows ordered by particle id (the step may bin rows by z)."""
    pos, vel, xy = st.current()
    tag = st.tag.cpu().numpy()
    offs, cnt = st.offset.cpu().numpy(), st.count.cpu().numpy()
    order = np.concatenate([offs[s] + np.argsort(tag[offs[s]:offs[s] + cnt[s], 0], kind="stable")
                            for s in range(len(cnt))])
    out = [t.cpu().numpy()[order] for t in (pos, vel) + ((xy,) if xy is not None else ())]
    return out + [tag[order], cnt]


def test_autotune_leaves_fp64_state_unchanged_and_results_identical(pdq):
    counts = [700, 333]
    field, phys, a, prm = _setup(pdq, 0, counts)
    cfg = pdq.step_cfg(0.1, window_start=2)
    before = _by_id(a)
    cur, step = a.cur, a.step_index
    pdq.autotune(field, phys, a, prm, cfg)
    assert cfg.block in (32, 64, 128, 256) and cfg.variant == 0
    after = _by_id(a)
    # the autotuner bins the state by z (a permutation within each sample) and leaves the rest
    assert a.step_index == step and int(a.ctl[0]) == step
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    # tuned run with graph replays (3 calls of 2 steps: the 2nd and 3rd replay the 1st's graph)
    stream = torch.cuda.Stream()
    ta = pdq.Tally(2, 3)
    cfg.use_graph = 1
    wa = pdq.workspace(a, cfg)
    with torch.cuda.stream(stream):
        for _ in range(3):
            pdq.step_particles(field, phys, a, prm, cfg, 2, ta, wa, stream)
    stream.synchronize()
    # untuned reference, no graph
    _, _, b, _ = _setup(pdq, 0, counts)
    tb = pdq.Tally(2, 3)
    cfg_b = pdq.step_cfg(0.1, window_start=2, block=64 if cfg.block != 64 else 256)
    pdq.step_particles(field, phys, b, prm, cfg_b, 6, tb, pdq.workspace(b, cfg_b))
    assert a.step_index == b.step_index == 6 and int(a.ctl[0]) == 6
    for x, y in zip(_by_id(a), _by_id(b)):
        assert np.array_equal(x, y)
    assert torch.equal(ta.n_dep, tb.n_dep) and torch.equal(ta.n_alive, tb.n_alive)
    pdq.release_graphs()


def test_autotune_mixed_binned(pdq):
    counts = [3000, 1500]
    field, phys, a, prm = _setup(pdq, 1, counts)
    cfg = pdq.step_cfg(0.05, compact_every=10)
    pdq.autotune(field, phys, a, prm, cfg)
    assert cfg.block in (64, 128, 256) and cfg.variant in (0, 1, 2, 3)
    assert not (cfg.variant == 3 and cfg.block == 256)
    # a second call for the same size bucket is served from the cache
    cfg2 = pdq.step_cfg(0.05, compact_every=10)
    pdq.autotune(field, phys, a, prm, cfg2)
    assert (cfg2.block, cfg2.variant) == (cfg.block, cfg.variant)
    # the binned, tuned state still advances consistently with an untuned run (by particle id)
    tally = pdq.Tally(2, 3)
    pdq.step_particles(field, phys, a, prm, cfg, 20, tally, pdq.workspace(a, cfg))
    _, _, b, _ = _setup(pdq, 1, counts)
    tb = pdq.Tally(2, 3)
    cfg_b = pdq.step_cfg(0.05)
    pdq.step_particles(field, phys, b, prm, cfg_b, 20, tb, pdq.workspace(b, cfg_b))
    pa = {}
    for st, d in ((a, pa),):
        pos, vel, xy = st.current()
        tag = st.tag.cpu().numpy()
        cnt, off = st.count.cpu().numpy(), st.offset.cpu().numpy()
        x = xy.cpu().numpy()
        al = vel[:, 3].cpu().numpy()
        for s in range(2):
            for g in range(off[s], off[s] + cnt[s]):
                if al[g] > 0.5:
                    d[(s, tag[g, 0])] = x[g]
    pos, vel, xy = b.current()
    xb, tb_ = xy.cpu().numpy(), b.tag.cpu().numpy()
    alb = vel[:, 3].cpu().numpy()
    off = b.offset.cpu().numpy()
    n_cmp = 0
    for s in range(2):
        for g in range(off[s], off[s + 1]):
            k = (s, tb_[g, 0])
            if alb[g] > 0.5 and k in pa:
                assert np.all(np.abs(pa[k] - xb[g]) < 1e-3)
                n_cmp += 1
    assert n_cmp > 0.99 * sum(counts) * 0.9


def test_graph_prepare_then_replay_matches_direct_run(pdq):
    # use_graph = 2 captures and instantiates the call's graph without running it; the state,
    # tallies and host fields stay as they were, and the next use_graph = 1 call replays it
    counts = [700, 333]
    field, phys, a, prm = _setup(pdq, 0, counts)
    stream = torch.cuda.Stream()
    cfg = pdq.step_cfg(0.1, window_start=2, block=64, use_graph=2)
    ta = pdq.Tally(2, 3)
    wa = pdq.workspace(a, cfg)
    with torch.cuda.stream(stream):
        pdq.step_particles(field, phys, a, prm, cfg, 3, ta, wa, stream)      # capture only
    stream.synchronize()
    before = _by_id(a)
    assert a.step_index == 0 and int(a.ctl[0]) == 0 and int(ta.n_alive.sum()) == 0
    _, _, b, _ = _setup(pdq, 0, counts)
    assert all(np.array_equal(x, y) for x, y in zip(before, _by_id(b)))
    cfg.use_graph = 1
    with torch.cuda.stream(stream):
        pdq.step_particles(field, phys, a, prm, cfg, 3, ta, wa, stream)      # replays the prepared graph
        pdq.step_particles(field, phys, a, prm, cfg, 3, ta, wa, stream)      # another phase: captured now
    stream.synchronize()
    tb = pdq.Tally(2, 3)
    cfg_b = pdq.step_cfg(0.1, window_start=2, block=64)
    pdq.step_particles(field, phys, b, prm, cfg_b, 6, tb, pdq.workspace(b, cfg_b))
    assert a.step_index == b.step_index == 6 and int(a.ctl[0]) == 6
    for x, y in zip(_by_id(a), _by_id(b)):
        assert np.array_equal(x, y)
    assert torch.equal(ta.n_dep, tb.n_dep) and torch.equal(ta.n_alive, tb.n_alive)
    pdq.release_graphs()
