"""Sobol' analysis of the deposition velocity with the batched particle model.

The uncertain inputs (xi, zeta, theta) of Secs. 2.1 and 4.3 are drawn uniform
over their ranges; each pick-freeze group (x, x', z^(1..d)) becomes d + 2
Monte Carlo samples of one batched run of the particle step (common random
particle seeds), whose V_dep+ per size class feeds pdq_mfmc_sobol.
sobol_deposition runs the particle model alone, i.e. the one-model case of the
MFMC formulas (k = 1), with bootstrap intervals; a low-fidelity model (the 1-D
Eulerian model, pdq_lf_vdep, or a cheaper particle model) joins as model 2 of
pdq_mfmc_sobol.  Every numerical step runs in libpdq; this module only arranges
the inputs.
"""
import numpy as np
import torch

from . import pdq


def pick_freeze(x, xp):
    """[m, d+2, d] inputs per group: x, x', then x' with input j taken from x."""
    m, d = x.shape
    out = np.empty((m, d + 2, d))
    out[:, 0], out[:, 1] = x, xp
    for j in range(d):
        z = xp.copy()
        z[:, j] = x[:, j]
        out[:, 2 + j] = z
    return out


def vdep_runs(inputs, particles, steps, st_plus=(0.1, 1.0, 10.0), dt=0.05, t_window=10.0, mode=pdq.STICK,
              forces=pdq.F_ALL, grid=(64, 32, 64), n_modes=64, seed=0, precision=pdq.MIXED, stream=None,
              field=None):
    """V_dep+ [n, C] of n particle-model runs, one per row of inputs [n, 3] = (xi, zeta, theta),
    all in one batched state (common random particle seeds), and the device time of the steps (ms).

    One evaluation of the model f(x) of Sec. 3 per sample; `forces`, `dt` and `particles` define
    the model (a cheaper setting serves as a low-fidelity model).
    """
    n = len(inputs)
    stream = stream or torch.cuda.Stream()
    with torch.cuda.stream(stream):
        phys = pdq.phys_default()
        if field is None:
            field = pdq.Field(pdq.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2], n_modes=n_modes), seed, stream)
        state = pdq.State(precision, [particles] * n, list(st_plus))
        params = pdq.params_tensor(np.asarray(inputs, np.float64))
        pdq.seed_particles(field, phys, state, params, seed + 1, 0.0, stream)
        w0 = int(np.ceil(t_window / dt - 1e-9))
        cfg = pdq.step_cfg(dt, mode=mode, window_start=w0, compact_every=100, forces=forces)
        pdq.autotune(field, phys, state, params, cfg, stream)
        tally = pdq.Tally(n, len(st_plus))
        ws = pdq.workspace(state, cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pdq.step_particles(field, phys, state, params, cfg, steps, tally, ws, stream)
        e1.record(stream)
        vdep, _, _ = pdq.deposition_tally(tally, dt, stream=stream)
        e1.synchronize()
    return vdep.cpu().numpy(), e0.elapsed_time(e1)


def sobol_deposition(m, particles, steps, st_plus=(0.1, 1.0, 10.0), ranges=((0.0, 0.1), (0.0, 1.0), (0.0, 1.0)),
                     dt=0.05, t_window=10.0, mode=pdq.STICK, grid=(64, 32, 64), n_modes=64, seed=0, n_boot=200,
                     precision=pdq.MIXED, qoi="vdep", stream=None, rank=0, world=1):
    """Main and total Sobol' indices of V_dep+ (qoi="vdep") or of the capture efficiency
    (qoi="ce", Sec. 4.3; use mode=pdq.REBOUND) per class from m pick-freeze groups.

    Returns a dict with s_main / s_total [d, C], their bootstrap intervals, mean and variance of
    V_dep+ [C], the V_dep+ table [m, d+2, C] and the device time of the particle runs (ms).
    With world > 1 (torch.distributed initialised, one GPU per rank) the groups are split into
    contiguous ranges, each rank runs its own, and the V_dep+ tables are gathered so that every
    rank evaluates the estimators on all m groups.
    """
    from . import shard
    rng = np.random.Generator(np.random.Philox(seed))
    lo = np.array([r[0] for r in ranges])
    hi = np.array([r[1] for r in ranges])
    d = len(ranges)
    x = lo + (hi - lo) * rng.random((m, d))
    xp = lo + (hi - lo) * rng.random((m, d))
    granges = shard.partition([particles] * m, world)         # equal groups: equal split
    g0, g1 = granges[rank]
    inputs = pick_freeze(x[g0:g1], xp[g0:g1]).reshape(-1, d)  # [(d+2) (g1-g0), d], group-major
    S = inputs.shape[0]
    stream = stream or torch.cuda.Stream()
    with torch.cuda.stream(stream):
        phys = pdq.phys_default()
        field = pdq.Field(pdq.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2], n_modes=n_modes), seed, stream)
        state = pdq.State(precision, [particles] * S, list(st_plus))
        params = pdq.params_tensor(inputs)
        pdq.seed_particles(field, phys, state, params, seed + 1, 0.0, stream)
        w0 = int(np.ceil(t_window / dt - 1e-9))
        cfg = pdq.step_cfg(dt, mode=mode, window_start=w0, compact_every=100)
        pdq.autotune(field, phys, state, params, cfg, stream)      # tile shape and pair variant
        tally = pdq.Tally(S, len(st_plus))
        ws = pdq.workspace(state, cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pdq.step_particles(field, phys, state, params, cfg, steps, tally, ws, stream)
        e1.record(stream)
        vdep, _, _ = pdq.deposition_tally(tally, dt, stream=stream)
        if qoi == "ce":
            vdep = pdq.capture_efficiency(field, phys, vdep, stream)
        e1.synchronize()
        y = vdep.reshape(g1 - g0, d + 2, len(st_plus)).contiguous()
        if world > 1:
            y = shard.gather_rows(y, granges, rank)
        out = pdq.mfmc_sobol([y], [m], [1.0], n_boot=n_boot, seed=seed + 2, stream=stream)
    out["vdep"] = y.cpu().numpy()
    out["ms"] = e0.elapsed_time(e1)
    out["particle_steps"] = float(S) * particles * steps
    return out


def dgsm_deposition(samples, particles, steps, st_plus=(0.1, 1.0, 10.0),
                    ranges=((0.0, 0.1), (0.0, 1.0), (0.0, 1.0)), dt=0.05, t_window=10.0, eps=0.1, K=50,
                    mode=pdq.STICK, eps_stick=10.0, grid=(64, 32, 64), n_modes=64, seed=0, precision=pdq.MIXED,
                    stream=None):
    """Derivative-based bounds on the total Sobol' indices of the smoothed V_dep+ per class.

    The adjoint (pdq_adjoint_run_seeded) gives dJ/d(xi, zeta, theta) for every sample with one cotangent
    vector per class; pdq_dgsm_bounds turns them into s_j^t <= (b_j - a_j)^2 E[(dJ/dx_j)^2] /
    (pi^2 Var J).  Returns dict(J [S, C], grad [S, C, 3], nu [3, C], bound [3, C]).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    lo = np.array([r[0] for r in ranges])
    hi = np.array([r[1] for r in ranges])
    x = lo + (hi - lo) * rng.random((samples, len(ranges)))
    stream = stream or torch.cuda.Stream()
    with torch.cuda.stream(stream):
        phys = pdq.phys_default()
        field = pdq.Field(pdq.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2], n_modes=n_modes), seed, stream)
        batch = pdq.Batch(precision, [particles] * samples, list(st_plus))
        w0 = int(np.ceil(t_window / dt - 1e-9))
        cfg = pdq.step_cfg(dt, mode=mode, window_start=w0)
        C = len(st_plus)
        gbar = torch.zeros((C, samples, C), dtype=torch.float64, device="cuda")
        for c in range(C):
            gbar[c, :, c] = 1.0
        J, pbar = pdq.adjoint_run_seeded(field, phys, batch, pdq.params_tensor(x), cfg, steps, min(K, steps),
                                         eps, seed + 1, gbar=gbar, stream=stream, eps_stick=eps_stick)
        grad = pbar.permute(1, 0, 2).contiguous()          # [S, C, 3]
        nu, bound = pdq.dgsm_bounds(grad, J, hi - lo, stream=stream)
    return {"J": J.cpu().numpy(), "grad": grad.cpu().numpy(), "nu": nu, "bound": bound, "inputs": x}


def mfmc_sobol_deposition(budget, particles, steps, st_plus=(0.1, 1.0, 10.0),
                          ranges=((0.0, 0.1), (0.0, 1.0), (0.0, 1.0)), dt=0.05, t_window=10.0, pilot=64,
                          alloc_class=None, allocation=None, lf_nodes=2048, lf_precision=pdq.MIXED,
                          grid=(64, 32, 64), n_modes=64, seed=0, n_boot=200, precision=pdq.MIXED, stream=None):
    """Two-model MFMC Sobol' study of V_dep+ (Sec. 3): model 1 the batched particle model, model 2
    the 1-D Eulerian model of App. B (pdq_lf_vdep), as in the paper's study.

    A pilot of `pilot` input samples gives rho and sigma per class and the GPU cost per sample of
    each model (model 2 timed on a batch of 65,536 samples, large enough to fill the GPU);
    pdq_mfmc_allocate splits `budget` (in units of one particle-model pick-freeze group) for the
    class `alloc_class` (default: the class with the largest mean V_dep+) into m_1 groups of both
    models and m_2 >= m_1 groups of the 1-D model, nested (the first m_1 shared).  `allocation` =
    (m, alpha) skips the pilot.  Raises PdqError (PDQ_ERR_PRECOND) when the pilot correlation makes
    MFMC no better than plain Monte Carlo, and ValueError when the pilot's V_dep+ of that class does
    not vary.  Returns pdq.mfmc_sobol's dict plus the allocation, the
    pilot statistics, the two models' tables and their device times (ms).
    """
    lo = np.array([r[0] for r in ranges])
    hi = np.array([r[1] for r in ranges])
    d, C = len(ranges), len(st_plus)
    rng = np.random.Generator(np.random.Philox(seed))
    stream = stream or torch.cuda.Stream()
    with torch.cuda.stream(stream):
        phys = pdq.phys_default()
        field = pdq.Field(pdq.field_desc(n_r=grid[0], n_th=grid[1], n_z=grid[2], n_modes=n_modes), seed, stream)
        var = pdq.lf_fluid_variance(field, stream)
        lfd = pdq.lf_desc(n_y=lf_nodes, precision=lf_precision)

    def hf_run(inputs):
        return vdep_runs(inputs, particles, steps, st_plus=st_plus, dt=dt, t_window=t_window, precision=precision,
                         stream=stream, field=field, seed=seed)

    def lf_run(inputs):
        with torch.cuda.stream(stream):
            prm = pdq.params_tensor(np.asarray(inputs, np.float64))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y = pdq.lf_vdep(field, phys, lfd, var, st_plus, prm, stream=stream)
            e1.record(stream)
            e1.synchronize()
        return y.cpu().numpy(), e0.elapsed_time(e1)

    info = {}
    if allocation is None:
        xp_ = lo + (hi - lo) * rng.random((pilot, d))
        yh, th = hf_run(xp_)
        yl, _ = lf_run(xp_)
        _, tl = lf_run(lo + (hi - lo) * rng.random((65536, d)))
        w = np.array([th / pilot, tl / 65536])
        rho = np.array([np.corrcoef(yh[:, c], yl[:, c])[0, 1] if yh[:, c].std() > 0 and yl[:, c].std() > 0
                        else 0.0 for c in range(C)])
        sig = np.stack([yh.std(0, ddof=1), yl.std(0, ddof=1)], 1)
        cq = int(np.argmax(yh.mean(0))) if alloc_class is None else int(alloc_class)
        if not np.all(sig[cq] > 0):
            raise ValueError("the pilot saw no variation of V_dep+ in class %d: nothing to allocate for" % cq)
        m, alpha, m_real, gamma = pdq.mfmc_allocate([1.0, rho[cq]], sig[cq], w / w[0], budget)
        info.update(pilot={"samples": pilot, "rho": rho, "sigma": sig.T, "w_ms_per_sample": w, "class": cq},
                    gamma=gamma, m_real=m_real)
    else:
        m, alpha = allocation
    m1, m2 = max(2, int(m[0])), int(m[1])
    x = lo + (hi - lo) * rng.random((m2, d))
    xp = lo + (hi - lo) * rng.random((m2, d))
    groups = pick_freeze(x, xp)                                   # [m2, d+2, d]
    yh, th = hf_run(groups[:m1].reshape(-1, d))
    yl, tl = lf_run(groups.reshape(-1, d))
    yh = yh.reshape(m1, d + 2, C)
    yl = yl.reshape(m2, d + 2, C)
    with torch.cuda.stream(stream):
        out = pdq.mfmc_sobol([torch.tensor(yh, device="cuda"), torch.tensor(yl, device="cuda")], [m1, m2],
                             np.asarray(alpha, np.float64), n_boot=n_boot, seed=seed + 2, stream=stream)
    out.update(info)
    out.update(m=[m1, m2], alpha=np.asarray(alpha, np.float64), hf=yh, lf=yl, hf_ms=th, lf_ms=tl, inputs=groups)
    return out
