#!/usr/bin/env python
"""Throughput of the batched mixed-precision particle step on GB300.

One bench step = one time step of the whole ``batched_mixed`` workload (1,024
Monte Carlo samples, 4,096..32,768 particles each, 5 St+ classes): the
all-pairs Coulomb sum, interpolation, local forces, integration, wall contact,
tallies (and compaction every 100 steps), i.e. every per-step row of the hot
path.  Field build and seeding happen once before timing.

value  = particle-steps/s = sum over timed steps and samples of live particles
         / device time (CUDA events on the launching stream), summed over ranks
         and divided by the slowest rank's time.
e2e    = the same metric through the public API with the particle state in
         pinned host memory: each step uploads the state (positions, velocities,
         tags, counts), advances one step and downloads the state and the tallies.

``--impl reference`` times the FP64 CPU oracle (the only reference this paper
has) on a bounded sample of the same workload, on the host cores.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_2205_04979_gb300.clocks import ClockSampler  # noqa: E402

METRIC = "particle-steps/s, batched mixed vs plain FP64 on GB300 at ≤1e-3 rel V_dep error"
FLOPS_PER_PAIR = 21          # 3 sub, 4 minimum image, 5 r^2, 3 r^-3 q, 6 accumulate (FMA = 2); + 1 rsqrt
# pair variant 3 (Newton pairs, each unordered pair once): 3 sub, 5 r^2, 2 r^-3, 2 charge products and
# 12 for the six accumulating FMAs = 24 flops from 16 FP32-pipe lane-operations per unordered pair
NEWTON_FLOPS_PER_PAIR = 12   # per ordered pair
NEWTON_FLOPS_PER_LANE_OP = 24.0 / 16.0
# DRAM bytes per launch of the dominant kernel on 4,557,792 particles (ncu): k_step for pair variant 2,
# k_pairs_sym for pair variant 3
KSTEP_DRAM_BYTES = {2: 495.4e6, 3: 176.6e6}
# pipe peaks measured by the project microbenchmarks (python -m paper_2205_04979_gb300.peaks)
PEAKS_FILE = os.path.join(ROOT, "profiles", "peaks.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_mixed")
    ap.add_argument("--samples", type=int, default=None, help="truncate the workload (testing only)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-groups", type=int, default=2,
                    help="sample groups pipelined in the e2e measurement (1 = upload, step, download in turn)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--block", type=int, default=0, help="threads per CTA of the step kernel (0 = library default)")
    ap.add_argument("--variant", type=int, default=0, help="MIXED pair-math variant")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time direct launches instead of one graph launch")
    ap.add_argument("--vdep-classes", type=float, nargs="+", default=[0.1, 0.316, 1.0, 3.16, 10.0],
                    help="St+ classes of --workload vdep_validation")
    ap.add_argument("--vdep-steps", type=int, default=1200, help="steps of --workload vdep_validation")
    ap.add_argument("--clamp-check", action="store_true",
                    help="--workload vdep_validation: compare the Coulomb clamp at the largest and smallest diameter")
    ap.add_argument("--adjoint-config4", action="store_true",
                    help="--workload adjoint as stated: 2,000 steps, checkpoints every 100, three widths")
    ap.add_argument("--no-vdep-check", action="store_true")
    ap.add_argument("--particles", type=int, default=100_000, help="P3M workload: particles in the sample")
    ap.add_argument("--p3m-mesh", type=int, nargs=2, default=None, metavar=("M", "NZ"),
                    help="P3M mesh: cells across the diameter and nodes along z (default by particle count)")
    ap.add_argument("--lf", default="particle", choices=["particle", "eulerian"],
                    help="--workload mfmc: low-fidelity model (the particle model without the pair sum, or the "
                         "1-D Eulerian model of App. B)")
    ap.add_argument("--hf-particles", type=int, default=4096, help="--workload mfmc: particles per HF sample")
    ap.add_argument("--hf-steps", type=int, default=600, help="--workload mfmc: HF steps at dt+ = 0.05")
    ap.add_argument("--mfmc-budget", type=int, default=24, help="--workload mfmc: HF pick-freeze groups per study")
    ap.add_argument("--study-budget", type=int, default=200,
                    help="--workload mfmc: HF groups of the single study with bootstrap intervals (0: none)")
    ap.add_argument("--replicates", type=int, default=100,
                    help="--workload mfmc: replicate studies (0: pilot and allocation only)")
    ap.add_argument("--contact", action="store_true",
                    help="half the charges negative, soft-sphere collisions and particle-particle vdW on")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def pipe_peak(mixed, newton):
    """(peak TFLOP/s, note, instruction-mix peak or None) of the pair kernel's pipe, measured.

    FP32: the packed FFMA2 rate (fma.rn.f32x2, 4 flops per lane per instruction), the pipe's
    highest flop rate.  FP64: the DFMA rate.  The Newton-pair kernels issue 16 pipe operations
    (packed FP32 lane-operations, or FP64 operations) for 24 flops, so the secondary figure is
    the pipe's operation rate x 24/16: what the pipe delivers for that instruction mix.
    """
    from paper_2205_04979_gb300 import peaks as pk
    rec = pk.load(PEAKS_FILE)
    if rec is None:
        raise RuntimeError("no measured pipe peaks: run python -m paper_2205_04979_gb300.peaks --write %s"
                           % PEAKS_FILE)
    k = rec["kernels"]
    clk = rec["clocks"].get("sm_mhz")
    if mixed:
        peak = k["ffma2"]["flops_per_s"] / 1e12
        note = ("measured FP32 FFMA2 (packed f32x2) peak, %.2f TFLOP/s at %.0f MHz on %d SMs" %
                (peak, clk, rec["sms"]))
        ops = 2 * k["ffma2"]["lane_ops_per_s"]          # FP32 lane-operations per second
    else:
        peak = k["dfma"]["flops_per_s"] / 1e12
        note = "measured FP64 DFMA peak, %.3f TFLOP/s at %.0f MHz on %d SMs" % (peak, clk, rec["sms"])
        ops = k["dfma"]["lane_ops_per_s"]
    mix = None
    if newton:
        mix = {"peak": ops * NEWTON_FLOPS_PER_LANE_OP / 1e12,
               "note": "the measured pipe operation rate x 24 flops / 16 operations (Newton-pair mix)"}
    return peak, note, mix


def cpu_baseline(name, params, counts, seconds, steps_max=50):
    """Time the FP64 oracle on a bounded sample of the workload; extrapolate by pair count."""
    import oracle
    w = workloads.WORKLOADS[name]
    of = oracle.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    grid = oracle.field_grid(of, oracle.field_modes(of, w["field_seed"]))
    # sample: the first two samples of the workload
    k = min(2, len(counts))
    sp, sc = params[:k], counts[:k]
    ost, off = oracle.seed(of, w["st_plus"], sc, sp, w["particle_seed"], charge_sigma=w.get("charge_sigma", 0.0))
    c = oracle.cfg(w["dt"])
    t0 = time.perf_counter()
    n = 0
    nd = na = None
    while n < steps_max and (n == 0 or time.perf_counter() - t0 < seconds):
        nd, na = oracle.run(of, grid, c, w["st_plus"], off, sp, ost, 1, step0=n,
                            tallies=None if nd is None else (nd, na))
        n += 1
    dt = time.perf_counter() - t0
    pairs_sample = float(np.sum(np.asarray(sc, np.float64) ** 2)) * n
    t_pair = dt / pairs_sample
    full_pairs = float(np.sum(np.asarray(counts, np.float64) ** 2))
    value = float(np.sum(counts)) / (t_pair * full_pairs)
    return {"value": value, "unit": "particle-steps/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "FP64 oracle, %d samples (%s particles) x %d steps = %.1f s; extrapolated to the full "
                      "workload by sum N_s^2 (pair-dominated)" % (k, "+".join(str(int(x)) for x in sc), n, dt)}


def rank_workload(name, rank, world, samples=None):
    """(params, counts, ranges) of one rank.

    Under N ranks the study holds N times the workload's samples (drawn by the same seeded
    recipe, so its first samples are the single-GPU workload), partitioned into contiguous
    ranges balanced by sum N_s^2: each rank steps about one workload's worth (weak scaling).
    """
    from paper_2205_04979_gb300 import shard
    w = workloads.WORKLOADS[name]
    params, counts = workloads.workload_inputs(name, samples)
    if world == 1 or w["samples"] == 1:
        return params, counts, [(0, len(counts))]
    S = len(counts) * world
    params = workloads.sample_params(S, w["param_seed"])
    counts = workloads.sample_counts(S, w["count"][0], w["count"][1], w["param_seed"])
    ranges = shard.partition(counts, world)
    lo, hi = ranges[rank]
    return params[lo:hi], counts[lo:hi], ranges


def study_vdep(pdq, tally, ranges, rank, dt, r_plus, stream):
    """V_dep+ per class over the whole study: the ranks' tallies gathered in sample order, then
    pdq_deposition_tally once on the full [S][C] table (MC mean and SE over all samples)."""
    import torch
    from paper_2205_04979_gb300 import shard
    nd = shard.gather_rows(tally.n_dep, ranges, rank)
    na = shard.gather_rows(tally.n_alive, ranges, rank)
    full = pdq.Tally(nd.shape[0], nd.shape[1])
    full.n_dep.copy_(nd)
    full.n_alive.copy_(na)
    vdep, mean, se = pdq.deposition_tally(full, dt, r_plus, stream=stream)
    return {"samples": int(nd.shape[0]), "ranges": [list(r) for r in ranges],
            "deposits": int(nd.sum().item()), "vdep_mean": mean.cpu().tolist(), "vdep_se": se.cpu().tolist()}


def reduce_over_ranks(ms, psteps, world, device):
    """(slowest rank's time, particle-steps summed over ranks); no collective when world == 1."""
    if world == 1:
        return ms, float(psteps)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(psteps)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def vdep_check(pdq, stream, block, variant, samples=16, count=4096, steps=1200, dt=0.05, t_window=10.0,
               st_plus=None, param_seed=4242, min_deposits=1000):
    """V_dep+ of the batched MIXED path, in the timed launch configuration (block, pair variant),
    against the plain FP64 GPU path (Newton-pair sums in double) on the same seeds and inputs.

    Each sample draws its own particles (a Philox stream per sample), so the deposits are
    distinct events; both runs start from the same particles, so an event differs only where
    rounding moved a particle across the wall.  Per class: the deposits of
    each run, the events that differ (summed over samples), the relative error of the MC mean
    of V_dep+ and that error over the FP64 run's MC standard error.  The validity bar of the
    metric, relative error <= 1e-3 and error <= one SE, is judged only for classes with at
    least `min_deposits` FP64 deposits (fewer leave the relative error unresolved).
    """
    import torch
    w = workloads.WORKLOADS["batched_mixed"]
    st_plus = list(w["st_plus"] if st_plus is None else st_plus)
    params = workloads.sample_params(samples, param_seed)
    phys = pdq.phys_default()
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    field = pdq.Field(desc, w["field_seed"], stream)
    out, ms = {}, {}
    for name, prec in (("mixed", pdq.MIXED), ("fp64", pdq.FP64)):
        with torch.cuda.stream(stream):
            st = pdq.State(prec, [count] * samples, st_plus)
            prm = pdq.params_tensor(params)
            pdq.seed_particles_independent(field, phys, st, prm, w["particle_seed"], 0.0, stream)
            tile = dict(block=block, variant=variant) if prec == pdq.MIXED else dict(block=64, variant=3)
            cfg = pdq.step_cfg(dt, window_start=workloads.window_start_step(t_window, dt), compact_every=100, **tile)
            tally = pdq.Tally(samples, len(st_plus))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pdq.step_particles(field, phys, st, prm, cfg, steps, tally, pdq.workspace(st, cfg), stream)
            e1.record(stream)
            vdep, _, _ = pdq.deposition_tally(tally, dt, stream=stream)
            stream.synchronize()
            ms[name] = e0.elapsed_time(e1)
            out[name] = (vdep.cpu().numpy(), tally.n_dep.cpu().numpy())
            del st, tally
    vm, nm = out["mixed"]
    vf, nf = out["fp64"]
    mean_m, mean_f = vm.mean(0), vf.mean(0)
    se = vf.std(0, ddof=1) / np.sqrt(samples)
    diff = np.abs(mean_m - mean_f)
    rel = diff / np.where(mean_f > 0, mean_f, 1.0)
    over_se = diff / np.where(se > 0, se, 1.0)
    dep_f = nf.sum(0)
    judged = dep_f >= min_deposits
    return {"workload": "%d samples x %d particles (a particle stream per sample), St+ classes %s, %d steps at "
                        "dt+=%g, window t+>=%g" % (samples, count, st_plus, steps, dt, t_window),
            "mixed_tile": {"block": block, "variant": variant}, "fp64_tile": {"block": 64, "variant": 3},
            "vdep_fp64_mean": mean_f.tolist(), "vdep_mixed_mean": mean_m.tolist(), "mc_se_fp64": se.tolist(),
            "rel_err": rel.tolist(), "err_over_se": over_se.tolist(),
            "deposits_fp64": dep_f.tolist(), "deposits_mixed": nm.sum(0).tolist(),
            "events_differing": np.abs(nm - nf).sum(0).tolist(),
            "bar": "rel_err <= 1e-3 and err <= 1 SE, judged where the FP64 run has >= %d deposits" % min_deposits,
            "bar_met": [bool(rel[c] <= 1e-3 and diff[c] <= se[c]) if judged[c] else None
                        for c in range(len(st_plus))],
            "ms": {"mixed": ms["mixed"], "fp64": ms["fp64"]}}


def workload_label(name, counts, contact=False):
    """The workload description both arms print in config.workload."""
    w = workloads.WORKLOADS[name]
    return ("%s: %d samples, %d..%d particles each (%d total), %d St+ classes, %dx%dx%d field, dt+=%g, "
            "compaction every %d steps, %s" % (
                name, len(counts), int(np.min(counts)), int(np.max(counts)), int(np.sum(counts)),
                len(w["st_plus"]), *w["grid"], w["dt"], w.get("compact_every", 0), w["precision"]) +
            (" (z-binned, re-binned and compacted every 10 steps)"
             if w["precision"] == "mixed" and w.get("compact_every", 0) > 0 else "") +
            ("; half the charges negative, soft-sphere collisions and particle-particle vdW" if contact else ""))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "lf_eulerian":
        w = workloads.WORKLOADS["lf_eulerian"]
        S = args.samples or w["samples"]
        params = workloads.sample_params(S, w["param_seed"], spread=w["spread"])
        base = lf_cpu_baseline(w, params, seconds=max(5.0, 2.0 * (args.steps + args.warmup)))
        print(json.dumps({"impl": "reference", "metric": "low-fidelity evaluations/s (1-D Eulerian model of App. B, "
                                                         "sample x class items)",
                          "value": base["value"], "unit": "evaluations/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "lf_eulerian: %d samples x %d St+ classes" % (S, len(w["st_plus"]))},
                          "cpu_baseline": base,
                          "e2e": {"value": base["value"], "unit": "evaluations/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    params, counts = workloads.workload_inputs(args.workload, args.samples)
    base = cpu_baseline(args.workload, params, counts, seconds=max(5.0, 4.0 * (args.steps + args.warmup)),
                        steps_max=args.steps + args.warmup)
    out = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "particle-steps/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_label(args.workload, counts, args.contact)},
           "cpu_baseline": base,
           "e2e": {"value": base["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_e2e(pdq, field, phys, state, prm, cfg, w, args, stream):
    """End-to-end particle-steps/s through the public API, host state in pinned memory."""
    import torch
    S = state.n_samples
    G = max(1, min(args.e2e_groups, S))
    bounds = [S * k // G for k in range(G + 1)]
    off = state.offset.cpu().numpy()
    pos, vel, xy = state.current()
    groups = []
    for k in range(G):
        s0, s1 = bounds[k], bounds[k + 1]
        o0, o1 = int(off[s0]), int(off[s1])
        st = pdq.State(state.precision, state.counts0[s0:s1], state.st_plus)
        st.pos[0].copy_(pos[o0:o1])
        st.vel[0].copy_(vel[o0:o1])
        if xy is not None:
            st.xy[0].copy_(xy[o0:o1])
        st.tag.copy_(state.tag[o0:o1])
        st.count.copy_(state.count[s0:s1])
        st.ctl[0] = state.step_index
        st.st.step = state.step_index
        tl = pdq.Tally(s1 - s0, state.n_classes)
        dev = [t for t in st.current() if t is not None] + [st.tag, st.count]
        hosts = [t.cpu().pin_memory() for t in dev]
        htal = [tl.n_alive.cpu().pin_memory(), tl.n_dep.cpu().pin_memory()]
        groups.append(dict(st=st, tally=tl, prm=prm[s0:s1], ws=pdq.workspace(st, cfg), hosts=hosts, htal=htal))
    torch.cuda.synchronize()

    def dev_state(st):
        return [t for t in st.current() if t is not None] + [st.tag, st.count]

    h2d = sum(sum(t.numel() * t.element_size() for t in g["hosts"]) for g in groups)
    d2h = h2d + sum(sum(t.numel() * t.element_size() for t in g["htal"]) for g in groups)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def one_step():
        # no host synchronisation between steps: a group's upload waits on the copy-out stream's
        # event of its previous download (the host buffers it reads), so copies of one step
        # overlap the other groups' steps of the next one as well
        for g in groups:
            with torch.cuda.stream(s_in):
                if g.get("ev_out") is not None:
                    s_in.wait_event(g["ev_out"])
                for dst, src in zip(dev_state(g["st"]), g["hosts"]):
                    dst.copy_(src, non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(s_in)
            stream.wait_event(ev_in)
            pdq.step_particles(field, phys, g["st"], g["prm"], cfg, 1, g["tally"], g["ws"], stream)
            ev_done = torch.cuda.Event()
            ev_done.record(stream)
            s_out.wait_event(ev_done)
            with torch.cuda.stream(s_out):
                for dst, src in zip(g["hosts"], dev_state(g["st"])):
                    dst.copy_(src, non_blocking=True)
                g["htal"][0].copy_(g["tally"].n_alive, non_blocking=True)
                g["htal"][1].copy_(g["tally"].n_dep, non_blocking=True)
                g["ev_out"] = torch.cuda.Event()
                g["ev_out"].record(s_out)

    one_step()                                       # untimed warm-up (first calls read offsets)
    torch.cuda.synchronize()
    alive0 = sum(int(g["tally"].n_alive.sum().item()) for g in groups)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        one_step()
    s_out.synchronize()                              # every download of the last step has landed
    te = time.perf_counter() - t0
    torch.cuda.synchronize()
    alive = sum(int(g["tally"].n_alive.sum().item()) for g in groups) - alive0
    return {"value": float(alive) / te, "unit": "particle-steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "sample_groups": G, "ms": te * 1e3, "particle_steps": float(alive)}


def run_ours(args):
    import torch
    import paper_2205_04979_gb300.pdq as pdq

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = workloads.WORKLOADS[args.workload]
    params, counts, ranges = rank_workload(args.workload, rank, world, args.samples)
    prec = pdq.MIXED if w["precision"] == "mixed" else pdq.FP64
    phys = pdq.phys_default()
    if args.contact:
        phys.neg_charge_frac = 0.5
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        field = pdq.Field(desc, w["field_seed"], stream)
        state = pdq.State(prec, counts, w["st_plus"])
        prm = pdq.params_tensor(params)
        pdq.seed_particles(field, phys, state, prm, w["particle_seed"], w.get("charge_sigma", 0.0), stream)
        cfg = pdq.step_cfg(w["dt"], window_start=0, compact_every=w.get("compact_every", 0), block=args.block,
                           variant=args.variant, forces=pdq.F_ALL | (pdq.F_CONTACT if args.contact else 0))
        tally = pdq.Tally(len(counts), len(w["st_plus"]))
        if args.block == 0 and args.variant == 0 and not args.no_autotune:
            pdq.autotune(field, phys, state, prm, cfg, stream)      # project autotuner picks block / variant
        ws = pdq.workspace(state, cfg)
        pdq.step_particles(field, phys, state, prm, cfg, args.warmup, tally, ws, stream)
        stream.synchronize()
        assert pdq.check_state(state, stream) == 0
        cnt0 = state.count.cpu().numpy().astype(np.float64)
        alive0 = int(tally.n_alive.sum().item())
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        # the K timed steps run as one CUDA-graph launch: captured and instantiated here (use_graph
        # = 2 runs nothing), replayed in the timed region
        gcfg = pdq.StepCfg.from_buffer_copy(cfg)
        if not args.no_graph:
            gcfg.use_graph = 2
            pdq.step_particles(field, phys, state, prm, gcfg, args.steps, tally, ws, stream)
            gcfg.use_graph = 1
            stream.synchronize()
        clk = ClockSampler(uuid)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pdq.step_particles(field, phys, state, prm, gcfg, args.steps, tally, ws, stream)
        e1.record(stream)
        e1.synchronize()
        clocks = clk.stop()
        pdq.release_graphs()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        assert pdq.check_state(state, stream) == 0
        cnt1 = state.count.cpu().numpy().astype(np.float64)
        psteps = int(tally.n_alive.sum().item()) - alive0
        pairs = 0.5 * (np.sum(cnt0 ** 2) + np.sum(cnt1 ** 2)) * args.steps
        s0 = state.step_index - args.steps
        # the step z-bins (and compacts, when compaction is on) at the start of a call and every
        # min(compact_every, 10) steps, 10 without compaction; both precisions
        ci = min(cfg.compact_every, 10) if cfg.compact_every > 0 else 10
        n_rebin = sum(1 for k in range(args.steps - 1) if (s0 + k + 1) % ci == 0)
        # sort, build_items, the step kernel(s) per step (Newton pairs: pair sums + update), re-bin + items
        per_step = 2 if cfg.variant == 3 and (not args.contact or prec == pdq.MIXED) else 1
        launches = 1 + 1 + per_step * args.steps + 2 * n_rebin

        # e2e: state in pinned host memory; every step uploads the state, steps it and downloads the
        # state and the tallies.  The batch is cut into --e2e-groups contiguous sample groups, each
        # a state of its own; group g's upload (copy-in stream), step (compute stream) and
        # download (copy-out stream) are ordered by events, so copies overlap other groups' steps.
        e2e = None
        if args.e2e_steps > 0:
            e2e = run_e2e(pdq, field, phys, state, prm, cfg, w, args, stream)
            # whole job: particle-steps of all ranks over the slowest rank's time, bytes summed
            te_ms, alive_all = reduce_over_ranks(e2e.pop("ms"), e2e.pop("particle_steps"), world, "cuda")
            e2e["value"] = alive_all / (te_ms / 1e3)
            if world > 1:
                _, h2d_all = reduce_over_ranks(0.0, e2e["h2d_bytes_per_step"], world, "cuda")
                _, d2h_all = reduce_over_ranks(0.0, e2e["d2h_bytes_per_step"], world, "cuda")
                e2e["h2d_bytes_per_step"], e2e["d2h_bytes_per_step"] = int(h2d_all), int(d2h_all)

        # plain FP64 single-sample path (the comparison the metric names)
        fp64 = None
        if not args.no_fp64 and rank == 0 and args.workload == "batched_mixed":
            w1 = workloads.WORKLOADS["single_fp64"]
            d1 = pdq.field_desc(n_r=w1["grid"][0], n_th=w1["grid"][1], n_z=w1["grid"][2], n_modes=w1["n_modes"])
            f1 = pdq.Field(d1, w1["field_seed"], stream)
            s1 = pdq.State(pdq.FP64, [w1["count"]], w1["st_plus"])
            p1 = pdq.params_tensor([workloads.NOMINAL])
            pdq.seed_particles(f1, phys, s1, p1, w1["particle_seed"], 0.0, stream)
            c1 = pdq.step_cfg(w1["dt"], window_start=0, use_graph=True)
            pdq.autotune(f1, phys, s1, p1, c1, stream)
            t1 = pdq.Tally(1, 1)
            ws1 = pdq.workspace(s1, c1)
            pdq.step_particles(f1, phys, s1, p1, c1, 20, t1, ws1, stream)
            a1 = t1.n_alive.sum().item()
            x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x0.record(stream)
            pdq.step_particles(f1, phys, s1, p1, c1, w1["steps"], t1, ws1, stream)
            x1.record(stream)
            x1.synchronize()
            fp64 = {"workload": "single_fp64 (1 sample x 1,000 particles, St+=10, 64x32x64 field, dt+=0.1)",
                    "value": (t1.n_alive.sum().item() - a1) / (x0.elapsed_time(x1) / 1e3),
                    "unit": "particle-steps/s", "steps": w1["steps"], "block": c1.block}

    ms_max, psteps_all = reduce_over_ranks(ms, psteps, world, "cuda")
    study = None
    if world > 1:
        with torch.cuda.stream(stream):
            study = study_vdep(pdq, tally, ranges, rank, w["dt"], desc.r_plus, stream)
    if rank != 0:
        return
    newton = cfg.variant == 3 and (not args.contact or prec == pdq.MIXED)
    flops_per_pair = NEWTON_FLOPS_PER_PAIR if newton else FLOPS_PER_PAIR
    peak_tflops, peak_note, mix = pipe_peak(prec == pdq.MIXED, newton)
    achieved = flops_per_pair * pairs / (ms / 1e3) / 1e12
    if mix is not None:
        mix["frac"] = achieved / mix["peak"]
    out = {
        "metric": METRIC, "value": psteps_all / (ms_max / 1e3), "unit": "particle-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == pdq.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": workload_label(args.workload, counts, args.contact),
                   "l2": "inputs larger than L2 (particle state %.2f GB)" % (
                       sum(t.numel() * t.element_size() for t in state.current() if t is not None) / 1e9),
                   "parallelism": ("one study of %d samples in contiguous ranges balanced by sum N_s^2, one "
                                   "per rank; tallies gathered at the end" % sum(h - l for l, h in ranges))
                   if world > 1 else "1 GPU",
                   "launch": "direct" if args.no_graph else "one CUDA-graph launch of the timed steps",
                   "tile": {"block": cfg.block,
                            "i_per_thread": ((12 if not args.contact else 8) if newton else
                                             8 if cfg.variant == 2 and not args.contact else 4)
                            if prec == pdq.MIXED else (2 if newton else 1),
                            "variant": cfg.variant, "autotuned": args.block == 0 and not args.no_autotune}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "instruction_mix": mix,
                     # dram bytes read + written per launch from ncu captures of the pair
                     # kernels (pair variant 2: 495.4 MB, variant 3: 176.6 MB, both on
                     # 4,557,792 particles), scaled by the particle count of this launch; null
                     # for a variant without a capture of its kernel
                     "traffic": KSTEP_DRAM_BYTES[cfg.variant] / 4557792 * float(np.sum(counts))
                     if prec == pdq.MIXED and cfg.variant in KSTEP_DRAM_BYTES and not args.contact else None,
                     "kernel": ("k_pairs_sym (Newton-pair Coulomb sums), then the k_step contact variant "
                                "taking them (near pairs, contact forces, update)" if args.contact else
                                "k_pairs_sym (Newton-pair Coulomb sums), then the given-sums k_step update"
                                if prec == pdq.MIXED else
                                "k_pairs_sym64 (FP64 Newton-pair Coulomb sums), then the given-sums k_step update")
                               if newton else "k_step (all-pairs Coulomb + local step)",
                     "note": "%s; %d flops per ordered pair; time per step from CUDA events over the timed "
                             "region%s" % (peak_note, flops_per_pair,
                                           " (both kernels and the zeroing of the sums: a lower bound on the "
                                           "pair kernel's own rate)" if newton else "")},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "plain_fp64": fp64,
    }
    if study is not None:
        out["study"] = study
    if not args.no_vdep_check and rank == 0 and args.workload == "batched_mixed":
        out["vdep_check"] = vdep_check(pdq, stream, cfg.block, cfg.variant)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, params, counts, args.cpu_seconds)
    print(json.dumps(out), flush=True)


def run_adjoint_config4(args):
    """The adjoint workload as stated: 256 samples x 16,384 particles, 2,000 steps, a checkpoint
    every 100 steps, eps+ = 0.5, 0.1, 0.02: one forward + reverse sweep per width."""
    import torch
    import paper_2205_04979_gb300.pdq as pdq
    w = workloads.WORKLOADS["adjoint"]
    S, steps, K = w["samples"], w["steps"], w["checkpoint"]
    params = workloads.sample_params(S, w["param_seed"])
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    phys = pdq.phys_default()
    out = {"metric": "gradient particle-steps/s (smoothed V_dep, forward + reverse sweep)", "unit": "particle-steps/s",
           "n_gpus": 1, "steps": steps, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "adjoint: %d samples x %d particles, classes %s, %d steps, checkpoint every %d steps"
                                  % (S, w["count"], w["st_plus"], steps, K)}, "eps": {}}
    with torch.cuda.stream(stream):
        field = pdq.Field(pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2],
                                         n_modes=w["n_modes"]), w["field_seed"], stream)
        batch = pdq.Batch(pdq.MIXED, [w["count"]] * S, w["st_plus"])
        cfg = pdq.step_cfg(w["dt"], window_start=workloads.window_start_step(w["t_window"], w["dt"]))
        prm = pdq.params_tensor(params)
        C = len(w["st_plus"])
        gbar = torch.ones((1, S, C), dtype=torch.float64, device="cuda")   # d(sum_c J_c)/d(xi, zeta, theta)
        # keep every step's Newton-pair sums for the reverse sweep when the GPU has room for them
        need = pdq.adjoint_workspace_bytes(batch.b, steps, K)
        extra = pdq.adjoint_workspace_bytes(batch.b, steps, K, store_sums=True) - need
        store = torch.cuda.mem_get_info()[0] > need + extra + (8 << 30)
        ws = pdq.adjoint_workspace(batch.b, steps, K, store_sums=store)
        out["workspace_bytes"] = int(ws.numel())
        out["stored_sums"] = bool(store)
        pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, 4, 2, w["eps"][0], w["particle_seed"], gbar=gbar,
                               stream=stream)             # warm-up
        for eps in w["eps"]:
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            J, _ = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, steps, K, eps, w["particle_seed"], ws=ws,
                                          stream=stream)     # forward sweep alone (checkpoints kept)
            e1.record(stream)
            pbar = pdq.adjoint_reverse(field, phys, batch.b, prm, cfg, steps, K, eps, gbar, ws, stream=stream)
            e2.record(stream)
            e2.synchronize()
            fwd, rev = e0.elapsed_time(e1), e1.elapsed_time(e2)
            psteps = float(S) * w["count"] * steps
            g = pbar.cpu().numpy()[0]                       # [S, 3]
            out["eps"][str(eps)] = {
                "forward_ms": fwd, "reverse_ms": rev,
                "value": psteps / ((fwd + rev) / 1e3), "forward_only": psteps / (fwd / 1e3),
                "J_mean": J.mean(0).cpu().numpy().tolist(),
                "grad_sumJ_mean_abs": np.abs(g).mean(axis=0).tolist()}
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Forward + reverse sweep of the smoothed-V_dep adjoint on 256 samples x 16,384 particles, with
    the forward sweep's Newton-pair sums kept for the reverse sweep (and, for comparison, with the
    reverse sweep recomputing them)."""
    import torch
    import paper_2205_04979_gb300.pdq as pdq
    if args.adjoint_config4:
        return run_adjoint_config4(args)
    w = workloads.WORKLOADS["adjoint"]
    S = args.samples or w["samples"]
    params = workloads.sample_params(S, w["param_seed"])
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    phys = pdq.phys_default()
    K = min(w["checkpoint"], max(1, args.steps // 2))
    with torch.cuda.stream(stream):
        field = pdq.Field(pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2],
                                         n_modes=w["n_modes"]), w["field_seed"], stream)
        batch = pdq.Batch(pdq.MIXED, [w["count"]] * S, w["st_plus"])
        cfg = pdq.step_cfg(w["dt"], window_start=0)
        prm = pdq.params_tensor(params)
        gbar = torch.ones((1, S, len(w["st_plus"])), dtype=torch.float64, device="cuda")
        timed = {}
        for store in (False, True):
            pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, max(2, args.warmup), 1, w["eps"][1],
                                   w["particle_seed"], gbar=gbar, stream=stream, store_sums=store)
            ws = pdq.adjoint_workspace(batch.b, args.steps, K, store_sums=store)
            stream.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            J, _ = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, args.steps, K, w["eps"][1],
                                          w["particle_seed"], stream=stream, ws=ws)
            e[1].record(stream)
            J2, pbar = pdq.adjoint_run_seeded(field, phys, batch, prm, cfg, args.steps, K, w["eps"][1],
                                              w["particle_seed"], gbar=gbar, stream=stream, ws=ws)
            e[2].record(stream)
            e[2].synchronize()
            timed[store] = (e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), J2, pbar)
            del ws
    fwd_ms, tot_ms, J2, pbar = timed[True]
    rec_ms = timed[False][1]
    psteps = float(S) * w["count"] * args.steps
    out = {"metric": "gradient particle-steps/s (smoothed V_dep, forward + reverse sweep)",
           "value": psteps / (tot_ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "adjoint: %d samples x %d particles, classes %s, checkpoint every %d steps, "
                                  "eps+=%g, forward sweep's pair sums kept for the reverse sweep"
                                  % (S, w["count"], w["st_plus"], K, w["eps"][1])},
           "forward_only": {"value": psteps / (fwd_ms / 1e3), "unit": "particle-steps/s"},
           "recomputed_sums": {"value": psteps / (rec_ms / 1e3), "unit": "particle-steps/s",
                               "ms_per_step": rec_ms / args.steps},
           "grad_mean_abs": np.abs(pbar.cpu().numpy()).mean(axis=(0, 1)).tolist(),
           "J_mean": J2.mean(0).cpu().numpy().tolist()}
    print(json.dumps(out), flush=True)


def _finite(x):
    """JSON-safe copy of nested lists: non-finite entries (classes with zero variance) become null."""
    if isinstance(x, list):
        return [_finite(v) for v in x]
    return x if np.isfinite(x) else None


def run_sobol(args):
    """End-to-end Sobol' study of V_dep+ (high-fidelity model only) through paper_2205_04979_gb300.uq."""
    import torch
    from paper_2205_04979_gb300 import uq, pdq
    torch.cuda.set_device(0)
    m = args.samples or 64
    uq.sobol_deposition(4, 1024, 10)                          # warm-up (builds, first launches)
    r = uq.sobol_deposition(m, 4096, args.steps, n_boot=200)
    rc = uq.sobol_deposition(m, 4096, args.steps, n_boot=200, mode=pdq.REBOUND, qoi="ce")
    out = {"metric": "Sobol' study: particle-steps/s of the pick-freeze runs", "value": r["particle_steps"] / (
               r["ms"] / 1e3), "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "sobol: %d pick-freeze groups x 5 runs x 4096 particles, classes (0.1, 1, 10), "
                                  "xi in [0, 0.1], zeta in [0, 1], theta in [0, 1]" % m},
           "mean_vdep": _finite(r["mean"].tolist()), "s_main": _finite(r["s_main"].tolist()), "s_total": _finite(r["s_total"].tolist()),
           "s_main_ci": _finite(r["s_main_ci"].tolist()),
           "ce_rebound": {"mean": _finite(rc["mean"].tolist()), "s_main": _finite(rc["s_main"].tolist()),
                          "s_total": _finite(rc["s_total"].tolist())}}
    print(json.dumps(out), flush=True)


def run_mfmc(args):
    """Config 5 with the models this build has: MFMC (Sec. 3) against plain MC at equal GPU cost.

    High fidelity: the batched particle model, 4,096 particles per sample, dt+ = 0.05, 600 steps.
    Low fidelity: the same particles without the particle-particle Coulomb sum and with 2x dt
    (300 steps to the same t+ = 30).  A pilot gives rho, sigma and the measured GPU time per sample w of each model;
    pdq_mfmc_allocate gives m and alpha.  R replicate studies, each with fresh pick-freeze
    groups, measure the variance of the MFMC and plain-MC estimates of the mean V_dep+ and of
    the Sobol' indices at the same budget; the variance ratio of the mean is reported beside
    gamma(rho, w).  Then one MFMC and one plain-MC Sobol' study at a larger budget, and the
    MIXED-vs-FP64 comparison of the Sobol' indices on the same inputs.

    --lf eulerian: the low-fidelity model is the 1-D Eulerian model of App. B (pdq_lf_vdep, the
    paper's own choice of low-fidelity model), its cost per sample measured on a batch of 65,536
    samples; the MIXED-vs-FP64 comparison is left to the default mode.  --hf-particles and
    --hf-steps size the particle model; --replicates 0 stops after the pilot and the allocation.
    """
    import torch
    from paper_2205_04979_gb300 import pdq, uq
    torch.cuda.set_device(0)
    st_plus = (0.1, 1.0, 10.0)
    ranges = ((0.0, 0.1), (0.0, 1.0), (0.0, 1.0))
    lo, hi = np.array([r[0] for r in ranges]), np.array([r[1] for r in ranges])
    d, C = 3, len(st_plus)
    hf = dict(particles=args.hf_particles, steps=args.hf_steps, dt=0.05, forces=pdq.F_ALL)
    lf = dict(particles=args.hf_particles, steps=args.hf_steps // 2, dt=0.10, forces=pdq.F_ALL & ~pdq.F_COULOMB)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        field = pdq.Field(pdq.field_desc(n_r=64, n_th=32, n_z=64), 0, stream)

    eulerian = args.lf == "eulerian"
    if eulerian:
        with torch.cuda.stream(stream):
            lf_var = pdq.lf_fluid_variance(field, stream)
        lf_desc = pdq.lf_desc()
        lf_phys = pdq.phys_default()

    def run_eulerian(inputs):
        with torch.cuda.stream(stream):
            prm = pdq.params_tensor(np.asarray(inputs, np.float64))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y = pdq.lf_vdep(field, lf_phys, lf_desc, lf_var, st_plus, prm, stream=stream)
            e1.record(stream)
            e1.synchronize()
        return y.cpu().numpy(), e0.elapsed_time(e1)

    def run(model, inputs, precision=pdq.MIXED, chunk=12000):
        if eulerian and model is lf:
            return run_eulerian(inputs)
        outs, ms = [], 0.0
        for a in range(0, len(inputs), chunk):
            y, t = uq.vdep_runs(inputs[a:a + chunk], model["particles"], model["steps"], st_plus=st_plus,
                                dt=model["dt"], forces=model["forces"], precision=precision, stream=stream,
                                field=field)
            outs.append(y)
            ms += t
        return np.concatenate(outs, 0), ms

    def draw(n, seed):
        rng = np.random.Generator(np.random.Philox(seed))
        x = lo + (hi - lo) * rng.random((n, d))
        xp = lo + (hi - lo) * rng.random((n, d))
        return uq.pick_freeze(x, xp)                        # [n, d+2, d]

    run(hf, draw(4, 1).reshape(-1, d))                      # warm-up: builds, autotuner caches
    run(lf, draw(4, 1).reshape(-1, d))
    # pilot: rho, sigma per class and the GPU cost per sample of each model
    npil = args.samples or 256
    xpil = lo + (hi - lo) * np.random.Generator(np.random.Philox(11)).random((npil, d))
    yh, th = run(hf, xpil)
    yl, tl = run(lf, xpil)
    w = np.array([th / npil, tl / npil])                    # ms per sample
    if eulerian:                                            # cost per sample on a batch that fills the GPU
        nb = 65536
        _, tb = run(lf, lo + (hi - lo) * np.random.Generator(np.random.Philox(12)).random((nb, d)))
        w[1] = tb / nb
    rho = np.array([np.corrcoef(yh[:, c], yl[:, c])[0, 1] for c in range(C)])
    sig = np.stack([yh.std(0, ddof=1), yl.std(0, ddof=1)], 1)
    cq = int(np.argmax(yh.mean(0)))                         # allocate for the class with most deposition
    p_eff = args.mfmc_budget                                # budget: HF pick-freeze groups per study
    wn = w / w[0]                                           # costs in units of one HF evaluation
    try:
        m, alpha, m_real, gamma = pdq.mfmc_allocate([1.0, rho[cq]], sig[cq], wn, p_eff)
    except pdq.PdqError as e:                               # precondition violated: MFMC does not pay
        print(json.dumps({"metric": "MFMC vs plain MC", "pilot": {"rho": _finite(rho.tolist()),
                          "w_ms_per_sample": w.tolist()}, "allocation_error": str(e)}), flush=True)
        return
    m1, m2 = max(2, int(m[0])), int(m[1])
    gam = [float((np.sqrt(1 - r ** 2) + r * np.sqrt(w[1] / w[0])) ** 2) for r in rho]

    def fin(a):
        return _finite(np.asarray(a).tolist())
    pilot = {"samples": npil, "rho": fin(rho), "sigma": fin(sig.T), "w_ms_per_sample": fin(w),
             "allocation_class": st_plus[cq], "m": [m1, m2], "alpha": fin(alpha),
             "gamma_predicted_per_class": fin(gam), "gamma_allocation": gamma,
             "hf_mean": fin(yh.mean(0)), "lf_mean": fin(yl.mean(0)),
             "hf_deposits_per_sample_approx": fin(yh.mean(0) * (args.hf_particles / C) *
                                                (hf["steps"] * hf["dt"] - 10.0) / 90.0)}
    hf_label = ("HF = particle model %d particles/sample, dt+ 0.05, %d steps" % (args.hf_particles, args.hf_steps))
    if args.replicates == 0:
        print(json.dumps({"metric": "MFMC pilot: correlation of the low-fidelity model with the particle model",
                          "config": {"workload": "mfmc pilot: %s; LF = %s; classes %s; inputs xi [0,0.1], zeta "
                                                 "[0,1], theta [0,1]" % (hf_label, "1-D Eulerian model" if eulerian
                                                                         else "particle model without the pair "
                                                                              "sum, 2x dt", list(st_plus))},
                          "pilot": pilot}), flush=True)
        return
    # replicates: HF on the first p_eff groups (MC uses them all, MFMC the first m1), LF on m2
    R = args.replicates
    groups = [draw(max(p_eff, m2), 1000 + r) for r in range(R)]
    y_hf, t_hf = run(hf, np.concatenate([g[:p_eff] for g in groups]).reshape(-1, d))
    y_lf, t_lf = run(lf, np.concatenate([g[:m2] for g in groups]).reshape(-1, d))
    y_hf = y_hf.reshape(R, p_eff, d + 2, C)
    y_lf = y_lf.reshape(R, m2, d + 2, C)
    est = {"mc": [], "mfmc": []}
    for r in range(R):
        a = torch.tensor(y_hf[r], device="cuda")
        b = torch.tensor(y_lf[r], device="cuda")
        est["mc"].append(pdq.mfmc_sobol([a], [p_eff], [1.0], stream=stream))
        est["mfmc"].append(pdq.mfmc_sobol([a[:m1], b], [m1, m2], alpha, stream=stream))

    def var_of(key, q):
        return np.var(np.array([e[q] for e in est[key]]), axis=0, ddof=1)
    def ratio(q):
        a, b = var_of("mfmc", q), var_of("mc", q)
        return np.where(b > 0, a / np.where(b > 0, b, 1.0), np.nan)
    ratio_mean, ratio_sm, ratio_st = ratio("mean"), ratio("s_main"), ratio("s_total")
    rep_means = {key: fin(np.mean(np.array([e["mean"] for e in est[key]]), axis=0)) for key in est}
    if eulerian and args.study_budget == 0:
        print(json.dumps({
            "metric": "MFMC vs plain MC at equal GPU cost, low fidelity = the 1-D Eulerian model (App. B)",
            "config": {"workload": "mfmc: %s; LF = 1-D Eulerian model, %d wall-normal nodes; classes %s; inputs xi "
                                   "[0,0.1], zeta [0,1], theta [0,1]" % (hf_label, lf_desc.n_y, list(st_plus))},
            "pilot": pilot,
            "replicates": {"R": R, "budget_hf_groups": p_eff, "mc_groups": p_eff, "mfmc_groups": [m1, m2],
                           "var_ratio_mean": fin(ratio_mean), "var_ratio_s_main": fin(ratio_sm),
                           "var_ratio_s_total": fin(ratio_st), "mean_of_estimates": rep_means,
                           "gpu_ms": {"hf_all": t_hf, "lf_all": t_lf, "mc_per_study": w[0] * p_eff * (d + 2),
                                      "mfmc_per_study": (w[0] * m1 + w[1] * m2) * (d + 2)}}}), flush=True)
        return
    # one study at a larger budget, MFMC and plain MC, with bootstrap intervals
    pb = args.study_budget
    mb, ab, _, gb = pdq.mfmc_allocate([1.0, rho[cq]], sig[cq], wn, pb)
    gbig = draw(max(pb, int(mb[1])), 7)
    yhb, thb = run(hf, gbig[:pb].reshape(-1, d))
    ylb, tlb = run(lf, gbig[:int(mb[1])].reshape(-1, d))
    yhb = torch.tensor(yhb.reshape(pb, d + 2, C), device="cuda")
    ylb = torch.tensor(ylb.reshape(-1, d + 2, C), device="cuda")
    big_mc = pdq.mfmc_sobol([yhb], [pb], [1.0], n_boot=200, seed=3, stream=stream)
    big_mf = pdq.mfmc_sobol([yhb[:int(mb[0])], ylb], [int(mb[0]), int(mb[1])], ab, n_boot=200, seed=3,
                            stream=stream)
    if eulerian:
        print(json.dumps({
            "metric": "MFMC vs plain MC at equal GPU cost, low fidelity = the 1-D Eulerian model (App. B)",
            "config": {"workload": "mfmc: %s; LF = 1-D Eulerian model, %d wall-normal nodes; classes %s; inputs xi "
                                   "[0,0.1], zeta [0,1], theta [0,1]" % (hf_label, lf_desc.n_y, list(st_plus))},
            "pilot": pilot,
            "replicates": {"R": R, "budget_hf_groups": p_eff, "mc_groups": p_eff, "mfmc_groups": [m1, m2],
                           "var_ratio_mean": fin(ratio_mean), "var_ratio_s_main": fin(ratio_sm),
                           "var_ratio_s_total": fin(ratio_st),
                           "gpu_ms": {"hf_all": t_hf, "lf_all": t_lf, "mc_per_study": w[0] * p_eff * (d + 2),
                                      "mfmc_per_study": (w[0] * m1 + w[1] * m2) * (d + 2)}},
            "study": {"budget_hf_groups": pb, "mfmc_m": [int(mb[0]), int(mb[1])], "gamma": gb,
                      "mc": {k: fin(v) for k, v in big_mc.items()},
                      "mfmc": {k: fin(v) for k, v in big_mf.items()}}}), flush=True)
        return
    # MIXED vs FP64 Sobol' indices of the high-fidelity model on the same 64 groups
    g64 = draw(64, 9).reshape(-1, d)
    ym, tm = run(hf, g64, pdq.MIXED)
    yf, tf = run(hf, g64, pdq.FP64)
    sm = pdq.mfmc_sobol([torch.tensor(ym.reshape(64, d + 2, C), device="cuda")], [64], [1.0], n_boot=200, seed=5)
    sf = pdq.mfmc_sobol([torch.tensor(yf.reshape(64, d + 2, C), device="cuda")], [64], [1.0], n_boot=200, seed=5)
    half = 0.5 * (sf["s_main_ci"][..., 1] - sf["s_main_ci"][..., 0])
    halft = 0.5 * (sf["s_total_ci"][..., 1] - sf["s_total_ci"][..., 0])
    dm, dt_ = np.abs(sm["s_main"] - sf["s_main"]), np.abs(sm["s_total"] - sf["s_total"])
    out = {"metric": "MFMC vs plain MC at equal GPU cost: variance of the estimates over replicate studies",
           "config": {"workload": "mfmc: HF = particle model 4,096 particles/sample, dt+ 0.05, 600 steps; LF = same "
                                  "without the Coulomb pair sum, dt+ 0.1, 300 steps; classes %s; inputs xi [0,0.1], "
                                  "zeta [0,1], theta [0,1]" % (list(st_plus),)},
           "pilot": {"samples": npil, "rho": fin(rho), "sigma": fin(sig.T), "w_ms_per_sample": fin(w),
                     "allocation_class": st_plus[cq], "m": [m1, m2], "alpha": fin(alpha),
                     "gamma_predicted_per_class": fin(gam), "gamma_allocation": gamma},
           "replicates": {"R": R, "budget_hf_groups": p_eff, "mc_groups": p_eff, "mfmc_groups": [m1, m2],
                          "var_ratio_mean": fin(ratio_mean), "var_ratio_s_main": fin(ratio_sm),
                          "var_ratio_s_total": fin(ratio_st),
                          "gpu_ms": {"hf_all": t_hf, "lf_all": t_lf,
                                     "mc_per_study": w[0] * p_eff * (d + 2),
                                     "mfmc_per_study": (w[0] * m1 + w[1] * m2) * (d + 2)}},
           "study": {"budget_hf_groups": pb, "mfmc_m": [int(mb[0]), int(mb[1])], "gamma": gb,
                     "mc": {k: fin(v) for k, v in big_mc.items()}, "mfmc": {k: fin(v) for k, v in big_mf.items()}},
           "mixed_vs_fp64_sobol": {"groups": 64, "s_main_mixed": fin(sm["s_main"]), "s_main_fp64": fin(sf["s_main"]),
                                   "s_total_mixed": fin(sm["s_total"]), "s_total_fp64": fin(sf["s_total"]),
                                   "abs_diff_main": fin(dm), "abs_diff_total": fin(dt_),
                                   # a class without variance has no interval (NaN): equal values pass
                                   "within_fp64_ci_halfwidth": bool(np.all((dm <= half + 1e-15) | (dm == 0)) and
                                                                    np.all((dt_ <= halft + 1e-15) | (dt_ == 0))),
                                   "vdep_max_abs_diff": float(np.max(np.abs(ym - yf))),
                                   "gpu_ms": {"mixed": tm, "fp64": tf}}}
    print(json.dumps(out), flush=True)


def run_p3m(args):
    """Paper-scale single sample (FP64, 10 classes, lognormal charges) with P3M electrostatics,
    against the all-pairs FP64 step on the same state."""
    import torch
    import paper_2205_04979_gb300.pdq as pdq
    torch.cuda.set_device(0)
    w = workloads.WORKLOADS["paper_scale_fp64"]
    n = args.particles
    phys = pdq.phys_default()
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        field = pdq.Field(desc, w["field_seed"], stream)
        M, Nz = args.p3m_mesh or ((61, 128) if n <= 200_000 else (123, 256))
        plan = pdq.P3M(field, M=M, Nz=Nz, max_particles=n, stream=stream)
        prm = pdq.params_tensor([workloads.NOMINAL])

        def fresh():
            st = pdq.State(pdq.FP64, [n], w["st_plus"])
            pdq.seed_particles(field, phys, st, prm, w["particle_seed"], w["charge_sigma"], stream)
            return st

        state = fresh()
        cfg = pdq.step_cfg(w["dt"], window_start=0)
        tally = pdq.Tally(1, len(w["st_plus"]))
        ws = pdq.workspace(state, cfg)
        pdq.step_particles_p3m(field, phys, state, prm, cfg, args.warmup, tally, plan, ws, stream)
        stream.synchronize()
        alive0 = int(tally.n_alive.sum().item())
        clk = ClockSampler(None)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pdq.step_particles_p3m(field, phys, state, prm, cfg, args.steps, tally, plan, ws, stream)
        e1.record(stream)
        e1.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        assert pdq.check_state(state, stream) == 0
        psteps = int(tally.n_alive.sum().item()) - alive0
        # the all-pairs FP64 step (nearest image only) on the same initial state, 2 steps
        ref_ms = None
        if n <= 200_000:
            st2 = fresh()
            t2 = pdq.Tally(1, len(w["st_plus"]))
            ws2 = pdq.workspace(st2, cfg)
            pdq.step_particles(field, phys, st2, prm, cfg, 1, t2, ws2, stream)
            e0.record(stream)
            pdq.step_particles(field, phys, st2, prm, cfg, 2, t2, ws2, stream)
            e1.record(stream)
            e1.synchronize()
            ref_ms = e0.elapsed_time(e1) / 2
    out = {"metric": "particle-steps/s, P3M electrostatics (periodic pipe), FP64", "value": psteps / (ms / 1e3),
           "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "p3m: 1 sample x %d particles, 10 St+ classes, lognormal charges (sigma 0.5), "
                                  "128x64x128 field, dt+=%g; mesh M=%d across (h=%.2f), Nz=%d, transform "
                                  "%dx%dx%d, alpha=%.4f, r_cut=%.2f" % (n, w["dt"], M, 360.0 / M, Nz, plan.nx,
                                                                      plan.nx, Nz, plan.alpha, plan.r_cut)},
           "all_pairs_fp64_ms_per_step": ref_ms, "clocks": clocks,
           "gpu_launches": int(args.steps * 16)}
    print(json.dumps(out), flush=True)


# FP64 operations per (item, cell) of the low-fidelity march, as written in k_lf_vdep: momentum
# c = V^2/2 + dw + dPhi (7), root -2c/(a + sqrt(a^2 + 2c)) (7, sqrt and the division counted as
# one each), cell means and exponential fitting vm, a', expm1, G = em/vm, E (6), Q += P G, P *= E (3)
LF_FLOPS_PER_CELL = 23
# FP64-pipe lane instructions per (item, cell) as executed (ncu instruction counters on a launch of
# 16,384 samples x 10 classes: the square root, divisions and expm1 expand to seeds plus Newton or
# polynomial steps), and the DRAM bytes (read + write) of a 65,536-sample launch, scaled by samples
LF_FP64_OPS_PER_CELL = 61.41
LF_DRAM_BYTES_PER_SAMPLE = 2.172e6 / 65536
# the FP32 march: (what bounds it, thread instructions per (item, cell) as executed (ncu, same capture
# size), the measured rate it is compared with): every instruction takes an issue slot, and the issue
# limit of 4 warp instructions per clock per SM equals the measured scalar FFMA lane rate
LF_F32_PIPE = ("instruction issue", 56.48, "ffma")


def lf_cpu_baseline(w, params, seconds):
    """Time the numpy FP64 oracle of the 1-D Eulerian model on a bounded sample of the samples."""
    import oracle
    from oracle import lf_eulerian as lfo
    of = oracle.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    var = lfo.fluid_variance(oracle.field_grid(of, oracle.field_modes(of, w["field_seed"])))
    p = oracle.phys()
    n, done, t = 8, 0, 0.0
    while t < seconds and done < len(params):
        k = min(n, len(params) - done)
        t0 = time.perf_counter()
        lfo.lf_vdep(p, w["st_plus"], params[done:done + k], var, of.r_plus, of.beta, lfo.lf_params(n_y=w["n_y"]))
        t += time.perf_counter() - t0
        done += k
        n *= 2
    C = len(w["st_plus"])
    return {"value": done * C / t, "unit": "low-fidelity evaluations/s (sample x class)", "cores": 1,
            "kind": "oracle", "sample": "numpy FP64 oracle (vectorised over the items of a chunk, one thread), "
                                        "%d samples x %d classes in %.1f s" % (done, C, t)}


def run_lf(args):
    """The 1-D Eulerian low-fidelity model (App. B) at the Sobol' study's low-fidelity size.

    One bench step = one evaluation of V_dep+ for every (sample, class) item: 262,144 samples x 10
    St+ classes at 2,048 wall-normal nodes (pdq_lf_vdep, one kernel launch).  The headline is the
    PDQ_MIXED march (FP32, wall condition and ratio in FP64); the FP64 march is timed beside it and
    every item of the two is compared.  L2 is flushed between timed steps.  e2e: the inputs
    uploaded from pinned host memory and V_dep+ downloaded every step.
    """
    import torch
    import paper_2205_04979_gb300.pdq as pdq
    torch.cuda.set_device(0)
    w = workloads.WORKLOADS["lf_eulerian"]
    S = args.samples or w["samples"]
    params = workloads.sample_params(S, w["param_seed"], spread=w["spread"])
    st = w["st_plus"]
    C = len(st)
    phys = pdq.phys_default()
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    stream = torch.cuda.Stream()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    with torch.cuda.stream(stream):
        field = pdq.Field(desc, w["field_seed"], stream)
        var = pdq.lf_fluid_variance(field, stream)
        prm = pdq.params_tensor(params)
        out = torch.empty((S, C), dtype=torch.float64, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def timed(lfd):
            for _ in range(args.warmup):
                pdq.lf_vdep(field, phys, lfd, var, st, prm, out=out, stream=stream)
            stream.synchronize()
            clk = ClockSampler(uuid)
            clk.start()
            evs = []
            for k in range(args.steps):
                flush.fill_(k & 255)                    # evict L2 between timed evaluations
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pdq.lf_vdep(field, phys, lfd, var, st, prm, out=out, stream=stream)
                e1.record(stream)
                evs.append((e0, e1))
            stream.synchronize()
            clocks = clk.stop()
            return sum(a.elapsed_time(b) for a, b in evs), out.cpu().numpy(), clocks

        lfm = pdq.lf_desc(n_y=w["n_y"], precision=pdq.MIXED)
        lfd = pdq.lf_desc(n_y=w["n_y"], precision=pdq.FP64)
        ms, vd, clocks = timed(lfm)
        ms64, vd64, clocks64 = timed(lfd)
        # end to end: pinned host inputs in, V_dep+ out, every step
        host_in = torch.zeros((S, 4), dtype=torch.float64).pin_memory()
        host_in[:, :3] = torch.from_numpy(params)
        host_out = torch.empty((S, C), dtype=torch.float64).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            prm.copy_(host_in, non_blocking=True)
            pdq.lf_vdep(field, phys, lfm, var, st, prm, out=out, stream=stream)
            host_out.copy_(out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        ms_e2e = e0.elapsed_time(e1)
        assert np.array_equal(host_out.numpy(), vd)
    from paper_2205_04979_gb300 import peaks as pk
    rec = pk.load(PEAKS_FILE)
    k = rec["kernels"] if rec else None
    items = S * C
    cells = w["n_y"] - 1
    sec, sec64 = ms / args.steps / 1e3, ms64 / args.steps / 1e3
    rel = np.abs(vd / vd64 - 1)
    roof = {"bound": "alu", "kernel": "k_lf_vdep<float>", "unit": "TFLOP/s", "traffic": LF_DRAM_BYTES_PER_SAMPLE * S,
            "achieved": LF_FLOPS_PER_CELL * cells * items / sec / 1e12,
            "peak": k["ffma2"]["flops_per_s"] / 1e12 if k else None,
            "note": "%d operations per (item, cell) of the scheme, sqrt, expm1 and divisions counted as one each "
                    "(each expands to several FP32 instructions), against the measured FFMA2 peak; traffic "
                    "scaled from a 65,536-sample capture" % LF_FLOPS_PER_CELL}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
    if LF_F32_PIPE is not None and k:
        # the pipe that bounds the FP32 march, its instructions as executed against the measured rate
        name, per_cell, rate = LF_F32_PIPE
        got = per_cell * cells * items / sec
        roof["pipe"] = {"pipe": name, "lane_ops_per_cell": per_cell, "achieved_gops": got / 1e9,
                        "peak_gops": k[rate]["lane_ops_per_s"] / 1e9, "frac": got / k[rate]["lane_ops_per_s"]}
    out_json = {
        "metric": "low-fidelity evaluations/s (1-D Eulerian model of App. B, sample x class items)",
        "value": items * args.steps / (ms / 1e3), "unit": "evaluations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "lf_eulerian: %d samples x %d St+ classes (log-spaced 0.1..100), inputs xi in "
                               "[0, 0.1], zeta in [0, 1], theta in [0, 1], %d wall-normal nodes, v_f'^2 from the "
                               "128x64x128 field" % (S, C, w["n_y"]),
                   "l2": "flushed between timed steps (256 MiB write)", "precision": "PDQ_MIXED (FP32 march)"},
        "roofline": roof,
        "clocks": clocks, "gpu_launches": args.steps,
        "e2e": {"value": items * args.steps / (ms_e2e / 1e3), "unit": "evaluations/s",
                "h2d_bytes_per_step": int(S * 32), "d2h_bytes_per_step": int(S * C * 8)},
        "fp64": {"value": items * args.steps / (ms64 / 1e3), "ms_per_step": ms64 / args.steps, "clocks": clocks64,
                 "roofline": {"bound": "alu", "kernel": "k_lf_vdep<double>", "unit": "Gop/s",
                              "achieved": LF_FP64_OPS_PER_CELL * cells * items / sec64 / 1e9,
                              "peak": k["dfma"]["lane_ops_per_s"] / 1e9 if k else None,
                              "frac": (LF_FP64_OPS_PER_CELL * cells * items / sec64 / k["dfma"]["lane_ops_per_s"]
                                       if k else None),
                              "note": "%.2f FP64-pipe lane operations per (item, cell) as executed (ncu "
                                      "instruction counters), against the measured DFMA lane-operation rate"
                                      % LF_FP64_OPS_PER_CELL}},
        "mixed_vs_fp64": {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)), "items": int(items)},
        "us_per_sample_all_classes": ms / args.steps / S * 1e3,
        "vdep_mean": np.mean(vd64, 0).tolist(),
    }
    if not args.no_cpu_baseline:
        out_json["cpu_baseline"] = lf_cpu_baseline(w, params, min(args.cpu_seconds, 15.0))
    print(json.dumps(out_json), flush=True)


def clamp_check(pdq, stream, block, variant, samples, count, steps, st_plus, dt=0.05, t_window=10.0,
                param_seed=4242):
    """Does V_dep+ depend on the Coulomb distance clamp (reading c1: the largest class diameter for
    every pair)?  The batched MIXED step with the clamp at the largest class diameter and at the
    smallest (contact_scale = d_min / d_max), same particles (a stream per sample) and inputs;
    any pair-dependent contact distance lies between the two."""
    import torch
    w = workloads.WORKLOADS["batched_mixed"]
    params = workloads.sample_params(samples, param_seed)
    desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
    scale = float(np.sqrt(min(st_plus) / max(st_plus)))       # d+ grows as sqrt(St+)
    res = {}
    for name, sc in (("largest", 1.0), ("smallest", scale)):
        phys = pdq.phys_default()
        phys.contact_scale = sc
        with torch.cuda.stream(stream):
            field = pdq.Field(desc, w["field_seed"], stream)
            st = pdq.State(pdq.MIXED, [count] * samples, list(st_plus))
            prm = pdq.params_tensor(params)
            pdq.seed_particles_independent(field, phys, st, prm, w["particle_seed"], 0.0, stream)
            cfg = pdq.step_cfg(dt, window_start=workloads.window_start_step(t_window, dt), compact_every=100,
                               block=block, variant=variant)
            tally = pdq.Tally(samples, len(st_plus))
            pdq.step_particles(field, phys, st, prm, cfg, steps, tally, pdq.workspace(st, cfg), stream)
            vdep, _, _ = pdq.deposition_tally(tally, dt, stream=stream)
            stream.synchronize()
            res[name] = (vdep.cpu().numpy(), tally.n_dep.cpu().numpy())
            del st, tally
    va, na = res["largest"]
    vb, nb = res["smallest"]
    se = va.std(0, ddof=1) / np.sqrt(samples)
    diff = np.abs(vb.mean(0) - va.mean(0))
    return {"contact_scale": [1.0, scale], "deposits": [na.sum(0).tolist(), nb.sum(0).tolist()],
            "events_differing": np.abs(na - nb).sum(0).tolist(),
            "vdep_mean": [va.mean(0).tolist(), vb.mean(0).tolist()],
            "rel_diff": (diff / np.where(va.mean(0) > 0, va.mean(0), 1.0)).tolist(),
            "diff_over_se": (diff / np.where(se > 0, se, 1.0)).tolist()}


def run_vdep_validation(args):
    """The metric's validity condition at scale: V_dep+ of the batched MIXED path (autotuned
    launch configuration, or --block / --variant) against the FP64 GPU path, the latter pinned to the oracle by the
    parity tests, on --samples samples of 4,096 particles over 1,200 steps (t+ = 60, window
    from t+ = 10), with enough samples for >= 1,000 FP64 deposits in every class St+ >= 1."""
    import torch
    import paper_2205_04979_gb300.pdq as pdq
    S = args.samples or 1024
    classes = args.vdep_classes
    stream = torch.cuda.Stream()
    w = workloads.WORKLOADS["batched_mixed"]
    # the MIXED step's launch configuration: --block / --variant when given (e.g. the one the
    # batched workload autotunes to), else autotuned on this batch
    if args.block:
        cfg = pdq.step_cfg(w["dt"], window_start=0, compact_every=100, block=args.block, variant=args.variant)
    else:
        with torch.cuda.stream(stream):
            phys = pdq.phys_default()
            desc = pdq.field_desc(n_r=w["grid"][0], n_th=w["grid"][1], n_z=w["grid"][2], n_modes=w["n_modes"])
            field = pdq.Field(desc, w["field_seed"], stream)
            st = pdq.State(pdq.MIXED, [4096] * S, classes)
            prm = pdq.params_tensor(workloads.sample_params(S, 4242))
            pdq.seed_particles(field, phys, st, prm, w["particle_seed"], 0.0, stream)
            cfg = pdq.step_cfg(w["dt"], window_start=0, compact_every=100)
            pdq.autotune(field, phys, st, prm, cfg, stream)
            del st
    if args.clamp_check:
        res = clamp_check(pdq, stream, cfg.block, cfg.variant, S, 4096, args.vdep_steps, classes)
        print(json.dumps({"metric": "V_dep+ with the Coulomb clamp at the largest vs the smallest class diameter",
                          "workload": "%d samples x 4096 particles (a particle stream per sample), St+ classes %s, "
                                      "%d steps" % (S, classes, args.vdep_steps), "clamp_check": res}), flush=True)
        return
    res = vdep_check(pdq, stream, cfg.block, cfg.variant, samples=S, count=4096, steps=args.vdep_steps,
                     st_plus=classes)
    print(json.dumps({"metric": "V_dep+ of batched MIXED vs FP64 GPU (relative error, error / MC SE)",
                      "validation": res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "sobol":
        run_sobol(args)
    elif args.workload == "p3m":
        run_p3m(args)
    elif args.workload == "vdep_validation":
        run_vdep_validation(args)
    elif args.workload == "mfmc":
        run_mfmc(args)
    elif args.workload == "lf_eulerian":
        run_lf(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
