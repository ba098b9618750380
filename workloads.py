"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle runs.

This module only draws the random inputs that the method takes from outside
(the uncertain parameters of each Monte Carlo sample and the per-sample
particle counts) and lists the sizes of each workload.  It holds none of the
method's arithmetic: the field, the particle seeds and every force are
computed on each side (CUDA library, oracle) from these inputs.

Workloads (paper Sec. 2.1 fixes Re_tau = 180 and the St+ classes; the uncertain
inputs are charge scale xi in [0, 0.1], Hamaker ratio zeta in [0, 1] and
temperature theta in [0, 1], Secs. 2.1 and 4.3):

* ``single_fp64``: 1 sample, 1,000 particles of St+ = 10, 64x32x64 grid,
  500 steps at dt+ = 0.1, nominal inputs.
* ``paper_scale_fp64``: 1 sample, 100,000 particles in 10 St+ classes
  log-spaced 0.1..100, lognormal(0.5) charge factor, 128x64x128 grid,
  20,000 steps at dt+ = 0.05.
* ``batched_mixed``: 1,024 samples, inputs uniform over +-50 % of nominal,
  counts uniform in 4,096..32,768, 5 St+ classes, 10,000 steps at dt+ = 0.05.
* ``adjoint``: 256 samples x 16,384 particles, 2,000 steps, checkpoints every 100.
* ``lf_eulerian``: the low-fidelity side of the MFMC Sobol' study, the 1-D
  Eulerian model of App. B on 262,144 samples x 10 St+ classes (log-spaced
  0.1..100), inputs uniform over the paper's ranges, the 128x64x128 field.
"""
import numpy as np

NOMINAL = (0.05, 0.5, 0.5)          # range midpoints of xi, zeta, theta


def st_plus_log(n, lo=0.1, hi=100.0):
    return list(np.geomspace(lo, hi, n))


WORKLOADS = {
    "single_fp64": dict(samples=1, count=1000, st_plus=[10.0], grid=(64, 32, 64), n_modes=64,
                        field_seed=0, particle_seed=1, dt=0.1, steps=500, t_window=10.0,
                        charge_sigma=0.0, precision="fp64"),
    "paper_scale_fp64": dict(samples=1, count=100_000, st_plus=st_plus_log(10), grid=(128, 64, 128),
                             n_modes=64, field_seed=0, particle_seed=1, dt=0.05, steps=20_000,
                             t_window=10.0, charge_sigma=0.5, precision="fp64"),
    "batched_mixed": dict(samples=1024, count=(4096, 32768), st_plus=[0.1, 0.316, 1.0, 3.16, 10.0],
                          grid=(128, 64, 128), n_modes=64, field_seed=0, particle_seed=1, param_seed=2,
                          dt=0.05, steps=10_000, t_window=10.0, charge_sigma=0.0, compact_every=100,
                          precision="mixed"),
    "adjoint": dict(samples=256, count=16384, st_plus=[0.1, 1.0, 10.0], grid=(64, 32, 64), n_modes=64,
                    field_seed=0, particle_seed=1, param_seed=3, dt=0.05, steps=2000, checkpoint=100,
                    t_window=10.0, eps=(0.5, 0.1, 0.02), precision="mixed"),
    "lf_eulerian": dict(samples=262144, st_plus=st_plus_log(10), grid=(128, 64, 128), n_modes=64, field_seed=0,
                        param_seed=5, spread=1.0, n_y=2048, precision="fp64"),
}


def sample_params(n, seed, spread=0.5, nominal=NOMINAL):
    """[n, 3] inputs (xi, zeta, theta) uniform over nominal * (1 +- spread)."""
    rng = np.random.Generator(np.random.Philox(seed))
    lo = np.asarray(nominal) * (1 - spread)
    hi = np.asarray(nominal) * (1 + spread)
    return lo + (hi - lo) * rng.random((n, 3))


def sample_counts(n, lo, hi, seed):
    """Per-sample particle counts uniform in lo..hi inclusive."""
    rng = np.random.Generator(np.random.Philox(seed + 1000))
    return rng.integers(lo, hi + 1, size=n).astype(np.int64)


def workload_inputs(name, samples=None):
    """(params [S,3], counts [S]) of a named workload, optionally truncated to ``samples``."""
    w = WORKLOADS[name]
    S = w["samples"] if samples is None else samples
    if w["samples"] == 1:
        params = np.array([NOMINAL], np.float64)
    else:
        params = sample_params(w["samples"], w["param_seed"])[:S]
    if isinstance(w["count"], tuple):
        counts = sample_counts(w["samples"], w["count"][0], w["count"][1], w["param_seed"])[:S]
    else:
        counts = np.full(S, w["count"], np.int64)
    return params, counts


def window_start_step(t_window, dt):
    """First step index inside the tally window t+ >= t_window."""
    return int(np.ceil(t_window / dt - 1e-9))
