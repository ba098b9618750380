"""Measured roofline denominators of the particle kernels on the GPU at hand.

Runs the microbenchmarks of csrc_peaks/pdq_peaks.cu (FP32 FMA scalar and packed f32x2, packed
FP32 add, FP64 FMA, MUFU rsqrt, L2 reads) with nvidia-smi clock samples taken during the runs,
and reports each rate both as measured and per SM per clock, so that a rate can be restated at
another clock.  `python -m paper_2205_04979_gb300.peaks --write FILE` also writes a markdown
summary whose ```json block the benchmark reads.  It changes no GPU setting.
"""
import argparse
import ctypes as C
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))

# kind: (name, unit of one counted operation, flops (or bytes) per counted operation per lane)
KINDS = {
    0: ("ffma", "FP32 FMA, scalar", 2),
    1: ("ffma2", "FP32 FMA, packed f32x2 (one instruction = 2 FMAs per lane)", 4),
    2: ("fadd2", "FP32 add, packed f32x2 (one instruction = 2 adds per lane)", 2),
    3: ("dfma", "FP64 FMA", 2),
    4: ("rsqrt", "MUFU rsqrt.approx.ftz.f32", 1),
}


def _lib():
    from . import build
    path = build.build_peaks()
    L = C.CDLL(path)
    L.pk_time.restype = C.c_int
    L.pk_time.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_float)]
    L.pk_ops_per_iter.restype = C.c_int
    return L


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def measure(reps=5):
    """Best-of-reps rates of every kernel, with the clocks sampled meanwhile."""
    import torch
    from .clocks import ClockSampler
    torch.cuda.init()
    L = _lib()
    sms = _sm_count()
    ops_iter = L.pk_ops_per_iter()
    threads, blocks = 256, sms * 8
    out = {"gpu": torch.cuda.get_device_name(0), "sms": sms, "threads": threads, "blocks": blocks, "kernels": {}}
    clk = ClockSampler(None)
    clk.start()
    time.sleep(0.5)
    t0 = time.time()
    # about 50 ms per launch (first GB300 measurement: FP32 ~120, packed ~62, FP64 ~1.7, MUFU ~15.5
    # instructions per lane per clock per SM), long enough for the clock samples to see the load
    iters = {0: 192 * 1024, 1: 96 * 1024, 2: 96 * 1024, 3: 2560, 4: 24 * 1024}
    for kind, (name, what, per) in KINDS.items():
        best = None
        for _ in range(reps):
            ms = C.c_float()
            rc = L.pk_time(kind, blocks, threads, iters[kind], 0, C.byref(ms))
            if rc != 0:
                raise RuntimeError("pk_time(%s) failed with CUDA error %d" % (name, rc))
            best = ms.value if best is None else min(best, ms.value)
        ops = float(blocks) * threads * iters[kind] * ops_iter          # lane-operations
        out["kernels"][name] = {"what": what, "ms": best, "lane_ops_per_s": ops / (best * 1e-3),
                                "flops_per_s": ops * per / (best * 1e-3) if kind != 4 else None}
    # L2: 48 MB read 6,400 times (~20 ms) by one wave of 8 CTAs of 256 threads per SM
    l2_bytes, passes = 48 << 20, 6400
    best = None
    for _ in range(reps):
        ms = C.c_float()
        rc = L.pk_time(5, blocks, threads, passes, l2_bytes, C.byref(ms))
        if rc != 0:
            raise RuntimeError("pk_time(l2) failed with CUDA error %d" % rc)
        best = ms.value if best is None else min(best, ms.value)
    out["kernels"]["l2_read"] = {"what": "L2 reads, 48 MB buffer (L2-resident), float4 __ldcg", "ms": best,
                                 "bytes_per_s": float(l2_bytes) * passes / (best * 1e-3)}
    out["seconds"] = time.time() - t0
    out["clocks"] = clk.stop()
    f = out["clocks"].get("sm_mhz") or 0.0
    for k in out["kernels"].values():
        rate = k.get("lane_ops_per_s") or k.get("bytes_per_s")
        k["per_sm_per_clock"] = rate / (sms * f * 1e6) if f else None
    return out


def summary_md(res, cmd):
    f = res["clocks"].get("sm_mhz")
    fmax = res["clocks"].get("sm_max_mhz")
    rows = []
    for name, k in res["kernels"].items():
        if name == "l2_read":
            rows.append("| %s | %s | %.1f GB/s | %.1f B/clk/SM |" % (name, k["what"], k["bytes_per_s"] / 1e9,
                                                                   k["per_sm_per_clock"] or float("nan")))
        else:
            fl = k["flops_per_s"]
            rows.append("| %s | %s | %s | %.1f lane-ops/clk/SM |" % (
                name, k["what"], ("%.2f TFLOP/s" % (fl / 1e12)) if fl else
                ("%.2f Tops/s" % (k["lane_ops_per_s"] / 1e12)), k["per_sm_per_clock"] or float("nan")))
    return "\n".join([
        "# Measured peaks: FP32 / FP64 / MUFU pipes and L2 reads (%s)" % res["gpu"],
        "",
        "Command: `%s`" % cmd,
        "",
        "Microbenchmarks `csrc_peaks/pdq_peaks.cu`: %d CTAs x %d threads (8 per SM), 8 independent chains "
        "per thread, best of 5 launches timed with CUDA events. SM clock median %s MHz during the runs "
        "(max %s), throttle reasons %s. Per-clock rates divide by %d SMs and that median clock." % (
            res["blocks"], res["threads"], f, fmax, res["clocks"].get("reasons"), res["sms"]),
        "",
        "| kernel | operation | measured | per SM per clock |",
        "|---|---|---|---|",
    ] + rows + ["", "```json", json.dumps(res, indent=1, sort_keys=True), "```", ""])


def load(path):
    """The measured record from a summary file (its ```json block), or None."""
    try:
        txt = open(path).read()
        a = txt.index("```json") + len("```json")
        b = txt.index("```", a)
        return json.loads(txt[a:b])
    except Exception:
        return None


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--write", default=None, help="markdown summary to write")
    args = ap.parse_args(argv)
    res = measure()
    print(json.dumps(res))
    if args.write:
        cmd = "python -m paper_2205_04979_gb300.peaks --write %s" % args.write
        open(args.write, "w").write(summary_md(res, cmd))
    return 0


if __name__ == "__main__":
    sys.exit(main())
