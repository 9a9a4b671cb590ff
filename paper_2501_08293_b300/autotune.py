"""Autotuner of the automatic chunking (CTAs of the local update and of the
persistent kernels).

A problem is cut into chunks of about `work_per_chunk` units of
n_s^2 + 4 n_s + 16; one CTA runs one chunk.  Few large chunks exchange less
between neighbours, many small ones spread the arithmetic over more SMs; the
best size depends on the GPU and the feeder's size.  For each size bucket a
synthetic feeder of that size is built with every candidate chunk size and
its persistent solve is timed on the device (CUDA events on the solve
stream, a fixed iteration count after a warm-up solve, the same parameters
for every candidate).  Iterates do not depend on the chunking (every
engine computes the same arithmetic per component), so time per iteration
is the figure of merit.  The winners go to a JSON file keyed by the GPU's
name and the bucket; the library reads it with opf_tuning_load and
opf_problem_create with chunks = 0 then uses it.

    python -m paper_2501_08293_b300.autotune [--out FILE] [--iters N] [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import feeders as F

# (lower bus count, upper bus count, representative size); the last bucket's
# feeder is the 8500-class configuration (11,932 buses)
BUCKETS = [(1, 60, 30), (60, 200, 120), (200, 700, 400), (700, 2500, 1300), (2500, 7000, 4000), (7000, 1 << 30, 11932)]
CANDIDATES = (256, 512, 1024, 2048, 4096, 8192, 16384)
DEFAULT_WORK, DEFAULT_CAP = 4096, 296
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def representative(n_bus: int, seed: int = 1):
    """Synthetic feeder of about n_bus buses shaped like the configurations
    (12.47 kV, ~1 load per 8 buses, lognormal loads, a PV per 60 buses)."""
    if n_bus >= 11932:
        return F.feeder_8500(seed)
    return F.make_feeder(n_bus, seed, n_loads=max(1, n_bus // 8), load_sampler=lambda r: r.lognormal(-4.0, 1.0),
                         n_pv=max(1, n_bus // 60), n_switches=4, line_mix=(0.6, 0.15, 0.25), v_ll_kv=12.47,
                         lateral_mean=5.0)


def work_total(prob) -> int:
    ns = np.diff(prob.structure()["comp_ptr"]).astype(np.int64)
    return int(np.sum(ns * ns + 4 * ns + 16))


def chunks_for(total: int, work: int, cap: int, n_comp: int) -> int:
    """The packer's rule for automatic chunking."""
    return max(1, min(cap, max(1, total // work), n_comp))


def time_per_iter(opf, feeder, chunks: int, params, iters: int, reps: int = 3) -> float:
    """Microseconds per iteration of the persistent solve (median of reps)."""
    import torch
    p = opf.Problem.from_feeder(feeder, chunks=chunks)
    try:
        if not p.persistent_ok(params):
            return float("inf")             # does not fit co-resident: the graph engine would run
        p.solve(params)                     # warm-up (module load, first touch)
        stream = torch.cuda.current_stream()
        out = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = p.solve(params)
            e1.record(stream)
            e1.synchronize()
            out.append(1e3 * e0.elapsed_time(e1) / max(1, info.iters))
        return float(np.median(out))
    finally:
        p.close()


def tune(buckets=BUCKETS, candidates=CANDIDATES, iters: int = 3000, precision=None, rho: float = 10.0,
         seed: int = 1, cap: int = DEFAULT_CAP, log=print) -> dict:
    import torch
    from . import opf
    if not torch.cuda.is_available():
        raise RuntimeError("the tuner times kernels: it needs a CUDA device")
    prec = opf.FP32 if precision is None else precision
    params = opf.default_params(rho=rho, precision=prec, criterion=opf.CRIT_NEVER, max_iter=iters, check_every=50,
                                engine=opf.ENGINE_PERSISTENT)
    gpu = torch.cuda.get_device_name()
    entries = []
    t0 = time.perf_counter()
    for lo, hi, size in buckets:
        f = representative(size, seed)
        probe = opf.Problem.from_feeder(f, upload=False)
        total, ncomp = work_total(probe), probe.dims.n_comp
        probe.close()
        # candidate -> chunk count (several candidates may give the same count)
        tried = {w: chunks_for(total, w, cap, ncomp) for w in sorted(set(candidates) | {DEFAULT_WORK})}
        times = {}
        for work, ch in tried.items():
            if ch not in times:
                times[ch] = time_per_iter(opf, f, ch, params, iters)
        best_work = min(tried, key=lambda w: (times[tried[w]], -w))
        e = {"n_bus_lo": lo, "n_bus_hi": hi, "work_per_chunk": int(best_work), "max_chunks": int(cap),
             "representative_n_bus": int(f.n_bus), "chunks": int(tried[best_work]),
             "us_per_iter": times[tried[best_work]],
             "default_chunks": int(tried[DEFAULT_WORK]), "default_us_per_iter": times[tried[DEFAULT_WORK]],
             "candidates": {str(w): {"chunks": int(c), "us_per_iter": times[c]} for w, c in sorted(tried.items())}}
        entries.append(e)
        log(f"bucket [{lo}, {hi}) n_bus {f.n_bus}: best {best_work} units/chunk ({e['chunks']} chunks, "
            f"{e['us_per_iter']:.2f} us/it) vs default {e['default_chunks']} chunks "
            f"{e['default_us_per_iter']:.2f} us/it")
    return {"gpu": gpu, "precision": "fp32" if prec == opf.FP32 else "fp64", "rho": rho, "iters": iters,
            "seconds": time.perf_counter() - t0, "entries": entries}


def save(table: dict, path: str = DEFAULT_PATH) -> None:
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--quick", action="store_true", help="three buckets and four candidates")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    buckets = BUCKETS[::2] if a.quick else BUCKETS
    cands = (512, 2048, 4096, 8192) if a.quick else CANDIDATES
    table = tune(buckets, cands, iters=a.iters)
    save(table, a.out)
    print(json.dumps({k: v for k, v in table.items() if k != "entries"}), flush=True)


if __name__ == "__main__":
    main()
