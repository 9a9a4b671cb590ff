"""The benchmark's contract on a machine without a GPU.

* The reference arm (the FP64 CPU oracle, timed on a bounded sample of the
  8500-class workload) prints one JSON line with the keys the harness reads.
* The product path has no CPU fallback: without a CUDA device the solver and
  the default benchmark fail loudly instead of quietly computing on the host.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_available():
    import torch
    return torch.cuda.is_available()


def _run_bench(args, timeout):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["unit"] == "iters/s" and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(_cuda_available(), reason="a CUDA device is present: the product path runs there")
def test_no_cpu_fallback_without_a_gpu():
    from paper_2501_08293_b300 import feeders as F
    from paper_2501_08293_b300 import opf
    with pytest.raises(Exception, match="CUDA"):
        opf.Problem.from_feeder(F.feeder_13(1))
    r = _run_bench(["--steps", "1", "--warmup", "0", "--no-cpu-baseline", "--no-serve"], timeout=600)
    assert r.returncode != 0
    assert not any(ln.strip().startswith("{") for ln in r.stdout.splitlines())


def test_batch_kernel_bytes_split_the_iteration_formula():
    """The per-kernel byte counts of the batched graph engine add up to the
    per-iteration formula the batch line's roofline uses (host-only
    problems, no device needed)."""
    import importlib.util
    from paper_2501_08293_b300 import feeders as F
    from paper_2501_08293_b300 import opf
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    probs = [opf.Problem.from_feeder(f, upload=False) for f in (F.feeder_13(1), F.feeder_123(2), F.feeder_tiny(5, 1))]
    try:
        for w in (4, 8):
            kb = bench.batch_kernel_bytes(probs, w)
            total = sum(w * (7 * p.dims.n_local + 6 * p.dims.n_global) + w * p.dims.sum_n2
                        + 4 * (2 * p.dims.n_local + p.dims.n_global) for p in probs)
            assert kb["z"] + kb["x"] == total
            assert kb["z"] > 0 and kb["x"] > kb["z"]
    finally:
        for p in probs:
            p.close()
