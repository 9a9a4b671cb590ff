"""Failure detection on the device without any GPU fault.

A non-finite value is planted on the host through the C ABI
(opf_set_state); the residual check of Eq. (termination) sees NaN and the
solve stops with OPF_ERR_NUMERIC instead of iterating on garbage.  The
context stays usable: a cold solve afterwards matches the oracle.  (The
bounded-wait timeout path is covered in test_gpu_parity.py.)
"""
import numpy as np
import pytest

from paper_2501_08293_b300 import feeders as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08293_b300 import build
    build.build()
    from paper_2501_08293_b300 import opf as mod
    return mod


@pytest.mark.parametrize("engine", ["graph", "hostloop", "persistent"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("where", ["lam", "x_local"])
def test_nan_state_stops_with_numeric_status(opf, engine, prec, where):
    from oracle import admm as OA, model as OM, precompute as OP
    eng = {"graph": opf.ENGINE_GRAPH, "hostloop": opf.ENGINE_HOSTLOOP, "persistent": opf.ENGINE_PERSISTENT}[engine]
    pc = opf.FP64 if prec == "fp64" else opf.FP32
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f)
    p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=60, check_every=20, precision=pc, engine=eng))
    xg, xl, lam = p.state()
    j = len(xl) // 3
    if where == "lam":
        lam[j] = np.nan       # a NaN dual stays NaN and reaches the residual sums
    else:
        xl[j] = np.inf        # x_prev of the first iteration: dres is not finite
    p.set_state(xl, lam)
    # the check runs on the first iteration after the warm start
    with pytest.raises(opf.OpfError) as ei:
        p.solve(opf.default_params(max_iter=5000, check_every=1, warm_start=1, precision=pc, engine=eng))
    assert ei.value.status == -3, ei.value
    # the same handle and context solve normally from a cold start
    info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=50, check_every=50, precision=pc,
                                      engine=eng))
    assert info.status == opf.OK and np.isfinite(info.pres) and np.isfinite(info.objective)
    m = OM.build_feeder(f)
    s = OA.ADMM(m, OP.precompute(m), 100.0)
    for _ in range(50):
        r = s.step()
    xg2, _, _ = p.state()
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.linalg.norm(xg2 - s.x) <= tol * np.linalg.norm(s.x)
    assert abs(info.pres - r.pres) <= (1e-9 if prec == "fp64" else 1e-3) * r.pres
    p.close()
