"""Batch dimension: several feeders of uneven size solved together, in one
cooperative launch (persistent engine) or in one while-node graph over all
instances (batched graph engine).  Each instance keeps its own chunks,
parameters, checks and stopping decision, so its result in the batch is
bit-identical to its result alone (same chunk layout) and matches the FP64
oracle."""
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


def rel(a, b):
    """Normwise relative difference (0 when both are exactly zero), and the
    largest element-wise ratio |a_i - b_i| / (|b_i| + ||b||_inf); the larger
    of the two is returned so that one bound checks both."""
    nb = float(np.linalg.norm(b))
    d = a - b
    if nb == 0.0:
        return 0.0 if not np.any(d) else float("inf")
    scale = np.abs(b) + float(np.max(np.abs(b)))
    return max(float(np.linalg.norm(d)) / nb, float(np.max(np.abs(d) / scale)))


def feeders_mix():
    return [F.feeder_13(1), F.feeder_123(1), F.feeder_tiny(6, 2), F.feeder_123(2), F.feeder_13(3),
            F.feeder_8500(1, n_bus=1500)]


@pytest.mark.parametrize("engine", ["auto", "graph"])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_alone(opf, prec, engine):
    eng = opf.ENGINE_AUTO if engine == "auto" else opf.ENGINE_GRAPH
    fs = feeders_mix()
    chunks = [1, 4, 1, 3, 2, 8]
    rhos = [100.0, 10.0, 10.0, 1000.0, 100.0, 10.0]
    params = [opf.default_params(rho=r, precision=prec, max_iter=3000 + 500 * i, check_every=50, engine=eng)
              for i, r in enumerate(rhos)]
    alone = []
    for f, c, prm in zip(fs, chunks, params):
        p = opf.Problem.from_feeder(f, chunks=c)
        info = p.solve(opf.default_params(rho=prm.rho, precision=prec, max_iter=prm.max_iter,
                                          check_every=50))   # alone, default engine
        alone.append((info, p.state()))
        p.close()
    probs = [opf.Problem.from_feeder(f, chunks=c) for f, c in zip(fs, chunks)]
    b = opf.Batch(probs)
    # a small batch: every chunk fits co-resident in shared memory
    assert b.auto_engine(prec) == opf.ENGINE_PERSISTENT
    infos = b.solve(params)
    for i, (p, info) in enumerate(zip(probs, infos)):
        ia, sa = alone[i]
        assert info.iters == ia.iters and info.status == ia.status, i
        sb = p.state()
        for x, y in zip(sb, sa):
            assert np.array_equal(x, y), (i, rel(x, y))
        assert info.pres == ia.pres and info.dres == ia.dres
    # a second batch solve, warm-started, continues every instance
    more = [opf.default_params(rho=r, precision=prec, max_iter=100, check_every=50, warm_start=1,
                               criterion=opf.CRIT_NEVER, engine=eng) for r in rhos]
    infos2 = b.solve(more)
    for i in range(len(fs)):
        assert infos2[i].iters == infos[i].iters + 100
    b.close()
    for p in probs:
        p.close()


def test_batch_fp64_matches_oracle(opf):
    from oracle import admm as OA, model as OM, precompute as OP
    fs = [F.feeder_13(2), F.feeder_123(3), F.feeder_tiny(5, 1)]
    probs = [opf.Problem.from_feeder(f, chunks=c) for f, c in zip(fs, [1, 5, 1])]
    b = opf.Batch(probs)
    infos = b.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=250, check_every=25))
    for f, p, info in zip(fs, probs, infos):
        m = OM.build_feeder(f)
        s = OA.ADMM(m, OP.precompute(m), 100.0)
        for _ in range(250):
            r = s.step()
        xg, xl, lam = p.state()
        assert rel(xg, s.x) <= 1e-9 and rel(xl, s.z) <= 1e-9 and rel(lam, s.lam) <= 1e-9
        assert abs(info.pres - r.pres) <= 1e-9 * r.pres
    b.close()


def test_batch_graph_engine_many_chunks(opf):
    """More chunks than fit co-resident: the persistent engine refuses, the
    graph engine runs, and each instance equals its graph-engine solve alone."""
    cap = opf.batch_capacity(opf.FP32)
    fs = [F.feeder_8500(s, n_bus=1500) for s in (1, 2, 3)]
    chunks = cap // 2 + 1
    prm = opf.default_params(rho=10.0, precision=opf.FP32, max_iter=600, check_every=50, engine=opf.ENGINE_GRAPH)
    alone = []
    for f in fs:
        p = opf.Problem.from_feeder(f, chunks=chunks)
        alone.append((p.solve(prm), p.state()))
        p.close()
    probs = [opf.Problem.from_feeder(f, chunks=chunks) for f in fs]
    b = opf.Batch(probs)
    with pytest.raises(RuntimeError):
        b.solve(opf.default_params(rho=10.0, precision=opf.FP32, max_iter=600, check_every=50,
                                   engine=opf.ENGINE_PERSISTENT))
    infos = b.solve(prm)
    for i, p in enumerate(probs):
        ia, sa = alone[i]
        assert infos[i].iters == ia.iters and infos[i].status == ia.status
        for x, y in zip(p.state(), sa):
            assert np.array_equal(x, y), (i, rel(x, y))
    b.close()
    for p in probs:
        p.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_graph_partial_last_round(opf, prec):
    """Iteration budgets that are not multiples of the check interval: each
    instance's last round ends with a check before the body's last offset,
    so its check iteration runs on the chunk kernel inside the tile-parallel
    launch (check role) while the other instances take plain iterations.
    Every instance still equals its solve alone bit for bit."""
    fs = feeders_mix()
    chunks = [1, 4, 1, 3, 2, 8]
    budgets = [137, 263, 50, 411, 99, 321]
    params = [opf.default_params(rho=10.0, precision=prec, max_iter=m, check_every=50, criterion=opf.CRIT_NEVER,
                                 engine=opf.ENGINE_GRAPH) for m in budgets]
    alone = []
    for f, c, prm in zip(fs, chunks, params):
        p = opf.Problem.from_feeder(f, chunks=c)
        info = p.solve(opf.default_params(rho=10.0, precision=prec, max_iter=prm.max_iter, check_every=50,
                                          criterion=opf.CRIT_NEVER))
        alone.append((info, p.state()))
        p.close()
    probs = [opf.Problem.from_feeder(f, chunks=c) for f, c in zip(fs, chunks)]
    b = opf.Batch(probs)
    infos = b.solve(params)
    for i, (p, info) in enumerate(zip(probs, infos)):
        ia, sa = alone[i]
        assert info.iters == ia.iters == budgets[i], i
        for x, y in zip(p.state(), sa):
            assert np.array_equal(x, y), (i, rel(x, y))
        assert info.pres == ia.pres and info.dres == ia.dres, i
    b.close()
    for p in probs:
        p.close()


def test_batch_profile_kernels_restores_state(opf):
    """The kernel-timing hook of the batched graph engine leaves every
    instance's iterate, duals and global vector as they were, and a solve
    afterwards continues as if it had not run."""
    fs = feeders_mix()[:4]
    probs = [opf.Problem.from_feeder(f, chunks=c) for f, c in zip(fs, [1, 4, 1, 3])]
    b = opf.Batch(probs)
    prm = opf.default_params(rho=10.0, precision=opf.FP32, max_iter=120, check_every=50, criterion=opf.CRIT_NEVER,
                             engine=opf.ENGINE_GRAPH)
    b.solve(prm)
    before = [p.state() for p in probs]
    us = b.profile_kernels(prm, reps=3)
    assert all(v > 0 for v in us.values()), us
    for p, sa in zip(probs, before):
        for x, y in zip(p.state(), sa):
            assert np.array_equal(x, y)
    b.close()
    for p in probs:
        p.close()
