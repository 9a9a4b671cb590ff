"""Serving: continuous batching of OPF requests (opf_server_*).

Requests arrive while others are being iterated; they are admitted as slots,
memory and co-resident capacity free up, and every round iterates all active
instances in one launch.  Each request's result is the same alone and in
the mix: served, it stops at the same iteration with bit-identical iterates
as when solved alone with the same parameters and chunking."""
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


def chunks_for(f):
    return max(1, min(64, f.n_bus // 50))      # the server's default chunking


def drain(srv, want, max_steps=100000):
    done = {}
    for _ in range(max_steps):
        srv.step()
        for rid, info in srv.poll():
            done[rid] = info
        if len(done) >= want:
            return done
    raise AssertionError("server did not finish")


@pytest.mark.parametrize("prec", [1, 0])
def test_served_result_equals_alone(opf, prec):
    fs = [F.feeder_13(1), F.feeder_123(1), F.feeder_tiny(6, 3), F.feeder_123(4), F.feeder_8500(2, n_bus=900),
          F.feeder_13(5), F.feeder_tiny(4, 7)]
    cfg = dict(precision=prec, rho=10.0, max_iter=60000, check_every=50, round_iters=500)
    srv = opf.Server(**cfg)
    ids = []
    # staggered arrivals: some while others are already on the device
    ids += [srv.submit(f) for f in fs[:3]]
    srv.step()
    ids += [srv.submit(f) for f in fs[3:5]]
    srv.step()
    srv.step()
    ids += [srv.submit(f) for f in fs[5:]]
    done = drain(srv, len(fs))
    for f, rid in zip(fs, ids):
        info = done[rid]
        p = opf.Problem.from_feeder(f, chunks=chunks_for(f))
        alone = p.solve(opf.default_params(precision=prec, rho=10.0, max_iter=60000, check_every=50))
        assert info.iters == alone.iters and info.status == alone.status, (f.name, info.iters, alone.iters)
        assert info.pres == alone.pres and info.dres == alone.dres
        sp = srv.problem(rid)
        for x, y in zip(sp.state(), p.state()):
            assert np.array_equal(x, y)
        p.close()
    st = srv.stats()
    assert st["completed"] == len(fs) and st["rounds"] > 1
    srv.close()


def test_warm_start_after_topology_switch(opf):
    """A switch flip of a resident feeder warm-starts from its last iterate
    on the device and reaches the cold-start optimum: both run to a tight
    residual (FP64, 1e-7) so their objectives agree to 1e-4 relative (at a
    1e-4 residual the ADMM objective itself is only within ~1e-3)."""
    f = F.feeder_123(1)
    g = F.reconfigure(f, np.random.default_rng(3))
    assert (f.lines["in_service"] != g.lines["in_service"]).sum() == 2
    tight = dict(precision=0, rho=10.0, max_iter=400000, check_every=50, eps_abs_prim=1e-7, eps_abs_dual=1e-7)
    srv = opf.Server(round_iters=1000, **tight)
    a = srv.submit(f)
    first = drain(srv, 1)[a]
    assert first.status == opf.OK
    b = srv.submit(g, warm_from=a)
    warm = drain(srv, 1)[b]
    p = opf.Problem.from_feeder(g)
    cold = p.solve(opf.default_params(**tight))
    assert warm.status == opf.OK and cold.status == opf.OK
    assert abs(warm.objective - cold.objective) <= 1e-4 * abs(cold.objective)
    assert srv.stats()["warm_started"] == 1
    p.close()
    srv.close()


def test_admission_by_memory(opf):
    """With a budget for only a few instances, requests wait in the queue,
    finished residents are evicted, and every request completes."""
    fs = [F.feeder_13(s) for s in range(1, 9)]
    p0 = opf.Problem.from_feeder(fs[0], upload=False)
    budget = int(p0.dims.device_bytes * 2.5)
    srv = opf.Server(device_budget_bytes=budget, precision=1, rho=10.0, max_iter=50000, check_every=50,
                     round_iters=500)
    ids = [srv.submit(f) for f in fs]
    na, npend = srv.step()
    assert na <= 2 and npend >= 6
    done = drain(srv, len(fs))
    assert set(done) == set(ids)
    st = srv.stats()
    assert st["evicted"] >= 5 and st["resident_bytes"] <= budget
    srv.close()


def test_warm_start_source_evicted_when_budget_holds_one(opf):
    """A warm-start request whose source feeder and itself do not fit the
    memory budget together, with nothing else active: the source is evicted
    and the request runs cold to convergence instead of waiting for memory
    that nothing would free."""
    f = F.feeder_123(1)
    g = F.reconfigure(f, np.random.default_rng(3))
    nch = chunks_for(f)
    bf = opf.Problem.from_feeder(f, chunks=nch, upload=False).dims.device_bytes
    bg = opf.Problem.from_feeder(g, chunks=nch, upload=False).dims.device_bytes
    budget = max(bf, bg) + min(bf, bg) // 2
    srv = opf.Server(device_budget_bytes=budget, precision=1, rho=10.0, max_iter=200000, check_every=50,
                     round_iters=500)
    a = srv.submit(f, chunks=nch)
    assert drain(srv, 1)[a].status == opf.OK
    b = srv.submit(g, warm_from=a, chunks=nch)
    info = drain(srv, 1, max_steps=2000)[b]
    alone = opf.Problem.from_feeder(g, chunks=nch)
    ref = alone.solve(opf.default_params(precision=1, rho=10.0, max_iter=200000, check_every=50))
    st = srv.stats()
    assert info.status == opf.OK and info.iters == ref.iters
    assert st["warm_started"] == 0 and st["evicted"] >= 1 and st["resident_bytes"] <= budget
    alone.close()
    srv.close()


def test_served_fp64_matches_oracle(opf):
    """Requests served in a mix (FP64, rho = 100, residuals checked every 50
    iterations) stop where the FP64 oracle stops with the same check
    interval, at the oracle's iterate (element-wise, 1e-9), and report its
    objective.  Ties the server to the paper's Algorithm 1 directly, not only
    through the solve alone."""
    from oracle import admm as OA, model as OM, precompute as OP

    def rel(a, b):
        nb = float(np.linalg.norm(b))
        d = a - b
        scale = np.abs(b) + float(np.max(np.abs(b)))
        return max(float(np.linalg.norm(d)) / nb, float(np.max(np.abs(d) / scale)))

    fs = [F.feeder_13(1), F.feeder_123(2), F.feeder_tiny(5, 1)]
    srv = opf.Server(precision=0, rho=100.0, max_iter=200000, check_every=50, round_iters=500)
    ids = [srv.submit(fs[0]), srv.submit(fs[1])]
    srv.step()
    ids.append(srv.submit(fs[2]))
    done = drain(srv, len(fs))
    for k in (0, 2):
        f, info = fs[k], done[ids[k]]
        m = OM.build_feeder(f)
        s = OA.ADMM(m, OP.precompute(m), 100.0)
        o = s.run(200000, criterion=OA.CRIT_ABS, check_every=50)
        assert info.status == opf.OK and info.iters == o["iters"], (k, info.iters, o["iters"])
        xg, xl, lam = srv.problem(ids[k]).state()
        assert rel(xg, s.x) <= 1e-9 and rel(xl, s.z) <= 1e-9, k
        assert abs(info.objective - o["objective"]) <= 1e-9 * abs(o["objective"])
    srv.close()
