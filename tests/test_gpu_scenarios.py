"""Multi-scenario engine: S load draws on one topology iterated together.
Each scenario's iterates must equal a single-instance FP32 solve of that
scenario (same arithmetic); its residuals agree to the rounding of their
sums, converged scenarios reach the same check, and the FP32 objective is
within 1e-4 of the FP64 path's at the same iteration."""
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


def alone(opf, f, loads_k, prm):
    g = f.copy()
    g.loads = loads_k.copy()
    p = opf.Problem.from_feeder(g)
    info = p.solve(prm)
    st = p.state()
    p.close()
    return info, st


@pytest.mark.parametrize("S, picks", [(8, range(8)), (70, (0, 1, 63, 64, 69))])
def test_scenarios_equal_alone_fixed_iterations(opf, S, picks):
    f = F.feeder_123(1)
    loads = F.load_scenarios(f, S, seed=7)
    sc = opf.Scenarios.from_feeder(f, loads)
    prm = opf.default_params(precision=opf.FP32, rho=10.0, criterion=opf.CRIT_NEVER, max_iter=300, check_every=50)
    infos = sc.solve(prm)
    for k in picks:
        ia, sa = alone(opf, f, loads[k], opf.default_params(precision=opf.FP32, rho=10.0, criterion=opf.CRIT_NEVER,
                                                             max_iter=300, check_every=50))
        assert infos[k].iters == ia.iters == 300
        sb = sc.state(k)
        for x, y in zip(sb, sa):
            assert np.array_equal(x, y), k
        # residual sums: FP32 within a component, FP64 across (single instance:
        # FP64 throughout), different order
        assert abs(infos[k].pres - ia.pres) <= 1e-5 * ia.pres
        assert abs(infos[k].dres - ia.dres) <= 1e-5 * ia.dres
        assert abs(infos[k].objective - ia.objective) <= 1e-12 * abs(ia.objective)
    # a second solve continues from the state (warm start)
    prm.warm_start = 1
    prm.max_iter = 50
    infos2 = sc.solve(prm)
    assert all(i.iters == 350 for i in infos2)
    sc.close()


def test_scenarios_short_last_body(opf):
    """A sweep body with fewer than K iterations left runs them at its last
    positions, so its check is still the last one: 130 = 2 x 50 + 30
    iterations, then one warm iteration (a one-iteration body whose previous
    x comes from the last check), each equal to solving alone."""
    f = F.feeder_123(1)
    S = 4
    loads = F.load_scenarios(f, S, seed=5)
    sc = opf.Scenarios.from_feeder(f, loads)
    for warm, iters, total in ((0, 130, 130), (1, 1, 131)):
        prm = opf.default_params(precision=opf.FP32, rho=10.0, criterion=opf.CRIT_NEVER, max_iter=iters,
                                 check_every=50)
        prm.warm_start = warm
        infos = sc.solve(prm)
        for k in range(S):
            ia, sa = alone(opf, f, loads[k], opf.default_params(precision=opf.FP32, rho=10.0,
                                                                 criterion=opf.CRIT_NEVER, max_iter=total,
                                                                 check_every=50))
            assert infos[k].iters == ia.iters == total
            for x, y in zip(sc.state(k), sa):
                assert np.array_equal(x, y), (k, total)
            assert abs(infos[k].pres - ia.pres) <= 1e-5 * ia.pres
            assert abs(infos[k].dres - ia.dres) <= 1e-5 * ia.dres
    sc.close()


def test_scenarios_converge_like_alone(opf):
    f = F.feeder_123(2)
    S = 6
    loads = F.load_scenarios(f, S, seed=3)
    sc = opf.Scenarios.from_feeder(f, loads)
    prm = opf.default_params(precision=opf.FP32, rho=10.0, max_iter=200000, check_every=50)
    infos = sc.solve(prm)
    for k in range(S):
        ia, sa = alone(opf, f, loads[k], prm)
        assert infos[k].status == ia.status == 0
        # the residual sums differ only in summation order: same deciding check
        assert infos[k].iters == ia.iters, k
        for x, y in zip(sc.state(k), sa):
            assert np.array_equal(x, y), k
        # FP32 sweeps against the FP64 path, same scenario and iteration count
        i64, _ = alone(opf, f, loads[k], opf.default_params(precision=opf.FP64, rho=10.0, criterion=opf.CRIT_NEVER,
                                                             max_iter=infos[k].iters, check_every=50))
        assert abs(infos[k].objective - i64.objective) <= 1e-4 * abs(i64.objective)
        assert infos[k].pres <= 1e-4 and infos[k].dres <= 1e-4
    sc.close()


def test_scenarios_reject_bad_input(opf):
    f = F.feeder_13(1)
    loads = F.load_scenarios(f, 3, seed=1)
    loads[2]["alpha"][0] = (loads[2]["alpha"][0] + 1) % 3
    with pytest.raises(opf.OpfError):
        opf.Scenarios.from_feeder(f, loads)
    sc = opf.Scenarios.from_feeder(f, F.load_scenarios(f, 3, seed=1))
    with pytest.raises(opf.OpfError):
        sc.solve(opf.default_params(precision=opf.FP64))
    with pytest.raises(opf.OpfError):
        sc.solve(opf.default_params(precision=opf.FP32, check_every=4097))
    with pytest.raises(opf.OpfError):
        sc.solve(opf.default_params(precision=opf.FP32, rho=float("inf")))
    with pytest.raises(opf.OpfError):
        sc.state(3)
    sc.close()


# Tolerances at t = 200 (derivation as in test_gpu_parity.py: sqrt(t n) u for
# x and z, t 4 u for the scaled dual).  CUDA cores: FP32, u = 2^-24.  Tensor
# cores: operands carried as two TF32 parts, about 22 significant bits, so
# u_eff = 2^-22 (4x) and the bounds are 4x larger.
TOLS = {0: (1e-5, 5e-5), 1: (4e-5, 2e-4)}


@pytest.mark.parametrize("xupdate", [0, 1])
@pytest.mark.parametrize("name,maker,picks", [("123", lambda: F.feeder_123(1), (0, 5, 63)),
                                              ("8500", lambda: F.feeder_8500(1), (0, 40))])
def test_scenarios_match_fp64_oracle(opf, name, maker, picks, xupdate):
    """Each scenario of the multi-scenario engine (FP32 sweeps; the small
    shared-operator local update on CUDA cores or on tensor cores in 3xTF32)
    against the FP64 oracle built from that scenario's loads, at t = 200
    (rho = 10): x, z and the scaled dual lambda / rho within TOLS."""
    from oracle import admm as OA, model as OM, precompute as OP
    f = maker()
    loads = F.load_scenarios(f, 64, seed=11)
    sc = opf.Scenarios.from_feeder(f, loads)
    sc.set_xupdate(xupdate)
    tol_x, tol_d = TOLS[xupdate]
    sc.solve(opf.default_params(precision=opf.FP32, rho=10.0, criterion=opf.CRIT_NEVER, max_iter=200, check_every=50))
    for k in picks:
        g = f.copy()
        g.loads = loads[k].copy()
        m = OM.build_feeder(g)
        s = OA.ADMM(m, OP.precompute(m), 10.0)
        for _ in range(200):
            s.step()
        xg, xl, lam = sc.state(k)
        rel = lambda a, b: max(np.linalg.norm(a - b) / np.linalg.norm(b),
                               np.max(np.abs(a - b) / (np.abs(b) + np.max(np.abs(b)))))
        d = (lam - s.lam) / 10.0
        sd = np.max(np.abs(d) / (np.abs(s.lam) / 10.0 + np.max(np.abs(s.lam)) / 10.0 + np.max(np.abs(s.z))))
        assert rel(xg, s.x) <= tol_x and rel(xl, s.z) <= tol_x and sd <= tol_d, (k, rel(xg, s.x), rel(xl, s.z), sd)
    sc.close()


def test_tensor_core_scenarios_converge(opf):
    """Both x-update kinds solve all 64 draws of the 123-bus feeder to ABS
    1e-4 (rho = 10).  Stopped at that residual, the objective is still
    moving (about 5e-3 from the optimum on this feeder; two trajectories
    with different rounding stop at different points), so each result is
    compared with that scenario's LP optimum (HiGHS on the oracle's model) at
    2e-2; a fixed-length run on the CUDA cores after switching back is
    bit-identical to a fresh one."""
    from oracle import lp as OL, model as OM
    f = F.feeder_123(1)
    loads = F.load_scenarios(f, 64, seed=3)
    prm = opf.default_params(precision=opf.FP32, rho=10.0, max_iter=300000, check_every=50)
    res = {}
    for kind in (0, 1):
        sc = opf.Scenarios.from_feeder(f, loads)
        sc.set_xupdate(kind)
        res[kind] = sc.solve(prm)
        sc.close()
    assert all(i.status == opf.OK for kind in (0, 1) for i in res[kind])
    for k in (0, 9, 33, 63):
        g = f.copy()
        g.loads = loads[k].copy()
        lp = OL.solve_lp(OM.build_feeder(g))
        assert lp.status == 0
        for kind in (0, 1):
            assert abs(res[kind][k].objective - lp.fun) <= 2e-2 * abs(lp.fun), (k, kind, res[kind][k].objective, lp.fun)
    sc = opf.Scenarios.from_feeder(f, loads)
    short = opf.default_params(precision=opf.FP32, rho=10.0, criterion=opf.CRIT_NEVER, max_iter=150, check_every=50)
    sc.set_xupdate(1)
    sc.solve(short)
    sc.set_xupdate(0)
    sc.solve(short)          # cold start again, CUDA cores
    x0 = sc.state(7)
    sc.close()
    sc = opf.Scenarios.from_feeder(f, loads)
    sc.solve(short)
    for x, y in zip(x0, sc.state(7)):
        assert np.array_equal(x, y)
    sc.close()
