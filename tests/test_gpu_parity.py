"""GPU parity: the sm_103a path through the C ABI against the FP64 oracle on
the same seeded feeders.

Tolerance (FP64 path): 1e-9 relative per iterate, for the global vector,
the stacked locals and the duals, at several iterations, checked two ways:
normwise, ||gpu - oracle|| <= 1e-9 ||oracle||, and element by element,
|gpu_i - oracle_i| <= 1e-9 (|oracle_i| + ||oracle||_inf), so that a wrong
small entry (a near-zero dual, a slack flow) cannot hide behind the large
ones; residuals likewise.  Both sides run Algorithm 1 in FP64 with
different summation orders and different (but equivalent) precompute
factorizations (operators agree to ~1e-11), and ADMM is non-expansive, so
the gap stays at rounding level.
"""
import numpy as np
import pytest

from paper_2501_08293_b300 import feeders as F

pytestmark = pytest.mark.gpu
TOL = 1e-9


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


def oracle_solver(f, rho):
    from oracle import admm as OA, model as OM, precompute as OP
    m = OM.build_feeder(f)
    pre = OP.precompute(m)
    return m, pre, OA.ADMM(m, pre, rho)


def run_pair(opf, f, rho, checkpoints, variant=0, **kw):
    """Advance GPU (warm-started in chunks) and oracle to each checkpoint."""
    p = opf.Problem.from_feeder(f)
    if variant:
        p.debug_config(variant=variant)
    m, pre, s = oracle_solver(f, rho)
    out = []
    done = 0
    for t in checkpoints:
        info = p.solve(opf.default_params(rho=rho, criterion=opf.CRIT_NEVER, max_iter=t - done,
                                          check_every=min(t - done, 50), warm_start=int(done > 0), **kw))
        assert info.iters == t
        for _ in range(t - done):
            r = s.step()
        done = t
        out.append((t, info, p.state(), (s.x.copy(), s.z.copy(), s.lam.copy()), r))
    return p, out


@pytest.mark.parametrize("maker,rho", [(lambda: F.feeder_13(1), 100.0), (lambda: F.feeder_123(1), 100.0),
                                       (lambda: F.feeder_tiny(6, 2), 10.0), (lambda: F.feeder_13(3), 1000.0)])
def test_fp64_per_iterate_parity(opf, maker, rho):
    f = maker()
    p, out = run_pair(opf, f, rho, [1, 2, 3, 10, 100, 1000])
    c = oracle_cost(f)
    for t, info, (xg, xl, lam), (ox, oz, ol), r in out:
        assert rel(xg, ox) <= TOL, (t, rel(xg, ox))
        assert rel(xl, oz) <= TOL, (t, rel(xl, oz))
        assert rel(lam, ol) <= TOL, (t, rel(lam, ol))
        assert abs(info.pres - r.pres) <= TOL * max(r.pres, 1e-6)
        assert abs(info.dres - r.dres) <= TOL * max(r.dres, 1e-6)
        assert abs(info.eps_prim - r.eps_prim) <= TOL * r.eps_prim
        assert abs(info.eps_dual - r.eps_dual) <= TOL * max(r.eps_dual, 1e-12)
        assert abs(info.objective - float(c @ ox)) <= TOL * max(1.0, abs(info.objective))
    p.close()


def oracle_cost(f):
    from oracle import model as OM
    return OM.build_feeder(f).c


def test_fp64_converges_like_oracle(opf):
    """Same stopping iteration (check every iteration) and the same
    solution at ABS 1e-4 on the 13-bus configuration (rho = 100)."""
    from oracle import admm as OA
    f = F.feeder_13(1)
    m, pre, s = oracle_solver(f, 100.0)
    o = s.run(200000, criterion=OA.CRIT_ABS)
    p = opf.Problem.from_feeder(f)
    info = p.solve(opf.default_params(check_every=1))
    assert info.status == opf.OK
    assert info.iters == o["iters"]
    xg, xl, lam = p.state()
    assert rel(xg, s.x) <= TOL
    assert abs(info.objective - o["objective"]) <= 1e-9 * abs(o["objective"])
    assert info.first_rel_iter == o["first_rel"]
    sol = p.solution()
    w = sol["w"]
    for i in range(f.n_bus):
        for ph in range(3):
            if (int(f.buses["phases"][i]) >> ph) & 1:
                assert w[i, ph] == xg[m.gidx["w"][i, ph]]
            else:
                assert np.isnan(w[i, ph])
    p.close()


def test_engines_and_chunking_are_bitwise_identical(opf):
    """Graph engine (device while-node) == host loop == warm-started chunks,
    bit for bit (fixed-order reductions, no atomics)."""
    f = F.feeder_123(3)
    res = []
    for engine, chunks in ((opf.ENGINE_GRAPH, [300]), (opf.ENGINE_HOSTLOOP, [300]),
                           (opf.ENGINE_GRAPH, [7, 93, 200])):
        p = opf.Problem.from_feeder(f)
        done = 0
        for c in chunks:
            info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=c, check_every=10,
                                              engine=engine, warm_start=int(done > 0)))
            done += c
        assert info.iters == 300
        res.append((p.state(), info.pres, info.dres))
        p.close()
    for (a, pa, da) in res[1:]:
        for x, y in zip(a, res[0][0]):
            assert np.array_equal(x, y)
    assert res[1][1] == res[0][1] and res[1][2] == res[0][2]


def test_full_size_8500_class_parity(opf):
    """8500-class feeder (11,932 nodes, S ~ 25k) in the bench's launch
    configuration: 200 iterations (check every 50) against the oracle."""
    f = F.feeder_8500(1)
    p = opf.Problem.from_feeder(f)
    m, pre, s = oracle_solver(f, 100.0)
    info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=200, check_every=50))
    for _ in range(200):
        r = s.step()
    xg, xl, lam = p.state()
    assert rel(xg, s.x) <= TOL and rel(xl, s.z) <= TOL and rel(lam, s.lam) <= TOL
    assert abs(info.pres - r.pres) <= TOL * r.pres and abs(info.dres - r.dres) <= TOL * r.dres
    # invariants at full size: bounds hold exactly, local rows hold
    assert np.all(xg >= m.lo) and np.all(xg <= m.hi)
    p.close()


# FP32 sweeps against the FP64 oracle: FP32 unit roundoff u = 2^-24 = 6e-8.
# Per iteration each local entry is a sum of at most n_s (<= 39) products and
# each global a sum over its copies; ADMM is non-expansive, so rounding
# errors add up at most linearly over iterations and, being of random sign,
# typically as the square root: sqrt(t * mean n_s) u ~ sqrt(200 * 7) * 6e-8
# ~ 2e-6 at t = 200, plus the one-time rounding of the operators to FP32 (u
# per entry).  The bound below keeps a factor of ~2-5 over that estimate
# (measured on B300: 2.4e-6 to 4.9e-6 for x and z).  The dual update
# lambda += rho (B x - x_s) multiplies the local rounding errors by rho, so
# lambda is compared in the variable in which ADMM is non-expansive, the
# scaled dual lambda / rho, against the scale of the local iterate:
# |dlambda_i| / rho <= TOL (|lambda_i| / rho + max |lambda| / rho + max |z|).
# The scaled dual is a running sum of the primal residuals B x - x_s of all
# iterations so far, so its rounding errors add up linearly in t rather than
# as a square root: t * 4u ~ 200 * 4 * 6e-8 = 4.8e-5 at t = 200 (two
# roundings in the residual, one in the sum, one in the division by rho);
# measured on B300: 1.7e-5 (rho = 100) and 2.8e-5 (rho = 10).
TOL_FP32_T200 = 1e-5
TOL_FP32_DUAL_T200 = 5e-5


def rel_scaled_dual(lam, lam_ref, z_ref, rho):
    d = (lam - lam_ref) / rho
    scale = np.abs(lam_ref) / rho + float(np.max(np.abs(lam_ref))) / rho + float(np.max(np.abs(z_ref)))
    nrm = float(np.linalg.norm(lam_ref)) / rho + float(np.linalg.norm(z_ref))
    return max(float(np.linalg.norm(d)) / nrm, float(np.max(np.abs(d) / scale)))


@pytest.mark.parametrize("rho", [10.0, 100.0])
def test_fp32_per_iterate_parity_8500_class(opf, rho):
    """The headline configuration (8500-class feeder, FP32 sweeps with FP64
    residual sums, default engine and chunking, check every 50) against the
    FP64 oracle at t = 200: x and z within TOL_FP32_T200, lambda / rho
    within TOL_FP32_DUAL_T200, normwise and element by element; residuals
    within 1e-3 relative."""
    f = F.feeder_8500(1)
    p = opf.Problem.from_feeder(f)
    m, pre, s = oracle_solver(f, rho)
    info = p.solve(opf.default_params(rho=rho, criterion=opf.CRIT_NEVER, max_iter=200, check_every=50,
                                      precision=opf.FP32))
    for _ in range(200):
        r = s.step()
    xg, xl, lam = p.state()
    errs = {"x": rel(xg, s.x), "z": rel(xl, s.z), "lam/rho": rel_scaled_dual(lam, s.lam, s.z, rho)}
    assert errs["x"] <= TOL_FP32_T200 and errs["z"] <= TOL_FP32_T200, errs
    assert errs["lam/rho"] <= TOL_FP32_DUAL_T200, errs
    assert abs(info.pres - r.pres) <= 1e-3 * r.pres and abs(info.dres - r.dres) <= 1e-3 * r.dres
    assert abs(info.eps_prim - r.eps_prim) <= 1e-5 * r.eps_prim
    p.close()


def test_edge_cases(opf):
    """max_iter = 0 leaves the initial point; a star feeder whose root bus
    component has n > 32 (one-warp tile path); a generator-only feeder."""
    f = F.feeder_13(2)
    p = opf.Problem.from_feeder(f)
    info = p.solve(opf.default_params(max_iter=0))
    _, xl, lam = p.state()
    m, pre, s = oracle_solver(f, 100.0)
    assert np.array_equal(xl, s.z) and np.all(lam == 0) and info.iters == 0
    p.close()
    # star: 20 single-phase laterals on the root -> root component n = 3 + 20*2 + 6
    star = F.make_feeder(21, 5, n_loads=20, load_sampler=lambda r: r.uniform(0.01, 0.05),
                         line_mix=(0.0, 0.0, 1.0), chain_prob=0.0)
    star.lines["from_bus"] = 0
    star.parent[1:] = 0
    ps = opf.Problem.from_feeder(star)
    assert ps.dims.max_n > 32
    p2, out = run_pair(opf, star, 100.0, [1, 50, 300])
    for t, info, (xg, xl, lam), (ox, oz, ol), r in out:
        assert rel(xg, ox) <= TOL and rel(xl, oz) <= TOL and rel(lam, ol) <= TOL
    p2.close(); ps.close()
    buses = np.zeros(1, F.BUS_DTYPE); buses["phases"] = 1; buses["w_lo"] = 0.9; buses["w_hi"] = 1.1
    # feasible only at pg = 0 (no load, no shunt): pg in [0, 1]
    gens = np.zeros(1, F.GEN_DTYPE); gens["phases"] = 1; gens["pg_lo"] = 0.0; gens["pg_hi"] = 1
    gens["qg_lo"] = -1; gens["qg_hi"] = 1; gens["cost"] = 1
    pg = opf.Problem(buses, np.zeros(0, F.LINE_DTYPE), gens, np.zeros(0, F.LOAD_DTYPE))
    info = pg.solve(opf.default_params(max_iter=5000, check_every=1))
    assert info.status == opf.OK


def test_fp32_path_reaches_tolerance(opf):
    """Reduced-precision sweeps (FP32 x/z/dual, FP64 residual accumulation):
    objective within 1e-4 relative of the FP64 oracle optimum and residuals
    at the 1e-4 target on the 13-bus configuration."""
    from oracle import admm as OA
    f = F.feeder_13(1)
    m, pre, s = oracle_solver(f, 100.0)
    o = s.run(400000, eps_abs_prim=1e-7, eps_abs_dual=1e-7)
    p = opf.Problem.from_feeder(f)
    info = p.solve(opf.default_params(precision=opf.FP32, max_iter=400000, check_every=10))
    assert info.status == opf.OK, info.as_dict()
    assert info.pres <= 1e-4 and info.dres <= 1e-4
    assert abs(info.objective - o["objective"]) <= 1e-4 * abs(o["objective"])
    p.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("maker,rho", [(lambda: F.feeder_13(1), 100.0), (lambda: F.feeder_123(1), 10.0),
                                       (lambda: F.feeder_123(2), 1000.0)])
def test_persistent_engine_parity(opf, maker, rho, variant):
    """Persistent engine (neighbour-synchronized CTAs, ping-pong buffers),
    both kernels: global-memory iterate (1) and shared-memory iterate with
    TMA-staged operators (2), against the oracle per iterate, with odd and
    even solve lengths (the final copy-home path)."""
    f = maker()
    p, out = run_pair(opf, f, rho, [1, 2, 5, 37, 300, 1001], variant=variant, engine=opf.ENGINE_PERSISTENT)
    assert p.dims.n_blocks >= 1
    for t, info, (xg, xl, lam), (ox, oz, ol), r in out:
        assert rel(xg, ox) <= TOL, (t, rel(xg, ox))
        assert rel(xl, oz) <= TOL, (t, rel(xl, oz))
        assert rel(lam, ol) <= TOL, (t, rel(lam, ol))
        assert abs(info.pres - r.pres) <= TOL * max(r.pres, 1e-6)
        assert abs(info.dres - r.dres) <= TOL * max(r.dres, 1e-6)
    p.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_matches_graph_engine_8500(opf, prec):
    """Engines and persistent kernels on the 8500-class feeder (hundreds of
    CTAs): every engine runs the same arithmetic (explicit fused
    multiply-adds, same summation orders), so after 500 iterations the
    iterates and residuals are bit-identical in FP64 and in FP32 -- the
    graph engine, the global-memory persistent kernel and the shared-memory
    one with the gathered (2) and the per-entry (3) boundary exchange."""
    f = F.feeder_8500(1)
    res = []
    for engine, variant in ((opf.ENGINE_GRAPH, 0), (opf.ENGINE_PERSISTENT, 1), (opf.ENGINE_PERSISTENT, 2),
                            (opf.ENGINE_PERSISTENT, 3)):
        p = opf.Problem.from_feeder(f)
        assert p.dims.n_blocks > 100
        p.debug_config(variant=variant)
        info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=500, check_every=50, engine=engine,
                                          precision=prec))
        res.append((p.state(), info))
        p.close()
    (a, ia) = res[0]
    for (b, ib) in res[1:]:
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert ia.iters == ib.iters == 500
        assert ia.pres == ib.pres and ia.dres == ib.dres
    # converging solves stop at the same check
    f = F.feeder_13(1)
    its = []
    for engine in (opf.ENGINE_GRAPH, opf.ENGINE_PERSISTENT):
        p = opf.Problem.from_feeder(f)
        its.append(p.solve(opf.default_params(check_every=10, engine=engine)).iters)
        p.close()
    assert its[0] == its[1]


def test_persistent_wait_expires_cleanly(opf):
    """Failure detection on the device without a fault: one CTA withholds its
    iteration flag, its neighbours' bounded waits expire (50 ms), the solve
    returns OPF_ERR_TIMEOUT, and the same context then solves normally."""
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f)
    assert p.dims.n_blocks >= 2
    p.debug_config(wait_limit_ns=50_000_000, withhold_block=1)
    with pytest.raises(opf.OpfError) as ei:
        p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=1000, check_every=50,
                                   engine=opf.ENGINE_PERSISTENT))
    assert ei.value.status == -6
    p.debug_config(wait_limit_ns=2_000_000_000, withhold_block=-1)
    p2, out = run_pair(opf, f, 100.0, [50], engine=opf.ENGINE_PERSISTENT)
    t, info, (xg, xl, lam), (ox, oz, ol), r = out[0]
    assert rel(xg, ox) <= TOL and rel(xl, oz) <= TOL
    p.close(); p2.close()


def test_residual_balancing_matches_oracle(opf):
    """Residual balancing (optional, Section III-D): rho changes at checks;
    the device and the oracle take the same decisions and stay at 1e-9."""
    from oracle import admm as OA
    f = F.feeder_123(1)
    m, pre, s = oracle_solver(f, 100.0)
    o = s.run(3000, criterion=OA.CRIT_NEVER, check_every=100, adaptive_rho=True)
    for engine in (opf.ENGINE_GRAPH, opf.ENGINE_PERSISTENT):
        p = opf.Problem.from_feeder(f)
        info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=3000, check_every=100,
                                          adaptive_rho=1, engine=engine))
        assert info.rho_changes == o["rho_changes"] and info.rho_changes > 0
        assert info.rho == o["rho"]
        xg, xl, lam = p.state()
        assert rel(xg, s.x) <= TOL and rel(xl, s.z) <= TOL and rel(lam, s.lam) <= TOL
        p.close()


def test_persistent_phase_profile(opf):
    """opf_profile_persistent: per-phase times are positive, the phases add
    up to about the event-timed iteration, and the iterate it leaves is the
    ordinary 300-iteration iterate (profiling does not change the arithmetic)."""
    import torch
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f)
    prm = opf.default_params(precision=1, rho=10.0, check_every=50)
    prof = p.profile_persistent(prm, iters=300)
    a = p.state()
    assert all(v >= 0 for v in prof["mean"].values()) and prof["mean"]["local_interior_check"] > 0
    q = opf.Problem.from_feeder(f)
    q.solve(opf.default_params(precision=1, rho=10.0, check_every=50, criterion=opf.CRIT_NEVER, max_iter=300,
                               engine=opf.ENGINE_PERSISTENT))
    for x, y in zip(a, q.state()):
        assert np.array_equal(x, y)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    q.solve(opf.default_params(precision=1, rho=10.0, check_every=50, criterion=opf.CRIT_NEVER, max_iter=300,
                               engine=opf.ENGINE_PERSISTENT))
    e1.record(); e1.synchronize()
    per_iter = e0.elapsed_time(e1) * 1e3 / 300
    assert 0.3 * per_iter <= sum(prof["mean"].values()) <= 1.5 * per_iter
    p.close(); q.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_nonblocking_checks_return_the_deciding_iterate(opf, prec):
    """The shared-memory persistent kernel does not wait for the residual
    decision: each check leaves a snapshot in the primary buffers and CTAs
    run on until they learn the outcome.  The result must still be the
    iterate of the deciding check: same iteration count, state and residuals
    as the graph engine, for a converging solve on a multi-chunk feeder and
    for a fixed iteration count that is not a multiple of the check interval."""
    f = F.feeder_123(2)
    for crit, max_iter in ((opf.CRIT_ABS, 200000), (opf.CRIT_NEVER, 1234)):
        res = []
        for engine, variant in ((opf.ENGINE_GRAPH, 0), (opf.ENGINE_PERSISTENT, 2)):
            p = opf.Problem.from_feeder(f, chunks=12)
            p.debug_config(variant=variant)
            info = p.solve(opf.default_params(criterion=crit, max_iter=max_iter, check_every=50, engine=engine,
                                              precision=prec, rho=10.0))
            res.append((p.state(), info))
            p.close()
        (a, ia), (b, ib) = res
        assert ia.iters == ib.iters and ia.status == ib.status
        if crit == opf.CRIT_NEVER:
            assert ib.iters == 1234
        else:
            assert ib.status == 0 and ib.iters % 50 == 0
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert ia.pres == ib.pres and ia.dres == ib.dres and ia.objective == ib.objective


@pytest.mark.parametrize("engine", ["graph", "hostloop", "auto"])
def test_textbook_residual_form_matches_oracle(opf, engine):
    """residual_form TEXTBOOK (the sum over components inside the norm of
    Eq. termination): the iterates are those of the paper form, the four
    residual quantities equal the oracle's textbook values at 1e-9 at every
    check, and a REL-criterion solve stops at the oracle's iteration.  The
    persistent engine refuses the form."""
    from oracle import admm as OA
    eng = {"graph": opf.ENGINE_GRAPH, "hostloop": opf.ENGINE_HOSTLOOP, "auto": opf.ENGINE_AUTO}[engine]
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f)
    m, pre, s = oracle_solver(f, 100.0)
    done = 0
    for t in (1, 7, 60, 400):
        info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=t - done, check_every=t - done,
                                          warm_start=int(done > 0), residual_form=opf.RES_TEXTBOOK, engine=eng))
        for _ in range(t - done):
            r = s.step(form=OA.RES_TEXTBOOK)
        done = t
        xg, xl, lam = p.state()
        assert rel(xg, s.x) <= TOL and rel(xl, s.z) <= TOL and rel(lam, s.lam) <= TOL
        for k in ("pres", "dres", "eps_prim", "eps_dual"):
            assert abs(getattr(info, k) - getattr(r, k)) <= TOL * abs(getattr(r, k)), (t, k, getattr(info, k),
                                                                                     getattr(r, k))
    # the two forms differ (a copy's change is spread over its siblings)
    rp = s.residuals(s.B @ s.x, s.z, s.z, s.lam, form=OA.RES_PAPER)
    assert abs(rp.eps_dual - r.eps_dual) > 1e-6 * r.eps_dual
    # stopping on the paper's relative criterion with the textbook norms
    m, pre, s2 = oracle_solver(f, 100.0)
    o = s2.run(200000, criterion=OA.CRIT_REL, form=OA.RES_TEXTBOOK, check_every=10)
    info = p.solve(opf.default_params(criterion=opf.CRIT_REL, max_iter=200000, check_every=10,
                                      residual_form=opf.RES_TEXTBOOK, engine=eng))
    assert info.status == opf.OK and info.iters == o["iters"] and info.first_rel_iter == o["first_rel"]
    if engine == "graph":
        with pytest.raises(opf.OpfError) as ei:
            p.solve(opf.default_params(residual_form=opf.RES_TEXTBOOK, engine=opf.ENGINE_PERSISTENT))
        assert ei.value.status == -1
    p.close()


@pytest.mark.parametrize("engine", ["graph", "persistent"])
@pytest.mark.parametrize("maker,rho", [(lambda: F.feeder_13(1), 100.0), (lambda: F.feeder_123(1), 10.0)])
def test_paper_decomposition_parity(opf, engine, maker, rho):
    """The paper's decomposition (Section V-A: nodes with their loads and
    generators, leaf nodes combined with their lines) through the C ABI
    against the oracle's, per iterate at 1e-9 (normwise and element-wise)."""
    from oracle import admm as OA, model as OM, precompute as OP
    eng = opf.ENGINE_GRAPH if engine == "graph" else opf.ENGINE_PERSISTENT
    f = maker()
    p = opf.Problem.from_feeder(f, decomposition=opf.DECOMP_PAPER)
    m = OM.build_feeder(f, "paper")
    s = OA.ADMM(m, OP.precompute(m), rho)
    assert p.dims.n_comp == m.S and p.dims.n_local == m.nl
    done = 0
    for t in (1, 2, 10, 300, 1001):
        info = p.solve(opf.default_params(rho=rho, criterion=opf.CRIT_NEVER, max_iter=t - done,
                                          check_every=min(50, t - done), warm_start=int(done > 0), engine=eng))
        for _ in range(t - done):
            r = s.step()
        done = t
        xg, xl, lam = p.state()
        assert rel(xg, s.x) <= TOL and rel(xl, s.z) <= TOL and rel(lam, s.lam) <= TOL, t
        assert abs(info.pres - r.pres) <= TOL * max(r.pres, 1e-6)
        assert abs(info.dres - r.dres) <= TOL * max(r.dres, 1e-6)
    p.close()


def test_paper_decomposition_8500_class(opf):
    """Full-size feeder under the paper's decomposition: 200 FP64 iterations
    against the oracle; and both decompositions of the 13-bus feeder solved
    tightly (FP64, ABS 1e-8) reach the LP optimum (stored HiGHS objective)
    to 1e-6, while FP32 solves of the 123-bus feeder converge to ABS 1e-4."""
    from oracle import admm as OA, model as OM, precompute as OP
    f = F.feeder_8500(1)
    p = opf.Problem.from_feeder(f, decomposition=opf.DECOMP_PAPER)
    m = OM.build_feeder(f, "paper")
    s = OA.ADMM(m, OP.precompute(m), 100.0)
    info = p.solve(opf.default_params(criterion=opf.CRIT_NEVER, max_iter=200, check_every=50))
    for _ in range(200):
        r = s.step()
    xg, xl, lam = p.state()
    assert rel(xg, s.x) <= TOL and rel(xl, s.z) <= TOL and rel(lam, s.lam) <= TOL
    assert abs(info.pres - r.pres) <= TOL * r.pres
    p.close()
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "lp_objectives.json")) as fh:
        lp13 = json.load(fh)["feeders"]["13"]["objective"]
    for d in (opf.DECOMP_FINE, opf.DECOMP_PAPER):
        q = opf.Problem.from_feeder(F.feeder_13(1), decomposition=d)
        inf = q.solve(opf.default_params(rho=100.0, max_iter=2000000, eps_abs_prim=1e-8, eps_abs_dual=1e-8))
        assert inf.status == opf.OK and abs(inf.objective - lp13) <= 1e-6 * abs(lp13), (d, inf.objective, lp13)
        q.close()
        q = opf.Problem.from_feeder(F.feeder_123(1), decomposition=d)
        inf = q.solve(opf.default_params(rho=10.0, precision=opf.FP32, max_iter=400000))
        assert inf.status == opf.OK
        q.close()
