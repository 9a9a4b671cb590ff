"""Pins for the CPU oracle: each test ties an oracle function to something
other than itself (an independent derivation, a library routine on a special
case, brute force, or a hand-solvable feeder).  CPU only."""
import math

import numpy as np
import pytest

from oracle import admm as OA
from oracle import lp as OL
from oracle import model as OM
from oracle import precompute as OP
from paper_2501_08293_b300 import feeders as F

ALPHA = np.exp(-2j * np.pi / 3)
PHASOR = np.array([1.0, ALPHA, ALPHA ** 2])   # balanced positive sequence


# ---------------------------------------------------------------- model pins
def test_m_matrices_match_phasor_derivation():
    """M^p, M^q (Section II-A) against the linearized voltage drop derived
    from phasors: with balanced voltages V_phi = a_phi |V| and series power
    S_psi, d w_phi = 2 sum_psi Re[gamma_{phi psi} Z_{phi psi} conj(S_psi)],
    gamma_{phi psi} = a_psi / a_phi.  Then w_j = w_i + Mp p + Mq q means
    Mp = -2 Re(gamma Z), Mq = -2 Im(gamma Z)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        r = rng.uniform(0.0, 1.0, (3, 3)); r = r + r.T
        x = rng.uniform(0.0, 1.0, (3, 3)); x = x + x.T
        Z = r + 1j * x
        gamma = PHASOR[None, :] / PHASOR[:, None]
        mp_ref = -2.0 * (gamma * Z).real
        mq_ref = -2.0 * (gamma * Z).imag
        mp, mq = OM.m_matrices(r.ravel(), x.ravel(), [0, 1, 2])
        np.testing.assert_allclose(mp, mp_ref, rtol=0, atol=1e-13)
        np.testing.assert_allclose(mq, mq_ref, rtol=0, atol=1e-13)
        mp2, mq2 = OM.m_matrices(r.ravel(), x.ravel(), [0, 2])
        np.testing.assert_allclose(mp2, mp_ref[np.ix_([0, 2], [0, 2])], atol=1e-13)
        np.testing.assert_allclose(mq2, mq_ref[np.ix_([0, 2], [0, 2])], atol=1e-13)


def _one_load_model(conn, alpha, a, b):
    buses = np.zeros(1, F.BUS_DTYPE); buses["phases"] = 7
    buses["w_lo"] = 0.81; buses["w_hi"] = 1.21
    loads = np.zeros(1, F.LOAD_DTYPE)
    loads["bus"] = 0; loads["phases"] = 7; loads["conn"] = conn
    loads["a"] = a; loads["b"] = b; loads["alpha"] = alpha; loads["beta"] = alpha
    m = OM.build(buses, np.zeros(0, F.LINE_DTYPE), np.zeros(0, F.GEN_DTYPE), loads)
    return m, [c for c in m.comps if c.kind == OM.KIND_LOAD][0]


def test_delta_rows_match_phasor_delta_to_wye():
    """VDLM-6..10 against circuit theory: delta branch powers S_ab, S_bc, S_ca
    (pd_1, pd_2, pd_3) under balanced phase voltages give bus withdrawals
    S_phi = V_phi conj(I_phi) with I_a = I_ab - I_ca etc.  Those (pb, qb)
    must satisfy the oracle's delta rows exactly."""
    rng = np.random.default_rng(5)
    m, comp = _one_load_model(1, [0, 0, 0], [0.1, 0.2, 0.3], [0.05, 0.01, 0.02])
    for _ in range(10):
        Sd = rng.normal(size=3) + 1j * rng.normal(size=3)
        I = np.zeros(3, complex)
        for k, (i, j) in enumerate(((0, 1), (1, 2), (2, 0))):
            Ib = np.conj(Sd[k] / (PHASOR[i] - PHASOR[j]))
            I[i] += Ib; I[j] -= Ib
        Sb = PHASOR * np.conj(I)
        # local order: pb(3), qb(3), pd(3), qd(3), w(3); rows 6.. are VDLM-6..10
        xs = np.concatenate([Sb.real, Sb.imag, Sd.real, Sd.imag, np.ones(3)])
        rows = comp.A[6:]
        np.testing.assert_allclose(rows @ xs, comp.b[6:], atol=1e-12)
        # and a perturbed withdrawal violates them
        xs[1] += 1e-3
        assert np.abs(rows @ xs - comp.b[6:]).max() > 1e-4


@pytest.mark.parametrize("conn", [0, 1])
@pytest.mark.parametrize("alpha", [0.0, 1.0, 2.0])
def test_load_rows_are_first_order_expansion(conn, alpha):
    """VDLM-1..4: pd = a (what)^{alpha/2} linearized at what = 1, what = w
    (wye) or 3w (delta).  The slope is checked against a central finite
    difference of the exponential load model, independent of the rows."""
    a = np.array([0.1, 0.2, 0.15]); b = 0.3 * a
    m, comp = _one_load_model(conn, [alpha] * 3, a, b)
    mul = 3.0 if conn else 1.0
    for w in (0.9, 1.0, 1.1):
        what = mul * w
        h = 1e-6
        slope = a * ((1 + h) ** (alpha / 2) - (1 - h) ** (alpha / 2)) / (2 * h)
        pd_lin = a + slope * (what - 1.0)
        # solve the pd rows (0, 2, 4 by phase: rows alternate pd, qd per phase)
        for p in range(3):
            row, rhs = comp.A[2 * p], comp.b[2 * p]
            jpd = 6 + p
            jw = 12 + p
            pd = (rhs - row[jw] * w) / row[jpd]
            assert abs(pd - pd_lin[p]) < 1e-8


def _two_bus(phases=1, conn=0, shunt=False, tap=1.0, P=(0.2, 0.15, 0.1), seed=0):
    """Root bus 0 (w fixed at 1) -- line -- bus 1 with one constant-power load."""
    rng = np.random.default_rng(seed)
    mask = {1: 1, 3: 7}[phases]
    buses = np.zeros(2, F.BUS_DTYPE)
    buses["phases"] = mask
    buses["w_lo"] = 0.5; buses["w_hi"] = 1.5
    buses["w_lo"][0] = 1.0; buses["w_hi"][0] = 1.0
    lines = np.zeros(1, F.LINE_DTYPE)
    lines["from_bus"] = 0; lines["to_bus"] = 1; lines["phases"] = mask; lines["in_service"] = 1
    r = rng.uniform(0.01, 0.05, (3, 3)); r = r + r.T
    x = rng.uniform(0.01, 0.05, (3, 3)); x = x + x.T
    lines["r"] = r.ravel(); lines["x"] = x.ravel(); lines["tap"] = tap
    for k in ("p_lo", "q_lo"):
        lines[k] = -5.0
    for k in ("p_hi", "q_hi"):
        lines[k] = 5.0
    if shunt:
        lines["g_fr"] = [0.01, 0.02, 0.015]; lines["b_fr"] = [0.03, 0.01, 0.02]
        lines["g_to"] = [0.005, 0.01, 0.02]; lines["b_to"] = [0.02, 0.02, 0.01]
    gens = np.zeros(1, F.GEN_DTYPE)
    gens["bus"] = 0; gens["phases"] = mask; gens["pg_lo"] = -5; gens["pg_hi"] = 5
    gens["qg_lo"] = -5; gens["qg_hi"] = 5; gens["cost"] = 1.0
    loads = np.zeros(1, F.LOAD_DTYPE)
    loads["bus"] = 1; loads["phases"] = mask; loads["conn"] = conn
    loads["a"] = P; loads["b"] = 0.3 * np.array(P)
    return buses, lines, gens, loads, r, x


@pytest.mark.parametrize("shunt", [False, True])
@pytest.mark.parametrize("tap", [1.0, 1.03])
def test_two_bus_three_phase_circuit_solution(shunt, tap):
    """A 2-bus three-phase feeder with a constant-power wye load has exactly
    one feasible point.  Derived by circuit reasoning (no oracle rows):
    receiving end withdraws the load, the sending end adds the pi-model shunt
    power conj(y_sh) w at both ends, the series power S = S_ij - conj(y_fr) w_i
    drops the voltage by the phasor formula, w_i = tap * w_j - drop."""
    P = np.array([0.2, 0.15, 0.1])
    buses, lines, gens, loads, r, x = _two_bus(3, 0, shunt, tap, P)
    m = OM.build(buses, lines, gens, loads)
    res = OL.solve_lp(m)
    assert res.status == 0
    xs = res.x
    T = m.gidx
    Sload = P + 1j * 0.3 * P
    g_fr = lines["g_fr"][0] + 1j * lines["b_fr"][0]     # y = g + j b
    g_to = lines["g_to"][0] + 1j * lines["b_to"][0]
    Z = r + 1j * x
    gamma = PHASOR[None, :] / PHASOR[:, None]
    # unknown w1 enters the shunt terms: iterate the (linear) relation to a fixed point
    w1 = np.ones(3)
    for _ in range(200):
        S_ji = -Sload                                   # bus 1 balance
        S_ij = -S_ji + np.conj(g_fr) * 1.0 + np.conj(g_to) * w1   # lossless series + shunts
        S_ser = S_ij - np.conj(g_fr) * 1.0              # series power at the sending end
        drop = 2.0 * ((gamma * Z) @ np.conj(S_ser)).real
        w1 = (1.0 - drop) / tap
    for p in range(3):
        assert abs(xs[T["w"][1, p]] - w1[p]) < 1e-9
        assert abs(xs[T["p_ij"][0, p]] - S_ij[p].real) < 1e-9
        assert abs(xs[T["q_ij"][0, p]] - S_ij[p].imag) < 1e-9
        assert abs(xs[T["pg"][0, p]] - S_ij[p].real) < 1e-9
    assert abs(res.fun - S_ij.real.sum()) < 1e-9


def test_bus_shunt_and_generator_signs():
    """Bus balance signs (Eq. balance_eqns): a single bus with a generator,
    a wye constant-power load and shunts g_sh, b_sh at fixed w: pg = pd + g w,
    qg = qd - b w."""
    buses = np.zeros(1, F.BUS_DTYPE); buses["phases"] = 1
    buses["w_lo"] = 1.1; buses["w_hi"] = 1.1
    buses["g_sh"] = 0.02; buses["b_sh"] = 0.05
    gens = np.zeros(1, F.GEN_DTYPE); gens["phases"] = 1; gens["pg_lo"] = -3; gens["pg_hi"] = 3
    gens["qg_lo"] = -3; gens["qg_hi"] = 3; gens["cost"] = 1
    loads = np.zeros(1, F.LOAD_DTYPE); loads["phases"] = 1; loads["a"] = 0.3; loads["b"] = 0.1
    m = OM.build(buses, np.zeros(0, F.LINE_DTYPE), gens, loads)
    res = OL.solve_lp(m)
    assert res.status == 0
    assert abs(res.x[m.gidx["pg"][0, 0]] - (0.3 + 0.02 * 1.1)) < 1e-10
    assert abs(res.x[m.gidx["qg"][0, 0]] - (0.1 - 0.05 * 1.1)) < 1e-10


def test_fine_decomposition_counts():
    """Sizes implied by the fine decomposition: Ng = 2G + B + 4E + 4L,
    Nl = 4G + B + 10E + 7L (phase-unit counts), S = buses + lines + loads + gens;
    every global variable has at least one copy, and B_s maps to distinct
    globals (column sums <= 1, Section II-B)."""
    f = F.feeder_123(2)
    m = OM.build_feeder(f)
    cnt = lambda arr: int(sum(bin(int(v)).count("1") for v in arr["phases"]))
    live = f.lines[f.lines["in_service"] == 1]
    G, B, E, L = cnt(f.gens), cnt(f.buses), cnt(live), cnt(f.loads)
    assert m.n == 2 * G + B + 4 * E + 4 * L
    assert m.nl == 4 * G + B + 10 * E + 7 * L
    assert m.S == len(f.buses) + len(live) + len(f.loads) + len(f.gens)
    k = np.zeros(m.n, int)
    for c in m.comps:
        assert len(set(c.gvars.tolist())) == len(c.gvars)
        k[c.gvars] += 1
    assert k.min() >= 1


def test_generator_radial_and_phase_nesting():
    for f in (F.feeder_13(3), F.feeder_123(3), F.feeder_8500(2, n_bus=3000)):
        live = f.lines[f.lines["in_service"] == 1]
        assert len(live) == f.n_bus - 1
        par = {}
        for ln in live:
            assert int(ln["to_bus"]) not in par
            par[int(ln["to_bus"])] = int(ln["from_bus"])
            assert int(ln["phases"]) & ~int(f.buses[ln["from_bus"]]["phases"]) == 0
            assert int(ln["phases"]) == int(f.buses[ln["to_bus"]]["phases"])
        for j in range(1, f.n_bus):          # every bus reaches the root
            seen = 0
            while j != 0:
                j = par[j]; seen += 1
                assert seen <= f.n_bus


# ----------------------------------------------------------- precompute pins
def test_rref_rank_and_consistency():
    """Section IV-B row reduction on constructed rank-deficient systems."""
    rng = np.random.default_rng(7)
    for m, n, r in ((6, 9, 3), (5, 5, 5), (8, 10, 1), (4, 7, 2)):
        R = rng.normal(size=(r, n)); C = rng.normal(size=(m, r))
        A = C @ R
        b = C @ rng.normal(size=r)
        Ar, br, piv = OP.rref(A, b)
        assert Ar.shape == (r, n) and len(piv) == r
        # same row space (projectors agree) and same solution set
        Pr = R.T @ np.linalg.solve(R @ R.T, R)
        Pa = Ar.T @ np.linalg.solve(Ar @ Ar.T, Ar)
        np.testing.assert_allclose(Pa, Pr, atol=1e-10)
        x0 = np.linalg.lstsq(A, b, rcond=None)[0]
        np.testing.assert_allclose(Ar @ x0, br, atol=1e-9)
        # pivot columns hold the identity (reduced echelon form)
        np.testing.assert_allclose(Ar[:, piv], np.eye(r), atol=1e-12)
        if r < m:
            bad = b.copy(); bad += rng.normal(size=m) * 1e-2
            with pytest.raises(OP.InconsistentError):
                OP.rref(A, bad)


def test_closed_form_matches_dense_kkt_and_svd():
    """Eq. (closed_2) against (i) the dense KKT system of Eq.
    (quadratic_problem) [rho I, A^T; A, 0][x; mu] = [-d; b] and (ii) the SVD:
    -Abar is the projector onto null(A), bbar the minimum-norm solution."""
    rng = np.random.default_rng(11)
    for m, n in ((3, 7), (1, 2), (6, 6), (4, 12)):
        A = rng.normal(size=(m, n)); b = rng.normal(size=m)
        Abar, bbar = OP.closed_form(A, b)
        for rho in (10.0, 100.0, 1000.0):
            d = rng.normal(size=n) * rho
            K = np.block([[rho * np.eye(n), A.T], [A, np.zeros((m, m))]])
            sol = np.linalg.solve(K, np.concatenate([-d, b]))
            np.testing.assert_allclose(Abar @ d / rho + bbar, sol[:n], atol=1e-12 * max(1, np.abs(sol).max()))
        U, s, Vt = np.linalg.svd(A)
        N = Vt[m:].T
        np.testing.assert_allclose(-Abar, N @ N.T, atol=1e-12)
        np.testing.assert_allclose(bbar, np.linalg.pinv(A) @ b, atol=1e-12)


def test_component_projectors_on_feeder():
    """On every component of a feeder: -Abar symmetric, idempotent, A Abar = -A
    (so A x_s = b_s for any update), and A bbar = b."""
    m = OM.build_feeder(F.feeder_13(2))
    pre = OP.precompute(m)
    for s, comp in enumerate(m.comps):
        P = -pre.Abar[s]
        np.testing.assert_allclose(P, P.T, atol=1e-13)
        np.testing.assert_allclose(P @ P, P, atol=1e-12)
        if comp.A.shape[0]:
            np.testing.assert_allclose(comp.A @ P, 0, atol=1e-10)
            np.testing.assert_allclose(comp.A @ pre.bbar[s], comp.b, atol=1e-10)


# ------------------------------------------------------------------ ADMM pins
def test_global_update_matches_bruteforce_1d():
    """Eq. (ADMM-1) is separable; each coordinate minimizes
    (c_i + sum lam_j) x + rho/2 sum (x - z_j)^2 over [lo, hi].  Compare the
    oracle's global update with a dense grid search plus golden refinement."""
    rng = np.random.default_rng(2)
    m = OM.build_feeder(F.feeder_tiny(4, 5))
    pre = OP.precompute(m)
    s = OA.ADMM(m, pre, 37.0)
    s.z = rng.normal(size=len(s.gidx)) * 0.5 + 1.0
    s.lam = rng.normal(size=len(s.gidx)) * 3
    x = s.global_update()
    for i in rng.choice(m.n, size=25, replace=False):
        js = np.nonzero(s.gidx == i)[0]
        lo, hi = m.lo[i], m.hi[i]
        lo_ = lo if np.isfinite(lo) else -20.0
        hi_ = hi if np.isfinite(hi) else 20.0
        f = lambda t: (m.c[i] + s.lam[js].sum()) * t + 0.5 * s.rho * np.sum((t - s.z[js]) ** 2)
        grid = np.linspace(lo_, hi_, 200001)
        vals = (m.c[i] + s.lam[js].sum()) * grid + 0.5 * s.rho * ((grid[:, None] - s.z[js][None, :]) ** 2).sum(1)
        t0 = grid[np.argmin(vals)]
        step = (hi_ - lo_) / 200000
        a_, b_ = max(lo_, t0 - step), min(hi_, t0 + step)
        for _ in range(100):                     # golden-section refinement
            c1 = b_ - 0.618 * (b_ - a_); c2 = a_ + 0.618 * (b_ - a_)
            if f(c1) < f(c2):
                b_ = c2
            else:
                a_ = c1
        # minimizing by function values resolves the argmin to ~sqrt(eps)
        assert abs(x[i] - 0.5 * (a_ + b_)) < 1e-7 * max(1.0, abs(x[i]))


def test_initialization_rule():
    """Section V-A: lam = 0; local entries 1 for voltages, midpoint if both
    bounds finite, 0 if unbounded."""
    m = OM.build_feeder(F.feeder_tiny(5, 3))
    s = OA.ADMM(m, OP.precompute(m), 100.0)
    assert np.all(s.lam == 0)
    for j, g in enumerate(s.gidx):
        nm = m.names[g][0]
        if nm == "w":
            assert s.z[j] == 1.0
        elif nm in ("pb", "qb", "pd", "qd"):
            assert s.z[j] == 0.0
        else:
            assert s.z[j] == 0.5 * (m.lo[g] + m.hi[g])


def test_residual_forms_bruteforce():
    """Eq. (termination) evaluated literally per component (B_s^T scatter)
    matches the oracle's residuals, both forms."""
    m = OM.build_feeder(F.feeder_tiny(4, 2))
    pre = OP.precompute(m)
    s = OA.ADMM(m, pre, 100.0)
    for _ in range(5):
        s.step()
    z_prev = s.z.copy()
    s.step()
    x, z, lam = s.x, s.z, s.lam
    acc = dict(p=0.0, d=0.0, bx=0.0, z=0.0, l=0.0)
    tot_d = np.zeros(m.n); tot_l = np.zeros(m.n)
    for k, comp in enumerate(m.comps):
        sl = slice(s.comp_ptr[k], s.comp_ptr[k + 1])
        Bs = np.zeros((len(comp.gvars), m.n)); Bs[np.arange(len(comp.gvars)), comp.gvars] = 1
        acc["p"] += np.sum((Bs @ x - z[sl]) ** 2)
        acc["d"] += np.sum((Bs.T @ (z[sl] - z_prev[sl])) ** 2)
        acc["bx"] += np.sum((Bs @ x) ** 2); acc["z"] += np.sum(z[sl] ** 2)
        acc["l"] += np.sum((Bs.T @ lam[sl]) ** 2)
        tot_d += Bs.T @ (z[sl] - z_prev[sl]); tot_l += Bs.T @ lam[sl]
    r = s.residuals(s.B @ x, z, z_prev, lam, OA.RES_PAPER, 1e-3)
    assert math.isclose(r.pres, math.sqrt(acc["p"]), rel_tol=1e-12)
    assert math.isclose(r.dres, 100.0 * math.sqrt(acc["d"]), rel_tol=1e-12)
    assert math.isclose(r.eps_prim, 1e-3 * max(math.sqrt(acc["bx"]), math.sqrt(acc["z"])), rel_tol=1e-12)
    assert math.isclose(r.eps_dual, 1e-3 * math.sqrt(acc["l"]), rel_tol=1e-12)
    r2 = s.residuals(s.B @ x, z, z_prev, lam, OA.RES_TEXTBOOK, 1e-3)
    assert math.isclose(r2.dres, 100.0 * np.linalg.norm(tot_d), rel_tol=1e-12)
    assert math.isclose(r2.eps_dual, 1e-3 * np.linalg.norm(tot_l), rel_tol=1e-12)


def test_local_update_equals_kkt_per_component():
    """Eq. (closed_2) inside the stacked update equals a per-component dense
    KKT solve of Eq. (quadratic_problem) with d_s = -rho B_s x - lam_s."""
    rng = np.random.default_rng(4)
    m = OM.build_feeder(F.feeder_13(4))
    pre = OP.precompute(m)
    s = OA.ADMM(m, pre, 100.0)
    s.lam = rng.normal(size=len(s.gidx))
    x = rng.uniform(0.9, 1.1, m.n)
    z = s.local_update(x)
    for k in range(m.S):
        sl = slice(s.comp_ptr[k], s.comp_ptr[k + 1])
        A, b = pre.Ared[k], pre.bred[k]
        n, mm = A.shape[1], A.shape[0]
        d = -s.rho * x[s.gidx[sl]] - s.lam[sl]
        K = np.block([[s.rho * np.eye(n), A.T], [A, np.zeros((mm, mm))]])
        sol = np.linalg.solve(K, np.concatenate([-d, b]))
        np.testing.assert_allclose(z[sl], sol[:n], atol=1e-11)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_iterate_invariants(seed):
    """At every iterate: A_s x_s = b_s (closed-form local solution) and
    xlo <= x <= xhi (clipped global update)."""
    m = OM.build_feeder(F.feeder_tiny(6, seed))
    pre = OP.precompute(m)
    s = OA.ADMM(m, pre, 100.0)
    for t in range(30):
        s.step()
        assert np.all(s.x >= m.lo) and np.all(s.x <= m.hi)
        for k, comp in enumerate(m.comps):
            if comp.A.shape[0]:
                zs = s.z[s.comp_ptr[k]:s.comp_ptr[k + 1]]
                np.testing.assert_allclose(comp.A @ zs, comp.b, atol=1e-11)


@pytest.mark.parametrize("maker", [lambda: F.feeder_13(1), lambda: F.feeder_tiny(5, 4)])
def test_fixed_point_matches_highs_and_gap_closes(maker):
    """Eq. (OurModel) is equivalent to Eq. (LP_model): the ADMM limit attains
    the HiGHS optimum, and the duality gap of the ADMM duals closes."""
    f = maker()
    m = OM.build_feeder(f)
    pre = OP.precompute(m)
    lp = OL.solve_lp(m)
    assert lp.status == 0
    s = OA.ADMM(m, pre, 100.0)
    out = s.run(400000, eps_abs_prim=1e-8, eps_abs_dual=1e-8, criterion=OA.CRIT_ABS)
    assert out["converged"]
    obj = out["objective"]
    assert abs(obj - lp.fun) <= 1e-6 * max(1.0, abs(lp.fun))
    cert = OA.dual_certificate(m, pre, s)
    assert abs(cert["primal"] - cert["dual"]) <= 1e-5 * max(1.0, abs(lp.fun))
    assert cert["free_residual"] < 1e-5
    # per-phase power balance from the solution (bus rows hold to ~pres)
    A, b = OM.stacked_A(m)
    assert np.abs(A @ s.x - b).max() < 1e-6


def test_two_bus_admm_reaches_unique_point():
    """ADMM on the 2-bus single-phase feeder converges to its unique feasible
    point: pg = load, w1 = 1 + Mp_aa p + Mq_aa q (derived by hand)."""
    buses, lines, gens, loads, r, x = _two_bus(1, 0, False, 1.0, (0.2, 0, 0))
    m = OM.build(buses, lines, gens, loads)
    pre = OP.precompute(m)
    s = OA.ADMM(m, pre, 100.0)
    out = s.run(200000, eps_abs_prim=1e-9, eps_abs_dual=1e-9)
    assert out["converged"]
    P, Q = 0.2, 0.06
    assert abs(s.x[m.gidx["pg"][0, 0]] - P) < 1e-7
    assert abs(s.x[m.gidx["w"][1, 0]] - (1 - 2 * r[0, 0] * P - 2 * x[0, 0] * Q)) < 1e-7


def test_paper_table3_component_identity():
    """Table III: S = nodes + lines - leaves for IEEE13/123/8500 (golden)."""
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")) as fh:
        g = json.load(fh)
    for name, row in g["table3"].items():
        if name.startswith("_"):
            continue
        assert row["nodes"] + row["lines"] - row["leaves"] == row["S"]
    t4 = g["table4_8500"]
    # Table IV: printed means (two decimals, truncated) are the sums over S
    S = g["table3"]["IEEE8500"]["S"]
    assert 0 <= t4["n_sum"] / S - t4["n_mean"] < 0.01
    assert 0 <= t4["m_sum"] / S - t4["m_mean"] < 0.01


def test_precompute_accurate_on_short_lines():
    """8500-class short lines give tiny per-unit impedances; the operators
    must still equal the SVD null-space projector and minimum-norm solution
    to FP64 accuracy (the library and oracle are compared at 1e-10)."""
    f = F.feeder_8500(1, n_bus=600)
    m = OM.build_feeder(f)
    pre = OP.precompute(m)
    for s, comp in enumerate(m.comps):
        if comp.kind != OM.KIND_LINE:
            continue
        A = comp.A
        U, S, Vt = np.linalg.svd(A)
        N = Vt[A.shape[0]:].T
        np.testing.assert_allclose(-pre.Abar[s], N @ N.T, atol=1e-12)
        np.testing.assert_allclose(pre.bbar[s], np.linalg.pinv(A) @ comp.b, atol=1e-12)


def test_rank_deficient_component_uses_row_reduction():
    """A bus phase with nothing attached and no shunt gives a zero balance
    row (0 = 0): row reduction drops it and the operators still match SVD."""
    buses = np.zeros(2, F.BUS_DTYPE); buses["phases"] = [7, 7]
    buses["w_lo"] = 0.9; buses["w_hi"] = 1.1
    lines = np.zeros(1, F.LINE_DTYPE); lines["from_bus"] = 0; lines["to_bus"] = 1
    lines["phases"] = 1; lines["in_service"] = 1; lines["r"] = 0.01; lines["x"] = 0.02; lines["tap"] = 1
    lines["p_lo"] = -1; lines["p_hi"] = 1; lines["q_lo"] = -1; lines["q_hi"] = 1
    m = OM.build(buses, lines, np.zeros(0, F.GEN_DTYPE), np.zeros(0, F.LOAD_DTYPE))
    pre = OP.precompute(m)
    bus1 = m.comps[1]
    assert bus1.A.shape[0] == 6 and pre.m_red[1] == 2
    U, S, Vt = np.linalg.svd(bus1.A)
    N = Vt[2:].T
    np.testing.assert_allclose(-pre.Abar[1], N @ N.T, atol=1e-12)


def test_golden_lp_objectives_reproduce():
    """tests/golden/lp_objectives.json (written by make_lp_objectives.py,
    oracle only) matches a fresh HiGHS solve on the small feeders."""
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "lp_objectives.json")) as fh:
        g = json.load(fh)["feeders"]
    for name, f in (("13", F.feeder_13(1)), ("123", F.feeder_123(1))):
        r = OL.solve_lp(OM.build_feeder(f))
        assert r.status == 0 and abs(r.fun - g[name]["objective"]) <= 1e-9 * abs(r.fun)


def test_residual_balancing_rule_on_scripted_residuals():
    """Residual balancing (Section III-D names it; the rule is the standard
    one of Boyd et al., 2011, "Distributed Optimization and Statistical
    Learning via the ADMM", Sec. 3.4.1, Eq. 3.13): at a check that does not
    stop, rho -> tau rho if ||r|| > mu ||s||, rho -> rho / tau if
    ||s|| > mu ||r||, else unchanged (r = primal, s = dual residual).  The
    oracle's step is replaced by a scripted residual sequence; the rho in
    effect at each step is worked out by hand below (mu = 10, tau = 2,
    rho0 = 100), including the strict comparison, no change at max_iter and
    no change on the check that stops."""
    m = OM.build_feeder(F.feeder_tiny(3, 1))
    s = OA.ADMM(m, OP.precompute(m), 100.0)
    script = [(1.0, 0.01), (1.0, 0.2), (0.001, 1.0), (0.001, 1.0), (10.0, 1.0), (10.0001, 1.0), (1.0, 0.0)]
    seen = []

    def fake_step(form=OA.RES_PAPER, eps_rel=1e-3):
        seen.append(s.rho)
        pr, du = script[len(seen) - 1]
        s.t += 1
        return OA.Residuals(pr, du, 1.0, 1.0)

    s.step = fake_step
    out = s.run(len(script), criterion=OA.CRIT_NEVER, check_every=1, adaptive_rho=True, rb_mu=10.0, rb_tau=2.0)
    assert seen == [100.0, 200.0, 200.0, 100.0, 50.0, 50.0, 100.0]
    assert out["rho"] == 100.0 and out["rho_changes"] == 4
    # checks every 2 iterations: only the residuals at t = 2 (no change),
    # 4 (halve), 6 (double) count; t = 7 is max_iter (no change)
    s.rho, s.t = 100.0, 0
    seen.clear()
    out = s.run(len(script), criterion=OA.CRIT_NEVER, check_every=2, adaptive_rho=True)
    assert seen == [100.0, 100.0, 100.0, 100.0, 50.0, 50.0, 100.0]
    assert out["rho_changes"] == 2
    # the check that stops leaves rho alone
    script[:] = [(1.0, 0.001), (1e-6, 1e-3)]
    s.rho, s.t = 100.0, 0
    seen.clear()
    out = s.run(10, criterion=OA.CRIT_ABS, eps_abs_prim=1e-4, eps_abs_dual=1e-2, check_every=1, adaptive_rho=True)
    assert out["converged"] and out["iters"] == 2 and seen == [100.0, 200.0] and out["rho"] == 200.0


def test_residual_balancing_equals_restart_at_new_rho():
    """Abar_s and bbar_s do not depend on rho and the duals are unscaled, so
    continuing after a residual-balancing change of rho is the same as a
    fresh Algorithm 1 at the new rho started from the same (x, z, lambda):
    the adaptive run must equal, bit for bit, a chain of fixed-rho runs
    restarted at every change.  (A plausible slip -- rescaling lambda as in
    the scaled-dual form, or applying the new rho one iteration late --
    breaks the equality.)"""
    f = F.feeder_13(2)
    m = OM.build_feeder(f)
    pre = OP.precompute(m)
    K, T = 40, 800
    a = OA.ADMM(m, pre, 100.0)
    ref = a.run(T, criterion=OA.CRIT_NEVER, check_every=K, adaptive_rho=True)
    assert ref["rho_changes"] >= 2
    # rho in effect after each check j (a run of K j + 1 iterations applies
    # the decision of check j and stops before the next one)
    rhos = [100.0]
    for j in range(1, T // K):
        r = OA.ADMM(m, pre, 100.0).run(K * j + 1, criterion=OA.CRIT_NEVER, check_every=K, adaptive_rho=True)
        rhos.append(r["rho"])
    assert len(set(rhos)) >= 3
    b = OA.ADMM(m, pre, rhos[0])
    for j in range(T // K):
        if j and rhos[j] != rhos[j - 1]:
            fresh = OA.ADMM(m, pre, rhos[j])
            fresh.x, fresh.z, fresh.lam, fresh.t = b.x, b.z, b.lam, b.t
            b = fresh
        for _ in range(K):
            b.step()
    assert b.t == a.t == T and b.rho == ref["rho"]
    assert np.array_equal(b.x, a.x) and np.array_equal(b.z, a.z) and np.array_equal(b.lam, a.lam)


def _leaves_and_nodes(f):
    live = np.flatnonzero(f.lines["in_service"] == 1)
    deg = np.zeros(f.n_bus, dtype=int)
    for e in live:
        deg[int(f.lines["from_bus"][e])] += 1
        deg[int(f.lines["to_bus"][e])] += 1
    return live, deg


@pytest.mark.parametrize("maker", [lambda: F.feeder_13(1), lambda: F.feeder_123(2), lambda: F.feeder_tiny(6, 3),
                                   lambda: F.feeder_8500(1, n_bus=2000)])
def test_paper_decomposition_counts(maker):
    """Section V-A / Table III: with the paper's decomposition S = nodes +
    lines - leaves (a leaf = a node with one in-service line); rows are
    neither lost nor added (sum m_s equal to the fine decomposition's); and
    every local copy that the combination removes is one that two parts
    shared: a load shares pb, qb, w with its bus (3 |P_l|), a generator pg,
    qg (2 |P_k|), a leaf node the flows leaving it and its w with its line
    (3 |P_e|), so sum n_s drops by exactly that."""
    f = maker()
    fine = OM.build_feeder(f)
    paper = OM.build_feeder(f, "paper")
    live, deg = _leaves_and_nodes(f)
    leaves = int(np.sum(deg == 1))
    assert paper.S == f.n_bus + len(live) - leaves
    assert sum(c.A.shape[0] for c in paper.comps) == sum(c.A.shape[0] for c in fine.comps)
    npl = lambda mask: bin(int(mask)).count("1")
    drop = sum(3 * npl(d["phases"]) for d in f.loads) + sum(2 * npl(g["phases"]) for g in f.gens)
    for e in live:
        for end in ("from_bus", "to_bus"):
            if deg[int(f.lines[end][e])] == 1:
                drop += 3 * npl(f.lines["phases"][e])
    assert paper.nl == fine.nl - drop
    # every global keeps at least one copy, and no component copies a global twice
    for c in paper.comps:
        assert len(set(c.gvars.tolist())) == len(c.gvars)
    assert set(np.concatenate([c.gvars for c in paper.comps]).tolist()) == set(range(paper.n))


@pytest.mark.parametrize("maker", [lambda: F.feeder_13(1), lambda: F.feeder_123(2)])
def test_paper_decomposition_is_the_same_lp(maker):
    """Both decompositions split the same centralized rows of Eq. (LP_model):
    the stacked rows A_s B_s (mapped to global columns) are the same set of
    rows, with the same right-hand sides."""
    f = maker()
    A1, b1 = OM.stacked_A(OM.build_feeder(f))
    A2, b2 = OM.stacked_A(OM.build_feeder(f, "paper"))
    key = lambda A, b: sorted((tuple(sorted(zip(A.getrow(r).indices.tolist(), A.getrow(r).data.tolist()))), b[r])
                              for r in range(A.shape[0]))
    assert key(A1.tocsr(), b1) == key(A2.tocsr(), b2)


@pytest.mark.parametrize("maker", [lambda: F.feeder_tiny(5, 1), lambda: F.feeder_13(1)])
def test_paper_decomposition_fixed_point_matches_highs(maker):
    """Algorithm 1 on the paper's decomposition reaches the same LP optimum
    (HiGHS) and its duality gap closes."""
    f = maker()
    m = OM.build_feeder(f, "paper")
    pre = OP.precompute(m)
    lp = OL.solve_lp(OM.build_feeder(f))
    s = OA.ADMM(m, pre, 100.0)
    out = s.run(400000, eps_abs_prim=1e-8, eps_abs_dual=1e-8, criterion=OA.CRIT_ABS)
    assert out["converged"]
    assert abs(out["objective"] - lp.fun) <= 1e-6 * max(1.0, abs(lp.fun))
    cert = OA.dual_certificate(m, pre, s)
    assert abs(cert["primal"] - cert["dual"]) <= 1e-5 * max(1.0, abs(lp.fun))
