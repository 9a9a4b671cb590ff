"""C-ABI library: loads, exports every declared symbol, record layouts, and
host-side logic (assembly, precompute, packing) against the oracle.  CPU only:
no call here touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2501_08293_b300 import feeders as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def opf():
    from paper_2501_08293_b300 import build
    build.build()
    from paper_2501_08293_b300 import opf as mod
    return mod


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(opf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(opf):
    names = declared_functions()
    assert len(names) >= 14
    lib = C.CDLL(opf._LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(opf.EXPORTS), "binding misses a declared entry point"


def test_record_layouts(opf):
    lib = opf.lib
    assert lib.opf_abi_version() == 1
    assert lib.opf_record_size(0) == F.BUS_DTYPE.itemsize
    assert lib.opf_record_size(1) == F.LINE_DTYPE.itemsize
    assert lib.opf_record_size(2) == F.GEN_DTYPE.itemsize
    assert lib.opf_record_size(3) == F.LOAD_DTYPE.itemsize
    assert lib.opf_record_size(4) == C.sizeof(opf.Params)
    assert lib.opf_record_size(5) == C.sizeof(opf.Info)
    assert lib.opf_record_size(6) == C.sizeof(opf.Dims)
    assert lib.opf_record_size(99) == 0
    p = opf.default_params()
    assert p.rho == 100.0 and p.eps_abs_prim == 1e-4 and p.eps_rel == 1e-3


@pytest.mark.parametrize("decomp", ["fine", "paper"])
@pytest.mark.parametrize("maker", [lambda: F.feeder_13(1), lambda: F.feeder_123(2),
                                   lambda: F.feeder_tiny(6, 3), lambda: F.feeder_8500(1, n_bus=1500)])
def test_host_precompute_matches_oracle(opf, maker, decomp):
    """Independent C++ assembly + QR projector vs the oracle's rows + RREF +
    Cholesky: same canonical structure, ranks and operators (P = -Abar), for
    the fine decomposition and the paper's (Section V-A)."""
    from oracle import model as OM, precompute as OP
    f = maker()
    p = opf.Problem.from_feeder(f, upload=False,
                                decomposition=opf.DECOMP_PAPER if decomp == "paper" else opf.DECOMP_FINE)
    m = OM.build_feeder(f, decomp)
    pre = OP.precompute(m)
    st = p.structure()
    assert p.dims.n_global == m.n and p.dims.n_local == m.nl and p.dims.n_comp == m.S
    assert p.dims.n_rows == sum(c.A.shape[0] for c in m.comps)
    assert (st["m_reduced"] == pre.m_red).all()
    assert (st["gidx"] == np.concatenate([c.gvars for c in m.comps])).all()
    assert (st["kind"] == np.array([c.kind for c in m.comps])).all()
    assert (st["index"] == np.array([c.index for c in m.comps])).all()
    ns = np.diff(st["comp_ptr"])
    assert p.dims.sum_n2 == int((ns.astype(np.int64) ** 2).sum()) and p.dims.max_n == ns.max()
    for s in range(m.S):
        P, b = p.operator(s)
        np.testing.assert_allclose(P, -pre.Abar[s], atol=1e-10)
        np.testing.assert_allclose(b, pre.bbar[s], atol=1e-10)
    p.close()


def _err(opf, f):
    with pytest.raises(opf.OpfError) as ei:
        opf.Problem.from_feeder(f, upload=False)
    return ei.value.status


def test_invalid_inputs_are_rejected(opf):
    base = F.feeder_tiny(5, 1)
    f = base.copy(); f.lines["to_bus"][0] = 99
    assert _err(opf, f) == -1
    f = base.copy(); f.lines["to_bus"][0] = f.lines["from_bus"][0]
    assert _err(opf, f) == -1
    f = base.copy(); f.buses["w_lo"][1] = 2.0
    assert _err(opf, f) == -1
    f = base.copy(); f.buses["phases"][0] = 0
    assert _err(opf, f) == -1
    f = base.copy(); f.loads["phases"][0] = 1; f.loads["conn"][0] = 1
    f.buses["phases"][f.loads["bus"][0]] |= 1
    assert _err(opf, f) == -1       # delta on one phase
    f = base.copy(); f.lines["r"][0][0] = np.nan
    assert _err(opf, f) == -1
    f = base.copy(); f.gens["bus"][0] = -1
    assert _err(opf, f) == -1
    assert "line" in opf.lib.opf_last_error().decode() or True


def test_out_of_service_line_and_degenerate_feeders(opf):
    """An open line leaves the model (no variables, no component); a single
    bus with a generator only (no lines, no loads) still builds."""
    f = F.feeder_123(1)
    p1 = opf.Problem.from_feeder(f, upload=False)
    g = f.copy()
    live = np.nonzero(g.lines["in_service"] == 1)[0]
    assert (g.lines["in_service"] == 0).sum() >= 1
    p2 = opf.Problem.from_feeder(g, upload=False)
    assert p2.dims.n_comp == p1.dims.n_comp
    buses = np.zeros(1, F.BUS_DTYPE); buses["phases"] = 7; buses["w_lo"] = 0.9; buses["w_hi"] = 1.1
    gens = np.zeros(1, F.GEN_DTYPE); gens["phases"] = 7; gens["pg_hi"] = 1; gens["qg_hi"] = 1; gens["cost"] = 1
    p = opf.Problem(buses, np.zeros(0, F.LINE_DTYPE), gens, np.zeros(0, F.LOAD_DTYPE), upload=False)
    assert p.dims.n_comp == 2 and p.dims.n_global == 9
    assert len(live) == f.n_bus - 1


def test_scenario_inputs_are_validated_on_the_host(opf):
    """opf_scenarios_create rejects scenarios whose loads differ in anything
    but the draw (a, b) before it touches a device; load_scenarios keeps
    everything but the draw."""
    import ctypes as C
    f = F.feeder_13(1)
    loads = F.load_scenarios(f, 3, seed=2)
    assert loads.shape == (3, len(f.loads)) and loads.dtype == F.LOAD_DTYPE
    for k in range(3):
        for fld in ("bus", "phases", "conn", "alpha", "beta"):
            assert np.array_equal(loads[k][fld], f.loads[fld])
    assert np.array_equal(loads[0]["a"], f.loads["a"])
    assert not np.array_equal(loads[1]["a"], f.loads["a"])
    bad = loads.copy()
    bad[1]["conn"][0] = 1 - bad[1]["conn"][0]
    arrs = [np.ascontiguousarray(a) for a in (f.buses, f.lines, f.gens)]
    h = C.c_void_p()
    st = opf.lib.opf_scenarios_create(arrs[0].ctypes.data, len(arrs[0]), arrs[1].ctypes.data, len(arrs[1]),
                                      arrs[2].ctypes.data, len(arrs[2]), bad.ctypes.data, len(f.loads), 3,
                                      C.byref(h))
    assert st == -1 and not h.value
    assert b"only the load draw" in opf.lib.opf_last_error()
    st = opf.lib.opf_scenarios_create(arrs[0].ctypes.data, len(arrs[0]), arrs[1].ctypes.data, len(arrs[1]),
                                      arrs[2].ctypes.data, len(arrs[2]), loads.ctypes.data, len(f.loads), 0,
                                      C.byref(h))
    assert st == -1


def test_line_updates_are_validated_on_the_host(opf):
    """opf_update_lines checks every record before touching a device: a
    line that is not in service, other ends or phases are rejected; a valid
    update of a problem that is not uploaded reports the state."""
    import ctypes as C
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f, upload=False)
    live = int(np.flatnonzero(f.lines["in_service"] == 1)[3])
    dead = np.flatnonzero(f.lines["in_service"] == 0)

    def call(idx, rec):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        rec = np.ascontiguousarray(rec)
        return opf.lib.opf_update_lines(p._h, idx.ctypes.data_as(opf._I), rec.ctypes.data, len(idx), None)

    rec = f.lines[[live]].copy()
    rec["r"] *= 1.1
    assert call([live], rec) == -7                  # valid, but not uploaded
    bad = rec.copy(); bad["to_bus"] = (bad["to_bus"] + 1) % len(f.buses)
    assert call([live], bad) == -1
    bad = rec.copy(); bad["in_service"] = 0
    assert call([live], bad) == -1
    bad = rec.copy(); bad["phases"] = 7 if int(bad["phases"][0]) != 7 else 1
    assert call([live], bad) == -1
    bad = rec.copy(); bad["p_lo"] = 1.0; bad["p_hi"] = 0.0
    assert call([live], bad) == -1
    if len(dead):
        assert call([int(dead[0])], f.lines[[int(dead[0])]]) == -1
    assert call([len(f.lines)], rec) == -1


def test_component_operator_inconsistent_rows(opf):
    """Rows that contradict each other (x0 + x1 = 1 and 2 x0 + 2 x1 = 3)
    are refused with OPF_ERR_INCONSISTENT through the C ABI: the row
    reduction of Section IV-B meets 0 = b, b != 0.  The physical model's
    rows are always consistent, so this is the way to reach that status."""
    A = np.array([[1.0, 1.0, 0.0], [2.0, 2.0, 0.0]])
    for b, ok in (([1.0, 3.0], False), ([1.0, 2.0], True)):
        b = np.array(b)
        P = np.empty((3, 3)); bb = np.empty(3); mr = C.c_int32()
        st = opf.lib.opf_component_operator(A.ctypes.data_as(opf._D), b.ctypes.data_as(opf._D), 2, 3,
                                            P.ctypes.data_as(opf._D), bb.ctypes.data_as(opf._D), C.byref(mr))
        if ok:
            assert st == 0 and mr.value == 1
            # the minimum-norm solution of x0 + x1 = 1 and the projector onto its null space
            np.testing.assert_allclose(bb, [0.5, 0.5, 0.0], atol=1e-15)
            np.testing.assert_allclose(P, [[0.5, -0.5, 0.0], [-0.5, 0.5, 0.0], [0.0, 0.0, 1.0]], atol=1e-15)
        else:
            assert st == -2, st
            assert "no common solution" in opf.lib.opf_last_error().decode()
    # a zero row with a nonzero right-hand side
    A = np.zeros((1, 2)); b = np.array([1.0])
    assert opf.lib.opf_component_operator(A.ctypes.data_as(opf._D), b.ctypes.data_as(opf._D), 1, 2,
                                          None, None, None) == -2
    # non-finite entries and bad sizes
    A = np.array([[np.nan, 1.0]]); b = np.array([0.0])
    assert opf.lib.opf_component_operator(A.ctypes.data_as(opf._D), b.ctypes.data_as(opf._D), 1, 2,
                                          None, None, None) == -1
    assert opf.lib.opf_component_operator(None, None, 0, 0, None, None, None) == -1


def test_component_operator_matches_oracle_row_reduction(opf):
    """Random rank-deficient but consistent systems: the library's QR
    precompute agrees with the oracle's row reduction + Cholesky (ranks,
    projectors, minimum-norm bbar); m = 0 gives P = I, bbar = 0."""
    from oracle import precompute as OP
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(2, 30))
        r = int(rng.integers(1, n))
        m = int(rng.integers(r, r + 5))
        A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))     # rank r
        b = A @ rng.standard_normal(n)                                    # consistent
        P, bb, mr = opf.component_operator(A, b)
        Ar, br, piv = OP.rref(A, b)
        Abar, bbar = OP.closed_form(Ar, br)
        assert mr == Ar.shape[0] == r
        np.testing.assert_allclose(P, -Abar, atol=1e-9)
        np.testing.assert_allclose(bb, bbar, atol=1e-9 * max(1.0, np.abs(bbar).max()))
    P, bb, mr = opf.component_operator(np.zeros((0, 4)), np.zeros(0))
    assert mr == 0 and np.array_equal(P, np.eye(4)) and np.array_equal(bb, np.zeros(4))


@pytest.mark.parametrize("decomp", ["fine", "paper"])
def test_set_line_status_host_rebuild(opf, decomp):
    """opf_set_line_status on a problem that is not uploaded: the rebuilt
    host problem equals one created from the new records (structure and
    operators bit for bit); only the components whose rows changed are
    re-precomputed, counted independently from the oracle's models; and
    switching back restores the original problem."""
    from oracle import model as OM
    d = opf.DECOMP_PAPER if decomp == "paper" else opf.DECOMP_FINE
    f = F.feeder_123(1)
    rng = np.random.default_rng(3)
    g = F.reconfigure(f, rng)
    changed = np.flatnonzero(g.lines["in_service"] != f.lines["in_service"])
    assert len(changed) == 2
    p = opf.Problem.from_feeder(f, upload=False, decomposition=d)
    base = [p.operator(s) for s in range(p.dims.n_comp)]
    cur = f.copy()
    for e in changed:
        old_m = OM.build_feeder(cur, decomp)
        cur.lines["in_service"][e] = g.lines["in_service"][e]
        new_m = OM.build_feeder(cur, decomp)
        before = {(c.kind, c.index): c for c in old_m.comps}
        touched = sum(1 for c in new_m.comps
                      if (c.kind, c.index) not in before
                      or not (np.array_equal(before[c.kind, c.index].A, c.A)
                              and np.array_equal(before[c.kind, c.index].b, c.b)))
        n = p.set_line_status(int(e), bool(g.lines["in_service"][e]))
        assert n == touched and 1 <= n <= 6, (n, touched)
        q = opf.Problem.from_feeder(cur, upload=False, decomposition=d)
        sp, sq = p.structure(), q.structure()
        for k in sp:
            assert np.array_equal(sp[k], sq[k]), k
        assert p.dims.n_global == q.dims.n_global and p.dims.n_blocks == q.dims.n_blocks
        for s in range(q.dims.n_comp):
            a, b = p.operator(s), q.operator(s)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        q.close()
    assert p.set_line_status(int(changed[0]), bool(g.lines["in_service"][changed[0]])) == 0   # no change
    for e in changed[::-1]:
        p.set_line_status(int(e), bool(f.lines["in_service"][e]))
    assert p.dims.n_comp == len(base)
    for s in range(p.dims.n_comp):
        a = p.operator(s)
        assert np.array_equal(a[0], base[s][0]) and np.array_equal(a[1], base[s][1])
    with pytest.raises(opf.OpfError):
        p.set_line_status(len(f.lines), True)
    p.close()


def test_tuning_table(opf, tmp_path):
    """Automatic chunking reads the tuning table: an entry for every GPU
    ("*") and a bus-count bucket sets the chunk size and cap; entries for
    another GPU name do not apply here (no device: empty name); a JSON file
    in the tuner's format loads (extra keys ignored); malformed files and
    out-of-range values are refused."""
    opf.tuning_clear()
    try:
        assert opf.tuning_lookup(150) == (4096, 296)
        from paper_2501_08293_b300 import autotune
        f = autotune.representative(150, 3)
        p0 = opf.Problem.from_feeder(f, upload=False)
        opf.tuning_set("*", 100, 200, 256, 7)
        assert opf.tuning_lookup(150) == (256, 7) and opf.tuning_lookup(99) == (4096, 296)
        p1 = opf.Problem.from_feeder(f, upload=False)
        ns = np.diff(p1.structure()["comp_ptr"]).astype(np.int64)
        total = int(np.sum(ns * ns + 4 * ns + 16))
        assert p1.dims.n_blocks == min(7, total // 256) and p1.dims.n_blocks != p0.dims.n_blocks
        for x, y in zip(p0.structure().values(), p1.structure().values()):
            assert np.array_equal(x, y)          # same problem, other chunking
        opf.tuning_set("Some Other GPU", 0, 1000, 512, 3)
        opf.tuning_clear()
        opf.tuning_set("Some Other GPU", 0, 1000, 512, 3)
        assert opf.tuning_lookup(150) == (4096, 296)
        path = tmp_path / "t.json"
        path.write_text('{"gpu": "*", "precision": "fp32", "entries": [{"n_bus_lo": 1, "n_bus_hi": 60, '
                        '"work_per_chunk": 1024, "max_chunks": 296, "us_per_iter": 1.5, "candidates": {"256": {}}},'
                        ' {"n_bus_lo": 60, "n_bus_hi": 200, "work_per_chunk": 2048, "max_chunks": 100}]}')
        assert opf.tuning_load(str(path)) == 2
        assert opf.tuning_lookup(30) == (1024, 296) and opf.tuning_lookup(150) == (2048, 100)
        for bad in ('{"gpu": "*", "entries": [{"n_bus_lo": 5, "n_bus_hi": 1, "work_per_chunk": 64, "max_chunks": 1}]}',
                    '{"gpu": "*", "entries": [{"n_bus_lo": 1}]}', '{"gpu": "*", "entries": [', '[1, 2]'):
            path.write_text(bad)
            with pytest.raises(opf.OpfError):
                opf.tuning_load(str(path))
        with pytest.raises(opf.OpfError):
            opf.tuning_set("*", 0, 10, 8, 1)
    finally:
        opf.tuning_clear()
        if os.path.exists(opf._TUNING_PATH):
            opf.tuning_load(opf._TUNING_PATH)
