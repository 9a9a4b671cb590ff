"""Linearized multi-phase OPF model and its componentwise decomposition.

Follows Section II of the paper:

* Eq. (operational): bounds on pg, qg, w and line flows -- these are the only
  inequalities, and after the reformulation of Eq. (OurModel) they live on
  the global variable vector only.
* Eq. (balance_eqns): per bus and phase, outgoing line flows + load
  withdrawals pb/qb + shunt terms = generation.
* Eq. (volt_load_model): VDLM-1..4 (voltage-dependent load), VDLM-5 (wye),
  VDLM-6..10 (three-phase delta).
* Eq. (power_flow_eqns): powerloss-1/2 and voltage_mag_diff with M^p, M^q.
* Eq. (LP_model): the global variable order [gens; w; loads; lines].
* Eq. (OurModel) with the fine decomposition the hot path uses by default:
  one component per bus, in-service line, load and generator; or the
  paper's decomposition of Section V-A ("paper"): one component per node of
  the feeder graph (a bus together with its loads and generators) and one
  per line, except that a leaf node is combined with the line that connects
  it, so S = nodes + lines - leaves (Table III).

Readings where the paper is silent: M^p/M^q of a line with fewer than three
phases is the sub-block on its phases; delta loads must be three-phase (the
paper writes VDLM-7..10 for phases 1, 2, 3 only); a variable counts as
bounded only when both bounds are finite.  Paper decomposition: a leaf is a
bus with exactly one in-service line (graph degree one, the substation bus
included when it has one line); when both ends of a line are leaves both
are combined with it; a bus with no in-service line stays a node.

Canonical orders (shared by contract with the library's state export):

* globals: gens k: pg(phases), qg(phases); buses i: w(phases);
  loads l: pb, qb, pd, qd (each over phases); in-service lines e:
  p_ij, q_ij, p_ji, q_ji (each over phases).
* components: buses, in-service lines, loads, generators (input order).
  Paper decomposition: nodes that are not leaves (bus order), then
  in-service lines (line order), each combined with its leaf end(s).
* bus i locals: w(P_i); for each in-service line touching i, in line order,
  the flow leaving i: p(P_e), q(P_e); loads at i: pb(P_l), qb(P_l);
  generators at i: pg(P_k), qg(P_k).
* line locals: p_ij, q_ij, p_ji, q_ji (each over P_e), w_i(P_e), w_j(P_e).
* load locals: pb, qb, pd, qd (each over P_l), w_i(P_l).
* generator locals: pg(P_k), qg(P_k).
* paper decomposition, combined parts: the locals of the parts concatenated
  (node: bus, then its loads in load order, then its generators; line with
  leaves: line, then the from-end node if a leaf, then the to-end node if a
  leaf) keeping the first copy of a global that appears twice; rows of the
  parts stacked in the same order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SQRT3 = math.sqrt(3.0)
KIND_BUS, KIND_LINE, KIND_LOAD, KIND_GEN = 0, 1, 2, 3
VAR_OTHER, VAR_W = 0, 1


class ModelError(ValueError):
    """Invalid feeder data (the library answers OPF_ERR_INVALID_ARG)."""


def phase_list(mask: int) -> list[int]:
    return [p for p in range(3) if (int(mask) >> p) & 1]


def m_matrices(r: np.ndarray, x: np.ndarray, ph: list[int]):
    """M^p and M^q of Section II-A (3x3, phases a, b, c), restricted to ph."""
    r = np.asarray(r, dtype=np.float64).reshape(3, 3)
    x = np.asarray(x, dtype=np.float64).reshape(3, 3)
    mp = np.array([
        [-2 * r[0, 0], r[0, 1] - SQRT3 * x[0, 1], r[0, 2] + SQRT3 * x[0, 2]],
        [r[1, 0] + SQRT3 * x[1, 0], -2 * r[1, 1], r[1, 2] - SQRT3 * x[1, 2]],
        [r[2, 0] - SQRT3 * x[2, 0], r[2, 1] + SQRT3 * x[2, 1], -2 * r[2, 2]],
    ])
    mq = np.array([
        [-2 * x[0, 0], x[0, 1] + SQRT3 * r[0, 1], x[0, 2] - SQRT3 * r[0, 2]],
        [x[1, 0] - SQRT3 * r[1, 0], -2 * x[1, 1], x[1, 2] + SQRT3 * r[1, 2]],
        [x[2, 0] + SQRT3 * r[2, 0], x[2, 1] - SQRT3 * r[2, 1], -2 * x[2, 2]],
    ])
    idx = np.ix_(ph, ph)
    return mp[idx], mq[idx]


@dataclasses.dataclass
class Component:
    kind: int                 # KIND_*
    index: int                # bus / line / load / generator index in the input
    gvars: np.ndarray         # global index of each local variable (B_s as a map)
    A: np.ndarray             # m_s x n_s equality rows (before row reduction)
    b: np.ndarray             # m_s


@dataclasses.dataclass
class Model:
    n: int                    # number of global variables
    lo: np.ndarray
    hi: np.ndarray
    c: np.ndarray
    vtype: np.ndarray         # VAR_W for squared voltage magnitudes
    names: list
    comps: list               # list[Component], canonical order
    gidx: dict                # lookup tables of global indices

    @property
    def S(self) -> int:
        return len(self.comps)

    @property
    def nl(self) -> int:
        return int(sum(len(c.gvars) for c in self.comps))


def _validate(buses, lines, gens, loads):
    nb = len(buses)
    if nb == 0:
        raise ModelError("no buses")
    for i, bus in enumerate(buses):
        if not (0 < int(bus["phases"]) < 8):
            raise ModelError(f"bus {i}: bad phase mask")
    for e, ln in enumerate(lines):
        f, t = int(ln["from_bus"]), int(ln["to_bus"])
        if not (0 <= f < nb and 0 <= t < nb) or f == t:
            raise ModelError(f"line {e}: bad ends")
        pm = int(ln["phases"])
        if not (0 < pm < 8) or (pm & ~int(buses[f]["phases"])) or (pm & ~int(buses[t]["phases"])):
            raise ModelError(f"line {e}: phases not on both buses")
    for k, g in enumerate(gens):
        bi = int(g["bus"])
        if not (0 <= bi < nb) or not (0 < int(g["phases"]) < 8) or (int(g["phases"]) & ~int(buses[bi]["phases"])):
            raise ModelError(f"gen {k}: bad bus/phases")
    for l, d in enumerate(loads):
        bi = int(d["bus"])
        if not (0 <= bi < nb) or not (0 < int(d["phases"]) < 8) or (int(d["phases"]) & ~int(buses[bi]["phases"])):
            raise ModelError(f"load {l}: bad bus/phases")
        if int(d["conn"]) not in (0, 1):
            raise ModelError(f"load {l}: bad connection")
        if int(d["conn"]) == 1 and int(d["phases"]) != 7:
            raise ModelError(f"load {l}: delta loads must be three-phase")


def build(buses, lines, gens, loads) -> Model:
    """Global variables (Eq. LP_model) and fine components (Eq. OurModel)."""
    _validate(buses, lines, gens, loads)
    lo, hi, c, vt, names = [], [], [], [], []

    def new(name, l, h, cost=0.0, t=VAR_OTHER):
        lo.append(float(l)); hi.append(float(h)); c.append(float(cost))
        vt.append(t); names.append(name)
        return len(lo) - 1

    g_pg, g_qg = {}, {}
    for k, g in enumerate(gens):
        for p in phase_list(g["phases"]):
            g_pg[k, p] = new(("pg", k, p), g["pg_lo"][p], g["pg_hi"][p], g["cost"][p])
        for p in phase_list(g["phases"]):
            g_qg[k, p] = new(("qg", k, p), g["qg_lo"][p], g["qg_hi"][p])
    g_w = {}
    for i, bus in enumerate(buses):
        for p in phase_list(bus["phases"]):
            g_w[i, p] = new(("w", i, p), bus["w_lo"][p], bus["w_hi"][p], t=VAR_W)
    g_pb, g_qb, g_pd, g_qd = {}, {}, {}, {}
    for l, d in enumerate(loads):
        for tab, nm in ((g_pb, "pb"), (g_qb, "qb"), (g_pd, "pd"), (g_qd, "qd")):
            for p in phase_list(d["phases"]):
                tab[l, p] = new((nm, l, p), -np.inf, np.inf)
    live = [e for e in range(len(lines)) if int(lines[e]["in_service"]) != 0]
    g_pij, g_qij, g_pji, g_qji = {}, {}, {}, {}
    for e in live:
        ln = lines[e]
        for tab, nm, lk, hk in ((g_pij, "p_ij", "p_lo", "p_hi"), (g_qij, "q_ij", "q_lo", "q_hi"),
                                (g_pji, "p_ji", "p_lo", "p_hi"), (g_qji, "q_ji", "q_lo", "q_hi")):
            for p in phase_list(ln["phases"]):
                tab[e, p] = new((nm, e, p), ln[lk][p], ln[hk][p])

    comps = []
    # --- bus components: Eq. (balance_eqns) ---------------------------------
    lines_at = [[] for _ in range(len(buses))]
    for e in live:
        lines_at[int(lines[e]["from_bus"])].append(e)
        lines_at[int(lines[e]["to_bus"])].append(e)
    loads_at = [[] for _ in range(len(buses))]
    for l, d in enumerate(loads):
        loads_at[int(d["bus"])].append(l)
    gens_at = [[] for _ in range(len(buses))]
    for k, g in enumerate(gens):
        gens_at[int(g["bus"])].append(k)
    for i, bus in enumerate(buses):
        ph = phase_list(bus["phases"])
        gv = [g_w[i, p] for p in ph]
        for e in sorted(lines_at[i]):
            lp = phase_list(lines[e]["phases"])
            if int(lines[e]["from_bus"]) == i:
                gv += [g_pij[e, p] for p in lp] + [g_qij[e, p] for p in lp]
            else:
                gv += [g_pji[e, p] for p in lp] + [g_qji[e, p] for p in lp]
        for l in loads_at[i]:
            lp = phase_list(loads[l]["phases"])
            gv += [g_pb[l, p] for p in lp] + [g_qb[l, p] for p in lp]
        for k in gens_at[i]:
            kp = phase_list(gens[k]["phases"])
            gv += [g_pg[k, p] for p in kp] + [g_qg[k, p] for p in kp]
        col = {g: j for j, g in enumerate(gv)}
        rows, rhs = [], []
        for p in ph:
            # real:  sum_e p_e + sum_l pb + gsh*w - sum_k pg = 0
            a = np.zeros(len(gv))
            for e in lines_at[i]:
                if p in phase_list(lines[e]["phases"]):
                    a[col[g_pij[e, p] if int(lines[e]["from_bus"]) == i else g_pji[e, p]]] += 1.0
            for l in loads_at[i]:
                if p in phase_list(loads[l]["phases"]):
                    a[col[g_pb[l, p]]] += 1.0
            a[col[g_w[i, p]]] += float(bus["g_sh"][p])
            for k in gens_at[i]:
                if p in phase_list(gens[k]["phases"]):
                    a[col[g_pg[k, p]]] -= 1.0
            rows.append(a); rhs.append(0.0)
            # reactive:  sum_e q_e + sum_l qb - bsh*w - sum_k qg = 0
            a = np.zeros(len(gv))
            for e in lines_at[i]:
                if p in phase_list(lines[e]["phases"]):
                    a[col[g_qij[e, p] if int(lines[e]["from_bus"]) == i else g_qji[e, p]]] += 1.0
            for l in loads_at[i]:
                if p in phase_list(loads[l]["phases"]):
                    a[col[g_qb[l, p]]] += 1.0
            a[col[g_w[i, p]]] -= float(bus["b_sh"][p])
            for k in gens_at[i]:
                if p in phase_list(gens[k]["phases"]):
                    a[col[g_qg[k, p]]] -= 1.0
            rows.append(a); rhs.append(0.0)
        comps.append(Component(KIND_BUS, i, np.array(gv, dtype=np.int64),
                               np.array(rows).reshape(len(rows), len(gv)), np.array(rhs)))
    # --- line components: Eq. (power_flow_eqns) -----------------------------
    for e in live:
        ln = lines[e]
        i, j = int(ln["from_bus"]), int(ln["to_bus"])
        ph = phase_list(ln["phases"])
        gv = ([g_pij[e, p] for p in ph] + [g_qij[e, p] for p in ph] +
              [g_pji[e, p] for p in ph] + [g_qji[e, p] for p in ph] +
              [g_w[i, p] for p in ph] + [g_w[j, p] for p in ph])
        col = {g: jj for jj, g in enumerate(gv)}
        mp, mq = m_matrices(ln["r"], ln["x"], ph)
        rows = []
        for a_, p in enumerate(ph):
            # powerloss-1: p_ij + p_ji - gs_ij w_i - gs_ji w_j = 0
            a = np.zeros(len(gv))
            a[col[g_pij[e, p]]] += 1.0
            a[col[g_pji[e, p]]] += 1.0
            a[col[g_w[i, p]]] -= float(ln["g_fr"][p])
            a[col[g_w[j, p]]] -= float(ln["g_to"][p])
            rows.append(a)
            # powerloss-2: q_ij + q_ji + bs_ij w_i + bs_ji w_j = 0
            a = np.zeros(len(gv))
            a[col[g_qij[e, p]]] += 1.0
            a[col[g_qji[e, p]]] += 1.0
            a[col[g_w[i, p]]] += float(ln["b_fr"][p])
            a[col[g_w[j, p]]] += float(ln["b_to"][p])
            rows.append(a)
            # voltage_mag_diff:
            # w_i - tau w_j + sum_psi Mp (p_ij - gs_ij w_i) + Mq (q_ij + bs_ij w_i) = 0
            a = np.zeros(len(gv))
            a[col[g_w[i, p]]] += 1.0
            a[col[g_w[j, p]]] -= float(ln["tap"][p])
            for b_, s in enumerate(ph):
                a[col[g_pij[e, s]]] += mp[a_, b_]
                a[col[g_w[i, s]]] -= mp[a_, b_] * float(ln["g_fr"][s])
                a[col[g_qij[e, s]]] += mq[a_, b_]
                a[col[g_w[i, s]]] += mq[a_, b_] * float(ln["b_fr"][s])
            rows.append(a)
        comps.append(Component(KIND_LINE, e, np.array(gv, dtype=np.int64),
                               np.array(rows), np.zeros(len(rows))))
    # --- load components: Eq. (volt_load_model) -----------------------------
    for l, d in enumerate(loads):
        i = int(d["bus"])
        ph = phase_list(d["phases"])
        gv = ([g_pb[l, p] for p in ph] + [g_qb[l, p] for p in ph] +
              [g_pd[l, p] for p in ph] + [g_qd[l, p] for p in ph] +
              [g_w[i, p] for p in ph])
        col = {g: jj for jj, g in enumerate(gv)}
        delta = int(d["conn"]) == 1
        wmul = 3.0 if delta else 1.0          # VDLM-4 / VDLM-3
        rows, rhs = [], []
        for p in ph:
            a_, al = float(d["a"][p]), float(d["alpha"][p])
            b_, be = float(d["b"][p]), float(d["beta"][p])
            # VDLM-1: pd = (a alpha / 2)(what - 1) + a
            r = np.zeros(len(gv))
            r[col[g_pd[l, p]]] = 1.0
            r[col[g_w[i, p]]] -= 0.5 * a_ * al * wmul
            rows.append(r); rhs.append(a_ - 0.5 * a_ * al)
            # VDLM-2: qd = (b beta / 2)(what - 1) + b
            r = np.zeros(len(gv))
            r[col[g_qd[l, p]]] = 1.0
            r[col[g_w[i, p]]] -= 0.5 * b_ * be * wmul
            rows.append(r); rhs.append(b_ - 0.5 * b_ * be)
        if not delta:
            for p in ph:            # VDLM-5
                r = np.zeros(len(gv)); r[col[g_pb[l, p]]] = 1.0; r[col[g_pd[l, p]]] = -1.0
                rows.append(r); rhs.append(0.0)
                r = np.zeros(len(gv)); r[col[g_qb[l, p]]] = 1.0; r[col[g_qd[l, p]]] = -1.0
                rows.append(r); rhs.append(0.0)
        else:
            def lin(terms):
                r = np.zeros(len(gv))
                for coef, tab, p in terms:
                    r[col[tab[l, p]]] += coef
                return r
            h = 0.5 * SQRT3
            # VDLM-6
            rows.append(lin([(1, g_pb, p) for p in range(3)] + [(-1, g_pd, p) for p in range(3)])); rhs.append(0.0)
            rows.append(lin([(1, g_qb, p) for p in range(3)] + [(-1, g_qd, p) for p in range(3)])); rhs.append(0.0)
            # VDLM-7: 3/2 pb2 - r3/2 qb2 = pd2 + 1/2 pd1 - r3/2 qd1
            rows.append(lin([(1.5, g_pb, 1), (-h, g_qb, 1), (-1, g_pd, 1), (-0.5, g_pd, 0), (h, g_qd, 0)])); rhs.append(0.0)
            # VDLM-8: r3/2 pb2 + 3/2 qb2 = r3/2 pd1 + 1/2 qd1 + qd2
            rows.append(lin([(h, g_pb, 1), (1.5, g_qb, 1), (-h, g_pd, 0), (-0.5, g_qd, 0), (-1, g_qd, 1)])); rhs.append(0.0)
            # VDLM-9: r3 qb2 + 3/2 pb3 - r3/2 qb3 = 1/2 pd1 + r3/2 qd1 + pd3
            rows.append(lin([(SQRT3, g_qb, 1), (1.5, g_pb, 2), (-h, g_qb, 2), (-0.5, g_pd, 0), (-h, g_qd, 0), (-1, g_pd, 2)])); rhs.append(0.0)
            # VDLM-10: -r3 pb2 + r3/2 pb3 + 3/2 qb3 = -r3/2 pd1 + 1/2 qd1 + qd3
            rows.append(lin([(-SQRT3, g_pb, 1), (h, g_pb, 2), (1.5, g_qb, 2), (h, g_pd, 0), (-0.5, g_qd, 0), (-1, g_qd, 2)])); rhs.append(0.0)
        comps.append(Component(KIND_LOAD, l, np.array(gv, dtype=np.int64),
                               np.array(rows), np.array(rhs)))
    # --- generator components: no equality rows -----------------------------
    for k, g in enumerate(gens):
        kp = phase_list(g["phases"])
        gv = [g_pg[k, p] for p in kp] + [g_qg[k, p] for p in kp]
        comps.append(Component(KIND_GEN, k, np.array(gv, dtype=np.int64),
                               np.zeros((0, len(gv))), np.zeros(0)))
    tables = dict(pg=g_pg, qg=g_qg, w=g_w, pb=g_pb, qb=g_qb, pd=g_pd, qd=g_qd,
                  p_ij=g_pij, q_ij=g_qij, p_ji=g_pji, q_ji=g_qji)
    return Model(len(lo), np.array(lo), np.array(hi), np.array(c), np.array(vt),
                 names, comps, tables)


def combine(kind: int, index: int, parts) -> Component:
    """One component from several (Section V-A): the union of their local
    variables (first occurrence kept, so a global shared by two parts gets
    one local copy) and all of their rows, stacked in order."""
    gv = []
    seen = {}
    for c in parts:
        for g in c.gvars:
            if int(g) not in seen:
                seen[int(g)] = len(gv)
                gv.append(int(g))
    rows, rhs = [], []
    for c in parts:
        for a in range(c.A.shape[0]):
            r = np.zeros(len(gv))
            for j, g in enumerate(c.gvars):
                r[seen[int(g)]] += c.A[a, j]
            rows.append(r)
            rhs.append(c.b[a])
    A = np.array(rows).reshape(len(rows), len(gv))
    return Component(kind, index, np.array(gv, dtype=np.int64), A, np.array(rhs, dtype=np.float64))


def paper_decomposition(model: Model, buses, lines, gens, loads) -> Model:
    """Components of Section V-A from the fine ones: node = bus + its loads
    + its generators; a leaf node (one in-service line) is combined with
    that line; S = nodes + lines - leaves."""
    fine = {(c.kind, c.index): c for c in model.comps}
    nb = len(buses)
    live = [e for e in range(len(lines)) if int(lines[e]["in_service"]) != 0]
    degree = [0] * nb
    for e in live:
        degree[int(lines[e]["from_bus"])] += 1
        degree[int(lines[e]["to_bus"])] += 1
    node = {}
    for i in range(nb):
        parts = [fine[KIND_BUS, i]]
        parts += [fine[KIND_LOAD, l] for l in range(len(loads)) if int(loads[l]["bus"]) == i]
        parts += [fine[KIND_GEN, k] for k in range(len(gens)) if int(gens[k]["bus"]) == i]
        node[i] = combine(KIND_BUS, i, parts)
    leaf = [degree[i] == 1 for i in range(nb)]
    comps = [node[i] for i in range(nb) if not leaf[i]]
    for e in live:
        i, j = int(lines[e]["from_bus"]), int(lines[e]["to_bus"])
        parts = [fine[KIND_LINE, e]] + ([node[i]] if leaf[i] else []) + ([node[j]] if leaf[j] else [])
        comps.append(combine(KIND_LINE, e, parts))
    return dataclasses.replace(model, comps=comps)


def build_feeder(f, decomposition: str = "fine") -> Model:
    m = build(f.buses, f.lines, f.gens, f.loads)
    if decomposition == "paper":
        return paper_decomposition(m, f.buses, f.lines, f.gens, f.loads)
    if decomposition != "fine":
        raise ValueError(decomposition)
    return m


def stacked_A(model: Model):
    """Centralized rows A x = b of Eq. (LP_model): each component's rows
    mapped to global columns (A_s B_s)."""
    import scipy.sparse as sp
    ri, ci, vv, bb = [], [], [], []
    r0 = 0
    for comp in model.comps:
        m = comp.A.shape[0]
        for a in range(m):
            for j in range(comp.A.shape[1]):
                if comp.A[a, j] != 0.0:
                    ri.append(r0 + a); ci.append(int(comp.gvars[j])); vv.append(comp.A[a, j])
        bb.extend(comp.b.tolist())
        r0 += m
    A = sp.csr_matrix((vv, (ri, ci)), shape=(r0, model.n))
    return A, np.array(bb)
