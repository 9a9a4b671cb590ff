"""Seeded synthetic radial distribution feeders (input data only).

The IEEE 13/123/8500-bus test feeders used in the paper's experiments
(Section V-A, Tables II-IV) are not available, so every workload here is a
seeded synthetic feeder shaped like them: a radial tree with a three-phase
backbone and two- and single-phase laterals, 3x3 line impedances, wye and
delta loads of constant power / current / impedance type, PV inverters and
one substation source.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.
It holds no arithmetic of the ADMM method or of the OPF model: it only
draws feeder data (topology, impedances, loads, bounds) and packs it into
numpy structured arrays whose layout is the C ABI's record layout
(``opf_bus``, ``opf_line``, ``opf_gen``, ``opf_load`` in ``include/opf_admm.h``).

Phase sets are bit masks: phase a = 1, b = 2, c = 4.  Per-phase arrays are
indexed by phase 0..2 (a, b, c); entries of absent phases are ignored.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "BUS_DTYPE", "LINE_DTYPE", "GEN_DTYPE", "LOAD_DTYPE", "Feeder",
    "phases_of", "make_feeder", "feeder_13", "feeder_123", "feeder_8500",
    "feeder_tiny", "feeder_batch", "CONFIG_FEEDERS",
]

# Record layouts.  Field order, padding and sizes match include/opf_admm.h
# (104, 376, 128 and 104 bytes); tests check them against the library.
BUS_DTYPE = np.dtype([
    ("phases", "u1"), ("_pad", "u1", 7),
    ("w_lo", "f8", 3), ("w_hi", "f8", 3),
    ("g_sh", "f8", 3), ("b_sh", "f8", 3),
], align=True)

LINE_DTYPE = np.dtype([
    ("from_bus", "i4"), ("to_bus", "i4"),
    ("phases", "u1"), ("in_service", "u1"), ("_pad", "u1", 6),
    ("r", "f8", 9), ("x", "f8", 9),
    ("g_fr", "f8", 3), ("b_fr", "f8", 3), ("g_to", "f8", 3), ("b_to", "f8", 3),
    ("tap", "f8", 3),
    ("p_lo", "f8", 3), ("p_hi", "f8", 3), ("q_lo", "f8", 3), ("q_hi", "f8", 3),
], align=True)

GEN_DTYPE = np.dtype([
    ("bus", "i4"), ("phases", "u1"), ("_pad", "u1", 3),
    ("pg_lo", "f8", 3), ("pg_hi", "f8", 3),
    ("qg_lo", "f8", 3), ("qg_hi", "f8", 3),
    ("cost", "f8", 3),
], align=True)

LOAD_DTYPE = np.dtype([
    ("bus", "i4"), ("phases", "u1"), ("conn", "u1"), ("_pad", "u1", 2),
    ("a", "f8", 3), ("b", "f8", 3), ("alpha", "f8", 3), ("beta", "f8", 3),
], align=True)

assert BUS_DTYPE.itemsize == 104 and LINE_DTYPE.itemsize == 376
assert GEN_DTYPE.itemsize == 128 and LOAD_DTYPE.itemsize == 104

WYE, DELTA = 0, 1


def phases_of(mask: int) -> list[int]:
    """Phase indices (0=a, 1=b, 2=c) present in a bit mask, ascending."""
    return [p for p in range(3) if (int(mask) >> p) & 1]


@dataclasses.dataclass
class Feeder:
    """One feeder as four record arrays plus the generator's bookkeeping."""
    buses: np.ndarray
    lines: np.ndarray
    gens: np.ndarray
    loads: np.ndarray
    name: str = "feeder"
    seed: int = 0
    load_scale: float = 1.0
    parent: np.ndarray | None = None       # parent bus of each bus (-1 at root)
    switches: np.ndarray | None = None     # line indices that carry a switch

    @property
    def n_bus(self) -> int:
        return len(self.buses)

    def copy(self) -> "Feeder":
        return Feeder(self.buses.copy(), self.lines.copy(), self.gens.copy(),
                      self.loads.copy(), self.name, self.seed, self.load_scale,
                      None if self.parent is None else self.parent.copy(),
                      None if self.switches is None else self.switches.copy())

    def stats(self) -> dict:
        ph = np.array([bin(int(m)).count("1") for m in self.lines["phases"]])
        ins = self.lines["in_service"] == 1
        return {
            "buses": self.n_bus, "lines": int(ins.sum()),
            "lines_1ph": int(((ph == 1) & ins).sum()),
            "lines_2ph": int(((ph == 2) & ins).sum()),
            "lines_3ph": int(((ph == 3) & ins).sum()),
            "gens": len(self.gens), "loads": len(self.loads),
            "delta_loads": int((self.loads["conn"] == DELTA).sum()),
            "load_scale": self.load_scale,
        }


_PHASE_SUBSETS = {
    7: {3: [7], 2: [3, 5, 6], 1: [1, 2, 4]},
    3: {2: [3], 1: [1, 2]},
    5: {2: [5], 1: [1, 4]},
    6: {2: [6], 1: [2, 4]},
    1: {1: [1]}, 2: {1: [2]}, 4: {1: [4]},
}


def _impedance(rng, length_km, z_base):
    """Symmetric 3x3 R, X in per unit: self U[0.3,0.6], mutual U[0.1,0.3] ohm/km."""
    r = np.empty((3, 3))
    x = np.empty((3, 3))
    for m in (r, x):
        for i in range(3):
            m[i, i] = rng.uniform(0.3, 0.6)
            for j in range(i + 1, 3):
                m[i, j] = m[j, i] = rng.uniform(0.1, 0.3)
    return r * length_km / z_base, x * length_km / z_base


def make_feeder(n_bus: int, seed: int, *, n_loads: int, load_sampler,
                n_pv: int = 0, pv_pmax=(0.02, 0.2), n_switches: int = 0,
                line_mix=(0.34, 0.33, 0.33), v_ll_kv: float = 4.16,
                s_base_mva: float = 1.0, delta_prob: float = 0.3,
                lateral_mean: float = 4.0, shunts: bool = True,
                taps: bool = False, source_limit: float | None = None,
                drop_budget: float = 0.4, line_len=(0.1, 1.0),
                chain_prob: float = 0.6, name: str = "feeder") -> Feeder:
    """Grow a seeded radial feeder.

    * A three-phase backbone of about ``line_mix[2] * n_bus`` buses; two- and
      single-phase laterals (geometric length, mean ``lateral_mean``) hang
      off earlier buses.  A child's phases are a subset of its parent's.
    * Lines ``line_len`` km (default 0.1-1); R, X symmetric 3x3 (self 0.3-0.6, mutual 0.1-0.3
      ohm/km) converted to per unit with Z_base = V_LL^2 / S_base.
    * Loads on random non-root buses: delta with probability ``delta_prob``
      when three-phase, else wye; type alpha = beta in {0, 1, 2} (constant
      power / current / impedance); P from ``load_sampler``, Q = 0.3 P,
      split evenly over the load's phases.
    * PV inverters: pg in [0, pmax], |qg| <= 0.44 pmax, pmax ~ U(pv_pmax).
    * Bounds: w in [0.81, 1.21] (root fixed at 1.0); flows within
      +-(1.5 x a downstream demand proxy + 0.1) per phase.
    * Switches: ``n_switches`` lines carry a switch; half of them are open
      tie lines that would close a loop, half are closed tree lines.
    * Load level: all loads are scaled by 0.9 until a worst-case
      impedance x downstream-demand sum along every root path (absolute
      3x3 row sums times a per-phase demand proxy, several times the actual
      drop) stays within ``drop_budget``; the factor is kept in
      ``Feeder.load_scale``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    z_base = v_ll_kv ** 2 / s_base_mva
    w1, w2, w3 = line_mix
    tot = w1 + w2 + w3
    n_bb = max(2, int(round(n_bus * w3 / tot)))
    parent = np.full(n_bus, -1, dtype=np.int64)
    phases = np.zeros(n_bus, dtype=np.int64)
    phases[0] = 7
    # Three-phase backbone: random recursive tree biased toward chains.
    for i in range(1, min(n_bb, n_bus)):
        if rng.random() < chain_prob:
            p = i - 1
        else:
            p = int(rng.integers(max(0, i - 40), i))
        parent[i] = p
        phases[i] = 7
    # Laterals: the remaining buses in short chains; target phase counts
    # follow the 1/2-phase shares of line_mix.
    i = n_bb
    want2 = w2 / max(w1 + w2, 1e-12)
    while i < n_bus:
        p = int(rng.integers(0, i))
        k = 2 if (rng.random() < want2) else 1
        if bin(int(phases[p])).count("1") < k:
            k = bin(int(phases[p])).count("1")
        choices = _PHASE_SUBSETS[int(phases[p])][k]
        ph = int(choices[rng.integers(0, len(choices))])
        run = 1 + int(rng.geometric(1.0 / lateral_mean)) - 1
        run = max(1, min(run, n_bus - i))
        prev = p
        for _ in range(run):
            parent[i] = prev
            phases[i] = ph
            prev = i
            i += 1
    # Buses.
    buses = np.zeros(n_bus, dtype=BUS_DTYPE)
    buses["phases"] = phases
    buses["w_lo"] = 0.81
    buses["w_hi"] = 1.21
    buses["w_lo"][0] = 1.0
    buses["w_hi"][0] = 1.0
    if shunts:
        # A few capacitor banks (shunt susceptance) on three-phase buses.
        cap = rng.choice(np.arange(1, n_bus), size=max(1, n_bus // 200), replace=False)
        for c in cap:
            if phases[c] == 7:
                buses["b_sh"][c] = rng.uniform(0.0, 0.002)
    # Lines: tree lines first (line e connects parent[e+1] -> e+1).
    n_tree = n_bus - 1
    n_tie = n_switches // 2
    lines = np.zeros(n_tree + n_tie, dtype=LINE_DTYPE)
    for e in range(n_tree):
        j = e + 1
        ln = lines[e]
        ln["from_bus"] = parent[j]
        ln["to_bus"] = j
        ln["phases"] = phases[j]
        ln["in_service"] = 1
        r, x = _impedance(rng, rng.uniform(*line_len), z_base)
        ln["r"] = r.ravel()
        ln["x"] = x.ravel()
        if shunts:
            bc = rng.uniform(0.0, 2e-5) * 0.5
            ln["b_fr"] = bc
            ln["b_to"] = bc
        ln["tap"] = rng.uniform(0.98, 1.02) if taps else 1.0
    # Tie lines (normally open) between two same-phase buses.
    for t in range(n_tie):
        for _ in range(1000):
            a, b = rng.integers(1, n_bus, size=2)
            if a != b and phases[a] == phases[b] and parent[a] != b and parent[b] != a:
                break
        ln = lines[n_tree + t]
        ln["from_bus"] = a
        ln["to_bus"] = b
        ln["phases"] = phases[a]
        ln["in_service"] = 0
        r, x = _impedance(rng, rng.uniform(0.1, 1.0), z_base)
        ln["r"] = r.ravel()
        ln["x"] = x.ravel()
        ln["tap"] = 1.0
    sw = list(range(n_tree, n_tree + n_tie))
    if n_switches - n_tie > 0:
        sw += list(rng.choice(np.arange(1, n_tree), size=n_switches - n_tie, replace=False))
    # Loads.
    n_loads = min(n_loads, n_bus - 1)
    load_bus = np.sort(rng.choice(np.arange(1, n_bus), size=n_loads, replace=False))
    loads = np.zeros(n_loads, dtype=LOAD_DTYPE)
    for k, bidx in enumerate(load_bus):
        ph = int(phases[bidx])
        ld = loads[k]
        ld["bus"] = bidx
        ld["phases"] = ph
        ld["conn"] = DELTA if (ph == 7 and rng.random() < delta_prob) else WYE
        ty = float(rng.integers(0, 3))
        P = float(load_sampler(rng))
        pp = phases_of(ph)
        for p in pp:
            ld["a"][p] = P / len(pp)
            ld["b"][p] = 0.3 * P / len(pp)
            ld["alpha"][p] = ty
            ld["beta"][p] = ty
    # Generators: source at the root + PV inverters.
    pv_bus = rng.choice(np.arange(1, n_bus), size=min(n_pv, n_bus - 1), replace=False)
    gens = np.zeros(1 + len(pv_bus), dtype=GEN_DTYPE)
    gens[0]["bus"] = 0
    gens[0]["phases"] = 7
    gens[0]["cost"] = 1.0
    for g, bidx in enumerate(pv_bus, start=1):
        ph = int(phases[bidx])
        pmax = rng.uniform(*pv_pmax)
        gn = gens[g]
        gn["bus"] = bidx
        gn["phases"] = ph
        pp = phases_of(ph)
        for p in pp:
            gn["pg_hi"][p] = pmax / len(pp)
            gn["qg_lo"][p] = -0.44 * pmax / len(pp)
            gn["qg_hi"][p] = 0.44 * pmax / len(pp)
            gn["cost"][p] = 1.0
    # Load level and flow bounds from a demand proxy summed downstream.
    children = [[] for _ in range(n_bus)]
    for j in range(1, n_bus):
        children[parent[j]].append(j)
    order = []
    stack = [0]
    while stack:
        u = stack.pop()
        order.append(u)
        stack.extend(children[u])
    # Per-phase demand proxy of each bus (worst phase): |a| + |b| scaled by
    # (1 + alpha) to cover voltage dependence and delta connection.
    dem = np.zeros(n_bus)
    for ld in loads:
        per = (np.abs(ld["a"]) + np.abs(ld["b"])) * (1.0 + ld["alpha"])
        dem[ld["bus"]] += float(per.max())
    zrow = np.zeros(n_bus)
    for e in range(n_tree):
        zr = np.abs(lines[e]["r"]).reshape(3, 3).sum(1) + np.abs(lines[e]["x"]).reshape(3, 3).sum(1)
        zrow[e + 1] = zr.max()
    scale = 1.0
    for _ in range(200):
        down = dem * scale
        for u in reversed(order):
            if parent[u] >= 0:
                down[parent[u]] += down[u]
        budget = np.zeros(n_bus)
        for u in order:
            if parent[u] >= 0:
                budget[u] = budget[parent[u]] + 2.0 * zrow[u] * down[u]
        if budget.max() <= drop_budget:
            break
        scale *= 0.9
    loads["a"] *= scale
    loads["b"] *= scale
    down = dem * scale
    for u in reversed(order):
        if parent[u] >= 0:
            down[parent[u]] += down[u]
    for e in range(n_tree):
        lim = 1.5 * down[e + 1] + 0.1
        lines[e]["p_lo"] = -lim
        lines[e]["p_hi"] = lim
        lines[e]["q_lo"] = -lim
        lines[e]["q_hi"] = lim
    for t in range(n_tie):
        lim = 1.5 * down.max() + 0.1
        ln = lines[n_tree + t]
        ln["p_lo"] = -lim
        ln["p_hi"] = lim
        ln["q_lo"] = -lim
        ln["q_hi"] = lim
    src = source_limit if source_limit is not None else max(10.0, 2.0 * down[0])
    gens[0]["pg_lo"] = -src
    gens[0]["pg_hi"] = src
    gens[0]["qg_lo"] = -src
    gens[0]["qg_hi"] = src
    return Feeder(buses, lines, gens, loads, name=name, seed=seed,
                  load_scale=scale, parent=parent, switches=np.array(sw, dtype=np.int64))


def feeder_13(seed: int = 1) -> Feeder:
    """13 buses, 12 lines (mixed 1/2/3-phase), 1 source, 9 loads P~U[0.01,0.4] pu."""
    return make_feeder(13, seed, n_loads=9, load_sampler=lambda r: r.uniform(0.01, 0.4),
                       line_mix=(0.34, 0.33, 0.33), v_ll_kv=4.16, lateral_mean=2.0,
                       name=f"synthetic-13bus-s{seed}")


def feeder_123(seed: int = 1) -> Feeder:
    """123 buses, ~85 loads P~U[0.005,0.1] pu, 10 PV, 4 switches."""
    return make_feeder(123, seed, n_loads=85, load_sampler=lambda r: r.uniform(0.005, 0.1),
                       n_pv=10, pv_pmax=(0.02, 0.2), n_switches=4,
                       line_mix=(0.45, 0.15, 0.40), v_ll_kv=4.16, lateral_mean=4.0,
                       name=f"synthetic-123bus-s{seed}")


def feeder_8500(seed: int = 1, n_bus: int = 11932) -> Feeder:
    """8500-class: 11,932 nodes (Table III node count), ~80/10/10 % 1/2/3-phase
    lines, 1200 loads lognormal(mu=-4, sigma=1) pu, 200 PV."""
    return make_feeder(n_bus, seed, n_loads=1200,
                       load_sampler=lambda r: r.lognormal(-4.0, 1.0),
                       n_pv=200, pv_pmax=(0.02, 0.2), n_switches=0,
                       line_mix=(0.80, 0.10, 0.10), v_ll_kv=12.47, lateral_mean=6.0,
                       line_len=(0.02, 0.3), chain_prob=0.5,
                       name=f"synthetic-8500class-{n_bus}node-s{seed}")


def feeder_tiny(n_bus: int, seed: int, *, shunts: bool = True, taps: bool = True,
                delta_prob: float = 0.5) -> Feeder:
    """Small feeders (3-8 buses) for oracle pins; exercises shunts, taps, delta loads."""
    return make_feeder(n_bus, seed, n_loads=max(1, n_bus - 2),
                       load_sampler=lambda r: r.uniform(0.02, 0.3), n_pv=1,
                       line_mix=(0.3, 0.3, 0.4), v_ll_kv=4.16, lateral_mean=2.0,
                       shunts=shunts, taps=taps, delta_prob=delta_prob,
                       name=f"tiny-{n_bus}-s{seed}")


def feeder_batch(n: int, seed: int, lo: int = 100, hi: int = 2500) -> list[Feeder]:
    """Feeders of uneven size (n_bus ~ U[lo, hi]) with their own switch state
    and load draw, for batched solves."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        nb = int(rng.integers(lo, hi + 1))
        s = int(rng.integers(0, 2 ** 31 - 1))
        out.append(make_feeder(nb, s, n_loads=max(1, nb // 8),
                               load_sampler=lambda r: r.lognormal(-4.0, 1.0),
                               n_pv=max(1, nb // 60), n_switches=4,
                               line_mix=(0.6, 0.15, 0.25), v_ll_kv=12.47,
                               lateral_mean=5.0, name=f"batch-{k}-{nb}bus"))
    return out


def reconfigure(f: Feeder, rng) -> Feeder:
    """A topology switch that keeps the feeder radial and connected: close
    one open tie line and open an in-service line on the loop it closes.
    Returns a copy; if the feeder has no open tie, a closed tree switch is
    opened and closed again elsewhere is not attempted (the copy is equal)."""
    g = f.copy()
    ties = [e for e in range(len(g.lines)) if g.lines["in_service"][e] == 0]
    if not ties:
        return g
    tie = int(ties[rng.integers(0, len(ties))])
    a, b = int(g.lines["from_bus"][tie]), int(g.lines["to_bus"][tie])
    # parent pointers of the current spanning tree (BFS from the root)
    adj = [[] for _ in range(g.n_bus)]
    for e in range(len(g.lines)):
        if g.lines["in_service"][e]:
            u, v = int(g.lines["from_bus"][e]), int(g.lines["to_bus"][e])
            adj[u].append((v, e)); adj[v].append((u, e))
    par = [(-1, -1)] * g.n_bus
    seen = [False] * g.n_bus
    seen[0] = True
    queue = [0]
    for u in queue:
        for v, e in adj[u]:
            if not seen[v]:
                seen[v] = True
                par[v] = (u, e)
                queue.append(v)
    def path(u):
        out = []
        while u != 0:
            out.append(par[u][1]); u = par[u][0]
        return out
    pa, pb = path(a), path(b)
    common = set(pa) & set(pb)
    loop = [e for e in pa + pb if e not in common]
    # open a line on the loop whose phases match the tie's (keeps every bus fed)
    cand = [e for e in loop if int(g.lines["phases"][e]) == int(g.lines["phases"][tie])]
    if not cand:
        return g
    off = int(cand[rng.integers(0, len(cand))])
    g.lines["in_service"][tie] = 1
    g.lines["in_service"][off] = 0
    return g


CONFIG_FEEDERS = {
    "13": feeder_13,
    "123": feeder_123,
    "8500": feeder_8500,
}


def load_scenarios(f: Feeder, n: int, seed: int, lo: float = 0.5, hi: float = 1.0) -> np.ndarray:
    """n load draws on the feeder's loads, scenario-major (n x n_load LOAD
    records): scenario 0 is the feeder's own draw, scenario k scales each
    load's a and b by its own factor ~ U[lo, hi] (Q/P kept; bus, phases,
    connection and load model unchanged, so only the draw differs)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = np.empty((n, len(f.loads)), dtype=LOAD_DTYPE)
    for k in range(n):
        out[k] = f.loads
        if k == 0:
            continue
        fac = rng.uniform(lo, hi, size=len(f.loads))
        out[k]["a"] = f.loads["a"] * fac[:, None]
        out[k]["b"] = f.loads["b"] * fac[:, None]
    return out
