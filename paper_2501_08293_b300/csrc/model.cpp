// Model assembly: the linearized multi-phase OPF of Section II-A written as
// the LP of Eq. (LP_model), split into fine components (Eq. OurModel).
//
// Rows per component (each over the element's phases):
//   bus   Eq. (balance_eqns): sum flows leaving + sum pb + g^sh w - sum pg = 0
//                             sum q leaving + sum qb - b^sh w - sum qg = 0
//   line  Eq. (power_flow_eqns): powerloss-1, powerloss-2, voltage_mag_diff
//   load  Eq. (volt_load_model): VDLM-1/2 with what = w (wye) or 3w (delta),
//         then VDLM-5 (wye) or VDLM-6..10 (three-phase delta)
//   gen   no rows
// The ordering of globals, components and locals is the canonical order
// documented in opf_admm.h.
//
// Decomposition of Section V-A (OPF_DECOMP_PAPER): one component per node
// of the feeder graph -- a bus together with its loads and generators --
// and one per in-service line, except that a node with exactly one
// in-service line (a leaf) is combined with that line, so S = nodes + lines
// - leaves (Table III).  A combined component's locals are its parts'
// locals in order, a global already present keeping its first local; its
// rows are its parts' rows stacked in the same order.
#include <cmath>
#include <cstring>
#include <map>

#include "internal.hpp"

namespace opf {
namespace {

constexpr double kSqrt3 = 1.7320508075688772935;


inline void phases(uint8_t m, int* out, int* cnt) {
    int k = 0;
    for (int p = 0; p < 3; ++p)
        if (m & (1u << p)) out[k++] = p;
    *cnt = k;
}

void check_bounds(double lo, double hi, const char* what, int idx) {
    if (std::isnan(lo) || std::isnan(hi) || lo > hi)
        throw Error(OPF_ERR_INVALID_ARG, std::string(what) + " " + std::to_string(idx) + ": bad bounds");
}

void check_finite(double v, const char* what, int idx) {
    if (!std::isfinite(v))
        throw Error(OPF_ERR_INVALID_ARG, std::string(what) + " " + std::to_string(idx) + ": non-finite value");
}

// Dense row builder for one component: column lookup by global index.
struct RowSet {
    const std::vector<int32_t>& gv;
    std::map<int32_t, int> col;
    std::vector<double> A, b;
    int m = 0;
    explicit RowSet(const std::vector<int32_t>& g) : gv(g) {
        for (int j = 0; j < (int)g.size(); ++j) col[g[j]] = j;
    }
    // rows are referred to by index: A may reallocate when a row is added
    int row(double rhs) {
        A.resize(A.size() + gv.size(), 0.0);
        b.push_back(rhs);
        return m++;
    }
    void add(int r, int32_t g, double v) { A[(size_t)r * gv.size() + col.at(g)] += v; }
};

}  // namespace

// Line component of Eq. (power_flow_eqns) for in-service line e, on the
// global indices already assigned in M.
Component line_component(const Model& M, const opf_line& L, int e) {
    int ph[3], np;
    Component C;
    C.kind = COMP_LINE; C.index = e;
    phases(L.phases, ph, &np);
    const int i = L.from_bus, j = L.to_bus;
    for (const std::vector<int32_t>* t : {&M.pij_idx, &M.qij_idx, &M.pji_idx, &M.qji_idx})
        for (int a = 0; a < np; ++a) C.gvars.push_back((*t)[3 * e + ph[a]]);
    for (int a = 0; a < np; ++a) C.gvars.push_back(M.w_idx[3 * i + ph[a]]);
    for (int a = 0; a < np; ++a) C.gvars.push_back(M.w_idx[3 * j + ph[a]]);
    // M^p, M^q (Section II-A) on phases a, b, c; sub-block read by phase.
    double Mp[3][3], Mq[3][3];
    const double* r = L.r;
    const double* x = L.x;
    auto R_ = [&](int u, int v) { return r[3 * u + v]; };
    auto X_ = [&](int u, int v) { return x[3 * u + v]; };
    // diagonal
    for (int u = 0; u < 3; ++u) { Mp[u][u] = -2.0 * R_(u, u); Mq[u][u] = -2.0 * X_(u, u); }
    // off-diagonal: sign s = +1 where the paper writes r - sqrt3 x (Mp) / x + sqrt3 r (Mq)
    // pairs (1,2),(2,3),(3,1) take "- sqrt3 x"; pairs (1,3),(2,1),(3,2) take "+ sqrt3 x"
    const int lag[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    const int lead[3][2] = {{0, 2}, {1, 0}, {2, 1}};
    for (auto& pq : lag) {
        int u = pq[0], v = pq[1];
        Mp[u][v] = R_(u, v) - kSqrt3 * X_(u, v);
        Mq[u][v] = X_(u, v) + kSqrt3 * R_(u, v);
    }
    for (auto& pq : lead) {
        int u = pq[0], v = pq[1];
        Mp[u][v] = R_(u, v) + kSqrt3 * X_(u, v);
        Mq[u][v] = X_(u, v) - kSqrt3 * R_(u, v);
    }
    RowSet Rs(C.gvars);
    for (int a = 0; a < np; ++a) {
        const int p = ph[a];
        const int32_t wi = M.w_idx[3 * i + p], wj = M.w_idx[3 * j + p];
        int r1 = Rs.row(0.0);     // powerloss-1
        Rs.add(r1, M.pij_idx[3 * e + p], 1.0);
        Rs.add(r1, M.pji_idx[3 * e + p], 1.0);
        Rs.add(r1, wi, -L.g_fr[p]);
        Rs.add(r1, wj, -L.g_to[p]);
        int r2 = Rs.row(0.0);     // powerloss-2
        Rs.add(r2, M.qij_idx[3 * e + p], 1.0);
        Rs.add(r2, M.qji_idx[3 * e + p], 1.0);
        Rs.add(r2, wi, L.b_fr[p]);
        Rs.add(r2, wj, L.b_to[p]);
        int r3 = Rs.row(0.0);     // voltage_mag_diff
        Rs.add(r3, wi, 1.0);
        Rs.add(r3, wj, -L.tap[p]);
        for (int bb = 0; bb < np; ++bb) {
            const int s = ph[bb];
            const int32_t wis = M.w_idx[3 * i + s];
            Rs.add(r3, M.pij_idx[3 * e + s], Mp[p][s]);
            Rs.add(r3, wis, -Mp[p][s] * L.g_fr[s]);
            Rs.add(r3, M.qij_idx[3 * e + s], Mq[p][s]);
            Rs.add(r3, wis, Mq[p][s] * L.b_fr[s]);
        }
    }
    C.m = Rs.m; C.A = std::move(Rs.A); C.b = std::move(Rs.b);
    return C;
}

Component line_update(const Model& M, const opf_line& L, int e) {
    if (e < 0 || e >= M.n_line) throw Error(OPF_ERR_INVALID_ARG, "line index out of range");
    if (L.from_bus != M.line_from[e] || L.to_bus != M.line_to[e])
        throw Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": ends differ from the problem's");
    if (!L.in_service) throw Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": out of service in the update");
    for (int p = 0; p < 3; ++p) {
        const bool here = M.pij_idx[3 * e + p] >= 0;
        if (here != (((L.phases >> p) & 1u) != 0))
            throw Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": phases or service state differ");
        if (!here) continue;
        check_bounds(L.p_lo[p], L.p_hi[p], "line", e);
        check_bounds(L.q_lo[p], L.q_hi[p], "line", e);
        for (double v : {L.g_fr[p], L.b_fr[p], L.g_to[p], L.b_to[p], L.tap[p]}) check_finite(v, "line", e);
        for (int q = 0; q < 3; ++q)
            if ((L.phases >> q) & 1u) {
                check_finite(L.r[3 * p + q], "line", e);
                check_finite(L.x[3 * p + q], "line", e);
            }
    }
    return line_component(M, L, e);
}

Model build_model(const opf_bus* buses, int nb, const opf_line* lines, int nl,
                  const opf_gen* gens, int ng, const opf_load* loads, int nd) {
    if (nb <= 0 || !buses) throw Error(OPF_ERR_INVALID_ARG, "no buses");
    if (nl < 0 || ng < 0 || nd < 0) throw Error(OPF_ERR_INVALID_ARG, "negative count");
    if ((nl && !lines) || (ng && !gens) || (nd && !loads)) throw Error(OPF_ERR_INVALID_ARG, "null record array");

    // ---- validation
    for (int i = 0; i < nb; ++i) {
        uint8_t m = buses[i].phases;
        if (m == 0 || m > 7) throw Error(OPF_ERR_INVALID_ARG, "bus " + std::to_string(i) + ": bad phase mask");
        for (int p = 0; p < 3; ++p)
            if (m & (1u << p)) {
                check_bounds(buses[i].w_lo[p], buses[i].w_hi[p], "bus", i);
                check_finite(buses[i].g_sh[p], "bus", i);
                check_finite(buses[i].b_sh[p], "bus", i);
            }
    }
    for (int e = 0; e < nl; ++e) {
        const opf_line& L = lines[e];
        if (L.from_bus < 0 || L.from_bus >= nb || L.to_bus < 0 || L.to_bus >= nb || L.from_bus == L.to_bus)
            throw Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": bad ends");
        if (L.phases == 0 || L.phases > 7 || (L.phases & ~buses[L.from_bus].phases) ||
            (L.phases & ~buses[L.to_bus].phases))
            throw Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": phases not on both buses");
        if (!L.in_service) continue;
        for (int p = 0; p < 3; ++p) {
            if (!(L.phases & (1u << p))) continue;
            check_bounds(L.p_lo[p], L.p_hi[p], "line", e);
            check_bounds(L.q_lo[p], L.q_hi[p], "line", e);
            for (double v : {L.g_fr[p], L.b_fr[p], L.g_to[p], L.b_to[p], L.tap[p]}) check_finite(v, "line", e);
            for (int q = 0; q < 3; ++q)
                if (L.phases & (1u << q)) {
                    check_finite(L.r[3 * p + q], "line", e);
                    check_finite(L.x[3 * p + q], "line", e);
                }
        }
    }
    for (int k = 0; k < ng; ++k) {
        const opf_gen& G = gens[k];
        if (G.bus < 0 || G.bus >= nb || G.phases == 0 || G.phases > 7 || (G.phases & ~buses[G.bus].phases))
            throw Error(OPF_ERR_INVALID_ARG, "gen " + std::to_string(k) + ": bad bus/phases");
        for (int p = 0; p < 3; ++p)
            if (G.phases & (1u << p)) {
                check_bounds(G.pg_lo[p], G.pg_hi[p], "gen", k);
                check_bounds(G.qg_lo[p], G.qg_hi[p], "gen", k);
                check_finite(G.cost[p], "gen", k);
            }
    }
    for (int l = 0; l < nd; ++l) {
        const opf_load& D = loads[l];
        if (D.bus < 0 || D.bus >= nb || D.phases == 0 || D.phases > 7 || (D.phases & ~buses[D.bus].phases))
            throw Error(OPF_ERR_INVALID_ARG, "load " + std::to_string(l) + ": bad bus/phases");
        if (D.conn > 1) throw Error(OPF_ERR_INVALID_ARG, "load " + std::to_string(l) + ": bad connection");
        if (D.conn == 1 && D.phases != 7)
            throw Error(OPF_ERR_INVALID_ARG, "load " + std::to_string(l) + ": delta loads must be three-phase");
        for (int p = 0; p < 3; ++p)
            if (D.phases & (1u << p))
                for (double v : {D.a[p], D.b[p], D.alpha[p], D.beta[p]}) check_finite(v, "load", l);
    }

    Model M;
    M.n_bus = nb; M.n_line = nl; M.n_gen = ng; M.n_load = nd;
    for (int e = 0; e < nl; ++e) { M.line_from.push_back(lines[e].from_bus); M.line_to.push_back(lines[e].to_bus); }
    for (int l = 0; l < nd; ++l) M.load_bus.push_back(loads[l].bus);
    for (int k = 0; k < ng; ++k) M.gen_bus.push_back(gens[k].bus);
    auto var = [&](double lo, double hi, double c, bool w) {
        M.lo.push_back(lo); M.hi.push_back(hi); M.c.push_back(c); M.is_w.push_back(w ? 1 : 0);
        return (int32_t)(M.lo.size() - 1);
    };
    const double inf = INFINITY;
    M.w_idx.assign((size_t)nb * 3, -1);
    M.pg_idx.assign((size_t)ng * 3, -1); M.qg_idx.assign((size_t)ng * 3, -1);
    M.pij_idx.assign((size_t)nl * 3, -1); M.qij_idx.assign((size_t)nl * 3, -1);
    M.pji_idx.assign((size_t)nl * 3, -1); M.qji_idx.assign((size_t)nl * 3, -1);
    M.pb_idx.assign((size_t)nd * 3, -1); M.qb_idx.assign((size_t)nd * 3, -1);
    M.pd_idx.assign((size_t)nd * 3, -1); M.qd_idx.assign((size_t)nd * 3, -1);

    int ph[3], np;
    // ---- global variables, Eq. (LP_model) order
    for (int k = 0; k < ng; ++k) {
        phases(gens[k].phases, ph, &np);
        for (int a = 0; a < np; ++a) M.pg_idx[3 * k + ph[a]] = var(gens[k].pg_lo[ph[a]], gens[k].pg_hi[ph[a]], gens[k].cost[ph[a]], false);
        for (int a = 0; a < np; ++a) M.qg_idx[3 * k + ph[a]] = var(gens[k].qg_lo[ph[a]], gens[k].qg_hi[ph[a]], 0.0, false);
    }
    for (int i = 0; i < nb; ++i) {
        phases(buses[i].phases, ph, &np);
        for (int a = 0; a < np; ++a) M.w_idx[3 * i + ph[a]] = var(buses[i].w_lo[ph[a]], buses[i].w_hi[ph[a]], 0.0, true);
    }
    for (int l = 0; l < nd; ++l) {
        phases(loads[l].phases, ph, &np);
        std::vector<int32_t>* tabs[4] = {&M.pb_idx, &M.qb_idx, &M.pd_idx, &M.qd_idx};
        for (auto* t : tabs)
            for (int a = 0; a < np; ++a) (*t)[3 * l + ph[a]] = var(-inf, inf, 0.0, false);
    }
    for (int e = 0; e < nl; ++e) {
        if (!lines[e].in_service) continue;
        phases(lines[e].phases, ph, &np);
        const opf_line& L = lines[e];
        for (int a = 0; a < np; ++a) M.pij_idx[3 * e + ph[a]] = var(L.p_lo[ph[a]], L.p_hi[ph[a]], 0.0, false);
        for (int a = 0; a < np; ++a) M.qij_idx[3 * e + ph[a]] = var(L.q_lo[ph[a]], L.q_hi[ph[a]], 0.0, false);
        for (int a = 0; a < np; ++a) M.pji_idx[3 * e + ph[a]] = var(L.p_lo[ph[a]], L.p_hi[ph[a]], 0.0, false);
        for (int a = 0; a < np; ++a) M.qji_idx[3 * e + ph[a]] = var(L.q_lo[ph[a]], L.q_hi[ph[a]], 0.0, false);
    }
    M.n = (int)M.lo.size();

    // incidence lists in input order
    std::vector<std::vector<int>> lines_at(nb), loads_at(nb), gens_at(nb);
    for (int e = 0; e < nl; ++e)
        if (lines[e].in_service) {
            lines_at[lines[e].from_bus].push_back(e);
            lines_at[lines[e].to_bus].push_back(e);
        }
    for (int l = 0; l < nd; ++l) loads_at[loads[l].bus].push_back(l);
    for (int k = 0; k < ng; ++k) gens_at[gens[k].bus].push_back(k);

    // ---- bus components, Eq. (balance_eqns)
    for (int i = 0; i < nb; ++i) {
        Component C;
        C.kind = COMP_BUS; C.index = i;
        phases(buses[i].phases, ph, &np);
        for (int a = 0; a < np; ++a) C.gvars.push_back(M.w_idx[3 * i + ph[a]]);
        for (int e : lines_at[i]) {
            int lp[3], ln;
            phases(lines[e].phases, lp, &ln);
            bool from = lines[e].from_bus == i;
            for (int a = 0; a < ln; ++a) C.gvars.push_back(from ? M.pij_idx[3 * e + lp[a]] : M.pji_idx[3 * e + lp[a]]);
            for (int a = 0; a < ln; ++a) C.gvars.push_back(from ? M.qij_idx[3 * e + lp[a]] : M.qji_idx[3 * e + lp[a]]);
        }
        for (int l : loads_at[i]) {
            int lp[3], ln;
            phases(loads[l].phases, lp, &ln);
            for (int a = 0; a < ln; ++a) C.gvars.push_back(M.pb_idx[3 * l + lp[a]]);
            for (int a = 0; a < ln; ++a) C.gvars.push_back(M.qb_idx[3 * l + lp[a]]);
        }
        for (int k : gens_at[i]) {
            int lp[3], ln;
            phases(gens[k].phases, lp, &ln);
            for (int a = 0; a < ln; ++a) C.gvars.push_back(M.pg_idx[3 * k + lp[a]]);
            for (int a = 0; a < ln; ++a) C.gvars.push_back(M.qg_idx[3 * k + lp[a]]);
        }
        RowSet R(C.gvars);
        for (int a = 0; a < np; ++a) {
            const int p = ph[a];
            int rp = R.row(0.0);
            int rq = R.row(0.0);
            for (int e : lines_at[i]) {
                if (!(lines[e].phases & (1u << p))) continue;
                bool from = lines[e].from_bus == i;
                R.add(rp, from ? M.pij_idx[3 * e + p] : M.pji_idx[3 * e + p], 1.0);
                R.add(rq, from ? M.qij_idx[3 * e + p] : M.qji_idx[3 * e + p], 1.0);
            }
            for (int l : loads_at[i]) {
                if (!(loads[l].phases & (1u << p))) continue;
                R.add(rp, M.pb_idx[3 * l + p], 1.0);
                R.add(rq, M.qb_idx[3 * l + p], 1.0);
            }
            R.add(rp, M.w_idx[3 * i + p], buses[i].g_sh[p]);
            R.add(rq, M.w_idx[3 * i + p], -buses[i].b_sh[p]);
            for (int k : gens_at[i]) {
                if (!(gens[k].phases & (1u << p))) continue;
                R.add(rp, M.pg_idx[3 * k + p], -1.0);
                R.add(rq, M.qg_idx[3 * k + p], -1.0);
            }
        }
        C.m = R.m; C.A = std::move(R.A); C.b = std::move(R.b);
        M.comps.push_back(std::move(C));
    }

    // ---- line components, Eq. (power_flow_eqns)
    for (int e = 0; e < nl; ++e) {
        if (!lines[e].in_service) continue;
        M.comps.push_back(line_component(M, lines[e], e));
    }

    // ---- load components, Eq. (volt_load_model)
    for (int l = 0; l < nd; ++l) {
        const opf_load& D = loads[l];
        Component C;
        C.kind = COMP_LOAD; C.index = l;
        phases(D.phases, ph, &np);
        for (const std::vector<int32_t>* t : {&M.pb_idx, &M.qb_idx, &M.pd_idx, &M.qd_idx})
            for (int a = 0; a < np; ++a) C.gvars.push_back((*t)[3 * l + ph[a]]);
        for (int a = 0; a < np; ++a) C.gvars.push_back(M.w_idx[3 * D.bus + ph[a]]);
        const bool delta = D.conn == 1;
        const double wm = delta ? 3.0 : 1.0;    // VDLM-4 : VDLM-3
        RowSet Rs(C.gvars);
        for (int a = 0; a < np; ++a) {
            const int p = ph[a];
            const int32_t w = M.w_idx[3 * D.bus + p];
            // VDLM-1: pd - (a alpha/2) what = a - a alpha / 2
            int r1 = Rs.row(D.a[p] - 0.5 * D.a[p] * D.alpha[p]);
            Rs.add(r1, M.pd_idx[3 * l + p], 1.0);
            Rs.add(r1, w, -0.5 * D.a[p] * D.alpha[p] * wm);
            // VDLM-2
            int r2 = Rs.row(D.b[p] - 0.5 * D.b[p] * D.beta[p]);
            Rs.add(r2, M.qd_idx[3 * l + p], 1.0);
            Rs.add(r2, w, -0.5 * D.b[p] * D.beta[p] * wm);
        }
        auto pb = [&](int p) { return M.pb_idx[3 * l + p]; };
        auto qb = [&](int p) { return M.qb_idx[3 * l + p]; };
        auto pd = [&](int p) { return M.pd_idx[3 * l + p]; };
        auto qd = [&](int p) { return M.qd_idx[3 * l + p]; };
        if (!delta) {
            for (int a = 0; a < np; ++a) {     // VDLM-5
                const int p = ph[a];
                int r = Rs.row(0.0); Rs.add(r, pb(p), 1.0); Rs.add(r, pd(p), -1.0);
                r = Rs.row(0.0); Rs.add(r, qb(p), 1.0); Rs.add(r, qd(p), -1.0);
            }
        } else {
            const double h = 0.5 * kSqrt3;
            int r = Rs.row(0.0);           // VDLM-6 (real)
            for (int p = 0; p < 3; ++p) { Rs.add(r, pb(p), 1.0); Rs.add(r, pd(p), -1.0); }
            r = Rs.row(0.0);                   // VDLM-6 (reactive)
            for (int p = 0; p < 3; ++p) { Rs.add(r, qb(p), 1.0); Rs.add(r, qd(p), -1.0); }
            // VDLM-7: 3/2 pb2 - h qb2 - pd2 - 1/2 pd1 + h qd1 = 0
            r = Rs.row(0.0);
            Rs.add(r, pb(1), 1.5); Rs.add(r, qb(1), -h); Rs.add(r, pd(1), -1.0);
            Rs.add(r, pd(0), -0.5); Rs.add(r, qd(0), h);
            // VDLM-8: h pb2 + 3/2 qb2 - h pd1 - 1/2 qd1 - qd2 = 0
            r = Rs.row(0.0);
            Rs.add(r, pb(1), h); Rs.add(r, qb(1), 1.5); Rs.add(r, pd(0), -h);
            Rs.add(r, qd(0), -0.5); Rs.add(r, qd(1), -1.0);
            // VDLM-9: sqrt3 qb2 + 3/2 pb3 - h qb3 - 1/2 pd1 - h qd1 - pd3 = 0
            r = Rs.row(0.0);
            Rs.add(r, qb(1), kSqrt3); Rs.add(r, pb(2), 1.5); Rs.add(r, qb(2), -h);
            Rs.add(r, pd(0), -0.5); Rs.add(r, qd(0), -h); Rs.add(r, pd(2), -1.0);
            // VDLM-10: -sqrt3 pb2 + h pb3 + 3/2 qb3 + h pd1 - 1/2 qd1 - qd3 = 0
            r = Rs.row(0.0);
            Rs.add(r, pb(1), -kSqrt3); Rs.add(r, pb(2), h); Rs.add(r, qb(2), 1.5);
            Rs.add(r, pd(0), h); Rs.add(r, qd(0), -0.5); Rs.add(r, qd(2), -1.0);
        }
        C.m = Rs.m; C.A = std::move(Rs.A); C.b = std::move(Rs.b);
        M.comps.push_back(std::move(C));
    }

    // ---- generator components: no rows
    for (int k = 0; k < ng; ++k) {
        Component C;
        C.kind = COMP_GEN; C.index = k;
        phases(gens[k].phases, ph, &np);
        for (int a = 0; a < np; ++a) C.gvars.push_back(M.pg_idx[3 * k + ph[a]]);
        for (int a = 0; a < np; ++a) C.gvars.push_back(M.qg_idx[3 * k + ph[a]]);
        C.m = 0;
        M.comps.push_back(std::move(C));
    }
    return M;
}

Component combine_parts(int kind, int index, const std::vector<const Component*>& parts) {
    Component C;
    C.kind = kind;
    C.index = index;
    std::map<int32_t, int> at;           // global -> local position in C
    for (const Component* q : parts)
        for (int32_t g : q->gvars)
            if (at.emplace(g, (int)C.gvars.size()).second) C.gvars.push_back(g);
    const int n = C.n();
    for (const Component* q : parts) {
        const int qn = q->n();
        for (int r = 0; r < q->m; ++r) {
            C.A.resize(C.A.size() + n, 0.0);
            double* row = &C.A[(size_t)C.m * n];
            for (int c = 0; c < qn; ++c) row[at[q->gvars[c]]] += q->A[(size_t)r * qn + c];
            C.b.push_back(q->b[r]);
            ++C.m;
        }
    }
    return C;
}

void paper_decomposition(Model& M) {
    const int nb = M.n_bus, nl = M.n_line;
    std::vector<int> bus_comp(nb, -1), line_comp(nl, -1);
    std::vector<std::vector<int>> parts_of(nb);     // loads, then generators, at each bus
    for (int c = 0; c < (int)M.comps.size(); ++c) {
        const Component& C = M.comps[c];
        if (C.kind == COMP_BUS) bus_comp[C.index] = c;
        else if (C.kind == COMP_LINE) line_comp[C.index] = c;
    }
    for (int c = 0; c < (int)M.comps.size(); ++c)
        if (M.comps[c].kind == COMP_LOAD) parts_of[M.load_bus[M.comps[c].index]].push_back(c);
    for (int c = 0; c < (int)M.comps.size(); ++c)
        if (M.comps[c].kind == COMP_GEN) parts_of[M.gen_bus[M.comps[c].index]].push_back(c);
    std::vector<int> degree(nb, 0);
    for (int e = 0; e < nl; ++e)
        if (line_comp[e] >= 0) {
            ++degree[M.line_from[e]];
            ++degree[M.line_to[e]];
        }
    std::vector<Component> node(nb);
    for (int i = 0; i < nb; ++i) {
        std::vector<const Component*> parts{&M.comps[bus_comp[i]]};
        for (int c : parts_of[i]) parts.push_back(&M.comps[c]);
        node[i] = combine_parts(COMP_BUS, i, parts);
    }
    std::vector<Component> out;
    for (int i = 0; i < nb; ++i)
        if (degree[i] != 1) out.push_back(std::move(node[i]));
    for (int e = 0; e < nl; ++e) {
        if (line_comp[e] < 0) continue;
        const int i = M.line_from[e], j = M.line_to[e];
        std::vector<const Component*> parts{&M.comps[line_comp[e]]};
        if (degree[i] == 1) parts.push_back(&node[i]);
        if (degree[j] == 1) parts.push_back(&node[j]);
        out.push_back(combine_parts(COMP_LINE, e, parts));
    }
    M.comps = std::move(out);
    M.decomposition = OPF_DECOMP_PAPER;
}

}  // namespace opf
