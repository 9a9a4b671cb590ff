// Device layout of the problem.
//
// 1. Component order for locality: a depth-first walk over the feeder; each
//    bus brings its own component, the in-service line that reaches it
//    (emitted when its second end is visited), its loads and its generators
//    (under the paper's decomposition a node already holds its loads and
//    generators, and a leaf node travels with its line).
// 2. The order is cut into `nblocks` contiguous chunks of about equal work
//    (n_s^2 + 4 n_s + 16 per component); chunk b is processed by CTA b.
// 3. Inside a chunk, components are sorted by decreasing n and packed into
//    warp tiles first-fit-decreasing: a small tile holds components with
//    sum n_g <= 32 lanes, lane (g, r) owning local r of component g; a
//    component with n > 32 gets a whole warp (big tile).
//    Small-tile operator elements are stored column by column across the
//    lanes: element (c, lane) at mat0 + c*L + lane holds P_g[c][r] (zero
//    when c >= n_g), so step c of the GEMV is one contiguous load for the
//    warp.  P_g is symmetric, so column c is also row c.  Big tiles store
//    (c, r) at mat0 + c*n + r.
// 4. Per chunk: the distinct globals its locals copy (its "halo"), which of
//    them it owns (holds their first copy, so it writes x_i), and its
//    neighbour chunks (chunks that copy one of its globals).
// The global update also has a CSR list of each global's copies (gptr/gcol,
// canonical order); invk = 1/k_i and cik = c_i/k_i carry (B^T B)^{-1} and
// (B^T B)^{-1} c of Eq. (global_sparse).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "internal.hpp"

namespace opf {

namespace {

std::vector<int> locality_order(const Model& M) {
    const int nb = M.n_bus;
    // component index per element
    std::vector<int> bus_comp(nb, -1), line_comp(M.n_line, -1);
    std::vector<std::vector<int>> loads_at(nb), gens_at(nb), lines_at(nb);
    for (int s = 0; s < (int)M.comps.size(); ++s) {
        const Component& c = M.comps[s];
        if (c.kind == COMP_BUS) bus_comp[c.index] = s;
        else if (c.kind == COMP_LINE) line_comp[c.index] = s;
        else if (c.kind == COMP_LOAD) loads_at[M.load_bus[c.index]].push_back(s);
        else gens_at[M.gen_bus[c.index]].push_back(s);
    }
    for (int e = 0; e < M.n_line; ++e)
        if (line_comp[e] >= 0) {
            lines_at[M.line_from[e]].push_back(e);
            lines_at[M.line_to[e]].push_back(e);
        }
    std::vector<int> order;
    order.reserve(M.comps.size());
    std::vector<char> seen(nb, 0), line_done(M.n_line, 0);
    std::vector<int> stack;
    for (int root = 0; root < nb; ++root) {
        if (seen[root]) continue;
        stack.push_back(root);
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            if (seen[u]) continue;
            seen[u] = 1;
            if (bus_comp[u] >= 0) order.push_back(bus_comp[u]);   // a leaf combined with its line has none
            for (int e : lines_at[u]) {
                const int v = M.line_from[e] == u ? M.line_to[e] : M.line_from[e];
                if (seen[v] && !line_done[e]) {          // second end visited
                    line_done[e] = 1;
                    order.push_back(line_comp[e]);
                }
            }
            for (int s : loads_at[u]) order.push_back(s);
            for (int s : gens_at[u]) order.push_back(s);
            for (auto it = lines_at[u].rbegin(); it != lines_at[u].rend(); ++it) {
                const int v = M.line_from[*it] == u ? M.line_to[*it] : M.line_from[*it];
                if (!seen[v]) stack.push_back(v);
            }
        }
    }
    return order;
}

// Every index the kernels dereference, checked once on the host: a layout
// that fails here is an internal error, never a device fault.
void validate(const Packed& K) {
    auto fail = [](const char* what) { throw Error(OPF_ERR_INVALID_ARG, std::string("internal layout check: ") + what); };
    std::vector<char> seen(K.nl, 0);
    if ((int)K.blocks.size() != K.nblocks || K.hcp.size() != K.halo_gid.size() + 1 || K.hcx.size() != K.hci.size())
        fail("sizes");
    for (int b = 0; b < K.nblocks; ++b) {
        const BlockInfo& bi = K.blocks[b];
        if (bi.loc0 < 0 || bi.loc1 > K.nl || bi.loc0 > bi.loc1) fail("chunk locals");
        if (bi.mat0 < 0 || bi.mat1 > K.mat_elems || bi.mat0 > bi.mat1 || (bi.mat0 & 3)) fail("chunk operators");
        if (bi.tile0 < 0 || bi.tile1 > (int)K.tiles.size() || bi.tile0 > bi.tile1) fail("chunk tiles");
        const int nh = bi.halo1 - bi.halo0;
        if (nh < 0 || nh > K.max_halo || nh > 0x10000) fail("chunk halo");
        if (bi.loc1 - bi.loc0 > K.max_loc || bi.mat1 - bi.mat0 > K.max_mat || bi.cp1 - bi.cp0 > K.max_copies) fail("maxima");
        for (int q = bi.nbr0; q < bi.nbr1; ++q)
            if (K.nbrs[q] < 0 || K.nbrs[q] >= K.nblocks || K.nbrs[q] == b) fail("neighbour");
        if (bi.tileb < bi.tile0 || bi.tileb > bi.tile1 || bi.halob < bi.halo0 || bi.halob > bi.halo1) fail("interior split");
        for (int h = bi.halo0; h < bi.halob; ++h)
            for (int q = K.hcp[h]; q < K.hcp[h + 1]; ++q)
                if (K.hci[q] < 0) fail("interior halo entry with an outside copy");
        for (int t = bi.tile0; t < bi.tileb; ++t)
            for (int r = 0; r < K.tiles[t].L; ++r)
                if ((K.meta[K.tiles[t].loc0 + r] & 0xFFFF) >= bi.halob - bi.halo0) fail("interior tile reads a boundary global");
        for (int t = bi.tile0; t < bi.tile1; ++t) {
            const Tile& tl = K.tiles[t];
            const int lanes = tl.L;
            const int64_t span = tl.big ? (int64_t)tl.L * tl.L : (int64_t)((tl.nmax + 3) / 4) * 4 * tl.L;
            if (tl.loc0 < bi.loc0 || tl.loc0 + lanes > bi.loc1) fail("tile locals");
            if (tl.mat0 < bi.mat0 || tl.mat0 + span > bi.mat1 || (tl.mat0 & 3)) fail("tile operators");
            if (!tl.big && lanes == 0 && tl.nmax != 0) fail("padding tile shape");
            if (!tl.big && lanes != 0 && (lanes < 1 || lanes > 32 || tl.nmax < 1 || tl.nmax > 32)) fail("small tile shape");
            if (tl.big && (tl.nmax != tl.L || tl.L <= 32 || tl.L > 255)) fail("big tile shape");
            for (int r = 0; r < lanes; ++r) {
                const int j = tl.loc0 + r;
                if (seen[j]) fail("local placed twice");
                seen[j] = 1;
                const int m = K.meta[j], n = (m >> 16) & 0xFF, base = (m >> 24) & 0x1F;
                if ((m & 0xFFFF) >= nh) fail("halo index");
                if (!tl.big && (n < 1 || n > tl.nmax || base + n > lanes || r < base || r >= base + n)) fail("lane meta");
                if (K.halo_gid[bi.halo0 + (m & 0xFFFF)] != K.gidx[j]) fail("halo entry of a local");
            }
        }
        if (bi.cp0 != K.hcp[bi.halo0] || bi.cp1 != K.hcp[bi.halo1]) fail("copy list range");
        if (bi.ext0 < 0 || bi.ext1 > (int)K.ext.size() || bi.ext0 > bi.ext1 || bi.ext1 - bi.ext0 > K.max_ext)
            fail("gather list range");
        for (int q = bi.cp0; q < bi.cp1; ++q) {
            const int c = K.hcx[q];
            if (c >= 0) {
                if (c != K.hci[q]) fail("gather copy index");
            } else if (~c >= bi.ext1 - bi.ext0 || K.ext[bi.ext0 + ~c] != ~K.hci[q]) {
                fail("gather slot");
            }
        }
        for (int h = bi.halo0; h < bi.halo1; ++h) {
            const int g = K.halo_gid[h];
            if (g < 0 || g >= K.ng) fail("halo global");
            if (K.hcp[h + 1] - K.hcp[h] != K.gptr[g + 1] - K.gptr[g]) fail("copy count");
            for (int q = K.hcp[h]; q < K.hcp[h + 1]; ++q) {
                const int c = K.hci[q];
                if (c >= 0) {
                    if (c >= bi.loc1 - bi.loc0 || K.gidx[bi.loc0 + c] != g) fail("internal copy");
                } else {
                    const int l = ~c;
                    if (l < 0 || l >= K.nl || (l >= bi.loc0 && l < bi.loc1) || K.gidx[l] != g) fail("external copy");
                    if (!(K.meta[l] & (1 << 30))) fail("external copy not exported");
                }
            }
        }
    }
    for (int j = 0; j < K.nl; ++j)
        if (!seen[j]) fail("local not placed");
}

}  // namespace

Packed pack(const Model& M, const std::vector<Operator>& ops, int nblocks_hint) {
    Packed K;
    K.ng = M.n;
    K.ncomp = (int)M.comps.size();
    std::vector<int64_t> cptr(K.ncomp + 1, 0);
    int64_t work_total = 0;
    for (int s = 0; s < K.ncomp; ++s) {
        const int n = M.comps[s].n();
        cptr[s + 1] = cptr[s] + n;
        K.sum_n2 += (int64_t)n * n;
        K.max_n = std::max(K.max_n, n);
        work_total += (int64_t)n * n + 4 * n + 16;
    }
    if (cptr[K.ncomp] > INT32_MAX / 2) throw Error(OPF_ERR_INVALID_ARG, "problem too large");
    K.nl = (int)cptr[K.ncomp];
    if (K.max_n > 255) throw Error(OPF_ERR_INVALID_ARG, "a component has more than 255 local variables");

    // ---- chunks
    int nblk = nblocks_hint;
    if (nblk <= 0) {
        int64_t work = 4096;
        int cap = 296;
        auto_chunking(M.n_bus, &work, &cap);
        nblk = (int)std::min<int64_t>(cap, std::max<int64_t>(1, work_total / work));
    }
    nblk = std::max(1, std::min(nblk, std::max(1, K.ncomp)));
    const std::vector<int> order = locality_order(M);
    std::vector<int> chunk_start;   // index into order
    {
        int64_t acc = 0;
        int b = 0;
        chunk_start.push_back(0);
        for (int q = 0; q < (int)order.size(); ++q) {
            const int n = M.comps[order[q]].n();
            acc += (int64_t)n * n + 4 * n + 16;
            if (b + 1 < nblk && acc * nblk >= (int64_t)(b + 1) * work_total && q + 1 < (int)order.size()) {
                chunk_start.push_back(q + 1);
                ++b;
            }
        }
        chunk_start.push_back((int)order.size());
    }
    K.nblocks = (int)chunk_start.size() - 1;

    K.comp_tile.assign(K.ncomp, -1);
    K.dev_of_canon.assign(K.nl, -1);
    K.canon_of_dev.assign(K.nl, -1);
    K.meta.assign(K.nl, 0);
    std::vector<int> comp_block(K.ncomp, -1);
    for (int b = 0; b < K.nblocks; ++b)
        for (int q = chunk_start[b]; q < chunk_start[b + 1]; ++q) comp_block[order[q]] = b;
    // a global is interior to a chunk when every copy is in that chunk
    std::vector<int> gblock(K.ng, -1);
    std::vector<char> gshared(K.ng, 0);
    for (int s2 = 0; s2 < K.ncomp; ++s2)
        for (int g : M.comps[s2].gvars) {
            if (gblock[g] < 0) gblock[g] = comp_block[s2];
            else if (gblock[g] != comp_block[s2]) gshared[g] = 1;
        }
    auto comp_boundary = [&](int s2) {
        for (int g : M.comps[s2].gvars)
            if (gshared[g]) return true;
        return false;
    };
    int loc = 0;
    int64_t mat = 0;
    for (int b = 0; b < K.nblocks; ++b) {
        BlockInfo bi;
        bi.tile0 = (int)K.tiles.size();
        bi.loc0 = loc;
        mat = (mat + 3) & ~int64_t(3);
        bi.mat0 = (int32_t)mat;
        std::vector<int> comps(order.begin() + chunk_start[b], order.begin() + chunk_start[b + 1]);
        // interior components first, each group by decreasing n
        std::stable_sort(comps.begin(), comps.end(), [&](int a, int c) {
            const bool ba = comp_boundary(a), bc = comp_boundary(c);
            if (ba != bc) return !ba;
            return M.comps[a].n() > M.comps[c].n();
        });
        // first-fit-decreasing into warps, interior and boundary apart
        std::vector<std::vector<int>> warps;
        std::vector<int> lanes;
        size_t first_boundary_warp = 0;
        bool in_boundary = false;
        for (int s : comps) {
            if (!in_boundary && comp_boundary(s)) {
                in_boundary = true;
                first_boundary_warp = warps.size();
            }
            const int n = M.comps[s].n();
            if (n == 0) continue;
            if (n > 32) {
                K.max_big = std::max(K.max_big, n);
                warps.push_back({s});
                lanes.push_back(-1);
                continue;
            }
            bool placed = false;
            for (size_t w = in_boundary ? first_boundary_warp : 0; w < warps.size(); ++w)
                if (lanes[w] >= 0 && lanes[w] + n <= 32) {
                    warps[w].push_back(s);
                    lanes[w] += n;
                    placed = true;
                    break;
                }
            if (!placed) {
                warps.push_back({s});
                lanes.push_back(n);
            }
        }
        if (!in_boundary) first_boundary_warp = warps.size();
        // balance each range (interior, boundary) over the CTA's warps:
        // longest tile first to the least loaded warp, then lay the tiles out
        // so that position q of the range is run by warp q % kTileWarps
        // (empty padding tiles where a warp has fewer tiles)
        // tile cost in units of one group of four operator columns (two
        // vector loads and two packed fmas per lane), plus the per-tile work
        auto tile_cost = [&](size_t w) {
            if (lanes[w] < 0) {
                const int n = M.comps[warps[w][0]].n();
                return (int64_t)(n * ((n + 31) / 32) + 3) / 4 + 6;
            }
            int nmax = 0;
            for (int s2 : warps[w]) nmax = std::max(nmax, M.comps[s2].n());
            return (int64_t)(nmax + 3) / 4 + 6;
        };
        // the local update runs the boundary range, then the interior range,
        // with no barrier in between: balance boundary tiles first, then the
        // interior ones on top of each warp's boundary load
        std::vector<int64_t> load(kTileWarps, 0);
        std::vector<std::vector<size_t>> per_range[2];
        for (int range : {1, 0}) {
            const size_t r0 = range == 0 ? 0 : first_boundary_warp;
            const size_t r1 = range == 0 ? first_boundary_warp : warps.size();
            std::vector<size_t> idx;
            for (size_t w = r0; w < r1; ++w) idx.push_back(w);
            std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t c) { return tile_cost(a) > tile_cost(c); });
            std::vector<std::vector<size_t>>& per = per_range[range];
            per.assign(kTileWarps, {});
            for (size_t w : idx) {
                int best = 0;
                for (int k = 1; k < kTileWarps; ++k)
                    if (load[k] < load[best]) best = k;
                per[best].push_back(w);
                load[best] += tile_cost(w);
            }
        }
        // lay each range out so that position q of the range is run by warp
        // q % kTileWarps (empty padding tiles where a warp has fewer tiles)
        std::vector<long> layout;              // indices into warps, -1 = padding
        for (int range = 0; range < 2; ++range) {
            if (range == 1) bi.tileb = bi.tile0 + (int)layout.size();
            const std::vector<std::vector<size_t>>& per = per_range[range];
            size_t rows = 0;
            for (auto& v2 : per) rows = std::max(rows, v2.size());
            for (size_t k = 0; k < rows; ++k)
                for (int w = 0; w < kTileWarps; ++w) layout.push_back(k < per[w].size() ? (long)per[w][k] : -1L);
            while (!layout.empty() && layout.back() < 0 && (int)layout.size() > bi.tileb - bi.tile0) layout.pop_back();
        }
        for (long lw : layout) {
            if (lw < 0) {                          // padding tile: no lanes, no operator
                Tile t;
                t.loc0 = bi.loc0; t.mat0 = bi.mat0; t.L = 0; t.nmax = 0; t.big = 0;
                K.tiles.push_back(t);
                continue;
            }
            const size_t w = (size_t)lw;
            for (int s2 : warps[w]) K.comp_tile[s2] = (int32_t)K.tiles.size();
            mat = (mat + 3) & ~int64_t(3);   // 32-byte aligned tile start (f64)
            if (mat > INT32_MAX) throw Error(OPF_ERR_INVALID_ARG, "problem too large");
            Tile t;
            t.loc0 = loc;
            t.mat0 = (int32_t)mat;
            if (lanes[w] < 0) {
                const int s = warps[w][0], n = M.comps[s].n();
                t.L = (int16_t)n; t.nmax = (int16_t)n; t.big = 1;
                K.P.resize((size_t)mat + (size_t)n * n, 0.0);
                for (int c = 0; c < n; ++c)
                    for (int r = 0; r < n; ++r) K.P[(size_t)mat + (size_t)c * n + r] = ops[s].P[(size_t)c * n + r];
                for (int r = 0; r < n; ++r) {
                    K.dev_of_canon[cptr[s] + r] = loc + r;
                    K.canon_of_dev[loc + r] = (int32_t)(cptr[s] + r);
                    K.meta[loc + r] = (n << 16);
                }
                mat += (int64_t)n * n;
                loc += n;
            } else {
                const int L = lanes[w];
                int nmax = 0;
                for (int s : warps[w]) nmax = std::max(nmax, M.comps[s].n());
                t.L = (int16_t)L; t.nmax = (int16_t)nmax; t.big = 0;
                // columns in groups of four, lane-interleaved: column c of
                // lane r at ((c / 4) * L + r) * 4 + c % 4, zero beyond n
                const int nq = (nmax + 3) / 4;
                K.P.resize((size_t)mat + (size_t)nq * 4 * L, 0.0);
                int base = 0;
                for (int s : warps[w]) {
                    const int n = M.comps[s].n();
                    for (int r = 0; r < n; ++r) {
                        const int lane = base + r;
                        K.dev_of_canon[cptr[s] + r] = loc + lane;
                        K.canon_of_dev[loc + lane] = (int32_t)(cptr[s] + r);
                        K.meta[loc + lane] = (n << 16) | (base << 24);
                        for (int c = 0; c < n; ++c)
                            K.P[(size_t)mat + ((size_t)(c / 4) * L + lane) * 4 + c % 4] = ops[s].P[(size_t)c * n + r];
                    }
                    base += n;
                }
                mat += (int64_t)nq * 4 * L;
                loc += L;
            }
            K.tiles.push_back(t);
        }
        bi.tile1 = (int)K.tiles.size();
        bi.loc1 = loc;
        bi.mat1 = (int32_t)mat;
        K.max_tiles = std::max(K.max_tiles, bi.tile1 - bi.tile0);
        K.max_loc = std::max(K.max_loc, bi.loc1 - bi.loc0);
        K.max_mat = std::max(K.max_mat, bi.mat1 - bi.mat0);
        K.blocks.push_back(bi);
    }
    if (loc != K.nl) throw Error(OPF_ERR_INVALID_ARG, "internal: locals not all placed");
    K.mat_elems = (int64_t)K.P.size();

    // ---- local vectors in device order
    K.gidx.resize(K.nl);
    K.bbar.resize(K.nl);
    K.xl0.resize(K.nl);
    std::vector<int> kcount(K.ng, 0);
    for (int s = 0; s < K.ncomp; ++s) {
        const Component& C = M.comps[s];
        for (int r = 0; r < C.n(); ++r) {
            const int d = K.dev_of_canon[cptr[s] + r];
            const int g = C.gvars[r];
            K.gidx[d] = g;
            K.bbar[d] = ops[s].bbar[r];
            // Section V-A: 1 for voltages, midpoint when both bounds are finite, else 0
            double x0 = 0.0;
            if (M.is_w[g]) x0 = 1.0;
            else if (std::isfinite(M.lo[g]) && std::isfinite(M.hi[g])) x0 = 0.5 * (M.lo[g] + M.hi[g]);
            K.xl0[d] = x0;
            ++kcount[g];
        }
    }
    // ---- CSR of copies, canonical order
    K.gptr.assign(K.ng + 1, 0);
    for (int i = 0; i < K.ng; ++i) {
        if (kcount[i] == 0) throw Error(OPF_ERR_INVALID_ARG, "a global variable has no local copy");
        K.gptr[i + 1] = K.gptr[i] + kcount[i];
    }
    K.gcol.assign(K.nl, 0);
    std::vector<int> fill(K.gptr.begin(), K.gptr.end() - 1);
    for (int s = 0; s < K.ncomp; ++s) {
        const Component& C = M.comps[s];
        for (int r = 0; r < C.n(); ++r) K.gcol[fill[C.gvars[r]]++] = K.dev_of_canon[cptr[s] + r];
    }
    K.invk.resize(K.ng);
    K.cik.resize(K.ng);
    for (int i = 0; i < K.ng; ++i) {
        K.invk[i] = 1.0 / (double)kcount[i];
        K.cik[i] = M.c[i] / (double)kcount[i];
    }

    // ---- halos, owners, neighbours
    std::vector<int> owner(K.ng, -1);          // block of the first copy (device order)
    std::vector<int> block_of_loc(K.nl);
    for (int b = 0; b < K.nblocks; ++b)
        for (int j = K.blocks[b].loc0; j < K.blocks[b].loc1; ++j) block_of_loc[j] = b;
    for (int j = 0; j < K.nl; ++j)
        if (owner[K.gidx[j]] < 0) owner[K.gidx[j]] = block_of_loc[j];
    std::vector<int> hmark(K.ng, -1), hpos(K.ng, 0), bmark(K.nblocks, -1);
    for (int b = 0; b < K.nblocks; ++b) {
        BlockInfo& bi = K.blocks[b];
        bi.halo0 = (int)K.halo_gid.size();
        for (int pass = 0; pass < 2; ++pass) {           // interior globals, then boundary
            if (pass == 1) bi.halob = (int)K.halo_gid.size();
            for (int j = bi.loc0; j < bi.loc1; ++j) {
                const int g = K.gidx[j];
                if ((int)gshared[g] != pass || hmark[g] == b) continue;
                hmark[g] = b;
                hpos[g] = (int)K.halo_gid.size() - bi.halo0;
                K.halo_gid.push_back(g);
                K.halo_own.push_back(owner[g] == b ? 1 : 0);
            }
        }
        for (int j = bi.loc0; j < bi.loc1; ++j) {
            const int g = K.gidx[j];
            if (hpos[g] > 0xFFFF) throw Error(OPF_ERR_INVALID_ARG, "chunk halo too large");
            K.meta[j] |= hpos[g];
        }
        bi.halo1 = (int)K.halo_gid.size();
        K.max_halo = std::max(K.max_halo, bi.halo1 - bi.halo0);
        // copy lists of the halo globals, canonical copy order; a copy held by
        // this chunk is referenced by its chunk-relative local index
        // (hcx: a copy of another chunk as ~slot in the chunk's list of such
        // copies, ext, which the persistent kernel gathers in one pass)
        bi.cp0 = (int)K.hci.size();
        bi.ext0 = (int)K.ext.size();
        for (int h = bi.halo0; h < bi.halo1; ++h) {
            K.hcp.push_back((int)K.hci.size());
            const int g = K.halo_gid[h];
            for (int q = K.gptr[g]; q < K.gptr[g + 1]; ++q) {
                const int l = K.gcol[q];
                if (l >= bi.loc0 && l < bi.loc1) {
                    K.hci.push_back(l - bi.loc0);
                    K.hcx.push_back(l - bi.loc0);
                } else {
                    K.hci.push_back(~l);
                    K.hcx.push_back(~((int)K.ext.size() - bi.ext0));
                    K.ext.push_back(l);
                    K.meta[l] |= (1 << 30);        // read by another chunk: exported
                }
            }
        }
        bi.cp1 = (int)K.hci.size();
        bi.ext1 = (int)K.ext.size();
        K.max_copies = std::max(K.max_copies, bi.cp1 - bi.cp0);
        K.max_ext = std::max(K.max_ext, bi.ext1 - bi.ext0);
        bi.nbr0 = (int)K.nbrs.size();
        for (int h = bi.halo0; h < bi.halo1; ++h) {
            const int g = K.halo_gid[h];
            for (int q = K.gptr[g]; q < K.gptr[g + 1]; ++q) {
                const int d = block_of_loc[K.gcol[q]];
                if (d != b && bmark[d] != b) {
                    bmark[d] = b;
                    K.nbrs.push_back(d);
                }
            }
        }
        std::sort(K.nbrs.begin() + bi.nbr0, K.nbrs.end());
        bi.nbr1 = (int)K.nbrs.size();
    }
    K.hcp.push_back((int)K.hci.size());
    validate(K);
    return K;
}

}  // namespace opf
