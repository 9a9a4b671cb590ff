// Device layout of the problem.
//
// Components are grouped by size n_s and cut into warp tiles:
//   n <= 32: one tile holds k = floor(32/n) components of the same n; lane
//            (g, r) = (lane / n, lane % n) owns local r of component g.
//            Operator elements are stored column by column across the
//            tile's lanes: element (c, lane) at mat0 + c*L + lane holds
//            P_g[c][r] (L = k n), so step c of the GEMV is one contiguous,
//            coalesced load for the whole warp.  P_g is symmetric, so column
//            c is also row c.
//   n > 32:  one component per tile; element (c, r) at mat0 + c*n + r.
// Tiles are ordered by decreasing n; components keep canonical order
// within a size.  Device local order follows the tiles, so a tile's locals
// (x_s, lambda_s, bbar_s, gidx) are contiguous and lane-indexed.
// The global update reads the copies of global i through a CSR list
// (gptr/gcol) in canonical order; invk = 1/k_i and cik = c_i/k_i carry
// (B^T B)^{-1} and (B^T B)^{-1} c of Eq. (global_sparse).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.hpp"

namespace opf {

Packed pack(const Model& M, const std::vector<Operator>& ops) {
    Packed K;
    K.ng = M.n;
    K.ncomp = (int)M.comps.size();
    std::vector<int64_t> cptr(K.ncomp + 1, 0);
    for (int s = 0; s < K.ncomp; ++s) {
        cptr[s + 1] = cptr[s] + M.comps[s].n();
        K.sum_n2 += (int64_t)M.comps[s].n() * M.comps[s].n();
        K.max_n = std::max(K.max_n, M.comps[s].n());
    }
    if (cptr[K.ncomp] > INT32_MAX / 2) throw Error(OPF_ERR_INVALID_ARG, "problem too large");
    K.nl = (int)cptr[K.ncomp];
    if (K.max_n > 256) throw Error(OPF_ERR_INVALID_ARG, "a component has more than 256 local variables");

    // component order: by decreasing n, canonical within a size
    std::vector<int> order(K.ncomp);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return M.comps[a].n() > M.comps[b].n(); });

    K.dev_of_canon.assign(K.nl, -1);
    K.canon_of_dev.assign(K.nl, -1);
    int loc = 0;
    int64_t mat = 0;
    size_t pos = 0;
    while (pos < order.size()) {
        const int n = M.comps[order[pos]].n();
        if (n == 0) { ++pos; continue; }
        int k = n <= 32 ? 32 / n : 1;
        size_t end = pos;
        while (end < order.size() && (int)(end - pos) < k && M.comps[order[end]].n() == n) ++end;
        const int kk = (int)(end - pos);
        mat = (mat + 3) & ~int64_t(3);           // 32-byte aligned tile start (f64)
        Tile t;
        t.n = n; t.ncomp = kk; t.loc0 = loc;
        if (mat > INT32_MAX) throw Error(OPF_ERR_INVALID_ARG, "problem too large");
        t.mat0 = (int32_t)mat;
        K.tiles.push_back(t);
        const int L = kk * n;
        K.P.resize((size_t)mat + (size_t)n * (n <= 32 ? L : n), 0.0);
        for (int g = 0; g < kk; ++g) {
            const int s = order[pos + g];
            const Operator& op = ops[s];
            for (int r = 0; r < n; ++r) {
                K.dev_of_canon[cptr[s] + r] = loc + g * n + r;
                K.canon_of_dev[loc + g * n + r] = (int32_t)(cptr[s] + r);
            }
            for (int c = 0; c < n; ++c)
                for (int r = 0; r < n; ++r) {
                    const double v = op.P[(size_t)c * n + r];
                    if (n <= 32) K.P[(size_t)mat + (size_t)c * L + g * n + r] = v;
                    else K.P[(size_t)mat + (size_t)c * n + r] = v;
                }
        }
        mat += (int64_t)n * (n <= 32 ? L : n);
        loc += L;
        pos = end;
    }
    K.mat_elems = (int64_t)K.P.size();

    // local vectors in device order
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
    // CSR of copies, canonical order
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
    return K;
}

}  // namespace opf
