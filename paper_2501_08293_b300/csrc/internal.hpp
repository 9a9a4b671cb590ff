// Internal host-side structures of libopf_admm (not part of the C ABI).
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "opf_admm.h"

namespace opf {

struct Error : std::runtime_error {
    int32_t status;
    Error(int32_t s, const std::string& m) : std::runtime_error(m), status(s) {}
};

enum CompKind { COMP_BUS = 0, COMP_LINE = 1, COMP_LOAD = 2, COMP_GEN = 3 };

// One fine-grained component of Eq. (OurModel): its local variables (as
// global indices, i.e. the 0-1 map B_s) and its equality rows A_s x_s = b_s
// (row-major m x n).
struct Component {
    int kind = 0;
    int index = 0;
    std::vector<int32_t> gvars;
    int m = 0;
    std::vector<double> A;
    std::vector<double> b;
    int n() const { return (int)gvars.size(); }
};

// Global vector of Eq. (LP_model) plus lookups for unscattering.
struct Model {
    int n = 0;
    std::vector<double> lo, hi, c;
    std::vector<uint8_t> is_w;                // squared voltage magnitude
    std::vector<Component> comps;             // canonical order
    int n_bus = 0, n_line = 0, n_gen = 0, n_load = 0;
    std::vector<int32_t> line_from, line_to, load_bus, gen_bus;   // topology
    // element lookups, -1 for absent phases / out-of-service lines
    std::vector<int32_t> w_idx, pg_idx, qg_idx;                 // *3
    std::vector<int32_t> pij_idx, qij_idx, pji_idx, qji_idx;    // n_line*3
    std::vector<int32_t> pb_idx, qb_idx, pd_idx, qd_idx;        // n_load*3
    int decomposition = OPF_DECOMP_FINE;
};

// Closed-form operator of one component (Eq. closed_2), P = -Abar.
struct Operator {
    int n = 0;
    int m_reduced = 0;
    std::vector<double> P;      // n x n, symmetric
    std::vector<double> bbar;   // n
};

// Warps per CTA of the local-update kernels; the packer balances tiles over
// this many warps (a tile at chunk position q is run by warp q % kTileWarps).
constexpr int kTileWarps = 8;

// Work item of the local-update kernel: one warp.  Small tiles hold whole
// components (sizes n_g <= 32, sum n_g = L <= 32 lanes, nmax = max n_g);
// a big tile holds one component with n > 32 (flag big = 1); L = 0 marks an
// empty padding tile.
struct Tile {
    int32_t loc0;   // first local (device order)
    int32_t mat0;   // first operator element
    int16_t L;      // lanes used (small) or n (big)
    int16_t nmax;   // loop length: max n_g over the tile's components
    int32_t big;
};

// One CTA's share of a problem: a contiguous chunk of the component order
// (a DFS over the feeder, so chunks are subtrees with few neighbours).
struct BlockInfo {
    int32_t tile0, tile1;   // tiles [tile0, tile1); [tile0, tileb) are interior
    int32_t halo0, halo1;   // globals read by the chunk [halo0, halo1); [halo0, halob) are interior
    int32_t nbr0, nbr1;     // neighbour CTAs (share a global) [nbr0, nbr1)
    int32_t loc0, loc1;     // locals [loc0, loc1)
    int32_t mat0, mat1;     // operator elements [mat0, mat1) of the chunk's tiles
    int32_t cp0, cp1;       // copy list entries of the chunk's halo [cp0, cp1)
    int32_t tileb, halob;   // first boundary tile / halo entry
    int32_t ext0, ext1;     // copies of other chunks that the chunk reads [ext0, ext1) (device locals)
};

// Device-ordered problem, ready to upload.
struct Packed {
    int ng = 0, nl = 0, ncomp = 0;
    int nblocks = 0;
    std::vector<Tile> tiles;
    std::vector<BlockInfo> blocks;
    std::vector<int32_t> halo_gid;       // global id per halo entry
    std::vector<uint8_t> halo_own;       // 1 if this chunk writes x_i (first copy)
    std::vector<int32_t> nbrs;
    std::vector<int32_t> meta;           // per local: hidx | n << 16 | base lane << 24 | exported << 30
    std::vector<int32_t> hcp;            // per halo entry (+1): start of its copy list in hci
    std::vector<int32_t> hci;            // copy of a halo global: chunk-relative local (>= 0) or ~device local (< 0)
    std::vector<int32_t> hcx;            // the same, copies of other chunks as ~slot in the chunk's ext list
    std::vector<int32_t> ext;            // per chunk: device locals of other chunks it reads, in copy-list order
    std::vector<int32_t> dev_of_canon;   // local: canonical -> device
    std::vector<int32_t> canon_of_dev;   // local: device -> canonical
    std::vector<int32_t> gidx;           // device order
    std::vector<int32_t> gptr, gcol;     // CSR: global -> device locals
    std::vector<double> invk, cik;       // 1/k_i, c_i/k_i
    std::vector<double> bbar, xl0;       // device order
    std::vector<double> P;               // operator elements, tile layout
    std::vector<int32_t> comp_tile;      // tile holding each (canonical) component
    int64_t mat_elems = 0;
    int64_t sum_n2 = 0;
    int max_n = 0;
    int max_halo = 0;                    // largest chunk halo (shared memory)
    int max_loc = 0;                     // largest chunk local count
    int max_mat = 0;                     // largest chunk operator span (elements)
    int max_copies = 0;                  // largest chunk halo copy list
    int max_ext = 0;                     // most copies of other chunks read by one chunk
    int max_big = 0;                     // largest component with n > 32 (0: none)
    int max_tiles = 0;                   // most tiles in one chunk
};

Model build_model(const opf_bus* buses, int nb, const opf_line* lines, int nl,
                  const opf_gen* gens, int ng, const opf_load* loads, int nd);
// Section V-A: replace M's fine components by nodes (bus + its loads + its
// generators) and lines, each leaf node (one in-service line) combined with
// its line; canonical order: non-leaf nodes, then lines.
void paper_decomposition(Model& M);
// Rows and locals of the parts stacked into one component (first copy of a
// global kept).
Component combine_parts(int kind, int index, const std::vector<const Component*>& parts);
Operator make_operator(const Component& c);
// Line component of Eq. (power_flow_eqns) for in-service line e on the
// global indices of M; line_update validates a new record for line e (same
// ends, phases and service state) and returns its component.
Component line_component(const Model& M, const opf_line& L, int e);
Component line_update(const Model& M, const opf_line& L, int e);
Packed pack(const Model& m, const std::vector<Operator>& ops, int nblocks_hint = 0);
// Automatic chunking (nblocks_hint = 0): chunk size in units of
// n_s^2 + 4 n_s + 16 and the chunk cap for a feeder of n_bus buses on the
// current device, from the tuning table (default 4096, 296).
void auto_chunking(int n_bus, int64_t* work_per_chunk, int* max_chunks);
void set_last_error(const std::string& m);

}  // namespace opf
