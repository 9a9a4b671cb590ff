// The opf_problem handle and the device-side control block.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <utility>

#include "internal.hpp"

namespace opf {

// Device control block: solve parameters written by the host before a
// solve, iteration state and residuals written by the kernels.
struct Ctl {
    double rho, inv_rho, eps_abs_prim, eps_abs_dual, eps_rel;
    int32_t criterion;
    int32_t max_iter;     // absolute bound on iter for this solve
    int32_t K;            // check interval
    int32_t iter;         // iterations since the last cold start
    int32_t status;       // CTL_*
    int32_t first_rel;
    int32_t stop;
    int32_t checks;
    double pres, dres, eps_prim, eps_dual, objective;
    // persistent engine
    unsigned long long arrive;    // check tickets taken
    unsigned long long timeout_ns;
    int32_t decided;              // checks decided
    int32_t abort;                // a wait gave up: every CTA leaves
    int32_t halt;                 // a check decided to stop (non-blocking checks): CTAs leave
    int32_t skip_block;           // test hook: this CTA withholds its flag (-1: none)
    int32_t timeout_where;        // 1 neighbour wait, 2 check wait, 3 final wait, 4 staging, 5 staging copy never landed,
                                  // 6 operator block of a tile (batched graph engine)
    int32_t profile_phases;       // persistent kernel: accumulate per-phase time
    int32_t adaptive;             // residual balancing on
    int32_t rho_changes;
    double rb_mu, rb_tau;
    int32_t res_form;             // OPF_RES_PAPER or OPF_RES_TEXTBOOK (graph / host-loop engines)
    int32_t _pad_res;
};
enum { CTL_RUNNING = 0, CTL_CONVERGED = 1, CTL_MAXITER = 2, CTL_NUMERIC = 3, CTL_TIMEOUT = 4 };

template <typename T>
struct View {
    const T* lo;
    const T* hi;
    const T* invk;
    const T* cik;
    T* zg;
    const int32_t* gptr;
    const int32_t* gcol;
    T* xl;
    T* lam;
    T* xl2;           // ping-pong partners of xl, lam (persistent engine)
    T* lam2;
    const T* bbar;
    const T* xl0;
    const int32_t* gidx;
    const int32_t* meta;
    const Tile* tiles;
    const BlockInfo* blocks;
    const int32_t* halo_gid;
    const uint8_t* halo_own;
    const int32_t* nbrs;
    const int32_t* hcp;
    const int32_t* hci;
    const int32_t* hcx;               // copy lists with copies of other chunks as ~slot (gathered exchange)
    const int32_t* ext;               // per chunk: device locals of other chunks it reads
    int32_t* flags;                   // per chunk: iteration flag (global-memory kernel) or claim word (shared-memory kernel)
    const T* P;
    const double* cost;
    double* partials;
    unsigned long long* phase;        // per CTA: interior, wait, boundary, release+check (ns)
    unsigned long long* mbox;         // tagged boundary values, 2 slots x nl x (1 f32 | 2 f64) words
    Ctl* ctl;
    double* tdz;                      // textbook residual form: x_s - x_s(prev) per local on a check iteration
    double* tpart;                    // textbook residual form: 2 partial sums per global-update block
    int32_t ng, nl, nblocks, nzb;
};

struct DevPrec {            // one precision's arrays
    void* lo = nullptr; void* hi = nullptr; void* invk = nullptr; void* cik = nullptr; void* zg = nullptr;
    void* xl = nullptr; void* lam = nullptr; void* xl2 = nullptr; void* lam2 = nullptr;
    void* bbar = nullptr; void* xl0 = nullptr; void* P = nullptr;
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace opf

struct opf_batch {
    std::vector<opf_problem*> probs;
    void* dev_buf = nullptr;          // views, CTA map, control read-back (cudaMallocAsync)
    size_t dev_bytes = 0;
    char* host_buf = nullptr;         // pinned staging of the same
    size_t host_bytes = 0;
    int device = -1;
    cudaEvent_t done = nullptr;       // end of the last launched batch
    int n_launched = 0;
    // batched graph engine: cached while-node graph and what it was built for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* g_buf = nullptr;
    int g_n = 0, g_nz = 0, g_nx = 0, g_K = 0, g_prec = -1, g_ni = 0;
    // persistent engine: the flag clear, the cooperative launch and the
    // finish kernel captured once as a graph, and what it was captured for
    cudaGraph_t pgraph = nullptr;
    cudaGraphExec_t pexec = nullptr;
    const void* p_buf = nullptr;
    int p_n = 0, p_nx = 0, p_nz = 0, p_prec = -1, p_var = 0;
    unsigned char p_plan[128] = {};
};

struct opf_problem {
    // the records the problem was built from (kept for topology changes)
    std::vector<opf_bus> rec_bus;
    std::vector<opf_line> rec_line;
    std::vector<opf_gen> rec_gen;
    std::vector<opf_load> rec_load;
    int create_chunks = 0;              // chunk option of the create call
    opf::Model model;
    std::vector<opf::Operator> ops;
    opf::Packed pk;
    std::vector<int32_t> canon_comp_ptr;
    std::vector<int32_t> m_reduced;
    int64_t n_rows = 0, n_rows_reduced = 0;

    // device side
    bool uploaded = false;
    bool owns_arena = false;
    int device = -1;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    opf::DevPrec d64, d32;
    int32_t* gptr = nullptr;
    int32_t* gcol = nullptr;
    int32_t* gidx = nullptr;
    int32_t* meta = nullptr;
    opf::Tile* tiles = nullptr;
    opf::BlockInfo* blocks = nullptr;
    int32_t* halo_gid = nullptr;
    uint8_t* halo_own = nullptr;
    int32_t* nbrs = nullptr;
    int32_t* hcp = nullptr;
    int32_t* hci = nullptr;
    int32_t* hcx = nullptr;
    int32_t* ext = nullptr;
    int32_t* flags = nullptr;
    double* cost = nullptr;
    double* partials = nullptr;
    double* tdz = nullptr;
    double* tpart = nullptr;
    // graph engine's tile-parallel local update: the problem's View in both
    // precisions (device copies) and its work items of tiles
    void* xt_views = nullptr;
    void* xt_items = nullptr;
    int xt_nitems = 0;
    unsigned long long* phase = nullptr;
    unsigned long long* mbox = nullptr;
    opf::Ctl* ctl = nullptr;
    opf::Ctl* ctl_host = nullptr;       // pinned mirror
    int cur_prec = 0;                   // precision holding the current state
    bool cold = true;                   // state is at the initial point
    unsigned long long timeout_ns = 2000000000ull;   // bounded waits (persistent engine)
    int skip_block = -1;                              // test hook
    int force_variant = 0;                            // persistent kernel: 0 auto, 1 global, 2 shared, 3 shared with per-entry exchange
    int profile_phases = 0;
    std::map<std::pair<int, int>, opf::GraphEntry> graphs;   // (precision + 2 * residual form, K)
};

namespace opf {
// Operators (reusing those of old_model's components with unchanged rows),
// canonical offsets, ranks and the device layout of p->model.
void finish_host(opf_problem* p, const Model* old_model, const std::vector<Operator>* old_ops, int* recomputed);
void set_line_status(opf_problem* p, int line, bool in_service, cudaStream_t s, int* recomputed);
std::vector<int32_t> warm_map(const opf_problem* dst, const opf_problem* src);
}  // namespace opf
