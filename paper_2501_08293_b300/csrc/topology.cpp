// Topology changes of an existing problem: a line switched in or out of
// service (opf_set_line_status).
//
// A switch changes the set of global variables (the line's flows appear or
// disappear) and the rows of the components at the line's ends, so the
// problem is rebuilt: the model is assembled from the stored records with
// the new service state, and the operators of Eq. (closed_2) are
// recomputed only for components whose rows changed (the line itself and
// the nodes at its ends; a component with the same rows has the same
// operator, it is only renumbered).  The new layout is uploaded and the
// iterate and duals are carried over on the device for every local copy
// whose component and global variable exist on both sides (identified by
// element and phase, not by index); new copies start from the initial
// point of Section V-A.
#include <cuda_runtime.h>

#include <map>
#include <unordered_map>
#include <utility>

#include "problem.hpp"

namespace opf {
void device_upload(opf_problem* p, void* arena, size_t bytes, cudaStream_t s);
void device_warm_transfer(opf_problem* dst, const opf_problem* src, const std::vector<int32_t>& map, cudaStream_t s);
void device_free(opf_problem* p);

namespace {

// Identity of a global variable independent of the numbering: kind, element, phase.
std::vector<int64_t> global_keys(const Model& M) {
    std::vector<int64_t> key(M.n, -1);
    auto put = [&](const std::vector<int32_t>& idx, int64_t kind) {
        for (size_t q = 0; q < idx.size(); ++q)
            if (idx[q] >= 0) key[idx[q]] = (kind << 40) | ((int64_t)(q / 3) << 4) | (int64_t)(q % 3);
    };
    put(M.w_idx, 1); put(M.pg_idx, 2); put(M.qg_idx, 3);
    put(M.pij_idx, 4); put(M.qij_idx, 5); put(M.pji_idx, 6); put(M.qji_idx, 7);
    put(M.pb_idx, 8); put(M.qb_idx, 9); put(M.pd_idx, 10); put(M.qd_idx, 11);
    return key;
}

struct CudaDeviceScope {
    int prev = -1;
    explicit CudaDeviceScope(int dev) {
        if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~CudaDeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// New device local -> old device local for copies of the same global
// variable in the same component (kind, element); -1 elsewhere.
std::vector<int32_t> warm_map(const opf_problem* dst, const opf_problem* src) {
    const std::vector<int64_t> kd = global_keys(dst->model), ks = global_keys(src->model);
    std::map<std::pair<int, int>, int> src_comp;
    for (int s = 0; s < (int)src->model.comps.size(); ++s)
        src_comp[{src->model.comps[s].kind, src->model.comps[s].index}] = s;
    std::vector<int32_t> map(dst->pk.nl, -1);
    for (int s = 0; s < (int)dst->model.comps.size(); ++s) {
        const Component& C = dst->model.comps[s];
        auto it = src_comp.find({C.kind, C.index});
        if (it == src_comp.end()) continue;
        const Component& D = src->model.comps[it->second];
        std::unordered_map<int64_t, int> pos;
        for (int r = 0; r < D.n(); ++r) pos[ks[D.gvars[r]]] = r;
        for (int r = 0; r < C.n(); ++r) {
            auto f = pos.find(kd[C.gvars[r]]);
            if (f == pos.end()) continue;
            map[dst->pk.dev_of_canon[dst->canon_comp_ptr[s] + r]] =
                src->pk.dev_of_canon[src->canon_comp_ptr[it->second] + f->second];
        }
    }
    return map;
}

void finish_host(opf_problem* p, const Model* old_model, const std::vector<Operator>* old_ops, int* recomputed) {
    std::map<std::pair<int, int>, int> old_at;
    if (old_model)
        for (int s = 0; s < (int)old_model->comps.size(); ++s)
            old_at[{old_model->comps[s].kind, old_model->comps[s].index}] = s;
    p->ops.clear();
    p->ops.reserve(p->model.comps.size());
    p->canon_comp_ptr.assign(1, 0);
    p->m_reduced.clear();
    p->n_rows = p->n_rows_reduced = 0;
    int fresh = 0;
    for (const Component& c : p->model.comps) {
        const Operator* same = nullptr;
        if (old_model) {
            auto it = old_at.find({c.kind, c.index});
            if (it != old_at.end()) {
                const Component& d = old_model->comps[it->second];
                if (d.m == c.m && d.n() == c.n() && d.A == c.A && d.b == c.b) same = &(*old_ops)[it->second];
            }
        }
        if (same) {
            p->ops.push_back(*same);
        } else {
            p->ops.push_back(make_operator(c));
            ++fresh;
        }
        p->m_reduced.push_back(p->ops.back().m_reduced);
        p->canon_comp_ptr.push_back(p->canon_comp_ptr.back() + c.n());
        p->n_rows += c.m;
        p->n_rows_reduced += p->ops.back().m_reduced;
    }
    p->pk = pack(p->model, p->ops, p->create_chunks);
    if (recomputed) *recomputed = fresh;
}

void set_line_status(opf_problem* p, int line, bool in_service, cudaStream_t s, int* recomputed) {
    if (line < 0 || line >= (int)p->rec_line.size()) throw Error(OPF_ERR_INVALID_ARG, "line index out of range");
    if ((p->rec_line[line].in_service != 0) == in_service) {
        if (recomputed) *recomputed = 0;
        return;
    }
    std::vector<opf_line> lines = p->rec_line;
    lines[line].in_service = in_service ? 1 : 0;
    opf_problem* q = new opf_problem();
    try {
        q->model = build_model(p->rec_bus.data(), (int)p->rec_bus.size(), lines.data(), (int)lines.size(),
                               p->rec_gen.data(), (int)p->rec_gen.size(), p->rec_load.data(), (int)p->rec_load.size());
        if (p->model.decomposition == OPF_DECOMP_PAPER) paper_decomposition(q->model);
        q->create_chunks = p->create_chunks;
        finish_host(q, &p->model, &p->ops, recomputed);
        q->rec_bus = p->rec_bus;
        q->rec_line = std::move(lines);
        q->rec_gen = p->rec_gen;
        q->rec_load = p->rec_load;
        if (p->uploaded) {
            CudaDeviceScope dev(p->device);
            device_upload(q, nullptr, 0, s);
            device_warm_transfer(q, p, warm_map(q, p), s);
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) throw Error(OPF_ERR_CUDA, std::string("set_line_status: ") + cudaGetErrorString(e));
            q->timeout_ns = p->timeout_ns;
            q->force_variant = p->force_variant;
            q->profile_phases = p->profile_phases;
            device_free(p);
            p->uploaded = false;
        }
    } catch (...) {
        if (q->uploaded) device_free(q);
        delete q;
        throw;
    }
    std::swap(*p, *q);
    delete q;
}

}  // namespace opf
