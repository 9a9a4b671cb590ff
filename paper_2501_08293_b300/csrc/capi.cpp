// extern "C" entry points of libopf_admm (declared in include/opf_admm.h).
// Every call converts internal exceptions into status codes and records a
// message retrievable with opf_last_error() on the same thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "problem.hpp"

namespace opf {
size_t device_bytes(const opf_problem* p);
void device_upload(opf_problem* p, void* arena, size_t bytes, cudaStream_t s);
int32_t device_solve(opf_problem* p, const opf_params& prm, cudaStream_t s, opf_info* info);
void device_get_state(const opf_problem* p, double* xg, double* xl, double* lam, cudaStream_t s);
void device_set_state(opf_problem* p, const double* xl, const double* lam, cudaStream_t s);
void device_free(opf_problem* p);
int device_auto_engine(const opf_problem* p, int precision);
void device_profile(opf_problem* p, const opf_params& prm, int reps, cudaStream_t s, double* us);
void device_batch_solve(opf_batch* B, const opf_params* prm, int nprm, cudaStream_t s, opf_info* infos);
void device_batch_profile(opf_batch* B, const opf_params& prm, int reps, cudaStream_t s, double* us);
void device_profile_persistent(opf_problem* p, const opf_params& prm, int iters, cudaStream_t s, double* out,
                               double* per_cta);
void device_batch_free(opf_batch* B);
int device_batch_capacity(int precision);
int device_batch_auto_engine(const opf_batch* B, int precision);
void residuals_noalloc(const double* v, const double* z, const double* zp, const double* lam, long long n,
                       double rho, double eps_rel, double* out, cudaStream_t s);
opf_scenarios* scenarios_create(const opf_bus* buses, int nb, const opf_line* lines, int nl, const opf_gen* gens,
                                int ng, const opf_load* loads, int nd, int S);
void scenarios_destroy(opf_scenarios* sc);
void scenarios_solve(opf_scenarios* sc, const opf_params& prm, cudaStream_t s, opf_info* infos);
void scenarios_get_state(const opf_scenarios* sc, int k, double* xg, double* xl, double* lam, cudaStream_t s);
void scenarios_dims(const opf_scenarios* sc, int32_t* n_global, int32_t* n_local, int64_t* device_bytes);
void scenarios_profile(opf_scenarios* sc, const opf_params& prm, int reps, cudaStream_t s, double* us);
void scenarios_set_xupdate(opf_scenarios* sc, int kind);
void device_reprecompute(opf_problem* p, const std::vector<int>& comps, cudaStream_t s);
void device_update_bounds(opf_problem* p, const std::vector<std::pair<int, int>>& ranges, cudaStream_t s);
}  // namespace opf

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace opf {
void set_last_error(const std::string& m) { g_last_error = m; }
}  // namespace opf

namespace {

template <typename F>
int32_t guarded(F&& f) {
    try {
        g_last_error.clear();
        return f();
    } catch (const opf::Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return OPF_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return OPF_ERR_INVALID_ARG;
    } catch (...) {
        g_last_error = "unknown error";
        return OPF_ERR_INVALID_ARG;
    }
}
}  // namespace

extern "C" {

int32_t opf_abi_version(void) { return OPF_ABI_VERSION; }

size_t opf_record_size(int32_t which) {
    switch (which) {
        case 0: return sizeof(opf_bus);
        case 1: return sizeof(opf_line);
        case 2: return sizeof(opf_gen);
        case 3: return sizeof(opf_load);
        case 4: return sizeof(opf_params);
        case 5: return sizeof(opf_info);
        case 6: return sizeof(opf_dims);
        default: return 0;
    }
}

const char* opf_status_string(int32_t s) {
    switch (s) {
        case OPF_OK: return "OPF_OK";
        case OPF_NOT_CONVERGED: return "OPF_NOT_CONVERGED";
        case OPF_ERR_INVALID_ARG: return "OPF_ERR_INVALID_ARG";
        case OPF_ERR_INCONSISTENT: return "OPF_ERR_INCONSISTENT";
        case OPF_ERR_NUMERIC: return "OPF_ERR_NUMERIC";
        case OPF_ERR_OOM: return "OPF_ERR_OOM";
        case OPF_ERR_CUDA: return "OPF_ERR_CUDA";
        case OPF_ERR_TIMEOUT: return "OPF_ERR_TIMEOUT";
        case OPF_ERR_STATE: return "OPF_ERR_STATE";
        default: return "OPF_UNKNOWN_STATUS";
    }
}

const char* opf_last_error(void) { return g_last_error.c_str(); }

void opf_params_default(opf_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->rho = 100.0;
    p->eps_abs_prim = 1e-4;
    p->eps_abs_dual = 1e-4;
    p->eps_rel = 1e-3;
    p->criterion = OPF_CRIT_ABS;
    p->max_iter = 1000000;
    p->check_every = 50;
    p->precision = OPF_FP64;
    p->residual_form = OPF_RES_PAPER;
    p->warm_start = 0;
    p->engine = OPF_ENGINE_AUTO;
    p->adaptive_rho = 0;
    p->rb_mu = 10.0;
    p->rb_tau = 2.0;
}

int32_t opf_problem_create_ex(const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                              const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                              const opf_create_options* options, opf_problem** out) {
    return guarded([&]() -> int32_t {
        if (!out) throw opf::Error(OPF_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        const int chunks = options ? options->chunks : 0;
        const int decomp = options ? options->decomposition : OPF_DECOMP_FINE;
        if (chunks < 0 || chunks > 65536) throw opf::Error(OPF_ERR_INVALID_ARG, "chunks out of [0, 65536]");
        if (decomp != OPF_DECOMP_FINE && decomp != OPF_DECOMP_PAPER)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad decomposition");
        opf_problem* p = new opf_problem();
        try {
            p->model = opf::build_model(buses, n_bus, lines, n_line, gens, n_gen, loads, n_load);
            if (decomp == OPF_DECOMP_PAPER) opf::paper_decomposition(p->model);
            p->create_chunks = chunks;
            opf::finish_host(p, nullptr, nullptr, nullptr);
            p->rec_bus.assign(buses, buses + n_bus);
            p->rec_line.assign(lines, lines + n_line);
            p->rec_gen.assign(gens, gens + n_gen);
            p->rec_load.assign(loads, loads + n_load);
        } catch (...) {
            delete p;
            throw;
        }
        *out = p;
        return OPF_OK;
    });
}

int32_t opf_problem_create(const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                           const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                           opf_problem** out) {
    return opf_problem_create_ex(buses, n_bus, lines, n_line, gens, n_gen, loads, n_load, nullptr, out);
}

int32_t opf_update_lines(opf_problem* p, const int32_t* line_idx, const opf_line* records, int32_t count,
                         void* stream) {
    return guarded([&]() -> int32_t {
        if (!p || (count > 0 && (!line_idx || !records)) || count < 0)
            throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        opf::Model& M = p->model;
        // component of each line (canonical order)
        std::vector<int> line_comp(M.n_line, -1);
        for (size_t c = 0; c < M.comps.size(); ++c)
            if (M.comps[c].kind == opf::COMP_LINE) line_comp[M.comps[c].index] = (int)c;
        // validate everything before changing anything
        std::vector<opf::Component> fresh;
        fresh.reserve(count);
        for (int k = 0; k < count; ++k) {
            const int e = line_idx[k];
            if (e < 0 || e >= M.n_line || line_comp[e] < 0)
                throw opf::Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": no in-service line there");
            const opf::Component& cur = M.comps[line_comp[e]];
            opf::Component nc = opf::line_update(M, records[k], e);
            if (M.decomposition == OPF_DECOMP_PAPER) {
                // a line with leaf ends: the line's locals and rows come first
                // in its component; only those rows change
                if (cur.n() < nc.n() || cur.m < nc.m || !std::equal(nc.gvars.begin(), nc.gvars.end(), cur.gvars.begin()))
                    throw opf::Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": structure differs");
                opf::Component merged = cur;
                for (int r = 0; r < nc.m; ++r) {
                    for (int c = 0; c < cur.n(); ++c)
                        merged.A[(size_t)r * cur.n() + c] = c < nc.n() ? nc.A[(size_t)r * nc.n() + c] : 0.0;
                    merged.b[r] = nc.b[r];
                }
                nc = std::move(merged);
            } else if (nc.gvars != cur.gvars) {
                throw opf::Error(OPF_ERR_INVALID_ARG, "line " + std::to_string(e) + ": structure differs");
            }
            fresh.push_back(std::move(nc));
        }
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "update before upload");
        std::vector<int> comps;
        std::vector<std::pair<int, int>> ranges;
        for (int k = 0; k < count; ++k) {
            const int e = line_idx[k];
            const int c = line_comp[e];
            M.comps[c].A = fresh[k].A;
            M.comps[c].b = fresh[k].b;
            M.comps[c].m = fresh[k].m;
            comps.push_back(c);
            // flow bounds: p_ij, q_ij, p_ji, q_ji on the line's phases (contiguous globals)
            const opf_line& L = records[k];
            int g0 = INT32_MAX, g1 = -1;
            for (int ph = 0; ph < 3; ++ph) {
                if (M.pij_idx[3 * e + ph] < 0) continue;
                M.lo[M.pij_idx[3 * e + ph]] = L.p_lo[ph]; M.hi[M.pij_idx[3 * e + ph]] = L.p_hi[ph];
                M.lo[M.pji_idx[3 * e + ph]] = L.p_lo[ph]; M.hi[M.pji_idx[3 * e + ph]] = L.p_hi[ph];
                M.lo[M.qij_idx[3 * e + ph]] = L.q_lo[ph]; M.hi[M.qij_idx[3 * e + ph]] = L.q_hi[ph];
                M.lo[M.qji_idx[3 * e + ph]] = L.q_lo[ph]; M.hi[M.qji_idx[3 * e + ph]] = L.q_hi[ph];
                for (int32_t gi : {M.pij_idx[3 * e + ph], M.pji_idx[3 * e + ph], M.qij_idx[3 * e + ph],
                                   M.qji_idx[3 * e + ph]}) {
                    g0 = std::min(g0, (int)gi);
                    g1 = std::max(g1, (int)gi + 1);
                }
            }
            ranges.emplace_back(g0, g1);
        }
        opf::device_update_bounds(p, ranges, (cudaStream_t)stream);
        opf::device_reprecompute(p, comps, (cudaStream_t)stream);
        for (int k = 0; k < count; ++k) p->rec_line[line_idx[k]] = records[k];
        return OPF_OK;
    });
}

int32_t opf_set_line_status(opf_problem* p, int32_t line, int32_t in_service, void* stream, int32_t* n_recomputed) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (in_service != 0 && in_service != 1) throw opf::Error(OPF_ERR_INVALID_ARG, "in_service must be 0 or 1");
        int rec = 0;
        opf::set_line_status(p, line, in_service != 0, (cudaStream_t)stream, &rec);
        if (n_recomputed) *n_recomputed = rec;
        return OPF_OK;
    });
}

int32_t opf_get_dims(const opf_problem* p, opf_dims* d) {
    return guarded([&]() -> int32_t {
        if (!p || !d) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        std::memset(d, 0, sizeof(*d));
        d->n_global = p->pk.ng;
        d->n_local = p->pk.nl;
        d->n_comp = p->pk.ncomp;
        d->n_rows = (int32_t)p->n_rows;
        d->n_rows_reduced = (int32_t)p->n_rows_reduced;
        d->max_n = p->pk.max_n;
        d->n_tiles = (int32_t)p->pk.tiles.size();
        d->n_blocks = p->pk.nblocks;
        d->sum_n2 = p->pk.sum_n2;
        d->device_bytes = (int64_t)opf::device_bytes(p);
        d->max_chunk_locals = p->pk.max_loc;
        d->max_chunk_halo = p->pk.max_halo;
        d->max_chunk_operator = p->pk.max_mat;
        d->max_chunk_copies = p->pk.max_copies;
        return OPF_OK;
    });
}

int32_t opf_problem_upload(opf_problem* p, void* arena, size_t arena_bytes, void* stream) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        opf::device_upload(p, arena, arena_bytes, (cudaStream_t)stream);
        return OPF_OK;
    });
}

int32_t opf_admm_solve(opf_problem* p, const opf_params* prm, void* stream, opf_info* info) {
    return guarded([&]() -> int32_t {
        if (!p || !prm) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "solve before upload");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho)) throw opf::Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
        if (prm->check_every < 1 || prm->check_every > 4096) throw opf::Error(OPF_ERR_INVALID_ARG, "check_every out of [1, 4096]");
        if (prm->max_iter < 0) throw opf::Error(OPF_ERR_INVALID_ARG, "max_iter < 0");
        if (prm->criterion < 0 || prm->criterion > 3) throw opf::Error(OPF_ERR_INVALID_ARG, "bad criterion");
        if (prm->precision != OPF_FP64 && prm->precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        if (prm->residual_form != OPF_RES_PAPER && prm->residual_form != OPF_RES_TEXTBOOK)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad residual form");
        if (prm->engine < 0 || prm->engine > 3) throw opf::Error(OPF_ERR_INVALID_ARG, "bad engine");
        if (prm->adaptive_rho && !(prm->rb_mu > 1.0 && prm->rb_tau > 1.0))
            throw opf::Error(OPF_ERR_INVALID_ARG, "residual balancing needs rb_mu > 1 and rb_tau > 1");
        return opf::device_solve(p, *prm, (cudaStream_t)stream, info);
    });
}

int32_t opf_get_state(const opf_problem* p, double* xg, double* xl, double* lam, void* stream) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "no device state");
        opf::device_get_state(p, xg, xl, lam, (cudaStream_t)stream);
        return OPF_OK;
    });
}

int32_t opf_set_state(opf_problem* p, const double* xl, const double* lam, void* stream) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "no device state");
        opf::device_set_state(p, xl, lam, (cudaStream_t)stream);
        return OPF_OK;
    });
}

int32_t opf_get_structure(const opf_problem* p, int32_t* comp_ptr, int32_t* comp_kind, int32_t* comp_index,
                          int32_t* gidx, int32_t* m_reduced) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        const int S = (int)p->model.comps.size();
        if (comp_ptr) std::memcpy(comp_ptr, p->canon_comp_ptr.data(), (S + 1) * sizeof(int32_t));
        for (int s = 0; s < S; ++s) {
            const auto& c = p->model.comps[s];
            if (comp_kind) comp_kind[s] = c.kind;
            if (comp_index) comp_index[s] = c.index;
            if (m_reduced) m_reduced[s] = p->m_reduced[s];
            if (gidx)
                for (int r = 0; r < c.n(); ++r) gidx[p->canon_comp_ptr[s] + r] = c.gvars[r];
        }
        return OPF_OK;
    });
}

int32_t opf_get_solution(const opf_problem* p, double* w, double* pg, double* qg, double* p_ij, double* q_ij,
                         double* p_ji, double* q_ji, double* pd, double* qd, double* pb, double* qb, void* stream) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "no device state");
        std::vector<double> x(p->pk.ng);
        opf::device_get_state(p, x.data(), nullptr, nullptr, (cudaStream_t)stream);
        const opf::Model& M = p->model;
        auto scat = [&](double* dst, const std::vector<int32_t>& idx) {
            if (!dst) return;
            for (size_t k = 0; k < idx.size(); ++k) dst[k] = idx[k] >= 0 ? x[idx[k]] : NAN;
        };
        scat(w, M.w_idx); scat(pg, M.pg_idx); scat(qg, M.qg_idx);
        scat(p_ij, M.pij_idx); scat(q_ij, M.qij_idx); scat(p_ji, M.pji_idx); scat(q_ji, M.qji_idx);
        scat(pd, M.pd_idx); scat(qd, M.qd_idx); scat(pb, M.pb_idx); scat(qb, M.qb_idx);
        return OPF_OK;
    });
}

int32_t opf_profile_kernels(opf_problem* p, const opf_params* prm, int32_t reps, void* stream, double* us) {
    return guarded([&]() -> int32_t {
        if (!p || !prm || !us) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "profile before upload");
        if (reps < 1 || reps > 100000) throw opf::Error(OPF_ERR_INVALID_ARG, "reps out of [1, 100000]");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho)) throw opf::Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
        if (prm->precision != OPF_FP64 && prm->precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        opf::device_profile(p, *prm, reps, (cudaStream_t)stream, us);
        return OPF_OK;
    });
}

int32_t opf_profile_persistent(opf_problem* p, const opf_params* prm, int32_t iters, void* stream, double* out) {
    return guarded([&]() -> int32_t {
        if (!p || !prm || !out) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "profile before upload");
        if (iters < 1) throw opf::Error(OPF_ERR_INVALID_ARG, "iters must be >= 1");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho) || (prm->precision != OPF_FP64 && prm->precision != OPF_FP32) ||
            prm->check_every < 1 || prm->check_every > 4096)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad parameters");
        opf::device_profile_persistent(p, *prm, iters, (cudaStream_t)stream, out, nullptr);
        return OPF_OK;
    });
}

int32_t opf_profile_persistent_ctas(opf_problem* p, const opf_params* prm, int32_t iters, void* stream,
                                    double* per_cta) {
    return guarded([&]() -> int32_t {
        if (!p || !prm || !per_cta) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "profile before upload");
        if (iters < 1) throw opf::Error(OPF_ERR_INVALID_ARG, "iters must be >= 1");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho) || (prm->precision != OPF_FP64 && prm->precision != OPF_FP32) ||
            prm->check_every < 1 || prm->check_every > 4096)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad parameters");
        double agg[8];
        opf::device_profile_persistent(p, *prm, iters, (cudaStream_t)stream, agg, per_cta);
        return OPF_OK;
    });
}

int32_t opf_chunk_stats(const opf_problem* p, int32_t* out) {
    return guarded([&]() -> int32_t {
        if (!p || !out) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        const opf::Packed& k = p->pk;
        for (int b = 0; b < k.nblocks; ++b) {
            const opf::BlockInfo& bi = k.blocks[b];
            int32_t* o = out + (size_t)OPF_CHUNK_STATS * b;
            int tiles = 0, itiles = 0, quads = 0;
            std::vector<int> wq(opf::kTileWarps, 0);
            for (int q = bi.tile0; q < bi.tile1; ++q) {
                const opf::Tile& t = k.tiles[q];
                if (!t.big && t.L == 0) continue;
                const int nq = t.big ? t.L * ((t.L + 3) / 4) / 32 + 1 : (t.nmax + 3) / 4;
                ++tiles;
                itiles += q < bi.tileb;
                quads += nq;
                wq[(q - (q < bi.tileb ? bi.tile0 : bi.tileb)) % opf::kTileWarps] += nq + 2;
            }
            int ext = 0;
            for (int q = bi.cp0; q < bi.cp1; ++q) ext += k.hci[q] < 0;
            o[0] = tiles; o[1] = itiles; o[2] = quads;
            o[3] = *std::max_element(wq.begin(), wq.end());
            o[4] = bi.halo1 - bi.halo0; o[5] = bi.halo1 - bi.halob;
            o[6] = bi.cp1 - bi.cp0; o[7] = ext; o[8] = bi.nbr1 - bi.nbr0; o[9] = bi.loc1 - bi.loc0;
        }
        return OPF_OK;
    });
}

int32_t opf_engine_for(const opf_problem* p, int32_t precision, int32_t* engine) {
    return guarded([&]() -> int32_t {
        if (!p || !engine) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (!p->uploaded) throw opf::Error(OPF_ERR_STATE, "problem not uploaded");
        if (precision != OPF_FP64 && precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        *engine = opf::device_auto_engine(p, precision);
        return OPF_OK;
    });
}

int32_t opf_debug_config(opf_problem* p, int64_t wait_limit_ns, int32_t withhold_block, int32_t persistent_variant) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (wait_limit_ns < 1000 || wait_limit_ns > 600000000000LL)
            throw opf::Error(OPF_ERR_INVALID_ARG, "wait limit out of [1 us, 600 s]");
        if (withhold_block < -1 || withhold_block >= p->pk.nblocks)
            throw opf::Error(OPF_ERR_INVALID_ARG, "withhold_block out of range");
        if (persistent_variant < 0 || persistent_variant > 3) throw opf::Error(OPF_ERR_INVALID_ARG, "bad persistent variant");
        p->timeout_ns = (unsigned long long)wait_limit_ns;
        p->skip_block = withhold_block;
        p->force_variant = persistent_variant;
        return OPF_OK;
    });
}

int32_t opf_residuals_noalloc(const double* v, const double* x_local, const double* x_local_prev, const double* lam,
                              int64_t n_local, double rho, double eps_rel, double* out, void* stream) {
    return guarded([&]() -> int32_t {
        opf::residuals_noalloc(v, x_local, x_local_prev, lam, (long long)n_local, rho, eps_rel, out,
                               (cudaStream_t)stream);
        return OPF_OK;
    });
}

int32_t opf_get_operator(const opf_problem* p, int32_t s, double* P, double* bbar, int32_t* n_s) {
    return guarded([&]() -> int32_t {
        if (!p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem");
        if (s < 0 || s >= (int32_t)p->ops.size()) throw opf::Error(OPF_ERR_INVALID_ARG, "component index out of range");
        const opf::Operator& op = p->ops[s];
        if (n_s) *n_s = op.n;
        if (P) std::memcpy(P, op.P.data(), op.P.size() * sizeof(double));
        if (bbar) std::memcpy(bbar, op.bbar.data(), op.bbar.size() * sizeof(double));
        return OPF_OK;
    });
}

int32_t opf_component_operator(const double* A, const double* b, int32_t m, int32_t n, double* P, double* bbar,
                               int32_t* m_reduced) {
    return guarded([&]() -> int32_t {
        if (m < 0 || m > 4096 || n < 1 || n > 4096) throw opf::Error(OPF_ERR_INVALID_ARG, "m or n out of range");
        if ((m > 0 && (!A || !b))) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL rows");
        opf::Component c;
        c.kind = -1;
        c.index = -1;
        c.gvars.assign(n, 0);
        c.m = m;
        c.A.assign(A, A + (size_t)m * n);
        c.b.assign(b, b + m);
        for (double a : c.A)
            if (!std::isfinite(a)) throw opf::Error(OPF_ERR_INVALID_ARG, "non-finite entry in A");
        for (double a : c.b)
            if (!std::isfinite(a)) throw opf::Error(OPF_ERR_INVALID_ARG, "non-finite entry in b");
        const opf::Operator op = opf::make_operator(c);
        if (P) std::memcpy(P, op.P.data(), op.P.size() * sizeof(double));
        if (bbar) std::memcpy(bbar, op.bbar.data(), op.bbar.size() * sizeof(double));
        if (m_reduced) *m_reduced = op.m_reduced;
        return OPF_OK;
    });
}

void opf_destroy(opf_problem* p) {
    if (!p) return;
    try {
        if (p->uploaded) opf::device_free(p);
    } catch (...) {
    }
    delete p;
}

int32_t opf_batch_create(opf_problem* const* problems, int32_t n, opf_batch** out) {
    return guarded([&]() -> int32_t {
        if (!out || !problems || n < 1) throw opf::Error(OPF_ERR_INVALID_ARG, "need at least one problem");
        *out = nullptr;
        int dev = -1;
        for (int i = 0; i < n; ++i) {
            if (!problems[i]) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL problem in batch");
            if (!problems[i]->uploaded) throw opf::Error(OPF_ERR_STATE, "batch problem not uploaded");
            if (i && problems[i]->device != dev) throw opf::Error(OPF_ERR_INVALID_ARG, "batch spans devices");
            dev = problems[i]->device;
            for (int j = 0; j < i; ++j)
                if (problems[j] == problems[i]) throw opf::Error(OPF_ERR_INVALID_ARG, "problem listed twice");
        }
        opf_batch* b = new opf_batch();
        b->probs.assign(problems, problems + n);
        b->device = dev;
        *out = b;
        return OPF_OK;
    });
}

int32_t opf_batch_solve(opf_batch* b, const opf_params* prm, int32_t n_params, void* stream, opf_info* infos) {
    return guarded([&]() -> int32_t {
        if (!b || !prm) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        const int n = (int)b->probs.size();
        if (n_params != 1 && n_params != n) throw opf::Error(OPF_ERR_INVALID_ARG, "n_params must be 1 or the batch size");
        for (int i = 0; i < n_params; ++i) {
            const opf_params& q = prm[i];
            if (!(q.rho > 0.0) || !std::isfinite(q.rho)) throw opf::Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
            if (q.check_every < 1 || q.check_every > 4096) throw opf::Error(OPF_ERR_INVALID_ARG, "check_every out of [1, 4096]");
            if (q.max_iter < 0 || q.criterion < 0 || q.criterion > 3) throw opf::Error(OPF_ERR_INVALID_ARG, "bad max_iter or criterion");
            if (q.precision != prm[0].precision || (q.precision != OPF_FP64 && q.precision != OPF_FP32))
                throw opf::Error(OPF_ERR_INVALID_ARG, "batch precision must be FP64 or FP32 for every instance");
            if (q.residual_form != OPF_RES_PAPER)
                throw opf::Error(OPF_ERR_INVALID_ARG, "batch: only the paper's residual form (OPF_RES_PAPER)");
            if (q.adaptive_rho && !(q.rb_mu > 1.0 && q.rb_tau > 1.0))
                throw opf::Error(OPF_ERR_INVALID_ARG, "residual balancing needs rb_mu > 1 and rb_tau > 1");
        }
        opf::device_batch_solve(b, prm, n_params, (cudaStream_t)stream, infos);
        return OPF_OK;
    });
}

int32_t opf_batch_profile_kernels(opf_batch* b, const opf_params* prm, int32_t reps, void* stream, double* us) {
    return guarded([&]() -> int32_t {
        if (!b || !prm || !us) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (reps < 1 || reps > 100000) throw opf::Error(OPF_ERR_INVALID_ARG, "reps out of [1, 100000]");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho)) throw opf::Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
        if (prm->precision != OPF_FP64 && prm->precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        if (prm->check_every < 1 || prm->check_every > 4096)
            throw opf::Error(OPF_ERR_INVALID_ARG, "check_every out of [1, 4096]");
        opf::device_batch_profile(b, *prm, reps, (cudaStream_t)stream, us);
        return OPF_OK;
    });
}

int32_t opf_batch_engine_for(const opf_batch* b, int32_t precision, int32_t* engine) {
    return guarded([&]() -> int32_t {
        if (!b || !engine) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (precision != OPF_FP64 && precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        *engine = opf::device_batch_auto_engine(b, precision);
        return OPF_OK;
    });
}

int32_t opf_batch_capacity(int32_t precision, int32_t* max_chunks) {
    return guarded([&]() -> int32_t {
        if (!max_chunks) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (precision != OPF_FP64 && precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "bad precision");
        *max_chunks = opf::device_batch_capacity(precision);
        return OPF_OK;
    });
}

int32_t opf_scenarios_create(const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                             const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                             int32_t n_scenarios, opf_scenarios** out) {
    return guarded([&]() -> int32_t {
        if (!out) throw opf::Error(OPF_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        *out = opf::scenarios_create(buses, n_bus, lines, n_line, gens, n_gen, loads, n_load, n_scenarios);
        return OPF_OK;
    });
}

int32_t opf_scenarios_solve(opf_scenarios* sc, const opf_params* prm, void* stream, opf_info* infos) {
    return guarded([&]() -> int32_t {
        if (!sc || !prm) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (prm->precision != OPF_FP32) throw opf::Error(OPF_ERR_INVALID_ARG, "scenarios: precision must be FP32");
        if (prm->adaptive_rho) throw opf::Error(OPF_ERR_INVALID_ARG, "scenarios: residual balancing not supported");
        if (prm->residual_form != OPF_RES_PAPER)
            throw opf::Error(OPF_ERR_INVALID_ARG, "scenarios: only the paper's residual form (OPF_RES_PAPER)");
        if (!(prm->rho > 0.0) || !std::isfinite(prm->rho) || prm->max_iter < 0)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad parameters");
        // the solve graph's body holds check_every iterations of kernel nodes
        if (prm->check_every < 1 || prm->check_every > 4096)
            throw opf::Error(OPF_ERR_INVALID_ARG, "check_every out of [1, 4096]");
        opf::scenarios_solve(sc, *prm, (cudaStream_t)stream, infos);
        return OPF_OK;
    });
}

int32_t opf_scenarios_get_state(const opf_scenarios* sc, int32_t scenario, double* x, double* xl, double* lam,
                                void* stream) {
    return guarded([&]() -> int32_t {
        if (!sc) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        opf::scenarios_get_state(sc, scenario, x, xl, lam, (cudaStream_t)stream);
        return OPF_OK;
    });
}

int32_t opf_scenarios_dims(const opf_scenarios* sc, int32_t* n_global, int32_t* n_local, int64_t* device_bytes) {
    return guarded([&]() -> int32_t {
        if (!sc) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        opf::scenarios_dims(sc, n_global, n_local, device_bytes);
        return OPF_OK;
    });
}

int32_t opf_scenarios_profile(opf_scenarios* sc, const opf_params* prm, int32_t reps, void* stream, double* us) {
    return guarded([&]() -> int32_t {
        if (!sc || !prm || !us) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        if (reps < 1 || reps > 100000 || !(prm->rho > 0.0) || !std::isfinite(prm->rho))
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad parameters");
        opf::scenarios_profile(sc, *prm, reps, (cudaStream_t)stream, us);
        return OPF_OK;
    });
}

int32_t opf_scenarios_set_xupdate(opf_scenarios* sc, int32_t kind) {
    return guarded([&]() -> int32_t {
        if (!sc) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        opf::scenarios_set_xupdate(sc, kind);
        return OPF_OK;
    });
}

void opf_scenarios_destroy(opf_scenarios* sc) {
    try {
        opf::scenarios_destroy(sc);
    } catch (...) {
    }
}

void opf_batch_destroy(opf_batch* b) {
    if (!b) return;
    try {
        opf::device_batch_free(b);
    } catch (...) {
    }
    delete b;
}

}  // extern "C"
