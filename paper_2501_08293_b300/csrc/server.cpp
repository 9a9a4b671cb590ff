// Continuous-batching OPF server (the serving pattern of the solver).
//
// Requests are feeders (host records).  opf_server_submit builds the model
// and the FP64 operators on the calling thread and queues the request.
// opf_server_step is one scheduling round:
//   1. collect the round in flight (if any): each active instance gets its
//      residuals; an instance that converged, failed or used up its
//      iteration budget (params.max_iter, or iters_per_bus times its bus
//      count when that is larger) is finished (its latency recorded) and
//      stays resident for warm starts until memory is needed;
//   2. admit queued requests in arrival order while a slot, the device
//      memory budget and the co-resident chunk capacity allow (finished
//      instances are evicted least recently used first; a request's own
//      warm-start source last, and only when nothing is active, in which
//      case it starts cold); uploads run on a
//      side stream, overlapping the round still queued on the main stream;
//      a request that modifies a resident feeder (warm_from) starts from
//      that feeder's iterate, copied on the device for every local copy
//      whose component and global variable are unchanged;
//   3. launch the next round, asynchronously: one cooperative batch launch
//      of round_iters iterations over every active instance, each with its
//      own control block (warm-started after its first round).
// Rounds are whole multiples of the check interval and every engine runs
// the same arithmetic, so a request's iterates and stopping iteration do not
// depend on what else was being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>

#include "problem.hpp"

namespace opf {
void device_batch_launch(opf_batch* B, const opf_params* prm, int nprm, cudaStream_t s);
void device_batch_collect(opf_batch* B, const opf_params* prm, int nprm, opf_info* infos);
void device_batch_free(opf_batch* B);
void device_upload(opf_problem* p, void* arena, size_t bytes, cudaStream_t s);
size_t device_bytes(const opf_problem* p);
void device_warm_transfer(opf_problem* dst, const opf_problem* src, const std::vector<int32_t>& map, cudaStream_t s);
void device_free(opf_problem* p);
void set_last_error(const std::string& m);
std::vector<int32_t> warm_map(const opf_problem* dst, const opf_problem* src);
}  // namespace opf

namespace {

enum { REQ_PENDING = 0, REQ_ACTIVE = 1, REQ_DONE = 2 };

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    opf_problem* p = nullptr;
    int64_t warm_from = -1;
    int state = REQ_PENDING;
    bool resident = false;
    bool started = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    opf_info info{};
    size_t bytes = 0;
    int chunks = 0;
    int32_t budget = 0;          // iteration budget of this request
    uint64_t last_use = 0;
};

}  // namespace

struct opf_server {
    opf_server_config cfg{};
    int device = -1;
    cudaStream_t upload = nullptr;
    cudaEvent_t uploaded = nullptr;
    std::mutex mu;                                  // guards submissions vs. steps
    std::map<int64_t, Request> reqs;
    std::deque<int64_t> pending;
    std::vector<int64_t> active;
    std::deque<int64_t> finished;                   // not yet polled
    std::vector<int64_t> round;                     // members of the round in flight
    std::vector<opf_params> round_params;
    bool in_flight = false;
    opf_batch batch;
    size_t used_bytes = 0;
    int64_t next_id = 1;
    uint64_t tick = 0;
    opf_server_stats stats{};
};

namespace {

void evict(opf_server* S, Request& r) {
    if (r.p) {
        S->used_bytes -= r.bytes;
        opf_destroy(r.p);
        r.p = nullptr;
    }
    r.resident = false;
    S->stats.evicted += 1;
}

int active_chunks(const opf_server* S) {
    int c = 0;
    for (int64_t id : S->active) c += S->reqs.at(id).chunks;
    return c;
}

void collect(opf_server* S) {
    if (!S->in_flight) return;
    std::vector<opf_info> infos(S->round.size());
    opf::device_batch_collect(&S->batch, S->round_params.data(), (int)S->round_params.size(), infos.data());
    S->in_flight = false;
    const double t = now_s();
    S->stats.rounds += 1;
    std::vector<int64_t> still;
    for (size_t i = 0; i < S->round.size(); ++i) {
        Request& r = S->reqs.at(S->round[i]);
        r.info = infos[i];
        r.started = true;
        r.last_use = ++S->tick;
        const bool budget_used = r.info.iters >= r.budget;
        if (r.info.status != OPF_NOT_CONVERGED || budget_used) {
            r.state = REQ_DONE;
            r.t_done = t;
            r.info.seconds = t - r.t_submit;
            S->finished.push_back(r.id);
            S->stats.completed += 1;
            if (r.info.status == OPF_OK) S->stats.converged += 1;
            S->stats.iterations += r.info.iters;
        } else {
            still.push_back(r.id);
        }
    }
    S->active.swap(still);
    S->round.clear();
}

bool admit(opf_server* S, Request& r) {
    const size_t budget = (size_t)S->cfg.device_budget_bytes;
    const int cap = S->cfg.max_chunks;
    if ((int)S->active.size() >= S->cfg.max_active) return false;
    if (active_chunks(S) + r.chunks > cap) return false;
    // make room: evict finished residents, least recently used first, but
    // never the feeder this request warm-starts from
    while (S->used_bytes + r.bytes > budget) {
        Request* lru = nullptr;
        for (auto& kv : S->reqs) {
            Request& q = kv.second;
            if (q.state == REQ_DONE && q.resident && q.id != r.warm_from && (!lru || q.last_use < lru->last_use)) lru = &q;
        }
        if (!lru) {
            // only the warm-start source is left to evict; with no instance
            // active nothing else will free memory, so the request gives up
            // its warm start (cold start below) instead of waiting forever
            auto src = S->reqs.find(r.warm_from);
            if (!S->active.empty() || src == S->reqs.end() || !src->second.resident) return false;
            evict(S, src->second);
            continue;
        }
        evict(S, *lru);
    }
    opf::device_upload(r.p, nullptr, 0, S->upload);
    r.p->uploaded = true;
    S->used_bytes += r.bytes;
    r.resident = true;
    if (r.warm_from >= 0) {
        auto it = S->reqs.find(r.warm_from);
        if (it != S->reqs.end() && it->second.resident && it->second.state == REQ_DONE && it->second.p) {
            opf::device_warm_transfer(r.p, it->second.p, opf::warm_map(r.p, it->second.p), S->upload);
            it->second.last_use = ++S->tick;
            S->stats.warm_started += 1;
        } else {
            r.warm_from = -1;                     // source gone: cold start
        }
    }
    r.state = REQ_ACTIVE;
    r.t_admit = now_s();
    S->active.push_back(r.id);
    S->stats.admitted += 1;
    return true;
}

void launch_round(opf_server* S, cudaStream_t s) {
    if (S->active.empty()) return;
    cudaError_t e = cudaEventRecord(S->uploaded, S->upload);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, S->uploaded, 0);
    if (e != cudaSuccess) throw opf::Error(OPF_ERR_CUDA, std::string("server round ordering: ") + cudaGetErrorString(e));
    S->round = S->active;
    S->round_params.clear();
    S->batch.probs.clear();
    // Every instance runs in the same launch, so a round lasts as long as its
    // slowest instance's iterations.  An instance's time per iteration grows
    // with its largest chunk (its CTAs run the chunk's tiles and halo every
    // iteration): the slowest instance gets round_iters iterations, faster
    // ones proportionally more (whole check intervals, at most 8x), so they
    // do not sit idle for the rest of the round.
    auto t_iter = [](const opf_problem* p) { return 1.5 + 0.004 * (double)p->pk.max_loc; };
    double t_max = 0;
    for (int64_t id : S->round) t_max = std::max(t_max, t_iter(S->reqs.at(id).p));
    const int K = std::max(1, S->cfg.params.check_every);
    for (int64_t id : S->round) {
        Request& r = S->reqs.at(id);
        opf_params q = S->cfg.params;
        q.warm_start = (r.started || r.warm_from >= 0) ? 1 : 0;
        const int left = r.budget - (r.started ? r.info.iters : 0);
        const double scale = std::min(8.0, t_max / t_iter(r.p));
        int iters = (int)(S->cfg.round_iters * scale) / K * K;
        iters = std::max(S->cfg.round_iters, iters);
        q.max_iter = std::max(0, std::min(iters, left));
        S->round_params.push_back(q);
        S->batch.probs.push_back(r.p);
    }
    opf::device_batch_launch(&S->batch, S->round_params.data(), (int)S->round_params.size(), s);
    S->in_flight = true;
}

template <typename F>
int32_t guard(F&& f) {
    opf::set_last_error("");
    try {
        return f();
    } catch (const opf::Error& e) {
        opf::set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc&) {
        opf::set_last_error("host allocation failed");
        return OPF_ERR_OOM;
    } catch (const std::exception& e) {
        opf::set_last_error(e.what());
        return OPF_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" {

void opf_server_config_default(opf_server_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->device_budget_bytes = (int64_t)8 << 30;
    c->max_active = 256;
    c->round_iters = 2000;
    c->max_chunks = 0;
    opf_params_default(&c->params);
    c->params.precision = OPF_FP32;
    c->params.rho = 10.0;
    c->params.max_iter = 1000000;
}

int32_t opf_server_create(const opf_server_config* cfg, opf_server** out) {
    return guard([&]() -> int32_t {
        if (!cfg || !out) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        if (cfg->max_active < 1 || cfg->round_iters < 1 || cfg->device_budget_bytes < 1 || cfg->iters_per_bus < 0 ||
            cfg->params.max_iter < 0)
            throw opf::Error(OPF_ERR_INVALID_ARG, "bad server configuration");
        if (cfg->params.check_every < 1 || cfg->params.check_every > 4096)
            throw opf::Error(OPF_ERR_INVALID_ARG, "params.check_every out of [1, 4096]");
        if (cfg->round_iters % cfg->params.check_every)
            throw opf::Error(OPF_ERR_INVALID_ARG, "round_iters must be a multiple of params.check_every");
        if (cfg->params.residual_form != OPF_RES_PAPER)
            throw opf::Error(OPF_ERR_INVALID_ARG, "server: only the paper's residual form (OPF_RES_PAPER)");
        opf_server* S = new opf_server();
        S->cfg = *cfg;
        int32_t cap = 0;
        const int32_t st = opf_batch_capacity(cfg->params.precision, &cap);
        if (st != OPF_OK) {
            delete S;
            throw opf::Error(st, "server: device capacity query failed");
        }
        if (S->cfg.max_chunks <= 0 || S->cfg.max_chunks > cap) S->cfg.max_chunks = cap;
        cudaGetDevice(&S->device);
        S->batch.device = S->device;
        cudaError_t e = cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->uploaded, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            delete S;
            throw opf::Error(OPF_ERR_CUDA, std::string("server streams: ") + cudaGetErrorString(e));
        }
        *out = S;
        return OPF_OK;
    });
}

int32_t opf_server_submit(opf_server* S, const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                          const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                          int32_t chunks, int64_t warm_from, int64_t* id) {
    return guard([&]() -> int32_t {
        if (!S || !id) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        const double t = now_s();
        opf_create_options o{};
        // default: one chunk per 50 buses (1..64) -- instances co-resident for
        // throughput, chunks small enough for short rounds
        o.chunks = chunks > 0 ? chunks : std::max(1, std::min(64, n_bus / 50));
        opf_problem* p = nullptr;
        const int32_t st = opf_problem_create_ex(buses, n_bus, lines, n_line, gens, n_gen, loads, n_load, &o, &p);
        if (st != OPF_OK) throw opf::Error(st, std::string("submit: ") + opf_last_error());
        std::lock_guard<std::mutex> lk(S->mu);
        Request r;
        r.id = S->next_id++;
        r.p = p;
        r.warm_from = warm_from;
        r.t_submit = t;
        r.bytes = opf::device_bytes(p);
        r.chunks = p->pk.nblocks;
        const int64_t scaled = (int64_t)S->cfg.iters_per_bus * n_bus;
        r.budget = (int32_t)std::min<int64_t>(INT32_MAX / 2, std::max<int64_t>(S->cfg.params.max_iter, scaled));
        if (r.chunks > S->cfg.max_chunks || r.bytes > (size_t)S->cfg.device_budget_bytes) {
            opf_destroy(p);
            throw opf::Error(OPF_ERR_INVALID_ARG, "request larger than the server's chunk or memory budget");
        }
        S->reqs[r.id] = r;
        S->pending.push_back(r.id);
        S->stats.submitted += 1;
        *id = r.id;
        return OPF_OK;
    });
}

int32_t opf_server_step(opf_server* S, void* stream, int32_t* n_active, int32_t* n_pending) {
    return guard([&]() -> int32_t {
        if (!S) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL server");
        std::lock_guard<std::mutex> lk(S->mu);
        collect(S);
        while (!S->pending.empty()) {
            Request& r = S->reqs.at(S->pending.front());
            if (!admit(S, r)) break;
            S->pending.pop_front();
        }
        launch_round(S, (cudaStream_t)stream);
        if (n_active) *n_active = (int32_t)S->active.size();
        if (n_pending) *n_pending = (int32_t)S->pending.size();
        return OPF_OK;
    });
}

int32_t opf_server_poll(opf_server* S, int64_t* ids, opf_info* infos, int32_t cap, int32_t* n) {
    return guard([&]() -> int32_t {
        if (!S || !n || (cap > 0 && (!ids || !infos))) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        int k = 0;
        while (k < cap && !S->finished.empty()) {
            const Request& r = S->reqs.at(S->finished.front());
            ids[k] = r.id;
            infos[k] = r.info;
            S->finished.pop_front();
            ++k;
        }
        *n = k;
        return OPF_OK;
    });
}

int32_t opf_server_problem(opf_server* S, int64_t id, opf_problem** p) {
    return guard([&]() -> int32_t {
        if (!S || !p) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second.resident || it->second.state != REQ_DONE)
            throw opf::Error(OPF_ERR_STATE, "request is not a finished resident instance");
        *p = it->second.p;
        return OPF_OK;
    });
}

int32_t opf_server_get_stats(opf_server* S, opf_server_stats* st) {
    return guard([&]() -> int32_t {
        if (!S || !st) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        *st = S->stats;
        st->active = (int32_t)S->active.size();
        st->pending = (int32_t)S->pending.size();
        st->resident_bytes = (int64_t)S->used_bytes;
        return OPF_OK;
    });
}

void opf_server_destroy(opf_server* S) {
    if (!S) return;
    try {
        if (S->in_flight) cudaEventSynchronize(S->batch.done);
        opf::device_batch_free(&S->batch);
    } catch (...) {
    }
    for (auto& kv : S->reqs)
        if (kv.second.p) opf_destroy(kv.second.p);
    if (S->uploaded) cudaEventDestroy(S->uploaded);
    if (S->upload) cudaStreamDestroy(S->upload);
    delete S;
}

}  // extern "C"
