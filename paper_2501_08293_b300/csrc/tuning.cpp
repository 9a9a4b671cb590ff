// Tuning table for the automatic chunking of a problem (the number of CTAs
// of the local update and of the persistent kernels).
//
// A problem is cut into chunks of about `work_per_chunk` units of
// n_s^2 + 4 n_s + 16 (at most `max_chunks`).  The best size depends on the
// GPU and on the feeder's size: few large chunks exchange less with their
// neighbours, many small ones spread the arithmetic over more SMs.  The
// project's tuner (paper_2501_08293_b300/autotune.py) times the candidates
// on the device for a few size buckets and writes the winners as JSON:
//
//   {"gpu": "<cudaDeviceProp::name>",
//    "entries": [{"n_bus_lo": 13, "n_bus_hi": 100, "work_per_chunk": 1024,
//                 "max_chunks": 296, ...}, ...]}
//
// (other keys are ignored).  opf_tuning_load reads such a file into the
// table; opf_problem_create with chunks = 0 looks up the current device's
// name and the feeder's bus count; without a matching entry the default is
// 4096 units per chunk, at most 296 chunks.
#include <cuda_runtime.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.hpp"

namespace opf {
namespace {

struct TuneEntry {
    std::string gpu;
    int lo = 0, hi = 0;
    int work = 4096;
    int max_chunks = 296;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> g_table;
std::map<int, std::string> g_names;     // device index -> name, looked up once

// ------------------------------------------------------------ JSON reader
// Enough JSON for the tuner's files: objects, arrays, strings (with the
// common escapes), numbers, true / false / null.
struct JVal {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0;
    bool b = false;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
    const JVal* get(const std::string& k) const {
        for (const auto& kv : obj)
            if (kv.first == k) return &kv.second;
        return nullptr;
    }
};

struct JParser {
    const std::string& s;
    size_t i = 0;
    explicit JParser(const std::string& src) : s(src) {}
    [[noreturn]] void fail(const char* what) const {
        throw Error(OPF_ERR_INVALID_ARG, std::string("tuning file: ") + what + " at byte " + std::to_string(i));
    }
    void ws() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    std::string string() {
        if (!eat('"')) fail("expected a string");
        std::string out;
        while (i < s.size() && s[i] != '"') {
            char c = s[i++];
            if (c == '\\') {
                if (i >= s.size()) fail("bad escape");
                const char e = s[i++];
                switch (e) {
                    case 'n': out += '\n'; break;
                    case 't': out += '\t'; break;
                    case 'r': out += '\r'; break;
                    case 'b': out += '\b'; break;
                    case 'f': out += '\f'; break;
                    case 'u':
                        if (i + 4 > s.size()) fail("bad escape");
                        out += '?';          // names in the table are ASCII
                        i += 4;
                        break;
                    default: out += e;
                }
            } else {
                out += c;
            }
        }
        if (i >= s.size()) fail("unterminated string");
        ++i;
        return out;
    }
    JVal value(int depth) {
        if (depth > 32) fail("nesting too deep");
        ws();
        if (i >= s.size()) fail("unexpected end");
        JVal v;
        const char c = s[i];
        if (c == '{') {
            ++i;
            v.kind = JVal::OBJ;
            if (eat('}')) return v;
            do {
                std::string k = string();
                if (!eat(':')) fail("expected ':'");
                v.obj.emplace_back(std::move(k), value(depth + 1));
            } while (eat(','));
            if (!eat('}')) fail("expected '}'");
        } else if (c == '[') {
            ++i;
            v.kind = JVal::ARR;
            if (eat(']')) return v;
            do {
                v.arr.push_back(value(depth + 1));
            } while (eat(','));
            if (!eat(']')) fail("expected ']'");
        } else if (c == '"') {
            v.kind = JVal::STR;
            v.str = string();
        } else if (s.compare(i, 4, "true") == 0) {
            v.kind = JVal::BOOL; v.b = true; i += 4;
        } else if (s.compare(i, 5, "false") == 0) {
            v.kind = JVal::BOOL; i += 5;
        } else if (s.compare(i, 4, "null") == 0) {
            i += 4;
        } else {
            const char* b = s.c_str() + i;
            char* e = nullptr;
            v.num = std::strtod(b, &e);
            if (e == b) fail("bad value");
            v.kind = JVal::NUM;
            i += (size_t)(e - b);
        }
        return v;
    }
};

int as_int(const JVal* v, const char* key) {
    if (!v || v->kind != JVal::NUM) throw Error(OPF_ERR_INVALID_ARG, std::string("tuning file: entry without ") + key);
    return (int)v->num;
}

void check_entry(const TuneEntry& e) {
    if (e.lo < 0 || e.hi <= e.lo) throw Error(OPF_ERR_INVALID_ARG, "tuning: need 0 <= n_bus_lo < n_bus_hi");
    if (e.work < 16 || e.work > (1 << 26)) throw Error(OPF_ERR_INVALID_ARG, "tuning: work_per_chunk out of [16, 2^26]");
    if (e.max_chunks < 1 || e.max_chunks > 65536) throw Error(OPF_ERR_INVALID_ARG, "tuning: max_chunks out of [1, 65536]");
}

void put_entry(const TuneEntry& e) {
    check_entry(e);
    for (TuneEntry& o : g_table)
        if (o.gpu == e.gpu && o.lo == e.lo && o.hi == e.hi) {
            o = e;
            return;
        }
    g_table.push_back(e);
}

// Name of the current device ("" when there is none), cached per index.
std::string current_gpu_name() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return "";
    }
    auto it = g_names.find(dev);
    if (it != g_names.end()) return it->second;
    cudaDeviceProp prop;
    std::string name;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    else cudaGetLastError();
    g_names[dev] = name;
    return name;
}

}  // namespace

void auto_chunking(int n_bus, int64_t* work_per_chunk, int* max_chunks) {
    *work_per_chunk = 4096;
    *max_chunks = 296;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_table.empty()) return;
    const std::string name = current_gpu_name();
    for (const TuneEntry& e : g_table)
        if ((e.gpu == name || e.gpu == "*") && n_bus >= e.lo && n_bus < e.hi) {
            *work_per_chunk = e.work;
            *max_chunks = e.max_chunks;
            return;
        }
}

}  // namespace opf

namespace {
template <typename F>
int32_t tune_guard(F&& f) {
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

int32_t opf_tuning_set(const char* gpu, int32_t n_bus_lo, int32_t n_bus_hi, int32_t work_per_chunk,
                       int32_t max_chunks) {
    return tune_guard([&]() -> int32_t {
        if (!gpu) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL gpu name");
        opf::TuneEntry e{gpu, n_bus_lo, n_bus_hi, work_per_chunk, max_chunks};
        std::lock_guard<std::mutex> lk(opf::g_tune_mu);
        opf::put_entry(e);
        return OPF_OK;
    });
}

int32_t opf_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(opf::g_tune_mu);
    opf::g_table.clear();
    return OPF_OK;
}

int32_t opf_tuning_load(const char* path, int32_t* n_entries) {
    return tune_guard([&]() -> int32_t {
        if (!path) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL path");
        std::unique_ptr<FILE, int (*)(FILE*)> fh(std::fopen(path, "rb"), &std::fclose);
        if (!fh) throw opf::Error(OPF_ERR_INVALID_ARG, std::string("cannot open ") + path);
        std::string src;
        char buf[4096];
        size_t k;
        while ((k = std::fread(buf, 1, sizeof(buf), fh.get())) > 0) {
            src.append(buf, k);
            if (src.size() > (1u << 22)) throw opf::Error(OPF_ERR_INVALID_ARG, "tuning file larger than 4 MiB");
        }
        opf::JParser ps(src);
        const opf::JVal root = ps.value(0);
        ps.ws();
        if (ps.i != src.size()) ps.fail("trailing characters");
        const opf::JVal* g = root.get("gpu");
        const opf::JVal* es = root.get("entries");
        if (root.kind != opf::JVal::OBJ || !g || g->kind != opf::JVal::STR || !es || es->kind != opf::JVal::ARR)
            throw opf::Error(OPF_ERR_INVALID_ARG, "tuning file: need {\"gpu\": name, \"entries\": [...]}");
        std::vector<opf::TuneEntry> add;
        for (const opf::JVal& e : es->arr) {
            if (e.kind != opf::JVal::OBJ) throw opf::Error(OPF_ERR_INVALID_ARG, "tuning file: entry is not an object");
            opf::TuneEntry t{g->str, opf::as_int(e.get("n_bus_lo"), "n_bus_lo"), opf::as_int(e.get("n_bus_hi"), "n_bus_hi"),
                             opf::as_int(e.get("work_per_chunk"), "work_per_chunk"),
                             opf::as_int(e.get("max_chunks"), "max_chunks")};
            opf::check_entry(t);
            add.push_back(t);
        }
        std::lock_guard<std::mutex> lk(opf::g_tune_mu);
        for (const opf::TuneEntry& t : add) opf::put_entry(t);
        if (n_entries) *n_entries = (int32_t)add.size();
        return OPF_OK;
    });
}

int32_t opf_tuning_lookup(int32_t n_bus, int32_t* work_per_chunk, int32_t* max_chunks) {
    return tune_guard([&]() -> int32_t {
        if (!work_per_chunk || !max_chunks) throw opf::Error(OPF_ERR_INVALID_ARG, "NULL argument");
        int64_t w = 0;
        int m = 0;
        opf::auto_chunking(n_bus, &w, &m);
        *work_per_chunk = (int32_t)w;
        *max_chunks = m;
        return OPF_OK;
    });
}

}  // extern "C"
