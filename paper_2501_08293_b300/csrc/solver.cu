// sm_103a kernels and the solve engines of the componentwise ADMM.
//
// One iteration of Algorithm 1 is two kernels:
//   z_kernel  global update, Eq. (global_sparse): for every global i, the
//             copies' (x_j - lambda_j / rho) are summed over the CSR list in a
//             fixed order, scaled by 1/k_i, shifted by -c_i/(rho k_i) and
//             clipped to [lo_i, hi_i].  One thread per global, no atomics.
//   x_kernel  local update, Eq. (closed_2), fused with the dual update of
//             Eq. (ADMM-3) and the residual sums of Eq. (termination): per
//             component u = B_s x + lambda_s / rho, x_s = P_s u + bbar_s
//             (P_s = -Abar_s), lambda_s += rho (B_s x - x_s).  One warp per
//             tile of components (see pack.cpp), operator elements streamed
//             with coalesced loads, u broadcast by warp shuffles.  On check
//             iterations each block writes five FP64 partial sums
//             (||Bx - z||^2, ||z - z_prev||^2, ||Bx||^2, ||z||^2, ||lambda||^2).
// finalize_kernel sums the block partials in a fixed order (deterministic),
// forms pres, dres, eps_prim, eps_dual, applies the stopping rule and, in the
// graph engine, sets the condition of the device-side while node so the
// whole solve runs as one CUDA graph launch without host round trips.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>

#include "problem.hpp"

namespace opf {

#define OPF_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw Error(e_ == cudaErrorMemoryAllocation ? OPF_ERR_OOM : OPF_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

constexpr int kXWarps = 8;          // warps per block of x_kernel
constexpr int kXBlocksMax = 148 * 8;
constexpr int kZThreads = 256;
constexpr int kFinThreads = 256;
constexpr int kMaxBigN = 256;

// ------------------------------------------------------------------ kernels
template <typename T>
__global__ void __launch_bounds__(kZThreads) z_kernel(View<T> v, int q) {
    const Ctl* ctl = v.ctl;
    if (ctl->iter + q >= ctl->max_iter) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.ng) return;
    const T inv_rho = (T)ctl->inv_rho;
    const int b = v.gptr[i], e = v.gptr[i + 1];
    T s = 0;
    for (int j = b; j < e; ++j) {
        const int l = v.gcol[j];
        s += v.xl[l] - v.lam[l] * inv_rho;
    }
    const T xh = s * v.invk[i] - v.cik[i] * inv_rho;
    v.zg[i] = fmin(fmax(xh, v.lo[i]), v.hi[i]);
}

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

template <typename T>
__global__ void __launch_bounds__(kXWarps * 32) x_kernel(View<T> v, int q) {
    const Ctl* ctl = v.ctl;
    const int iter = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    if (iter + q >= maxit) return;
    const bool want = (q == min(K, maxit - iter) - 1);
    const T rho = (T)ctl->rho, inv_rho = (T)ctl->inv_rho;
    __shared__ T us[kXWarps][kMaxBigN];
    __shared__ double red[kXWarps][5];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    for (int t = blockIdx.x * kXWarps + warp; t < v.ntiles; t += gridDim.x * kXWarps) {
        const Tile tl = v.tiles[t];
        const int n = tl.n;
        if (n <= 32) {
            const int L = tl.ncomp * n;
            const bool act = lane < L;
            const int base = (lane / n) * n;
            const int j = tl.loc0 + lane;
            T vv = 0, lo = 0, xo = 0, u = 0;
            if (act) {
                vv = v.zg[v.gidx[j]];
                lo = v.lam[j];
                xo = v.xl[j];
                u = vv + lo * inv_rho;
            }
            const T* Pm = v.P + tl.mat0 + lane;
            T y = 0;
#pragma unroll 4
            for (int c = 0; c < n; ++c) {
                const T uc = __shfl_sync(0xffffffffu, u, (base + c) & 31);
                if (act) y = fma(Pm[(size_t)c * L], uc, y);
            }
            if (act) {
                const T xn = y + v.bbar[j];
                const T ln = lo + rho * (vv - xn);
                v.xl[j] = xn;
                v.lam[j] = ln;
                if (want) {
                    const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                    a0 += pr * pr; a1 += dz * dz;
                    a2 += (double)vv * (double)vv; a3 += (double)xn * (double)xn; a4 += (double)ln * (double)ln;
                }
            }
        } else {
            for (int r = lane; r < n; r += 32) {
                const int j = tl.loc0 + r;
                us[warp][r] = v.zg[v.gidx[j]] + v.lam[j] * inv_rho;
            }
            __syncwarp();
            const T* Pm = v.P + tl.mat0;
            for (int r = lane; r < n; r += 32) {
                T y = 0;
                for (int c = 0; c < n; ++c) y = fma(Pm[(size_t)c * n + r], us[warp][c], y);
                const int j = tl.loc0 + r;
                const T vv = v.zg[v.gidx[j]];
                const T lo = v.lam[j], xo = v.xl[j];
                const T xn = y + v.bbar[j];
                const T ln = lo + rho * (vv - xn);
                v.xl[j] = xn;
                v.lam[j] = ln;
                if (want) {
                    const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                    a0 += pr * pr; a1 += dz * dz;
                    a2 += (double)vv * (double)vv; a3 += (double)xn * (double)xn; a4 += (double)ln * (double)ln;
                }
            }
            __syncwarp();
        }
    }
    if (!want) return;
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
    if (lane == 0) {
        red[warp][0] = a0; red[warp][1] = a1; red[warp][2] = a2; red[warp][3] = a3; red[warp][4] = a4;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0;
        for (int w = 0; w < kXWarps; ++w) s += red[w][threadIdx.x];
        v.partials[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(View<T> v, cudaGraphConditionalHandle h, int use_cond) {
    Ctl* ctl = v.ctl;
    const int iter = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    const int ndone = max(0, min(K, maxit - iter));
    __shared__ double sh[5][kFinThreads];
    double s[5] = {0, 0, 0, 0, 0};
    if (ndone > 0)
        for (int b = threadIdx.x; b < v.nparts; b += kFinThreads)
            for (int k = 0; k < 5; ++k) s[k] += v.partials[(size_t)b * 8 + k];
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const int it = iter + ndone;
    ctl->iter = it;
    int stop = 0;
    if (ndone > 0) {
        const double pres = sqrt(sh[0][0]);
        const double dres = ctl->rho * sqrt(sh[1][0]);
        const double ep = ctl->eps_rel * fmax(sqrt(sh[2][0]), sqrt(sh[3][0]));
        const double ed = ctl->eps_rel * sqrt(sh[4][0]);
        ctl->pres = pres; ctl->dres = dres; ctl->eps_prim = ep; ctl->eps_dual = ed;
        ctl->checks += 1;
        const bool ok_abs = pres <= ctl->eps_abs_prim && dres <= ctl->eps_abs_dual;
        const bool ok_rel = pres <= ep && dres <= ed;
        if (ok_rel && ctl->first_rel < 0) ctl->first_rel = it;
        const int cr = ctl->criterion;
        const bool conv = (cr == OPF_CRIT_ABS && ok_abs) || (cr == OPF_CRIT_REL && ok_rel) ||
                          (cr == OPF_CRIT_BOTH && ok_abs && ok_rel);
        if (!isfinite(pres) || !isfinite(dres)) {
            ctl->status = CTL_NUMERIC; stop = 1;
        } else if (conv) {
            ctl->status = CTL_CONVERGED; stop = 1;
        }
    }
    if (!stop && it >= maxit) {
        ctl->status = CTL_MAXITER; stop = 1;
    }
    ctl->stop = stop;
    if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

template <typename T>
__global__ void init_kernel(View<T> v) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < v.nl) {
        v.xl[j] = v.xl0[j];
        v.lam[j] = 0;
    }
    if (j < v.ng) v.zg[j] = 0;
    if (j == 0) {
        v.ctl->iter = 0;
        v.ctl->first_rel = -1;
        v.ctl->checks = 0;
        v.ctl->pres = v.ctl->dres = v.ctl->eps_prim = v.ctl->eps_dual = NAN;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) objective_kernel(View<T> v) {
    __shared__ double sh[256];
    double s = 0;
    for (int i = threadIdx.x; i < v.ng; i += 256) s += v.cost[i] * (double)v.zg[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) v.ctl->objective = sh[0];
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ src, B* __restrict__ dst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (B)src[i];
}

// ------------------------------------------------------------------- host
namespace {

struct Arena {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = (off + 255) & ~size_t(255);
        size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};

struct Layout {
    size_t lo, hi, invk, cik, zg, lo32, hi32, invk32, cik32, zg32;
    size_t gptr, gcol, gidx, tiles, cost, partials, ctl;
    size_t xl, lam, bbar, xl0, xl32, lam32, bbar32, xl0_32, P64, P32;
    size_t total;
};

Layout layout_of(const opf_problem* p, int nparts) {
    const Packed& k = p->pk;
    Arena a;
    Layout L;
    L.lo = a.take<double>(k.ng); L.hi = a.take<double>(k.ng); L.invk = a.take<double>(k.ng);
    L.cik = a.take<double>(k.ng); L.zg = a.take<double>(k.ng);
    L.lo32 = a.take<float>(k.ng); L.hi32 = a.take<float>(k.ng); L.invk32 = a.take<float>(k.ng);
    L.cik32 = a.take<float>(k.ng); L.zg32 = a.take<float>(k.ng);
    L.gptr = a.take<int32_t>(k.ng + 1); L.gcol = a.take<int32_t>(k.nl); L.gidx = a.take<int32_t>(k.nl);
    L.tiles = a.take<Tile>(k.tiles.size()); L.cost = a.take<double>(k.ng);
    L.partials = a.take<double>((size_t)nparts * 8); L.ctl = a.take<Ctl>(1);
    L.xl = a.take<double>(k.nl); L.lam = a.take<double>(k.nl); L.bbar = a.take<double>(k.nl); L.xl0 = a.take<double>(k.nl);
    L.xl32 = a.take<float>(k.nl); L.lam32 = a.take<float>(k.nl); L.bbar32 = a.take<float>(k.nl); L.xl0_32 = a.take<float>(k.nl);
    L.P64 = a.take<double>(k.mat_elems); L.P32 = a.take<float>(k.mat_elems);
    L.total = (a.off + 255) & ~size_t(255);
    return L;
}

int nparts_of(const opf_problem* p) {
    const int nt = (int)p->pk.tiles.size();
    int nb = (nt + kXWarps - 1) / kXWarps;
    if (nb < 1) nb = 1;
    if (nb > kXBlocksMax) nb = kXBlocksMax;
    return nb;
}

template <typename T>
View<T> view_of(const opf_problem* p, const DevPrec& d) {
    View<T> v;
    v.lo = (const T*)d.lo; v.hi = (const T*)d.hi; v.invk = (const T*)d.invk; v.cik = (const T*)d.cik;
    v.zg = (T*)d.zg; v.gptr = p->gptr; v.gcol = p->gcol; v.xl = (T*)d.xl; v.lam = (T*)d.lam;
    v.bbar = (const T*)d.bbar; v.xl0 = (const T*)d.xl0; v.gidx = p->gidx; v.tiles = p->tiles;
    v.P = (const T*)d.P; v.cost = p->cost; v.partials = p->partials; v.ctl = p->ctl;
    v.ng = p->pk.ng; v.nl = p->pk.nl; v.ntiles = (int)p->pk.tiles.size(); v.nparts = p->nparts;
    return v;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
void enqueue_init(opf_problem* p, cudaStream_t s) {
    const DevPrec& d = sizeof(T) == 8 ? p->d64 : p->d32;
    View<T> v = view_of<T>(p, d);
    const int n = std::max(p->pk.nl, p->pk.ng) + 1;
    init_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(v);
    OPF_CUDA(cudaGetLastError());
}

template <typename T>
void enqueue_iterations(opf_problem* p, int K, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
    const DevPrec& d = sizeof(T) == 8 ? p->d64 : p->d32;
    View<T> v = view_of<T>(p, d);
    const int zb = (p->pk.ng + kZThreads - 1) / kZThreads;
    for (int q = 0; q < K; ++q) {
        z_kernel<T><<<zb, kZThreads, 0, s>>>(v, q);
        x_kernel<T><<<p->nparts, kXWarps * 32, 0, s>>>(v, q);
    }
    finalize_kernel<T><<<1, kFinThreads, 0, s>>>(v, h, use_cond);
    OPF_CUDA(cudaGetLastError());
}

template <typename T>
GraphEntry& get_graph(opf_problem* p, int K, cudaStream_t s) {
    const int prec = sizeof(T) == 8 ? OPF_FP64 : OPF_FP32;
    auto key = std::make_pair(prec, K);
    auto it = p->graphs.find(key);
    if (it != p->graphs.end()) return it->second;
    GraphEntry g;
    OPF_CUDA(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle h;
    OPF_CUDA(cudaGraphConditionalHandleCreate(&h, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = cudaGraphNodeParams{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    OPF_CUDA(cudaGraphAddNode(&cnode, g.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture one body (K iterations + finalize) into the while node's graph
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    OPF_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_iterations<T>(p, K, cs, h, 1);
    } catch (...) {
        cudaGraph_t tmp;
        cudaStreamEndCapture(cs, &tmp);
        cudaStreamDestroy(cs);
        throw;
    }
    cudaGraph_t captured;
    OPF_CUDA(cudaStreamEndCapture(cs, &captured));
    OPF_CUDA(cudaStreamDestroy(cs));
    OPF_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    (void)s;
    return p->graphs.emplace(key, g).first->second;
}

template <typename T>
void run_solve(opf_problem* p, const opf_params& prm, cudaStream_t s) {
    const int engine = prm.engine == OPF_ENGINE_AUTO ? OPF_ENGINE_GRAPH : prm.engine;
    if (engine == OPF_ENGINE_GRAPH) {
        GraphEntry& g = get_graph<T>(p, prm.check_every, s);
        OPF_CUDA(cudaGraphLaunch(g.exec, s));
        OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaStreamSynchronize(s));
    } else {
        for (;;) {
            enqueue_iterations<T>(p, prm.check_every, s, 0, 0);
            OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            OPF_CUDA(cudaStreamSynchronize(s));
            if (p->ctl_host->stop) break;
        }
    }
    const DevPrec& d = sizeof(T) == 8 ? p->d64 : p->d32;
    objective_kernel<T><<<1, 256, 0, s>>>(view_of<T>(p, d));
    OPF_CUDA(cudaGetLastError());
    OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
}

template <typename A, typename B>
void enqueue_convert(const void* src, void* dst, int n, cudaStream_t s) {
    if (n <= 0) return;
    convert_kernel<A, B><<<(n + 255) / 256, 256, 0, s>>>((const A*)src, (B*)dst, n);
    OPF_CUDA(cudaGetLastError());
}

void sync_state_to(opf_problem* p, int prec, cudaStream_t s) {
    if (p->cur_prec == prec) return;
    const int nl = p->pk.nl, ng = p->pk.ng;
    if (prec == OPF_FP32) {
        enqueue_convert<double, float>(p->d64.xl, p->d32.xl, nl, s);
        enqueue_convert<double, float>(p->d64.lam, p->d32.lam, nl, s);
        enqueue_convert<double, float>(p->d64.zg, p->d32.zg, ng, s);
    } else {
        enqueue_convert<float, double>(p->d32.xl, p->d64.xl, nl, s);
        enqueue_convert<float, double>(p->d32.lam, p->d64.lam, nl, s);
        enqueue_convert<float, double>(p->d32.zg, p->d64.zg, ng, s);
    }
    p->cur_prec = prec;
}

}  // namespace

size_t device_bytes(const opf_problem* p) { return layout_of(p, nparts_of(p)).total; }

void device_upload(opf_problem* p, void* arena, size_t bytes, cudaStream_t s) {
    if (p->uploaded) throw Error(OPF_ERR_STATE, "problem already uploaded");
    const int np = nparts_of(p);
    const Layout L = layout_of(p, np);
    OPF_CUDA(cudaGetDevice(&p->device));
    if (arena) {
        if (bytes < L.total) throw Error(OPF_ERR_INVALID_ARG, "device arena too small");
        if (((uintptr_t)arena) & 255) throw Error(OPF_ERR_INVALID_ARG, "device arena must be 256-byte aligned");
        p->arena = (char*)arena;
        p->owns_arena = false;
    } else {
        void* ptr = nullptr;
        OPF_CUDA(cudaMallocAsync(&ptr, L.total, s));
        p->arena = (char*)ptr;
        p->owns_arena = true;
    }
    p->arena_bytes = L.total;
    p->nparts = np;
    char* a = p->arena;
    const Packed& k = p->pk;
    p->d64.lo = a + L.lo; p->d64.hi = a + L.hi; p->d64.invk = a + L.invk; p->d64.cik = a + L.cik; p->d64.zg = a + L.zg;
    p->d32.lo = a + L.lo32; p->d32.hi = a + L.hi32; p->d32.invk = a + L.invk32; p->d32.cik = a + L.cik32; p->d32.zg = a + L.zg32;
    p->d64.xl = a + L.xl; p->d64.lam = a + L.lam; p->d64.bbar = a + L.bbar; p->d64.xl0 = a + L.xl0; p->d64.P = a + L.P64;
    p->d32.xl = a + L.xl32; p->d32.lam = a + L.lam32; p->d32.bbar = a + L.bbar32; p->d32.xl0 = a + L.xl0_32; p->d32.P = a + L.P32;
    p->gptr = (int32_t*)(a + L.gptr); p->gcol = (int32_t*)(a + L.gcol); p->gidx = (int32_t*)(a + L.gidx);
    p->tiles = (Tile*)(a + L.tiles); p->cost = (double*)(a + L.cost); p->partials = (double*)(a + L.partials);
    p->ctl = (Ctl*)(a + L.ctl);
    if (!p->ctl_host) OPF_CUDA(cudaMallocHost((void**)&p->ctl_host, sizeof(Ctl)));
    std::memset(p->ctl_host, 0, sizeof(Ctl));

    // host staging of every array (pageable; the copies are synchronized below)
    auto h2d = [&](void* dst, const void* src, size_t n) {
        if (n) OPF_CUDA(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s));
    };
    const Model& M = p->model;
    std::vector<float> f;
    auto h2d32 = [&](void* dst, const std::vector<double>& src) {
        f.assign(src.begin(), src.end());
        h2d(dst, f.data(), f.size() * sizeof(float));
        OPF_CUDA(cudaStreamSynchronize(s));
    };
    h2d(p->d64.lo, M.lo.data(), k.ng * 8); h2d(p->d64.hi, M.hi.data(), k.ng * 8);
    h2d(p->d64.invk, k.invk.data(), k.ng * 8); h2d(p->d64.cik, k.cik.data(), k.ng * 8);
    h2d32(p->d32.lo, M.lo); h2d32(p->d32.hi, M.hi); h2d32(p->d32.invk, k.invk); h2d32(p->d32.cik, k.cik);
    h2d(p->gptr, k.gptr.data(), (k.ng + 1) * 4); h2d(p->gcol, k.gcol.data(), k.nl * 4); h2d(p->gidx, k.gidx.data(), k.nl * 4);
    h2d(p->tiles, k.tiles.data(), k.tiles.size() * sizeof(Tile));
    h2d(p->cost, M.c.data(), k.ng * 8);
    h2d(p->d64.bbar, k.bbar.data(), k.nl * 8); h2d(p->d64.xl0, k.xl0.data(), k.nl * 8);
    h2d32(p->d32.bbar, k.bbar); h2d32(p->d32.xl0, k.xl0);
    h2d(p->d64.P, k.P.data(), k.mat_elems * 8);
    h2d32(p->d32.P, k.P);
    OPF_CUDA(cudaMemsetAsync(p->partials, 0, (size_t)np * 8 * sizeof(double), s));
    OPF_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), s));
    enqueue_init<double>(p, s);
    enqueue_init<float>(p, s);
    OPF_CUDA(cudaStreamSynchronize(s));
    p->cur_prec = OPF_FP64;
    p->cold = true;
    p->uploaded = true;
}

int32_t device_solve(opf_problem* p, const opf_params& prm, cudaStream_t s, opf_info* info) {
    DeviceGuard g(p->device);
    auto t0 = std::chrono::steady_clock::now();
    const int prec = prm.precision;
    if (!prm.warm_start) {
        if (prec == OPF_FP64) enqueue_init<double>(p, s);
        else enqueue_init<float>(p, s);
        p->cur_prec = prec;
    } else {
        sync_state_to(p, prec, s);
    }
    // parameters -> device control block (iteration state kept)
    OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    Ctl c = *p->ctl_host;
    c.rho = prm.rho; c.inv_rho = 1.0 / prm.rho;
    c.eps_abs_prim = prm.eps_abs_prim; c.eps_abs_dual = prm.eps_abs_dual; c.eps_rel = prm.eps_rel;
    c.criterion = prm.criterion; c.K = prm.check_every;
    const long long mi = (long long)c.iter + prm.max_iter;
    c.max_iter = (int32_t)(mi > INT32_MAX ? INT32_MAX : mi);
    c.status = CTL_RUNNING; c.stop = 0;
    *p->ctl_host = c;
    OPF_CUDA(cudaMemcpyAsync(p->ctl, p->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    if (prm.max_iter > 0) {
        if (prec == OPF_FP64) run_solve<double>(p, prm, s);
        else run_solve<float>(p, prm, s);
    } else {
        OPF_CUDA(cudaStreamSynchronize(s));
    }
    p->cold = false;
    const Ctl& r = *p->ctl_host;
    int32_t st = OPF_NOT_CONVERGED;
    if (r.status == CTL_CONVERGED) st = OPF_OK;
    else if (r.status == CTL_NUMERIC) st = OPF_ERR_NUMERIC;
    else if (prm.criterion == OPF_CRIT_NEVER && r.status == CTL_MAXITER) st = OPF_OK;
    if (info) {
        info->status = st;
        info->iters = r.iter;
        info->first_rel_iter = r.first_rel;
        info->pres = r.pres; info->dres = r.dres; info->eps_prim = r.eps_prim; info->eps_dual = r.eps_dual;
        info->objective = r.objective;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

void device_get_state(const opf_problem* p, double* xg, double* xl, double* lam, cudaStream_t s) {
    DeviceGuard g(p->device);
    const int nl = p->pk.nl, ng = p->pk.ng;
    const DevPrec& d = p->cur_prec == OPF_FP64 ? p->d64 : p->d32;
    const size_t w = p->cur_prec == OPF_FP64 ? 8 : 4;
    std::vector<char> bz(ng * w), bx(nl * w), bl(nl * w);
    if (xg) OPF_CUDA(cudaMemcpyAsync(bz.data(), d.zg, ng * w, cudaMemcpyDeviceToHost, s));
    if (xl) OPF_CUDA(cudaMemcpyAsync(bx.data(), d.xl, nl * w, cudaMemcpyDeviceToHost, s));
    if (lam) OPF_CUDA(cudaMemcpyAsync(bl.data(), d.lam, nl * w, cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    auto get = [&](const std::vector<char>& b, int i) {
        return w == 8 ? ((const double*)b.data())[i] : (double)((const float*)b.data())[i];
    };
    if (xg)
        for (int i = 0; i < ng; ++i) xg[i] = get(bz, i);
    for (int c = 0; c < nl; ++c) {
        const int dv = p->pk.dev_of_canon[c];
        if (xl) xl[c] = get(bx, dv);
        if (lam) lam[c] = get(bl, dv);
    }
}

void device_set_state(opf_problem* p, const double* xl, const double* lam, cudaStream_t s) {
    DeviceGuard g(p->device);
    const int nl = p->pk.nl;
    std::vector<double> a(nl), b(nl);
    std::vector<float> af(nl), bf(nl);
    for (int c = 0; c < nl; ++c) {
        const int dv = p->pk.dev_of_canon[c];
        a[dv] = xl ? xl[c] : 0.0;
        b[dv] = lam ? lam[c] : 0.0;
        af[dv] = (float)a[dv];
        bf[dv] = (float)b[dv];
    }
    OPF_CUDA(cudaMemcpyAsync(p->d64.xl, a.data(), nl * 8, cudaMemcpyHostToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(p->d64.lam, b.data(), nl * 8, cudaMemcpyHostToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(p->d32.xl, af.data(), nl * 4, cudaMemcpyHostToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(p->d32.lam, bf.data(), nl * 4, cudaMemcpyHostToDevice, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    p->cold = false;
}

namespace {

template <typename T>
double time_graph(opf_problem* p, int which, int reps, cudaStream_t s) {
    const DevPrec& d = sizeof(T) == 8 ? p->d64 : p->d32;
    View<T> v = view_of<T>(p, d);
    const int zb = (p->pk.ng + kZThreads - 1) / kZThreads;
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    OPF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < reps; ++r) {
        if (which == 0) z_kernel<T><<<zb, kZThreads, 0, cs>>>(v, 0);
        else if (which <= 2) x_kernel<T><<<p->nparts, kXWarps * 32, 0, cs>>>(v, 0);
        else finalize_kernel<T><<<1, kFinThreads, 0, cs>>>(v, 0, 0);
    }
    OPF_CUDA(cudaStreamEndCapture(cs, &g));
    OPF_CUDA(cudaStreamDestroy(cs));
    OPF_CUDA(cudaGraphInstantiate(&ge, g, 0));
    cudaEvent_t e0, e1;
    OPF_CUDA(cudaEventCreate(&e0));
    OPF_CUDA(cudaEventCreate(&e1));
    OPF_CUDA(cudaGraphLaunch(ge, s));            // warm
    OPF_CUDA(cudaEventRecord(e0, s));
    OPF_CUDA(cudaGraphLaunch(ge, s));
    OPF_CUDA(cudaEventRecord(e1, s));
    OPF_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    OPF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    return 1e3 * (double)ms / reps;
}

}  // namespace

void device_profile(opf_problem* p, const opf_params& prm, int reps, cudaStream_t s, double* us) {
    DeviceGuard g(p->device);
    const int prec = prm.precision;
    sync_state_to(p, prec, s);
    const DevPrec& d = prec == OPF_FP64 ? p->d64 : p->d32;
    const size_t w = prec == OPF_FP64 ? 8 : 4;
    const size_t nl = p->pk.nl, ng = p->pk.ng;
    char* save = nullptr;
    const size_t bytes = 2 * nl * w + ng * w + sizeof(Ctl);
    OPF_CUDA(cudaMallocAsync((void**)&save, bytes, s));
    OPF_CUDA(cudaMemcpyAsync(save, d.xl, nl * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(save + nl * w, d.lam, nl * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(save + 2 * nl * w, d.zg, ng * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(save + 2 * nl * w + ng * w, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    // control block for timing: no launch is skipped (huge bound); K = 1 makes
    // every local-update launch compute residual partials (which == 2)
    Ctl c = *p->ctl_host;
    c.rho = prm.rho; c.inv_rho = 1.0 / prm.rho; c.iter = 0; c.max_iter = INT32_MAX;
    for (int which = 0; which < 4; ++which) {
        c.K = (which == 2) ? 1 : (1 << 20);
        c.iter = 0;
        *p->ctl_host = c;
        OPF_CUDA(cudaMemcpyAsync(p->ctl, p->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        us[which] = prec == OPF_FP64 ? time_graph<double>(p, which, reps, s) : time_graph<float>(p, which, reps, s);
    }
    OPF_CUDA(cudaMemcpyAsync(d.xl, save, nl * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(d.lam, save + nl * w, nl * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(d.zg, save + 2 * nl * w, ng * w, cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaMemcpyAsync(p->ctl, save + 2 * nl * w + ng * w, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
    OPF_CUDA(cudaFreeAsync(save, s));
    OPF_CUDA(cudaStreamSynchronize(s));
}

void device_free(opf_problem* p) {
    DeviceGuard g(p->device);
    for (auto& kv : p->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    p->graphs.clear();
    if (p->owns_arena && p->arena) cudaFree(p->arena);
    p->arena = nullptr;
    if (p->ctl_host) cudaFreeHost(p->ctl_host);
    p->ctl_host = nullptr;
}

}  // namespace opf
