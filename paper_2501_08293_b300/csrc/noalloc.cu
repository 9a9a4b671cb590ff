// Residual norms for caller-owned device vectors, with no device allocation
// at all: pres = ||v - z||, dres = rho ||z - z_prev||, eps_prim = eps_rel
// max(||v||, ||z||), eps_dual = eps_rel ||lambda|| (2-norms over all locals).
//
// Who needs this: code that runs where cudaMalloc / cudaFree (and any
// allocating library routine) are off limits -- inside a caller's memory
// pool that must not grow, in a plugin that is handed pre-allocated buffers,
// or in a process that forbids allocations after start-up.  Such a caller
// brings its inputs and its output buffer; the per-CTA partial sums that the
// reduction needs live in a fixed array of this library's module instead.
//
// The reduction is the same two-stage scheme as the solver's residual
// check: each CTA sums its slice of the five squared norms in FP64
// (||v - z||^2, ||z - z_prev||^2, ||v||^2, ||z||^2, ||lambda||^2) and writes
// them to its slot of the scratch array; one CTA then adds the slots in a
// fixed order.  Every slot that the second stage reads is written by the
// first stage of the same call, so nothing has to be cleared between calls.
#include <cuda.h>            // driver types only (entry points resolved through the runtime)
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.hpp"

namespace opf {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 8;                               // locals per thread
constexpr int kNaMaxBlocks = 2048;                            // scratch slots
constexpr long long kNaMaxLocals = (long long)kNaMaxBlocks * kNaThreads * kNaPerThread;   // 4,194,304

// One record of 8 doubles per CTA (5 used): 128 KiB held by every device
// that loads the library, for the life of the process.
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks * 8];

__global__ void __launch_bounds__(kNaThreads) noalloc_partials(const double* __restrict__ v, const double* __restrict__ z,
                                                               const double* __restrict__ zp, const double* __restrict__ lam,
                                                               int n, double* scratch) {
    __shared__ double red[kNaThreads / 32][5];
    double a[5] = {0, 0, 0, 0, 0};
    const int base = blockIdx.x * kNaThreads * kNaPerThread;
    for (int q = 0; q < kNaPerThread; ++q) {
        const int j = base + q * kNaThreads + threadIdx.x;
        if (j < n) {
            const double vv = v[j], zz = z[j], dz = zz - zp[j], pr = vv - zz, l = lam[j];
            a[0] += pr * pr; a[1] += dz * dz; a[2] += vv * vv; a[3] += zz * zz; a[4] += l * l;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < 5; ++k)
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    if (lane == 0)
        for (int k = 0; k < 5; ++k) red[warp][k] = a[k];
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0;
        for (int w = 0; w < kNaThreads / 32; ++w) s += red[w][threadIdx.x];
        scratch[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kNaThreads) noalloc_finish(const double* scratch, int nblocks, double rho,
                                                             double eps_rel, double* out) {
    __shared__ double sh[5][kNaThreads];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kNaThreads)
        for (int k = 0; k < 5; ++k) s[k] += scratch[(size_t)b * 8 + k];
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(sh[0][0]);
        out[1] = rho * sqrt(sh[1][0]);
        out[2] = eps_rel * fmax(sqrt(sh[2][0]), sqrt(sh[3][0]));
        out[3] = eps_rel * sqrt(sh[4][0]);
    }
}

// Device address of the scratch array.  The array's host-side name is not a
// device address: cudaGetSymbolAddress gives the address in the current
// context's copy of this module.  A context has its own copy (a non-primary
// context, or the primary context again after cudaDeviceReset, loads the
// module anew, possibly at another address), so the address is cached per
// context, keyed by the driver's unique context id (cuCtxGetId, never
// reused within a process), and looked up once per context.
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);
std::mutex g_mu;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
constexpr int kCacheSlots = 64;
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
ScratchSlot g_cache[kCacheSlots];
int g_cache_next = 0;

void resolve_driver_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return;
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e0 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
    cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
    if (e0 != cudaSuccess || e1 != cudaSuccess || q0 != cudaDriverEntryPointSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
        throw Error(OPF_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f0);
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f1);
}

// Unique id of the calling thread's current context; 0 when there is none.
unsigned long long current_context_id() {
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

double* symbol_address() {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        throw Error(OPF_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    return static_cast<double*>(ptr);
}

double* scratch_for_current_context() {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_driver_entry_points();
    unsigned long long id = current_context_id();
    if (id == 0) {
        // no current context yet: the runtime makes the device's primary
        // context current when it resolves the symbol
        double* p = symbol_address();
        id = current_context_id();
        if (id == 0) throw Error(OPF_ERR_CUDA, "no current CUDA context after resolving the scratch array");
        g_cache[g_cache_next] = ScratchSlot{id, p};
        g_cache_next = (g_cache_next + 1) % kCacheSlots;
        return p;
    }
    for (const ScratchSlot& c : g_cache)
        if (c.ctx_id == id) return c.ptr;
    double* p = symbol_address();
    g_cache[g_cache_next] = ScratchSlot{id, p};
    g_cache_next = (g_cache_next + 1) % kCacheSlots;
    return p;
}

}  // namespace

void residuals_noalloc(const double* v, const double* z, const double* zp, const double* lam, long long n,
                       double rho, double eps_rel, double* out, cudaStream_t s) {
    if (n < 0 || n > kNaMaxLocals)
        throw Error(OPF_ERR_INVALID_ARG, "n_local = " + std::to_string(n) + " is outside [0, " +
                                             std::to_string(kNaMaxLocals) + "], the size the fixed scratch supports");
    if (!out || (n > 0 && (!v || !z || !zp || !lam))) throw Error(OPF_ERR_INVALID_ARG, "NULL device pointer");
    if (!(rho > 0.0)) throw Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
    double* scratch = scratch_for_current_context();
    const int per_block = kNaThreads * kNaPerThread;
    const int nb = n > 0 ? (int)((n + per_block - 1) / per_block) : 1;
    noalloc_partials<<<nb, kNaThreads, 0, s>>>(v, z, zp, lam, (int)n, scratch);
    noalloc_finish<<<1, kNaThreads, 0, s>>>(scratch, nb, rho, eps_rel, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(OPF_ERR_CUDA, std::string("residual kernels: ") + cudaGetErrorString(e));
}

}  // namespace opf
