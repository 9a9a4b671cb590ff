// Residual norms of Eq. (termination) for caller-owned device vectors, with
// no device allocation at all.
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

// Device address of the scratch array, looked up once per device with that
// device current (the symbol's host-side name is not a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

double* scratch_for_current_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) throw Error(OPF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) throw Error(OPF_ERR_INVALID_ARG, "device index beyond 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            throw Error(OPF_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    return g_scratch_ptr[dev];
}

}  // namespace

void residuals_noalloc(const double* v, const double* z, const double* zp, const double* lam, long long n,
                       double rho, double eps_rel, double* out, cudaStream_t s) {
    if (n < 0 || n > kNaMaxLocals)
        throw Error(OPF_ERR_INVALID_ARG, "n_local = " + std::to_string(n) + " is outside [0, " +
                                             std::to_string(kNaMaxLocals) + "], the size the fixed scratch supports");
    if (!out || (n > 0 && (!v || !z || !zp || !lam))) throw Error(OPF_ERR_INVALID_ARG, "NULL device pointer");
    if (!(rho > 0.0)) throw Error(OPF_ERR_INVALID_ARG, "rho must be > 0");
    double* scratch = scratch_for_current_device();
    const int per_block = kNaThreads * kNaPerThread;
    const int nb = n > 0 ? (int)((n + per_block - 1) / per_block) : 1;
    noalloc_partials<<<nb, kNaThreads, 0, s>>>(v, z, zp, lam, (int)n, scratch);
    noalloc_finish<<<1, kNaThreads, 0, s>>>(scratch, nb, rho, eps_rel, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(OPF_ERR_CUDA, std::string("residual kernels: ") + cudaGetErrorString(e));
}

}  // namespace opf
