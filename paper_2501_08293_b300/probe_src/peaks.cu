// Device peaks that bound the solver's kernels, measured with CUDA events:
//   FP64 and FP32 FMA throughput (8 independent FMA chains per thread over
//   148 x 8 CTAs of 256 threads), and the read bandwidth of a 64 MB buffer
//   that stays in L2 (20 passes, __ldcg float4 loads).
// Built and run by paper_2501_08293_b300/probe.py.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void l2_read(const float4* __restrict__ in, size_t n, int reps, float* out) {
    float acc = 0;
    for (int r = 0; r < reps; ++r)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            float4 v = __ldcg(in + i); acc += v.x + v.y + v.z + v.w;
        }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}
template <typename T> void run(const char* name) {
    int blocks = 148 * 8, threads = 256, iters = 20000;
    T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    fma_kernel<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);
    cudaEventRecord(e0); fma_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001); cudaEventRecord(e1);
    cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * iters * (double)blocks * threads;
    printf("%s FMA: %.3f TFLOP/s (%.3f ms) err=%s\n", name, flops / (ms * 1e-3) / 1e12, ms, cudaGetErrorString(cudaGetLastError()));
    cudaFree(out);
}
int main() {
    run<double>("fp64"); run<float>("fp32");
    size_t bytes = 64ull << 20; size_t n = bytes / 16;
    float4* in; cudaMalloc(&in, bytes); cudaMemset(in, 0, bytes);
    float* out; int blocks = 148 * 4, threads = 512; cudaMalloc(&out, sizeof(float) * blocks * threads);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    l2_read<<<blocks, threads>>>(in, n, 2, out);
    cudaEventRecord(e0); l2_read<<<blocks, threads>>>(in, n, 20, out); cudaEventRecord(e1);
    cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms, e0, e1);
    printf("L2-resident read (64 MB x20): %.1f GB/s err=%s\n", 20.0 * bytes / (ms * 1e-3) / 1e9, cudaGetErrorString(cudaGetLastError()));
    return 0;
}
