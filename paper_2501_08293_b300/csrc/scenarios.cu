// Multi-scenario engine: one feeder topology, S load scenarios (different
// load draws a, b on the same loads) iterated together.
//
// Every scenario runs Algorithm 1 on its own model.  Only the load
// components depend on the draw: their right-hand sides always (b_s holds
// the constant-power part of Eq. volt_load_model), their rows A_s when the
// load is voltage dependent (alpha or beta != 0).  Bus, line and generator
// components, the bounds and the costs are shared, so for those components
// the local update of Eq. (closed_2) is one small matrix product
// X_s = P_s U_s + bbar_s over the S columns of U_s.
//
// Data layout is scenario-minor: element (j, k) of a per-local array at
// j * Sp + k (Sp = S rounded up to a multiple of 64), so the 32 lanes of a
// warp hold 64 consecutive scenarios as float2 pairs.  Kernels, FP32 sweeps
// with FP64 residual sums:
//   sc_z_kernel   one half-warp per global: the copy terms of every scenario,
//                 summed in the CSR order of the single-instance engines,
//                 Eq. (global_sparse); stopped scenarios are not written;
//   sc_xs_kernel  components of at most 8 locals, one warp each (grid-
//                 stride, fixed order): u of every column in registers, per
//                 row r the GEMV sum_c P[c][r] u_c with packed fmas on
//                 scenario pairs (P broadcast by shuffles; per-scenario P for
//                 voltage-dependent loads), the dual update of Eq. (ADMM-3)
//                 and the copy term for the next global update;
//   sc_x_kernel   larger components, one CTA each: u staged in shared
//                 memory, rows spread over the warps, same arithmetic;
//                 both come as a plain and a check instantiation, the check
//                 one also forming per-scenario FP64 partial sums of
//                 Eq. (termination);
//   sc_fin_kernel one CTA per scenario: fixed-order sum of the partials,
//                 the stopping rule; a stopped scenario keeps the state of
//                 its deciding check.
// A CUDA graph runs K iterations and the check in the body of a device-side
// while node until every scenario has stopped (a body that has fewer than K
// iterations left runs them at its last positions, so its check is still the
// last one).
//
// The arithmetic of a scenario is the same sequence of operations as the
// single-instance engines (same copy order, even/odd GEMV accumulators,
// same fused multiply-adds), so its iterates are bit-identical to solving
// that scenario alone in FP32; only the order of the residual sums differs.
//
// Tensor cores (opf_scenarios_set_xupdate): for the small components whose
// operator is shared by every scenario, the product X = P U over 64
// scenarios is D (16 scenarios x 8 rows) = U^T P^T per block of 16
// scenarios on mma.sync m16n8k8 with TF32 inputs, each operand split in two
// TF32 parts and three products (hi*hi + hi*lo + lo*hi) with FP32
// accumulation -- about FP32 accuracy, not the same bits.  It runs on the
// iterations between checks; check iterations and the per-scenario
// operators keep the CUDA-core path.  Per element and scenario the product
// reads u and writes x (8 bytes) against 2 n flops, about n/4 flop per byte
// with n ~ 7: far below either ridge point, so what the tensor-core path can
// change is the instruction count (no operator broadcast by shuffles) and
// the latency chain of the GEMV, not the bytes moved.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "arith.cuh"
#include "problem.hpp"

namespace opf {
namespace {

#define SC_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw Error(e_ == cudaErrorMemoryAllocation ? OPF_ERR_OOM : OPF_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

constexpr int kScWarps = 4;          // warps per CTA of sc_x_kernel

// per-scenario state (device)
struct ScState {
    int32_t active, status, iter, first_rel, checks;
    int32_t _pad;
    double pres, dres, eps_prim, eps_dual, objective;
};

// shared solve parameters (device)
struct ScCtl {
    float rho, inv_rho;
    double eps_abs_prim, eps_abs_dual, eps_rel;
    int32_t criterion, max_iter, K, iter;   // iter: iterations run by the sweep
    int32_t running;                        // scenarios still active
};

// component descriptor: canonical first local, size | flags << 16, offset of
// its operator (shared: n*n floats; per scenario: n*n*Sp floats, element
// (c*n + r)*Sp + k), offset of its bbar (shared: n floats; per scenario:
// (boff + r)*Sp + k)
struct ScComp {
    int32_t loc0, nf, poff, boff;
};
constexpr int kVarP = 1 << 16, kVarB = 2 << 16;

struct ScView {
    const ScComp* comps;
    const float* Ps;
    const float* Pv;
    const float* bs;
    const float* bv;
    const int32_t* gidx;
    const int32_t* gptr;
    const int32_t* gcol;
    const float* invk;
    const float* cik;
    const float* lo;
    const float* hi;
    const double* cost;
    const float* xl0;
    float* W;      // copy terms x - lambda / rho
    float* L;      // lambda
    float* X;      // x_s (written around checks)
    float* Z;      // global vector
    double* partials;
    ScState* st;
    uint32_t* amask;         // active scenarios, one bit each
    ScCtl* ctl;
    int32_t ncomp, nl, ng, Sp, nctas, maxn;
    int32_t nsmall;          // comps[0, nsmall) have n <= kSmallN, the rest more
    int32_t nctas_s;         // CTAs of sc_xs_kernel (partials slots [0, nctas_s))
};
constexpr int kSmallN = 8;
constexpr int kXsWarps = 8;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// A body of the sweep runs r = min(K, max_iter - iter) iterations at its
// last r positions q = K - r, ..., K - 1, so the check iteration is always
// q = K - 1: the local-update kernels come in a check and a plain
// instantiation, and the plain one carries no residual code.
__device__ __forceinline__ int body_start(const ScCtl* ctl) {
    return ctl->K - min(ctl->K, ctl->max_iter - ctl->iter);
}

__global__ void sc_init_kernel(ScView v) {
    const size_t n = (size_t)v.nl * v.Sp;
    const float inv_rho = v.ctl->inv_rho;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float x = v.xl0[e / v.Sp];
        v.X[e] = x;
        v.L[e] = 0.f;
        v.W[e] = copy_term(x, 0.f, inv_rho);
    }
}

// Eq. (global_sparse) for global i, every scenario: one half-warp per
// global, four scenarios per lane (16-byte loads of the copies' terms).  The
// copy list is loaded by the lanes together and broadcast, so the copies'
// rows are fetched without a dependent load between them.
__global__ void __launch_bounds__(256) sc_z_kernel(ScView v, int q) {
    const ScCtl* ctl = v.ctl;
    if (q < body_start(ctl)) return;
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 4);
    const int hl = threadIdx.x & 15;
    const unsigned hm = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    if (i >= v.ng) return;                          // whole half-warps leave together
    const float inv_rho = ctl->inv_rho;
    const int b = v.gptr[i], e = v.gptr[i + 1];
    const float invk = v.invk[i], cik = v.cik[i], lo = v.lo[i], hi = v.hi[i];
    for (int k0 = 4 * hl; k0 < v.Sp; k0 += 64) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int qb = b; qb < e; qb += 16) {
            const int cnt = min(16, e - qb);
            const int my = hl < cnt ? v.gcol[qb + hl] : 0;
            int c = 0;
            for (; c + 3 < cnt; c += 4) {
                float4 w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    w[h] = *reinterpret_cast<const float4*>(v.W + (size_t)__shfl_sync(hm, my, c + h, 16) * v.Sp + k0);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    s.x += w[h].x; s.y += w[h].y; s.z += w[h].z; s.w += w[h].w;
                }
            }
            for (; c < cnt; ++c) {
                const float4 w = *reinterpret_cast<const float4*>(v.W + (size_t)__shfl_sync(hm, my, c, 16) * v.Sp + k0);
                s.x += w.x; s.y += w.y; s.z += w.z; s.w += w.w;
            }
        }
        const unsigned act = (v.amask[k0 >> 5] >> (k0 & 31)) & 0xFu;
        float* zp = v.Z + (size_t)i * v.Sp + k0;
        if (act == 0xFu) {
            *reinterpret_cast<float4*>(zp) = make_float4(global_from_sum(s.x, invk, cik, inv_rho, lo, hi),
                                                         global_from_sum(s.y, invk, cik, inv_rho, lo, hi),
                                                         global_from_sum(s.z, invk, cik, inv_rho, lo, hi),
                                                         global_from_sum(s.w, invk, cik, inv_rho, lo, hi));
        } else {
            if (act & 1u) zp[0] = global_from_sum(s.x, invk, cik, inv_rho, lo, hi);
            if (act & 2u) zp[1] = global_from_sum(s.y, invk, cik, inv_rho, lo, hi);
            if (act & 4u) zp[2] = global_from_sum(s.z, invk, cik, inv_rho, lo, hi);
            if (act & 8u) zp[3] = global_from_sum(s.w, invk, cik, inv_rho, lo, hi);
        }
    }
}

// Residual terms of one local for the lane's two scenarios, summed in FP32
// within a component (at most a few dozen terms), then added to the FP64
// per-lane sums once per component.
__device__ __forceinline__ void sc_terms(float (&f)[2][5], float2 z, float2 xn, float2 xo, float2 ln) {
    const float zz[2] = {z.x, z.y}, xs[2] = {xn.x, xn.y}, xx[2] = {xo.x, xo.y}, ll[2] = {ln.x, ln.y};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float pr = zz[h] - xs[h], dz = xs[h] - xx[h];
        f[h][0] = fmaf(pr, pr, f[h][0]);
        f[h][1] = fmaf(dz, dz, f[h][1]);
        f[h][2] = fmaf(zz[h], zz[h], f[h][2]);
        f[h][3] = fmaf(xs[h], xs[h], f[h][3]);
        f[h][4] = fmaf(ll[h], ll[h], f[h][4]);
    }
}
__device__ __forceinline__ void sc_accumulate(double (&acc)[2][5], const float (&f)[2][5]) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int m = 0; m < 5; ++m) acc[h][m] += (double)f[h][m];
}

// Residual sums of one check: per-lane sums of the lane's two scenarios,
// reduced over the CTA's warps in a fixed order into partials slot `slot`.
template <int W>
__device__ __forceinline__ void sc_partials(const double (&acc)[2][5], double (*red)[5][64], double* partials,
                                            int slot, int Sp, int pass) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int m = 0; m < 5; ++m) {
        red[warp][m][2 * lane] = acc[0][m];
        red[warp][m][2 * lane + 1] = acc[1][m];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 5 * 64; t += blockDim.x) {
        const int m = t / 64, kk = t % 64;
        double a = 0;
        for (int w = 0; w < W; ++w) a += red[w][m][kk];
        partials[((size_t)slot * 5 + m) * Sp + pass * 64 + kk] = a;
    }
    __syncthreads();
}

// Components of at most kSmallN locals (most of a feeder): one warp per
// component.  u of every column for the lane's scenario pair is held in
// registers (the loads of all columns are issued together), then each row's
// GEMV runs over NC = 4, 6 or 8 columns (n rounded up; the padded operator
// is zero past n, so those columns add exact zeros) in the order of the
// single-instance engines: even columns into y0, odd into y1.  z and lambda
// of a row are read again at the row (first-level cache hits) instead of
// being kept in registers, which lets four CTAs share an SM.
template <bool check, int NC>
__device__ __forceinline__ void sc_small_rows(const ScView& v, const ScComp& cd, int gl, int k0, int lane, bool a0,
                                              bool a1, bool keepx, float rho, float inv_rho, const float2 (&u)[kSmallN],
                                              float (&f)[2][5]) {
    const int n = cd.nf & 0xFFFF, j0 = cd.loc0, Sp = v.Sp;
    const bool var = (cd.nf & kVarP) != 0;
    const float4 pq = (!var && lane < 16) ? reinterpret_cast<const float4*>(v.Ps + cd.poff)[lane]
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
    const float* Pv = v.Pv + cd.poff;
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        if (r < n) {
            float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
            if (!var) {
                // element (c, r) of the padded 8 x 8 operator: lane 2c + r/4
                const float pe = (r & 3) == 0 ? pq.x : (r & 3) == 1 ? pq.y : (r & 3) == 2 ? pq.z : pq.w;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float ps = __shfl_sync(0xffffffffu, pe, 2 * c + (r >> 2));
                    if (c & 1) y1 = ffma2(make_float2(ps, ps), u[c], y1);
                    else y0 = ffma2(make_float2(ps, ps), u[c], y0);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c < n) {
                        const float2 pv = *reinterpret_cast<const float2*>(Pv + (size_t)(c * n + r) * Sp + k0);
                        if (c & 1) y1 = ffma2(pv, u[c], y1);
                        else y0 = ffma2(pv, u[c], y0);
                    }
                }
            }
            const size_t e = (size_t)(j0 + r) * Sp + k0;
            const int g = __shfl_sync(0xffffffffu, gl, r);
            const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)g * Sp + k0);
            const float2 l = *reinterpret_cast<const float2*>(v.L + e);
            float2 bb;
            if (cd.nf & kVarB) bb = *reinterpret_cast<const float2*>(v.bv + (size_t)(cd.boff + r) * Sp + k0);
            else bb = make_float2(v.bs[cd.boff + r], v.bs[cd.boff + r]);
            const float xn0 = (y0.x + y1.x) + bb.x, xn1 = (y0.y + y1.y) + bb.y;
            const float ln0 = dual_of(l.x, rho, z.x, xn0), ln1 = dual_of(l.y, rho, z.y, xn1);
            const float wn0 = copy_term(xn0, ln0, inv_rho), wn1 = copy_term(xn1, ln1, inv_rho);
            if constexpr (check) {
                const float2 xo = *reinterpret_cast<const float2*>(v.X + e);
                sc_terms(f, z, make_float2(xn0, xn1), xo, make_float2(ln0, ln1));
            }
            if (a0) {
                v.L[e] = ln0;
                v.W[e] = wn0;
                if (keepx) v.X[e] = xn0;
            }
            if (a1) {
                v.L[e + 1] = ln1;
                v.W[e + 1] = wn1;
                if (keepx) v.X[e + 1] = xn1;
            }
        }
    }
}

// ---- tensor-core (3xTF32) local update of small shared-operator components
// x -> (hi, lo), both TF32 (hi = x rounded to TF32, lo = the remainder
// rounded to TF32): about 21 significant bits of x.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
// D += A B, A 16 x 8 (row-major), B 8 x 8 (column-major), TF32 in, FP32
// accumulate; fragment of lane l (g = l / 4, t = l % 4): a = {A[g][t],
// A[g+8][t], A[g][t+4], A[g+8][t+4]}, b = {B[t][g], B[t+4][g]},
// d = {D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]}.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One small component with a shared operator, the warp's 64 scenarios of
// this pass [base, base + 64) on tensor cores: for each block of 16
// scenarios, D (16 scenarios x 8 rows) = U^T (16 x 8 columns) P^T (8 x 8),
// i.e. D[s][r] = sum_c P[r][c] u_c(s), in three TF32 products (lo*hi +
// hi*lo + hi*hi, FP32 accumulation), then x = D + bbar, the dual update
// and the copy term for the next global update.  Columns and rows past n
// are zero in the padded operator (and u is zero there).  Fragment row g of
// a block holds scenario 2g and row g + 8 scenario 2g + 1, so a lane's two
// rows are adjacent scenarios: its A operands, its outputs of one matrix row
// and their z, lambda, bbar, x are float2 pairs (lanes g = 0..7 of one
// column cover 64 contiguous bytes).
__device__ __forceinline__ void sc_small_tc(const ScView& v, const ScComp& cd, int gl, int base, int lane, bool keepx,
                                            float rho, float inv_rho) {
    const int n = cd.nf & 0xFFFF, j0 = cd.loc0, Sp = v.Sp;
    const int g = lane >> 2, t = lane & 3;
    const float* Ps = v.Ps + cd.poff;              // P[r][c] at c * 8 + r
    uint32_t bh0, bl0, bh1, bl1;
    split_tf32(Ps[t * 8 + g], bh0, bl0);           // B[t][g] = P[g][t]
    split_tf32(Ps[(t + 4) * 8 + g], bh1, bl1);     // B[t+4][g] = P[g][t+4]
    const int gc0 = __shfl_sync(0xffffffffu, gl, t), gc1 = __shfl_sync(0xffffffffu, gl, t + 4);
    const int gr0 = __shfl_sync(0xffffffffu, gl, 2 * t), gr1 = __shfl_sync(0xffffffffu, gl, 2 * t + 1);
    const bool c0 = t < n, c1 = t + 4 < n;
    const int rr[2] = {2 * t, 2 * t + 1};
    const int gr[2] = {gr0, gr1};
    const bool var_b = (cd.nf & kVarB) != 0;
    float bsr[2] = {0.f, 0.f};                     // shared bbar of the lane's two rows
    if (!var_b)
        for (int h = 0; h < 2; ++h)
            if (rr[h] < n) bsr[h] = v.bs[cd.boff + rr[h]];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int sp = base + 16 * m + 2 * g;      // the lane's scenario pair (sp, sp + 1)
        auto upair = [&](bool live, int gc, int c) -> float2 {
            if (!live) return make_float2(0.f, 0.f);
            const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)gc * Sp + sp);
            const float2 l = *reinterpret_cast<const float2*>(v.L + (size_t)(j0 + c) * Sp + sp);
            return make_float2(u_of(z.x, l.x, inv_rho), u_of(z.y, l.y, inv_rho));
        };
        const float2 u0 = upair(c0, gc0, t), u1 = upair(c1, gc1, t + 4);
        uint32_t ah[4], al[4];
        split_tf32(u0.x, ah[0], al[0]);            // A[g][t]      (scenario sp,     column t)
        split_tf32(u0.y, ah[1], al[1]);            // A[g + 8][t]  (scenario sp + 1, column t)
        split_tf32(u1.x, ah[2], al[2]);            // A[g][t + 4]
        split_tf32(u1.y, ah[3], al[3]);            // A[g + 8][t + 4]
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_tf32(d, al, bh0, bh1);
        mma_tf32(d, ah, bl0, bl1);
        mma_tf32(d, ah, bh0, bh1);
        const unsigned act = (v.amask[sp >> 5] >> (sp & 31)) & 3u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {              // matrix row r = 2t + h: (d[h], d[h + 2]) = scenarios (sp, sp + 1)
            const int r = rr[h];
            if (r >= n) continue;
            const size_t e = (size_t)(j0 + r) * Sp + sp;
            const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)gr[h] * Sp + sp);
            const float2 l = *reinterpret_cast<const float2*>(v.L + e);
            const float2 bb = var_b ? *reinterpret_cast<const float2*>(v.bv + (size_t)(cd.boff + r) * Sp + sp)
                                    : make_float2(bsr[h], bsr[h]);
            const float xn0 = d[h] + bb.x, xn1 = d[h + 2] + bb.y;
            const float ln0 = dual_of(l.x, rho, z.x, xn0), ln1 = dual_of(l.y, rho, z.y, xn1);
            const float wn0 = copy_term(xn0, ln0, inv_rho), wn1 = copy_term(xn1, ln1, inv_rho);
            if (act == 3u) {
                *reinterpret_cast<float2*>(v.L + e) = make_float2(ln0, ln1);
                *reinterpret_cast<float2*>(v.W + e) = make_float2(wn0, wn1);
                if (keepx) *reinterpret_cast<float2*>(v.X + e) = make_float2(xn0, xn1);
            } else {
                if (act & 1u) {
                    v.L[e] = ln0;
                    v.W[e] = wn0;
                    if (keepx) v.X[e] = xn0;
                }
                if (act & 2u) {
                    v.L[e + 1] = ln1;
                    v.W[e + 1] = wn1;
                    if (keepx) v.X[e + 1] = xn1;
                }
            }
        }
    }
}

// kTC (plain iterations only): components with a shared operator go to the
// tensor-core path above, those with per-scenario operators keep the
// CUDA-core rows.
template <bool check, bool kTC = false>
__global__ void __launch_bounds__(kXsWarps * 32, check ? 2 : 4) sc_xs_kernel(ScView v, int q) {
    __shared__ double red[check ? kXsWarps : 1][5][64];
    const ScCtl* ctl = v.ctl;
    if (q < body_start(ctl)) return;
    const bool keepx = q >= ctl->K - 2;             // x before and at a check
    const float rho = ctl->rho, inv_rho = ctl->inv_rho;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kXsWarps + warp, nw = gridDim.x * kXsWarps;
    const int Sp = v.Sp;
    for (int k0 = 2 * lane, pass = 0; k0 < Sp; k0 += 64, ++pass) {
        const bool a0 = v.st[k0].active != 0, a1 = v.st[k0 + 1].active != 0;
        double acc[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
        // descriptor and globals of the next component are fetched while the
        // current one is computed
        ScComp ncd = gw < v.nsmall ? v.comps[gw] : ScComp{0, 0, 0, 0};
        int ngl = lane < (ncd.nf & 0xFFFF) ? v.gidx[ncd.loc0 + lane] : 0;
        for (int s = gw; s < v.nsmall; s += nw) {
            const ScComp cd = ncd;
            const int gl = ngl;
            const int n = cd.nf & 0xFFFF;
            const int j0 = cd.loc0;
            if constexpr (kTC) {
                if (!(cd.nf & kVarP)) {
                    if (s + nw < v.nsmall) {
                        ncd = v.comps[s + nw];
                        ngl = lane < (ncd.nf & 0xFFFF) ? v.gidx[ncd.loc0 + lane] : 0;
                    }
                    sc_small_tc(v, cd, gl, k0 - 2 * lane, lane, keepx, rho, inv_rho);
                    continue;
                }
            }
            float2 u[kSmallN];
#pragma unroll
            for (int c = 0; c < kSmallN; ++c) {
                const int g = __shfl_sync(0xffffffffu, gl, c);
                if (c < n) {
                    const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)g * Sp + k0);
                    const float2 l = *reinterpret_cast<const float2*>(v.L + (size_t)(j0 + c) * Sp + k0);
                    u[c] = make_float2(u_of(z.x, l.x, inv_rho), u_of(z.y, l.y, inv_rho));
                } else {
                    u[c] = make_float2(0.f, 0.f);
                }
            }
            if (s + nw < v.nsmall) {
                ncd = v.comps[s + nw];
                ngl = lane < (ncd.nf & 0xFFFF) ? v.gidx[ncd.loc0 + lane] : 0;
            }
            float f[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
            if (n <= 4) sc_small_rows<check, 4>(v, cd, gl, k0, lane, a0, a1, keepx, rho, inv_rho, u, f);
            else if (n <= 6) sc_small_rows<check, 6>(v, cd, gl, k0, lane, a0, a1, keepx, rho, inv_rho, u, f);
            else sc_small_rows<check, 8>(v, cd, gl, k0, lane, a0, a1, keepx, rho, inv_rho, u, f);
            if constexpr (check) sc_accumulate(acc, f);
        }
        if constexpr (check) sc_partials<kXsWarps>(acc, red, v.partials, blockIdx.x, Sp, pass);
    }
}

// Components of more than kSmallN locals: one CTA per component (grid-
// stride).  Its warps stage u of every column for the lane's scenario pair
// in shared memory (and the component's operator when it is shared), then
// warp w updates rows r = w, w + kScWarps, ... -- the rows whose columns it
// staged, so z and lambda of a row are read again from the first-level
// cache.  GEMV order as the single-instance engines: even columns into y0,
// odd into y1 up to 32 locals, one sequential accumulator above.
template <bool check>
__global__ void __launch_bounds__(kScWarps * 32, check ? 4 : 8) sc_x_kernel(ScView v, int q) {
    extern __shared__ float2 sdyn[];               // u: maxn x 32, then the operator
    __shared__ double red[check ? kScWarps : 1][5][64];
    const ScCtl* ctl = v.ctl;
    if (q < body_start(ctl)) return;
    const bool keepx = q >= ctl->K - 2;             // x before and at a check
    const float rho = ctl->rho, inv_rho = ctl->inv_rho;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Sp = v.Sp, mn = v.maxn;
    float2* us = sdyn;
    float* psm = reinterpret_cast<float*>(sdyn + (size_t)mn * 32);   // shared operator, mn * mn
    for (int k0 = 2 * lane, pass = 0; k0 < Sp; k0 += 64, ++pass) {
        const bool a0 = v.st[k0].active != 0, a1 = v.st[k0 + 1].active != 0;
        double acc[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
        for (int s = v.nsmall + blockIdx.x; s < v.ncomp; s += gridDim.x) {
            const ScComp cd = v.comps[s];
            const int n = cd.nf & 0xFFFF;
            const int j0 = cd.loc0;
            if (!(cd.nf & kVarP))
                for (int e = threadIdx.x; e < n * n; e += blockDim.x) psm[e] = __ldg(v.Ps + cd.poff + e);
            for (int c = warp; c < n; c += kScWarps) {
                const int g = v.gidx[j0 + c];
                const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)g * Sp + k0);
                const float2 l = *reinterpret_cast<const float2*>(v.L + (size_t)(j0 + c) * Sp + k0);
                us[c * 32 + lane] = make_float2(u_of(z.x, l.x, inv_rho), u_of(z.y, l.y, inv_rho));
            }
            __syncthreads();
            const bool var = (cd.nf & kVarP) != 0;
            const float* Pv = v.Pv + cd.poff;
            float f[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};   // FP32 sums within the component
            for (int r = warp; r < n; r += kScWarps) {
                const size_t e = (size_t)(j0 + r) * Sp + k0;
                float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
                if (!var) {
                    const float* pc = psm + r;              // column cc at pc[cc * n]
                    if (n <= 32) {
                        int cc = 0;
#pragma unroll 4
                        for (; cc + 1 < n; cc += 2) {
                            const float p0 = pc[cc * n], p1 = pc[(cc + 1) * n];
                            y0 = ffma2(make_float2(p0, p0), us[cc * 32 + lane], y0);
                            y1 = ffma2(make_float2(p1, p1), us[(cc + 1) * 32 + lane], y1);
                        }
                        if (cc < n) {
                            const float p0 = pc[cc * n];
                            y0 = ffma2(make_float2(p0, p0), us[cc * 32 + lane], y0);
                        }
                    } else {
#pragma unroll 4
                        for (int cc = 0; cc < n; ++cc) {
                            const float p0 = pc[cc * n];
                            y0 = ffma2(make_float2(p0, p0), us[cc * 32 + lane], y0);
                        }
                    }
                } else {
                    const float* pc = Pv + (size_t)r * Sp + k0;   // column cc at pc[cc * n * Sp]
                    const size_t cs = (size_t)n * Sp;
                    if (n <= 32) {
                        int cc = 0;
#pragma unroll 4
                        for (; cc + 1 < n; cc += 2) {
                            const float2 p0 = *reinterpret_cast<const float2*>(pc + cc * cs);
                            const float2 p1 = *reinterpret_cast<const float2*>(pc + (cc + 1) * cs);
                            y0 = ffma2(p0, us[cc * 32 + lane], y0);
                            y1 = ffma2(p1, us[(cc + 1) * 32 + lane], y1);
                        }
                        if (cc < n) y0 = ffma2(*reinterpret_cast<const float2*>(pc + cc * cs), us[cc * 32 + lane], y0);
                    } else {
#pragma unroll 4
                        for (int cc = 0; cc < n; ++cc)
                            y0 = ffma2(*reinterpret_cast<const float2*>(pc + cc * cs), us[cc * 32 + lane], y0);
                    }
                }
                const int g = v.gidx[j0 + r];
                const float2 z = *reinterpret_cast<const float2*>(v.Z + (size_t)g * Sp + k0);
                const float2 l = *reinterpret_cast<const float2*>(v.L + e);
                float2 bb;
                if (cd.nf & kVarB) bb = *reinterpret_cast<const float2*>(v.bv + (size_t)(cd.boff + r) * Sp + k0);
                else bb = make_float2(v.bs[cd.boff + r], v.bs[cd.boff + r]);
                const float xn0 = (y0.x + y1.x) + bb.x, xn1 = (y0.y + y1.y) + bb.y;
                const float ln0 = dual_of(l.x, rho, z.x, xn0), ln1 = dual_of(l.y, rho, z.y, xn1);
                const float wn0 = copy_term(xn0, ln0, inv_rho), wn1 = copy_term(xn1, ln1, inv_rho);
                if constexpr (check) {
                    const float2 xo = *reinterpret_cast<const float2*>(v.X + e);
                    sc_terms(f, z, make_float2(xn0, xn1), xo, make_float2(ln0, ln1));
                }
                if (a0) {
                    v.L[e] = ln0;
                    v.W[e] = wn0;
                    if (keepx) v.X[e] = xn0;
                }
                if (a1) {
                    v.L[e + 1] = ln1;
                    v.W[e + 1] = wn1;
                    if (keepx) v.X[e + 1] = xn1;
                }
            }
            if constexpr (check) sc_accumulate(acc, f);
            __syncthreads();                        // before the next component's staging
        }
        if constexpr (check) sc_partials<kScWarps>(acc, red, v.partials, v.nctas_s + blockIdx.x, Sp, pass);
    }
}

// One CTA per scenario: Eq. (termination) from the fixed-order sum of the
// per-CTA partials (each thread a fixed set of CTAs, then a fixed tree)
// after the body's iterations.
__global__ void __launch_bounds__(256) sc_fin_kernel(ScView v) {
    __shared__ double sh[5][256];
    const ScCtl* ctl = v.ctl;
    const int k = blockIdx.x;
    ScState& st = v.st[k];
    if (!st.active) return;
    const int iter = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    const int ndone = max(0, min(K, maxit - iter));
    const int it = iter + ndone;
    double a[5] = {0, 0, 0, 0, 0};
    if (ndone > 0)
        for (int b = threadIdx.x; b < v.nctas; b += blockDim.x)
            for (int m = 0; m < 5; ++m) a[m] += v.partials[((size_t)b * 5 + m) * v.Sp + k];
    for (int m = 0; m < 5; ++m) sh[m][threadIdx.x] = a[m];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int m = 0; m < 5; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    st.iter = it;
    if (ndone > 0) {
        const double pres = sqrt(sh[0][0]);
        const double dres = (double)ctl->rho * sqrt(sh[1][0]);
        const double ep = ctl->eps_rel * fmax(sqrt(sh[2][0]), sqrt(sh[3][0]));
        const double ed = ctl->eps_rel * sqrt(sh[4][0]);
        st.pres = pres; st.dres = dres; st.eps_prim = ep; st.eps_dual = ed;
        st.checks += 1;
        const bool ok_abs = pres <= ctl->eps_abs_prim && dres <= ctl->eps_abs_dual;
        const bool ok_rel = pres <= ep && dres <= ed;
        if (ok_rel && st.first_rel < 0) st.first_rel = it;
        const int cr = ctl->criterion;
        const bool conv = (cr == OPF_CRIT_ABS && ok_abs) || (cr == OPF_CRIT_REL && ok_rel) ||
                          (cr == OPF_CRIT_BOTH && ok_abs && ok_rel);
        if (!isfinite(pres) || !isfinite(dres)) { st.status = 3; st.active = 0; }
        else if (conv) { st.status = 1; st.active = 0; }
    }
    if (st.active && it >= maxit) { st.status = 2; st.active = 0; }
}

// Advance the sweep's iteration count, count the scenarios still running
// and set the while node's condition.
__global__ void __launch_bounds__(256) sc_cond_kernel(ScView v, int S, cudaGraphConditionalHandle h, int use_cond) {
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    int mine = 0;
    for (int k = threadIdx.x; k < S; k += blockDim.x) mine += v.st[k].active;
    atomicAdd(&running, mine);
    for (int w = threadIdx.x; w < v.Sp / 32; w += blockDim.x) {
        uint32_t m = 0;
        for (int b = 0; b < 32; ++b) m |= (uint32_t)(v.st[32 * w + b].active != 0) << b;
        v.amask[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ScCtl* ctl = v.ctl;
        ctl->iter += max(0, min(ctl->K, ctl->max_iter - ctl->iter));
        ctl->running = running;
        if (use_cond) cudaGraphSetConditional(h, running > 0 ? 1u : 0u);
    }
}

// c^T x per scenario in FP64, fixed order.
__global__ void sc_objective_kernel(ScView v, int S) {
    __shared__ double sh[256];
    const int k = blockIdx.x;
    double s = 0;
    for (int i = threadIdx.x; i < v.ng; i += 256) s += v.cost[i] * (double)v.Z[(size_t)i * v.Sp + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) v.st[k].objective = sh[0];
}

}  // namespace
}  // namespace opf

struct opf_scenarios {
    int device = -1;
    int S = 0, Sp = 0, nl = 0, ng = 0, ncomp = 0, nctas = 0, maxn = 0;
    std::vector<int32_t> canon_comp_ptr;
    char* buf = nullptr;             // one device allocation
    size_t bytes = 0;
    opf::ScView view{};
    opf::ScCtl* ctl_host = nullptr;  // pinned
    opf::ScState* st_host = nullptr; // pinned, S entries
    uint32_t* am_host = nullptr;     // pinned, Sp / 32 words
    bool cold = true;
    int graph_K = -1;
    int xupdate = 0;                 // OPF_SC_XUPDATE_*: small-component local update of plain iterations
    int graph_xupdate = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
};

namespace opf {

void scenarios_destroy(opf_scenarios* sc);

void scenarios_set_xupdate(opf_scenarios* sc, int kind) {
    if (kind != OPF_SC_XUPDATE_CUDA_CORES && kind != OPF_SC_XUPDATE_TENSOR)
        throw Error(OPF_ERR_INVALID_ARG, "bad x-update kind");
    sc->xupdate = kind;
}

namespace {

struct ScArena {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = (off + 255) & ~size_t(255);
        const size_t o = off;
        off += std::max<size_t>(1, count) * sizeof(T);
        return o;
    }
};

size_t sc_x_smem(int maxn) {
    const size_t m = (size_t)std::max(1, maxn);
    return m * 32 * sizeof(float2) + ((m * m * sizeof(float) + 15) & ~size_t(15));
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// The active-scenario bitmask from the host copy of the states.
void upload_mask(opf_scenarios* sc, cudaStream_t s) {
    for (int w = 0; w < sc->Sp / 32; ++w) {
        uint32_t m = 0;
        for (int b = 0; b < 32; ++b) m |= (uint32_t)(sc->st_host[32 * w + b].active != 0) << b;
        sc->am_host[w] = m;
    }
    SC_CUDA(cudaMemcpyAsync(sc->view.amask, sc->am_host, (size_t)(sc->Sp / 32) * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, s));
}

void build_graph(opf_scenarios* sc, int K) {
    if (sc->exec) cudaGraphExecDestroy(sc->exec);
    if (sc->graph) cudaGraphDestroy(sc->graph);
    sc->exec = nullptr;
    sc->graph = nullptr;
    SC_CUDA(cudaGraphCreate(&sc->graph, 0));
    cudaGraphConditionalHandle h;
    SC_CUDA(cudaGraphConditionalHandleCreate(&h, sc->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = cudaGraphNodeParams{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    SC_CUDA(cudaGraphAddNode(&node, sc->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    SC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    SC_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const ScView v = sc->view;
    const int zblocks = (int)(((size_t)sc->ng * 16 + 255) / 256);
    // the two local-update kernels depend only on the global update and
    // write disjoint locals: they run as parallel branches of the body
    cudaStream_t cs2;
    SC_CUDA(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
    cudaEvent_t ev_z, ev_x;
    SC_CUDA(cudaEventCreateWithFlags(&ev_z, cudaEventDisableTiming));
    SC_CUDA(cudaEventCreateWithFlags(&ev_x, cudaEventDisableTiming));
    for (int q = 0; q < K; ++q) {
        sc_z_kernel<<<zblocks, 256, 0, cs>>>(v, q);
        cudaEventRecord(ev_z, cs);
        cudaStreamWaitEvent(cs2, ev_z, 0);
        if (q == K - 1) sc_x_kernel<true><<<v.nctas - v.nctas_s, kScWarps * 32, sc_x_smem(sc->maxn), cs2>>>(v, q);
        else sc_x_kernel<false><<<v.nctas - v.nctas_s, kScWarps * 32, sc_x_smem(sc->maxn), cs2>>>(v, q);
        cudaEventRecord(ev_x, cs2);
        if (q == K - 1) sc_xs_kernel<true><<<v.nctas_s, kXsWarps * 32, 0, cs>>>(v, q);
        else if (sc->xupdate == OPF_SC_XUPDATE_TENSOR) sc_xs_kernel<false, true><<<v.nctas_s, kXsWarps * 32, 0, cs>>>(v, q);
        else sc_xs_kernel<false><<<v.nctas_s, kXsWarps * 32, 0, cs>>>(v, q);
        cudaStreamWaitEvent(cs, ev_x, 0);
    }
    sc_fin_kernel<<<sc->S, 256, 0, cs>>>(v);
    sc_cond_kernel<<<1, 256, 0, cs>>>(v, sc->S, h, 1);
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t captured;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    cudaStreamDestroy(cs2);
    cudaEventDestroy(ev_z);
    cudaEventDestroy(ev_x);
    if (le != cudaSuccess || ee != cudaSuccess)
        throw Error(OPF_ERR_CUDA, std::string("scenario graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ee));
    SC_CUDA(cudaGraphInstantiate(&sc->exec, sc->graph, 0));
    sc->graph_K = K;
    sc->graph_xupdate = sc->xupdate;
}

}  // namespace

opf_scenarios* scenarios_create(const opf_bus* buses, int nb, const opf_line* lines, int nl, const opf_gen* gens,
                                int ng, const opf_load* loads, int nd, int S) {
    if (S < 1 || S > 1024) throw Error(OPF_ERR_INVALID_ARG, "n_scenarios out of [1, 1024]");
    if (nd > 0 && !loads) throw Error(OPF_ERR_INVALID_ARG, "loads is NULL");
    // scenario 0 defines the structure; the others must differ only in a, b
    const Model M = build_model(buses, nb, lines, nl, gens, ng, loads, nd);
    for (int k = 1; k < S; ++k)
        for (int l = 0; l < nd; ++l) {
            const opf_load& a = loads[l];
            const opf_load& b = loads[(size_t)k * nd + l];
            if (a.bus != b.bus || a.phases != b.phases || a.conn != b.conn ||
                std::memcmp(a.alpha, b.alpha, sizeof a.alpha) != 0 || std::memcmp(a.beta, b.beta, sizeof a.beta) != 0)
                throw Error(OPF_ERR_INVALID_ARG, "scenario " + std::to_string(k) + " load " + std::to_string(l) +
                                                     ": only the load draw (a, b) may differ between scenarios");
        }
    std::vector<Operator> ops;
    ops.reserve(M.comps.size());
    for (const auto& c : M.comps) ops.push_back(make_operator(c));
    const Packed K = pack(M, ops, 0);      // for the copy order and the initial point
    const int ncomp = (int)M.comps.size();
    std::vector<int> load_comps;
    for (int s = 0; s < ncomp; ++s)
        if (M.comps[s].kind == COMP_LOAD) load_comps.push_back(s);
    // every scenario's load components
    std::vector<std::vector<Operator>> lops(S);
    std::vector<std::vector<std::vector<double>>> lA(S);
    lops[0].reserve(load_comps.size());
    for (int s : load_comps) {
        lops[0].push_back(ops[s]);
        lA[0].push_back(M.comps[s].A);
    }
    for (int k = 1; k < S; ++k) {
        const Model Mk = build_model(buses, nb, lines, nl, gens, ng, loads + (size_t)k * nd, nd);
        if (Mk.comps.size() != M.comps.size()) throw Error(OPF_ERR_INVALID_ARG, "scenario structure differs");
        for (int s : load_comps) {
            if (Mk.comps[s].gvars != M.comps[s].gvars) throw Error(OPF_ERR_INVALID_ARG, "scenario structure differs");
            lops[k].push_back(make_operator(Mk.comps[s]));
            lA[k].push_back(Mk.comps[s].A);
        }
    }
    opf_scenarios* sc = new opf_scenarios();
    try {
        sc->S = S;
        sc->Sp = (S + 63) / 64 * 64;
        sc->nl = K.nl;
        sc->ng = K.ng;
        sc->ncomp = ncomp;
        const int Sp = sc->Sp;
        // host arrays in canonical order
        std::vector<ScComp> comps(ncomp);
        std::vector<float> Ps, Pv, bs, bv;
        std::vector<int32_t> gidx(K.nl), cptr(ncomp + 1, 0);
        for (int s = 0; s < ncomp; ++s) cptr[s + 1] = cptr[s] + M.comps[s].n();
        sc->canon_comp_ptr = cptr;
        std::vector<int> lpos(ncomp, -1);
        for (size_t i = 0; i < load_comps.size(); ++i) lpos[load_comps[i]] = (int)i;
        for (int s = 0; s < ncomp; ++s) {
            const int n = M.comps[s].n();
            if (n > 64) throw Error(OPF_ERR_INVALID_ARG, "scenarios: a component has more than 64 local variables");
            ScComp& cd = comps[s];
            cd.loc0 = cptr[s];
            int flags = 0;
            for (int r = 0; r < n; ++r) gidx[cptr[s] + r] = M.comps[s].gvars[r];
            const int li = lpos[s];
            bool varP = false, varB = false;
            if (li >= 0)
                for (int k = 1; k < S; ++k) {
                    varP |= lA[k][li] != lA[0][li];
                    varB |= lops[k][li].bbar != lops[0][li].bbar;
                }
            if (varP) {
                flags |= kVarP;
                cd.poff = (int32_t)Pv.size();
                Pv.resize(Pv.size() + (size_t)n * n * Sp, 0.f);
                for (int k = 0; k < Sp; ++k) {
                    const Operator& o = lops[std::min(k, S - 1)][li];
                    for (int e = 0; e < n * n; ++e) Pv[cd.poff + (size_t)e * Sp + k] = (float)o.P[e];
                }
            } else if (n <= kSmallN) {
                // 8 x 8, column-major, zero past n (16-byte aligned block)
                cd.poff = (int32_t)Ps.size();
                Ps.resize(Ps.size() + kSmallN * kSmallN, 0.f);
                for (int c = 0; c < n; ++c)
                    for (int r = 0; r < n; ++r) Ps[cd.poff + c * kSmallN + r] = (float)ops[s].P[(size_t)c * n + r];
            } else {
                cd.poff = (int32_t)Ps.size();
                for (int e = 0; e < n * n; ++e) Ps.push_back((float)ops[s].P[e]);
                while (Ps.size() % 4) Ps.push_back(0.f);
            }
            if (varB) {
                flags |= kVarB;
                cd.boff = (int32_t)(bv.size() / Sp);
                bv.resize(bv.size() + (size_t)n * Sp, 0.f);
                for (int k = 0; k < Sp; ++k) {
                    const Operator& o = lops[std::min(k, S - 1)][li];
                    for (int r = 0; r < n; ++r) bv[((size_t)cd.boff + r) * Sp + k] = (float)o.bbar[r];
                }
            } else {
                cd.boff = (int32_t)bs.size();
                for (int r = 0; r < n; ++r) bs.push_back((float)ops[s].bbar[r]);
            }
            cd.nf = n | flags;
        }
        // device order: components of at most kSmallN locals first
        std::vector<ScComp> dcomps;
        dcomps.reserve(ncomp);
        for (int s = 0; s < ncomp; ++s)
            if ((comps[s].nf & 0xFFFF) <= kSmallN) dcomps.push_back(comps[s]);
        const int nsmall = (int)dcomps.size();
        int maxn_large = 1;
        for (int s = 0; s < ncomp; ++s)
            if ((comps[s].nf & 0xFFFF) > kSmallN) {
                dcomps.push_back(comps[s]);
                maxn_large = std::max(maxn_large, comps[s].nf & 0xFFFF);
            }
        // largest first: CTA b takes components b, b + G, ... (balanced loads)
        std::stable_sort(dcomps.begin() + nsmall, dcomps.end(), [](const ScComp& x, const ScComp& y) {
            const int nx = x.nf & 0xFFFF, ny = y.nf & 0xFFFF;
            const int cx = nx * nx * ((x.nf & kVarP) ? 8 : 1), cy = ny * ny * ((y.nf & kVarP) ? 8 : 1);
            return cx > cy;
        });
        comps.swap(dcomps);
        sc->maxn = maxn_large;
        // copies of each global in the CSR order of the single-instance engines
        std::vector<int32_t> gptr = K.gptr, gcol(K.gcol.size());
        for (size_t q = 0; q < K.gcol.size(); ++q) gcol[q] = K.canon_of_dev[K.gcol[q]];
        std::vector<float> xl0(K.nl), invk(K.ng), cik(K.ng), lo(K.ng), hi(K.ng);
        for (int j = 0; j < K.nl; ++j) xl0[j] = (float)K.xl0[K.dev_of_canon[j]];
        for (int i = 0; i < K.ng; ++i) {
            invk[i] = (float)K.invk[i];
            cik[i] = (float)K.cik[i];
            lo[i] = (float)M.lo[i];
            hi[i] = (float)M.hi[i];
        }
        // device arena
        int dev = 0, sms = 0;
        SC_CUDA(cudaGetDevice(&dev));
        SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        sc->device = dev;
        const int nctas_s = 4 * sms, nctas_l = 8 * sms;   // one wave each (plain sweeps)
        sc->nctas = nctas_s + nctas_l;
        ScArena a;
        const size_t o_comps = a.take<ScComp>(ncomp), o_Ps = a.take<float>(Ps.size()), o_Pv = a.take<float>(Pv.size());
        const size_t o_bs = a.take<float>(bs.size()), o_bv = a.take<float>(bv.size());
        const size_t o_gidx = a.take<int32_t>(K.nl), o_gptr = a.take<int32_t>(K.ng + 1), o_gcol = a.take<int32_t>(K.nl);
        const size_t o_invk = a.take<float>(K.ng), o_cik = a.take<float>(K.ng), o_lo = a.take<float>(K.ng);
        const size_t o_hi = a.take<float>(K.ng), o_cost = a.take<double>(K.ng), o_xl0 = a.take<float>(K.nl);
        const size_t per = (size_t)K.nl * Sp;
        const size_t o_W = a.take<float>(per), o_L = a.take<float>(per), o_X = a.take<float>(per);
        const size_t o_Z = a.take<float>((size_t)K.ng * Sp);
        const size_t o_part = a.take<double>((size_t)sc->nctas * 5 * Sp);
        const size_t o_st = a.take<ScState>(Sp), o_ctl = a.take<ScCtl>(1), o_am = a.take<uint32_t>(Sp / 32);
        sc->bytes = (a.off + 255) & ~size_t(255);
        SC_CUDA(cudaMalloc((void**)&sc->buf, sc->bytes));
        char* d = sc->buf;
        auto up = [&](size_t off, const void* src, size_t n) {
            if (n) SC_CUDA(cudaMemcpy(d + off, src, n, cudaMemcpyHostToDevice));
        };
        up(o_comps, comps.data(), comps.size() * sizeof(ScComp));
        up(o_Ps, Ps.data(), Ps.size() * 4); up(o_Pv, Pv.data(), Pv.size() * 4);
        up(o_bs, bs.data(), bs.size() * 4); up(o_bv, bv.data(), bv.size() * 4);
        up(o_gidx, gidx.data(), gidx.size() * 4); up(o_gptr, gptr.data(), gptr.size() * 4);
        up(o_gcol, gcol.data(), gcol.size() * 4);
        up(o_invk, invk.data(), invk.size() * 4); up(o_cik, cik.data(), cik.size() * 4);
        up(o_lo, lo.data(), lo.size() * 4); up(o_hi, hi.data(), hi.size() * 4);
        up(o_cost, M.c.data(), M.c.size() * 8); up(o_xl0, xl0.data(), xl0.size() * 4);
        SC_CUDA(cudaMemset(d + o_st, 0, (size_t)Sp * sizeof(ScState)));
        SC_CUDA(cudaMemset(d + o_ctl, 0, sizeof(ScCtl)));
        ScView& v = sc->view;
        v.comps = (const ScComp*)(d + o_comps);
        v.Ps = (const float*)(d + o_Ps); v.Pv = (const float*)(d + o_Pv);
        v.bs = (const float*)(d + o_bs); v.bv = (const float*)(d + o_bv);
        v.gidx = (const int32_t*)(d + o_gidx); v.gptr = (const int32_t*)(d + o_gptr); v.gcol = (const int32_t*)(d + o_gcol);
        v.invk = (const float*)(d + o_invk); v.cik = (const float*)(d + o_cik);
        v.lo = (const float*)(d + o_lo); v.hi = (const float*)(d + o_hi);
        v.cost = (const double*)(d + o_cost); v.xl0 = (const float*)(d + o_xl0);
        v.W = (float*)(d + o_W); v.L = (float*)(d + o_L); v.X = (float*)(d + o_X); v.Z = (float*)(d + o_Z);
        v.partials = (double*)(d + o_part);
        v.st = (ScState*)(d + o_st);
        v.amask = (uint32_t*)(d + o_am);
        v.ctl = (ScCtl*)(d + o_ctl);
        v.ncomp = ncomp; v.nl = K.nl; v.ng = K.ng; v.Sp = Sp; v.nctas = sc->nctas; v.maxn = sc->maxn;
        v.nsmall = nsmall; v.nctas_s = nctas_s;
        const size_t xsm = sc_x_smem(sc->maxn);
        if (xsm > 200 * 1024) throw Error(OPF_ERR_INVALID_ARG, "a component is too large for the scenario engine");
        SC_CUDA(cudaFuncSetAttribute(sc_x_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
        SC_CUDA(cudaFuncSetAttribute(sc_x_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
        SC_CUDA(cudaMallocHost((void**)&sc->ctl_host, sizeof(ScCtl)));
        SC_CUDA(cudaMallocHost((void**)&sc->st_host, (size_t)Sp * sizeof(ScState)));
        SC_CUDA(cudaMallocHost((void**)&sc->am_host, (size_t)(Sp / 32) * sizeof(uint32_t)));
        std::memset(sc->ctl_host, 0, sizeof(ScCtl));
        std::memset(sc->st_host, 0, (size_t)Sp * sizeof(ScState));
        SC_CUDA(cudaEventCreateWithFlags(&sc->done, cudaEventDisableTiming));
    } catch (...) {
        scenarios_destroy(sc);
        throw;
    }
    return sc;
}

void scenarios_destroy(opf_scenarios* sc) {
    if (!sc) return;
    DevGuard g(sc->device);
    if (sc->exec) cudaGraphExecDestroy(sc->exec);
    if (sc->graph) cudaGraphDestroy(sc->graph);
    if (sc->done) cudaEventDestroy(sc->done);
    if (sc->buf) cudaFree(sc->buf);
    if (sc->ctl_host) cudaFreeHost(sc->ctl_host);
    if (sc->st_host) cudaFreeHost(sc->st_host);
    if (sc->am_host) cudaFreeHost(sc->am_host);
    delete sc;
}

void scenarios_solve(opf_scenarios* sc, const opf_params& prm, cudaStream_t s, opf_info* infos) {
    DevGuard g(sc->device);
    const auto t0 = std::chrono::steady_clock::now();
    const int S = sc->S, Sp = sc->Sp;
    ScCtl c = *sc->ctl_host;
    if (!prm.warm_start || sc->cold) c.iter = 0;
    c.rho = (float)prm.rho;
    c.inv_rho = (float)(1.0 / prm.rho);
    c.eps_abs_prim = prm.eps_abs_prim; c.eps_abs_dual = prm.eps_abs_dual; c.eps_rel = prm.eps_rel;
    c.criterion = prm.criterion; c.K = prm.check_every;
    const long long mi = (long long)c.iter + prm.max_iter;
    c.max_iter = (int32_t)std::min<long long>(mi, INT32_MAX);
    c.running = S;
    *sc->ctl_host = c;
    for (int k = 0; k < Sp; ++k) {
        ScState& st = sc->st_host[k];
        const bool keep = prm.warm_start && !sc->cold;
        if (!keep) {
            st = ScState{};
            st.first_rel = -1;
            st.pres = st.dres = st.eps_prim = st.eps_dual = NAN;
        }
        st.active = k < S ? 1 : 0;
        st.status = 0;
    }
    SC_CUDA(cudaMemcpyAsync(sc->view.ctl, sc->ctl_host, sizeof(ScCtl), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(sc->view.st, sc->st_host, (size_t)Sp * sizeof(ScState), cudaMemcpyHostToDevice, s));
    upload_mask(sc, s);
    if (!prm.warm_start || sc->cold) {
        sc_init_kernel<<<4 * 148, 256, 0, s>>>(sc->view);
        SC_CUDA(cudaGetLastError());
        sc->cold = false;
    }
    if (prm.max_iter > 0) {
        if (sc->graph_K != prm.check_every || sc->graph_xupdate != sc->xupdate) build_graph(sc, prm.check_every);
        SC_CUDA(cudaGraphLaunch(sc->exec, s));
    }
    sc_objective_kernel<<<S, 256, 0, s>>>(sc->view, S);
    SC_CUDA(cudaGetLastError());
    SC_CUDA(cudaMemcpyAsync(sc->ctl_host, sc->view.ctl, sizeof(ScCtl), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaMemcpyAsync(sc->st_host, sc->view.st, (size_t)Sp * sizeof(ScState), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (infos)
        for (int k = 0; k < S; ++k) {
            const ScState& st = sc->st_host[k];
            opf_info& inf = infos[k];
            std::memset(&inf, 0, sizeof inf);
            inf.status = st.status == 1 ? OPF_OK
                         : st.status == 3 ? OPF_ERR_NUMERIC
                         : (prm.criterion == OPF_CRIT_NEVER ? OPF_OK : OPF_NOT_CONVERGED);
            inf.iters = st.iter;
            inf.first_rel_iter = st.first_rel;
            inf.pres = st.pres; inf.dres = st.dres; inf.eps_prim = st.eps_prim; inf.eps_dual = st.eps_dual;
            inf.objective = st.objective;
            inf.seconds = sec;
            inf.rho = prm.rho;
        }
}

// Average device time of each kernel of one iteration (events around `reps`
// back-to-back launches of that kernel outside the graph): us[0] global
// update, us[1] small-component local update, us[2] large-component local
// update, us[3] the same two local updates on a check iteration, us[4] the
// per-scenario check.  Leaves the scenarios at a cold start.
void scenarios_profile(opf_scenarios* sc, const opf_params& prm, int reps, cudaStream_t s, double* us) {
    DevGuard g(sc->device);
    ScCtl c{};
    c.rho = (float)prm.rho;
    c.inv_rho = (float)(1.0 / prm.rho);
    c.eps_abs_prim = prm.eps_abs_prim; c.eps_abs_dual = prm.eps_abs_dual; c.eps_rel = prm.eps_rel;
    c.criterion = OPF_CRIT_NEVER; c.K = 1 << 20; c.max_iter = 1 << 30; c.iter = 0; c.running = sc->S;
    *sc->ctl_host = c;
    for (int k = 0; k < sc->Sp; ++k) {
        sc->st_host[k] = ScState{};
        sc->st_host[k].active = k < sc->S;
    }
    SC_CUDA(cudaMemcpyAsync(sc->view.ctl, sc->ctl_host, sizeof(ScCtl), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(sc->view.st, sc->st_host, (size_t)sc->Sp * sizeof(ScState), cudaMemcpyHostToDevice, s));
    upload_mask(sc, s);
    const ScView v = sc->view;
    sc_init_kernel<<<4 * 148, 256, 0, s>>>(v);
    cudaEvent_t e0, e1;
    SC_CUDA(cudaEventCreate(&e0));
    SC_CUDA(cudaEventCreate(&e1));
    const int zblocks = (int)(((size_t)sc->ng * 16 + 255) / 256);
    const size_t xsm = sc_x_smem(sc->maxn);
    auto timeit = [&](auto&& launch) {
        launch();
        SC_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) launch();
        SC_CUDA(cudaEventRecord(e1, s));
        SC_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        SC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return 1e3 * ms / reps;
    };
    // q = 0 with K = 2^20: a plain iteration; q = K - 1: a check iteration
    us[0] = timeit([&] { sc_z_kernel<<<zblocks, 256, 0, s>>>(v, 0); });
    us[1] = timeit([&] {
        if (sc->xupdate == OPF_SC_XUPDATE_TENSOR) sc_xs_kernel<false, true><<<v.nctas_s, kXsWarps * 32, 0, s>>>(v, 0);
        else sc_xs_kernel<false><<<v.nctas_s, kXsWarps * 32, 0, s>>>(v, 0);
    });
    us[2] = timeit([&] { sc_x_kernel<false><<<v.nctas - v.nctas_s, kScWarps * 32, xsm, s>>>(v, 0); });
    us[3] = timeit([&] {
        sc_xs_kernel<true><<<v.nctas_s, kXsWarps * 32, 0, s>>>(v, (1 << 20) - 1);
        sc_x_kernel<true><<<v.nctas - v.nctas_s, kScWarps * 32, xsm, s>>>(v, (1 << 20) - 1);
    });
    us[4] = timeit([&] {
        sc_fin_kernel<<<sc->S, 256, 0, s>>>(v);
        sc_cond_kernel<<<1, 256, 0, s>>>(v, sc->S, cudaGraphConditionalHandle{}, 0);
    });
    SC_CUDA(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sc->cold = true;
}

void scenarios_get_state(const opf_scenarios* sc, int k, double* xg, double* xl, double* lam, cudaStream_t s) {
    if (k < 0 || k >= sc->S) throw Error(OPF_ERR_INVALID_ARG, "scenario index out of range");
    DevGuard g(sc->device);
    const int Sp = sc->Sp;
    std::vector<float> h;
    auto col = [&](const float* dptr, size_t rows, double* out) {
        if (!out) return;
        h.resize(rows * Sp);
        SC_CUDA(cudaMemcpyAsync(h.data(), dptr, h.size() * 4, cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        for (size_t r = 0; r < rows; ++r) out[r] = h[r * Sp + k];
    };
    col(sc->view.Z, sc->ng, xg);
    col(sc->view.X, sc->nl, xl);
    col(sc->view.L, sc->nl, lam);
}

void scenarios_dims(const opf_scenarios* sc, int32_t* n_global, int32_t* n_local, int64_t* device_bytes) {
    if (n_global) *n_global = sc->ng;
    if (n_local) *n_local = sc->nl;
    if (device_bytes) *device_bytes = (int64_t)sc->bytes;
}

}  // namespace opf
