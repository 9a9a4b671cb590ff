// sm_103a kernels and the solve engines of the componentwise ADMM.
//
// Algorithm 1, one iteration:
//   global update, Eq. (global_sparse): for every global i the copies'
//     (x_j - lambda_j / rho) are summed over its CSR list in a fixed order,
//     scaled by 1/k_i, shifted by -c_i/(rho k_i), clipped to [lo_i, hi_i].
//   local update, Eq. (closed_2), fused with the dual update, Eq. (ADMM-3),
//     and the residual sums of Eq. (termination): per component
//     u = B_s x + lambda_s / rho, x_s = P_s u + bbar_s (P_s = -Abar_s),
//     lambda_s += rho (B_s x - x_s).  One warp per tile of components (see
//     pack.cpp); the tile's operator columns are stored in lane-interleaved
//     groups of four, so a lane reads four columns with one 16-byte load;
//     u is broadcast by warp shuffles (graph engine, FP64) or read from
//     shifted shared-memory rows (FP32 persistent kernel).  On check
//     iterations each CTA writes five FP64 partial sums: ||Bx - z||^2,
//     ||z - z_prev||^2, ||Bx||^2, ||z||^2, ||lambda||^2; they are summed in a
//     fixed order (deterministic).
//
// Engines:
//   GRAPH       z_kernel + x_kernel per iteration and finalize_kernel every
//               K iterations, captured once as the body of a device-side
//               while node: one graph launch runs the whole solve.
//   HOSTLOOP    the same kernels, stop test read back by the host.
//   PERSISTENT  one cooperative launch for the whole solve.  CTA b owns a
//               chunk of components; each iteration it recomputes the global
//               update for the globals its chunk copies (its halo) into
//               shared memory from ping-pong x_s / lambda buffers, then runs
//               the local and dual updates.  CTAs synchronize only with their
//               neighbours (chunks sharing a global) through per-CTA
//               iteration flags (release / acquire); every K iterations a
//               ticket counter elects the last CTA to finalize the residuals.
//               Every wait is bounded in time: on expiry the CTA records
//               where, sets OPF_ERR_TIMEOUT and all CTAs leave.
//               The shared-memory variant exchanges boundary values without
//               flags or fences: a CTA publishes, for each of its copies that
//               other chunks read, the term x_j - lambda_j / rho together
//               with the iteration number in one 64-bit word (two for FP64:
//               each half of the double with the tag) into a two-slot
//               mailbox; a reader polls exactly the words it needs until the
//               tags match.  A single-copy-atomic word carries its own
//               validity, so no release / acquire ordering is involved.  Its
//               checks do not wait for the decision: each leaves a snapshot
//               of the state, and a stop raises a halt flag that every CTA
//               sees at its next check or while polling a neighbour.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>

#include "arith.cuh"
#include "problem.hpp"

namespace opf {

#define OPF_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw Error(e_ == cudaErrorMemoryAllocation ? OPF_ERR_OOM : OPF_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

constexpr int kXWarps = kTileWarps;  // warps per CTA of x_kernel / persistent kernels
constexpr int kZThreads = 256;
constexpr int kFinThreads = 256;
constexpr int kMaxBigN = 256;

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tagged mailbox of boundary terms: slot s, device local j.  A word holds
// the value bits in its low half and the tag (iteration + 1, never 0 after
// the launch clears the mailbox) in its high half; an FP64 value takes two
// words, one per 32-bit half, each with the tag.
template <typename T>
struct Mail;
template <>
struct Mail<float> {
    static constexpr int kWords = 1;
    static __device__ __forceinline__ void fetch(const unsigned long long* mb, int nl, int slot, int j,
                                                 unsigned long long* r) {
        r[0] = ld_relaxed64(mb + (size_t)slot * nl + j);
    }
    static __device__ __forceinline__ bool decode(const unsigned long long* r, unsigned tag, float& w) {
        w = __uint_as_float((unsigned)r[0]);
        return (unsigned)(r[0] >> 32) == tag;
    }
    static __device__ __forceinline__ void put(unsigned long long* mb, int nl, int slot, int j, float w, unsigned tag) {
        st_relaxed64(mb + (size_t)slot * nl + j, ((unsigned long long)tag << 32) | __float_as_uint(w));
    }
    static __device__ __forceinline__ bool get(const unsigned long long* mb, int nl, int slot, int j, unsigned tag,
                                               float& w) {
        const unsigned long long v = ld_relaxed64(mb + (size_t)slot * nl + j);
        w = __uint_as_float((unsigned)v);
        return (unsigned)(v >> 32) == tag;
    }
};
template <>
struct Mail<double> {
    static constexpr int kWords = 2;
    static __device__ __forceinline__ void fetch(const unsigned long long* mb, int nl, int slot, int j,
                                                 unsigned long long* r) {
        const unsigned long long* q = mb + ((size_t)slot * nl + j) * 2;
        r[0] = ld_relaxed64(q);
        r[1] = ld_relaxed64(q + 1);
    }
    static __device__ __forceinline__ bool decode(const unsigned long long* r, unsigned tag, double& w) {
        w = __longlong_as_double((long long)(((r[1] & 0xFFFFFFFFull) << 32) | (r[0] & 0xFFFFFFFFull)));
        return (unsigned)(r[0] >> 32) == tag && (unsigned)(r[1] >> 32) == tag;
    }
    static __device__ __forceinline__ void put(unsigned long long* mb, int nl, int slot, int j, double w, unsigned tag) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(w);
        unsigned long long* q = mb + ((size_t)slot * nl + j) * 2;
        const unsigned long long t = (unsigned long long)tag << 32;
        st_relaxed64(q, t | (b & 0xFFFFFFFFull));
        st_relaxed64(q + 1, t | (b >> 32));
    }
    static __device__ __forceinline__ bool get(const unsigned long long* mb, int nl, int slot, int j, unsigned tag,
                                               double& w) {
        const unsigned long long* q = mb + ((size_t)slot * nl + j) * 2;
        const unsigned long long a = ld_relaxed64(q), c = ld_relaxed64(q + 1);
        w = __longlong_as_double((long long)(((c & 0xFFFFFFFFull) << 32) | (a & 0xFFFFFFFFull)));
        return (unsigned)(a >> 32) == tag && (unsigned)(c >> 32) == tag;
    }
};

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded poll of one mailbox entry until its tag matches; false once the
// deadline passed (the CTA then raises the abort flag and records `where`)
// or another CTA aborted.
template <typename T>
__device__ __forceinline__ bool mail_poll(const unsigned long long* mb, int nl, int slot, int j, unsigned tag, T& w,
                                          Ctl* ctl, unsigned long long tmo, int where) {
    unsigned spins = 0;
    unsigned long long deadline = 0;
    while (!Mail<T>::get(mb, nl, slot, j, tag, w)) {
        if ((++spins & 31u) == 0) {
            if (ld_acquire(&ctl->abort) || ld_acquire(&ctl->halt)) return false;
            const unsigned long long tn = now_ns();
            if (deadline == 0) {
                deadline = tn + tmo;
            } else if (tn > deadline) {
                if (atomicCAS(&ctl->abort, 0, 1) == 0) { ctl->status = CTL_TIMEOUT; ctl->timeout_where = where; }
                return false;
            }
        }
    }
    return true;
}
__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }


// Operator columns 4q .. 4q+3 of one lane (quad layout of pack.cpp: column c
// of lane r at ((c / 4) * L + r) * 4 + c % 4): one 16-byte load for FP32,
// two for FP64.
__device__ __forceinline__ void load_quad(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load_quad(const double* p, double (&o)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// y0 = fma(a0, b0, y0), y1 = fma(a1, b1, y1): one packed FP32 instruction on
// sm_100+ (two independent round-to-nearest fmas, so the same bits as two
// scalar fmas); two fmas for FP64.
__device__ __forceinline__ void fma_pair(float& y0, float& y1, float a0, float a1, float b0, float b1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(y0, y1));
    y0 = r.x;
    y1 = r.y;
}
__device__ __forceinline__ void fma_pair(double& y0, double& y1, double a0, double a1, double b0, double b1) {
    y0 = fma(a0, b0, y0);
    y1 = fma(a1, b1, y1);
}

// Small-tile GEMV of one lane, y = sum_c P[c][r] u_(base + c), with u
// broadcast by warp shuffles: even columns accumulate into y0, odd ones into
// y1 (the order of every engine).  Columns past the lane's component are
// zero in the packed operator, so they add exact zeros and need no test.
// Inactive lanes (act false) read lane 0's operator and discard y.
template <typename T>
__device__ __forceinline__ T tile_gemv(const T* Pt, int L, int lane, int nmax, int base, T u, bool act) {
    T y0 = 0, y1 = 0;
    const int r = act ? lane : 0;
    const int nq = (nmax + 3) >> 2;
    for (int q = 0; q < nq; ++q) {
        T p[4];
        load_quad(Pt + (q * L + r) * 4, p);
        const int c = base + 4 * q;
        const T u0 = __shfl_sync(0xffffffffu, u, c & 31), u1 = __shfl_sync(0xffffffffu, u, (c + 1) & 31);
        const T u2 = __shfl_sync(0xffffffffu, u, (c + 2) & 31), u3 = __shfl_sync(0xffffffffu, u, (c + 3) & 31);
        fma_pair(y0, y1, p[0], p[1], u0, u1);
        fma_pair(y0, y1, p[2], p[3], u2, u3);
    }
    return y0 + y1;
}

// The same GEMV with u from shared memory: ub is the lane's 16-byte-aligned
// view of the warp's u values, ub[4q + j] = u_(base + 4q + j) (zero past the
// tile), so each group of four columns is two vector loads and two packed
// fmas.  Same accumulation order as tile_gemv, hence the same bits.
constexpr int kUrow = 68;     // shifted u row: 64 entries + 4 of padding (bank spread)
template <typename T>
__device__ __forceinline__ T tile_gemv_sh(const T* Pt, int L, int r, int nq, const T* ub) {
    T y0 = 0, y1 = 0;
#pragma unroll 4
    for (int q = 0; q < nq; ++q) {
        T p[4], w[4];
        load_quad(Pt + (q * L + r) * 4, p);
        load_quad(ub + 4 * q, w);
        fma_pair(y0, y1, p[0], p[1], w[0], w[1]);
        fma_pair(y0, y1, p[2], p[3], w[2], w[3]);
    }
    return y0 + y1;
}
template <>
__device__ __forceinline__ float tile_gemv_sh<float>(const float* Pt, int L, int r, int nq, const float* ub) {
    float2 y = make_float2(0.f, 0.f);
    const float4* P4 = reinterpret_cast<const float4*>(Pt) + r;
    const float4* U4 = reinterpret_cast<const float4*>(ub);
#pragma unroll 4
    for (int q = 0; q < nq; ++q) {
        const float4 p = P4[q * L], u = U4[q];
        y = __ffma2_rn(make_float2(p.x, p.y), make_float2(u.x, u.y), y);
        y = __ffma2_rn(make_float2(p.z, p.w), make_float2(u.z, u.w), y);
    }
    return y.x + y.y;
}

// Eq. (global_sparse) from a halo entry's copy sum and its constants
// c = {lo, hi, 1/k, c/k} (one 16-byte load for FP32).
__device__ __forceinline__ float halo_global(float sum, const float* c, float inv_rho) {
    const float4 q = *reinterpret_cast<const float4*>(c);
    return global_from_sum(sum, q.z, q.w, inv_rho, q.x, q.y);
}
__device__ __forceinline__ double halo_global(double sum, const double* c, double inv_rho) {
    const double2 a = reinterpret_cast<const double2*>(c)[0], b = reinterpret_cast<const double2*>(c)[1];
    return global_from_sum(sum, b.x, b.y, inv_rho, a.x, a.y);
}

// Eq. (global_sparse) for global g from the copies in (xr, lr).
template <typename T, bool CG>
__device__ __forceinline__ T global_value(const View<T>& v, int g, const T* xr, const T* lr, T inv_rho) {
    const int b = v.gptr[g], e = v.gptr[g + 1];
    T s = 0;
    for (int j = b; j < e; ++j) {
        const int l = v.gcol[j];
        if (CG) s += copy_term(ldcg(xr + l), ldcg(lr + l), inv_rho);
        else s += copy_term(xr[l], lr[l], inv_rho);
    }
    return global_from_sum(s, v.invk[g], v.cik[g], inv_rho, v.lo[g], v.hi[g]);
}

// Local update + dual update of one tile (Eq. closed_2, Eq. ADMM-3).
// getv(j, meta) returns the gathered global value (B_s x)_j for local j.
// dzout (optional, check iterations only): x_s - x_s(prev) per local in
// FP64, for the textbook residual form.
template <typename T, typename GETV>
__device__ __forceinline__ void tile_update(const View<T>& v, const Tile tl, int lane, T rho, T inv_rho,
                                            const T* xr, const T* lr, T* xw, T* lw, bool want, double* acc,
                                            T* us, GETV getv, double* dzout = nullptr) {
    if (!tl.big) {
        const int L = tl.L, nmax = tl.nmax;
        const bool act = lane < L;
        const int j = tl.loc0 + lane;
        int base = 0;
        T vv = 0, lo = 0, xo = 0, u = 0;
        if (act) {
            const int m = v.meta[j];
            base = (m >> 24) & 0x1F;
            vv = getv(j, m);
            lo = ldcg(lr + j);
            xo = ldcg(xr + j);
            u = u_of(vv, lo, inv_rho);
        }
        const T y = tile_gemv(v.P + tl.mat0, L, lane, nmax, base, u, act);
        if (act) {
            const T xn = y + v.bbar[j];
            const T ln = dual_of(lo, rho, vv, xn);
            xw[j] = xn;
            lw[j] = ln;
            if (want) {
                const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                acc[0] += pr * pr; acc[1] += dz * dz;
                acc[2] += (double)vv * (double)vv; acc[3] += (double)xn * (double)xn; acc[4] += (double)ln * (double)ln;
                if (dzout) dzout[j] = dz;
            }
        }
    } else {
        const int n = tl.nmax;
        for (int r = lane; r < n; r += 32) {
            const int j = tl.loc0 + r;
            us[r] = u_of(getv(j, v.meta[j]), ldcg(lr + j), inv_rho);
        }
        __syncwarp();
        const T* Pm = v.P + tl.mat0;
        for (int r = lane; r < n; r += 32) {
            T y = 0;
            for (int c = 0; c < n; ++c) y = fma(Pm[c * n + r], us[c], y);
            const int j = tl.loc0 + r;
            const T vv = getv(j, v.meta[j]);
            const T lo = ldcg(lr + j), xo = ldcg(xr + j);
            const T xn = y + v.bbar[j];
            const T ln = dual_of(lo, rho, vv, xn);
            xw[j] = xn;
            lw[j] = ln;
            if (want) {
                const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                acc[0] += pr * pr; acc[1] += dz * dz;
                acc[2] += (double)vv * (double)vv; acc[3] += (double)xn * (double)xn; acc[4] += (double)ln * (double)ln;
                if (dzout) dzout[j] = dz;
            }
        }
        __syncwarp();
    }
}

// CTA-wide fixed-order reduction of acc[5]; threads 0..4 write out[0..4].
__device__ __forceinline__ void cta_partials(double* acc, double (*red)[5], double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < 5; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0)
        for (int k = 0; k < 5; ++k) red[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0;
        for (int w = 0; w < kXWarps; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Fixed-order sum of nparts partial records by one CTA using only the
// per-warp scratch red[][5]: thread-strided sums, a fixed shuffle tree per
// warp, then warps in order.  Thread 0 gets the five sums in tot.
__device__ __forceinline__ void sum_partials_small(const double* partials, int nparts, double (*red)[5], double* tot) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int k = 0; k < 5; ++k) s[k] += __ldcg(partials + (size_t)b * 8 + k);
    for (int k = 0; k < 5; ++k) s[k] = warp_sum(s[k]);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 5; ++k) red[warp][k] = s[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) {
            double a = 0;
            for (int w = 0; w < kXWarps; ++w) a += red[w][k];
            tot[k] = a;
        }
}

// Eq. (termination) from the five sums after `it` iterations; returns stop.
__device__ __forceinline__ int decide(Ctl* ctl, const double* s, int it) {
    const double pres = sqrt(s[0]);
    const double dres = ctl->rho * sqrt(s[1]);
    const double ep = ctl->eps_rel * fmax(sqrt(s[2]), sqrt(s[3]));
    const double ed = ctl->eps_rel * sqrt(s[4]);
    ctl->pres = pres; ctl->dres = dres; ctl->eps_prim = ep; ctl->eps_dual = ed;
    ctl->checks += 1;
    const bool ok_abs = pres <= ctl->eps_abs_prim && dres <= ctl->eps_abs_dual;
    const bool ok_rel = pres <= ep && dres <= ed;
    if (ok_rel && ctl->first_rel < 0) ctl->first_rel = it;
    const int cr = ctl->criterion;
    const bool conv = (cr == OPF_CRIT_ABS && ok_abs) || (cr == OPF_CRIT_REL && ok_rel) ||
                      (cr == OPF_CRIT_BOTH && ok_abs && ok_rel);
    if (!isfinite(pres) || !isfinite(dres)) {
        ctl->status = CTL_NUMERIC;
        return 1;
    }
    if (conv) {
        ctl->status = CTL_CONVERGED;
        return 1;
    }
    if (it >= ctl->max_iter) {
        ctl->status = CTL_MAXITER;
        return 1;
    }
    if (ctl->adaptive) {                // residual balancing
        double rho = ctl->rho;
        if (pres > ctl->rb_mu * dres) rho *= ctl->rb_tau;
        else if (dres > ctl->rb_mu * pres) rho /= ctl->rb_tau;
        if (rho != ctl->rho) {
            ctl->rho = rho;
            ctl->inv_rho = 1.0 / rho;
            ctl->rho_changes += 1;
        }
    }
    return 0;
}

// ----------------------------------------------------- graph / hostloop
// Globals per thread of the graph engines' global update, and its CTA
// count for an instance of ng globals.
constexpr int kZPer = 2;
inline int zb_blocks(int ng) { return (ng + kZThreads * kZPer - 1) / (kZThreads * kZPer); }

// Eq. (global_sparse) for kZPer globals g[k] of one instance (g[k] < 0:
// none): the copy lists are read four entries at a time and all their x,
// lambda loads are in flight together; each sum still adds the copies in
// list order, so the result is that of global_value.
template <typename T>
__device__ __forceinline__ void global_values_batched(const View<T>& v, const int (&g)[kZPer], T inv_rho,
                                                      T (&out)[kZPer]) {
    int b[kZPer], e[kZPer];
    T s[kZPer], lo[kZPer], hi[kZPer], ik[kZPer], ck[kZPer];
#pragma unroll
    for (int k = 0; k < kZPer; ++k) {
        b[k] = g[k] >= 0 ? v.gptr[g[k]] : 0;
        e[k] = g[k] >= 0 ? v.gptr[g[k] + 1] : 0;
        lo[k] = g[k] >= 0 ? v.lo[g[k]] : (T)0;
        hi[k] = g[k] >= 0 ? v.hi[g[k]] : (T)0;
        ik[k] = g[k] >= 0 ? v.invk[g[k]] : (T)0;
        ck[k] = g[k] >= 0 ? v.cik[g[k]] : (T)0;
        s[k] = 0;
    }
    const T* xr = v.xl;
    const T* lr = v.lam;
    for (int j0 = 0;; j0 += 4) {
        bool more = false;
        int l[kZPer][4];
#pragma unroll
        for (int k = 0; k < kZPer; ++k)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool in = b[k] + j0 + r < e[k];
                l[k][r] = in ? v.gcol[b[k] + j0 + r] : -1;
                more |= in;
            }
        if (!more) break;
        T xv[kZPer][4], lv[kZPer][4];
#pragma unroll
        for (int k = 0; k < kZPer; ++k)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                xv[k][r] = l[k][r] >= 0 ? xr[l[k][r]] : (T)0;
                lv[k][r] = l[k][r] >= 0 ? lr[l[k][r]] : (T)0;
            }
#pragma unroll
        for (int k = 0; k < kZPer; ++k)
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (l[k][r] >= 0) s[k] += copy_term(xv[k][r], lv[k][r], inv_rho);
    }
#pragma unroll
    for (int k = 0; k < kZPer; ++k) out[k] = global_from_sum(s[k], ik[k], ck[k], inv_rho, lo[k], hi[k]);
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) z_kernel(View<T> v, int q) {
    const Ctl* ctl = v.ctl;
    if (ctl->iter + q >= ctl->max_iter) return;
    int g[kZPer];
#pragma unroll
    for (int k = 0; k < kZPer; ++k) {
        const int i = blockIdx.x * (kZThreads * kZPer) + k * kZThreads + threadIdx.x;
        g[k] = i < v.ng ? i : -1;
    }
    if (g[0] < 0) return;
    T z[kZPer];
    global_values_batched<T>(v, g, (T)ctl->inv_rho, z);
#pragma unroll
    for (int k = 0; k < kZPer; ++k)
        if (g[k] >= 0) v.zg[g[k]] = z[k];
}

// Local + dual update of chunk b for iteration offset q of a graph body.
template <typename T>
__device__ __forceinline__ void x_chunk(const View<T>& v, const int b, const int q) {
    const Ctl* ctl = v.ctl;
    const int iter = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    if (iter + q >= maxit) return;
    const bool want = (q == min(K, maxit - iter) - 1);
    const T rho = (T)ctl->rho, inv_rho = (T)ctl->inv_rho;
    __shared__ T us[kXWarps][kMaxBigN];
    __shared__ double red[kXWarps][5];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const BlockInfo bi = v.blocks[b];
    double acc[5] = {0, 0, 0, 0, 0};
    const T* zg = v.zg;
    const int32_t* gidx = v.gidx;
    auto getv = [zg, gidx](int j, int) { return zg[gidx[j]]; };
    // boundary tiles first, then interior ones: the order of every engine
    // (the persistent kernel publishes boundary values early), so the
    // residual partial sums agree bit for bit
    double* dzo = (want && ctl->res_form == OPF_RES_TEXTBOOK) ? v.tdz : nullptr;
    for (int t = bi.tileb + warp; t < bi.tile1; t += kXWarps)
        tile_update<T>(v, v.tiles[t], lane, rho, inv_rho, v.xl, v.lam, v.xl, v.lam, want, acc, us[warp], getv, dzo);
    for (int t = bi.tile0 + warp; t < bi.tileb; t += kXWarps)
        tile_update<T>(v, v.tiles[t], lane, rho, inv_rho, v.xl, v.lam, v.xl, v.lam, want, acc, us[warp], getv, dzo);
    if (!want) return;
    cta_partials(acc, red, v.partials + (size_t)b * 8);
}

template <typename T>
__global__ void __launch_bounds__(kXWarps * 32) x_kernel(View<T> v, int q) {
    x_chunk(v, blockIdx.x, q);
}

// Textbook residual form of Eq. (termination) (the sum over components
// inside the norm): per global i, the copies' changes and duals summed in
// CSR order, D_i = sum_j (x_j - x_j(prev)), L_i = sum_j lambda_j; each block
// writes sum_i D_i^2 and sum_i L_i^2 over its globals (fixed-order tree), so
// dres = rho sqrt(sum D^2) and eps_dual = eps_rel sqrt(sum L^2).
template <typename T>
__global__ void __launch_bounds__(kZThreads) textbook_kernel(View<T> v) {
    const Ctl* ctl = v.ctl;
    __shared__ double sh[2][kZThreads];
    if (ctl->iter >= ctl->max_iter) return;       // no iteration ran in this body
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0, l = 0;
    if (i < v.ng) {
        for (int q = v.gptr[i]; q < v.gptr[i + 1]; ++q) {
            const int j = v.gcol[q];
            d += v.tdz[j];
            l += (double)v.lam[j];
        }
    }
    sh[0][threadIdx.x] = d * d;
    sh[1][threadIdx.x] = l * l;
    __syncthreads();
    for (int w = kZThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        v.tpart[2 * blockIdx.x] = sh[0][0];
        v.tpart[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// Residual check after a graph body (fixed-order sum, Eq. termination);
// returns the stop decision to thread 0.
template <typename T>
__device__ __forceinline__ int finalize_body(const View<T>& v) {
    Ctl* ctl = v.ctl;
    const int iter = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    const int ndone = max(0, min(K, maxit - iter));
    __shared__ double red[kXWarps][5];
    __shared__ double tot[5];
    static_assert(kFinThreads == kXWarps * 32, "finalize reduction layout");
    if (ndone > 0) sum_partials_small(v.partials, v.nblocks, red, tot);
    if (ndone > 0 && ctl->res_form == OPF_RES_TEXTBOOK && threadIdx.x == 0) {
        double d = 0, l = 0;
        for (int b = 0; b < v.nzb; ++b) {
            d += __ldcg(v.tpart + 2 * b);
            l += __ldcg(v.tpart + 2 * b + 1);
        }
        tot[1] = d;
        tot[4] = l;
    }
    if (threadIdx.x != 0) return 0;
    if (ctl->abort) {                   // a bounded wait gave up (status and place already recorded)
        ctl->stop = 1;
        return 1;
    }
    const int it = iter + ndone;
    ctl->iter = it;
    int stop = 0;
    if (ndone > 0) stop = decide(ctl, tot, it);
    if (!stop && it >= maxit) {
        ctl->status = CTL_MAXITER;
        stop = 1;
    }
    ctl->stop = stop;
    return stop;
}

template <typename T>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(View<T> v, cudaGraphConditionalHandle h, int use_cond) {
    const int stop = finalize_body(v);
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// ------------------------------------------------------------- persistent
// Bounded wait until every neighbour CTA has completed `t` iterations: each
// thread polls one neighbour's flag (acquire), the CTA combines the results.
// Returns false when the deadline passed or another CTA aborted.
template <typename T>
__device__ bool wait_neighbours(const View<T>& v, const BlockInfo& bi, int t, unsigned long long tmo, int*) {
    int ok = 1;
    if (bi.nbr1 > bi.nbr0) {
        const unsigned long long deadline = now_ns() + tmo;
        for (int q = bi.nbr0 + threadIdx.x; q < bi.nbr1 && ok; q += blockDim.x) {
            const int32_t* f = v.flags + v.nbrs[q];
            while (ld_acquire(f) < t) {
                if (ld_acquire(&v.ctl->abort)) { ok = 0; break; }
                if (now_ns() > deadline) {
                    if (atomicCAS(&v.ctl->abort, 0, 1) == 0) { v.ctl->status = CTL_TIMEOUT; v.ctl->timeout_where = 1; }
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

template <typename T>
__device__ __forceinline__ void chunk_global(const View<T>& v, const int b, unsigned char* smem_raw) {
    T* zs = reinterpret_cast<T*>(smem_raw);
    __shared__ T us[kXWarps][kMaxBigN];
    __shared__ double red[kXWarps][5];
    __shared__ double tot[5];
    __shared__ int s_last, s_stop, s_ok;
    __shared__ double s_rho;
    Ctl* ctl = v.ctl;
    const BlockInfo bi = v.blocks[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it0 = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    T rho = (T)ctl->rho, inv_rho = (T)ctl->inv_rho;
    const unsigned long long tmo = ctl->timeout_ns;
    const bool withhold = (ctl->skip_block == b);
    int t = 0, checkno = 0;
    bool done = it0 >= maxit;
    while (!done) {
        if (t > 0 && !wait_neighbours(v, bi, t, tmo, &s_ok)) return;
        const T* xr = (t & 1) ? v.xl2 : v.xl;
        const T* lr = (t & 1) ? v.lam2 : v.lam;
        T* xw = (t & 1) ? v.xl : v.xl2;
        T* lw = (t & 1) ? v.lam : v.lam2;
        // global update of the chunk's halo, Eq. (global_sparse)
        for (int h = bi.halo0 + threadIdx.x; h < bi.halo1; h += blockDim.x) {
            const int g = v.halo_gid[h];
            const T z = global_value<T, true>(v, g, xr, lr, inv_rho);
            zs[h - bi.halo0] = z;
            if (v.halo_own[h]) v.zg[g] = z;
        }
        __syncthreads();
        const int nrem = maxit - (it0 + t);
        const bool check = ((t + 1) % K == 0) || nrem == 1;
        double acc[5] = {0, 0, 0, 0, 0};
        auto getv = [zs](int, int m) { return zs[m & 0xFFFF]; };
        for (int q = bi.tileb + warp; q < bi.tile1; q += kXWarps)
            tile_update<T>(v, v.tiles[q], lane, rho, inv_rho, xr, lr, xw, lw, check, acc, us[warp], getv);
        for (int q = bi.tile0 + warp; q < bi.tileb; q += kXWarps)
            tile_update<T>(v, v.tiles[q], lane, rho, inv_rho, xr, lr, xw, lw, check, acc, us[warp], getv);
        __syncthreads();
        ++t;
        if (threadIdx.x == 0 && !withhold) st_release(v.flags + b, t);   // release: cumulative over the CTA barrier
        if (check) {
            cta_partials(acc, red, v.partials + (size_t)b * 8);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned long long ticket = atomicAdd(&ctl->arrive, 1ull);
                s_last = ticket == (unsigned long long)v.nblocks * (checkno + 1) - 1;
            }
            __syncthreads();
            if (s_last) {
                sum_partials_small(v.partials, v.nblocks, red, tot);
                if (threadIdx.x == 0) {
                    ctl->iter = it0 + t;
                    ctl->stop = decide(ctl, tot, it0 + t);
                    __threadfence();
                    st_release(&ctl->decided, checkno + 1);
                }
            }
            if (threadIdx.x == 0) {
                int ok = 1;
                const unsigned long long deadline = now_ns() + tmo;
                while (ld_acquire(&ctl->decided) < checkno + 1) {
                    if (ld_acquire(&ctl->abort)) { ok = 0; break; }
                    if (now_ns() > deadline) {
                        if (atomicCAS(&ctl->abort, 0, 1) == 0) { ctl->status = CTL_TIMEOUT; ctl->timeout_where = 2; }
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
                s_ok = ok;
                s_stop = ok ? ld_acquire(&ctl->stop) : 1;
                s_rho = __ldcg(&ctl->rho);
            }
            __syncthreads();
            rho = (T)s_rho;
            inv_rho = (T)(1.0 / s_rho);
            ++checkno;
            if (!s_ok) return;
            if (s_stop) done = true;
        }
        if (it0 + t >= maxit) done = true;
    }
    // after an odd count the newest iterate is in the second buffer: move the
    // chunk's locals home once the neighbours have finished reading
    if (t & 1) {
        if (!wait_neighbours(v, bi, t, tmo, &s_ok)) return;
        for (int j = bi.loc0 + threadIdx.x; j < bi.loc1; j += blockDim.x) {
            v.xl[j] = __ldcg(v.xl2 + j);
            v.lam[j] = __ldcg(v.lam2 + j);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kXWarps * 32) persistent_kernel(View<T> v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    chunk_global(v, blockIdx.x, smem_raw);
}

// ----------------------------------------------- persistent, shared-memory
// Per-launch shared-memory plan (byte offsets; every region 16-byte aligned).
struct SmemPlan {
    int P, xs, ls, ws, bb, mt, zs, hcon, hp, hc, us, big, tl, ush, rt, total;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Same iteration as persistent_kernel, but the chunk's operators (staged once
// by TMA bulk copies), its local iterate, duals, bbar, meta and the halo's
// bounds, scalings and copy lists stay in shared memory for the whole solve.
// Only copies read by another chunk (the "exported" locals) are written to
// the global ping-pong buffers each iteration; only copies held by another
// chunk are read from them.
// kGather selects how the terms of copies held by other chunks reach the
// boundary global update: true -- every thread first fetches its share of
// the chunk's list of such copies (one mailbox word each, all loads in
// flight together) into shared memory, then the boundary entries are summed
// from shared memory; false -- each thread polls the words of its own
// boundary entries as it sums them.  Same terms, same order, same bits.
template <typename T, bool kGather>
__device__ __forceinline__ void chunk_smem(const View<T>& v, const int b, const SmemPlan& sp, unsigned char* sm) {
    T* sP = reinterpret_cast<T*>(sm + sp.P);
    T* xs = reinterpret_cast<T*>(sm + sp.xs);
    T* ls = reinterpret_cast<T*>(sm + sp.ls);
    T* bb = reinterpret_cast<T*>(sm + sp.bb);
    int* mt = reinterpret_cast<int*>(sm + sp.mt);
    T* zs = reinterpret_cast<T*>(sm + sp.zs);
    T* hcon = reinterpret_cast<T*>(sm + sp.hcon);      // per halo entry: lo, hi, 1/k, c/k (one 4-vector)
    int* hp = reinterpret_cast<int*>(sm + sp.hp);
    int* hc = reinterpret_cast<int*>(sm + sp.hc);
    T* usw = reinterpret_cast<T*>(sm + sp.us);          // big-tile staging, sp.big per warp
    Tile* stl = reinterpret_cast<Tile*>(sm + sp.tl);    // the chunk's tile descriptors
    constexpr bool kF32 = sizeof(T) == 4;
    T* ws = reinterpret_cast<T*>(sm + sp.ws);           // per local: x_j - lambda_j / rho (FP32)
    // (FP32) per warp four shifted copies of a tile's u values, row k
    // holding u_(i + k) at i (zero for i + k >= 32), so that every lane
    // reads its operands u_(base + c) with 16-byte-aligned vector loads
    T* ush = reinterpret_cast<T*>(sm + sp.ush);
    T* rt = reinterpret_cast<T*>(sm + sp.rt);           // gathered exchange: term of each outside copy (aliases usw)
    __shared__ double red[kXWarps][5];
    __shared__ double tot[5];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_last, s_stop, s_ok;
    __shared__ double s_rho;
    Ctl* ctl = v.ctl;
    const BlockInfo bi = v.blocks[b];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it0 = ctl->iter, maxit = ctl->max_iter, K = ctl->K;
    T rho = (T)ctl->rho, inv_rho = (T)ctl->inv_rho;
    const unsigned long long tmo = ctl->timeout_ns;
    const bool withhold = (ctl->skip_block == b);
    const bool adaptive = ctl->adaptive != 0;
    const int nloc = bi.loc1 - bi.loc0, nh = bi.halo1 - bi.halo0, ncp = bi.cp1 - bi.cp0, next = bi.ext1 - bi.ext0;

    // ---- prologue: operators by TMA bulk copies, the rest by plain loads
    const unsigned pbytes = (unsigned)(((size_t)(bi.mat1 - bi.mat0) * sizeof(T) + 15) & ~size_t(15));
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    if constexpr (kF32)
        for (int i = threadIdx.x; i < kXWarps * 4 * kUrow; i += blockDim.x) ush[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0 && pbytes) {
        mbar_expect_tx(&mbar, pbytes);
        const char* src = reinterpret_cast<const char*>(v.P + bi.mat0);
        for (unsigned off = 0; off < pbytes; off += 32768u) {
            const unsigned len = min(32768u, pbytes - off);
            bulk_g2s(reinterpret_cast<char*>(sP) + off, src + off, len, &mbar);
        }
    }
    for (int j = threadIdx.x; j < nloc; j += blockDim.x) {
        xs[j] = v.xl[bi.loc0 + j];
        ls[j] = v.lam[bi.loc0 + j];
        if constexpr (kF32) ws[j] = copy_term(xs[j], ls[j], inv_rho);
        bb[j] = v.bbar[bi.loc0 + j];
        mt[j] = v.meta[bi.loc0 + j];
    }
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
        const int g = v.halo_gid[bi.halo0 + h];
        hcon[4 * h] = v.lo[g]; hcon[4 * h + 1] = v.hi[g]; hcon[4 * h + 2] = v.invk[g]; hcon[4 * h + 3] = v.cik[g];
        hp[h] = v.hcp[bi.halo0 + h] - bi.cp0;
    }
    if (threadIdx.x == 0) hp[nh] = ncp;
    for (int q = threadIdx.x; q < ncp; q += blockDim.x) hc[q] = kGather ? v.hcx[bi.cp0 + q] : v.hci[bi.cp0 + q];
    // gathered exchange: device local of the thread's first outside copy (in
    // a register for the whole solve); further slots are read from global
    const int32_t* gxg = v.ext + bi.ext0;
    const int gx0 = (kGather && (int)threadIdx.x < next) ? gxg[threadIdx.x] : 0;
    for (int q = threadIdx.x; q < bi.tile1 - bi.tile0; q += blockDim.x) stl[q] = v.tiles[bi.tile0 + q];
    const int hb = bi.halob - bi.halo0;                // interior halo entries [0, hb)
    int ok = 1;
    if (pbytes) {
        const unsigned long long deadline = now_ns() + tmo;
        while (!mbar_try_wait(&mbar, 0)) {
            if (now_ns() > deadline) {
                if (atomicCAS(&ctl->abort, 0, 1) == 0) { ctl->status = CTL_TIMEOUT; ctl->timeout_where = 4; }
                ok = 0;
                break;
            }
        }
    }
    if (!__syncthreads_and(ok)) {
        // The solve is abandoned (OPF_ERR_TIMEOUT), but the bulk copy still
        // targets this CTA's shared memory: stay resident until it lands.
        // The wait is bounded (8x the wait limit, at least 4 s); a copy that
        // has not landed by then is recorded as site 5 before the CTA leaves.
        if (threadIdx.x == 0) {
            const unsigned long long lim = max(tmo, 500000000ull) * 8ull;
            const unsigned long long deadline = now_ns() + lim;
            bool landed = false;
            while (!(landed = mbar_try_wait(&mbar, 0)) && now_ns() < deadline) __nanosleep(256);
            if (!landed) ctl->timeout_where = 5;
        }
        __syncthreads();
        return;
    }

    int t = 0, checkno = 0;
    bool done = it0 >= maxit;
    // global update of halo entries [h0, h1), Eq. (global_sparse), copies in
    // CSR order.  Copies of other chunks: at t == 0 the initial iterate from
    // the primary buffers, later the neighbour's term of iteration t - 1
    // from mailbox slot (t - 1) & 1, polled until its tag is t (bounded).
    const unsigned long long* mb = v.mbox;
    const int nlg = v.nl;
    // Mailbox words of the first boundary entry of each thread, loaded at
    // the start of an iteration so that their latency overlaps the
    // interior global update (kPre copies; raw words, tags checked later).
    constexpr int kW = Mail<T>::kWords;
    constexpr int kPre = 4;                     // copies prefetched per thread
    unsigned long long raw[kPre * kW];
    // halo entry h is handled by thread h % blockDim.x (interior and
    // boundary entries alike, so no thread gets a second entry before every
    // thread has one); hb1 = this thread's first boundary entry
    const int hb1 = hb + (int)((threadIdx.x + blockDim.x - (unsigned)hb % blockDim.x) % blockDim.x);
    auto prefetch = [&](int t) {
        if (t == 0) return;
        if constexpr (kGather) {
            // the thread's first slot of the gather list
            if ((int)threadIdx.x < next) Mail<T>::fetch(mb, nlg, (t - 1) & 1, gx0, raw);
        } else {
            const int h = hb1;
            if (h >= nh) return;
            const int q0 = hp[h], n = min(hp[h + 1] - q0, kPre);
#pragma unroll
            for (int k = 0; k < kPre; ++k)
                if (k < n && hc[q0 + k] < 0) Mail<T>::fetch(mb, nlg, (t - 1) & 1, ~hc[q0 + k], raw + k * kW);
        }
    };
    // term of an internal copy (chunk-relative local c)
    auto wint = [&](int c) -> T {
        if constexpr (kF32) return ws[c];
        else return copy_term(xs[c], ls[c], inv_rho);
    };
    // interior entries: every copy is in this chunk; pairs of loads, then
    // the adds in CSR order
    auto zinterior = [&]() {
        for (int h = threadIdx.x; h < hb; h += blockDim.x) {
            const int q0 = hp[h], q1 = hp[h + 1];
            T sum = 0;
            int q = q0;
            for (; q + 1 < q1; q += 2) {
                const T a = wint(hc[q]), c = wint(hc[q + 1]);
                sum += a;
                sum += c;
            }
            if (q < q1) sum += wint(hc[q]);
            zs[h] = halo_global(sum, hcon + 4 * h, inv_rho);
        }
    };
    // boundary entries: copies of other chunks come from the mailbox (or,
    // at t == 0, from the initial iterate)
    auto zboundary = [&](int t, bool& ok) {
        const int slot = (t - 1) & 1;
        const unsigned tag = (unsigned)t;
        for (int h = hb1; h < nh && ok; h += blockDim.x) {
            T sum = 0;
            const int q0 = hp[h], q1 = hp[h + 1];
            const bool pre = h == hb1 && t > 0;      // prefetched words of this entry
            for (int qb = q0; qb < q1 && ok; qb += 4) {
                T w[4];
                unsigned miss = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    w[k] = 0;
                    if (qb + k < q1) {
                        const int c = hc[qb + k];
                        if (c >= 0) {
                            w[k] = wint(c);
                        } else if (t == 0) {
                            w[k] = copy_term(__ldcg(v.xl + ~c), __ldcg(v.lam + ~c), inv_rho);
                        } else if (pre && qb == q0) {
                            if (!Mail<T>::decode(raw + k * kW, tag, w[k])) miss |= 1u << k;
                        } else if (!Mail<T>::get(mb, nlg, slot, ~c, tag, w[k])) {
                            miss |= 1u << k;
                        }
                    }
                }
                if (miss) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (((miss >> k) & 1u) && ok) ok = mail_poll(mb, nlg, slot, ~hc[qb + k], tag, w[k], ctl, tmo, 1);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (qb + k < q1) sum += w[k];
            }
            if (ok) zs[h] = halo_global(sum, hcon + 4 * h, inv_rho);
        }
    };
    // gathered exchange: the term of every outside copy of iteration t - 1
    // into rt (t == 0: from the initial iterate in the primary buffers)
    auto gather = [&](int t, bool& ok) {
        const int slot = (t - 1) & 1;
        const unsigned tag = (unsigned)t;
        for (int k = threadIdx.x; k < next && ok; k += blockDim.x) {
            T w;
            const int l = (k == (int)threadIdx.x) ? gx0 : gxg[k];
            if (t == 0) {
                w = copy_term(__ldcg(v.xl + l), __ldcg(v.lam + l), inv_rho);
            } else {
                const bool hit = (k == (int)threadIdx.x) ? Mail<T>::decode(raw, tag, w)
                                                         : Mail<T>::get(mb, nlg, slot, l, tag, w);
                if (!hit) ok = mail_poll(mb, nlg, slot, l, tag, w, ctl, tmo, 1);
            }
            rt[k] = w;
        }
    };
    // gathered exchange: boundary entries summed from shared memory, copies
    // in CSR order (the same additions as zboundary)
    auto zboundary_gathered = [&]() {
        for (int h = hb1; h < nh; h += blockDim.x) {
            const int q0 = hp[h], q1 = hp[h + 1];
            T sum = 0;
            for (int q = q0; q < q1; ++q) {
                const int c = hc[q];
                sum += c >= 0 ? wint(c) : rt[~c];
            }
            zs[h] = halo_global(sum, hcon + 4 * h, inv_rho);
        }
    };
    // publish the terms of this chunk's exported copies for iteration t
    auto publish = [&](int jl, T w, int t) {
        if (!withhold) Mail<T>::put(v.mbox, nlg, t & 1, bi.loc0 + jl, w, (unsigned)(t + 1));
    };
    // local + dual updates of tiles [q0, q1) (chunk-relative), Eq. (closed_2), Eq. (ADMM-3)
    auto xphase = [&](int q0, int q1, int t, bool pub, bool check, double* acc) {
        for (int q = q0 + warp; q < q1; q += kXWarps) {
            const Tile tl = stl[q];
            if (tl.L == 0) continue;                    // padding tile
            const int jl0 = tl.loc0 - bi.loc0;
            const T* Pt = sP + (tl.mat0 - bi.mat0);
            if (!tl.big) {
                const int L = tl.L, nmax = tl.nmax;
                const bool act = lane < L;
                const int jl = jl0 + lane;
                int base = 0, m = 0;
                T vv = 0, lo = 0, xo = 0, u = 0;
                if (act) {
                    m = mt[jl];
                    base = (m >> 24) & 0x1F;
                    vv = zs[m & 0xFFFF];
                    lo = ls[jl];
                    xo = xs[jl];
                    u = u_of(vv, lo, inv_rho);
                }
                T y;
                if constexpr (kF32) {
                    T* uw = ush + warp * 4 * kUrow;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (lane >= k) uw[k * kUrow + lane - k] = u;
                    __syncwarp();
                    y = tile_gemv_sh(Pt, L, act ? lane : 0, (nmax + 3) >> 2, uw + (base & 3) * kUrow + (base & ~3));
                    __syncwarp();
                } else {
                    y = tile_gemv(Pt, L, lane, nmax, base, u, act);
                }
                if (act) {
                    const T xn = y + bb[jl];
                    const T ln = dual_of(lo, rho, vv, xn);
                    const T wn = copy_term(xn, ln, inv_rho);
                    xs[jl] = xn;
                    ls[jl] = ln;
                    if constexpr (kF32) ws[jl] = wn;
                    if (pub && (m & (1 << 30))) publish(jl, wn, t);
                    if (check) {
                        const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                        acc[0] += pr * pr; acc[1] += dz * dz;
                        acc[2] += (double)vv * (double)vv; acc[3] += (double)xn * (double)xn;
                        acc[4] += (double)ln * (double)ln;
                    }
                }
            } else {
                const int n = tl.nmax;
                T* us = usw + warp * sp.big;
                for (int r = lane; r < n; r += 32) us[r] = u_of(zs[mt[jl0 + r] & 0xFFFF], ls[jl0 + r], inv_rho);
                __syncwarp();
                for (int r = lane; r < n; r += 32) {
                    T y = 0;
                    for (int c = 0; c < n; ++c) y = fma(Pt[c * n + r], us[c], y);
                    const int jl = jl0 + r;
                    const int m = mt[jl];
                    const T vv = zs[m & 0xFFFF];
                    const T lo = ls[jl], xo = xs[jl];
                    const T xn = y + bb[jl];
                    const T ln = dual_of(lo, rho, vv, xn);
                    const T wn = copy_term(xn, ln, inv_rho);
                    xs[jl] = xn;
                    ls[jl] = ln;
                    if constexpr (kF32) ws[jl] = wn;
                    if (pub && (m & (1 << 30))) publish(jl, wn, t);
                    if (check) {
                        const double pr = (double)vv - (double)xn, dz = (double)xn - (double)xo;
                        acc[0] += pr * pr; acc[1] += dz * dz;
                        acc[2] += (double)vv * (double)vv; acc[3] += (double)xn * (double)xn;
                        acc[4] += (double)ln * (double)ln;
                    }
                }
                __syncwarp();
            }
        }
    };
    const int ntl = bi.tile1 - bi.tile0, ntb = bi.tileb - bi.tile0;
    // phase marks in SM cycles (cheap), scaled to ns by the globaltimer over
    // the whole loop
    const bool prof = ctl->profile_phases != 0 && threadIdx.x == 0;
    unsigned long long ph[4] = {0, 0, 0, 0};
    long long tp = prof ? clock64() : 0;
    const long long c_start = tp;
    const unsigned long long g_start = prof ? now_ns() : 0;
    auto mark = [&](int k) {
        if (prof) {
            const long long tn = clock64();
            ph[k] += (unsigned long long)(tn - tp);
            tp = tn;
        }
    };
    auto flush_prof = [&]() {
        if (prof) {
            const double scale = (double)(now_ns() - g_start) / (double)max(1ll, clock64() - c_start);
            for (int k = 0; k < 4; ++k) v.phase[(size_t)b * 4 + k] = (unsigned long long)((double)ph[k] * scale);
        }
    };
    bool snap = false;          // the primary buffers hold the state of the last iteration
    while (!done) {
        const int nrem = maxit - (it0 + t);
        const bool check = ((t + 1) % K == 0) || nrem == 1;
        // with residual balancing rho may change at a check: publish after it
        const bool defer = check && adaptive;
        double acc[5] = {0, 0, 0, 0, 0};
        bool okz = true;
        // global update: interior halo entries (copies all in this chunk),
        // then boundary ones (the neighbours' terms of iteration t - 1)
        prefetch(t);
        zinterior();
        mark(0);
        if constexpr (kGather) {
            gather(t, okz);
            if (!__syncthreads_and(okz)) { flush_prof(); return; }
            zboundary_gathered();
            __syncthreads();
        } else {
            zboundary(t, okz);
            if (!__syncthreads_and(okz)) { flush_prof(); return; }
        }
        mark(1);
        // local update: boundary tiles first so that their terms reach the
        // neighbours while the interior tiles are computed
        xphase(ntb, ntl, t, !defer, check, acc);
        mark(2);
        xphase(0, ntb, t, !defer, check, acc);
        __syncthreads();
        ++t;
        snap = false;
        if (__builtin_expect(check, 0) && !adaptive && t >= 2) {
            // Non-blocking check: the chunk's state after iteration t goes to
            // the primary buffers (x_s, lambda; owners' x) as a snapshot,
            // the partials to slot checkno & 1, a ticket elects the last CTA
            // to decide, and nobody waits for the decision.  A stop decision
            // raises `halt`; every CTA sees it at its next check (or while
            // polling a neighbour that has left) and leaves: the snapshot of
            // the deciding check is the result.  Before a check a CTA waits
            // for the previous decision, so a slot and a snapshot are never
            // overwritten while still needed.
            if (checkno > 0) {
                if (threadIdx.x == 0) {
                    int okw = 1;
                    const unsigned long long deadline = now_ns() + tmo;
                    while (ld_acquire(&ctl->decided) < checkno) {
                        if (ld_acquire(&ctl->abort)) { okw = 0; break; }
                        if (now_ns() > deadline) {
                            if (atomicCAS(&ctl->abort, 0, 1) == 0) { ctl->status = CTL_TIMEOUT; ctl->timeout_where = 2; }
                            okw = 0;
                            break;
                        }
                        __nanosleep(20);
                    }
                    s_ok = okw && !ld_acquire(&ctl->halt);
                }
                __syncthreads();
                if (!s_ok) { flush_prof(); return; }
            }
            for (int h = threadIdx.x; h < nh; h += blockDim.x)
                if (v.halo_own[bi.halo0 + h]) v.zg[v.halo_gid[bi.halo0 + h]] = zs[h];
            for (int j = threadIdx.x; j < nloc; j += blockDim.x) {
                v.xl[bi.loc0 + j] = xs[j];
                v.lam[bi.loc0 + j] = ls[j];
            }
            double* slot = v.partials + (size_t)(checkno & 1) * v.nblocks * 8;
            cta_partials(acc, red, slot + (size_t)b * 8);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned long long ticket = atomicAdd(&ctl->arrive, 1ull);
                s_last = ticket == (unsigned long long)v.nblocks * (checkno + 1) - 1;
                s_stop = 0;
            }
            __syncthreads();
            if (s_last) {
                sum_partials_small(slot, v.nblocks, red, tot);
                if (threadIdx.x == 0) {
                    ctl->iter = it0 + t;
                    const int stop = decide(ctl, tot, it0 + t);
                    ctl->stop = stop;
                    if (stop) ctl->halt = 1;
                    __threadfence();
                    st_release(&ctl->decided, checkno + 1);
                    s_stop = stop;
                }
                __syncthreads();
            }
            ++checkno;
            snap = true;
            if (s_stop) done = true;
        } else if (__builtin_expect(check, 0)) {
            double* slot = v.partials + (size_t)(checkno & 1) * v.nblocks * 8;
            if (checkno > 0 && threadIdx.x == 0) {   // previous (non-blocking) decision consumed that slot
                const unsigned long long deadline = now_ns() + tmo;
                while (ld_acquire(&ctl->decided) < checkno && now_ns() < deadline && !ld_acquire(&ctl->abort))
                    __nanosleep(20);
            }
            cta_partials(acc, red, slot + (size_t)b * 8);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned long long ticket = atomicAdd(&ctl->arrive, 1ull);
                s_last = ticket == (unsigned long long)v.nblocks * (checkno + 1) - 1;
            }
            __syncthreads();
            if (s_last) {
                sum_partials_small(slot, v.nblocks, red, tot);
                if (threadIdx.x == 0) {
                    ctl->iter = it0 + t;
                    ctl->stop = decide(ctl, tot, it0 + t);
                    __threadfence();
                    st_release(&ctl->decided, checkno + 1);
                }
            }
            if (threadIdx.x == 0) {
                int okw = 1;
                const unsigned long long deadline = now_ns() + tmo;
                while (ld_acquire(&ctl->decided) < checkno + 1) {
                    if (ld_acquire(&ctl->abort)) { okw = 0; break; }
                    if (now_ns() > deadline) {
                        if (atomicCAS(&ctl->abort, 0, 1) == 0) { ctl->status = CTL_TIMEOUT; ctl->timeout_where = 2; }
                        okw = 0;
                        break;
                    }
                    __nanosleep(20);
                }
                s_ok = okw;
                s_stop = okw ? ld_acquire(&ctl->stop) : 1;
                s_rho = __ldcg(&ctl->rho);
            }
            __syncthreads();
            rho = (T)s_rho;
            inv_rho = (T)(1.0 / s_rho);
            ++checkno;
            if (!s_ok) return;
            if (s_stop) done = true;
            if (defer) {    // rho may have changed: terms with the new rho, then publish
                for (int j = threadIdx.x; j < nloc; j += blockDim.x) {
                    const T wn = copy_term(xs[j], ls[j], inv_rho);
                    if constexpr (kF32) ws[j] = wn;
                    if (mt[j] & (1 << 30)) publish(j, wn, t - 1);
                }
                __syncthreads();
            }
        }
        if (it0 + t >= maxit) done = true;
        mark(3);
    }
    flush_prof();
    if (snap) return;           // the last check's snapshot is the result
    // epilogue: owners publish the last global update, the chunk's iterate
    // goes back to the primary buffers.  Neighbours read those buffers only
    // at t == 0; after a one-iteration launch, wait until every neighbour
    // has published iteration 0 (which it does after reading them).
    for (int h = threadIdx.x; h < nh; h += blockDim.x)
        if (v.halo_own[bi.halo0 + h]) v.zg[v.halo_gid[bi.halo0 + h]] = zs[h];
    if (t == 1) {
        bool okz = true;
        if constexpr (kGather) {
            for (int k = threadIdx.x; k < next && okz; k += blockDim.x) {
                T w;
                okz = mail_poll(mb, nlg, 0, gxg[k], 1u, w, ctl, tmo, 3);
            }
        } else {
            for (int q = threadIdx.x; q < ncp && okz; q += blockDim.x) {
                T w;
                if (hc[q] < 0) okz = mail_poll(mb, nlg, 0, ~hc[q], 1u, w, ctl, tmo, 3);
            }
        }
        if (!__syncthreads_and(okz)) return;
    }
    for (int j = threadIdx.x; j < nloc; j += blockDim.x) {
        v.xl[bi.loc0 + j] = xs[j];
        v.lam[bi.loc0 + j] = ls[j];
    }
}

// Which chunk a CTA runs.  Chunks are numbered along the feeder, so most
// neighbours are adjacent numbers; the exchange between CTAs of one SM is
// the cheapest, so the k-th CTA to start on SM `smid` prefers chunk
// per * smid + k (`per`: CTAs resident per SM).  A CTA whose preferred
// chunks are out of range or already taken takes the first free one, so
// every chunk gets exactly one CTA whatever the placement (`claim`: one
// zeroed word per chunk).  Which CTA runs a chunk does not change any
// result: the chunk's work and its slot in the residual reduction depend
// only on the chunk number.
__device__ __forceinline__ int claim_chunk(int32_t* claim, int nblocks, int per) {
    __shared__ int s_b;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        int b = -1;
        if (per >= 1 && ((long long)smid + 1) * per <= nblocks)
            for (int k = 0; k < per && b < 0; ++k)
                if (atomicCAS(claim + (size_t)per * smid + k, 0, 1) == 0) b = per * (int)smid + k;
        for (int c = 0; b < 0 && c < nblocks; ++c)
            if (atomicCAS(claim + c, 0, 1) == 0) b = c;
        s_b = b;
    }
    __syncthreads();
    return s_b;
}

template <typename T, bool kGather>
__global__ void __launch_bounds__(kXWarps * 32, 2) persistent_smem_kernel(View<T> v, SmemPlan sp) {
    extern __shared__ __align__(128) unsigned char sm[];
    // nblocks CTAs claim nblocks chunks one each: the scan always finds one
    const int b = claim_chunk(v.flags, v.nblocks, 2);
    if (b < 0) return;
    chunk_smem<T, kGather>(v, b, sp, sm);
}

// ------------------------------------------------------------------ batch
// Many problems in one cooperative launch: CTA i runs chunk map[i].chunk of
// problem map[i].inst with that problem's own view, flags, control block and
// ticket counter, so an instance's iterates and stopping decision do not
// depend on the other instances in the launch.
struct CtaMap {
    int32_t inst, chunk;
};

// The map lists each instance's chunks consecutively; CTAs claim map
// entries by SM as above (`per` CTAs resident per SM), so an instance's
// neighbouring chunks tend to share an SM.
template <typename T>
__global__ void __launch_bounds__(kXWarps * 32, 3) batch_smem_kernel(const View<T>* views, const CtaMap* map, SmemPlan sp,
                                                                     int32_t* claim, int per) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ View<T> sv;
    const int i = claim_chunk(claim, gridDim.x, per);
    if (i < 0) return;
    const CtaMap m = map[i];
    if (threadIdx.x == 0) sv = views[m.inst];
    __syncthreads();
    chunk_smem<T, true>(sv, m.chunk, sp, sm);
}

template <typename T>
__global__ void __launch_bounds__(kXWarps * 32, 4) batch_global_kernel(const View<T>* views, const CtaMap* map,
                                                                       int32_t* claim, int per) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ View<T> sv;
    const int i = claim_chunk(claim, gridDim.x, per);
    if (i < 0) return;
    const CtaMap m = map[i];
    if (threadIdx.x == 0) sv = views[m.inst];
    __syncthreads();
    chunk_global(sv, m.chunk, smem_raw);
}

// Batched graph engine: the graph engine's kernels over many instances.
// Global update: CTA -> (instance, first global); local update: CTA ->
// (instance, chunk); one finalize CTA per instance.  Instances that have
// stopped skip their work; the body repeats while any instance runs.
struct ZMap {
    int32_t inst, g0;
};

template <typename T>
__global__ void __launch_bounds__(kZThreads) zb_kernel(const View<T>* views, const ZMap* zmap, int q) {
    const ZMap m = zmap[blockIdx.x];
    const View<T>& v = views[m.inst];
    const Ctl* ctl = v.ctl;
    if (ctl->stop || ctl->iter + q >= ctl->max_iter) return;
    int g[kZPer];
#pragma unroll
    for (int k = 0; k < kZPer; ++k) {
        const int i = m.g0 + k * kZThreads + threadIdx.x;
        g[k] = i < v.ng ? i : -1;
    }
    if (g[0] < 0) return;
    T z[kZPer];
    global_values_batched<T>(v, g, (T)ctl->inv_rho, z);
#pragma unroll
    for (int k = 0; k < kZPer; ++k)
        if (g[k] >= 0) v.zg[g[k]] = z[k];
}

template <typename T>
__global__ void __launch_bounds__(kXWarps * 32) xb_kernel(const View<T>* views, const CtaMap* map, int q) {
    __shared__ View<T> sv;
    const CtaMap m = map[blockIdx.x];
    if (threadIdx.x == 0) sv = views[m.inst];
    __syncthreads();
    if (sv.ctl->stop) return;
    x_chunk(sv, m.chunk, q);
}

// ---------------------------------------------- graph engines, tile-parallel
// Local update of the iterations that take no residual partials (graph and
// host-loop engines, one problem or a batch), with the tiles of every
// instance in work items of kItemTiles consecutive tiles (any warp may
// run any tile: x and lambda of a tile do not depend on who computes them,
// and no partial sums are taken), so the grid fills every SM whatever the
// problems' chunking.  Each warp copies the operator block of its next
// small tile into its own shared-memory buffer with one bulk copy (TMA,
// completion on the warp's mbarrier), issued as soon as the current tile's
// GEMV has read the buffer, so the copy overlaps the next tile's vector
// loads and gather.
constexpr int kItemTiles = 8;
constexpr int kStageBytes = 4096;          // a small FP32 tile's block: 8 column groups x 4 x 32 lanes x 4 B

template <typename T>
__device__ __forceinline__ unsigned stage_bytes(const Tile& tl) {
    if (tl.big || tl.L <= 0) return 0;
    const unsigned b = (unsigned)(((tl.nmax + 3) >> 2) * 4 * tl.L) * (unsigned)sizeof(T);
    return b <= (unsigned)kStageBytes ? b : 0;
}

// Lane 0 starts the bulk copy of tile tl's operator block (if it is staged).
template <typename T>
__device__ __forceinline__ void stage_issue(const T* P, const Tile& tl, T* buf, unsigned long long* bar, int lane) {
    const unsigned b = stage_bytes<T>(tl);
    if (lane == 0 && b) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, b);
        bulk_g2s(buf, P + tl.mat0, b, bar);
    }
}

// Bounded wait for the warp's staged block (phase parity `ph`): false after
// 0.5 s without completion (the copy is then waited for once more, again
// bounded, before the caller gives up).
__device__ __forceinline__ bool stage_wait(unsigned long long* bar, unsigned ph) {
    for (int round = 0; round < 2; ++round) {
        const unsigned long long deadline = now_ns() + 500000000ull;
        unsigned spins = 0;
        while (!mbar_try_wait(bar, ph)) {
            if ((++spins & 1023u) == 0 && now_ns() > deadline) break;
        }
        if (mbar_try_wait(bar, ph)) return round == 0;
    }
    return false;
}

// A big tile's local and dual update without partials (Eq. closed_2, Eq.
// ADMM-3): u staged in the warp's us, each lane's rows over the full
// operator in global memory (the order of every engine).
template <typename T>
__device__ __forceinline__ void tile_big_plain(const View<T>* vp, const Tile& tl, int lane, T rho, T inv_rho, T* us) {
    const T* zg = vp->zg;
    const int32_t* gidx = vp->gidx;
    T* xl = vp->xl;
    T* lam = vp->lam;
    const int n = tl.nmax;
    for (int r = lane; r < n; r += 32) {
        const int j = tl.loc0 + r;
        us[r] = u_of(zg[gidx[j]], ldcg(lam + j), inv_rho);
    }
    __syncwarp();
    const T* Pm = vp->P + tl.mat0;
    for (int r = lane; r < n; r += 32) {
        T y = 0;
        for (int c = 0; c < n; ++c) y = fma(Pm[c * n + r], us[c], y);
        const int j = tl.loc0 + r;
        const T vv = zg[gidx[j]];
        const T lo = ldcg(lam + j);
        const T xn = y + vp->bbar[j];
        xl[j] = xn;
        lam[j] = dual_of(lo, rho, vv, xn);
    }
    __syncwarp();
}

// Tile descriptor held by lane k of the warp, to every lane.
__device__ __forceinline__ Tile tile_from_lane(const Tile& mine, int k) {
    Tile t;
    t.loc0 = __shfl_sync(0xffffffffu, mine.loc0, k);
    t.mat0 = __shfl_sync(0xffffffffu, mine.mat0, k);
    const unsigned lm = __shfl_sync(0xffffffffu, (unsigned)(uint16_t)mine.L | ((unsigned)(uint16_t)mine.nmax << 16), k);
    t.L = (int16_t)(lm & 0xFFFFu);
    t.nmax = (int16_t)(lm >> 16);
    t.big = __shfl_sync(0xffffffffu, mine.big, k);
    return t;
}

// This lane's vector loads of a small tile (meta -> shuffle base, gather
// index, dual, bbar); g = -1 for lanes without a local or other tiles.
template <typename T>
__device__ __forceinline__ void vec_issue(const Tile& tl, int lane, const int32_t* meta, const int32_t* gidx,
                                          const T* lam, const T* bbar, int& base, int& g, T& lo, T& bb) {
    if (!tl.big && lane < tl.L) {
        const int j = tl.loc0 + lane;
        base = (meta[j] >> 24) & 0x1F;
        g = gidx[j];
        lo = ldcg(lam + j);
        bb = bbar[j];
    } else {
        base = 0; g = -1; lo = 0; bb = 0;
    }
}

// Work item of the tile-parallel local update: instance, tiles [t0, t1).
struct TileItem {
    int32_t inst, t0, t1, pad;
};

// Whether instance c's local update at offset q of the body takes residual
// partials (then the chunk kernel runs it) or has nothing to do.
__device__ __forceinline__ bool plain_iteration(const Ctl* c, int q) {
    const int iter = c->iter, maxit = c->max_iter, K = c->K;
    if (c->stop || iter + q >= maxit) return false;
    return q != min(K, maxit - iter) - 1;
}
__device__ __forceinline__ bool check_iteration(const Ctl* c, int q) {
    const int iter = c->iter, maxit = c->max_iter, K = c->K;
    return !c->stop && iter + q < maxit && q == min(K, maxit - iter) - 1;
}

// Check role of the tile-parallel kernel (kept out of line so that its
// registers do not constrain the tile role's).
template <typename T>
__device__ __noinline__ void xt_check_role(const View<T>* views, int ninst, int ntl, int q) {
    __shared__ View<T> sv;
    __shared__ int wl[kXWarps * 32];
    __shared__ int nwl;
    for (int i0 = 0; i0 < ninst; i0 += blockDim.x) {
        if (threadIdx.x == 0) nwl = 0;
        __syncthreads();
        const int i = i0 + threadIdx.x;
        if (i < ninst && check_iteration(views[i].ctl, q)) wl[atomicAdd(&nwl, 1)] = i;
        __syncthreads();
        const int n = nwl;
        for (int k = 0; k < n; ++k) {
            if (threadIdx.x == 0) sv = views[wl[k]];
            __syncthreads();
            for (int b = blockIdx.x - ntl; b < sv.nblocks; b += gridDim.x - ntl) {
                x_chunk(sv, b, q);
                __syncthreads();
            }
            __syncthreads();                            // sv is rewritten next
        }
        __syncthreads();
    }
}

// Blocks [0, ntl): warps take work items in turn (tile role).  Blocks
// [ntl, gridDim.x): instances whose check falls on this offset q (their
// last round ends before the body's) are run chunk by chunk with partials,
// as the chunk kernel does (check role; normally they find none and leave).
template <typename T>
__global__ void __launch_bounds__(kXWarps * 32, sizeof(T) == 4 ? 4 : 3)
    xt_kernel(const View<T>* views, const TileItem* items, int nitems, int ntl, int ninst, int q) {
    extern __shared__ __align__(128) unsigned char xt_smem[];
    __shared__ unsigned long long bars[kXWarps];
    __shared__ T us[kXWarps][kMaxBigN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x >= ntl) {
        xt_check_role<T>(views, ninst, ntl, q);
        return;
    }
    T* buf = reinterpret_cast<T*>(xt_smem + (size_t)warp * kStageBytes);
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    unsigned ph = 0;
    const int nw = ntl * kXWarps;
    Tile none;
    none.loc0 = 0; none.mat0 = 0; none.L = 0; none.nmax = 0; none.big = 0;
    for (int it = blockIdx.x * kXWarps + warp; it < nitems; it += nw) {
        const TileItem m = items[it];
        const View<T>* vp = views + m.inst;
        const Ctl* c = vp->ctl;
        if (!plain_iteration(c, q)) continue;
        const T rho = (T)c->rho, inv_rho = (T)c->inv_rho;
        const T* P = vp->P;
        const T* zg = vp->zg;
        const int32_t* gidx = vp->gidx;
        const int32_t* meta = vp->meta;
        const T* bbar = vp->bbar;
        T* xl = vp->xl;
        T* lam = vp->lam;
        // the item's tile descriptors, one per lane, passed round by shuffles
        const int nt = m.t1 - m.t0;
        Tile mine = none;
        if (lane < nt) mine = vp->tiles[m.t0 + lane];
        Tile cur = tile_from_lane(mine, 0);
        stage_issue<T>(P, cur, buf, bar, lane);
        // software pipeline: the next tile's vectors load while this tile runs,
        // and its gathered global value right after
        int cb, cg;
        T clo, cbb;
        vec_issue<T>(cur, lane, meta, gidx, lam, bbar, cb, cg, clo, cbb);
        T cvv = cg >= 0 ? zg[cg] : (T)0;
        for (int k = 0; k < nt; ++k) {
            const Tile nxt = (k + 1 < nt) ? tile_from_lane(mine, k + 1) : none;
            int nb, gn;
            T nlo, nbb;
            vec_issue<T>(nxt, lane, meta, gidx, lam, bbar, nb, gn, nlo, nbb);
            const bool staged = stage_bytes<T>(cur) != 0;
            if (!staged) stage_issue<T>(P, nxt, buf, bar, lane);   // the buffer is free
            if (cur.big) {
                tile_big_plain<T>(vp, cur, lane, rho, inv_rho, us[warp]);
            } else if (cur.L > 0) {
                const bool act = lane < cur.L;
                const T u = u_of(cvv, clo, inv_rho);
                if (staged) {
                    if (!__all_sync(0xffffffffu, stage_wait(bar, ph))) {
                        if (lane == 0) {
                            Ctl* cw = vp->ctl;
                            if (atomicCAS(&cw->abort, 0, 1) == 0) { cw->status = CTL_TIMEOUT; cw->timeout_where = 6; }
                        }
                        return;
                    }
                    ph ^= 1u;
                }
                const T y = tile_gemv(staged ? buf : P + cur.mat0, cur.L, lane, cur.nmax, cb, u, act);
                if (staged) {
                    __syncwarp();                           // every lane has read the buffer
                    stage_issue<T>(P, nxt, buf, bar, lane);
                }
                if (act) {
                    const int j = cur.loc0 + lane;
                    const T xn = y + cbb;
                    xl[j] = xn;
                    lam[j] = dual_of(clo, rho, cvv, xn);
                }
            }
            cvv = gn >= 0 ? zg[gn] : (T)0;
            cur = nxt; cb = nb; clo = nlo; cbb = nbb;
        }
    }
}

// Grid of the tile-parallel kernel: tile-role CTAs up to what is resident
// on every SM at once (warps then take items in turn), check-role CTAs one
// per SM at most.
constexpr size_t kXtSmem = (size_t)kXWarps * kStageBytes;
struct XtGrid {
    int ntl, nchk;
};
template <typename T>
XtGrid xt_grid(int nitems, int nctas) {
    int dev = 0, sms = 0, per = 0;
    OPF_CUDA(cudaGetDevice(&dev));
    OPF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OPF_CUDA(cudaFuncSetAttribute(xt_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXtSmem));
    OPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, xt_kernel<T>, kXWarps * 32, kXtSmem));
    XtGrid g;
    g.ntl = std::max(1, std::min((nitems + kXWarps - 1) / kXWarps, std::max(1, per) * sms));
    g.nchk = std::max(1, std::min(nctas, sms));
    return g;
}

template <typename T>
__global__ void __launch_bounds__(kFinThreads) finb_kernel(const View<T>* views, int* running) {
    const View<T>& v = views[blockIdx.x];
    const int stopped = v.ctl->stop;
    __syncthreads();                  // every thread has read stop before thread 0 may write it
    if (stopped) return;
    const int stop = finalize_body(v);
    if (threadIdx.x == 0 && stop) atomicSub(running, 1);
}

__global__ void batch_cond_kernel(const int* running, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, *running > 0 ? 1u : 0u);
}

// One CTA per instance: objective c^T x in a fixed order, then the instance's
// control block is copied to a contiguous array for one read-back.
template <typename T>
__global__ void __launch_bounds__(256) batch_finish_kernel(const View<T>* views, Ctl* out) {
    __shared__ double sh[256];
    const View<T>& v = views[blockIdx.x];
    double s = 0;
    for (int i = threadIdx.x; i < v.ng; i += 256) s += v.cost[i] * (double)v.zg[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        v.ctl->objective = sh[0];
        out[blockIdx.x] = *v.ctl;
    }
}

// Zero every instance's CTA flags and, for the shared-memory persistent
// kernel, its boundary mailbox (one launch for the whole batch).
template <typename T>
__global__ void batch_clear_flags(const View<T>* views, int n, int mailbox) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        for (int b = threadIdx.x; b < views[i].nblocks; b += blockDim.x) views[i].flags[b] = 0;
        if (mailbox) {
            const size_t words = (size_t)views[i].nl * 2 * Mail<T>::kWords;
            for (size_t j = threadIdx.x; j < words; j += blockDim.x) views[i].mbox[j] = 0;
        }
    }
}

// Warm start across a topology change: new local j takes the old iterate and
// dual of local map[j] (same component, same position, same global
// variable), or keeps its initial point when map[j] < 0.
template <typename T>
__global__ void warm_gather_kernel(const int32_t* __restrict__ map, const T* __restrict__ oxl, const T* __restrict__ olam,
                                   T* __restrict__ nxl, T* __restrict__ nlam, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && map[j] >= 0) {
        nxl[j] = oxl[map[j]];
        nlam[j] = olam[map[j]];
    }
}

// ------------------------------------------------------- re-precompute
// Device FP64 precompute of Eq. (closed_2) for components whose rows
// changed (a line's impedances, shunts or taps): with the Cholesky factor L
// of A A^T (A of full row rank), W = L^-1 A, P = I - W^T W (= -Abar) and
// bbar = W^T L^-1 b.  One warp per component; the result goes into both
// precisions' packed operators and bbar, and a dense copy for the host.
struct RpDesc {
    int32_t m, n, aoff, boff;      // rows, locals, offsets into the A (row-major) and b buffers
    int32_t mat0, L, base, big;    // destination tile: first element, lanes, lane base, big flag
    int32_t loc0, outoff, woff, _pad;   // device index of local 0; dense output; scratch offset
};

__global__ void __launch_bounds__(32) reprecompute_kernel(const RpDesc* __restrict__ ds, const double* __restrict__ A,
                                                         const double* __restrict__ bv, double* scratch, double* P64,
                                                         float* P32, double* bb64, float* bb32, double* out, int* err) {
    const RpDesc d = ds[blockIdx.x];
    const int lane = threadIdx.x, m = d.m, n = d.n;
    double* G = scratch + d.woff;                  // m x m, lower triangle
    double* W = G + m * m;                         // m x n
    double* y = W + (size_t)m * n;                 // m
    const double* Ar = A + d.aoff;
    // G = A A^T (lower triangle)
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, k = e % m;
        if (k > i) continue;
        double s = 0;
        for (int c = 0; c < n; ++c) s += Ar[i * n + c] * Ar[k * n + c];
        G[i * m + k] = s;
    }
    __syncwarp();
    double gmax = 0;
    for (int i = 0; i < m; ++i) gmax = fmax(gmax, G[i * m + i]);
    // right-looking Cholesky
    for (int k = 0; k < m; ++k) {
        if (lane == 0) {
            const double dk = G[k * m + k];
            if (!(dk > 1e-13 * gmax)) atomicExch(err, 1);   // rank deficient: the host path is needed
            G[k * m + k] = sqrt(fmax(dk, 1e-300));
        }
        __syncwarp();
        const double lkk = G[k * m + k];
        for (int i = k + 1 + lane; i < m; i += 32) G[i * m + k] /= lkk;
        __syncwarp();
        for (int e = lane; e < m * m; e += 32) {
            const int i = e / m, j = e % m;
            if (j > k && j <= i) G[i * m + j] -= G[i * m + k] * G[j * m + k];
        }
        __syncwarp();
    }
    // W = L^-1 A (columns in parallel), y = L^-1 b
    for (int c = lane; c < n; c += 32)
        for (int i = 0; i < m; ++i) {
            double s = Ar[i * n + c];
            for (int p = 0; p < i; ++p) s -= G[i * m + p] * W[p * n + c];
            W[i * n + c] = s / G[i * m + i];
        }
    if (lane == 0)
        for (int i = 0; i < m; ++i) {
            double s = bv[d.boff + i];
            for (int p = 0; p < i; ++p) s -= G[i * m + p] * y[p];
            y[i] = s / G[i * m + i];
        }
    __syncwarp();
    // P = I - W^T W (one triangle, mirrored: exactly symmetric), bbar = W^T y
    for (int e = lane; e < n * n; e += 32) {
        const int c = e / n, r = e % n;
        if (r < c) continue;
        double s = 0;
        for (int i = 0; i < m; ++i) s += W[i * n + c] * W[i * n + r];
        const double pv = (c == r ? 1.0 : 0.0) - s;
        auto put = [&](int cc, int rr) {
            const size_t at = d.big ? (size_t)d.mat0 + (size_t)cc * n + rr
                                    : (size_t)d.mat0 + ((size_t)(cc / 4) * d.L + d.base + rr) * 4 + cc % 4;
            P64[at] = pv;
            P32[at] = (float)pv;
            out[d.outoff + cc * n + rr] = pv;
        };
        put(c, r);
        if (r != c) put(r, c);
    }
    for (int c = lane; c < n; c += 32) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += W[i * n + c] * y[i];
        bb64[d.loc0 + c] = s;
        bb32[d.loc0 + c] = (float)s;
        out[d.outoff + n * n + c] = s;
    }
}

// ------------------------------------------------------------ misc kernels
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
    size_t gptr, gcol, gidx, meta, tiles, blocks, halo_gid, halo_own, nbrs, hcp, hci, flags, cost, partials, phase, ctl, mbox;
    size_t tdz, tpart, hcx, ext, xtv, xti;
    size_t xl, lam, xl2, lam2, bbar, xl0, xl32, lam32, xl2_32, lam2_32, bbar32, xl0_32, P64, P32;
    size_t total;
};

Layout layout_of(const opf_problem* p) {
    const Packed& k = p->pk;
    Arena a;
    Layout L;
    L.lo = a.take<double>(k.ng); L.hi = a.take<double>(k.ng); L.invk = a.take<double>(k.ng);
    L.cik = a.take<double>(k.ng); L.zg = a.take<double>(k.ng);
    L.lo32 = a.take<float>(k.ng); L.hi32 = a.take<float>(k.ng); L.invk32 = a.take<float>(k.ng);
    L.cik32 = a.take<float>(k.ng); L.zg32 = a.take<float>(k.ng);
    L.gptr = a.take<int32_t>(k.ng + 1); L.gcol = a.take<int32_t>(k.nl); L.gidx = a.take<int32_t>(k.nl);
    L.meta = a.take<int32_t>(k.nl);
    L.tiles = a.take<Tile>(k.tiles.size()); L.blocks = a.take<BlockInfo>(k.blocks.size());
    L.halo_gid = a.take<int32_t>(k.halo_gid.size()); L.halo_own = a.take<uint8_t>(k.halo_own.size());
    L.nbrs = a.take<int32_t>(k.nbrs.size() + 1);
    L.hcp = a.take<int32_t>(k.hcp.size()); L.hci = a.take<int32_t>(k.hci.size() + 1);
    L.hcx = a.take<int32_t>(k.hcx.size() + 1); L.ext = a.take<int32_t>(k.ext.size() + 1);
    L.flags = a.take<int32_t>(k.nblocks);
    L.cost = a.take<double>(k.ng);
    L.partials = a.take<double>((size_t)k.nblocks * 16); L.ctl = a.take<Ctl>(1);   // two check slots
    L.phase = a.take<unsigned long long>((size_t)k.nblocks * 4);
    L.mbox = a.take<unsigned long long>((size_t)k.nl * 4);     // 2 slots x 2 words (f64)
    L.tdz = a.take<double>(std::max(1, k.nl));
    L.tpart = a.take<double>((size_t)2 * ((k.ng + kZThreads - 1) / kZThreads + 1));
    L.xtv = a.take<View<double>>(2);
    L.xti = a.take<TileItem>(std::max<size_t>(1, (k.tiles.size() + kItemTiles - 1) / kItemTiles));
    L.xl = a.take<double>(k.nl); L.lam = a.take<double>(k.nl); L.xl2 = a.take<double>(k.nl); L.lam2 = a.take<double>(k.nl);
    L.bbar = a.take<double>(k.nl); L.xl0 = a.take<double>(k.nl);
    L.xl32 = a.take<float>(k.nl); L.lam32 = a.take<float>(k.nl); L.xl2_32 = a.take<float>(k.nl); L.lam2_32 = a.take<float>(k.nl);
    L.bbar32 = a.take<float>(k.nl); L.xl0_32 = a.take<float>(k.nl);
    // operators, padded so a chunk's 16-byte-rounded bulk copy stays inside
    L.P64 = a.take<double>(k.mat_elems + 8); L.P32 = a.take<float>(k.mat_elems + 8);
    L.total = (a.off + 255) & ~size_t(255);
    return L;
}

template <typename T>
View<T> view_of(const opf_problem* p, const DevPrec& d) {
    View<T> v;
    v.lo = (const T*)d.lo; v.hi = (const T*)d.hi; v.invk = (const T*)d.invk; v.cik = (const T*)d.cik;
    v.zg = (T*)d.zg; v.gptr = p->gptr; v.gcol = p->gcol;
    v.xl = (T*)d.xl; v.lam = (T*)d.lam; v.xl2 = (T*)d.xl2; v.lam2 = (T*)d.lam2;
    v.bbar = (const T*)d.bbar; v.xl0 = (const T*)d.xl0; v.gidx = p->gidx; v.meta = p->meta;
    v.tiles = p->tiles; v.blocks = p->blocks; v.halo_gid = p->halo_gid; v.halo_own = p->halo_own;
    v.nbrs = p->nbrs; v.hcp = p->hcp; v.hci = p->hci; v.hcx = p->hcx; v.ext = p->ext; v.flags = p->flags;
    v.P = (const T*)d.P; v.cost = p->cost; v.partials = p->partials; v.phase = p->phase; v.ctl = p->ctl;
    v.mbox = p->mbox;
    v.tdz = p->tdz; v.tpart = p->tpart;
    v.ng = p->pk.ng; v.nl = p->pk.nl; v.nblocks = p->pk.nblocks;
    v.nzb = (p->pk.ng + kZThreads - 1) / kZThreads;
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
const DevPrec& prec_of(const opf_problem* p) { return sizeof(T) == 8 ? p->d64 : p->d32; }

template <typename T>
void enqueue_init(opf_problem* p, cudaStream_t s) {
    View<T> v = view_of<T>(p, prec_of<T>(p));
    const int n = std::max(p->pk.nl, p->pk.ng) + 1;
    init_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(v);
    OPF_CUDA(cudaGetLastError());
}

// The problem's View on the device (slot 0 FP32, slot 1 FP64), as the
// tile-parallel kernel reads it.
template <typename T>
const View<T>* device_view(const opf_problem* p) {
    return reinterpret_cast<const View<T>*>(static_cast<const char*>(p->xt_views) +
                                            (sizeof(T) == 8 ? sizeof(View<double>) : 0));
}

// One graph body (or host-loop round) of K iterations: the global update,
// then the local update -- tile-parallel on the positions without residual
// partials, the chunk kernel on the last (the check) -- and the finalize.
// xg: the tile kernel's grid (computed here when null; a caller that
// captures the body computes it before the capture begins).
template <typename T>
void enqueue_iterations(opf_problem* p, int K, int form, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                        const XtGrid* xg = nullptr) {
    View<T> v = view_of<T>(p, prec_of<T>(p));
    const int zb = (p->pk.ng + kZThreads - 1) / kZThreads;
    const XtGrid g = xg ? *xg : xt_grid<T>(p->xt_nitems, p->pk.nblocks);
    const View<T>* dv = device_view<T>(p);
    const TileItem* di = static_cast<const TileItem*>(p->xt_items);
    for (int q = 0; q < K; ++q) {
        z_kernel<T><<<zb_blocks(p->pk.ng), kZThreads, 0, s>>>(v, q);
        if (q < K - 1)
            xt_kernel<T><<<g.ntl + g.nchk, kXWarps * 32, kXtSmem, s>>>(dv, di, p->xt_nitems, g.ntl, 1, q);
        else
            x_kernel<T><<<p->pk.nblocks, kXWarps * 32, 0, s>>>(v, q);
    }
    if (form == OPF_RES_TEXTBOOK) textbook_kernel<T><<<zb, kZThreads, 0, s>>>(v);
    finalize_kernel<T><<<1, kFinThreads, 0, s>>>(v, h, use_cond);
    OPF_CUDA(cudaGetLastError());
}

template <typename T>
GraphEntry& get_graph(opf_problem* p, int K, int form) {
    const int prec = sizeof(T) == 8 ? OPF_FP64 : OPF_FP32;
    auto key = std::make_pair(prec + 2 * form, K);
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
    const XtGrid xg = xt_grid<T>(p->xt_nitems, p->pk.nblocks);
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    OPF_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_iterations<T>(p, K, form, cs, h, 1, &xg);
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
    return p->graphs.emplace(key, g).first->second;
}

template <typename T>
size_t persistent_smem(const opf_problem* p) { return (size_t)std::max(1, p->pk.max_halo) * sizeof(T); }

struct ChunkMax {
    int mat = 0, loc = 0, halo = 0, copies = 0, big = 0, tiles = 0, ext = 0;
    void add(const Packed& k) {
        mat = std::max(mat, k.max_mat); loc = std::max(loc, k.max_loc); halo = std::max(halo, k.max_halo);
        copies = std::max(copies, k.max_copies); big = std::max(big, k.max_big); tiles = std::max(tiles, k.max_tiles);
        ext = std::max(ext, k.max_ext);
    }
};

template <typename T>
SmemPlan smem_plan_of(const ChunkMax& k) {
    SmemPlan sp;
    int off = 0;
    auto take = [&](size_t bytes) {
        const int o = off;
        off += (int)((bytes + 15) & ~size_t(15));
        return o;
    };
    const size_t w = sizeof(T);
    sp.P = take((size_t)k.mat * w + 16);
    // FP32 keeps x - lambda / rho per local and the shifted u rows; FP64
    // (bound by FP64 fma throughput) recomputes the former and shuffles u,
    // which keeps two of its CTAs within one SM's shared memory
    const bool f32 = w == 4;
    sp.xs = take((size_t)k.loc * w); sp.ls = take((size_t)k.loc * w); sp.ws = take(f32 ? (size_t)k.loc * w : 0);
    sp.bb = take((size_t)k.loc * w); sp.mt = take((size_t)k.loc * 4);
    sp.zs = take((size_t)k.halo * w); sp.hcon = take((size_t)k.halo * 4 * w);
    sp.hp = take((size_t)(k.halo + 1) * 4); sp.hc = take((size_t)std::max(1, k.copies) * 4);
    sp.big = k.big;
    // big-tile staging (tile phase) and the gathered outside terms (global
    // update phase) are never live at the same time: one region
    sp.us = take(std::max((size_t)kXWarps * k.big * w, (size_t)std::max(1, k.ext) * w));
    sp.rt = sp.us;
    sp.tl = take((size_t)std::max(1, k.tiles) * sizeof(Tile));
    sp.ush = take(f32 ? (size_t)kXWarps * 4 * kUrow * w : 0);
    sp.total = off;
    return sp;
}

template <typename T>
SmemPlan smem_plan(const opf_problem* p) {
    ChunkMax m;
    m.add(p->pk);
    return smem_plan_of<T>(m);
}


// CTAs of `kernel` (kXWarps warps, `smem` bytes dynamic) resident per SM;
// 0 if the query fails.
template <typename KernelT>
int resident_per_sm(KernelT kernel, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kXWarps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// Can every chunk's CTA be co-resident with `smem` dynamic bytes?
template <typename KernelT>
bool coop_fits(KernelT kernel, size_t smem, int nblocks) {
    int dev = 0, coop = 0, sms = 0, per_sm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || smem > (size_t)optin) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kXWarps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * sms >= nblocks;
}

// 0: none, 1: persistent (global-memory iterate), 2: persistent (shared-memory iterate)
template <typename T>
int persistent_variant(const opf_problem* p) {
    const size_t sm = (size_t)smem_plan<T>(p).total;
    const bool smem_ok = coop_fits(persistent_smem_kernel<T, true>, sm, p->pk.nblocks) &&
                         coop_fits(persistent_smem_kernel<T, false>, sm, p->pk.nblocks);
    if (p->force_variant >= 2) return smem_ok ? p->force_variant : 0;
    if (p->force_variant != 1 && smem_ok) return 2;
    if (coop_fits(persistent_kernel<T>, persistent_smem<T>(p), p->pk.nblocks)) return 1;
    return 0;
}

template <typename T>
bool persistent_fits(const opf_problem* p) { return persistent_variant<T>(p) != 0; }

template <typename T>
void launch_persistent(opf_problem* p, cudaStream_t s) {
    View<T> v = view_of<T>(p, prec_of<T>(p));
    OPF_CUDA(cudaMemsetAsync(p->flags, 0, sizeof(int32_t) * p->pk.nblocks, s));
    const int variant = persistent_variant<T>(p);
    if (variant >= 2) {
        OPF_CUDA(cudaMemsetAsync(p->mbox, 0, (size_t)p->pk.nl * 2 * Mail<T>::kWords * sizeof(unsigned long long), s));
        SmemPlan sp = smem_plan<T>(p);
        void* args[] = {&v, &sp};
        const void* kern = variant == 2 ? (const void*)persistent_smem_kernel<T, true>
                                        : (const void*)persistent_smem_kernel<T, false>;
        OPF_CUDA(cudaLaunchCooperativeKernel(kern, dim3(p->pk.nblocks), dim3(kXWarps * 32), args, (size_t)sp.total, s));
    } else if (variant == 1) {
        void* args[] = {&v};
        OPF_CUDA(cudaLaunchCooperativeKernel((const void*)persistent_kernel<T>, dim3(p->pk.nblocks),
                                             dim3(kXWarps * 32), args, persistent_smem<T>(p), s));
    } else {
        throw Error(OPF_ERR_INVALID_ARG, "persistent engine: the chunks do not fit co-resident on this device");
    }
}

template <typename T>
void run_solve(opf_problem* p, const opf_params& prm, cudaStream_t s) {
    int engine = prm.engine;
    const int form = prm.residual_form;
    if (engine == OPF_ENGINE_AUTO)
        engine = (form == OPF_RES_PAPER && persistent_fits<T>(p)) ? OPF_ENGINE_PERSISTENT : OPF_ENGINE_GRAPH;
    if (engine == OPF_ENGINE_PERSISTENT && form != OPF_RES_PAPER)
        throw Error(OPF_ERR_INVALID_ARG, "persistent engine: only the paper's residual form (OPF_RES_PAPER)");
    if (engine == OPF_ENGINE_PERSISTENT) {
        if (!persistent_fits<T>(p))
            throw Error(OPF_ERR_INVALID_ARG, "persistent engine: the chunks do not fit co-resident on this device");
        launch_persistent<T>(p, s);
        OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaStreamSynchronize(s));
    } else if (engine == OPF_ENGINE_GRAPH) {
        GraphEntry& g = get_graph<T>(p, prm.check_every, form);
        OPF_CUDA(cudaGraphLaunch(g.exec, s));
        OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaStreamSynchronize(s));
    } else {
        for (;;) {
            enqueue_iterations<T>(p, prm.check_every, form, s, 0, 0);
            OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            OPF_CUDA(cudaStreamSynchronize(s));
            if (p->ctl_host->stop) break;
        }
    }
    if (p->ctl_host->status == CTL_TIMEOUT) return;
    objective_kernel<T><<<1, 256, 0, s>>>(view_of<T>(p, prec_of<T>(p)));
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

template <typename T>
double time_graph(opf_problem* p, int which, int reps, cudaStream_t s) {
    View<T> v = view_of<T>(p, prec_of<T>(p));
    const XtGrid xg = xt_grid<T>(p->xt_nitems, p->pk.nblocks);
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    OPF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < reps; ++r) {
        if (which == 0) z_kernel<T><<<zb_blocks(p->pk.ng), kZThreads, 0, cs>>>(v, 0);
        else if (which == 1)
            xt_kernel<T><<<xg.ntl + xg.nchk, kXWarps * 32, kXtSmem, cs>>>(
                device_view<T>(p), static_cast<const TileItem*>(p->xt_items), p->xt_nitems, xg.ntl, 1, 0);
        else if (which == 2) x_kernel<T><<<p->pk.nblocks, kXWarps * 32, 0, cs>>>(v, 0);
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

size_t device_bytes(const opf_problem* p) { return layout_of(p).total; }

int device_auto_engine(const opf_problem* p, int precision) {
    DeviceGuard g(p->device);
    const bool ok = precision == OPF_FP64 ? persistent_fits<double>(p) : persistent_fits<float>(p);
    return ok ? OPF_ENGINE_PERSISTENT : OPF_ENGINE_GRAPH;
}

void device_upload(opf_problem* p, void* arena, size_t bytes, cudaStream_t s) {
    if (p->uploaded) throw Error(OPF_ERR_STATE, "problem already uploaded");
    const Layout L = layout_of(p);
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
    char* a = p->arena;
    const Packed& k = p->pk;
    p->d64.lo = a + L.lo; p->d64.hi = a + L.hi; p->d64.invk = a + L.invk; p->d64.cik = a + L.cik; p->d64.zg = a + L.zg;
    p->d32.lo = a + L.lo32; p->d32.hi = a + L.hi32; p->d32.invk = a + L.invk32; p->d32.cik = a + L.cik32; p->d32.zg = a + L.zg32;
    p->d64.xl = a + L.xl; p->d64.lam = a + L.lam; p->d64.xl2 = a + L.xl2; p->d64.lam2 = a + L.lam2;
    p->d64.bbar = a + L.bbar; p->d64.xl0 = a + L.xl0; p->d64.P = a + L.P64;
    p->d32.xl = a + L.xl32; p->d32.lam = a + L.lam32; p->d32.xl2 = a + L.xl2_32; p->d32.lam2 = a + L.lam2_32;
    p->d32.bbar = a + L.bbar32; p->d32.xl0 = a + L.xl0_32; p->d32.P = a + L.P32;
    p->gptr = (int32_t*)(a + L.gptr); p->gcol = (int32_t*)(a + L.gcol); p->gidx = (int32_t*)(a + L.gidx);
    p->meta = (int32_t*)(a + L.meta); p->tiles = (Tile*)(a + L.tiles); p->blocks = (BlockInfo*)(a + L.blocks);
    p->halo_gid = (int32_t*)(a + L.halo_gid); p->halo_own = (uint8_t*)(a + L.halo_own);
    p->nbrs = (int32_t*)(a + L.nbrs); p->flags = (int32_t*)(a + L.flags);
    p->hcp = (int32_t*)(a + L.hcp); p->hci = (int32_t*)(a + L.hci);
    p->hcx = (int32_t*)(a + L.hcx); p->ext = (int32_t*)(a + L.ext);
    p->cost = (double*)(a + L.cost); p->partials = (double*)(a + L.partials);
    p->phase = (unsigned long long*)(a + L.phase);
    p->mbox = (unsigned long long*)(a + L.mbox);
    p->tdz = (double*)(a + L.tdz);
    p->tpart = (double*)(a + L.tpart);
    p->xt_views = a + L.xtv;
    p->xt_items = a + L.xti;
    p->xt_nitems = (int)((k.tiles.size() + kItemTiles - 1) / kItemTiles);
    p->ctl = (Ctl*)(a + L.ctl);
    if (!p->ctl_host) OPF_CUDA(cudaMallocHost((void**)&p->ctl_host, sizeof(Ctl)));
    std::memset(p->ctl_host, 0, sizeof(Ctl));
    p->ctl_host->first_rel = -1;                 // mirror of the state init_kernel leaves

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
    h2d(p->meta, k.meta.data(), k.nl * 4);
    h2d(p->tiles, k.tiles.data(), k.tiles.size() * sizeof(Tile));
    h2d(p->blocks, k.blocks.data(), k.blocks.size() * sizeof(BlockInfo));
    h2d(p->halo_gid, k.halo_gid.data(), k.halo_gid.size() * 4);
    h2d(p->halo_own, k.halo_own.data(), k.halo_own.size());
    h2d(p->nbrs, k.nbrs.data(), k.nbrs.size() * 4);
    h2d(p->hcp, k.hcp.data(), k.hcp.size() * 4);
    h2d(p->hci, k.hci.data(), k.hci.size() * 4);
    h2d(p->hcx, k.hcx.data(), k.hcx.size() * 4);
    h2d(p->ext, k.ext.data(), k.ext.size() * 4);
    h2d(p->cost, M.c.data(), k.ng * 8);
    h2d(p->d64.bbar, k.bbar.data(), k.nl * 8); h2d(p->d64.xl0, k.xl0.data(), k.nl * 8);
    h2d32(p->d32.bbar, k.bbar); h2d32(p->d32.xl0, k.xl0);
    OPF_CUDA(cudaMemsetAsync(a + L.P64, 0, (k.mat_elems + 8) * 8, s));
    OPF_CUDA(cudaMemsetAsync(a + L.P32, 0, (k.mat_elems + 8) * 4, s));
    h2d(p->d64.P, k.P.data(), k.mat_elems * 8);
    h2d32(p->d32.P, k.P);
    OPF_CUDA(cudaMemsetAsync(p->partials, 0, (size_t)k.nblocks * 16 * sizeof(double), s));
    OPF_CUDA(cudaMemsetAsync(p->flags, 0, (size_t)k.nblocks * sizeof(int32_t), s));
    OPF_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), s));
    // the graph engine's tile-parallel kernel reads the View from the device
    static_assert(sizeof(View<float>) == sizeof(View<double>), "view slots");
    const View<double> vd = view_of<double>(p, p->d64);
    const View<float> vf = view_of<float>(p, p->d32);
    std::vector<TileItem> items;
    for (int t0 = 0; t0 < (int)k.tiles.size(); t0 += kItemTiles)
        items.push_back(TileItem{0, t0, std::min((int)k.tiles.size(), t0 + kItemTiles), 0});
    h2d(p->xt_views, &vf, sizeof(vf));
    h2d((char*)p->xt_views + sizeof(View<double>), &vd, sizeof(vd));
    h2d(p->xt_items, items.data(), items.size() * sizeof(TileItem));
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
    OPF_CUDA(cudaMemcpyAsync(p->ctl_host, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    Ctl c = *p->ctl_host;
    c.rho = prm.rho; c.inv_rho = 1.0 / prm.rho;
    c.eps_abs_prim = prm.eps_abs_prim; c.eps_abs_dual = prm.eps_abs_dual; c.eps_rel = prm.eps_rel;
    c.criterion = prm.criterion; c.K = prm.check_every;
    const long long mi = (long long)c.iter + prm.max_iter;
    c.max_iter = (int32_t)(mi > INT32_MAX ? INT32_MAX : mi);
    c.status = CTL_RUNNING; c.stop = 0;
    c.arrive = 0; c.decided = 0; c.abort = 0; c.halt = 0; c.timeout_where = 0;
    c.timeout_ns = p->timeout_ns; c.skip_block = p->skip_block;
    c.adaptive = prm.adaptive_rho; c.rb_mu = prm.rb_mu; c.rb_tau = prm.rb_tau; c.rho_changes = 0;
    c.profile_phases = p->profile_phases;
    c.res_form = prm.residual_form;
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
    else if (r.status == CTL_TIMEOUT) st = OPF_ERR_TIMEOUT;
    else if (prm.criterion == OPF_CRIT_NEVER && r.status == CTL_MAXITER) st = OPF_OK;
    if (info) {
        info->status = st;
        info->iters = r.iter;
        info->first_rel_iter = r.first_rel;
        info->pres = r.pres; info->dres = r.dres; info->eps_prim = r.eps_prim; info->eps_dual = r.eps_dual;
        info->objective = r.objective;
        info->rho = r.rho;
        info->rho_changes = r.rho_changes;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (st == OPF_ERR_TIMEOUT)
        throw Error(OPF_ERR_TIMEOUT, "persistent engine: a bounded wait expired (site " +
                                         std::to_string(r.timeout_where) + "); the iterate is undefined");
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
    c.rho = prm.rho; c.inv_rho = 1.0 / prm.rho; c.max_iter = INT32_MAX;
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

namespace {

// Control block for a solve: parameters from prm, iteration state from the
// host mirror (kept current after every synchronizing call).
Ctl solve_ctl(const opf_problem* p, const opf_params& prm, const Ctl& cur) {
    Ctl c = cur;
    c.rho = prm.rho; c.inv_rho = 1.0 / prm.rho;
    c.eps_abs_prim = prm.eps_abs_prim; c.eps_abs_dual = prm.eps_abs_dual; c.eps_rel = prm.eps_rel;
    c.criterion = prm.criterion; c.K = prm.check_every;
    const long long mi = (long long)c.iter + prm.max_iter;
    c.max_iter = (int32_t)(mi > INT32_MAX ? INT32_MAX : mi);
    c.status = CTL_RUNNING; c.stop = 0;
    c.arrive = 0; c.decided = 0; c.abort = 0; c.halt = 0; c.timeout_where = 0;
    c.timeout_ns = p->timeout_ns; c.skip_block = p->skip_block;
    c.adaptive = prm.adaptive_rho; c.rb_mu = prm.rb_mu; c.rb_tau = prm.rb_tau; c.rho_changes = 0;
    c.res_form = OPF_RES_PAPER;
    return c;
}

int32_t status_of(const Ctl& r, const opf_params& prm) {
    if (r.status == CTL_CONVERGED) return OPF_OK;
    if (r.status == CTL_NUMERIC) return OPF_ERR_NUMERIC;
    if (r.status == CTL_TIMEOUT) return OPF_ERR_TIMEOUT;
    if (prm.criterion == OPF_CRIT_NEVER && r.status == CTL_MAXITER) return OPF_OK;
    return OPF_NOT_CONVERGED;
}

// The batched graph engine's graph: a while node whose body runs K
// iterations of every instance (global then local update, one launch each
// over all instances), the per-instance checks, and sets the condition to
// "some instance still runs".
template <typename T>
GraphEntry build_batch_graph(const View<T>* dviews, const CtaMap* dmap, const ZMap* dzmap, const TileItem* ditems,
                             int* drun, int n, int nz, int nx, int nitems, int K) {
    const XtGrid xg = xt_grid<T>(nitems, nx);
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
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    OPF_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // iterations without partials on the tile-parallel kernel, the body's
    // last (the check) on the chunk kernel
    for (int q = 0; q < K; ++q) {
        zb_kernel<T><<<nz, kZThreads, 0, cs>>>(dviews, dzmap, q);
        if (q < K - 1)
            xt_kernel<T><<<xg.ntl + xg.nchk, kXWarps * 32, kXtSmem, cs>>>(dviews, ditems, nitems, xg.ntl, n, q);
        else
            xb_kernel<T><<<nx, kXWarps * 32, 0, cs>>>(dviews, dmap, q);
    }
    finb_kernel<T><<<n, kFinThreads, 0, cs>>>(dviews, drun);
    batch_cond_kernel<<<1, 1, 0, cs>>>(drun, h);
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t captured;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (le != cudaSuccess || ee != cudaSuccess)
        throw Error(OPF_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ee));
    OPF_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    return g;
}

// Enqueue a batch solve on `s` without waiting: initial points, control
// blocks built from each problem's host mirror, flags cleared, the
// iterations (one cooperative persistent launch, or the batched graph
// engine's while-node graph), objectives and a single read-back of all
// control blocks into pinned memory; B->done is recorded at the end.
// Engine that OPF_ENGINE_AUTO runs for a batch: persistent when every
// chunk fits co-resident, unless the chunks fit only with their iterate in
// global memory and what one iteration touches in this precision (vectors,
// index lists and the padded operators) is larger than L2 -- then the
// operators stream from HBM and the graph engine (full occupancy, no
// neighbour waits, tile-parallel local update) is the faster one.  On B300,
// feeders of 100-2500 buses, feeder-iterations/s persistent / graph: 16
// feeders (37 MB per iteration) 1.10M / 0.56M, 32 (72 MB) 1.23M / 0.96M,
// 64 (156 MB) 0.93M / 0.95M, 128 (312 MB) 0.88M / 1.17M, 256 (634 MB)
// 0.67M / 1.21M.
template <typename T>
int batch_auto_engine(const opf_batch* B) {
    int nctas = 0;
    ChunkMax cm;
    size_t batch_bytes = 0;
    for (opf_problem* p : B->probs) {
        nctas += p->pk.nblocks;
        cm.add(p->pk);
        const size_t nl = (size_t)p->pk.nl, ng = (size_t)p->pk.ng;
        batch_bytes += sizeof(T) * (7 * nl + 6 * ng + (size_t)p->pk.mat_elems) + 4 * (2 * nl + ng);
    }
    const SmemPlan sp = smem_plan_of<T>(cm);
    const size_t gsmem = (size_t)std::max(1, cm.halo) * sizeof(T);
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        l2 = 0;
    }
    if (coop_fits(batch_smem_kernel<T>, (size_t)sp.total, nctas)) return OPF_ENGINE_PERSISTENT;
    if (coop_fits(batch_global_kernel<T>, gsmem, nctas) && (l2 <= 0 || batch_bytes <= (size_t)l2))
        return OPF_ENGINE_PERSISTENT;
    return OPF_ENGINE_GRAPH;
}

// Byte offsets of a batch's descriptors in its device buffer and in the
// pinned staging copy: control read-back, views, CTA map, global-update
// map, running counter, claim words; 256-byte aligned slices.
struct BatchOffsets {
    size_t ctl, views, map, zmap, run, claim, items, bytes;
};
template <typename T>
BatchOffsets batch_offsets(int n, int nctas, int nz, int nitems) {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    BatchOffsets o;
    o.ctl = 0;
    o.views = up((size_t)n * sizeof(Ctl));
    o.map = o.views + up((size_t)n * sizeof(View<T>));
    o.zmap = o.map + up((size_t)nctas * sizeof(CtaMap));
    o.run = o.zmap + up((size_t)std::max(1, nz) * sizeof(ZMap));
    o.claim = o.run + 256;                                  // zeroed claim words, one per CTA
    o.items = o.claim + up((size_t)nctas * sizeof(int32_t));
    o.bytes = o.items + up((size_t)std::max(1, nitems) * sizeof(TileItem));
    return o;
}

template <typename T>
void batch_launch(opf_batch* B, const opf_params* prm, int nprm, cudaStream_t s) {
    const int n = (int)B->probs.size();
    const size_t ctl_off = 0;
    const size_t views_off = batch_offsets<T>(n, 0, 0, 0).views;
    int nctas = 0, nz = 0, nitems = 0;
    ChunkMax cm;
    for (opf_problem* p : B->probs) {
        nctas += p->pk.nblocks;
        nz += zb_blocks(p->pk.ng);
        nitems += ((int)p->pk.tiles.size() + kItemTiles - 1) / kItemTiles;
        cm.add(p->pk);
    }
    const BatchOffsets bo = batch_offsets<T>(n, nctas, nz, nitems);
    const size_t map_off = bo.map, zmap_off = bo.zmap, run_off = bo.run, claim_off = bo.claim, bytes = bo.bytes;
    if (bytes > B->dev_bytes) {
        if (B->dev_buf) OPF_CUDA(cudaFreeAsync(B->dev_buf, s));
        B->dev_buf = nullptr;
        OPF_CUDA(cudaMallocAsync(&B->dev_buf, bytes, s));
        B->dev_bytes = bytes;
    }
    if (bytes > B->host_bytes) {
        OPF_CUDA(cudaStreamSynchronize(s));
        if (B->host_buf) cudaFreeHost(B->host_buf);
        B->host_buf = nullptr;
        OPF_CUDA(cudaMallocHost((void**)&B->host_buf, bytes));
        B->host_bytes = bytes;
    }
    if (!B->done) OPF_CUDA(cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming));
    Ctl* hctl = reinterpret_cast<Ctl*>(B->host_buf + ctl_off);
    View<T>* hviews = reinterpret_cast<View<T>*>(B->host_buf + views_off);
    CtaMap* hmap = reinterpret_cast<CtaMap*>(B->host_buf + map_off);
    ZMap* hzmap = reinterpret_cast<ZMap*>(B->host_buf + zmap_off);
    int* hrun = reinterpret_cast<int*>(B->host_buf + run_off);
    SmemPlan sp = smem_plan_of<T>(cm);
    const size_t gsmem = (size_t)std::max(1, cm.halo) * sizeof(T);
    int engine = prm[0].engine;
    if (engine == OPF_ENGINE_HOSTLOOP) engine = OPF_ENGINE_GRAPH;
    if (engine == OPF_ENGINE_AUTO) engine = batch_auto_engine<T>(B);
    if (engine == OPF_ENGINE_GRAPH)
        for (int i = 0; i < nprm; ++i)
            if (prm[i].check_every != prm[0].check_every)
                throw Error(OPF_ERR_INVALID_ARG, "batch graph engine: every instance needs the same check_every");
    const int prec = sizeof(T) == 8 ? OPF_FP64 : OPF_FP32;
    int c = 0, cz = 0, running = 0;
    for (int i = 0; i < n; ++i) {
        opf_problem* p = B->probs[i];
        const opf_params& pr = prm[nprm == 1 ? 0 : i];
        Ctl cur = *p->ctl_host;
        if (!pr.warm_start) {
            enqueue_init<T>(p, s);
            p->cur_prec = prec;
            cur.iter = 0; cur.first_rel = -1; cur.checks = 0;
            cur.pres = cur.dres = cur.eps_prim = cur.eps_dual = NAN;
        } else {
            sync_state_to(p, prec, s);
        }
        hctl[i] = solve_ctl(p, pr, cur);
        if (pr.max_iter > 0) ++running;
        else if (engine == OPF_ENGINE_GRAPH) hctl[i].stop = 1;   // nothing to do: skipped by the graph body
        hviews[i] = view_of<T>(p, prec_of<T>(p));
        for (int b = 0; b < p->pk.nblocks; ++b) hmap[c++] = CtaMap{i, b};
        for (int g0 = 0; g0 < p->pk.ng; g0 += kZThreads * kZPer) hzmap[cz++] = ZMap{i, g0};
    }
    *hrun = running;
    std::memset(B->host_buf + claim_off, 0, bytes - claim_off);
    TileItem* hitems = reinterpret_cast<TileItem*>(B->host_buf + bo.items);
    for (int i = 0, k = 0; i < n; ++i) {
        const int nt = (int)B->probs[i]->pk.tiles.size();
        for (int t0 = 0; t0 < nt; t0 += kItemTiles) hitems[k++] = TileItem{i, t0, std::min(nt, t0 + kItemTiles), 0};
    }
    for (int i = 0; i < n; ++i)
        OPF_CUDA(cudaMemcpyAsync(B->probs[i]->ctl, hctl + i, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    char* d = static_cast<char*>(B->dev_buf);
    OPF_CUDA(cudaMemcpyAsync(d + views_off, B->host_buf + views_off, bytes - views_off, cudaMemcpyHostToDevice, s));
    const View<T>* dviews = reinterpret_cast<const View<T>*>(d + views_off);
    const CtaMap* dmap = reinterpret_cast<const CtaMap*>(d + map_off);
    const ZMap* dzmap = reinterpret_cast<const ZMap*>(d + zmap_off);
    int* drun = reinterpret_cast<int*>(d + run_off);
    int32_t* dclaim = reinterpret_cast<int32_t*>(d + claim_off);
    Ctl* dctl = reinterpret_cast<Ctl*>(d + ctl_off);
    const bool smem_var = engine == OPF_ENGINE_PERSISTENT && coop_fits(batch_smem_kernel<T>, (size_t)sp.total, nctas);
    if (running > 0 && engine == OPF_ENGINE_PERSISTENT) {
        // One persistent launch for the whole batch, captured once into a
        // CUDA graph (flag clear, cooperative kernel, per-instance finish)
        // and launched again while the batch layout, precision and kernel
        // plan are unchanged; the per-solve control blocks and descriptors
        // are copied in before it (same device addresses).
        const int variant = smem_var ? 2 : (coop_fits(batch_global_kernel<T>, gsmem, nctas) ? 1 : 0);
        if (!variant)
            throw Error(OPF_ERR_INVALID_ARG, "batch: " + std::to_string(nctas) +
                                                 " chunks do not fit co-resident; create the problems with fewer"
                                                 " chunks or use the graph engine");
        static_assert(sizeof(SmemPlan) <= sizeof(B->p_plan), "plan key");
        unsigned char plan[sizeof(B->p_plan)] = {};
        std::memcpy(plan, &sp, sizeof(SmemPlan));
        if (!B->pexec || B->p_buf != B->dev_buf || B->p_n != n || B->p_nx != nctas || B->p_nz != nz || B->p_prec != prec ||
            B->p_var != variant || std::memcmp(plan, B->p_plan, sizeof(plan)) != 0) {
            if (B->pexec) cudaGraphExecDestroy(B->pexec);
            if (B->pgraph) cudaGraphDestroy(B->pgraph);
            B->pexec = nullptr;
            B->pgraph = nullptr;
            cudaStream_t cs;
            OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            OPF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            batch_clear_flags<T><<<std::min(n, 1024), 256, 0, cs>>>(dviews, n, smem_var ? 1 : 0);
            cudaLaunchConfig_t lc = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            lc.gridDim = dim3(nctas);
            lc.blockDim = dim3(kXWarps * 32);
            lc.stream = cs;
            lc.attrs = at;
            lc.numAttrs = 1;
            if (variant == 2) {
                int per = resident_per_sm(batch_smem_kernel<T>, (size_t)sp.total);
                void* args[] = {&dviews, &dmap, &sp, &dclaim, &per};
                lc.dynamicSmemBytes = (size_t)sp.total;
                ce = cudaLaunchKernelExC(&lc, (const void*)batch_smem_kernel<T>, args);
            } else {
                int per = resident_per_sm(batch_global_kernel<T>, gsmem);
                void* args[] = {&dviews, &dmap, &dclaim, &per};
                lc.dynamicSmemBytes = gsmem;
                ce = cudaLaunchKernelExC(&lc, (const void*)batch_global_kernel<T>, args);
            }
            batch_finish_kernel<T><<<n, 256, 0, cs>>>(dviews, dctl);
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess || ee != cudaSuccess || !g) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw Error(OPF_ERR_CUDA, std::string("batch: capturing the persistent launch failed: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : ee));
            }
            cudaGraphExec_t ge = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(g);
                throw Error(OPF_ERR_CUDA, std::string("batch: instantiating the persistent launch: ") +
                                              cudaGetErrorString(ie));
            }
            B->pgraph = g;
            B->pexec = ge;
            B->p_buf = B->dev_buf; B->p_n = n; B->p_nx = nctas; B->p_nz = nz; B->p_prec = prec; B->p_var = variant;
            std::memcpy(B->p_plan, plan, sizeof(plan));
        }
        OPF_CUDA(cudaGraphLaunch(B->pexec, s));
        OPF_CUDA(cudaMemcpyAsync(hctl, dctl, (size_t)n * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaEventRecord(B->done, s));
        B->n_launched = n;
        return;
    }
    batch_clear_flags<T><<<std::min(n, 1024), 256, 0, s>>>(dviews, n, smem_var ? 1 : 0);
    OPF_CUDA(cudaGetLastError());
    if (running > 0) {
        const int K = prm[0].check_every;
        if (!B->gexec || B->g_buf != B->dev_buf || B->g_n != n || B->g_nz != nz || B->g_nx != nctas || B->g_K != K ||
            B->g_prec != prec || B->g_ni != nitems) {
            if (B->gexec) cudaGraphExecDestroy(B->gexec);
            if (B->graph) cudaGraphDestroy(B->graph);
            B->gexec = nullptr;
            B->graph = nullptr;
            const TileItem* ditems = reinterpret_cast<const TileItem*>(d + bo.items);
            GraphEntry ge = build_batch_graph<T>(dviews, dmap, dzmap, ditems, drun, n, nz, nctas, nitems, K);
            B->graph = ge.graph;
            B->gexec = ge.exec;
            B->g_buf = B->dev_buf; B->g_n = n; B->g_nz = nz; B->g_nx = nctas; B->g_K = K; B->g_prec = prec;
            B->g_ni = nitems;
        }
        OPF_CUDA(cudaGraphLaunch(B->gexec, s));
    }
    batch_finish_kernel<T><<<n, 256, 0, s>>>(dviews, dctl);
    OPF_CUDA(cudaGetLastError());
    OPF_CUDA(cudaMemcpyAsync(hctl, dctl, (size_t)n * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaEventRecord(B->done, s));
    B->n_launched = n;
}

// `reps` back-to-back launches of one kernel of the batched graph body
// (which: 0 global update, 1 tile-parallel local update, 2 chunk local
// update with partials, 3 chunk local update without) in a plain graph;
// microseconds per launch.
template <typename T>
double time_batch_graph(const View<T>* dv, const CtaMap* dm, const ZMap* dz, const TileItem* di, int n, int nz,
                        int nx, int ni, int which, int reps, cudaStream_t s) {
    const XtGrid xg = xt_grid<T>(ni, nx);
    cudaStream_t cs;
    OPF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    OPF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < reps; ++r) {
        if (which == 0) zb_kernel<T><<<nz, kZThreads, 0, cs>>>(dv, dz, 0);
        else if (which == 1) xt_kernel<T><<<xg.ntl + xg.nchk, kXWarps * 32, kXtSmem, cs>>>(dv, di, ni, xg.ntl, n, 0);
        else xb_kernel<T><<<nx, kXWarps * 32, 0, cs>>>(dv, dm, 0);
    }
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        throw Error(OPF_ERR_CUDA, std::string("batch profile capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ee));
    }
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

template <typename T>
void batch_profile(opf_batch* B, const opf_params& prm, int reps, cudaStream_t s, double* us) {
    const int n = (int)B->probs.size();
    const int prec = sizeof(T) == 8 ? OPF_FP64 : OPF_FP32;
    const size_t w = sizeof(T);
    size_t tot = 0;
    for (opf_problem* p : B->probs) {
        sync_state_to(p, prec, s);
        tot += (2 * (size_t)p->pk.nl + (size_t)p->pk.ng) * w;
    }
    // save every instance's iterate, duals, global vector and control block
    char* save = nullptr;
    OPF_CUDA(cudaMallocAsync((void**)&save, tot + (size_t)n * sizeof(Ctl), s));
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        opf_problem* p = B->probs[i];
        const DevPrec& d = prec == OPF_FP64 ? p->d64 : p->d32;
        const size_t nl = p->pk.nl, ng = p->pk.ng;
        OPF_CUDA(cudaMemcpyAsync(save + o, d.xl, nl * w, cudaMemcpyDeviceToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(save + o + nl * w, d.lam, nl * w, cudaMemcpyDeviceToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(save + o + 2 * nl * w, d.zg, ng * w, cudaMemcpyDeviceToDevice, s));
        o += (2 * nl + ng) * w;
        OPF_CUDA(cudaMemcpyAsync(save + tot + (size_t)i * sizeof(Ctl), p->ctl, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
    }
    // a graph-engine launch of zero iterations uploads the views and maps
    opf_params q = prm;
    q.engine = OPF_ENGINE_GRAPH;
    q.max_iter = 0;
    q.warm_start = 1;
    batch_launch<T>(B, &q, 1, s);
    OPF_CUDA(cudaEventSynchronize(B->done));
    int nctas = 0, nz = 0, ni = 0;
    for (opf_problem* p : B->probs) {
        nctas += p->pk.nblocks;
        nz += zb_blocks(p->pk.ng);
        ni += ((int)p->pk.tiles.size() + kItemTiles - 1) / kItemTiles;
    }
    const BatchOffsets bo = batch_offsets<T>(n, nctas, nz, ni);
    char* d = static_cast<char*>(B->dev_buf);
    const View<T>* dv = reinterpret_cast<const View<T>*>(d + bo.views);
    const CtaMap* dm = reinterpret_cast<const CtaMap*>(d + bo.map);
    const ZMap* dz = reinterpret_cast<const ZMap*>(d + bo.zmap);
    const TileItem* di = reinterpret_cast<const TileItem*>(d + bo.items);
    Ctl* hctl = reinterpret_cast<Ctl*>(B->host_buf + bo.ctl);
    // control blocks for timing: nothing skipped (huge bound); K = 1 makes
    // every local-update launch a check iteration (which == 2)
    for (int which = 0; which < 4; ++which) {
        for (int i = 0; i < n; ++i) {
            Ctl& c = hctl[i];
            c.stop = 0;
            c.iter = 0;
            c.max_iter = INT32_MAX;
            c.rho = prm.rho;
            c.inv_rho = 1.0 / prm.rho;
            c.K = (which == 2) ? 1 : (1 << 20);
            OPF_CUDA(cudaMemcpyAsync(B->probs[i]->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        }
        us[which] = time_batch_graph<T>(dv, dm, dz, di, n, nz, nctas, ni, which, reps, s);
    }
    o = 0;
    for (int i = 0; i < n; ++i) {
        opf_problem* p = B->probs[i];
        const DevPrec& dd = prec == OPF_FP64 ? p->d64 : p->d32;
        const size_t nl = p->pk.nl, ng = p->pk.ng;
        OPF_CUDA(cudaMemcpyAsync(dd.xl, save + o, nl * w, cudaMemcpyDeviceToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(dd.lam, save + o + nl * w, nl * w, cudaMemcpyDeviceToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(dd.zg, save + o + 2 * nl * w, ng * w, cudaMemcpyDeviceToDevice, s));
        o += (2 * nl + ng) * w;
        OPF_CUDA(cudaMemcpyAsync(p->ctl, save + tot + (size_t)i * sizeof(Ctl), sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
    }
    OPF_CUDA(cudaFreeAsync(save, s));
    OPF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

// Wait for the batch launched last and publish each instance's outcome.
void device_batch_collect(opf_batch* B, const opf_params* prm, int nprm, opf_info* infos) {
    DeviceGuard g(B->device);
    OPF_CUDA(cudaEventSynchronize(B->done));
    const int n = B->n_launched;
    const Ctl* hctl = reinterpret_cast<const Ctl*>(B->host_buf);
    for (int i = 0; i < n; ++i) {
        opf_problem* p = B->probs[i];
        *p->ctl_host = hctl[i];
        p->cold = false;
        const Ctl& r = hctl[i];
        if (infos) {
            opf_info& in = infos[i];
            in.status = status_of(r, prm[nprm == 1 ? 0 : i]);
            in.iters = r.iter;
            in.first_rel_iter = r.first_rel;
            in.pres = r.pres; in.dres = r.dres; in.eps_prim = r.eps_prim; in.eps_dual = r.eps_dual;
            in.objective = r.objective;
            in.rho = r.rho;
            in.rho_changes = r.rho_changes;
            in.seconds = 0;
        }
    }
    for (int i = 0; i < n; ++i)
        if (hctl[i].status == CTL_TIMEOUT)
            throw Error(OPF_ERR_TIMEOUT, "batch: instance " + std::to_string(i) + " hit a bounded-wait limit");
}

void device_batch_launch(opf_batch* B, const opf_params* prm, int nprm, cudaStream_t s) {
    DeviceGuard g(B->device);
    if (prm[0].precision == OPF_FP64) batch_launch<double>(B, prm, nprm, s);
    else batch_launch<float>(B, prm, nprm, s);
}

namespace {
}  // namespace

void device_batch_solve(opf_batch* B, const opf_params* prm, int nprm, cudaStream_t s, opf_info* infos) {
    DeviceGuard g(B->device);
    auto t0 = std::chrono::steady_clock::now();
    device_batch_launch(B, prm, nprm, s);
    device_batch_collect(B, prm, nprm, infos);
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (infos)
        for (size_t i = 0; i < B->probs.size(); ++i) infos[i].seconds = sec;
}

void device_batch_profile(opf_batch* B, const opf_params& prm, int reps, cudaStream_t s, double* us) {
    DeviceGuard g(B->device);
    if (prm.precision == OPF_FP64) batch_profile<double>(B, prm, reps, s, us);
    else batch_profile<float>(B, prm, reps, s, us);
}

// Co-resident CTAs a batch launch can use on the current device (the
// global-memory kernel with its smallest shared-memory footprint).
int device_batch_auto_engine(const opf_batch* B, int precision) {
    DeviceGuard g(B->device);
    return precision == OPF_FP64 ? batch_auto_engine<double>(B) : batch_auto_engine<float>(B);
}

int device_batch_capacity(int precision) {
    int dev = 0, sms = 0, per_sm = 0;
    OPF_CUDA(cudaGetDevice(&dev));
    OPF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = 4096;
    if (precision == OPF_FP64)
        OPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_global_kernel<double>, kXWarps * 32, smem));
    else
        OPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_global_kernel<float>, kXWarps * 32, smem));
    return per_sm * sms;
}

void device_batch_free(opf_batch* B) {
    DeviceGuard g(B->device);
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->gexec = nullptr;
    B->graph = nullptr;
    if (B->pexec) cudaGraphExecDestroy(B->pexec);
    if (B->pgraph) cudaGraphDestroy(B->pgraph);
    B->pexec = nullptr;
    B->pgraph = nullptr;
    if (B->done) cudaEventDestroy(B->done);
    B->done = nullptr;
    if (B->dev_buf) cudaFree(B->dev_buf);
    if (B->host_buf) cudaFreeHost(B->host_buf);
    B->dev_buf = nullptr;
    B->host_buf = nullptr;
}

// Copy the old problem's iterate into the new one where the local copies
// correspond (map built by the caller, device order of the new problem, old
// device indices).  Both problems on the same device; runs on `s`.
void device_warm_transfer(opf_problem* dst, const opf_problem* src, const std::vector<int32_t>& map, cudaStream_t s) {
    DeviceGuard g(dst->device);
    const int prec = src->cur_prec;
    const int n = dst->pk.nl;
    if ((int)map.size() != n) throw Error(OPF_ERR_INVALID_ARG, "warm map size");
    int32_t* dmap = nullptr;
    OPF_CUDA(cudaMallocAsync((void**)&dmap, sizeof(int32_t) * std::max(1, n), s));
    OPF_CUDA(cudaMemcpyAsync(dmap, map.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    // the new problem starts from its initial point in the old one's precision
    if (prec == OPF_FP64) enqueue_init<double>(dst, s);
    else enqueue_init<float>(dst, s);
    const DevPrec& sd = prec == OPF_FP64 ? src->d64 : src->d32;
    const DevPrec& dd = prec == OPF_FP64 ? dst->d64 : dst->d32;
    if (n > 0) {
        if (prec == OPF_FP64)
            warm_gather_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(dmap, (const double*)sd.xl, (const double*)sd.lam,
                                                                      (double*)dd.xl, (double*)dd.lam, n);
        else
            warm_gather_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(dmap, (const float*)sd.xl, (const float*)sd.lam,
                                                                     (float*)dd.xl, (float*)dd.lam, n);
        OPF_CUDA(cudaGetLastError());
    }
    OPF_CUDA(cudaFreeAsync(dmap, s));
    dst->cur_prec = prec;
    dst->cold = false;
    Ctl& m = *dst->ctl_host;
    m.iter = 0; m.first_rel = -1; m.checks = 0;
}

// Per-iteration time of each phase of the shared-memory persistent kernel,
// mean and max over CTAs: a solve of `iters` iterations from the initial
// point with the phase counters on.
void device_profile_persistent(opf_problem* p, const opf_params& prm, int iters, cudaStream_t s, double* out,
                               double* per_cta) {
    DeviceGuard g(p->device);
    opf_params q = prm;
    q.warm_start = 0;
    q.criterion = OPF_CRIT_NEVER;
    q.max_iter = iters;
    q.engine = OPF_ENGINE_PERSISTENT;
    const int saved = p->force_variant;
    p->force_variant = 2;
    p->profile_phases = 1;
    try {
        device_solve(p, q, s, nullptr);
    } catch (...) {
        p->force_variant = saved;
        p->profile_phases = 0;
        throw;
    }
    p->force_variant = saved;
    p->profile_phases = 0;
    const int nb = p->pk.nblocks;
    std::vector<unsigned long long> h((size_t)nb * 4);
    OPF_CUDA(cudaMemcpyAsync(h.data(), p->phase, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    OPF_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 4; ++k) {
        double sum = 0, mx = 0;
        for (int b = 0; b < nb; ++b) {
            const double us = 1e-3 * (double)h[(size_t)b * 4 + k] / iters;
            if (per_cta) per_cta[(size_t)b * 4 + k] = us;
            sum += us;
            mx = std::max(mx, us);
        }
        out[k] = sum / nb;
        out[4 + k] = mx;
    }
}

// Recompute the operators of components `comps` (whose A, b in p->model were
// updated) on the device and refresh the host copies in p->ops.
void device_reprecompute(opf_problem* p, const std::vector<int>& comps, cudaStream_t s) {
    if (comps.empty()) return;
    DeviceGuard g(p->device);
    const Packed& K = p->pk;
    std::vector<RpDesc> ds;
    std::vector<double> A, b;
    int32_t out = 0, wo = 0;
    for (int c : comps) {
        const Component& C = p->model.comps[c];
        const int n = C.n(), m = C.m;
        if (n == 0 || K.comp_tile[c] < 0) continue;
        if (m == 0) throw Error(OPF_ERR_INVALID_ARG, "component without rows");
        const Tile& t = K.tiles[K.comp_tile[c]];
        const int32_t loc0 = K.dev_of_canon[p->canon_comp_ptr[c]];
        RpDesc d{};
        d.m = m; d.n = n;
        d.aoff = (int32_t)A.size(); d.boff = (int32_t)b.size();
        d.mat0 = t.mat0; d.L = t.L; d.big = t.big;
        d.base = t.big ? 0 : (K.meta[loc0] >> 24) & 0x1F;
        d.loc0 = loc0;
        d.outoff = out; out += n * n + n;
        d.woff = wo; wo += m * m + m * n + m;
        A.insert(A.end(), C.A.begin(), C.A.end());
        b.insert(b.end(), C.b.begin(), C.b.end());
        ds.push_back(d);
    }
    if (ds.empty()) return;
    const size_t bd = ds.size() * sizeof(RpDesc), ba = A.size() * 8, bb = b.size() * 8;
    const size_t bs = (size_t)wo * 8, bo = (size_t)out * 8;
    const size_t o_d = 0, o_a = (bd + 255) & ~size_t(255), o_b = o_a + ((ba + 255) & ~size_t(255));
    const size_t o_s = o_b + ((bb + 255) & ~size_t(255)), o_o = o_s + ((bs + 255) & ~size_t(255));
    const size_t o_e = o_o + ((bo + 255) & ~size_t(255)), total = o_e + 256;
    char* buf = nullptr;
    OPF_CUDA(cudaMallocAsync((void**)&buf, total, s));
    std::vector<double> hout(out);
    int herr = 0;
    try {
        OPF_CUDA(cudaMemcpyAsync(buf + o_d, ds.data(), bd, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(buf + o_a, A.data(), ba, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemcpyAsync(buf + o_b, b.data(), bb, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemsetAsync(buf + o_e, 0, sizeof(int), s));
        reprecompute_kernel<<<(unsigned)ds.size(), 32, 0, s>>>(
            (const RpDesc*)(buf + o_d), (const double*)(buf + o_a), (const double*)(buf + o_b), (double*)(buf + o_s),
            (double*)p->d64.P, (float*)p->d32.P, (double*)p->d64.bbar, (float*)p->d32.bbar, (double*)(buf + o_o),
            (int*)(buf + o_e));
        OPF_CUDA(cudaGetLastError());
        OPF_CUDA(cudaMemcpyAsync(hout.data(), buf + o_o, bo, cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaMemcpyAsync(&herr, buf + o_e, sizeof(int), cudaMemcpyDeviceToHost, s));
        OPF_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFreeAsync(buf, s);
        throw;
    }
    OPF_CUDA(cudaFreeAsync(buf, s));
    if (herr) throw Error(OPF_ERR_NUMERIC, "re-precompute: a component's rows are rank deficient");
    size_t k = 0;
    for (int c : comps) {
        const Component& C = p->model.comps[c];
        if (C.n() == 0 || K.comp_tile[c] < 0) continue;
        const RpDesc& d = ds[k++];
        Operator& op = p->ops[c];
        op.n = d.n;
        op.P.assign(hout.begin() + d.outoff, hout.begin() + d.outoff + (size_t)d.n * d.n);
        op.bbar.assign(hout.begin() + d.outoff + (size_t)d.n * d.n, hout.begin() + d.outoff + (size_t)d.n * d.n + d.n);
        op.m_reduced = d.m;
    }
}

// Upload the bounds of the global ranges [g0, g1) from p->model to both
// precisions (one synchronization for all).
void device_update_bounds(opf_problem* p, const std::vector<std::pair<int, int>>& ranges, cudaStream_t s) {
    if (ranges.empty()) return;
    DeviceGuard g(p->device);
    const Model& M = p->model;
    std::vector<std::vector<float>> keep;
    for (const auto& r : ranges) {
        const int g0 = r.first, g1 = r.second;
        if (g1 <= g0) continue;
        const size_t n = (size_t)(g1 - g0);
        keep.emplace_back(2 * n);
        std::vector<float>& f = keep.back();
        for (size_t i = 0; i < n; ++i) {
            f[i] = (float)M.lo[g0 + i];
            f[n + i] = (float)M.hi[g0 + i];
        }
        OPF_CUDA(cudaMemcpyAsync((double*)p->d64.lo + g0, M.lo.data() + g0, n * 8, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemcpyAsync((double*)p->d64.hi + g0, M.hi.data() + g0, n * 8, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemcpyAsync((float*)p->d32.lo + g0, f.data(), n * 4, cudaMemcpyHostToDevice, s));
        OPF_CUDA(cudaMemcpyAsync((float*)p->d32.hi + g0, f.data() + n, n * 4, cudaMemcpyHostToDevice, s));
    }
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
