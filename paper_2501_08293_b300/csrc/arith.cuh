// The arithmetic of one ADMM iteration (Algorithm 1), written once with
// explicit fused multiply-adds.  The library is built with -fmad=false, so
// nothing else is contracted: every engine and kernel that uses these
// helpers in the same order computes bit-identical iterates.
#pragma once

namespace opf {

// Copy term of the global update, Eq. (global_sparse): x - lambda / rho.
template <typename T>
__device__ __forceinline__ T copy_term(T x, T l, T inv_rho) { return fma(-l, inv_rho, x); }

// Eq. (global_sparse): s / k - c / (rho k), clipped to [lo, hi]
// (invk = 1/k, cik = c/k).
template <typename T>
__device__ __forceinline__ T global_from_sum(T s, T invk, T cik, T inv_rho, T lo, T hi) {
    const T xh = fma(s, invk, -(cik * inv_rho));
    return fmin(fmax(xh, lo), hi);
}

// Operand of the local update, Eq. (closed_2): u = B x + lambda / rho.
template <typename T>
__device__ __forceinline__ T u_of(T v, T l, T inv_rho) { return fma(l, inv_rho, v); }

// Dual update, Eq. (ADMM-3): lambda + rho (B x - x_s).
template <typename T>
__device__ __forceinline__ T dual_of(T l, T rho, T v, T xn) { return fma(rho, v - xn, l); }

}  // namespace opf
