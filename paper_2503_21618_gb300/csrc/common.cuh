// Shared device/host helpers of the slrf library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slrf.h"

namespace slrf {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2 (x = real, y = imaginary)
// ---------------------------------------------------------------------------
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a + b * c
template <typename C> __host__ __device__ __forceinline__ C cfma(C b, C c, C a) {
    C r;
    r.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    r.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename C> __host__ __device__ __forceinline__ decltype(C().x) cabs2(C a) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------------------
// kernel classes (profiling buckets of slrf_report)
// ---------------------------------------------------------------------------
enum KernelClass {
    KC_SHIFTED_SPMM = 0,   // K1: (A - sigma_j B) P, fused dot
    KC_KRYLOV_UPDATE = 1,  // K3: COCG x/r update + U accumulation + dots
    KC_KRYLOV_DIR = 2,     // K3: search direction p = z + beta p
    KC_KRYLOV_REDUCE = 3,  // per-column scalar reductions
    KC_KRYLOV_INIT = 4,    // r0, z0, p0
    KC_SPMM_REAL = 5,      // K2: A X, B X in FP64
    KC_GRAM = 6,           // K6: X^T Y
    KC_TALL_GEMM = 7,      // K9: X T (n x m times m x m)
    KC_SMALL_DENSE = 8,    // K7/K8: Cholesky, inverse, small GEMMs, eigensolver
    KC_RESIDUAL = 9,       // residual R = B X Theta - A X and norms
    KC_FILTER_COMBINE = 10,// U = X Phi(Theta) + correction, conversions
    KC_OTHER = 11,
    KC_MG_FINE = 12,       // multigrid: finest-level shifted products (residual, Jacobi sweep)
    KC_MG_TRANSFER = 13,   // multigrid: restriction, prolongation, first sweep
    KC_MG_COARSE = 14,     // multigrid: coarser-level products and the coarsest solve
};

}  // namespace slrf
