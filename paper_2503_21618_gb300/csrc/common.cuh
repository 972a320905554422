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
// packed FP32x2 fused multiply-add: c = a * b + c on both lanes of a float2
// (one instruction for two FMAs: it halves the issue slots of the FP32
// products of the gathered kernels)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ffma2(float2 &c, float2 a, float2 b) {
    unsigned long long cu = (unsigned long long)__float_as_uint(c.x) | ((unsigned long long)__float_as_uint(c.y) << 32);
    const unsigned long long au =
        (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
    const unsigned long long bu =
        (unsigned long long)__float_as_uint(b.x) | ((unsigned long long)__float_as_uint(b.y) << 32);
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(cu) : "l"(au), "l"(bu));
    c.x = __uint_as_float((unsigned)(cu & 0xffffffffu));
    c.y = __uint_as_float((unsigned)(cu >> 32));
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (TMA engine) primitives for shared-memory pipelines
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(void *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(void *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(void *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(void *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity to complete, for at most limit_ns
// nanoseconds; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(void *bar, unsigned parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on the mbarrier's tx count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, void *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// ---- tcgen05 (5th-generation tensor cores) ----------------------------------
// Shared-memory matrix descriptor of a K-major operand without swizzle, in
// the canonical layout of 8 x 16-byte core matrices: 128 B between K-adjacent
// cores (leading offset), 512 B between 8-row groups (stride offset),
// descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t umma_desc(unsigned smem_byte_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_byte_addr >> 4) & 0x3fff);
    d |= (uint64_t)((128u >> 4) & 0x3fff) << 16;
    d |= (uint64_t)((512u >> 4) & 0x3fff) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor: bf16 x bf16 -> FP32, both operands K-major, M x N
// (M = 128: N a multiple of 16 up to 256)
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (TMEM) (+)= A (smem) x B (smem), issued by one thread
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread completes
__device__ __forceinline__ void umma_commit(void *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Prefetch [p, p + bytes) into L2 with bulk prefetches of at most 32 KB, one
// per lane of the calling (converged) warp; p 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void l2_prefetch_warp(const void *p, int64_t bytes, int lane) {
    const char *c = reinterpret_cast<const char *>(p);
    for (int64_t off = (int64_t)lane * 32768; off < bytes; off += 32 * 32768) {
        const unsigned sz = (unsigned)((bytes - off) < 32768 ? (bytes - off) : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(sz) : "memory");
    }
}

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
