// FP64-accurate Gram G = X^T Y on the integer tensor cores (Ozaki scheme).
//
// FP64 arithmetic on this GPU runs at ~1 TFLOP/s (CUDA cores and the FP64
// tensor path alike, measured), while int8 mma.sync runs at ~150 TOP/s.  The
// Gram of two tall n x m blocks is therefore computed from exact integer
// pieces (error-free splitting, Ozaki et al., Numer. Algorithms 59, 2012):
//
//  * every column a of X is scaled by 2^-e_a, e_a = exponent of max_i |X_ia|
//    plus one, so |X_ia 2^-e_a| < 1/2;
//  * the scaled value is rounded to a fixed-point integer F with 7S fraction
//    bits and cut into S balanced base-128 digits D_s in [-64, 64] (int8):
//    X_ia = 2^e_a sum_s D_s,ia 2^(-7(s+1)) + (rounding below 2^(e_a - 7S - 1));
//  * products of digits are exact in int32 (|D E| <= 2^12; a K-slice of at
//    most 2^19/(d+1) rows keeps every partial sum below 2^31), and all digit
//    pairs with the same s + t = d share one scale, so
//        G_ab = 2^(e_a + f_b) sum_{d < S} 2^(-7(d+2)) sum_{s+t=d} D_s^T E_t;
//  * the int32 sums are converted to FP64 once per (CTA, d) and the K-slices
//    are reduced in a fixed order.
// With S = 7 the truncation error is ~2^-50 relative to max|X_a| max|Y_b| n.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace slrf {

constexpr int OZ_S = 7;          // digits per value
constexpr int OZ_TM = 64;        // CTA output tile (rows a) = (cols b)

// ---------------------------------------------------------------------------
// column exponents: e[a] = ilogb(max_i |X_ia|) + 2 (so |X 2^-e| < 1/2)
// ---------------------------------------------------------------------------
__global__ void k_oz_colmax(int64_t n, int m, const double *__restrict__ X, int64_t ldx,
                            unsigned long long *__restrict__ maxbits) {
    const int a = blockIdx.x * 32 + threadIdx.x;
    if (a >= m) return;
    double mx = 0.0;
    for (int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; i < n; i += (int64_t)gridDim.y * blockDim.y)
        mx = fmax(mx, fabs(X[i * ldx + a]));
    // for non-negative doubles the bit pattern orders like the value
    atomicMax(maxbits + a, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_oz_exponent(int m, const unsigned long long *__restrict__ maxbits, int *__restrict__ e) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    const double mx = __longlong_as_double((long long)maxbits[a]);
    e[a] = mx > 0.0 ? ilogb(mx) + 2 : 0;
}

// ---------------------------------------------------------------------------
// digits: slices[s][a][i] (transposed, row pitch npad bytes), integer-exact
// ---------------------------------------------------------------------------
__device__ __forceinline__ void oz_digits(double x, int e, int8_t d[OZ_S]) {
    // F = round(x 2^(7S - e)) exactly, from the integer significand
    long long F = 0;
    if (x != 0.0) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
        const int ex = (int)((bits >> 52) & 0x7ff);
        unsigned long long mant = bits & ((1ull << 52) - 1);
        int E;
        if (ex == 0) {
            E = -1074;                 // subnormal
        } else {
            mant |= 1ull << 52;
            E = ex - 1075;
        }
        const int sh = E - e + 7 * OZ_S;   // x 2^(7S-e) = mant 2^sh
        unsigned long long mag;
        if (sh >= 0)
            mag = mant << sh;              // |x 2^-e| < 1/2 keeps this below 2^(7S-1)
        else if (sh > -64)
            mag = (mant + (1ull << (-sh - 1))) >> (-sh);
        else
            mag = 0;
        F = (bits >> 63) ? -(long long)mag : (long long)mag;
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        const int k = 7 * (OZ_S - 1 - s);
        long long D;
        if (k > 0)
            D = (F + (1ll << (k - 1))) >> k;   // balanced digit (round half up)
        else
            D = F;
        F -= D << k;
        d[s] = (int8_t)D;
    }
}

__global__ void __launch_bounds__(256)
k_oz_split(int64_t n, int m, int64_t npad, const double *__restrict__ X, int64_t ldx, const int *__restrict__ e,
           int8_t *__restrict__ slices, int mpad) {
    // 32 x 32 tile: read along a (coalesced), write along i (coalesced)
    __shared__ int8_t tile[OZ_S][32][33];
    const int a0 = blockIdx.x * 32, i0base = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int64_t i0 = i0base; i0 < npad; i0 += (int64_t)gridDim.y * 32) {
        for (int r = ty; r < 32; r += 8) {
            const int64_t i = i0 + r;
            const int a = a0 + tx;
            int8_t d[OZ_S];
            const double x = (i < n && a < m) ? X[i * ldx + a] : 0.0;
            oz_digits(x, a < m ? e[a] : 0, d);
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) tile[s][r][tx] = d[s];
        }
        __syncthreads();
        for (int c = ty; c < 32; c += 8) {
            const int a = a0 + c;
            if (a < mpad) {
                const int64_t i = i0 + tx;
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) slices[((int64_t)s * mpad + a) * npad + i] = tile[s][tx][c];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// IMMA Gram of digit slices: work[z][a][b] = sum_d 2^(-7(d+2)) sum_{s+t=d} D_s^T E_t
// over the K-slice z.  CTA = 4 warps, 64 x 64 tile, warp 32 x 32 (2 x 4 mma).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void imma16832(int c[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128)
k_oz_gram(int m, int mpad, int64_t npad, int64_t kslice, const int8_t *__restrict__ SX,
          const int8_t *__restrict__ SY, double *__restrict__ work, int symmetric) {
    // a symmetric Gram needs the tiles on and above the diagonal only
    if (symmetric && blockIdx.y > blockIdx.x) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int a_base = blockIdx.y * OZ_TM + (warp >> 1) * 32;
    const int b_base = blockIdx.x * OZ_TM + (warp & 1) * 32;
    const int64_t k_begin = blockIdx.z * kslice;
    const int64_t k_end = min(npad, k_begin + kslice);
    const int64_t plane = (int64_t)mpad * npad;
    double acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) acc[i][j][h] = 0.0;

    for (int d = 0; d < OZ_S; ++d) {
        int c[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) c[i][j][h] = 0;
        for (int s = 0; s <= d; ++s) {
            const int8_t *Xs = SX + s * plane;
            const int8_t *Yt = SY + (d - s) * plane;
            for (int64_t k = k_begin; k < k_end; k += 32) {
                unsigned af[2][4], bf[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int8_t *r0 = Xs + (int64_t)(a_base + i * 16 + g) * npad + k + 4 * q;
                    const int8_t *r1 = r0 + 8 * npad;
                    af[i][0] = __ldg(reinterpret_cast<const unsigned *>(r0));
                    af[i][1] = __ldg(reinterpret_cast<const unsigned *>(r1));
                    af[i][2] = __ldg(reinterpret_cast<const unsigned *>(r0 + 16));
                    af[i][3] = __ldg(reinterpret_cast<const unsigned *>(r1 + 16));
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int8_t *r = Yt + (int64_t)(b_base + j * 8 + g) * npad + k + 4 * q;
                    bf[j][0] = __ldg(reinterpret_cast<const unsigned *>(r));
                    bf[j][1] = __ldg(reinterpret_cast<const unsigned *>(r + 16));
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) imma16832(c[i][j], af[i], bf[j]);
            }
        }
        const double scale = ldexp(1.0, -7 * (d + 2));
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) acc[i][j][h] = fma((double)c[i][j][h], scale, acc[i][j][h]);
    }
    // C fragment: c0, c1 at (row g, cols 2q, 2q+1); c2, c3 at (row g+8, ...)
    double *W = work + (int64_t)blockIdx.z * m * m;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int a = a_base + i * 16 + g + (h >= 2 ? 8 : 0);
                const int b = b_base + j * 8 + 2 * q + (h & 1);
                if (a < m && b < m) W[(int64_t)a * m + b] = acc[i][j][h];
            }
}

__global__ void k_oz_reduce(int m, int split, const double *__restrict__ work, const int *__restrict__ ex,
                            const int *__restrict__ ey, double *__restrict__ G, int64_t ldg, int symmetric) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    int a = (int)(idx / m), b = (int)(idx % m);
    const int ga = a, gb = b;
    if (symmetric && a > b) {   // mirror the upper triangle (computed tiles only)
        a = gb;
        b = ga;
    }
    const int64_t src = (int64_t)a * m + b;
    double s = 0.0;
    for (int z = 0; z < split; ++z) s += work[(int64_t)z * m * m + src];
    G[(int64_t)ga * ldg + gb] = ldexp(s, ex[a] + ey[b]);
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) form of the same Gram.
//
// The digits are the seven balanced base-128 digits above, stored as bf16
// (|D| <= 64 is exact in bf16) and multiplied by tcgen05.mma (kind::f16, bf16
// operands, FP32 accumulation in tensor memory).  A digit product is at most
// 2^12 and a diagonal d sums at most 7 of them per row of K, so with K-slices
// of at most 512 rows every partial sum stays below 2^24 and the FP32
// accumulation is exact; the seven diagonals live in seven TMEM accumulators
// and are combined in FP64 once per K-slice, then the K-slices are reduced in
// a fixed order (k_oz_reduce).
//
// Operand "panel" layout (UMMA canonical K-major, no swizzle): an operand
// with R rows (the M or N side) and depth K is stored per digit s, K-step of
// 32, and 64-row panel as 8 x 4 core matrices of 8 rows x 8 K-elements
// (128 contiguous bytes, row r at 16 r):
//   [s][ks][panel][row%64 / 8][k%32 / 8][row%8][k%8]
// so one (digit, K-step) block of consecutive panels is contiguous, the
// 8-row groups of consecutive panels are 512 bytes apart (the descriptor's
// stride offset) and K-adjacent cores 128 bytes apart (its leading offset).
// ---------------------------------------------------------------------------
constexpr int TC_KSTEP = 32;        // K rows per pipeline stage
constexpr int TC_KSLICE = 512;      // K rows per CTA (exact FP32 accumulation)
constexpr int TC_TM = 128, TC_TN = 64;
constexpr unsigned TC_STAGE_A = OZ_S * 8192u, TC_STAGE_B = OZ_S * 4096u;
constexpr int TC_NS = 2;
// (16 KB of slack after the stages: no operand read can leave the allocation)
constexpr size_t TC_SMEM = 1024 + TC_NS * (size_t)(TC_STAGE_A + TC_STAGE_B) + 16384;

// digits of X (rows i < n, columns a < m, exponents e[a]) into the panel
// layout with K = rows of X and the panel rows = columns a; zero padding to
// ntr panels and nks K-steps.  One thread per (a, 8 consecutive i).
__global__ void __launch_bounds__(256)
k_oz_split_panel(int64_t n, int m, const double *__restrict__ X, int64_t ldx, const int *__restrict__ e, int64_t nks,
                 int ntr, __nv_bfloat16 *__restrict__ out) {
    const int a = blockIdx.x * 32 + (threadIdx.x & 31);
    if (a >= ntr * 64) return;
    const int ea = a < m ? e[a] : 0;
    for (int64_t i8 = blockIdx.y * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i8 < nks * 4;
         i8 += (int64_t)gridDim.y * (blockDim.x >> 5)) {
        int8_t d[8][OZ_S];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t i = i8 * 8 + k;
            const double x = (i < n && a < m) ? X[i * ldx + a] : 0.0;
            oz_digits(x, ea, d[k]);
        }
        const int64_t ks = i8 >> 2;
        const int kc = (int)(i8 & 3);
        const int panel = a >> 6, mg = (a & 63) >> 3, r = a & 7;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            const int64_t core = (((int64_t)s * nks + ks) * ntr + panel) * 32 + mg * 4 + kc;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __int2bfloat16_rn((int)d[k][s]);
            *reinterpret_cast<uint4 *>(out + core * 64 + r * 8) = *reinterpret_cast<const uint4 *>(v);
        }
    }
}

// M = 128, N = 64, bf16 x bf16 -> FP32, both operands K-major
constexpr uint32_t TC_IDESC = umma_idesc_bf16(TC_TM, TC_TN);

// sum_d v_d 2^(-7(d+2)) of the seven FP32 accumulators (exact integers,
// |v_d| <= (d+1) 2^12 K with K <= 512 rows per slice) with two FP64
// operations instead of seven: T = sum_{d>=1} v_d 2^(7(6-d)) is exact in
// int64 (|T| < K 2^49), and the result is 2^-14 (v_0 + 2^-42 T), whose one
// rounding is that of an FP64 sum.  FP64 runs at a small fraction of the
// integer rate here, and these epilogues make one such sum per output.
__device__ __forceinline__ double oz_combine(const float v[OZ_S]) {
    long long t = 0;
#pragma unroll
    for (int d = 1; d < OZ_S; ++d) t += (long long)__float2int_rn(v[d]) * (1ll << (7 * (OZ_S - 1 - d)));
    return fma((double)t, 0x1p-56, (double)__float2int_rn(v[0]) * 0x1p-14);
}

// x 2^e for the exponents of these products (power of two built from its
// bits while 2^e is a normal number, else ldexp)
__device__ __forceinline__ double oz_scale(double x, int e) {
    return (e >= -1022 && e <= 1023) ? x * __longlong_as_double((long long)(e + 1023) << 52) : ldexp(x, e);
}

// One CTA: output block a in [128 ta, +128), b in [64 tb, +64) of K-slice z
// (rows [512 z, 512 z + 512)).  Warp 0: TMEM allocation and the bulk copies
// of the digit panels; warp 1 lane 0: the MMAs; all four warps: epilogue
// (thread = TMEM lane = row a).  Gram (TALL = false): work[z][a][b] (m x m
// per slice) receives sum_d 2^(-7(d+2)) sum_{s+t=d} D_s^T E_t for a, b < m.
// Tall product (TALL = true, one slice: K <= 512): C[a][b] receives that sum
// times 2^(ea[a] + eb[b]) for a < nrows, b < m.
template <bool TALL>
__global__ void __launch_bounds__(128, 1)
k_oz_gram_tc(int m, int nta, int ntb, int64_t nks, int ntrx, int ntry, const __nv_bfloat16 *__restrict__ PX,
             const __nv_bfloat16 *__restrict__ PY, double *__restrict__ work, int symmetric, int32_t *__restrict__ err,
             int64_t nrows, double *__restrict__ C, int64_t ldc, const int *__restrict__ ea,
             const int *__restrict__ eb) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int ta = blockIdx.x / ntb, tb = blockIdx.x % ntb;
    if (!TALL && symmetric && tb < 2 * ta) return;   // block entirely below the diagonal
    const int z = blockIdx.y;
    const int64_t ks0 = (int64_t)z * (TC_KSLICE / TC_KSTEP);
    const int nsteps = (int)min((int64_t)(TC_KSLICE / TC_KSTEP), nks - ks0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr unsigned long long LIMIT_NS = 1000000000ull;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem);   // full[2], empty[2], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 64);
    unsigned char *stA = smem + 1024;
    unsigned char *stB = stA + TC_NS * TC_STAGE_A;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * TC_NS + 1; ++i) mbar_init(bars + i, 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tmem_slot);
    unsigned long long *full = bars, *empty = bars + TC_NS, *done = bars + 2 * TC_NS;

    if (warp == 0) {   // ---- producer: 7 A blocks (8 KB) and 7 B blocks (4 KB) per stage
        for (int it = 0; it < nsteps; ++it) {
            const int st = it % TC_NS, u = it / TC_NS;
            int ok = 1;
            if (u > 0 && lane == 0) ok = mbar_wait_bounded(empty + st, (u - 1) & 1, LIMIT_NS);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) atomicExch(err, 3);
                break;
            }
            if (lane == 0) mbar_expect_tx(full + st, TC_STAGE_A + TC_STAGE_B);
            __syncwarp();
            const int64_t ks = ks0 + it;
            if (lane < OZ_S) {
                const __nv_bfloat16 *src = PX + ((((int64_t)lane * nks + ks) * ntrx + 2 * ta) * 32) * 64;
                bulk_g2s(stA + st * TC_STAGE_A + lane * 8192u, src, 8192u, full + st);
            } else if (lane < 2 * OZ_S) {
                const int t = lane - OZ_S;
                const __nv_bfloat16 *src = PY + ((((int64_t)t * nks + ks) * ntry + tb) * 32) * 64;
                bulk_g2s(stB + st * TC_STAGE_B + t * 4096u, src, 4096u, full + st);
            }
        }
    } else if (warp == 1 && lane == 0) {   // ---- MMA issuer
        bool first = true;
        for (int it = 0; it < nsteps; ++it) {
            const int st = it % TC_NS, u = it / TC_NS;
            if (!mbar_wait_bounded(full + st, u & 1, LIMIT_NS)) {
                atomicExch(err, 4);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = smem_addr(stA + st * TC_STAGE_A), b0 = smem_addr(stB + st * TC_STAGE_B);
            for (int d = 0; d < OZ_S; ++d)
                for (int sd = 0; sd <= d; ++sd)
#pragma unroll
                    for (int k16 = 0; k16 < 2; ++k16) {
                        const uint64_t ad = umma_desc(a0 + sd * 8192u + k16 * 256u);
                        const uint64_t bd = umma_desc(b0 + (d - sd) * 4096u + k16 * 256u);
                        umma_bf16(tmem + (uint32_t)(d * TC_TN), ad, bd, TC_IDESC, (first && sd == 0 && k16 == 0) ? 0u : 1u);
                    }
            first = false;
            umma_commit(empty + st);   // stage free once these MMAs have read it
        }
        umma_commit(done);             // accumulators final once every MMA above completes
    }
    __syncwarp();
    // ---- epilogue: thread = row a of the block (TMEM lane 32 warp + lane)
    const bool ok = mbar_wait_bounded(done, 0, LIMIT_NS);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t a = (int64_t)ta * TC_TM + warp * 32 + lane;
    double *W = TALL ? nullptr : work + (int64_t)z * m * m;
    if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicExch(err, 5);
    } else if (TALL) {
        const int e_a = a < nrows ? ea[a] : 0;
        for (int c16 = 0; c16 < TC_TN / 16; ++c16) {
            float v[OZ_S][16];
#pragma unroll
            for (int d = 0; d < OZ_S; ++d)
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * TC_TN + c16 * 16), v[d]);
            if (a < nrows)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int b = tb * TC_TN + c16 * 16 + j;
                    if (b < m) {
                        float u[OZ_S];
#pragma unroll
                        for (int d = 0; d < OZ_S; ++d) u[d] = v[d][j];
                        C[a * ldc + b] = oz_scale(oz_combine(u), e_a + eb[b]);
                    }
                }
        }
    } else {
        for (int c16 = 0; c16 < TC_TN / 16; ++c16) {
            float v[OZ_S][16];
#pragma unroll
            for (int d = 0; d < OZ_S; ++d)
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * TC_TN + c16 * 16), v[d]);
            if (a < m)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int b = tb * TC_TN + c16 * 16 + j;
                    if (b < m) {
                        float u[OZ_S];
#pragma unroll
                        for (int d = 0; d < OZ_S; ++d) u[d] = v[d][j];
                        W[a * m + b] = oz_combine(u);
                    }
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// The kernels' shared-memory limit, raised once per device (attributes are
// process-wide and every launch uses the same size).
static void raise_tc_smem() {
    static bool raised[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !raised[dev]) {
        cudaFuncSetAttribute(k_oz_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        cudaFuncSetAttribute(k_oz_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        raised[dev] = true;
    }
}

static void ozaki_gram_tc(Ctx &ctx, int64_t n, int m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                          double *G, void *work, bool symmetric, int32_t *err) {
    const int64_t nks = (n + TC_KSTEP - 1) / TC_KSTEP;
    const int nta = (m + TC_TM - 1) / TC_TM, ntb = (m + TC_TN - 1) / TC_TN;
    const int ntrx = 2 * nta, ntry = ntb;
    const int nz = (int)((nks * TC_KSTEP + TC_KSLICE - 1) / TC_KSLICE);
    char *w = reinterpret_cast<char *>(work);
    __nv_bfloat16 *PX = reinterpret_cast<__nv_bfloat16 *>(w);
    __nv_bfloat16 *PY = PX + (size_t)OZ_S * nks * ntrx * 2048;
    char *tail = reinterpret_cast<char *>(PY + (size_t)OZ_S * nks * ntry * 2048);
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(tail);
    int *ex = reinterpret_cast<int *>(mb + 2 * m);
    int *ey = ex + m;
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(ey + m) + 16 - ((uintptr_t)(ey + m) & 15));
    raise_tc_smem();
    cudaMemsetAsync(mb, 0, 2 * (size_t)m * sizeof(unsigned long long), ctx.stream);
    const dim3 cgrid((m + 31) / 32, 64), cblock(32, 8);
    ctx.before(KC_GRAM, 8.0 * (double)n * m * 2, 0);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(n, m, X, ldx, mb);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(n, m, Y, ldy, mb + m);
    k_oz_exponent<<<(2 * m + 127) / 128, 128, 0, ctx.stream>>>(2 * m, mb, ex);
    ctx.after();
    const unsigned gy_split = (unsigned)std::min<int64_t>((nks * 4 + 7) / 8, 8192);
    ctx.before(KC_GRAM, 8.0 * (double)n * m * 2 + 2.0 * OZ_S * nks * TC_KSTEP * 64.0 * (ntrx + ntry), 0);
    k_oz_split_panel<<<dim3(ntrx * 2, gy_split), 256, 0, ctx.stream>>>(n, m, X, ldx, ex, nks, ntrx, PX);
    k_oz_split_panel<<<dim3(ntry * 2, gy_split), 256, 0, ctx.stream>>>(n, m, Y, ldy, ey, nks, ntry, PY);
    ctx.after();
    const int live = symmetric ? [&] {
        int c = 0;
        for (int a = 0; a < nta; ++a)
            for (int b = 0; b < ntb; ++b) c += b >= 2 * a;
        return c;
    }() : nta * ntb;
    const double pairs = OZ_S * (OZ_S + 1) / 2.0;
    ctx.before(KC_GRAM, 2.0 * OZ_S * (double)nks * TC_KSTEP * 64.0 * (2.0 * live + live) + 8.0 * nz * m * m,
               2.0 * pairs * (double)live * TC_TM * TC_TN * nks * TC_KSTEP);
    k_oz_gram_tc<false><<<dim3(nta * ntb, nz), 128, TC_SMEM, ctx.stream>>>(
        m, nta, ntb, nks, ntrx, ntry, PX, PY, part, symmetric ? 1 : 0, err, 0, nullptr, 0, nullptr, nullptr);
    ctx.after();
    ctx.before(KC_GRAM, 8.0 * (double)nz * m * m, 0);
    k_oz_reduce<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, ctx.stream>>>(m, nz, part, ex, ey, G, m,
                                                                                    symmetric ? 1 : 0);
    ctx.after();
}

// ---------------------------------------------------------------------------
size_t ozaki_gram_work_bytes(int64_t n, int m, int sm_count) {
    const int64_t npad = (n + 63) / 64 * 64;
    const int mpad = (m + OZ_TM - 1) / OZ_TM * OZ_TM;
    const size_t slices = 2 * (size_t)OZ_S * mpad * npad;
    const size_t split = (size_t)sm_count * 4;
    const size_t mma_sync = slices + split * m * m * sizeof(double) + 2 * (size_t)m * (sizeof(int) + 8) + 1024;
    // tensor-core form: bf16 digit panels of both operands and one m x m partial per 512-row slice
    const int64_t nks = (n + TC_KSTEP - 1) / TC_KSTEP;
    const int nta = (m + TC_TM - 1) / TC_TM, ntb = (m + TC_TN - 1) / TC_TN;
    const int64_t nz = (nks * TC_KSTEP + TC_KSLICE - 1) / TC_KSLICE;
    const size_t tc = (size_t)OZ_S * nks * (2 * nta + ntb) * 2048 * sizeof(__nv_bfloat16) +
                      (size_t)nz * m * m * sizeof(double) + 2 * (size_t)m * (sizeof(int) + 8) + 1024;
    return std::max(mma_sync, tc);
}

void ozaki_gram(Ctx &ctx, int64_t n, int m, const double *X, int64_t ldx, const double *Y, int64_t ldy, double *G,
                void *work, bool symmetric, int32_t *tc_err) {
    if (tc_err) {   // tensor-core form (tcgen05)
        ozaki_gram_tc(ctx, n, m, X, ldx, Y, ldy, G, work, symmetric, tc_err);
        return;
    }
    const int64_t npad = (n + 63) / 64 * 64;
    const int mpad = (m + OZ_TM - 1) / OZ_TM * OZ_TM;
    char *w = reinterpret_cast<char *>(work);
    int8_t *SX = reinterpret_cast<int8_t *>(w);
    int8_t *SY = SX + (size_t)OZ_S * mpad * npad;
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(SY + (size_t)OZ_S * mpad * npad);
    int *ex = reinterpret_cast<int *>(mb + 2 * m);
    int *ey = ex + m;
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(ey + m) + 16 - ((uintptr_t)(ey + m) & 15));
    const int tiles = mpad / OZ_TM;
    const int live = symmetric ? tiles * (tiles + 1) / 2 : tiles * tiles;   // tiles with work
    // K-slices: enough CTAs to fill the GPU, each at most 2^16 rows (int32 bound)
    int split = (ctx.sm_count * 4 + live - 1) / live;
    int64_t kslice = (npad + split - 1) / split;
    kslice = (kslice + 31) / 32 * 32;
    if (kslice > 65536) kslice = 65536;
    split = (int)((npad + kslice - 1) / kslice);

    cudaMemsetAsync(mb, 0, 2 * (size_t)m * sizeof(unsigned long long), ctx.stream);
    const dim3 cgrid((m + 31) / 32, 64), cblock(32, 8);
    ctx.before(KC_GRAM, 8.0 * (double)n * m * 2, 0);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(n, m, X, ldx, mb);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(n, m, Y, ldy, mb + m);
    k_oz_exponent<<<(2 * m + 127) / 128, 128, 0, ctx.stream>>>(2 * m, mb, ex);
    ctx.after();
    // digits (rows beyond n and columns beyond m become zeros)
    const dim3 sgrid(mpad / 32, (unsigned)std::min<int64_t>(npad / 32, 4096)), sblock(32, 8);
    ctx.before(KC_GRAM, 8.0 * (double)n * m * 2 + 2.0 * OZ_S * mpad * npad, 0);
    k_oz_split<<<sgrid, sblock, 0, ctx.stream>>>(n, m, npad, X, ldx, ex, SX, mpad);
    k_oz_split<<<sgrid, sblock, 0, ctx.stream>>>(n, m, npad, Y, ldy, ey, SY, mpad);
    ctx.after();
    const dim3 ggrid(tiles, tiles, split);
    const double pairs = OZ_S * (OZ_S + 1) / 2.0;
    ctx.before(KC_GRAM, 2.0 * OZ_S * mpad * npad,
               2.0 * pairs * (double)live * OZ_TM * OZ_TM * npad);
    k_oz_gram<<<ggrid, 128, 0, ctx.stream>>>(m, mpad, npad, kslice, SX, SY, part, symmetric ? 1 : 0);
    ctx.after();
    ctx.before(KC_GRAM, 8.0 * (double)split * m * m, 0);
    k_oz_reduce<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, ctx.stream>>>(m, split, part, ex, ey, G, m,
                                                                                    symmetric ? 1 : 0);
    ctx.after();
}

// ---------------------------------------------------------------------------
// Tall product C = (A diag(cs)) B on the same digits: A is n x k (row-major,
// n large, k small), B is k x m, C is n x m.  Rows of A take their own
// exponent (max over the row of |A_ai cs_i|), columns of B theirs, so the
// error is ~2^-50 of max_i |A_ai cs_i| * sum_i |B_ib|; the optional column
// scaling cs (nullptr = 1) lets a caller whose columns differ widely in size
// split the well-scaled A diag(cs) instead of A.
// ---------------------------------------------------------------------------
constexpr int OZ_TA = 128;       // tall product: CTA tile rows (4 warps x 32)
constexpr int OZ_TB = 32;        // tall product: CTA tile columns

// One warp per row: exponent e[a] and the digits of A_a diag(cs), written to
// slices[s][a][i] (row pitch kpad, zero beyond k and beyond n).
__global__ void __launch_bounds__(256)
k_oz_rowsplit(int64_t n, int k, int kpad, int64_t npad, const double *__restrict__ A, int64_t lda,
              const double *__restrict__ cs, int *__restrict__ e, int8_t *__restrict__ slices) {
    const int lane = threadIdx.x & 31;
    const int64_t a = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (a >= npad) return;
    const bool live = a < n;
    double mx = 0.0;
    if (live)
        for (int i = lane; i < k; i += 32) mx = fmax(mx, fabs(A[a * lda + i] * (cs ? cs[i] : 1.0)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const int ea = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (lane == 0 && live) e[a] = ea;
    for (int i = lane; i < kpad; i += 32) {
        const double x = (live && i < k) ? A[a * lda + i] * (cs ? cs[i] : 1.0) : 0.0;
        int8_t d[OZ_S];
        oz_digits(x, ea, d);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) slices[((int64_t)s * npad + a) * kpad + i] = d[s];
    }
}

// C tile 128 x 32 per CTA, warp 32 x 32 (2 x 4 mma), all of K per CTA (k is
// small: kpad <= 2^16 keeps each diagonal's int32 sum exact).
__global__ void __launch_bounds__(128)
k_oz_tall(int64_t n, int m, int kpad, int64_t npad, int mpad, const int8_t *__restrict__ SA,
          const int8_t *__restrict__ SB, const int *__restrict__ ea, const int *__restrict__ eb, double *__restrict__ C,
          int64_t ldc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int64_t a_base = blockIdx.y * (int64_t)OZ_TA + warp * 32;
    const int b_base = blockIdx.x * OZ_TB;
    const int64_t planeA = npad * kpad, planeB = (int64_t)mpad * kpad;
    double acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) acc[i][j][h] = 0.0;
    for (int d = 0; d < OZ_S; ++d) {
        int c[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) c[i][j][h] = 0;
        for (int s = 0; s <= d; ++s) {
            const int8_t *As = SA + s * planeA;
            const int8_t *Bt = SB + (d - s) * planeB;
            for (int kk = 0; kk < kpad; kk += 32) {
                unsigned af[2][4], bf[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int8_t *r0 = As + (a_base + i * 16 + g) * kpad + kk + 4 * q;
                    const int8_t *r1 = r0 + 8 * (int64_t)kpad;
                    af[i][0] = __ldg(reinterpret_cast<const unsigned *>(r0));
                    af[i][1] = __ldg(reinterpret_cast<const unsigned *>(r1));
                    af[i][2] = __ldg(reinterpret_cast<const unsigned *>(r0 + 16));
                    af[i][3] = __ldg(reinterpret_cast<const unsigned *>(r1 + 16));
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int8_t *r = Bt + (int64_t)(b_base + j * 8 + g) * kpad + kk + 4 * q;
                    bf[j][0] = __ldg(reinterpret_cast<const unsigned *>(r));
                    bf[j][1] = __ldg(reinterpret_cast<const unsigned *>(r + 16));
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) imma16832(c[i][j], af[i], bf[j]);
            }
        }
        const double scale = ldexp(1.0, -7 * (d + 2));
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 4; ++h) acc[i][j][h] = fma((double)c[i][j][h], scale, acc[i][j][h]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t a = a_base + i * 16 + g + (h >= 2 ? 8 : 0);
                const int b = b_base + j * 8 + 2 * q + (h & 1);
                if (a < n && b < m) C[a * ldc + b] = ldexp(acc[i][j][h], ea[a] + eb[b]);
            }
}

// Tall product on tcgen05: row exponents and digits of A diag(cs) into the
// K-major panel layout of k_oz_gram_tc's A operand (panel rows = rows a of
// A, K = its columns i, zero beyond k and beyond n).  One warp per row: the
// row maximum, then each lane the digits of 8 consecutive columns.
__global__ void __launch_bounds__(256)
k_oz_rowsplit_panel(int64_t n, int k, const double *__restrict__ A, int64_t lda, const double *__restrict__ cs,
                    int64_t nks, int ntr, int *__restrict__ e, __nv_bfloat16 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t a = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (a >= (int64_t)ntr * 64) return;
    const bool live = a < n;
    double mx = 0.0;
    if (live)
        for (int i = lane; i < k; i += 32) mx = fmax(mx, fabs(A[a * lda + i] * (cs ? cs[i] : 1.0)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const int ea = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (lane == 0 && live) e[a] = ea;
    const int panel = (int)(a >> 6), mg = (int)((a & 63) >> 3), r = (int)(a & 7);
    for (int64_t i8 = lane; i8 < nks * 4; i8 += 32) {
        int8_t d[8][OZ_S];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int64_t i = i8 * 8 + t;
            const double x = (live && i < k) ? A[a * lda + i] * (cs ? cs[i] : 1.0) : 0.0;
            oz_digits(x, ea, d[t]);
        }
        const int64_t ks = i8 >> 2;
        const int kc = (int)(i8 & 3);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            const int64_t core = (((int64_t)s * nks + ks) * ntr + panel) * 32 + mg * 4 + kc;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = __int2bfloat16_rn((int)d[t][s]);
            *reinterpret_cast<uint4 *>(out + core * 64 + r * 8) = *reinterpret_cast<const uint4 *>(v);
        }
    }
}

// C = (A diag(cs)) B with A n x k, B k x m, k <= 512 (one K-slice: the FP32
// tensor-memory sums of digit products stay exact), on tcgen05.  *err (a
// mapped host word) records a bounded wait that gave up.
static void ozaki_tall_tc(Ctx &ctx, int64_t n, int k, int m, const double *A, int64_t lda, const double *cs,
                          const double *B, int64_t ldb, double *C, int64_t ldc, void *work, int kc, int32_t *err) {
    const int64_t nks = (k + TC_KSTEP - 1) / TC_KSTEP;
    const int nta = (int)((n + TC_TM - 1) / TC_TM), ntb = (m + TC_TN - 1) / TC_TN;
    const int ntra = 2 * nta, ntrb = ntb;
    char *w = reinterpret_cast<char *>(work);
    __nv_bfloat16 *PA = reinterpret_cast<__nv_bfloat16 *>(w);
    __nv_bfloat16 *PB = PA + (size_t)OZ_S * nks * ntra * 2048;
    char *tail = reinterpret_cast<char *>(PB + (size_t)OZ_S * nks * ntrb * 2048);
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(tail);
    int *eb = reinterpret_cast<int *>(mb + m);
    int *ea = eb + m;
    raise_tc_smem();
    // B: column exponents and digit panels (panel rows = columns b, K = rows of B)
    cudaMemsetAsync(mb, 0, (size_t)m * sizeof(unsigned long long), ctx.stream);
    const dim3 cgrid((m + 31) / 32, (unsigned)std::min<int64_t>((k + 7) / 8, 64)), cblock(32, 8);
    ctx.before(kc, 8.0 * (double)k * m * 2 + 2.0 * OZ_S * nks * TC_KSTEP * 64.0 * ntrb, 0);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(k, m, B, ldb, mb);
    k_oz_exponent<<<(m + 127) / 128, 128, 0, ctx.stream>>>(m, mb, eb);
    const unsigned gy = (unsigned)std::min<int64_t>((nks * 4 + 7) / 8, 8192);
    k_oz_split_panel<<<dim3(ntrb * 2, gy), 256, 0, ctx.stream>>>(k, m, B, ldb, eb, nks, ntrb, PB);
    ctx.after();
    // A: row exponents and digit panels
    ctx.before(kc, 8.0 * (double)n * k + 2.0 * OZ_S * nks * TC_KSTEP * 64.0 * ntra, 0);
    k_oz_rowsplit_panel<<<(unsigned)((int64_t)ntra * 64 / 8), 256, 0, ctx.stream>>>(n, k, A, lda, cs, nks, ntra,
                                                                                   ea, PA);
    ctx.after();
    const double pairs = OZ_S * (OZ_S + 1) / 2.0;
    ctx.before(kc, 2.0 * OZ_S * (double)nks * TC_KSTEP * 64.0 * (2.0 * nta * ntb + (double)nta * ntb) +
                       8.0 * (double)n * m,
               2.0 * pairs * (double)nta * ntb * TC_TM * TC_TN * nks * TC_KSTEP);
    k_oz_gram_tc<true><<<dim3(nta * ntb, 1), 128, TC_SMEM, ctx.stream>>>(m, nta, ntb, nks, ntra, ntrb, PA, PB,
                                                                        nullptr, 0, err, n, C, ldc, ea, eb);
    ctx.after();
}

size_t ozaki_tall_work_bytes(int64_t n, int k, int m) {
    const int64_t npad = (n + OZ_TA - 1) / OZ_TA * OZ_TA;
    const int kpad = (k + 31) / 32 * 32, mpad = (m + OZ_TB - 1) / OZ_TB * OZ_TB;
    const size_t mma_sync = (size_t)OZ_S * npad * kpad + (size_t)OZ_S * mpad * kpad + 256 +
                            (size_t)npad * sizeof(int) + (size_t)m * (sizeof(int) + 8) + 1024;
    // tensor-core form: bf16 digit panels of A (rows) and B (columns), exponents
    const int64_t nks = (k + TC_KSTEP - 1) / TC_KSTEP;
    const int64_t nta = (n + TC_TM - 1) / TC_TM, ntb = (m + TC_TN - 1) / TC_TN;
    const size_t tc = (size_t)OZ_S * nks * (2 * nta + ntb) * 2048 * sizeof(__nv_bfloat16) + (size_t)m * 12 +
                      (size_t)nta * TC_TM * sizeof(int) + 1024;
    return std::max(mma_sync, tc);
}

bool ozaki_tall_fits(int k) { return (k + 31) / 32 * 32 <= 65536; }

void ozaki_tall(Ctx &ctx, int64_t n, int k, int m, const double *A, int64_t lda, const double *cs, const double *B,
                int64_t ldb, double *C, int64_t ldc, void *work, int kc, int32_t *tc_err) {
    if (tc_err && k <= TC_KSLICE) {
        ozaki_tall_tc(ctx, n, k, m, A, lda, cs, B, ldb, C, ldc, work, kc, tc_err);
        return;
    }
    const int64_t npad = (n + OZ_TA - 1) / OZ_TA * OZ_TA;
    const int kpad = (k + 31) / 32 * 32, mpad = (m + OZ_TB - 1) / OZ_TB * OZ_TB;
    char *w = reinterpret_cast<char *>(work);
    int8_t *SA = reinterpret_cast<int8_t *>(w);
    int8_t *SB = SA + (size_t)OZ_S * npad * kpad;
    char *tail = reinterpret_cast<char *>(SB + (size_t)OZ_S * mpad * kpad);
    tail += (256 - ((uintptr_t)tail & 255)) & 255;
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(tail);
    int *eb = reinterpret_cast<int *>(mb + m);
    int *ea = eb + m;
    // B: column exponents and transposed digits (rows = K, columns = m)
    cudaMemsetAsync(mb, 0, (size_t)m * sizeof(unsigned long long), ctx.stream);
    const dim3 cgrid((m + 31) / 32, (unsigned)std::min<int64_t>((k + 7) / 8, 64)), cblock(32, 8);
    ctx.before(kc, 8.0 * (double)k * m * 2 + 1.0 * OZ_S * mpad * kpad, 0);
    k_oz_colmax<<<cgrid, cblock, 0, ctx.stream>>>(k, m, B, ldb, mb);
    k_oz_exponent<<<(m + 127) / 128, 128, 0, ctx.stream>>>(m, mb, eb);
    const dim3 sgrid(mpad / 32, (unsigned)std::min<int64_t>(kpad / 32, 4096)), sblock(32, 8);
    k_oz_split<<<sgrid, sblock, 0, ctx.stream>>>(k, m, kpad, B, ldb, eb, SB, mpad);
    ctx.after();
    // A: row exponents and digits
    ctx.before(kc, 8.0 * (double)n * k + 1.0 * OZ_S * npad * kpad, 0);
    k_oz_rowsplit<<<(unsigned)(npad / 8), 256, 0, ctx.stream>>>(n, k, kpad, npad, A, lda, cs, ea, SA);
    ctx.after();
    const dim3 grid(mpad / OZ_TB, (unsigned)(npad / OZ_TA));
    const double pairs = OZ_S * (OZ_S + 1) / 2.0;
    ctx.before(kc, (double)OZ_S * (npad * kpad * (double)(mpad / OZ_TB) + (double)mpad * kpad) + 8.0 * (double)n * m,
               2.0 * pairs * (double)npad * mpad * kpad);
    k_oz_tall<<<grid, 128, 0, ctx.stream>>>(n, m, kpad, npad, mpad, SA, SB, ea, eb, C, ldc);
    ctx.after();
}

}  // namespace slrf
