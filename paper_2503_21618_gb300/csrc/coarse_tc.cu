// Application of the exact level's dense shifted inverses on the tcgen05
// tensor cores.
//
// Per cycle and pole, Z_j = R_j M_j^{-1} with R_j the level block's Lp columns
// (complex FP32) and M_j^{-1} the complex symmetric n x n inverse formed once
// per solve (coarse.cu).  As a real product, row-vector convention,
//   [Z_r  Z_i] = [R_r  R_i] [[M_r, M_i], [-M_i, M_r]],
// so Z^T (2n x Lp) = E_j (2n x 2n) R^T with E_j = [[M_r, -M_i], [M_i, M_r]]
// (M_r, M_i symmetric).  E_j is the MMA's M side (rows = output index o, K =
// input index k), the level block the N side (rows = column c of the pole).
//
// FP32 accuracy from bf16 operands: every value x is split into three bf16
// parts x = h0 + h1 + h2 + O(2^-25 |x|) (each the rounded remainder of the
// previous), and the six part products with s + t <= 2 are summed into one
// FP32 tensor-memory accumulator; the dropped products are O(2^-24).  The
// result is an FP32-accurate, fixed linear operator, as the cycle's
// symmetry (COCG) requires; it differs from an FP32 GEMM only in rounding.
//
// Both operands use the UMMA canonical K-major layout without swizzle (8 x 16 B
// core matrices, 128 B between K-adjacent cores, 512 B between 8-row groups);
// a (part, 32-wide K step) block of a 128-row A tile or of the whole N side is
// one contiguous run that one bulk copy moves into shared memory.  The K range
// is split between two CTAs per output tile (the 21 row tiles x 4 poles of
// the 2D workload would fill only 84 SMs), whose FP32 partial sums are added
// in a fixed order by k_inv_reduce.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace slrf {

namespace {

constexpr int CT_TM = 128;              // output rows (o) per CTA
constexpr int CT_KSTEP = 32;            // K per pipeline stage
constexpr int CT_PARTS = 3;             // bf16 parts per value
constexpr int CT_KSPLIT = 2;            // CTAs per output tile along K
constexpr int CT_PAIRS = 6;             // part products with s + t <= 2
constexpr unsigned CT_ABLK = 8192u;     // one part of a 128-row A tile per K step

__host__ __device__ inline int ct_ntb(int Lp) { return (Lp + 63) / 64; }         // 64-row B panels
__host__ __device__ inline int ct_nt(int Lp) { return (Lp + 15) / 16 * 16; }     // MMA N
__host__ __device__ inline unsigned ct_bblk(int Lp) { return 4096u * ct_ntb(Lp); }
__host__ __device__ inline unsigned ct_stage(int Lp) { return CT_PARTS * (CT_ABLK + ct_bblk(Lp)); }
__host__ __device__ inline int ct_nstages(int Lp) { return 1024 + 3 * ct_stage(Lp) <= 220 * 1024 ? 3 : 2; }
inline size_t ct_smem(int Lp) { return 1024 + (size_t)ct_nstages(Lp) * ct_stage(Lp); }

__device__ __forceinline__ void split3(float x, __nv_bfloat16 h[3]) {
    h[0] = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h[0]);
    h[1] = __float2bfloat16_rn(r1);
    h[2] = __float2bfloat16_rn(r1 - __bfloat162float(h[1]));
}

// core offset (in elements) of row `row`, 8-element K group `i8` of part `s`
__device__ __forceinline__ int64_t ct_core(int s, int64_t nks, int ntr, int row, int64_t i8) {
    const int64_t ks = i8 >> 2;
    const int kc = (int)(i8 & 3);
    const int panel = row >> 6, mg = (row & 63) >> 3, r = row & 7;
    return ((((int64_t)s * nks + ks) * ntr + panel) * 32 + mg * 4 + kc) * 64 + r * 8;
}

// E_j panels: one thread per (output row o, 8 consecutive k); grid.z = pole
__global__ void __launch_bounds__(256) k_inv_split_panel(int n, int64_t nks, int ntr, const float2 *__restrict__ Minv,
                                                         __nv_bfloat16 *__restrict__ Mpan) {
    const int j = blockIdx.z;
    const int o = blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t i8 = blockIdx.y * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (o >= ntr * 64 || i8 >= nks * 4) return;
    const float2 *M = Minv + (int64_t)j * n * n;
    const int oi = o < n ? o : o - n;
    __nv_bfloat16 h[8][CT_PARTS];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t k = i8 * 8 + t;
        float x = 0.f;
        if (o < 2 * n && k < 2 * n) {
            const int ki = (int)(k < n ? k : k - n);
            const float2 v = M[(int64_t)ki * n + oi];   // symmetric: (ki, oi) = (oi, ki)
            x = (o < n) == (k < n) ? v.x : (o < n ? -v.y : v.y);
        }
        split3(x, h[t]);
    }
    __nv_bfloat16 *P = Mpan + (size_t)j * CT_PARTS * nks * ntr * 2048;
#pragma unroll
    for (int s = 0; s < CT_PARTS; ++s) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = h[t][s];
        *reinterpret_cast<uint4 *>(P + ct_core(s, nks, ntr, o, i8)) = *reinterpret_cast<const uint4 *>(v);
    }
}

// level-block panels: rows c < Lp of pole j, K = 2n (real parts, then
// imaginary parts); one thread per (c, 8 consecutive k); grid.z = pole
__global__ void __launch_bounds__(256) k_vec_split_panel(int n, int Lp, int W, int64_t nks, int ntr,
                                                         const float2 *__restrict__ R, __nv_bfloat16 *__restrict__ Rpan) {
    const int j = blockIdx.z;
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t i8 = blockIdx.y * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ntr * 64 || i8 >= nks * 4) return;
    __nv_bfloat16 h[8][CT_PARTS];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t k = i8 * 8 + t;
        float x = 0.f;
        if (c < Lp && k < 2 * n) {
            const float2 v = R[(k < n ? k : k - n) * (int64_t)W + (int64_t)j * Lp + c];
            x = k < n ? v.x : v.y;
        }
        split3(x, h[t]);
    }
    __nv_bfloat16 *P = Rpan + (size_t)j * CT_PARTS * nks * ntr * 2048;
#pragma unroll
    for (int s = 0; s < CT_PARTS; ++s) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = h[t][s];
        *reinterpret_cast<uint4 *>(P + ct_core(s, nks, ntr, c, i8)) = *reinterpret_cast<const uint4 *>(v);
    }
}

// One CTA: output rows o in [128 mt, +128) of pole j, K steps of slice z.
// Warp 0: TMEM allocation (256 columns) and the bulk copies; warp 1 lane 0:
// the MMAs; all four warps: the epilogue (thread = TMEM lane = row o), which
// writes the FP32 partial sums part[z][j][o][c].
__global__ void __launch_bounds__(128, 1)
k_inv_apply_tc(int n, int Lp, int64_t nks, int ntra, int ntrb, const __nv_bfloat16 *__restrict__ Mpan,
               const __nv_bfloat16 *__restrict__ Rpan, float *__restrict__ part, int32_t *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int mt = blockIdx.x, j = blockIdx.y, z = blockIdx.z;
    const int64_t per = (nks + CT_KSPLIT - 1) / CT_KSPLIT;
    const int64_t ks0 = z * per;
    const int nsteps = (int)max((int64_t)0, min(per, nks - ks0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = ct_nstages(Lp);
    const unsigned bblk = ct_bblk(Lp), stage = ct_stage(Lp);
    const uint32_t idesc = umma_idesc_bf16(CT_TM, ct_nt(Lp));
    constexpr unsigned long long LIMIT_NS = 1000000000ull;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem);   // full[3], empty[3], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 64);
    unsigned char *stg = smem + 1024;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * NS + 1; ++i) mbar_init(bars + i, 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tmem_slot);
    unsigned long long *full = bars, *empty = bars + NS, *done = bars + 2 * NS;
    const __nv_bfloat16 *MA = Mpan + (size_t)j * CT_PARTS * nks * ntra * 2048;
    const __nv_bfloat16 *RB = Rpan + (size_t)j * CT_PARTS * nks * ntrb * 2048;

    if (warp == 0) {   // ---- producer: 3 A blocks (8 KB) and 3 B blocks per stage
        for (int it = 0; it < nsteps; ++it) {
            const int st = it % NS, u = it / NS;
            int ok = 1;
            if (u > 0 && lane == 0) ok = mbar_wait_bounded(empty + st, (u - 1) & 1, LIMIT_NS);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) atomicExch(err, 13);
                break;
            }
            if (lane == 0) mbar_expect_tx(full + st, stage);
            __syncwarp();
            const int64_t ks = ks0 + it;
            unsigned char *sa = stg + (size_t)st * stage, *sb = sa + CT_PARTS * CT_ABLK;
            if (lane < CT_PARTS) {
                const __nv_bfloat16 *src = MA + ((((int64_t)lane * nks + ks) * ntra + 2 * mt) * 32) * 64;
                bulk_g2s(sa + lane * CT_ABLK, src, CT_ABLK, full + st);
            } else if (lane < 2 * CT_PARTS) {
                const int t = lane - CT_PARTS;
                const __nv_bfloat16 *src = RB + ((((int64_t)t * nks + ks) * ntrb) * 32) * 64;
                bulk_g2s(sb + t * bblk, src, bblk, full + st);
            }
        }
    } else if (warp == 1 && lane == 0) {   // ---- MMA issuer
        bool first = true;
        for (int it = 0; it < nsteps; ++it) {
            const int st = it % NS, u = it / NS;
            if (!mbar_wait_bounded(full + st, u & 1, LIMIT_NS)) {
                atomicExch(err, 14);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = smem_addr(stg + (size_t)st * stage), b0 = a0 + CT_PARTS * CT_ABLK;
#pragma unroll
            for (int k16 = 0; k16 < 2; ++k16)
#pragma unroll
                for (int p = 0; p < CT_PAIRS; ++p) {
                    // (s, t) = (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
                    const int s = p < 1 ? 0 : (p < 3 ? p - 1 : p - 3);
                    const int t = p < 1 ? 0 : (p < 3 ? 2 - p : 5 - p);
                    const uint64_t ad = umma_desc(a0 + s * CT_ABLK + k16 * 256u);
                    const uint64_t bd = umma_desc(b0 + t * bblk + k16 * 256u);
                    umma_bf16(tmem, ad, bd, idesc, (first && k16 == 0 && p == 0) ? 0u : 1u);
                }
            first = false;
            umma_commit(empty + st);
        }
        umma_commit(done);
    }
    __syncwarp();
    // ---- epilogue
    const bool ok = nsteps == 0 || mbar_wait_bounded(done, 0, LIMIT_NS);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int o = mt * CT_TM + warp * 32 + lane;
    float *P = part + (((int64_t)z * gridDim.y + j) * 2 * n + o) * Lp;
    if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicExch(err, 15);
    } else {
        for (int c16 = 0; c16 < ct_nt(Lp) / 16; ++c16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c16 * 16), v);
            if (o < 2 * n)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c16 * 16 + q;
                    if (c < Lp) P[c] = nsteps ? v[q] : 0.f;
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// Z[i][j Lp + c] = (sum_z part[z][j][i][c], sum_z part[z][j][n + i][c])
__global__ void k_inv_reduce(int n, int N, int Lp, int W, const float *__restrict__ part, float2 *__restrict__ Z) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)N * n * Lp;
    if (e >= tot) return;
    const int c = (int)(e % Lp);
    const int i = (int)((e / Lp) % n);
    const int j = (int)(e / ((int64_t)Lp * n));
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int z = 0; z < CT_KSPLIT; ++z) {
        const float *P = part + ((int64_t)z * N + j) * 2 * n * Lp;
        re += P[(int64_t)i * Lp + c];
        im += P[(int64_t)(n + i) * Lp + c];
    }
    Z[(int64_t)i * W + (int64_t)j * Lp + c] = make_float2(re, im);
}

}  // namespace

bool coarse_tc_fits(int Lp) { return Lp >= 1 && Lp <= 256; }

size_t coarse_tc_panel_bytes(int n, int N) {
    const int64_t nks = (2 * (int64_t)n + CT_KSTEP - 1) / CT_KSTEP;
    const int ntra = 2 * ((2 * n + CT_TM - 1) / CT_TM);
    return (size_t)N * CT_PARTS * nks * ntra * 2048 * sizeof(__nv_bfloat16);
}

size_t coarse_tc_work_bytes(int n, int N, int Lp) {
    const int64_t nks = (2 * (int64_t)n + CT_KSTEP - 1) / CT_KSTEP;
    const size_t rpan = (size_t)N * CT_PARTS * nks * ct_ntb(Lp) * 2048 * sizeof(__nv_bfloat16);
    const size_t partb = (size_t)CT_KSPLIT * N * 2 * n * Lp * sizeof(float);
    return (rpan + 255) / 256 * 256 + partb + 256;
}

void coarse_tc_panels(Ctx &ctx, int n, int N, const float2 *Minv, void *Mpan) {
    const int64_t nks = (2 * (int64_t)n + CT_KSTEP - 1) / CT_KSTEP;
    const int ntra = 2 * ((2 * n + CT_TM - 1) / CT_TM);
    const dim3 grid((unsigned)(ntra * 2), (unsigned)((nks * 4 + 7) / 8), (unsigned)N);
    ctx.before(KC_MG_COARSE, (double)N * n * n * 8 + (double)coarse_tc_panel_bytes(n, N), 0);
    k_inv_split_panel<<<grid, 256, 0, ctx.stream>>>(n, nks, ntra, Minv, reinterpret_cast<__nv_bfloat16 *>(Mpan));
    ctx.after();
}

void coarse_tc_apply(Ctx &ctx, const KrylovDims &d, int n, const void *Mpan_v, const float2 *R, float2 *Z,
                     void *work, int32_t *err) {
    const __nv_bfloat16 *Mpan = reinterpret_cast<const __nv_bfloat16 *>(Mpan_v);
    const int Lp = d.Lp, N = d.N, W = d.W();
    const int64_t nks = (2 * (int64_t)n + CT_KSTEP - 1) / CT_KSTEP;
    const int mtiles = (2 * n + CT_TM - 1) / CT_TM, ntra = 2 * mtiles, ntrb = ct_ntb(Lp);
    char *w = reinterpret_cast<char *>(work);
    __nv_bfloat16 *Rpan = reinterpret_cast<__nv_bfloat16 *>(w);
    const size_t rpan = (size_t)N * CT_PARTS * nks * ntrb * 2048 * sizeof(__nv_bfloat16);
    float *part = reinterpret_cast<float *>(w + (rpan + 255) / 256 * 256);
    static bool raised[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !raised[dev]) {
        cudaFuncSetAttribute(k_inv_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        raised[dev] = true;
    }
    ctx.before(KC_MG_COARSE, 2.0 * n * W * 8 * d.frac + (double)rpan, 0);
    k_vec_split_panel<<<dim3((unsigned)(ntrb * 2), (unsigned)((nks * 4 + 7) / 8), (unsigned)N), 256, 0,
                        ctx.stream>>>(n, Lp, W, nks, ntrb, R, Rpan);
    ctx.after();
    ctx.before(KC_MG_COARSE, (double)coarse_tc_panel_bytes(n, N) + (double)rpan * mtiles,
               8.0 * N * (double)n * n * Lp);
    k_inv_apply_tc<<<dim3((unsigned)mtiles, (unsigned)N, CT_KSPLIT), 128, ct_smem(Lp), ctx.stream>>>(
        n, Lp, nks, ntra, ntrb, Mpan, Rpan, part, err);
    ctx.after();
    const int64_t tot = (int64_t)N * n * Lp;
    ctx.before(KC_MG_COARSE, (double)CT_KSPLIT * N * 2 * n * Lp * 4 + 8.0 * n * W, 0);
    k_inv_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(n, N, Lp, W, part, Z);
    ctx.after();
}

}  // namespace slrf
