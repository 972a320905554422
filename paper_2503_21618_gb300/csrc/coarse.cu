// Exact solve of one multigrid level by dense shifted inverses.
//
// The cycle's coarse-grid correction is only as good as the level it stops
// at.  Stopping at a level of ~10^3 unknowns with an exact solve there
// (instead of smoothing it and recursing once more) cuts the COCG
// iterations per pole on the 2D bench pencil from ~15 to ~10.  A level of
// that size is solved exactly by its shifted inverses: per solve, with the
// poles known, every matrix M_j = A_l - sigma_j B_l (complex symmetric,
// Im M_j = -Im(sigma_j) B_l definite, so every leading block is nonsingular
// and no pivoting is needed) is formed densely and inverted in place by
// blocked Gauss-Jordan elimination; the cycle then applies Z_j = M_j^{-1} R_j
// as one batched complex GEMM per visit.  The inverse is symmetrised, so the
// cycle stays a complex symmetric operator, as COCG requires.
//
// Blocked Gauss-Jordan (column-major view, blocks of CB rows/columns K, the
// rest R), per block step, in place:
//   P = M_KK^{-1} (one CTA per matrix, Gauss-Jordan in shared memory)
//   T = P M_K*            C = M_*K
//   M -= C T              (rank-CB update of the whole matrix)
//   M_K* = T,  M_*K = -C P,  M_KK = P
// after the last block M holds M^{-1}.  The GEMMs are plain complex FP32
// GEMMs (cuBLAS, batched over the poles).
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace slrf {

namespace {

constexpr int CB = 64;   // block size of the elimination

// M_j = A - sigma_j B on the level's CSR pattern of (a, b) pairs, dense n x n
__global__ void k_dense_shift(int n, int N, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const float2 *__restrict__ ab, PoleSet<float> ps, float2 *__restrict__ M) {
    const int row = blockIdx.x;
    const int j = blockIdx.y;
    float2 *Mr = M + ((int64_t)j * n + row) * n;
    for (int c = threadIdx.x; c < n; c += blockDim.x) Mr[c] = make_float2(0.f, 0.f);
    __syncthreads();
    const float sr = ps.re[j], si = ps.im[j];
    for (int k = ptr[row] + threadIdx.x; k < ptr[row + 1]; k += blockDim.x) {
        const float2 w = ab[k];
        Mr[col[k]] = make_float2(w.x - sr * w.y, -si * w.y);
    }
}

// In-place inverse of the b x b diagonal block at (k0, k0) of each of the
// N matrices (column-major, leading dimension n), copied out to P (b x b,
// column-major, ld CB) -- Gauss-Jordan without pivoting in shared memory.
// 1024 threads, thread (r, c0) owns rows r and columns c0, c0 + 16, ...: no
// index division in the elimination loop, four entries per thread.
__global__ void __launch_bounds__(1024) k_block_inverse(int n, int b, int k0, const float2 *__restrict__ M,
                                                       float2 *__restrict__ P) {
    __shared__ float2 S[CB][CB + 1];   // S[r][c]
    __shared__ float2 rowk[CB], colk[CB];
    const int j = blockIdx.x;
    const float2 *Mj = M + (int64_t)j * n * n;
    const int r = threadIdx.x & (CB - 1), c0 = threadIdx.x >> 6;   // c0 in [0, 16)
    for (int c = c0; c < b; c += 16)
        if (r < b) S[r][c] = Mj[(int64_t)(k0 + c) * n + k0 + r];
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x < b) {
            rowk[threadIdx.x] = S[k][threadIdx.x];
            colk[threadIdx.x] = S[threadIdx.x][k];
        }
        __syncthreads();
        const float2 p = rowk[k];
        const float den = p.x * p.x + p.y * p.y;
        const float2 pinv = make_float2(p.x / den, -p.y / den);
        if (r < b) {
            const float2 cr = colk[r];
            for (int c = c0; c < b; c += 16) {
                float2 v;
                if (r == k && c == k) {
                    v = pinv;
                } else if (r == k) {
                    v = cmul(rowk[c], pinv);
                } else if (c == k) {
                    v = cmul(cr, pinv);
                    v.x = -v.x;
                    v.y = -v.y;
                } else {
                    v = csub(S[r][c], cmul(cr, cmul(rowk[c], pinv)));
                }
                S[r][c] = v;
            }
        }
        __syncthreads();
    }
    float2 *Pj = P + (int64_t)j * CB * CB;
    for (int c = c0; c < b; c += 16)
        if (r < b) Pj[c * CB + r] = S[r][c];
}

// dst(r, c) = scale * src(r, c) for an rows x cols column-major block of
// each of N matrices
__global__ void k_copy_block(int N, int rows, int cols, const float2 *__restrict__ src, int64_t lds, int64_t ss,
                             float2 *__restrict__ dst, int64_t ldd, int64_t sd, float scale) {
    const int64_t tot = (int64_t)rows * cols;
    const int j = blockIdx.y;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % rows), c = (int)(e / rows);
        const float2 v = src[j * ss + (int64_t)c * lds + r];
        dst[j * sd + (int64_t)c * ldd + r] = make_float2(scale * v.x, scale * v.y);
    }
}

// M <- (M + M^T) / 2 for each matrix (upper triangle pairs)
__global__ void k_symmetrize_c(int n, float2 *__restrict__ M) {
    const int j = blockIdx.y;
    float2 *Mj = M + (int64_t)j * n * n;
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        if (c <= r) continue;
        const float2 a = Mj[(int64_t)r * n + c], b = Mj[(int64_t)c * n + r];
        const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
        Mj[(int64_t)r * n + c] = m;
        Mj[(int64_t)c * n + r] = m;
    }
}

}  // namespace

size_t coarse_inverse_work_bytes(int n, int N) {
    return (2 * (size_t)N * n * CB + (size_t)N * CB * CB) * sizeof(float2) + 1024;
}

int coarse_inverse(Ctx &ctx, void *cublas, int n, const PoleSet<float> &ps, const int32_t *ptr, const int32_t *col,
                   const float2 *ab, float2 *Minv, void *work) {
    cublasHandle_t hb = reinterpret_cast<cublasHandle_t>(cublas);
    const int N = ps.N;
    const int64_t nn = (int64_t)n * n;
    float2 *T = reinterpret_cast<float2 *>(work);          // N x (CB x n), ld CB
    float2 *C = T + (size_t)N * n * CB;                      // N x (n x CB), ld n
    float2 *P = C + (size_t)N * n * CB;                      // N x (CB x CB), ld CB
    cublasStatus_t st = cublasSetStream(hb, ctx.stream);
    if (st != CUBLAS_STATUS_SUCCESS) return (int)st;
    ctx.before(KC_MG_COARSE, (double)N * nn * 8, 0);
    k_dense_shift<<<dim3(n, N), 128, 0, ctx.stream>>>(n, N, ptr, col, ab, ps, Minv);
    ctx.after();
    const cuComplex one = make_cuComplex(1.f, 0.f), mone = make_cuComplex(-1.f, 0.f),
                    zero = make_cuComplex(0.f, 0.f);
    const unsigned cgrid = (unsigned)std::min<int64_t>(((int64_t)n * CB + 255) / 256, 4096);
    for (int k0 = 0; k0 < n; k0 += CB) {
        const int b = std::min(CB, n - k0);
        ctx.before(KC_MG_COARSE, (double)N * b * b * 16, 8.0 * N * b * b * b);
        k_block_inverse<<<N, 1024, 0, ctx.stream>>>(n, b, k0, Minv, P);
        ctx.after();
        // T = P M_K*  (b x n)
        ctx.before(KC_MG_COARSE, (double)N * b * n * 16, 8.0 * N * b * b * n);
        st = cublasCgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, b, n, b, &one, P, CB, (int64_t)CB * CB,
                                       Minv + k0, n, nn, &zero, T, CB, (int64_t)CB * n, N);
        ctx.after();
        if (st != CUBLAS_STATUS_SUCCESS) return (int)st;
        // C = M_*K  (n x b)
        ctx.before(KC_MG_COARSE, (double)N * b * n * 16, 0);
        k_copy_block<<<dim3(cgrid, N), 256, 0, ctx.stream>>>(N, n, b, Minv + (int64_t)k0 * n, n, nn, C, n,
                                                             (int64_t)n * CB, 1.f);
        ctx.after();
        // M -= C T
        ctx.before(KC_MG_COARSE, (double)N * nn * 16, 8.0 * N * b * (double)nn);
        st = cublasCgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, n, n, b, &mone, C, n, (int64_t)n * CB, T, CB,
                                       (int64_t)CB * n, &one, Minv, n, nn, N);
        ctx.after();
        if (st != CUBLAS_STATUS_SUCCESS) return (int)st;
        // M_K* = T
        ctx.before(KC_MG_COARSE, (double)N * b * n * 16, 0);
        k_copy_block<<<dim3(cgrid, N), 256, 0, ctx.stream>>>(N, b, n, T, CB, (int64_t)CB * n, Minv + k0, n, nn, 1.f);
        ctx.after();
        // M_*K = -C P
        ctx.before(KC_MG_COARSE, (double)N * b * n * 16, 8.0 * N * b * b * n);
        st = cublasCgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, n, b, b, &mone, C, n, (int64_t)n * CB, P, CB,
                                       (int64_t)CB * CB, &zero, Minv + (int64_t)k0 * n, n, nn, N);
        ctx.after();
        if (st != CUBLAS_STATUS_SUCCESS) return (int)st;
        // M_KK = P
        ctx.before(KC_MG_COARSE, (double)N * b * b * 16, 0);
        k_copy_block<<<dim3(1, N), 256, 0, ctx.stream>>>(N, b, b, P, CB, (int64_t)CB * CB, Minv + (int64_t)k0 * n + k0,
                                                         n, nn, 1.f);
        ctx.after();
    }
    ctx.before(KC_MG_COARSE, (double)N * nn * 16, 0);
    k_symmetrize_c<<<dim3((unsigned)std::min<int64_t>((nn + 255) / 256, 4096), N), 256, 0, ctx.stream>>>(n, Minv);
    ctx.after();
    return (int)CUBLAS_STATUS_SUCCESS;
}

int coarse_inverse_apply(Ctx &ctx, void *cublas, const KrylovDims &d, int n, const float2 *Minv, const float2 *R,
                         float2 *Z) {
    cublasHandle_t hb = reinterpret_cast<cublasHandle_t>(cublas);
    cublasStatus_t st = cublasSetStream(hb, ctx.stream);
    if (st != CUBLAS_STATUS_SUCCESS) return (int)st;
    const int W = d.W();
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
    // column-major: Z_j^T (Lp x n, ld W) = R_j^T (Lp x n, ld W) * Minv_j (symmetric)
    ctx.before(KC_MG_COARSE, (double)d.N * n * n * 8 + 2.0 * n * W * 8 * d.frac,
               8.0 * d.N * (double)n * n * d.Lp * d.frac);
    st = cublasCgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, d.Lp, n, n, &one, R, W, d.Lp, Minv, n,
                                   (int64_t)n * n, &zero, Z, W, d.Lp, d.N);
    ctx.after();
    return (int)st;
}

}  // namespace slrf
