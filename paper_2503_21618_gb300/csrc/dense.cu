// FP64 kernels of the projection step of Algorithm 1: real SpMM (A U, B U,
// A X, B X), tall-skinny GEMMs (Grams U^T B U, U^T A U and the basis changes
// X = U S), residuals rho_i, and the filter combination of the
// residual-corrected form.  Everything here is FP64: these quantities set the
// accuracy of the Ritz values (relative error 1e-10) and residuals (1e-8).
#include <cuda_runtime.h>

#include "internal.h"

namespace slrf {

// ---------------------------------------------------------------------------
// Y = A X, Z = B X (either may be null); thread per (row, column)
// ---------------------------------------------------------------------------
template <bool DO_A, bool DO_B>
__global__ void __launch_bounds__(256)
k_spmm_real(int n, int m, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
            const double2 *__restrict__ ab, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
            int64_t ldy, double *__restrict__ Z, int64_t ldz) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    if (c >= m) return;
    for (int row = blockIdx.y * 8 + threadIdx.y; row < n; row += gridDim.y * 8) {
        const int k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
        double ya = 0.0, zb = 0.0;
        for (int k = k0; k < k1; ++k) {
            const double x = X[(int64_t)__ldg(col + k) * ldx + c];
            const double2 w = __ldg(ab + k);
            if (DO_A) ya = fma(w.x, x, ya);
            if (DO_B) zb = fma(w.y, x, zb);
        }
        if (DO_A) Y[(int64_t)row * ldy + c] = ya;
        if (DO_B) Z[(int64_t)row * ldz + c] = zb;
    }
}

void spmm_real(Ctx &ctx, const DevPencil &A, int m, const double *X, int64_t ldx, double *Y, int64_t ldy,
               double *Z, int64_t ldz) {
    if (!Y && !Z) return;
    const int gx = (m + 31) / 32;
    int gy = ctx.sm_count * 8 / gx;
    if (gy > (A.n + 7) / 8) gy = (A.n + 7) / 8;
    if (gy < 1) gy = 1;
    dim3 grid(gx, gy), block(32, 8);
    const int nout = (Y ? 1 : 0) + (Z ? 1 : 0);
    const double bytes = 4.0 * (A.n + 1) + 20.0 * A.nnz + 8.0 * A.n * m * (1 + nout);
    ctx.before(KC_SPMM_REAL, bytes, 2.0 * nout * A.nnz * m);
    if (Y && Z)
        k_spmm_real<true, true><<<grid, block, 0, ctx.stream>>>(A.n, m, A.rowptr, A.col, A.ab64, X, ldx, Y, ldy, Z, ldz);
    else if (Y)
        k_spmm_real<true, false><<<grid, block, 0, ctx.stream>>>(A.n, m, A.rowptr, A.col, A.ab64, X, ldx, Y, ldy, Z, ldz);
    else
        k_spmm_real<false, true><<<grid, block, 0, ctx.stream>>>(A.n, m, A.rowptr, A.col, A.ab64, X, ldx, Y, ldy, Z, ldz);
    ctx.after();
}

// ---------------------------------------------------------------------------
// DGEMM, row-major, C = op(A) op(B) (+ beta C), 64x64x16 tiles, 4x4 per thread.
// On GB300 the FP64 tensor-core path (mma.sync m8n8k4 f64) measured slower
// than this CUDA-core kernel on the Gram shapes (0.62 vs 0.70 TFLOP/s at
// 89 401 x 150, 0.79 vs 0.90 at 187 200 x 300), so FP64 products stay here.
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 16;

template <int OPA, int OPB>
__global__ void __launch_bounds__(256)
k_dgemm(int M, int N, int K, int Kc, const double *__restrict__ A, int64_t lda, const double *__restrict__ B,
        int64_t ldb, double beta, double *__restrict__ C, int64_t ldc, double *__restrict__ work) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * Kc;
    const int kend = min(K, kbeg + Kc);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // load op(A) tile [BM x BK] into As[kk][ii]
#pragma unroll
        for (int t = 0; t < (BM * BK) / 256; ++t) {
            const int e = tid + t * 256;
            int ii, kk;
            if (OPA == 1) { ii = e % BM; kk = e / BM; }   // A is K x M: coalesce along i
            else { kk = e % BK; ii = e / BK; }             // A is M x K: coalesce along k
            const int gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < kend) v = OPA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
            As[kk][ii] = v;
        }
#pragma unroll
        for (int t = 0; t < (BN * BK) / 256; ++t) {
            const int e = tid + t * 256;
            int jj, kk;
            if (OPB == 0) { jj = e % BN; kk = e / BN; }   // B is K x N
            else { kk = e % BK; jj = e / BK; }             // B is N x K
            const int gj = j0 + jj, gk = k0 + kk;
            double v = 0.0;
            if (gj < N && gk < kend) v = OPB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int gi = i0 + ty + 16 * p;
        if (gi >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gj = j0 + tx + 16 * q;
            if (gj >= N) continue;
            if (work) {
                work[((int64_t)blockIdx.z * M + gi) * N + gj] = acc[p][q];
            } else {
                double *o = C + (int64_t)gi * ldc + gj;
                *o = (beta != 0.0 ? beta * *o : 0.0) + acc[p][q];
            }
        }
    }
}

__global__ void k_split_reduce(int M, int N, int split, const double *__restrict__ work, double beta,
                               double *__restrict__ C, int64_t ldc) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    double s = 0.0;
    for (int z = 0; z < split; ++z) s += work[(int64_t)z * M * N + e];
    const int i = (int)(e / N), j = (int)(e % N);
    double *o = C + (int64_t)i * ldc + j;
    *o = (beta != 0.0 ? beta * *o : 0.0) + s;
}

// Small products (the m x m x m GEMMs of the projection): one output per
// thread, 16 x 16 tiles staged in shared memory, so an m = 150 product runs on
// 100 CTAs instead of the 9 that the 64 x 64 tiling of k_dgemm gives it.
template <int OPA, int OPB>
__global__ void __launch_bounds__(256)
k_dgemm_small(int M, int N, int K, const double *__restrict__ A, int64_t lda, const double *__restrict__ B,
              int64_t ldb, double beta, double *__restrict__ C, int64_t ldc) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double s = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (i < M && ka < K) ? (OPA ? A[(int64_t)ka * lda + i] : A[(int64_t)i * lda + ka]) : 0.0;
        Bs[ty][tx] = (kb < K && j < N) ? (OPB ? B[(int64_t)j * ldb + kb] : B[(int64_t)kb * ldb + j]) : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) s = fma(As[ty][k], Bs[k][tx], s);
        __syncthreads();
    }
    if (i < M && j < N) {
        double *o = C + (int64_t)i * ldc + j;
        *o = (beta != 0.0 ? beta * *o : 0.0) + s;
    }
}

int gram_split(const Ctx &ctx, int m, int64_t n) {
    const int tiles = ((m + BM - 1) / BM) * ((m + BN - 1) / BN);
    int split = (ctx.sm_count * 4 + tiles - 1) / tiles;
    const int64_t maxs = (n + 255) / 256;    // keep at least 256 rows per slice
    if (split > maxs) split = (int)maxs;
    if (split < 1) split = 1;
    return split;
}

void dgemm(Ctx &ctx, int opA, int opB, int M, int N, int K, const double *A, int64_t lda, const double *B,
           int64_t ldb, double beta, double *C, int64_t ldc, int split, double *work, int kc) {
    if (M <= 0 || N <= 0) return;
    if (split < 1 || !work) split = 1;
    if (split == 1 && M <= 1024 && N <= 1024 && K <= 4096) {
        const dim3 grid((N + 15) / 16, (M + 15) / 16), block(16, 16);
        ctx.before(kc, 8.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * (double)K);
#define LS(a, b) k_dgemm_small<a, b><<<grid, block, 0, ctx.stream>>>(M, N, K, A, lda, B, ldb, beta, C, ldc)
        if (opA == 0 && opB == 0) LS(0, 0);
        else if (opA == 1 && opB == 0) LS(1, 0);
        else if (opA == 0 && opB == 1) LS(0, 1);
        else LS(1, 1);
#undef LS
        ctx.after();
        return;
    }
    int Kc = (K + split - 1) / split;
    Kc = (Kc + BK - 1) / BK * BK;
    split = (K + Kc - 1) / Kc;
    if (split < 1) split = 1;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, split);
    double *w = split > 1 ? work : nullptr;
    ctx.before(kc, 8.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * (double)K);
#define L(a, b) k_dgemm<a, b><<<grid, 256, 0, ctx.stream>>>(M, N, K, Kc, A, lda, B, ldb, beta, C, ldc, w)
    if (opA == 0 && opB == 0) L(0, 0);
    else if (opA == 1 && opB == 0) L(1, 0);
    else if (opA == 0 && opB == 1) L(0, 1);
    else L(1, 1);
#undef L
    ctx.after();
    if (split > 1) {
        const int64_t tot = (int64_t)M * N;
        ctx.before(kc, 8.0 * tot * (split + 1), 0);
        k_split_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(M, N, split, work, beta, C, ldc);
        ctx.after();
    }
}

// ---------------------------------------------------------------------------
// residuals: R = BX diag(theta) - AX, per-column ||R||^2, ||BX||^2, ||AX||^2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_residual(int n, int m, const double *__restrict__ AX, const double *__restrict__ BX, int64_t ld,
           const double *__restrict__ theta, double *__restrict__ R, int64_t ldr, double *__restrict__ part) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (c < m) {
        const double th = theta[c];
        for (int row = blockIdx.y * 8 + threadIdx.y; row < n; row += gridDim.y * 8) {
            const double ax = AX[(int64_t)row * ld + c];
            const double bx = BX[(int64_t)row * ld + c];
            const double r = fma(bx, th, -ax);
            if (R) R[(int64_t)row * ldr + c] = r;
            s0 = fma(r, r, s0);
            s1 = fma(bx, bx, s1);
            s2 = fma(ax, ax, s2);
        }
    }
    __shared__ double red[8][32][3];
    red[threadIdx.y][threadIdx.x][0] = s0;
    red[threadIdx.y][threadIdx.x][1] = s1;
    red[threadIdx.y][threadIdx.x][2] = s2;
    __syncthreads();
    if (threadIdx.y == 0 && c < m) {
        double a = 0, b = 0, d = 0;
        for (int y = 0; y < 8; ++y) {
            a += red[y][threadIdx.x][0];
            b += red[y][threadIdx.x][1];
            d += red[y][threadIdx.x][2];
        }
        double *o = part + ((int64_t)blockIdx.y * m + c) * 3;
        o[0] = a;
        o[1] = b;
        o[2] = d;
    }
}

__global__ void k_residual_reduce(int m, int gy, const double *__restrict__ part, const double *__restrict__ theta,
                                  double *__restrict__ rho, double *__restrict__ rho_ax) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= m) return;
    double a = 0, b = 0, d = 0;
    for (int g = lane; g < gy; g += 32) {
        const double *o = part + ((int64_t)g * m + c) * 3;
        a += o[0];
        b += o[1];
        d += o[2];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        d += __shfl_xor_sync(0xffffffffu, d, off);
    }
    if (lane == 0) {
        const double nr = sqrt(a);
        rho[c] = nr / (fabs(theta[c]) * sqrt(b));
        if (rho_ax) rho_ax[c] = nr / sqrt(d);
    }
}

void residual(Ctx &ctx, int n, int m, const double *AX, const double *BX, int64_t ld, const double *theta,
              double *Rout, int64_t ldr, double *rho, double *rho_ax, double *work) {
    const int gx = (m + 31) / 32;
    int gy = ctx.sm_count * 4 / gx;
    if (gy > (n + 7) / 8) gy = (n + 7) / 8;
    if (gy > 1024) gy = 1024;
    if (gy < 1) gy = 1;
    ctx.before(KC_RESIDUAL, 8.0 * n * m * (Rout ? 3 : 2), 8.0 * n * m);
    k_residual<<<dim3(gx, gy), dim3(32, 8), 0, ctx.stream>>>(n, m, AX, BX, ld, theta, Rout, ldr, work);
    ctx.after();
    ctx.before(KC_RESIDUAL, 24.0 * gy * m, 0);
    k_residual_reduce<<<(m * 32 + 255) / 256, 256, 0, ctx.stream>>>(m, gy, work, theta, rho, rho_ax);
    ctx.after();
}

// ---------------------------------------------------------------------------
// U = X diag(phi) + Ucorr
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_filter_combine(int n, int m, const double *__restrict__ X, int64_t ldx,
                                 const double *__restrict__ phi, const T *__restrict__ Uc, int ldc,
                                 double *__restrict__ U, int64_t ldu) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    if (c >= m) return;
    const double ph = phi ? phi[c] : 0.0;
    for (int row = blockIdx.y * 8 + threadIdx.y; row < n; row += gridDim.y * 8) {
        const double x = X ? X[(int64_t)row * ldx + c] * ph : 0.0;
        U[(int64_t)row * ldu + c] = x + (double)Uc[(int64_t)row * ldc + c];
    }
}

template <typename T>
void filter_combine(Ctx &ctx, int n, int m, const double *X, int64_t ldx, const double *phi, const T *Ucorr,
                    int ldc, double *U, int64_t ldu) {
    const int gx = (m + 31) / 32;
    int gy = ctx.sm_count * 8 / gx;
    if (gy > (n + 7) / 8) gy = (n + 7) / 8;
    if (gy < 1) gy = 1;
    ctx.before(KC_FILTER_COMBINE, (double)n * m * (8 * (X ? 2 : 1) + sizeof(T)), 2.0 * n * m);
    k_filter_combine<T><<<dim3(gx, gy), dim3(32, 8), 0, ctx.stream>>>(n, m, X, ldx, phi, Ucorr, ldc, U, ldu);
    ctx.after();
}
template void filter_combine<float>(Ctx &, int, int, const double *, int64_t, const double *, const float *, int,
                                    double *, int64_t);
template void filter_combine<double>(Ctx &, int, int, const double *, int64_t, const double *, const double *,
                                     int, double *, int64_t);

void fill_zero(Ctx &ctx, void *p, size_t bytes) { cudaMemsetAsync(p, 0, bytes, ctx.stream); }

void copy_block(Ctx &ctx, int n, int m, const double *src, int64_t lds, double *dst, int64_t ldd) {
    cudaMemcpy2DAsync(dst, (size_t)ldd * 8, src, (size_t)lds * 8, (size_t)m * 8, (size_t)n,
                      cudaMemcpyDeviceToDevice, ctx.stream);
}

}  // namespace slrf
