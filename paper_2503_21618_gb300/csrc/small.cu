// Small dense m x m kernels of the projection step (m = subspace size L):
// Cholesky factor and triangular inverse for Cholesky-QR2 B-orthonormalisation,
// and the symmetric eigensolver of the projected problem (Algorithm 1, "solve
// the eigenvalue problem A_hat s_i = theta_i B_hat s_i" once B_hat = I).
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so
// the eigensolver has two modes:
//  0. cyclic parallel Jacobi in FP64 (round-robin pair ordering, all m/2
//     rotations of a round applied at once) as ONE cooperative multi-block
//     kernel: each round is "rotations -> row phase -> grid barrier -> column
//     phase -> grid barrier", so the O(m^3) rotation work of a sweep is spread
//     over many SMs;
//  1. the same Jacobi in FP32 in one block's shared memory first (fast, gives
//     eigenvectors S0 good to ~1e-6), then S0 is re-orthonormalised in FP64
//     (Cholesky of S0^T S0 ~ I), T = S0^T A S0 is formed by FP64 GEMMs, and the
//     cooperative FP64 Jacobi polishes the nearly diagonal T in 2-3 sweeps
//     (Jacobi converges quadratically; unlike first-order refinement it is
//     robust to clustered and graded spectra).
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <float.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace slrf {

// ---------------------------------------------------------------------------
// column scaling of a Gram matrix: s_i = 1/sqrt(g_ii), G <- S G S
// ---------------------------------------------------------------------------
__global__ void k_colscale(int m, double *__restrict__ G, double *__restrict__ s) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e / m), j = (int)(e % m);
    const double gi = G[(int64_t)i * m + i], gj = G[(int64_t)j * m + j];
    const double si = gi > 0.0 ? 1.0 / sqrt(gi) : 0.0;
    const double sj = gj > 0.0 ? 1.0 / sqrt(gj) : 0.0;
    // every thread reads the diagonal before any writes it: write to a copy
    // is avoided by updating the diagonal last (see k_colscale_diag).
    if (i != j) G[e] *= si * sj;
    if (i == j) s[i] = si;
}
__global__ void k_colscale_diag(int m, double *__restrict__ G, const double *__restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) G[(int64_t)i * m + i] *= s[i] * s[i];
}

void small_colscale(Ctx &ctx, int m, double *G, double *s) {
    const int64_t tot = (int64_t)m * m;
    ctx.before(KC_SMALL_DENSE, 16.0 * tot, tot);
    k_colscale<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(m, G, s);
    ctx.after();
    ctx.before(KC_SMALL_DENSE, 16.0 * m, m);
    k_colscale_diag<<<(m + 255) / 256, 256, 0, ctx.stream>>>(m, G, s);
    ctx.after();
}

__global__ void k_scale_rows(int m, const double *__restrict__ s, double *__restrict__ T) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    T[e] *= s[e / m];
}
void small_scale_rows(Ctx &ctx, int m, const double *s, double *T) {
    const int64_t tot = (int64_t)m * m;
    ctx.before(KC_SMALL_DENSE, 16.0 * tot, tot);
    k_scale_rows<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(m, s, T);
    ctx.after();
}

// ---------------------------------------------------------------------------
// Cholesky G + shift I = R^T R (R upper), one block, right-looking.  G is read
// and left untouched; R is written to Rg.  If the factorisation of G breaks
// down (a pivot <= shift_on_fail, or non-finite) and shift_on_fail > 0, it is
// redone on G + shift_on_fail I (shifted Cholesky-QR) and *status = -1; an
// unrecoverable breakdown (pivot <= 0 with no shift) sets *status = k + 1
// (k = failing pivot).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_chol_upper(int m, const double *__restrict__ G, double *__restrict__ Rg,
                                                      int32_t *__restrict__ status, int use_smem,
                                                      double shift_on_fail, int only_if_failed) {
    extern __shared__ double sm[];
    double *A = use_smem ? sm : Rg;
    const int tid = threadIdx.x, bs = blockDim.x;
    __shared__ int bad;
    __shared__ double dinv;
    double shift = 0.0;
    int first = 0;
    if (only_if_failed) {   // the blocked form's breakdown fallback: shifted factor only
        if (*(volatile int32_t *)status <= 0) return;
        first = 1;
        shift = shift_on_fail;
    }
    for (int attempt = first; attempt < 2; ++attempt) {
        for (int e = tid; e < m * m; e += bs) A[e] = G[e] + ((e / m == e % m) ? shift : 0.0);
        if (tid == 0) bad = 0;
        __syncthreads();
        // unshifted: a pivot at or below the shift (a numerically dependent
        // column of the column-scaled Gram) counts as a breakdown too
        const double pmin = attempt == 0 ? shift_on_fail : 0.0;
        for (int k = 0; k < m; ++k) {
            if (tid == 0) {
                const double d = A[k * m + k];
                if (!(d > pmin) || !isfinite(d)) {
                    bad = k + 1;
                } else {
                    const double r = sqrt(d);
                    A[k * m + k] = r;
                    dinv = 1.0 / r;
                }
            }
            __syncthreads();
            if (bad) break;
            for (int j = k + 1 + tid; j < m; j += bs) A[k * m + j] *= dinv;
            __syncthreads();
            const int r = m - k - 1;
            for (int e = tid; e < r * r; e += bs) {
                const int i = k + 1 + e / r, j = k + 1 + e % r;
                if (j >= i) A[i * m + j] -= A[k * m + i] * A[k * m + j];
            }
            __syncthreads();
        }
        if (!bad || !(shift_on_fail > 0.0) || attempt == 1) break;
        shift = shift_on_fail;
        __syncthreads();
    }
    if (!bad)
        for (int e = tid; e < m * m; e += bs) {
            const int i = e / m, j = e % m;
            if (j < i) A[e] = 0.0;
        }
    __syncthreads();
    if (use_smem)
        for (int e = tid; e < m * m; e += bs) Rg[e] = A[e];
    if (tid == 0) *status = bad ? bad : (shift > 0.0 ? -1 : 0);
}

void raise_smem_limits();   // defined after the kernels it configures

// ---------------------------------------------------------------------------
// Blocked form for m >= 64: the CHB x CHB diagonal blocks on one CTA, the
// panel solves and the symmetric trailing updates spread over the GPU (FP64
// runs at a small fraction of the FP32 rate here, and one CTA would do all
// m^3/6 FMAs of the update alone).  Right-looking, in place in R (upper).
// A breakdown at pivot k (a pivot at or below shift_on_fail) sets *status =
// k + 1 and stops the later steps; with shift_on_fail > 0 the one-block
// kernel then refactors G + shift I.
// ---------------------------------------------------------------------------
constexpr int CHB = 32;

__global__ void k_chol_init(int m, const double *__restrict__ G, double *__restrict__ A, int32_t *__restrict__ status) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e == 0) *status = 0;
    if (e < (int64_t)m * m && G != A) A[e] = G[e];
}

// One warp factors the kb x kb diagonal block (lane j owns column j of its
// upper triangle; warp barriers only).
__global__ void __launch_bounds__(32) k_chol_diag(int m, int k0, int kb, double *__restrict__ A,
                                                 int32_t *__restrict__ status, double pmin) {
    __shared__ double S[CHB][CHB + 1];
    if (*(volatile int32_t *)status != 0) return;
    const int lane = threadIdx.x;
    for (int i = 0; i < kb; ++i)
        if (lane < kb) S[i][lane] = A[(int64_t)(k0 + i) * m + k0 + lane];
    __syncwarp();
    int bad = 0;
    for (int k = 0; k < kb; ++k) {
        const double d = S[k][k];
        if (!(d > pmin) || !isfinite(d)) {
            bad = k0 + k + 1;
            break;   // uniform: every lane read the same pivot
        }
        const double r = sqrt(d), dinv = 1.0 / r;
        __syncwarp();
        if (lane == k) S[k][k] = r;
        if (lane > k && lane < kb) S[k][lane] *= dinv;
        __syncwarp();
        if (lane > k && lane < kb) {
            const double skj = S[k][lane];
            for (int i = k + 1; i <= lane; ++i) S[i][lane] -= S[k][i] * skj;
        }
        __syncwarp();
    }
    if (bad) {
        if (lane == 0) *status = bad;
        return;
    }
    for (int i = 0; i < kb; ++i)
        if (lane < kb) A[(int64_t)(k0 + i) * m + k0 + lane] = lane >= i ? S[i][lane] : 0.0;
}

// rows k0 .. k0+kb of the columns right of the block: x = R_kk^{-T} a, one
// warp per column (lane i = row i; the forward substitution broadcasts
// x_p from lane p), four columns per block
__global__ void __launch_bounds__(128) k_chol_panel(int m, int k0, int kb, double *__restrict__ A,
                                                   const int32_t *__restrict__ status) {
    __shared__ double Rk[CHB][CHB + 1];
    if (*(volatile int32_t *)status != 0) return;
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x)
        Rk[e / kb][e % kb] = A[(int64_t)(k0 + e / kb) * m + k0 + e % kb];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = k0 + kb + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= m) return;
    double v = lane < kb ? A[(int64_t)(k0 + lane) * m + c] : 0.0;
    const double ri = lane < kb ? 1.0 / Rk[lane][lane] : 0.0;
    double x = 0.0;
    for (int p = 0; p < kb; ++p) {
        const double xp = __shfl_sync(0xffffffffu, v * ri, p);
        if (lane == p) x = xp;
        if (lane > p && lane < kb) v = fma(-Rk[p][lane], xp, v);
    }
    if (lane < kb) A[(int64_t)(k0 + lane) * m + c] = x;
}

// A[i][j] -= sum_p A[k0+p][i] A[k0+p][j] for k0+kb <= i <= j < m, 16 x 16
// output tiles (the tiles below the diagonal return at once)
__global__ void __launch_bounds__(256) k_chol_update(int m, int k0, int kb, double *__restrict__ A,
                                                    const int32_t *__restrict__ status) {
    __shared__ double Pi[CHB][17], Pj[CHB][17];
    if (*(volatile int32_t *)status != 0) return;
    const int r0 = k0 + kb;
    if (blockIdx.x < blockIdx.y) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = r0 + blockIdx.y * 16, j0 = r0 + blockIdx.x * 16;
    for (int e = threadIdx.x; e < kb * 16; e += 256) {
        const int p = e / 16, q = e % 16;
        Pi[p][q] = (i0 + q < m) ? A[(int64_t)(k0 + p) * m + i0 + q] : 0.0;
        Pj[p][q] = (j0 + q < m) ? A[(int64_t)(k0 + p) * m + j0 + q] : 0.0;
    }
    __syncthreads();
    const int i = i0 + ty, j = j0 + tx;
    if (i >= m || j >= m || j < i) return;
    double s = 0.0;
    for (int p = 0; p < kb; ++p) s = fma(Pi[p][ty], Pj[p][tx], s);
    A[(int64_t)i * m + j] -= s;
}

__global__ void k_chol_finish(int m, double *__restrict__ A, const int32_t *__restrict__ status) {
    if (*(volatile int32_t *)status != 0) return;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < (int64_t)m * m && e % m < e / m) A[e] = 0.0;
}

void small_chol_upper(Ctx &ctx, int m, const double *G, double *R, int32_t *status, double shift_on_fail) {
    const size_t smem = (size_t)m * m * sizeof(double);
    const int use_smem = smem <= 200 * 1024;
    raise_smem_limits();
    if (m < 64) {
        ctx.before(KC_SMALL_DENSE, 16.0 * m * m, (double)m * m * m / 3.0);
        k_chol_upper<<<1, 1024, use_smem ? smem : 0, ctx.stream>>>(m, G, R, status, use_smem, shift_on_fail, 0);
        ctx.after();
        return;
    }
    const int64_t m2 = (int64_t)m * m;
    const unsigned eg = (unsigned)((m2 + 255) / 256);
    ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
    k_chol_init<<<eg, 256, 0, ctx.stream>>>(m, G, R, status);
    ctx.after();
    for (int k0 = 0; k0 < m; k0 += CHB) {
        const int kb = std::min(CHB, m - k0), rest = m - k0 - kb;
        ctx.before(KC_SMALL_DENSE, 16.0 * kb * kb, (double)kb * kb * kb / 3.0);
        k_chol_diag<<<1, 32, 0, ctx.stream>>>(m, k0, kb, R, status, shift_on_fail);
        ctx.after();
        if (rest == 0) break;
        ctx.before(KC_SMALL_DENSE, 16.0 * kb * rest, 0.5 * kb * kb * rest);
        k_chol_panel<<<(rest + 3) / 4, 128, 0, ctx.stream>>>(m, k0, kb, R, status);
        ctx.after();
        const int tiles = (rest + 15) / 16;
        ctx.before(KC_SMALL_DENSE, 8.0 * rest * rest, 0.5 * (double)rest * rest * kb);
        k_chol_update<<<dim3(tiles, tiles), 256, 0, ctx.stream>>>(m, k0, kb, R, status);
        ctx.after();
    }
    ctx.before(KC_SMALL_DENSE, 8.0 * m2, 0);
    k_chol_finish<<<eg, 256, 0, ctx.stream>>>(m, R, status);
    ctx.after();
    if (shift_on_fail > 0.0 && G != R) {
        ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
        k_chol_upper<<<1, 1024, use_smem ? smem : 0, ctx.stream>>>(m, G, R, status, use_smem, shift_on_fail, 1);
        ctx.after();
    }
}

// ---------------------------------------------------------------------------
// X = R^{-1} for upper triangular R (m x m, row-major): one warp per column j,
// back substitution x_i = (delta_ij - sum_{k=i+1..j} R_ik x_k) / R_ii with the
// column in shared memory and each sum split over the lanes (R rows are read
// coalesced; R stays in L1/L2).  Entries below the diagonal are set to zero.
// ---------------------------------------------------------------------------
// The reciprocals of the diagonal are formed once per column block up front
// (FP64 division is slow here), so each step of the chain is FMAs and one
// warp reduction.
__global__ void __launch_bounds__(32) k_triinv_upper(int m, const double *__restrict__ R, double *__restrict__ X) {
    extern __shared__ double xcol[];
    double *rinv = xcol + m;
    const int j = blockIdx.x, lane = threadIdx.x;
    for (int i = lane; i <= j; i += 32) rinv[i] = 1.0 / R[(int64_t)i * m + i];
    for (int i = j + 1 + lane; i < m; i += 32) X[(int64_t)i * m + j] = 0.0;
    __syncwarp();
    for (int i = j; i >= 0; --i) {
        const double *Ri = R + (int64_t)i * m;
        double s = 0.0;
        for (int k = i + 1 + lane; k <= j; k += 32) s = fma(Ri[k], xcol[k], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            const double x = ((i == j ? 1.0 : 0.0) - s) * rinv[i];
            xcol[i] = x;
            X[(int64_t)i * m + j] = x;
        }
        __syncwarp();
    }
}

void small_triinv_upper(Ctx &ctx, int m, const double *R, double *Rinv) {
    const size_t smem = 2 * (size_t)m * sizeof(double);
    ctx.before(KC_SMALL_DENSE, 16.0 * m * m, (double)m * m * m / 3.0);
    raise_smem_limits();
    k_triinv_upper<<<m, 32, smem, ctx.stream>>>(m, R, Rinv);
    ctx.after();
}

// ---------------------------------------------------------------------------
// cyclic parallel Jacobi: round-robin pair ordering (circle method)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rr_pair(int k, int r, int mp, int &a, int &b) {
    // circle method: position 0 fixed, positions 1..mp-1 rotate by r
    a = (k == 0) ? 0 : ((k - 1 + r) % (mp - 1)) + 1;
    b = ((mp - 2 - k + r) % (mp - 1)) + 1;
}

// ---------------------------------------------------------------------------
// FP32 cyclic Jacobi for m <= JMAX in one block: all m/2 rotations of a
// round applied at once (rows, then columns), A and V in shared memory with
// an odd row pitch (the column phase's lanes walk a column without bank
// conflicts), every row and column loop unrolled to its fixed trip count
// (predicated on m), and the pivot pair's zeroing folded into the column
// phase (three block barriers per round).  A rotation is skipped below
// rel_tol of sqrt(|a_pp a_qq|); the sweeps stop once every rotation of a
// sweep was below sqrt(rel_tol) (quadratic convergence: the next sweep would
// find nothing).  Output: lam ascending (FP64), Q (FP64, columns =
// eigenvectors).
// ---------------------------------------------------------------------------
constexpr int JMAX = 160;

__global__ void __launch_bounds__(1024) k_jacobi32(int m, const double *__restrict__ S, double *__restrict__ lam,
                                                  double *__restrict__ Q, int max_sweeps, float rel_tol) {
    extern __shared__ float jsm[];
    const int ld = m | 1;
    float *A = jsm, *V = jsm + (size_t)m * ld;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
    const int mp = m + (m & 1);
    const int npair = mp / 2;
    constexpr int NIT = (JMAX + 31) / 32;
    __shared__ float cs[JMAX / 2], sn[JMAX / 2];
    __shared__ int pp[JMAX / 2], qq[JMAX / 2];
    __shared__ int nrot;
    __shared__ float maxrel;
    __shared__ double red[32];
    __shared__ float absmin;
    double fro = 0.0;
    for (int e = tid; e < m * m; e += bs) {
        const double v = S[e];
        A[(e / m) * ld + e % m] = (float)v;
        fro += v * v;
    }
    for (int e = tid; e < m * m; e += bs) V[(e / m) * ld + e % m] = (e / m == e % m) ? 1.f : 0.f;
    for (int off = 16; off > 0; off >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, off);
    if (lane == 0) red[warp] = fro;
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        for (int w = 0; w < nwarp; ++w) t += red[w];
        absmin = (float)(sqrt(t) * (double)rel_tol / sqrt((double)m));
    }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) {
            nrot = 0;
            maxrel = 0.f;
        }
        __syncthreads();
        for (int r = 0; r < mp - 1; ++r) {
            if (tid < npair) {
                int a, b;
                rr_pair(tid, r, mp, a, b);
                const int p = min(a, b), q = max(a, b);
                float c = 1.f, sv = 0.f;
                if (q < m) {
                    const float apq = A[p * ld + q];
                    const float app = A[p * ld + p], aqq = A[q * ld + q];
                    const float scale = sqrtf(fabsf(app * aqq));
                    if (fabsf(apq) > rel_tol * scale && fabsf(apq) > absmin) {
                        const float th = (aqq - app) / (2.f * apq);
                        const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(1.f + th * th));
                        c = 1.f / sqrtf(1.f + t * t);
                        sv = t * c;
                        atomicAdd(&nrot, 1);
                        const float rel = fabsf(apq) / (scale > 0.f ? scale : 1.f);
                        atomicMax(reinterpret_cast<int *>(&maxrel), __float_as_int(rel));
                    }
                }
                cs[tid] = c;
                sn[tid] = sv;
                pp[tid] = p;
                qq[tid] = (q < m && sv != 0.f) ? q : -1;
            }
            __syncthreads();
            // rows: A <- J^T A (warp per pair, lanes over columns)
            for (int k = warp; k < npair; k += nwarp) {
                const int q = qq[k];
                if (q < 0) continue;
                const int p = pp[k];
                const float c = cs[k], sv = sn[k];
                float *Ap = A + p * ld, *Aq = A + q * ld;
#pragma unroll
                for (int it = 0; it < NIT; ++it) {
                    const int col = lane + 32 * it;
                    if (col < m) {
                        const float x = Ap[col], y = Aq[col];
                        Ap[col] = c * x - sv * y;
                        Aq[col] = sv * x + c * y;
                    }
                }
            }
            __syncthreads();
            // columns: A <- A J, V <- V J; the pivot pair (p, q) / (q, p) becomes 0
            for (int k = warp; k < npair; k += nwarp) {
                const int q = qq[k];
                if (q < 0) continue;
                const int p = pp[k];
                const float c = cs[k], sv = sn[k];
#pragma unroll
                for (int it = 0; it < NIT; ++it) {
                    const int row = lane + 32 * it;
                    if (row < m) {
                        float *Ar = A + row * ld, *Vr = V + row * ld;
                        const float x = Ar[p], y = Ar[q];
                        Ar[p] = row == q ? 0.f : c * x - sv * y;
                        Ar[q] = row == p ? 0.f : sv * x + c * y;
                        const float vx = Vr[p], vy = Vr[q];
                        Vr[p] = c * vx - sv * vy;
                        Vr[q] = sv * vx + c * vy;
                    }
                }
            }
            __syncthreads();
        }
        if (nrot == 0 || maxrel < sqrtf(rel_tol)) break;
        __syncthreads();
    }
    // sort eigenvalues ascending (rank sort), permute columns into Q (FP64)
    for (int i = tid; i < m; i += bs) {
        const float di = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const float dj = A[j * ld + j];
            rank += (dj < di) || (dj == di && j < i);
        }
        lam[rank] = (double)di;
        for (int row = 0; row < m; ++row) Q[(int64_t)row * m + rank] = (double)V[row * ld + i];
    }
}

// ---------------------------------------------------------------------------
// cooperative FP64 Jacobi on a global m x m matrix A (overwritten; diag = lam)
// accumulating V <- V J.  cnt[4] (device): rotation counters of the last two
// sweeps (0, 1) and their pre-check flags (2, 3).  All blocks
// compute the same rotations from the same data, so no broadcast is needed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_jacobi_coop(int m, double *__restrict__ A, double *__restrict__ V, double *__restrict__ lam, int max_sweeps,
              const double *__restrict__ normA, int *__restrict__ cnt, int32_t *__restrict__ info) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int mp = m + (m & 1);
    const int npair = mp / 2;
    __shared__ double cs[512], sn[512], dp[512], dq[512];
    __shared__ int pp[512], qq[512];
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const double eps = DBL_EPSILON;
    const double absmin = (*normA) * eps * 0.5 / (double)m;
    // cnt[2 + (sweep & 1)]: set when some pair still passes the rotation test
    if (gtid == 0) cnt[2] = cnt[3] = 0;
    grid.sync();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[sweep & 1] = 0;
        // A sweep that would rotate nothing leaves A and V as they are: test
        // every pair against the rotation criterion first (one pass over A)
        // instead of running the sweep's 2 (mp - 1) grid barriers to find out.
        {
            int found = 0;
            for (int64_t e = gtid; e < (int64_t)m * m && !found; e += gsz) {
                const int p = (int)(e / m), q = (int)(e % m);
                if (q <= p) continue;
                const double apq = A[e];
                const double scale = sqrt(fabs(A[(int64_t)p * m + p] * A[(int64_t)q * m + q]));
                found = fabs(apq) > eps * scale && fabs(apq) > absmin;
            }
            if (found) atomicOr(&cnt[2 + (sweep & 1)], 1);
            grid.sync();
            const int any = *(volatile int *)&cnt[2 + (sweep & 1)];
            // the other flag was last read before this sweep's barriers: reset it for the next sweep
            if (gtid == 0) cnt[2 + ((sweep + 1) & 1)] = 0;
            if (!any) break;
        }
        __syncthreads();
        for (int r = 0; r < mp - 1; ++r) {
            // Every block derives all rotations of the round from the pair
            // blocks (p,p), (q,q), (p,q).  Those entries are not written by the
            // row phase (below), so a block still reading them here cannot race
            // with a block that has moved on to the row phase.
            for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                int a, b;
                rr_pair(k, r, mp, a, b);
                const int p = min(a, b), q = max(a, b);
                double c = 1, s = 0, t = 0, app = 0, aqq = 0, apq = 0;
                if (q < m) {
                    apq = A[(int64_t)p * m + q];
                    app = A[(int64_t)p * m + p];
                    aqq = A[(int64_t)q * m + q];
                    const double scale = sqrt(fabs(app * aqq));
                    if (fabs(apq) > eps * scale && fabs(apq) > absmin) {
                        const double th = (aqq - app) / (2 * apq);
                        t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        // every applied rotation counts: near-degenerate pairs
                        // converge only once they stop rotating
                        if (blockIdx.x == 0) atomicAdd(&cnt[sweep & 1], 1);
                    }
                }
                cs[k] = c;
                sn[k] = s;
                dp[k] = app - t * apq;   // rotated diagonal of the pair block
                dq[k] = aqq + t * apq;
                pp[k] = p;
                qq[k] = (q < m && s != 0.0) ? q : -1;
            }
            __syncthreads();
            // rows p, q <- J^T (rows p, q), except the pair block itself
            for (int64_t e = gtid; e < (int64_t)npair * m; e += gsz) {
                const int k = (int)(e / m), col = (int)(e % m);
                const int q = qq[k];
                if (q < 0) continue;
                const int p = pp[k];
                if (col == p || col == q) continue;
                const double c = cs[k], s = sn[k];
                const double apk = A[(int64_t)p * m + col], aqk = A[(int64_t)q * m + col];
                A[(int64_t)p * m + col] = c * apk - s * aqk;
                A[(int64_t)q * m + col] = s * apk + c * aqk;
            }
            grid.sync();
            // columns p, q <- (columns p, q) J; the pair block in closed form
            for (int64_t e = gtid; e < (int64_t)npair * m; e += gsz) {
                const int k = (int)(e / m), row = (int)(e % m);
                const int q = qq[k];
                if (q < 0) continue;
                const int p = pp[k];
                const double c = cs[k], s = sn[k];
                if (row == p) {
                    A[(int64_t)p * m + p] = dp[k];
                    A[(int64_t)p * m + q] = 0.0;
                } else if (row == q) {
                    A[(int64_t)q * m + q] = dq[k];
                    A[(int64_t)q * m + p] = 0.0;
                } else {
                    const double akp = A[(int64_t)row * m + p], akq = A[(int64_t)row * m + q];
                    A[(int64_t)row * m + p] = c * akp - s * akq;
                    A[(int64_t)row * m + q] = s * akp + c * akq;
                }
                const double vkp = V[(int64_t)row * m + p], vkq = V[(int64_t)row * m + q];
                V[(int64_t)row * m + p] = c * vkp - s * vkq;
                V[(int64_t)row * m + q] = s * vkp + c * vkq;
            }
            grid.sync();
        }
        const int n_rot = *(volatile int *)&cnt[sweep & 1];
        grid.sync();
        if (n_rot == 0) {
            ++sweep;
            break;
        }
    }
    for (int64_t i = gtid; i < m; i += gsz) lam[i] = A[i * m + i];
    if (gtid == 0 && info) *info = sweep;
}

__global__ void k_identity(int m, double *__restrict__ V) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < (int64_t)m * m) V[e] = (e / m == e % m) ? 1.0 : 0.0;
}

// final ordering: lam ascending, Q columns permuted
__global__ void k_sort_eig(int m, const double *__restrict__ lam_in, const double *__restrict__ S,
                           double *__restrict__ lam, double *__restrict__ Q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double di = lam_in[i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double dj = lam_in[j];
            rank += (dj < di) || (dj == di && j < i);
        }
        lam[rank] = di;
        for (int row = 0; row < m; ++row) Q[(int64_t)row * m + rank] = S[(int64_t)row * m + i];
    }
}

__global__ void k_fro(int m, const double *__restrict__ S, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) s += S[e] * S[e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) t += red[w];
        *out = sqrt(t);
    }
}

size_t small_syev_work_bytes(int m) {
    const size_t mp = (size_t)(m + (m & 1));
    const size_t m2 = (size_t)m * m;
    // A32/V32 global fallback (2 mp^2 doubles) + S0, S1, G, Y, T, V (6 m^2) + lam0, normA, counters,
    // component labels and sizes (2 m ints)
    return 2 * mp * mp * sizeof(double) + 6 * m2 * sizeof(double) + (2 * (size_t)m + 2) * sizeof(double) +
           2 * (size_t)m * sizeof(int) + 4096;
}

// ---------------------------------------------------------------------------
// Iterative refinement of an approximate eigendecomposition (Ogita and
// Aishima, "Iterative refinement for symmetric eigenvalue decomposition",
// Japan J. Indust. Appl. Math. 35, 2018).  With Xh the current eigenvector
// matrix, G = Xh^T Xh, T = Xh^T S Xh and R = I - G, the exact eigenvectors
// are X = Xh (I + E) with, to first order in the error,
//   E + E^T = R                         (orthonormality)
//   T + E^T D + D E = D                 (diagonalisation, D = eigenvalues)
// so lam_i = t_ii / g_ii, e_ii = r_ii / 2 and, for i != j,
//   e_ij = (t_ij + lam_j r_ij) / (lam_j - lam_i).
// A pair is refined this way only while the step is small: its eigenvalues
// more than delta = 2 ||T - D||_F apart and |e_ij| <= 1/8; other pairs get
// e_ij = r_ij / 2 (orthonormality only) and are left to k_oa_components.
// (The paper's delta also carries ||S|| ||R||; here every step is preceded
// by a Newton-Schulz orthonormalisation X <- X (3 I - X^T X) / 2, which
// keeps R at rounding level, so that term is dropped: with the FP32
// Jacobi's ||R|| ~ 1e-4 it would group most of a graded spectrum.)  The
// products are FP64 GEMMs; three steps reach FP64 accuracy from the FP32
// Jacobi's vectors wherever the pairs are separated.
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// lam_t = t_ii / g_ii and the pair threshold delta = 2 ||T - D||_F (one
// block: the norm is one fixed-order reduction)
__global__ void __launch_bounds__(1024) k_oa_norms(int m, const double *__restrict__ G, const double *__restrict__ T,
                                                  double *__restrict__ lam_t, double *__restrict__ delta) {
    __shared__ double red[32];
    const int tid = threadIdx.x, bs = blockDim.x;
    double off = 0.0;
    for (int e = tid; e < m * m; e += bs) {
        const int i = e / m, j = e % m;
        const double d = i == j ? T[e] - T[e] / G[e] : T[e];
        off += d * d;
    }
    off = block_sum(off, red);
    for (int i = tid; i < m; i += bs) lam_t[i] = T[(int64_t)i * m + i] / G[(int64_t)i * m + i];
    if (tid == 0) *delta = 2.0 * sqrt(off);
}

// Ep = I + E (row-major), one thread per entry over many blocks (the FP64
// divisions spread over the GPU)
__global__ void k_oa_step(int m, const double *__restrict__ G, const double *__restrict__ T,
                          const double *__restrict__ lam_t, const double *__restrict__ delta, double *__restrict__ Ep) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e / m), j = (int)(e % m);
    const double r = (i == j ? 1.0 : 0.0) - G[e];
    double v;
    if (i == j) {
        v = 1.0 + 0.5 * r;
    } else {
        const double li = lam_t[i], lj = lam_t[j], num = T[e] + lj * r;
        const bool sep = fabs(li - lj) > *delta && 8.0 * fabs(num) <= fabs(lj - li);
        v = sep ? num / (lj - li) : 0.5 * r;
    }
    Ep[e] = v;
}

// Newton-Schulz orthonormalisation factor: Ep = (3 I - G) / 2
__global__ void k_ns_factor(int m, const double *__restrict__ G, double *__restrict__ Ep) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    Ep[e] = (e / m == e % m ? 1.5 : 0.0) - 0.5 * G[e];
}

// After the refinement T = Q^T S Q is diagonal up to rounding except inside
// groups of (nearly) equal eigenvalues.  Indices joined by an off-diagonal
// entry above tau = 4 m u ||S||_F (about ten times the rounding of the FP64
// products) form components (label propagation); each
// component of two or more is diagonalised by cyclic FP64 Jacobi and its
// columns of Q rotated; lam receives the diagonal (unsorted).  Workspace:
// label, size (m ints each), blk, W (m^2 doubles each), Qc (m^2 doubles).
__global__ void __launch_bounds__(1024) k_oa_components(int m, const double *__restrict__ T,
                                                       const double *__restrict__ normS, double *__restrict__ Q,
                                                       double *__restrict__ lam, int *__restrict__ label,
                                                       int *__restrict__ size, double *__restrict__ blk,
                                                       double *__restrict__ Wm, double *__restrict__ Qc) {
    const int tid = threadIdx.x, bs = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
    __shared__ int changed, k, nrot;
    __shared__ int members[1024];
    __shared__ double cs[512], sn[512];
    __shared__ int pp[512], qq[512];
    const double tau = 4.0 * m * 1.1102230246251565e-16 * (*normS);
    auto joined = [&](int i, int j) {
        return fabs(T[(int64_t)i * m + j]) > tau || fabs(T[(int64_t)j * m + i]) > tau;
    };
    for (int i = tid; i < m; i += bs) {
        label[i] = i;
        size[i] = 0;
    }
    __syncthreads();
    // labels only decrease and label[i] <= i, so the jumps end; a chain of
    // m indices needs at most m passes
    for (int pass = 0; pass <= m; ++pass) {
        if (tid == 0) changed = 0;
        __syncthreads();
        for (int e = tid; e < m * m; e += bs) {
            const int i = e / m, j = e % m;
            if (j <= i || !joined(i, j)) continue;
            const int li = label[i], lj = label[j];
            if (li != lj) {
                const int l = min(li, lj);
                atomicMin(&label[i], l);
                atomicMin(&label[j], l);
                changed = 1;
            }
        }
        __syncthreads();
        for (int i = tid; i < m; i += bs) {
            int l = label[i];
            while (label[l] != l) l = label[l];
            atomicMin(&label[i], l);
        }
        __syncthreads();
        const int c = changed;
        __syncthreads();
        if (!c) break;
    }
    for (int i = tid; i < m; i += bs) atomicAdd(&size[label[i]], 1);
    __syncthreads();
    for (int i = tid; i < m; i += bs)
        if (size[label[i]] == 1) lam[i] = T[(int64_t)i * m + i];
    for (int r = 0; r < m; ++r) {
        if (size[r] < 2) continue;   // uniform: every thread reads the same entry
        if (tid == 0) {
            int c = 0;
            for (int i = r; i < m && c < 1024; ++i)
                if (label[i] == r) members[c++] = i;
            k = c;
        }
        __syncthreads();
        const int kk = k;
        for (int e = tid; e < kk * kk; e += bs) {
            const int a = e / kk, b = e % kk;
            const int ia = members[a], ib = members[b];
            blk[e] = 0.5 * (T[(int64_t)ia * m + ib] + T[(int64_t)ib * m + ia]);
            Wm[e] = a == b ? 1.0 : 0.0;
        }
        __syncthreads();
        const int kp = kk + (kk & 1), npair = kp / 2;
        for (int sweep = 0; sweep < 40; ++sweep) {
            if (tid == 0) nrot = 0;
            __syncthreads();
            for (int rd = 0; rd < kp - 1; ++rd) {
                for (int t = tid; t < npair; t += bs) {
                    int a, b;
                    rr_pair(t, rd, kp, a, b);
                    const int p = min(a, b), q = max(a, b);
                    double c = 1.0, s = 0.0;
                    if (q < kk) {
                        const double apq = blk[p * kk + q];
                        if (fabs(apq) > tau) {
                            const double app = blk[p * kk + p], aqq = blk[q * kk + q];
                            const double th = (aqq - app) / (2.0 * apq);
                            const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                            c = 1.0 / sqrt(1.0 + tt * tt);
                            s = tt * c;
                            atomicAdd(&nrot, 1);
                        }
                    }
                    cs[t] = c;
                    sn[t] = s;
                    pp[t] = p;
                    qq[t] = (q < kk && s != 0.0) ? q : -1;
                }
                __syncthreads();
                for (int t = warp; t < npair; t += nwarp) {
                    const int q = qq[t];
                    if (q < 0) continue;
                    const int p = pp[t];
                    const double c = cs[t], s = sn[t];
                    for (int col = lane; col < kk; col += 32) {
                        const double apk = blk[p * kk + col], aqk = blk[q * kk + col];
                        blk[p * kk + col] = c * apk - s * aqk;
                        blk[q * kk + col] = s * apk + c * aqk;
                    }
                }
                __syncthreads();
                for (int t = warp; t < npair; t += nwarp) {
                    const int q = qq[t];
                    if (q < 0) continue;
                    const int p = pp[t];
                    const double c = cs[t], s = sn[t];
                    for (int row = lane; row < kk; row += 32) {
                        const double akp = blk[row * kk + p], akq = blk[row * kk + q];
                        blk[row * kk + p] = c * akp - s * akq;
                        blk[row * kk + q] = s * akp + c * akq;
                        const double wkp = Wm[row * kk + p], wkq = Wm[row * kk + q];
                        Wm[row * kk + p] = c * wkp - s * wkq;
                        Wm[row * kk + q] = s * wkp + c * wkq;
                    }
                }
                __syncthreads();
                for (int t = tid; t < npair; t += bs) {
                    const int q = qq[t];
                    if (q < 0) continue;
                    const int p = pp[t];
                    blk[p * kk + q] = 0.0;
                    blk[q * kk + p] = 0.0;
                }
                __syncthreads();
            }
            const int nr = nrot;
            __syncthreads();
            if (nr == 0) break;
        }
        for (int a = tid; a < kk; a += bs) lam[members[a]] = blk[a * kk + a];
        for (int e = tid; e < m * kk; e += bs) {
            const int row = e / kk, b = e % kk;
            Qc[e] = Q[(int64_t)row * m + members[b]];
        }
        __syncthreads();
        for (int e = tid; e < m * kk; e += bs) {
            const int row = e / kk, a = e % kk;
            double v = 0.0;
            for (int b = 0; b < kk; ++b) v = fma(Qc[row * kk + b], Wm[b * kk + a], v);
            Q[(int64_t)row * m + members[a]] = v;
        }
        __syncthreads();
    }
}

// At most one cooperative (grid-barrier) kernel of this process is in flight
// on the device at any time: concurrent handles on other streams take turns,
// so two partially resident cooperative grids can never wait on each other.
static std::mutex g_coop_mutex;

// Returns the launch's or the wait's error: a refused cooperative launch (too
// few co-resident blocks, say) must not leave the caller polishing an
// unrotated matrix.
static cudaError_t coop_jacobi(Ctx &ctx, int m, double *A, double *V, double *lam, int max_sweeps,
                               const double *normA, int *cnt) {
    static const int per_sm = [] {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_jacobi_coop, 256, 0);
        return b;
    }();
    const int64_t work = (int64_t)((m + 1) / 2) * m;
    int blocks = (int)std::min<int64_t>((work + 255) / 256, std::min(per_sm * ctx.sm_count, ctx.sm_count));
    if (blocks < 1) blocks = 1;
    int32_t *info = nullptr;
    void *args[] = {&m, &A, &V, &lam, &max_sweeps, (void *)&normA, &cnt, &info};
    thread_local cudaEvent_t done = nullptr;
    if (!done) {
        const cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            done = nullptr;
            return e;
        }
    }
    std::lock_guard<std::mutex> lock(g_coop_mutex);
    ctx.before(KC_SMALL_DENSE, 24.0 * m * m, 9.0 * (double)m * m * m * 3);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_jacobi_coop, dim3(blocks), dim3(256), args, 0,
                                                ctx.stream);
    ctx.after();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(done, ctx.stream);
    if (e != cudaSuccess) return e;
    return cudaEventSynchronize(done);
}

cudaError_t small_syev(Ctx &ctx, int m, const double *S, double *lam, double *Q, double *work, int mode) {
    const size_t m2 = (size_t)m * m;
    const size_t mp = (size_t)(m + (m & 1));
    char *w = reinterpret_cast<char *>(work);
    void *Ag = w;
    void *Vg = w + mp * mp * sizeof(double);
    double *S0 = reinterpret_cast<double *>(w + 2 * mp * mp * sizeof(double));
    double *S1 = S0 + m2;
    double *G = S1 + m2;
    double *Ym = G + m2;
    double *Tm = Ym + m2;
    double *Vm = Tm + m2;
    double *lam0 = Vm + m2;
    double *normA = lam0 + m;   // [0] = ||S||_F, [1] = the refinement's pair threshold
    int *cnt = reinterpret_cast<int *>(normA + m + 2);
    int32_t *cst = cnt + 4;

    ctx.before(KC_SMALL_DENSE, 8.0 * m2, 2.0 * m2);
    k_fro<<<1, 1024, 0, ctx.stream>>>(m, S, normA);
    ctx.after();
    ctx.before(KC_SMALL_DENSE, 8.0 * m2, 0);
    k_identity<<<(unsigned)((m2 + 255) / 256), 256, 0, ctx.stream>>>(m, Vm);
    ctx.after();
    // The FP32 stage needs A and V in one block's shared memory (m <= 160:
    // 206 KB with the odd row pitch); larger problems go straight to the
    // cooperative FP64 Jacobi.
    if (mode == 0 || m > JMAX) {
        cudaMemcpyAsync(Tm, S, m2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx.stream);
        const cudaError_t e = coop_jacobi(ctx, m, Tm, Vm, lam0, 60, normA, cnt);
        if (e != cudaSuccess) return e;
        ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
        k_sort_eig<<<(m + 127) / 128, 128, 0, ctx.stream>>>(m, lam0, Vm, lam, Q);
        ctx.after();
        return cudaGetLastError();
    }
    // stage 1: FP32 Jacobi in shared memory
    raise_smem_limits();
    ctx.before(KC_SMALL_DENSE, 24.0 * m2, 9.0 * (double)m * m2 * 8);
    const size_t smem32 = 2 * (size_t)m * (m | 1) * sizeof(float);
    k_jacobi32<<<1, 1024, smem32, ctx.stream>>>(m, S, lam0, S0, 40, 1e-6f);
    ctx.after();
    if (mode == 2) {
        // stage 2: three rounds of an orthonormalisation step and a
        // refinement step X <- X (I + E) from the FP64 products G = X^T X and
        // T = X^T (S X); then the groups of nearly equal eigenvalues are
        // diagonalised and the pairs sorted
        double *X0 = S0, *X1 = S1;
        const unsigned eg = (unsigned)((m2 + 255) / 256);
        for (int it = 0; it < 3; ++it) {
            dgemm(ctx, 1, 0, m, m, m, X0, m, X0, m, 0.0, G, m, 1, nullptr, KC_SMALL_DENSE);
            ctx.before(KC_SMALL_DENSE, 16.0 * m2, 2.0 * m2);
            k_ns_factor<<<eg, 256, 0, ctx.stream>>>(m, G, Vm);
            ctx.after();
            dgemm(ctx, 0, 0, m, m, m, X0, m, Vm, m, 0.0, X1, m, 1, nullptr, KC_SMALL_DENSE);
            std::swap(X0, X1);
            dgemm(ctx, 1, 0, m, m, m, X0, m, X0, m, 0.0, G, m, 1, nullptr, KC_SMALL_DENSE);
            dgemm(ctx, 0, 0, m, m, m, S, m, X0, m, 0.0, Ym, m, 1, nullptr, KC_SMALL_DENSE);
            dgemm(ctx, 1, 0, m, m, m, X0, m, Ym, m, 0.0, Tm, m, 1, nullptr, KC_SMALL_DENSE);
            ctx.before(KC_SMALL_DENSE, 16.0 * m2, 4.0 * m2);
            k_oa_norms<<<1, 1024, 0, ctx.stream>>>(m, G, Tm, lam0, normA + 1);
            ctx.after();
            ctx.before(KC_SMALL_DENSE, 24.0 * m2, 8.0 * m2);
            k_oa_step<<<eg, 256, 0, ctx.stream>>>(m, G, Tm, lam0, normA + 1, Vm);
            ctx.after();
            dgemm(ctx, 0, 0, m, m, m, X0, m, Vm, m, 0.0, X1, m, 1, nullptr, KC_SMALL_DENSE);
            std::swap(X0, X1);
        }
        // the last refinement step leaves R at the square of its largest
        // accepted steps: three orthonormalisation steps bring it back to
        // rounding level before the groups are rotated
        for (int it = 0; it < 3; ++it) {
            dgemm(ctx, 1, 0, m, m, m, X0, m, X0, m, 0.0, G, m, 1, nullptr, KC_SMALL_DENSE);
            ctx.before(KC_SMALL_DENSE, 16.0 * m2, 2.0 * m2);
            k_ns_factor<<<eg, 256, 0, ctx.stream>>>(m, G, Vm);
            ctx.after();
            dgemm(ctx, 0, 0, m, m, m, X0, m, Vm, m, 0.0, X1, m, 1, nullptr, KC_SMALL_DENSE);
            std::swap(X0, X1);
        }
        dgemm(ctx, 0, 0, m, m, m, S, m, X0, m, 0.0, Ym, m, 1, nullptr, KC_SMALL_DENSE);
        dgemm(ctx, 1, 0, m, m, m, X0, m, Ym, m, 0.0, Tm, m, 1, nullptr, KC_SMALL_DENSE);
        int *label = cst + 4, *csize = label + m;
        ctx.before(KC_SMALL_DENSE, 24.0 * m2, 4.0 * m2);
        k_oa_components<<<1, 1024, 0, ctx.stream>>>(m, Tm, normA, X0, lam0, label, csize, (double *)Ag,
                                                     (double *)Vg, X1);
        ctx.after();
        ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
        k_sort_eig<<<(m + 127) / 128, 128, 0, ctx.stream>>>(m, lam0, X0, lam, Q);
        ctx.after();
        return cudaGetLastError();
    }
    // stage 2: FP64 re-orthonormalisation S1 = S0 R^{-1}, G = S0^T S0 = R^T R
    dgemm(ctx, 1, 0, m, m, m, S0, m, S0, m, 0.0, G, m, 1, nullptr, KC_SMALL_DENSE);
    small_chol_upper(ctx, m, G, G, cst, 0.0);
    small_triinv_upper(ctx, m, G, Ym);
    dgemm(ctx, 0, 0, m, m, m, S0, m, Ym, m, 0.0, S1, m, 1, nullptr, KC_SMALL_DENSE);
    // T = S1^T A S1, then polish T by FP64 Jacobi, S = S1 V
    dgemm(ctx, 0, 0, m, m, m, S, m, S1, m, 0.0, Ym, m, 1, nullptr, KC_SMALL_DENSE);
    dgemm(ctx, 1, 0, m, m, m, S1, m, Ym, m, 0.0, Tm, m, 1, nullptr, KC_SMALL_DENSE);
    const cudaError_t e = coop_jacobi(ctx, m, Tm, Vm, lam0, 20, normA, cnt);
    if (e != cudaSuccess) return e;
    dgemm(ctx, 0, 0, m, m, m, S1, m, Vm, m, 0.0, S0, m, 1, nullptr, KC_SMALL_DENSE);
    ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
    k_sort_eig<<<(m + 127) / 128, 128, 0, ctx.stream>>>(m, lam0, S0, lam, Q);
    ctx.after();
    return cudaGetLastError();
}

// Kernel attributes are process-wide: a handle lowering a kernel's dynamic
// shared-memory limit to its own size while another thread is about to launch
// with more would fail that launch ("invalid argument").  So the limits are
// raised once, to the most any launch here uses (200 KB), and never changed.
void raise_smem_limits() {
    constexpr int kMaxDevices = 64;
    static std::once_flag once[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(once[dev < 0 || dev >= kMaxDevices ? 0 : dev], [] {   // per device, with it current
        const int lim = 200 * 1024;
        cudaFuncSetAttribute(k_chol_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_triinv_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
}

}  // namespace slrf
