// Block COCG over all (pole, column) shifted systems (A - sigma_j B) y = f.
//
// Section 1, Eq. (2): each outer step of Algorithm 1 needs N shifted solves
// per column.  The paper solves them by preconditioned BiCGStab (Section
// 4.2.1); A - sigma B is complex symmetric, so this library uses the
// conjugate-orthogonal CG (unconjugated bilinear form x^T y) with a Jacobi
// preconditioner M_j = diag(A - sigma_j B), which keeps the iteration a short
// recurrence of SpMM + vector updates + per-column dot products.
//
// State layout ("column block"): complex n x W, W = N * Lp, row-major with row
// stride W; pole j owns columns [j*Lp, j*Lp + Lp).  One row of the block is
// W complex numbers, so a warp reading a row is fully coalesced, and every
// matrix entry (col, a, b) is loaded once per row for all poles and columns.
//
// One iteration = 5 launches:
//   spmm      Q = (A - sigma_j B) P        + partial mu = P^T Q per column
//   alpha     alpha = rho / mu, ua = 2 coef alpha
//   update    R -= alpha Q, U += Re(ua P)  + partial rho' = R^T M^{-1} R, |R|^2
//   beta      beta = rho'/rho, convergence mask
//   direction P = M^{-1} R + beta P
// The filter output sum_j 2 Re(coef_jc Y_jc) is accumulated directly in U
// (coef_jc = w_j in the plain filter, w_j/(theta_c - sigma_j) in the
// residual-corrected one), so the per-pole solutions are never stored.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace slrf {

template <typename T> struct VecN;
template <> struct VecN<float> { static constexpr int VC = 2; };   // one float4 = 2 complex
template <> struct VecN<double> { static constexpr int VC = 1; };  // one double2 = 1 complex

template <typename T> struct ABT;
template <> struct ABT<float> { using type = float2; };
template <> struct ABT<double> { using type = double2; };

template <typename T, int VC> struct CV { cplx<T> v[VC]; };

__device__ __forceinline__ CV<float, 2> ldcv(const float2 *p) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    CV<float, 2> r;
    r.v[0] = make_float2(t.x, t.y);
    r.v[1] = make_float2(t.z, t.w);
    return r;
}
__device__ __forceinline__ void stcv(float2 *p, const CV<float, 2> &a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0].x, a.v[0].y, a.v[1].x, a.v[1].y);
}
__device__ __forceinline__ CV<double, 1> ldcv(const double2 *p) {
    CV<double, 1> r;
    r.v[0] = *p;
    return r;
}
__device__ __forceinline__ void stcv(double2 *p, const CV<double, 1> &a) { *p = a.v[0]; }

constexpr int TY = 8;   // rows processed concurrently by a block (warps)

// ---------------------------------------------------------------------------
// Jacobi inverse diagonal dinv[i][j] = 1 / (a_ii - sigma_j b_ii)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_dinv(int n, int N, const double *__restrict__ da, const double *__restrict__ db,
                       PoleSet<T> ps, int precond, cplx<T> *__restrict__ dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * N) return;
    const int row = (int)(i / N), j = (int)(i % N);
    cplx<T> r;
    if (precond == SLRF_PRECOND_JACOBI) {
        // 1/(x + i y) = (x - i y)/(x^2 + y^2), evaluated in FP64
        const double x = da[row] - (double)ps.re[j] * db[row];
        const double y = -(double)ps.im[j] * db[row];
        const double den = x * x + y * y;
        r.x = (T)(x / den);
        r.y = (T)(-y / den);
    } else {
        r.x = (T)1;
        r.y = (T)0;
    }
    dinv[i] = r;
}

// ---------------------------------------------------------------------------
// init: r = b, p = z = M^{-1} r, partial rho = r^T z, |b|^2
// ---------------------------------------------------------------------------
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_init(int n, int W, int Lp, int N, int m, const double *__restrict__ rhs, int64_t ldr,
       const double2 *__restrict__ rhs_c, const cplx<T> *__restrict__ dinv, cplx<T> *__restrict__ R,
       cplx<T> *__restrict__ P, const int32_t *__restrict__ flag, T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    int j = 0, cl = 0;
    bool act[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) act[v] = false;
    if (cg < ng) {
        j = c0 / Lp;
        cl = c0 - j * Lp;
#pragma unroll
        for (int v = 0; v < VC; ++v) act[v] = flag[c0 + v] == 1;
    }
    T acc[VC][3];
#pragma unroll
    for (int v = 0; v < VC; ++v) acc[v][0] = acc[v][1] = acc[v][2] = (T)0;
    if (cg < ng) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            const C dv = dinv[(int64_t)row * N + j];
            CV<T, VC> r, p;
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                C b = mk((T)0, (T)0);
                if (act[v]) {
                    if (rhs_c) {
                        const double2 t = rhs_c[(int64_t)row * W + c0 + v];
                        b = mk((T)t.x, (T)t.y);
                    } else if (cl + v < m) {
                        b = mk((T)rhs[(int64_t)row * ldr + cl + v], (T)0);
                    }
                }
                r.v[v] = b;
                const C z = cmul(dv, b);
                p.v[v] = z;
                const C rz = cmul(b, z);
                acc[v][0] += rz.x;
                acc[v][1] += rz.y;
                acc[v][2] += cabs2(b);
            }
            stcv(R + (int64_t)row * W + c0, r);
            stcv(P + (int64_t)row * W + c0, p);
        }
    }
    __shared__ T red[TY][32][VC * 3];
#pragma unroll
    for (int v = 0; v < VC; ++v)
#pragma unroll
        for (int s = 0; s < 3; ++s) red[ty][tx][v * 3 + s] = acc[v][s];
    __syncthreads();
    if (ty == 0 && cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            T s0 = 0, s1 = 0, s2 = 0;
            for (int y = 0; y < TY; ++y) {
                s0 += red[y][tx][v * 3 + 0];
                s1 += red[y][tx][v * 3 + 1];
                s2 += red[y][tx][v * 3 + 2];
            }
            T *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
            o[2] = s2;
            o[3] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// K1: shifted block SpMM Q = (A - sigma_j B) P, fused mu = P^T Q partials.
// Two forms: plain CSR rows (rows_per_block consecutive rows per CTA) and row
// groups (below).  Measured on the 2D Q1 pencil (mean launch over a solve):
// grid-strided rows 330 us, contiguous row blocks 355 us, row groups of 2
// 280 us, row groups of 4 396 us.  Alternatives measured and dropped
// (standalone launch, all 600 columns, L2 flushed, row groups of 2: 371 us):
// warp-cooperative index loads broadcast by shuffles (same), cp.async
// staging of the gathers in shared memory (500-570 us), unroll depth 6 / 12
// (433 / 363 us).
// ---------------------------------------------------------------------------
// Variant with contiguous row blocks (rows_per_block consecutive rows per CTA,
// so consecutive warps reuse the same gathered P rows in L1) and the nonzeros
// of a row processed UNR at a time: all UNR indices, then all UNR gathers are
// issued before the FMAs, so each warp keeps UNR loads in flight.
template <typename T, int VC, int UNR>
__global__ void __launch_bounds__(32 * TY)
k_spmm_shifted_rb(int n, int W, int Lp, int rows_per_block, const int32_t *__restrict__ rowptr,
                  const int32_t *__restrict__ col, const typename ABT<T>::type *__restrict__ ab,
                  const cplx<T> *__restrict__ sig, const cplx<T> *__restrict__ P, cplx<T> *__restrict__ Q,
                  const int32_t *__restrict__ flag, T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    C s = mk((T)0, (T)0);
    if (cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[c0 + v] == 1;
        s = sig[c0 / Lp];
    }
    C mu[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) mu[v] = mk((T)0, (T)0);
    const int r_begin = blockIdx.y * rows_per_block;
    const int r_end = min(n, r_begin + rows_per_block);
    if (act) {
        for (int row = r_begin + ty; row < r_end; row += TY) {
            const int k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
            C sa[VC], sb[VC];
#pragma unroll
            for (int v = 0; v < VC; ++v) sa[v] = sb[v] = mk((T)0, (T)0);
            int k = k0;
            for (; k + UNR <= k1; k += UNR) {
                int cc[UNR];
                typename ABT<T>::type w[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    cc[u] = __ldg(col + k + u);
                    w[u] = __ldg(ab + k + u);
                }
                CV<T, VC> p[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) p[u] = ldcv(P + (int64_t)cc[u] * W + c0);
#pragma unroll
                for (int u = 0; u < UNR; ++u)
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        sa[v].x = fma(w[u].x, p[u].v[v].x, sa[v].x);
                        sa[v].y = fma(w[u].x, p[u].v[v].y, sa[v].y);
                        sb[v].x = fma(w[u].y, p[u].v[v].x, sb[v].x);
                        sb[v].y = fma(w[u].y, p[u].v[v].y, sb[v].y);
                    }
            }
            for (; k < k1; ++k) {
                const int c = __ldg(col + k);
                const auto w = __ldg(ab + k);
                const CV<T, VC> p = ldcv(P + (int64_t)c * W + c0);
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    sa[v].x = fma(w.x, p.v[v].x, sa[v].x);
                    sa[v].y = fma(w.x, p.v[v].y, sa[v].y);
                    sb[v].x = fma(w.y, p.v[v].x, sb[v].x);
                    sb[v].y = fma(w.y, p.v[v].y, sb[v].y);
                }
            }
            CV<T, VC> q;
#pragma unroll
            for (int v = 0; v < VC; ++v) q.v[v] = csub(sa[v], cmul(s, sb[v]));
            stcv(Q + (int64_t)row * W + c0, q);
            const CV<T, VC> pr = ldcv(P + (int64_t)row * W + c0);
#pragma unroll
            for (int v = 0; v < VC; ++v) mu[v] = cfma(pr.v[v], q.v[v], mu[v]);
        }
    }
    __shared__ T red[TY][32][VC * 2];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[ty][tx][2 * v] = mu[v].x;
        red[ty][tx][2 * v + 1] = mu[v].y;
    }
    __syncthreads();
    if (ty == 0 && cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            T s0 = 0, s1 = 0;
            for (int y = 0; y < TY; ++y) {
                s0 += red[y][tx][2 * v];
                s1 += red[y][tx][2 * v + 1];
            }
            T *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
        }
    }
}

// Row-group variant.  R consecutive rows share one merged (union) column
// list; every union entry stores R coefficient pairs (zero where a row lacks
// that column).  Each gathered row of P is then used for R output rows, which
// cuts the gather traffic by R on 3-dof elasticity (rows of one node share
// their columns exactly) and by ~R/2 on 2D stencils.  Groups are assigned to
// CTAs in contiguous ranges.
template <typename T, int VC, int R, int UNR>
__global__ void __launch_bounds__(32 * TY)
k_spmm_shifted_rg(int n, int W, int Lp, int ngroups, int groups_per_block, const int32_t *__restrict__ gptr,
                  const int32_t *__restrict__ ucol, const typename ABT<T>::type *__restrict__ uab,
                  const cplx<T> *__restrict__ sig, const cplx<T> *__restrict__ P, cplx<T> *__restrict__ Q,
                  const int32_t *__restrict__ flag, T *__restrict__ part) {
    using C = cplx<T>;
    using AB = typename ABT<T>::type;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    C s = mk((T)0, (T)0);
    if (cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[c0 + v] == 1;
        s = sig[c0 / Lp];
    }
    C mu[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) mu[v] = mk((T)0, (T)0);
    const int g_begin = blockIdx.y * groups_per_block;
    const int g_end = min(ngroups, g_begin + groups_per_block);
    if (blockIdx.x == 0 && ty == 0 && g_end > g_begin) {
        // this CTA's slab of rows (whole rows, every column chunk) into L2 up
        // front: their first gathers then hit L2 instead of DRAM
        const int64_t r0 = (int64_t)g_begin * R, r1 = min((int64_t)n, (int64_t)g_end * R);
        l2_prefetch_warp(P + r0 * W, (r1 - r0) * W * (int64_t)sizeof(C), tx);
    }
    if (act) {
        for (int g = g_begin + ty; g < g_end; g += TY) {
            const int e0 = __ldg(gptr + g), e1 = __ldg(gptr + g + 1);
            C sa[R][VC], sb[R][VC];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < VC; ++v) sa[r][v] = sb[r][v] = mk((T)0, (T)0);
            int e = e0;
            for (; e + UNR <= e1; e += UNR) {
                int cc[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) cc[u] = __ldg(ucol + e + u);
                CV<T, VC> p[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) p[u] = ldcv(P + (int64_t)cc[u] * W + c0);
#pragma unroll
                for (int u = 0; u < UNR; ++u)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const AB w = __ldg(uab + (int64_t)(e + u) * R + r);
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            sa[r][v].x = fma(w.x, p[u].v[v].x, sa[r][v].x);
                            sa[r][v].y = fma(w.x, p[u].v[v].y, sa[r][v].y);
                            sb[r][v].x = fma(w.y, p[u].v[v].x, sb[r][v].x);
                            sb[r][v].y = fma(w.y, p[u].v[v].y, sb[r][v].y);
                        }
                    }
            }
            for (; e < e1; ++e) {
                const int c = __ldg(ucol + e);
                const CV<T, VC> p = ldcv(P + (int64_t)c * W + c0);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const AB w = __ldg(uab + (int64_t)e * R + r);
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        sa[r][v].x = fma(w.x, p.v[v].x, sa[r][v].x);
                        sa[r][v].y = fma(w.x, p.v[v].y, sa[r][v].y);
                        sb[r][v].x = fma(w.y, p.v[v].x, sb[r][v].x);
                        sb[r][v].y = fma(w.y, p.v[v].y, sb[r][v].y);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = g * R + r;
                if (row >= n) break;
                CV<T, VC> q;
#pragma unroll
                for (int v = 0; v < VC; ++v) q.v[v] = csub(sa[r][v], cmul(s, sb[r][v]));
                stcv(Q + (int64_t)row * W + c0, q);
                const CV<T, VC> pr = ldcv(P + (int64_t)row * W + c0);
#pragma unroll
                for (int v = 0; v < VC; ++v) mu[v] = cfma(pr.v[v], q.v[v], mu[v]);
            }
        }
    }
    __shared__ T red[TY][32][VC * 2];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[ty][tx][2 * v] = mu[v].x;
        red[ty][tx][2 * v + 1] = mu[v].y;
    }
    __syncthreads();
    if (ty == 0 && cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            T s0 = 0, s1 = 0;
            for (int y = 0; y < TY; ++y) {
                s0 += red[y][tx][2 * v];
                s1 += red[y][tx][2 * v + 1];
            }
            T *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
        }
    }
}

// ---------------------------------------------------------------------------
// Node-block variant (FP32) for 3-dof pencils whose mass couples equal dofs
// only: per neighbour node j one index, the three gathered rows 3j..3j+2 of
// P, the 3 x 3 stiffness block and three mass weights.  Against the
// row-group kernel on the same pattern: a third of the index loads, a third
// of the coefficient loads and two thirds of the mass FMAs (the zero
// off-dof mass entries are skipped).  Same FMA order per row and column
// within the stiffness and the mass sums as the row-group kernel.
// ---------------------------------------------------------------------------
template <int UNR>
__global__ void __launch_bounds__(32 * TY)
k_spmm_shifted_nb(int n, int W, int Lp, int ngroups, int groups_per_block, const int32_t *__restrict__ nptr,
                  const int32_t *__restrict__ node, const float4 *__restrict__ coef, const float2 *__restrict__ sig,
                  const float2 *__restrict__ P, float2 *__restrict__ Q, const int32_t *__restrict__ flag,
                  float *__restrict__ part) {
    constexpr int VC = 2;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    float2 s = make_float2(0.f, 0.f);
    if (cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[c0 + v] == 1;
        s = sig[c0 / Lp];
    }
    float2 mu[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) mu[v] = make_float2(0.f, 0.f);
    const int g_begin = blockIdx.y * groups_per_block;
    const int g_end = min(ngroups, g_begin + groups_per_block);
    if (blockIdx.x == 0 && ty == 0 && g_end > g_begin) {
        const int64_t r0 = (int64_t)g_begin * 3, r1 = min((int64_t)n, (int64_t)g_end * 3);
        l2_prefetch_warp(P + r0 * W, (r1 - r0) * W * (int64_t)sizeof(float2), tx);
    }
    if (act) {
        const float2 *Pc = P + c0;
        for (int g = g_begin + ty; g < g_end; g += TY) {
            const int t0 = __ldg(nptr + g), t1 = __ldg(nptr + g + 1);
            float2 sa[3][VC], sb[3][VC];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int v = 0; v < VC; ++v) sa[r][v] = sb[r][v] = make_float2(0.f, 0.f);
            for (int t = t0; t < t1; t += UNR) {
                CV<float, VC> p[UNR][3];
                float4 w[UNR][3];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (t + u < t1) {
                        const int64_t j3 = 3 * (int64_t)__ldg(node + t + u);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            p[u][c] = ldcv(Pc + (j3 + c) * W);
                            w[u][c] = __ldg(coef + (int64_t)(t + u) * 3 + c);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (t + u >= t1) break;
                    const float a[3][3] = {{w[u][0].x, w[u][0].y, w[u][0].z},
                                           {w[u][0].w, w[u][1].x, w[u][1].y},
                                           {w[u][1].z, w[u][1].w, w[u][2].x}};
                    const float b[3] = {w[u][2].y, w[u][2].z, w[u][2].w};
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            const float2 x = p[u][c].v[v];
#pragma unroll
                            for (int r = 0; r < 3; ++r) ffma2(sa[r][v], make_float2(a[r][c], a[r][c]), x);
                            ffma2(sb[c][v], make_float2(b[c], b[c]), x);
                        }
                }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int row = g * 3 + r;
                if (row >= n) break;
                CV<float, VC> q;
#pragma unroll
                for (int v = 0; v < VC; ++v) q.v[v] = csub(sa[r][v], cmul(s, sb[r][v]));
                stcv(Q + (int64_t)row * W + c0, q);
                const CV<float, VC> pr = ldcv(P + (int64_t)row * W + c0);
#pragma unroll
                for (int v = 0; v < VC; ++v) mu[v] = cfma(pr.v[v], q.v[v], mu[v]);
            }
        }
    }
    __shared__ float red[TY][32][VC * 2];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[ty][tx][2 * v] = mu[v].x;
        red[ty][tx][2 * v + 1] = mu[v].y;
    }
    __syncthreads();
    if (ty == 0 && cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            float s0 = 0.f, s1 = 0.f;
            for (int y = 0; y < TY; ++y) {
                s0 += red[y][tx][2 * v];
                s1 += red[y][tx][2 * v + 1];
            }
            float *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
        }
    }
}

// ---------------------------------------------------------------------------
// SELL-C-sigma variant (FP32).  The chunks of C permuted rows are split
// between the CTAs of a column slice; warp ty takes rows ty, ty + TY, ... of
// each chunk and walks its row's slots k = 0 .. len-1 at cptr + k C + r (the
// padding slots of shorter rows are skipped, not multiplied).  Results go to
// the row's original position.
// ---------------------------------------------------------------------------
template <int UNR>
__global__ void __launch_bounds__(32 * TY)
k_spmm_shifted_sell(int n, int W, int Lp, int C, int nchunks, int chunks_per_block, const int32_t *__restrict__ cptr,
                    const int32_t *__restrict__ col, const float2 *__restrict__ ab, const int32_t *__restrict__ perm,
                    const int32_t *__restrict__ rlen, const float2 *__restrict__ sig, const float2 *__restrict__ P,
                    float2 *__restrict__ Q, const int32_t *__restrict__ flag, float *__restrict__ part) {
    constexpr int VC = 2;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    float2 s = make_float2(0.f, 0.f);
    if (cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[c0 + v] == 1;
        s = sig[c0 / Lp];
    }
    float2 mu[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) mu[v] = make_float2(0.f, 0.f);
    const int ch_begin = blockIdx.y * chunks_per_block;
    const int ch_end = min(nchunks, ch_begin + chunks_per_block);
    if (act) {
        const float2 *Pc = P + c0;
        for (int ch = ch_begin; ch < ch_end; ++ch) {
            const int64_t base = __ldg(cptr + ch);
            for (int r = ty; r < C; r += TY) {
                const int prow = ch * C + r;
                if (prow >= n) break;
                const int row = __ldg(perm + prow), len = __ldg(rlen + prow);
                float2 sa[VC], sb[VC];
#pragma unroll
                for (int v = 0; v < VC; ++v) sa[v] = sb[v] = make_float2(0.f, 0.f);
                int k = 0;
                for (; k + UNR <= len; k += UNR) {
                    int cc[UNR];
                    float2 w[UNR];
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        const int64_t e = base + (int64_t)(k + u) * C + r;
                        cc[u] = __ldg(col + e);
                        w[u] = __ldg(ab + e);
                    }
                    CV<float, VC> p[UNR];
#pragma unroll
                    for (int u = 0; u < UNR; ++u) p[u] = ldcv(Pc + (int64_t)cc[u] * W);
#pragma unroll
                    for (int u = 0; u < UNR; ++u)
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            ffma2(sa[v], make_float2(w[u].x, w[u].x), p[u].v[v]);
                            ffma2(sb[v], make_float2(w[u].y, w[u].y), p[u].v[v]);
                        }
                }
                for (; k < len; ++k) {
                    const int64_t e = base + (int64_t)k * C + r;
                    const float2 w = __ldg(ab + e);
                    const CV<float, VC> p = ldcv(Pc + (int64_t)__ldg(col + e) * W);
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        ffma2(sa[v], make_float2(w.x, w.x), p.v[v]);
                        ffma2(sb[v], make_float2(w.y, w.y), p.v[v]);
                    }
                }
                CV<float, VC> q;
#pragma unroll
                for (int v = 0; v < VC; ++v) q.v[v] = csub(sa[v], cmul(s, sb[v]));
                stcv(Q + (int64_t)row * W + c0, q);
                const CV<float, VC> pr = ldcv(P + (int64_t)row * W + c0);
#pragma unroll
                for (int v = 0; v < VC; ++v) mu[v] = cfma(pr.v[v], q.v[v], mu[v]);
            }
        }
    }
    __shared__ float red[TY][32][VC * 2];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[ty][tx][2 * v] = mu[v].x;
        red[ty][tx][2 * v + 1] = mu[v].y;
    }
    __syncthreads();
    if (ty == 0 && cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            float s0 = 0.f, s1 = 0.f;
            for (int y = 0; y < TY; ++y) {
                s0 += red[y][tx][2 * v];
                s1 += red[y][tx][2 * v + 1];
            }
            float *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
        }
    }
}

// ---------------------------------------------------------------------------
// Staged (warp-specialized) variant of the FP32 row-group product.
//
// The row-group kernel above is latency-bound: every warp waits on its own
// gathers from L2, and a third of its instructions are index loads and
// address arithmetic.  Here one producer warp per CTA moves the gathered rows
// with bulk copies (the TMA engine) into shared-memory slots, and NC consumer
// warps only read shared memory and multiply:
//   * a CTA owns one column chunk (CW = 32 VC complex columns) of a range of
//     row groups; task t (one row group) goes to consumer warp t % NC, which
//     has NS private slots used in turn;
//   * a slot holds the group's gathered rows (union entry e at row e of the
//     slot, CW columns each) and its coefficient pairs in the packed layout
//     (a, a, b, b), so each entry costs one shared load of the rows, R of the
//     pairs and 2 R VC packed FP32x2 FMAs;
//   * slot handover uses two mbarriers per slot: "full" completes when the
//     producer's copies have landed (transaction count), "empty" when the
//     consumer is done with it.  Every wait is bounded (1 s); a wait that
//     gives up sets *err and the kernel winds down.
// The product and the partial sums mu = p^T q per column are those of the
// row-group kernel (same union lists, same per-column order of the FMAs
// within a row), so both kernels satisfy the same parity tests.
// ---------------------------------------------------------------------------
template <int R, int VC, int NC, int NS>
__global__ void __launch_bounds__(32 * (NC + 1), 1)
k_spmm_staged(int n, int W, int Lp, int ngroups, int gpb, int emax, const int32_t *__restrict__ gptr,
              const int32_t *__restrict__ ucol, const float4 *__restrict__ ab4, const uint8_t *__restrict__ dpos,
              const float2 *__restrict__ sig, const float2 *__restrict__ P, float2 *__restrict__ Q,
              const int32_t *__restrict__ flag, float *__restrict__ part, int gy_part, int32_t *__restrict__ err) {
    constexpr int CW = 32 * VC;
    constexpr unsigned long long LIMIT_NS = 1000000000ull;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem);   // full[NC][NS], empty[NC][NS]
    const size_t slot_bytes = ((size_t)emax * CW * 8 + (size_t)emax * R * 16 + 127) & ~(size_t)127;
    unsigned char *slots = smem + 128 * ((2 * NC * NS * 8 + 127) / 128);
    float *red = reinterpret_cast<float *>(slots + NC * NS * slot_bytes);   // [NC][32][2 VC]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * CW;
    const int cw = min(CW, W - c0);
    const int cl = c0 + lane * VC;   // first column of this lane (consumers)
    const bool live = lane * VC < cw;
    const int g_begin = blockIdx.y * gpb;
    const int T = max(0, min(ngroups, g_begin + gpb) - g_begin);
    bool act = false;
    if (warp < NC && live) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[cl + v] == 1;
    }
    // The partial sums have gy_part rows (the layout the reductions read);
    // this grid has gridDim.y <= gy_part of them, and the CTAs of row 0 zero
    // the rest for their columns.
    if (blockIdx.y == 0 && warp == 0 && live)
        for (int yy = gridDim.y; yy < gy_part; ++yy)
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                float *o = part + ((int64_t)yy * W + cl + v) * 4;
                o[0] = 0.f;
                o[1] = 0.f;
            }
    if (!__syncthreads_or(act)) {
        // no active column in the chunk: zero partial sums keep the per-column sums complete
        if (warp == 0 && live)
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                float *o = part + ((int64_t)blockIdx.y * W + cl + v) * 4;
                o[0] = 0.f;
                o[1] = 0.f;
            }
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * NC * NS; ++i) mbar_init(bars + i, 1);
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == NC) {   // ---- producer
        // Rounds of NC consecutive groups (one per consumer, slot k % NS).  A
        // round's union entries are one contiguous range of the lists, so the
        // lanes load its column indices together (coalesced) and each lane
        // issues the copies of every 32nd entry; lane w < NC handles the
        // slot handshake and the coefficient copy of consumer w.
        const unsigned row_bytes = (unsigned)cw * 8u;
        const int rounds = (T + NC - 1) / NC;
        for (int k = 0; k < rounds; ++k) {
            const int s = k % NS, u = k / NS;
            const int t = k * NC + lane;                 // this lane's task (lane < NC)
            const bool mine = lane < NC && t < T;
            int e0 = 0, ne = 0;
            if (mine) {
                const int g = g_begin + t;
                e0 = __ldg(gptr + g);
                ne = __ldg(gptr + g + 1) - e0;
            }
            int ok = 1;
            if (mine && u > 0) ok = mbar_wait_bounded(bars + NC * NS + lane * NS + s, (u - 1) & 1, LIMIT_NS);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            unsigned long long *full = bars + lane * NS + s;
            if (mine) mbar_expect_tx(full, row_bytes * (unsigned)ne + (unsigned)ne * R * 16u);
            // entry prefix over the round's groups (lanes 0..NC-1 hold ne)
            int pre = ne;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, off);
                if (lane >= off) pre += y;
            }
            const int total = __shfl_sync(0xffffffffu, pre, 31);
            const int ebase = __shfl_sync(0xffffffffu, e0, 0);   // first entry of the round
            int pq[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) pq[q] = __shfl_sync(0xffffffffu, pre, q);
            __syncwarp();
            for (int j = lane; j < total; j += 32) {
                // consumer w of entry j: pq[w - 1] <= j < pq[w]
                int w = 0, start = 0;
#pragma unroll
                for (int q = 0; q < NC - 1; ++q)
                    if (pq[q] <= j) {
                        w = q + 1;
                        start = pq[q];
                    }
                unsigned char *slot = slots + (size_t)(w * NS + s) * slot_bytes;
                bulk_g2s(slot + (size_t)(j - start) * CW * 8, P + (int64_t)__ldg(ucol + ebase + j) * W + c0, row_bytes,
                         bars + w * NS + s);
            }
            if (mine)
                bulk_g2s(slots + (size_t)(lane * NS + s) * slot_bytes + (size_t)emax * CW * 8, ab4 + (int64_t)e0 * R,
                         (unsigned)ne * R * 16u, full);
        }
        return;
    }

    // ---- consumers
    const float2 sg = sig[min(cl, W - 1) / Lp];
    float2 mu[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) mu[v] = make_float2(0.f, 0.f);
    for (int k = 0;; ++k) {
        const int t = warp + k * NC;
        if (t >= T) break;
        const int s = k % NS, u = k / NS;
        unsigned long long *full = bars + warp * NS + s;
        unsigned long long *empty = bars + NC * NS + warp * NS + s;
        const bool ok = mbar_wait_bounded(full, u & 1, LIMIT_NS);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) atomicExch(err, 2);
            break;
        }
        const int g = g_begin + t;
        const int ne = __ldg(gptr + g + 1) - __ldg(gptr + g);
        const unsigned char *slot = slots + (size_t)(warp * NS + s) * slot_bytes;
        const float2 *xs = reinterpret_cast<const float2 *>(slot) + lane * VC;
        const float4 *ws = reinterpret_cast<const float4 *>(slot + (size_t)emax * CW * 8);
        float2 sa[R][VC], sb[R][VC];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < VC; ++v) sa[r][v] = sb[r][v] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int e = 0; e < ne; ++e) {
            float2 x[VC];
            if constexpr (VC == 2) {
                const float4 t4 = *reinterpret_cast<const float4 *>(xs + (size_t)e * CW);
                x[0] = make_float2(t4.x, t4.y);
                x[1] = make_float2(t4.z, t4.w);
            } else {
                x[0] = xs[(size_t)e * CW];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 w4 = ws[e * R + r];
                const float2 aa = make_float2(w4.x, w4.y), bb = make_float2(w4.z, w4.w);
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    ffma2(sa[r][v], aa, x[v]);
                    ffma2(sb[r][v], bb, x[v]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = g * R + r;
            if (row >= n) break;
            const int dp = __ldg(dpos + (int64_t)g * R + r);
            float2 q[VC];
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                q[v] = csub(sa[r][v], cmul(sg, sb[r][v]));
                const float2 pr = xs[(size_t)dp * CW + v];
                mu[v] = cfma(pr, q[v], mu[v]);
            }
            if (live) {
                if constexpr (VC == 2)
                    *reinterpret_cast<float4 *>(Q + (int64_t)row * W + cl) = make_float4(q[0].x, q[0].y, q[1].x, q[1].y);
                else
                    Q[(int64_t)row * W + cl] = q[0];
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty);
    }
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[(warp * 32 + lane) * 2 * VC + 2 * v] = mu[v].x;
        red[(warp * 32 + lane) * 2 * VC + 2 * v + 1] = mu[v].y;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NC * 32) : "memory");   // consumers only
    if (warp == 0 && live) {
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            float s0 = 0.f, s1 = 0.f;
            for (int w = 0; w < NC; ++w) {
                s0 += red[(w * 32 + lane) * 2 * VC + 2 * v];
                s1 += red[(w * 32 + lane) * 2 * VC + 2 * v + 1];
            }
            float *o = part + ((int64_t)blockIdx.y * W + cl + v) * 4;
            o[0] = s0;
            o[1] = s1;
        }
    }
}

// Shapes of the staged kernel by rows per group: two complex columns per
// lane and 8 consumers for R <= 2; one column per lane and 4 consumers for
// longer groups (3-dof elasticity: 81 union entries per group).
template <int R> struct StagedShape;
template <> struct StagedShape<2> { static constexpr int VC = 2, NC = 8, NS = 2; };
template <> struct StagedShape<3> { static constexpr int VC = 1, NC = 4, NS = 2; };
template <> struct StagedShape<4> { static constexpr int VC = 1, NC = 4, NS = 2; };

template <int R>
static size_t staged_smem_bytes(int emax) {
    using S = StagedShape<R>;
    const size_t slot = ((size_t)emax * 32 * S::VC * 8 + (size_t)emax * R * 16 + 127) & ~(size_t)127;
    return 128 * ((2 * S::NC * S::NS * 8 + 127) / 128) + S::NC * S::NS * slot + (size_t)S::NC * 32 * 2 * S::VC * 4;
}

size_t spmm_staged_smem(const DevPencil &A) {
    if (A.rg_rows < 2 || A.rg_rows > 4 || !A.rg_ab4 || !A.rg_dpos || A.rg_emax < 1 || A.rg_emax > 255) return 0;
    size_t b = 0;
    if (A.rg_rows == 2) b = staged_smem_bytes<2>(A.rg_emax);
    else if (A.rg_rows == 3) b = staged_smem_bytes<3>(A.rg_emax);
    else b = staged_smem_bytes<4>(A.rg_emax);
    return b <= 227 * 1024 ? b : 0;
}

template <int R>
static void launch_staged(Ctx &ctx, const KrylovDims &d, const DevPencil &A, const float2 *sig, const float2 *P,
                          float2 *Q, const int32_t *flag, float *part, int gy) {
    using S = StagedShape<R>;
    constexpr int CW = 32 * S::VC;
    const int W = d.W();
    const size_t smem = staged_smem_bytes<R>(A.rg_emax);
    static bool raised[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !raised[dev]) {   // per device, before the first launch there
        cudaFuncSetAttribute(k_spmm_staged<R, S::VC, S::NC, S::NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        raised[dev] = true;
    }
    // about two waves of CTAs, each streaming a long contiguous range of row
    // groups (long producer/consumer pipelines); at most gy rows of partials
    const int gx = (W + CW - 1) / CW;
    const int per_sm = std::max(1, (int)((228 * 1024) / (smem + 1024)));
    int gy2 = A.spmm_gpb > 0 ? (A.rg_ngroups + A.spmm_gpb - 1) / A.spmm_gpb
                             : (2 * per_sm * ctx.sm_count + gx - 1) / gx;
    gy2 = std::max(1, std::min(gy2, std::min(gy, A.rg_ngroups)));
    const int gpb = (A.rg_ngroups + gy2 - 1) / gy2;
    dim3 grid(gx, gy2);
    k_spmm_staged<R, S::VC, S::NC, S::NS><<<grid, 32 * (S::NC + 1), smem, ctx.stream>>>(
        d.n, W, d.Lp, A.rg_ngroups, gpb, A.rg_emax, A.rg_ptr, A.rg_col, A.rg_ab4, A.rg_dpos, sig, P, Q, flag, part,
        gy, A.dev_err);
}

// ---------------------------------------------------------------------------
// update: r -= alpha q ; U += Re(ua p) ; partial |r|^2 and, with the Jacobi
// preconditioner (JAC), z = M^{-1} r and partial r^T z (with multigrid the
// cycle that follows forms z and r^T z).
// One thread owns VC columns of one pole-slot c and walks all N poles, so the
// pole sum of the filter is formed in registers.
// ---------------------------------------------------------------------------
// With the multigrid preconditioner (MGY) the update also writes y = D r
// (D: the cycle's finest damped Jacobi diagonal) over Q, which is dead once
// read here: the block the cycle's gathered products read.
template <typename T, int VC, int NP, bool JAC, bool MGY>
__global__ void __launch_bounds__(32 * TY)
k_update(int n, int W, int Lp, int N, cplx<T> *__restrict__ R, const cplx<T> *__restrict__ P,
         cplx<T> *__restrict__ Q, const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ alpha,
         const cplx<T> *__restrict__ ua, const int32_t *__restrict__ flag, T *__restrict__ U,
         T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ngl = Lp / VC;
    const int cgl = blockIdx.x * 32 + tx;
    const int c0 = cgl * VC;
    const bool live = cgl < ngl;
    unsigned actmask = 0;   // bit j*VC + v
    if (live) {
#pragma unroll
        for (int j = 0; j < NP; ++j)
            if (j < N)
#pragma unroll
                for (int v = 0; v < VC; ++v)
                    if (flag[j * Lp + c0 + v] == 1) actmask |= 1u << (j * VC + v);
    }
    T acc[NP][VC][3];
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int v = 0; v < VC; ++v) acc[j][v][0] = acc[j][v][1] = acc[j][v][2] = (T)0;

    if (actmask) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            T u[VC];
#pragma unroll
            for (int v = 0; v < VC; ++v) u[v] = (T)0;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                if (j >= N) break;
                const unsigned mj = (actmask >> (j * VC)) & ((1u << VC) - 1);
                if (!mj) continue;
                const int64_t base = (int64_t)row * W + j * Lp + c0;
                CV<T, VC> r = ldcv(R + base);
                const CV<T, VC> p = ldcv(P + base);
                const CV<T, VC> q = ldcv(Q + base);
                C dv = mk((T)0, (T)0);
                if (JAC || MGY) dv = dinv[(int64_t)row * N + j];
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    if (!(mj & (1u << v))) continue;
                    const C a = alpha[j * Lp + c0 + v];
                    const C w = ua[j * Lp + c0 + v];
                    r.v[v] = csub(r.v[v], cmul(a, q.v[v]));
                    u[v] += w.x * p.v[v].x - w.y * p.v[v].y;
                    if (JAC) {
                        const C z = cmul(dv, r.v[v]);
                        const C rz = cmul(r.v[v], z);
                        acc[j][v][0] += rz.x;
                        acc[j][v][1] += rz.y;
                    }
                    acc[j][v][2] += cabs2(r.v[v]);
                }
                stcv(R + base, r);
                if (MGY) {
                    CV<T, VC> y;
#pragma unroll
                    for (int v = 0; v < VC; ++v) y.v[v] = cmul(dv, r.v[v]);
                    stcv(Q + base, y);
                }
            }
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                bool any = false;
#pragma unroll
                for (int j = 0; j < NP; ++j)
                    if (j < N) any |= (actmask >> (j * VC + v)) & 1u;
                if (any) U[(int64_t)row * Lp + c0 + v] += u[v];
            }
        }
    }
    __shared__ T red[TY][32][VC * 3];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        if (j >= N) break;
#pragma unroll
        for (int v = 0; v < VC; ++v)
#pragma unroll
            for (int s = 0; s < 3; ++s) red[ty][tx][v * 3 + s] = acc[j][v][s];
        __syncthreads();
        if (ty == 0 && live) {
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                T s0 = 0, s1 = 0, s2 = 0;
                for (int y = 0; y < TY; ++y) {
                    s0 += red[y][tx][v * 3 + 0];
                    s1 += red[y][tx][v * 3 + 1];
                    s2 += red[y][tx][v * 3 + 2];
                }
                T *o = part + ((int64_t)blockIdx.y * W + j * Lp + c0 + v) * 4;
                if (JAC) {
                    o[0] = s0;
                    o[1] = s1;
                }
                o[2] = s2;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// direction: p = z + beta p, z = Z (multigrid) or M^{-1} r (Jacobi); init: p = z
// ---------------------------------------------------------------------------
template <typename T, int VC, bool MGZ>
__global__ void __launch_bounds__(32 * TY)
k_direction(int n, int W, int Lp, int N, const cplx<T> *__restrict__ R, const cplx<T> *__restrict__ Z,
            cplx<T> *__restrict__ P, const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ beta,
            const int32_t *__restrict__ flag, int init) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    if (cg >= ng) return;
    const int c0 = cg * VC;
    const int j = c0 / Lp;
    bool act[VC];
    bool any = false;
    C b[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        act[v] = flag[c0 + v] == 1;
        any |= act[v];
        b[v] = init ? mk((T)0, (T)0) : beta[c0 + v];
    }
    if (!any) return;
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        CV<T, VC> z;
        if (MGZ) {
            z = ldcv(Z + base);
        } else {
            const C dv = dinv[(int64_t)row * N + j];
            z = ldcv(R + base);
#pragma unroll
            for (int v = 0; v < VC; ++v) z.v[v] = cmul(dv, z.v[v]);
        }
        CV<T, VC> p;
        if (init) {
            p = z;
        } else {
            p = ldcv(P + base);
#pragma unroll
            for (int v = 0; v < VC; ++v)
                if (act[v]) p.v[v] = cfma(b[v], p.v[v], z.v[v]);
        }
        stcv(P + base, p);
    }
}

// ---------------------------------------------------------------------------
// per-column reductions (one warp per column, lanes over row groups, FP64)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void warp_sum3(const T *part, int gy, int W, int col, double &s0, double &s1,
                                          double &s2) {
    const int lane = threadIdx.x & 31;
    s0 = s1 = s2 = 0.0;
    for (int g = lane; g < gy; g += 32) {
        const T *o = part + ((int64_t)g * W + col) * 4;
        s0 += (double)o[0];
        s1 += (double)o[1];
        s2 += (double)o[2];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
}

template <typename T>
__global__ void k_reduce_init(int W, int gy, const T *__restrict__ part, KrylovScalars<T> s) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    if ((threadIdx.x & 31) == 0) {
        s.rho[col] = mk((T)s0, (T)s1);
        s.bnorm2[col] = s2;
        s.rnorm2[col] = s2;
        s.iters[col] = 0;
        if (s.flag[col] == 1 && !(s2 > 0.0)) s.flag[col] = 0;   // zero right-hand side: y = 0
    }
}

template <typename T>
__global__ void k_reduce_alpha(int W, int gy, const T *__restrict__ part, KrylovScalars<T> s) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    if ((threadIdx.x & 31) == 0 && s.flag[col] == 1) {
        const double den = s0 * s0 + s1 * s1;
        const double rr = (double)s.rho[col].x, ri = (double)s.rho[col].y;
        if (!(den > 0.0) || !isfinite(den)) {
            s.flag[col] = 2;
            return;
        }
        // alpha = rho / mu
        const double ar = (rr * s0 + ri * s1) / den;
        const double ai = (ri * s0 - rr * s1) / den;
        s.alpha[col] = mk((T)ar, (T)ai);
        const double2 c = s.coef[col];
        s.ua[col] = mk((T)(2.0 * (c.x * ar - c.y * ai)), (T)(2.0 * (c.x * ai + c.y * ar)));
    }
}

template <typename T>
__global__ void k_reduce_beta(int W, int gy, const T *__restrict__ part, KrylovScalars<T> s, double tol2,
                              int maxit) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    if ((threadIdx.x & 31) == 0 && s.flag[col] == 1) {
        const int it = s.iters[col] + 1;
        s.iters[col] = it;
        s.rnorm2[col] = s2;
        if (s2 <= tol2 * s.bnorm2[col]) {
            s.flag[col] = 0;
            return;
        }
        if (it >= maxit) {
            s.flag[col] = 3;
            return;
        }
        const double rr = (double)s.rho[col].x, ri = (double)s.rho[col].y;
        const double den = rr * rr + ri * ri;
        if (!(den > 0.0) || !isfinite(s2)) {
            s.flag[col] = 2;
            return;
        }
        // beta = rho' / rho
        const double br = (s0 * rr + s1 * ri) / den;
        const double bi = (s1 * rr - s0 * ri) / den;
        s.beta[col] = mk((T)br, (T)bi);
        s.rho[col] = mk((T)s0, (T)s1);
    }
}

__global__ void k_count_active(int W, const int32_t *__restrict__ flag, int32_t *__restrict__ count) {
    __shared__ int tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < W; i += blockDim.x) c += flag[i] == 1;
    atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) *count = tot;
}

template <typename T>
__global__ void k_reduce_mu(int W, int gy, const T *__restrict__ part, cplx<T> *__restrict__ mu, int Lp, int m) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    const int j = col / Lp, c = col - j * Lp;
    if ((threadIdx.x & 31) == 0 && c < m) mu[j * m + c] = mk((T)s0, (T)s1);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int krylov_row_groups(const Ctx &ctx, const KrylovDims &d, int prec_fp32) {
    // The update kernel has the narrowest grid (one pole-slot of Lp columns in
    // x), so the shared row-group count is sized for it: ~8 CTAs per SM.
    const int VC = prec_fp32 ? 2 : 1;
    const int gx = (d.Lp / VC + 31) / 32;
    const int target = ctx.sm_count * 8;
    int gy = target / (gx > 0 ? gx : 1);
    const int maxgy = (d.n + TY - 1) / TY;
    if (gy > maxgy) gy = maxgy;
    if (gy < 1) gy = 1;
    return gy;
}

template <typename T>
void krylov_dinv(Ctx &ctx, const DevPencil &A, const PoleSet<T> &ps, int precond, cplx<T> *dinv) {
    const int64_t tot = (int64_t)A.n * ps.N;
    ctx.before(KC_KRYLOV_INIT, (double)tot * sizeof(cplx<T>) + 16.0 * A.n, 0);
    k_dinv<T><<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(A.n, ps.N, A.diag_a, A.diag_b, ps, precond, dinv);
    ctx.after();
}

template <typename T>
void krylov_init(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, const double *rhs, int64_t ldr,
                 const cplx<double> *rhs_c) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_INIT, 2 * vb + (double)d.n * d.m * 8, 0);
    k_init<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, d.m, rhs, ldr, rhs_c, kb.dinv, kb.R, kb.P,
                                                  kb.s.flag, kb.s.part);
    ctx.after();
}

template <typename T>
void krylov_reduce_init(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb) {
    const int W = d.W();
    ctx.before(KC_KRYLOV_REDUCE, (double)kb.gy * W * 4 * sizeof(T), 0);
    k_reduce_init<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, kb.gy, kb.s.part, kb.s);
    ctx.after();
}

template <typename T>
void krylov_spmm(Ctx &ctx, const KrylovDims &d, const DevPencil &A, const cplx<T> *sig, const cplx<T> *P,
                 cplx<T> *Q, const int32_t *flag, T *part, int gy) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    // algorithmic bytes: pattern + (a,b) pairs once, P read once and Q written
    // once for the active columns (converged columns are skipped)
    const double bytes = 4.0 * (d.n + 1) + (double)A.nnz * (4 + 2 * sizeof(T)) +
                         2.0 * d.n * W * d.frac * sizeof(cplx<T>);
    const double flops = 8.0 * (double)A.nnz * W * d.frac;
    const auto *abp =
        reinterpret_cast<const typename ABT<T>::type *>(sizeof(T) == 4 ? (const void *)A.ab32 : (const void *)A.ab64);
    ctx.before(KC_SHIFTED_SPMM, bytes, flops);
    if constexpr (sizeof(T) == 4) {
        if (A.spmm_kind == SPMM_NODEBLOCK && A.nb_coef) {
            const int gpb = (A.rg_ngroups + gy - 1) / gy;
            // one neighbour node in flight per warp (three 16-B gathers and
            // three coefficient loads): two in flight measured 30% slower
            k_spmm_shifted_nb<1><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, A.rg_ngroups, gpb, A.nb_ptr, A.nb_node,
                                                                 A.nb_coef, reinterpret_cast<const float2 *>(sig), P,
                                                                 Q, flag, part);
            ctx.after();
            return;
        }
        if (A.spmm_kind == SPMM_SELL && A.sell_ab) {
            const int cpb = (A.sell_nchunks + gy - 1) / gy;
            k_spmm_shifted_sell<4><<<grid, block, 0, ctx.stream>>>(
                d.n, W, d.Lp, A.sell_c, A.sell_nchunks, cpb, A.sell_cptr, A.sell_col, A.sell_ab, A.sell_perm,
                A.sell_rlen, reinterpret_cast<const float2 *>(sig), P, Q, flag, part);
            ctx.after();
            return;
        }
        if (A.spmm_kind == SPMM_STAGED && spmm_staged_smem(A) > 0) {
            const float2 *s2 = reinterpret_cast<const float2 *>(sig);
            if (A.rg_rows == 2) launch_staged<2>(ctx, d, A, s2, P, Q, flag, part, gy);
            else if (A.rg_rows == 3) launch_staged<3>(ctx, d, A, s2, P, Q, flag, part, gy);
            else launch_staged<4>(ctx, d, A, s2, P, Q, flag, part, gy);
            ctx.after();
            return;
        }
    }
    if (A.rg_rows > 1) {
        const int gpb = (A.rg_ngroups + gy - 1) / gy;
        const auto *uab = reinterpret_cast<const typename ABT<T>::type *>(sizeof(T) == 4 ? (const void *)A.rg_ab32
                                                                                          : (const void *)A.rg_ab64);
#define RGL(RR)                                                                                                  \
    k_spmm_shifted_rg<T, VC, RR, 4><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, A.rg_ngroups, gpb, A.rg_ptr,     \
                                                                    A.rg_col, uab, sig, P, Q, flag, part)
        if (A.rg_rows == 2) RGL(2);
        else if (A.rg_rows == 3) RGL(3);
        else RGL(4);
#undef RGL
    } else {
        const int rpb = (d.n + gy - 1) / gy;
        k_spmm_shifted_rb<T, VC, 4><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, rpb, A.rowptr, A.col, abp, sig, P,
                                                                     Q, flag, part);
    }
    ctx.after();
}

template <typename T>
void krylov_reduce_alpha(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb) {
    const int W = d.W();
    ctx.before(KC_KRYLOV_REDUCE, (double)kb.gy * W * 4 * sizeof(T), 0);
    k_reduce_alpha<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, kb.gy, kb.s.part, kb.s);
    ctx.after();
}

template <typename T, int NP>
static void launch_update(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((d.Lp / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_UPDATE,
               (kb.mgd ? 5 : 4) * vb + 2.0 * d.n * d.Lp * sizeof(T) + (double)d.n * d.N * sizeof(cplx<T>),
               16.0 * d.n * W * d.frac);
    if (kb.Z && kb.mgd)
        k_update<T, VC, NP, false, true><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, kb.P, kb.Q, kb.mgd,
                                                                          kb.s.alpha, kb.s.ua, kb.s.flag, kb.Uacc,
                                                                          kb.s.part);
    else if (kb.Z)
        k_update<T, VC, NP, false, false><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, kb.P, kb.Q,
                                                                           kb.dinv, kb.s.alpha, kb.s.ua, kb.s.flag,
                                                                           kb.Uacc, kb.s.part);
    else
        k_update<T, VC, NP, true, false><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, kb.P, kb.Q, kb.dinv,
                                                                          kb.s.alpha, kb.s.ua, kb.s.flag, kb.Uacc,
                                                                          kb.s.part);
    ctx.after();
}

template <typename T>
void krylov_update(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb) {
    if (d.N <= 2)
        launch_update<T, 2>(ctx, d, kb);
    else if (d.N <= 4)
        launch_update<T, 4>(ctx, d, kb);
    else if (d.N <= 8)
        launch_update<T, 8>(ctx, d, kb);
    else
        launch_update<T, 16>(ctx, d, kb);
}

template <typename T>
void krylov_reduce_beta(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, double tol2, int maxit) {
    const int W = d.W();
    ctx.before(KC_KRYLOV_REDUCE, (double)kb.gy * W * 4 * sizeof(T), 0);
    k_reduce_beta<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, kb.gy, kb.s.part, kb.s, tol2, maxit);
    ctx.after();
}

template <typename T>
void krylov_direction(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, int init) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_DIR, (init ? 2 : 3) * vb + (kb.Z ? 0.0 : (double)d.n * d.N * sizeof(cplx<T>)),
               10.0 * d.n * W * d.frac);
    if (kb.Z)
        k_direction<T, VC, true><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, kb.Z, kb.P, kb.dinv,
                                                                 kb.s.beta, kb.s.flag, init);
    else
        k_direction<T, VC, false><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, kb.Z, kb.P, kb.dinv,
                                                                  kb.s.beta, kb.s.flag, init);
    ctx.after();
}

void krylov_count_active(Ctx &ctx, int W, const int32_t *flag, int32_t *count) {
    ctx.before(KC_KRYLOV_REDUCE, 4.0 * W, 0);
    k_count_active<<<1, 256, 0, ctx.stream>>>(W, flag, count);
    ctx.after();
}

template <typename T>
void krylov_reduce_mu(Ctx &ctx, const KrylovDims &d, const T *part, int gy, cplx<T> *mu) {
    const int W = d.W();
    ctx.before(KC_KRYLOV_REDUCE, (double)gy * W * 4 * sizeof(T), 0);
    k_reduce_mu<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, gy, part, mu, d.Lp, d.m);
    ctx.after();
}

#define INST(T)                                                                                                \
    template void krylov_dinv<T>(Ctx &, const DevPencil &, const PoleSet<T> &, int, cplx<T> *);                \
    template void krylov_init<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, const double *, int64_t,       \
                                 const cplx<double> *);                                                       \
    template void krylov_reduce_init<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &);                       \
    template void krylov_spmm<T>(Ctx &, const KrylovDims &, const DevPencil &, const cplx<T> *,               \
                                 const cplx<T> *, cplx<T> *, const int32_t *, T *, int);                       \
    template void krylov_reduce_alpha<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &);                      \
    template void krylov_update<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &);                            \
    template void krylov_reduce_beta<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, double, int);          \
    template void krylov_direction<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, int);                    \
    template void krylov_reduce_mu<T>(Ctx &, const KrylovDims &, const T *, int, cplx<T> *);
INST(float)
INST(double)
#undef INST

}  // namespace slrf
