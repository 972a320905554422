// Multigrid V/W-cycle preconditioner for the block COCG of krylov.cu.
//
// One cycle is applied to all (pole, column) systems at once: every level
// keeps the column-block layout of the Krylov state (complex n_l x W, row
// stride W, pole j in columns [j*Lp, j*Lp + Lp)), the level operator of pole
// j is M_l = A_l - sigma_j B_l with the Galerkin pencil of mg_setup.cpp, and
// the smoother is damped Jacobi, D_lj = omega_l / (a_ii - sigma_j b_ii) with
// omega_l = omega / rho(D_l^{-1} A_l) (4/3 by default: the high-frequency
// modes are damped whatever the level's diagonal dominance).  With
// R_l = P_l^T, equal pre- and post-smoothing and the exact coarsest solve
// V (Lambda - sigma_j)^{-1} V^T, the cycle is a complex symmetric linear
// operator, as COCG requires of its preconditioner.
//
// Finest level, one sweep each side with the pre-smoothing from zero:
//   x = D r,  r1 = P^T (r - M x),  e = cycle(1, r1),
//   z1 = x + P e,  z = z1 + D (r - M z1).
// With F = (M - D^{-1}) P (a pair matrix like the pencil's: F_a - sigma F_b)
// the two ends fold into one gathered product each, and neither the fine
// residual nor z1 is ever stored:
//   r1 = -F^T y                             k_mg_sspmm<DOWN>  (coarse rows)
//   z  = D (2 r - M y - F e),  r^T z        k_mg_sspmm<UP>    (fine row groups)
// with y = D r formed once (fused into the Krylov update that produces r).
// (P^T (I - M D) = -((M - D^{-1}) P)^T D and (I - D M) P = -D F.)  The fine
// level is read twice and written once per cycle.
// Coarser levels run nu sweeps on each side and gamma coarse visits
// (gamma = 2: W-cycle) with materialised iterates.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "internal.h"

namespace slrf {

namespace {

constexpr int TY = 8;

template <typename T> struct VecN;
template <> struct VecN<float> { static constexpr int VC = 2; };
template <> struct VecN<double> { static constexpr int VC = 1; };

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

enum { MG_RESID = 0, MG_SMOOTH = 1, MG_DOWN = 2, MG_UP = 3 };
enum { MG_RESTRICT = 0, MG_PROLONG_ADD = 1 };

// Column group of a thread: VC consecutive columns of one pole (Lp is even).
template <int VC>
__device__ __forceinline__ bool col_active(const int32_t *flag, int c0) {
    bool a = false;
#pragma unroll
    for (int v = 0; v < VC; ++v) a |= flag[c0 + v] == 1;
    return a;
}

// One segment of a row group's union column list [e0, e1): gathers x_k = X[k]
// and accumulates sa[r] += a_rk x_k, sb[r] += b_rk x_k.  Full batches of UNR
// entries issue all their index loads, then all their gathers, then the FMAs
// (UNR gathers in flight per warp), and a remainder loop takes the rest.
template <typename T, int VC, int R, int UNR>
__device__ __forceinline__ void seg_accum(int e0, int e1, const int32_t *__restrict__ ucol,
                                          const cplx<T> *__restrict__ uab, const cplx<T> *__restrict__ X, int W,
                                          int c0, cplx<T> (&sa)[R][VC], cplx<T> (&sb)[R][VC]) {
    using C = cplx<T>;
    const cplx<T> *Xc = X + c0;
    int e = e0;
    for (; e + UNR <= e1; e += UNR) {
        int cc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) cc[u] = __ldg(ucol + e + u);
        CV<T, VC> x[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) x[u] = ldcv(Xc + (int64_t)cc[u] * W);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const C w = __ldg(uab + (int64_t)(e + u) * R + r);
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    sa[r][v].x = fma(w.x, x[u].v[v].x, sa[r][v].x);
                    sa[r][v].y = fma(w.x, x[u].v[v].y, sa[r][v].y);
                    sb[r][v].x = fma(w.y, x[u].v[v].x, sb[r][v].x);
                    sb[r][v].y = fma(w.y, x[u].v[v].y, sb[r][v].y);
                }
            }
    }
    for (; e < e1; ++e) {
        const CV<T, VC> x = ldcv(Xc + (int64_t)__ldg(ucol + e) * W);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const C w = __ldg(uab + (int64_t)e * R + r);
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                sa[r][v].x = fma(w.x, x.v[v].x, sa[r][v].x);
                sa[r][v].y = fma(w.x, x.v[v].y, sa[r][v].y);
                sb[r][v].x = fma(w.y, x.v[v].x, sb[r][v].x);
                sb[r][v].y = fma(w.y, x.v[v].y, sb[r][v].y);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Shifted level product in row-group form (R rows per group share one union
// column list with R (a, b) pairs per entry; R = 1 is plain CSR), with
// y = (sa - sigma sb) the gathered shifted product of the group's rows:
//   RESID : out = r - M x
//   SMOOTH: out = x + D (r - M x), optional partial r^T out per column
//   DOWN  : out = -F^T y                   (rows: coarse; gathers: fine y = D r)
//   UP    : out = D (2 r - M y - F e),      (gathers y = D r and, by the
//           second list, F over e), optional partial r^T out
// The finest-level block y = D r is formed once per cycle (by the Krylov
// update, or k_mg_scale), so the gathers carry no per-entry diagonal.
// ---------------------------------------------------------------------------
// 40 registers, 6 resident CTAs per SM: measured on the 2D bench, the finest
// UP product of row groups runs faster there (282 us per launch, with some
// spills) than at 64 registers and 4 CTAs without spills (323 us).
template <typename T, int VC, int R, int MODE>
__global__ void __launch_bounds__(32 * TY, 6)
k_mg_sspmm(int n, int W, int Lp, int N, int ngroups, const int32_t *__restrict__ gptr,
           const int32_t *__restrict__ ucol, const cplx<T> *__restrict__ uab, const cplx<T> *__restrict__ sig,
           const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ X, const cplx<T> *__restrict__ Rv,
           cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag, T *__restrict__ part,
           const int32_t *__restrict__ g2ptr, const int32_t *__restrict__ u2col, const cplx<T> *__restrict__ u2ab,
           const cplx<T> *__restrict__ X2) {
    using C = cplx<T>;
    constexpr bool DOTS = MODE == MG_SMOOTH || MODE == MG_UP;
    constexpr int UNR = (MODE == MG_DOWN) ? 4 : 2;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    int j = 0;
    C s = mk((T)0, (T)0);
    if (cg < ng) {
        act = col_active<VC>(flag, c0);
        j = c0 / Lp;
        s = sig[j];
    }
    C rz[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) rz[v] = mk((T)0, (T)0);
    // Row groups are dealt grid-strided: the CTAs resident at any moment then
    // work on one contiguous band of rows, whose gathered neighbours stay in
    // L2 (contiguous slabs per CTA scattered the neighbourhoods over ~280 MB
    // and re-read 1.6-1.9x the algorithmic bytes from DRAM; 124 -> 109 ms per
    // 2D solve)
    if (act) {
        for (int g = blockIdx.y * TY + ty; g < ngroups; g += gridDim.y * TY) {
            if constexpr (MODE == MG_UP) {
                // the grid's next band of row groups: this CTA's part of it,
                // whole rows of the gathered block, moved into L2 ahead of use
                if (blockIdx.x == 0 && ty == 0) {
                    const int64_t gn = (int64_t)g + (int64_t)gridDim.y * TY;
                    if (gn < ngroups) {
                        const int64_t r0 = gn * R, r1 = min((int64_t)n, r0 + (int64_t)TY * R);
                        l2_prefetch_warp(X + r0 * W, (r1 - r0) * W * (int64_t)sizeof(C), tx);
                    }
                }
            }
            C sa[R][VC], sb[R][VC];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < VC; ++v) sa[r][v] = sb[r][v] = mk((T)0, (T)0);
            seg_accum<T, VC, R, UNR>(__ldg(gptr + g), __ldg(gptr + g + 1), ucol, uab, X, W, c0, sa, sb);
            if constexpr (MODE == MG_UP)
                seg_accum<T, VC, R, UNR>(__ldg(g2ptr + g), __ldg(g2ptr + g + 1), u2col, u2ab, X2, W, c0, sa, sb);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = g * R + r;
                if (row >= n) break;
                const int64_t base = (int64_t)row * W + c0;
                CV<T, VC> o;
                if constexpr (MODE == MG_DOWN) {
#pragma unroll
                    for (int v = 0; v < VC; ++v) o.v[v] = csub(cmul(s, sb[r][v]), sa[r][v]);
                } else {
                    const CV<T, VC> rr = ldcv(Rv + base);
                    if constexpr (MODE == MG_RESID) {
#pragma unroll
                        for (int v = 0; v < VC; ++v) o.v[v] = csub(rr.v[v], csub(sa[r][v], cmul(s, sb[r][v])));
                    } else {
                        const C d = dinv[(int64_t)row * N + j];
                        CV<T, VC> xr;
                        if constexpr (MODE == MG_SMOOTH) xr = ldcv(X + base);
#pragma unroll
                        for (int v = 0; v < VC; ++v) {
                            const C y = csub(sa[r][v], cmul(s, sb[r][v]));
                            if constexpr (MODE == MG_SMOOTH)
                                o.v[v] = cfma(d, csub(rr.v[v], y), xr.v[v]);
                            else
                                o.v[v] = cmul(d, csub(cadd(rr.v[v], rr.v[v]), y));
                            rz[v] = cfma(rr.v[v], o.v[v], rz[v]);
                        }
                    }
                }
                stcv(Out + base, o);
            }
        }
    }
    if constexpr (DOTS) {
        if (part == nullptr) return;   // uniform over the block
        __shared__ T red[TY][32][VC * 2];
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            red[ty][tx][2 * v] = rz[v].x;
            red[ty][tx][2 * v + 1] = rz[v].y;
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
}

// ---------------------------------------------------------------------------
// Grid transfers below the finest level with a real CSR matrix (P or P^T),
// all W columns:
//   RESTRICT   : out = M x
//   PROLONG_ADD: out += M x           (out is the level iterate, updated in place)
// ---------------------------------------------------------------------------
template <typename T, int VC, int MODE>
__global__ void __launch_bounds__(32 * TY)
k_mg_xfer(int n_out, int W, int rows_per_block, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
          const T *__restrict__ val, const cplx<T> *__restrict__ X, cplx<T> *Out, const int32_t *__restrict__ flag) {
    using C = cplx<T>;
    constexpr int UNR = 4;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    if (cg >= ng) return;
    const int c0 = cg * VC;
    if (!col_active<VC>(flag, c0)) return;
    const int r_begin = blockIdx.y * rows_per_block;
    const int r_end = min(n_out, r_begin + rows_per_block);
    for (int row = r_begin + ty; row < r_end; row += TY) {
        const int k0 = __ldg(ptr + row), k1 = __ldg(ptr + row + 1);
        C acc[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v) acc[v] = mk((T)0, (T)0);
        for (int k = k0; k < k1; k += UNR) {
            int cc[UNR];
            T w[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const bool ok = k + u < k1;
                cc[u] = ok ? __ldg(col + k + u) : -1;
                w[u] = ok ? __ldg(val + k + u) : (T)0;
            }
            CV<T, VC> x[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                if (cc[u] >= 0) {
                    x[u] = ldcv(X + (int64_t)cc[u] * W + c0);
                } else {
#pragma unroll
                    for (int v = 0; v < VC; ++v) x[u].v[v] = mk((T)0, (T)0);
                }
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u)
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    acc[v].x = fma(w[u], x[u].v[v].x, acc[v].x);
                    acc[v].y = fma(w[u], x[u].v[v].y, acc[v].y);
                }
        }
        const int64_t base = (int64_t)row * W + c0;
        CV<T, VC> o;
        if (MODE == MG_RESTRICT) {
#pragma unroll
            for (int v = 0; v < VC; ++v) o.v[v] = acc[v];
        } else {
            o = ldcv(Out + base);
#pragma unroll
            for (int v = 0; v < VC; ++v) o.v[v] = cadd(o.v[v], acc[v]);
        }
        stcv(Out + base, o);
    }
}

// out = D r (first pre-smoothing sweep from a zero iterate)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_mg_jacobi0(int n, int W, int Lp, int N, const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ Rv,
             cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    if (cg >= ng) return;
    const int c0 = cg * VC;
    if (!col_active<VC>(flag, c0)) return;
    const int j = c0 / Lp;
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        const cplx<T> d = dinv[(int64_t)row * N + j];
        CV<T, VC> o = ldcv(Rv + base);
#pragma unroll
        for (int v = 0; v < VC; ++v) o.v[v] = cmul(d, o.v[v]);
        stcv(Out + base, o);
    }
}

// y = D x on the finest level (the block the DOWN / UP products gather)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_mg_scale(int n, int W, int Lp, int N, const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ Xv,
           cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    if (cg >= ng) return;
    const int c0 = cg * VC;
    if (!col_active<VC>(flag, c0)) return;
    const int j = c0 / Lp;
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        const cplx<T> d = dinv[(int64_t)row * N + j];
        CV<T, VC> o = ldcv(Xv + base);
#pragma unroll
        for (int v = 0; v < VC; ++v) o.v[v] = cmul(d, o.v[v]);
        stcv(Out + base, o);
    }
}

// Coarsest solve, one of its two products (n_c x n_c real V times the
// complex block X, n_c x W):  Out = op(V) X, op(V) = V^T if trans, and if
// cinv != nullptr each output row k of pole j is scaled by cinv[k*N + j].
// 32 x 32-column tiles of Out per CTA (32 x 8 threads, 4 rows per thread).
template <typename T>
__global__ void __launch_bounds__(256)
k_mg_coarse_gemm(int nc, int W, int Lp, int N, int trans, const T *__restrict__ V, const cplx<T> *__restrict__ X,
                 const cplx<T> *__restrict__ cinv, cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag) {
    using C = cplx<T>;
    __shared__ T sV[32][33];
    __shared__ C sX[32][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int colb = blockIdx.x * 32, rowb = blockIdx.y * 32;
    const int ccol = colb + tx;
    C acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = mk((T)0, (T)0);
    for (int k0 = 0; k0 < nc; k0 += 32) {
        // sV[r][k] = op(V)[rowb + r][k0 + k]
        for (int idx = ty * 32 + tx; idx < 32 * 32; idx += 256) {
            const int r = idx / 32, k = idx % 32;
            const int gr = rowb + r, gk = k0 + k;
            T v = (T)0;
            if (gr < nc && gk < nc) v = trans ? V[(int64_t)gk * nc + gr] : V[(int64_t)gr * nc + gk];
            sV[r][k] = v;
        }
        for (int k = ty; k < 32; k += 8) {
            const int gk = k0 + k;
            sX[k][tx] = (gk < nc && ccol < W) ? X[(int64_t)gk * W + ccol] : mk((T)0, (T)0);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const C x = sX[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T v = sV[ty * 4 + q][k];
                acc[q].x = fma(v, x.x, acc[q].x);
                acc[q].y = fma(v, x.y, acc[q].y);
            }
        }
        __syncthreads();
    }
    if (ccol >= W || flag[ccol] != 1) return;
    const int j = ccol / Lp;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = rowb + ty * 4 + q;
        if (r >= nc) continue;
        C o = acc[q];
        if (cinv) o = cmul(o, cinv[(int64_t)r * N + j]);
        Out[(int64_t)r * W + ccol] = o;
    }
}

// partial r^T z per column (used when the hierarchy is a single level)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_mg_rz(int n, int W, const cplx<T> *__restrict__ Rv, const cplx<T> *__restrict__ Z, const int32_t *__restrict__ flag,
        T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    C rz[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) rz[v] = mk((T)0, (T)0);
    if (cg < ng && col_active<VC>(flag, c0)) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            const int64_t base = (int64_t)row * W + c0;
            const CV<T, VC> r = ldcv(Rv + base), z = ldcv(Z + base);
#pragma unroll
            for (int v = 0; v < VC; ++v) rz[v] = cfma(r.v[v], z.v[v], rz[v]);
        }
    }
    __shared__ T red[TY][32][VC * 2];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        red[ty][tx][2 * v] = rz[v].x;
        red[ty][tx][2 * v + 1] = rz[v].y;
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

template <typename T>
__global__ void k_mg_dinv(int n, int N, const double *__restrict__ da, const double *__restrict__ db,
                          PoleSet<T> ps, double omega, cplx<T> *__restrict__ dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * N) return;
    const int row = (int)(i / N), j = (int)(i % N);
    const double x = da[row] - (double)ps.re[j] * db[row];
    const double y = -(double)ps.im[j] * db[row];
    const double den = x * x + y * y;
    cplx<T> r;
    r.x = (T)(omega * x / den);
    r.y = (T)(-omega * y / den);
    dinv[i] = r;
}

// F = (M - D^{-1}) P of the finest level in pair form for the current damping:
// per stored pair, q = (A P, B P) and (a_ii P, b_ii P); out = first - kappa
// second with kappa = rho_0 / omega (D^{-1} = (rho_0 / omega) (a_ii - sigma b_ii)).
template <typename T>
__global__ void k_mg_fold(int64_t ns, const double2 *__restrict__ q, double kappa, cplx<T> *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const double2 a = q[2 * i], b = q[2 * i + 1];
    out[i] = mk((T)(a.x - kappa * b.x), (T)(a.y - kappa * b.y));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
double vec_bytes(const KrylovDims &d, int n) {
    return (double)n * d.W() * d.frac * sizeof(cplx<T>);
}

// One level product.  Bytes: the pattern and pairs once, the gathered input
// block once (its own rows are part of it), the other vector blocks read or
// written once, the Jacobi diagonals of the gathered rows; for UP also F and
// the coarse iterate.
template <typename T, int MODE>
void launch_sspmm(Ctx &ctx, const KrylovDims &d, int kc, int n_rows, int R, int ngroups, const int32_t *gptr,
                  const int32_t *gcol, const cplx<T> *ab, int64_t nnz_union, int n_in, int gy, const cplx<T> *sig,
                  const cplx<T> *dinv, const cplx<T> *X, const cplx<T> *Rv, cplx<T> *Out, const int32_t *flag,
                  T *part, const int32_t *g2ptr = nullptr, const int32_t *g2col = nullptr,
                  const cplx<T> *ab2 = nullptr, int64_t nnz2 = 0, const cplx<T> *X2 = nullptr, int n2 = 0) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    // gy is used as given: with partial dots every one of the gy partial rows
    // must be written (CTAs without row groups write zeros)
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    const double vin = vec_bytes<T>(d, n_in), vout = vec_bytes<T>(d, n_rows);
    double bytes = 4.0 * (ngroups + 1) + (double)nnz_union * (4 + R * sizeof(cplx<T>)) + vin + vout;
    if (MODE == MG_RESID || MODE == MG_SMOOTH || MODE == MG_UP) bytes += vout;   // r of the rows
    if (MODE == MG_SMOOTH || MODE == MG_UP) bytes += (double)n_rows * d.N * sizeof(cplx<T>);   // D of the rows
    if (MODE == MG_UP) bytes += 4.0 * (ngroups + 1) + (double)nnz2 * (4 + R * sizeof(cplx<T>)) + vec_bytes<T>(d, n2);
    ctx.before(kc, bytes, 8.0 * (double)(nnz_union + nnz2) * R * W * d.frac);
#define SSP(RR)                                                                                                     \
    k_mg_sspmm<T, VC, RR, MODE><<<grid, block, 0, ctx.stream>>>(n_rows, W, d.Lp, d.N, ngroups, gptr, gcol, ab, sig, \
                                                               dinv, X, Rv, Out, flag, part, g2ptr, g2col, ab2, X2)
    switch (R) {
        case 1: SSP(1); break;
        case 2: SSP(2); break;
        case 3: SSP(3); break;
        default: SSP(4); break;
    }
#undef SSP
    ctx.after();
}

// RESID / SMOOTH on a level below the finest
template <typename T, int MODE>
void level_sspmm(Ctx &ctx, const KrylovDims &d, const MgLevel<T> &L, int gy, const cplx<T> *sig, const cplx<T> *X,
                 const cplx<T> *Rv, cplx<T> *Out, const int32_t *flag) {
    launch_sspmm<T, MODE>(ctx, d, KC_MG_COARSE, L.n, L.R, L.ngroups, L.gptr, L.gcol, L.ab, L.nnz_union, L.n, gy, sig,
                          L.dinv, X, Rv, Out, flag, nullptr);
}

template <typename T, int MODE>
void launch_xfer(Ctx &ctx, const KrylovDims &d, int n_out, int n_in, int64_t nnz, const int32_t *ptr,
                 const int32_t *col, const T *val, int gy, const cplx<T> *X, cplx<T> *Out, const int32_t *flag) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    int gyy = std::min(gy, (n_out + TY - 1) / TY);
    if (gyy < 1) gyy = 1;
    dim3 grid((W / VC + 31) / 32, gyy), block(32, TY);
    const int rpb = (n_out + gyy - 1) / gyy;
    const double bytes = 4.0 * (n_out + 1) + (double)nnz * (4 + sizeof(T)) + vec_bytes<T>(d, n_in) +
                         (MODE == MG_RESTRICT ? 1 : 2) * vec_bytes<T>(d, n_out);
    ctx.before(KC_MG_TRANSFER, bytes, 4.0 * (double)nnz * W * d.frac);
    k_mg_xfer<T, VC, MODE><<<grid, block, 0, ctx.stream>>>(n_out, W, rpb, ptr, col, val, X, Out, flag);
    ctx.after();
}

template <typename T>
void coarse_solve(Ctx &ctx, const KrylovDims &d, const MgSolve<T> &mg, const cplx<T> *Rv, cplx<T> *Y, cplx<T> *Z,
                  const int32_t *flag) {
    if constexpr (sizeof(T) == 4) {
        if (mg.Mpan) {   // dense shifted inverses of this level on the tensor cores
            coarse_tc_apply(ctx, d, mg.nc, mg.Mpan, Rv, Z, mg.ct_work, mg.ct_err);
            return;
        }
        if (mg.Minv) {   // dense shifted inverses of this level (FP32 cycles)
            coarse_inverse_apply(ctx, mg.cublas, d, mg.nc, mg.Minv, Rv, Z);
            return;
        }
    }
    const int nc = mg.nc, W = d.W();
    dim3 grid((W + 31) / 32, (nc + 31) / 32), block(32, 8);
    const double bytes = (double)nc * nc * sizeof(T) + 2.0 * vec_bytes<T>(d, nc);
    const double flops = 4.0 * (double)nc * nc * W;
    ctx.before(KC_MG_COARSE, bytes, flops);
    k_mg_coarse_gemm<T><<<grid, block, 0, ctx.stream>>>(nc, W, d.Lp, d.N, 1, mg.V, Rv, mg.cinv, Y, flag);
    ctx.after();
    ctx.before(KC_MG_COARSE, bytes, flops);
    k_mg_coarse_gemm<T><<<grid, block, 0, ctx.stream>>>(nc, W, d.Lp, d.N, 0, mg.V, Y, nullptr, Z, flag);
    ctx.after();
}

template <typename T>
void launch_rz(Ctx &ctx, const KrylovDims &d, int gy, const cplx<T> *R, const cplx<T> *Z, const int32_t *flag,
               T *part) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    ctx.before(KC_MG_TRANSFER, 2 * vec_bytes<T>(d, d.n), 0);
    k_mg_rz<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, R, Z, flag, part);
    ctx.after();
}

// Cycle on level l >= 1 from its restricted residual lv[l].r; returns the
// buffer holding the level iterate.
template <typename T>
cplx<T> *cycle(Ctx &ctx, const KrylovDims &d, MgSolve<T> &mg, int l, int gy, const cplx<T> *sig,
               const int32_t *flag) {
    constexpr int VC = VecN<T>::VC;
    MgLevel<T> &L = mg.lv[l];
    if (l == mg.nlev - 1) {
        coarse_solve<T>(ctx, d, mg, L.r, L.t, L.z, flag);
        return L.z;
    }
    int gyl = std::min(gy, (L.n + TY - 1) / TY);
    if (gyl < 1) gyl = 1;
    cplx<T> *z = L.z, *t = L.t;
    {
        const int W = d.W();
        dim3 grid((W / VC + 31) / 32, gyl), block(32, TY);
        ctx.before(KC_MG_TRANSFER, 2 * vec_bytes<T>(d, L.n) + (double)L.n * d.N * sizeof(cplx<T>), 0);
        k_mg_jacobi0<T, VC><<<grid, block, 0, ctx.stream>>>(L.n, W, d.Lp, d.N, L.dinv, L.r, z, flag);
        ctx.after();
    }
    for (int s = 1; s < mg.nu; ++s) {
        level_sspmm<T, MG_SMOOTH>(ctx, d, L, gyl, sig, z, L.r, t, flag);
        std::swap(z, t);
    }
    const MgLevel<T> &Lc = mg.lv[l + 1];
    for (int v = 0; v < mg.gamma; ++v) {
        level_sspmm<T, MG_RESID>(ctx, d, L, gyl, sig, z, L.r, t, flag);
        launch_xfer<T, MG_RESTRICT>(ctx, d, Lc.n, L.n, L.r_nnz, L.rptr, L.rcol, L.rval, gy, t, Lc.r, flag);
        cplx<T> *e = cycle<T>(ctx, d, mg, l + 1, gy, sig, flag);
        launch_xfer<T, MG_PROLONG_ADD>(ctx, d, L.n, Lc.n, L.p_nnz, L.pptr, L.pcol, L.pval, gy, e, z, flag);
    }
    for (int s = 0; s < mg.nu; ++s) {
        level_sspmm<T, MG_SMOOTH>(ctx, d, L, gyl, sig, z, L.r, t, flag);
        std::swap(z, t);
    }
    return z;
}

}  // namespace

template <typename T>
void mg_dinv(Ctx &ctx, MgSolve<T> &mg, const PoleSet<T> &ps) {
    for (int l = 0; l < mg.nlev; ++l) {
        MgLevel<T> &L = mg.lv[l];
        if (l == mg.nlev - 1 && mg.nlev > 1) break;   // the coarsest level is solved exactly
        const int64_t tot = (int64_t)L.n * ps.N;
        ctx.before(KC_KRYLOV_INIT, (double)tot * sizeof(cplx<T>) + 16.0 * L.n, 0);
        k_mg_dinv<T><<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(L.n, ps.N, L.diag_a, L.diag_b, ps,
                                                                              mg.omega / L.rho, L.dinv);
        ctx.after();
    }
    MgLevel<T> &L0 = mg.lv[0];
    if (mg.nlev > 1) {
        const int64_t ns = L0.fu_nnz * L0.R + L0.fd_nnz;
        ctx.before(KC_KRYLOV_INIT, (double)ns * (32 + sizeof(cplx<T>)), 0);
        k_mg_fold<T><<<(unsigned)((ns + 255) / 256), 256, 0, ctx.stream>>>(ns, L0.f_q, L0.rho / mg.omega, L0.f_ab);
        ctx.after();
    }
}

template <typename T>
void mg_scale(Ctx &ctx, const KrylovDims &d, const MgSolve<T> &mg, int gy, const cplx<T> *X, cplx<T> *Y,
              const int32_t *flag) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    ctx.before(KC_MG_TRANSFER, 2 * vec_bytes<T>(d, d.n) + (double)d.n * d.N * sizeof(cplx<T>), 0);
    k_mg_scale<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, mg.lv[0].dinv, X, Y, flag);
    ctx.after();
}

template <typename T>
void mg_apply(Ctx &ctx, const KrylovDims &d, MgSolve<T> &mg, const cplx<T> *sig, const int32_t *flag, T *part,
              int gy, const cplx<T> *R0, cplx<T> *Z0, cplx<T> *T0, const cplx<T> *Y0) {
    if (mg.nlev == 1) {
        coarse_solve<T>(ctx, d, mg, R0, T0, Z0, flag);
        launch_rz<T>(ctx, d, gy, R0, Z0, flag, part);
        return;
    }
    const MgLevel<T> &L = mg.lv[0];
    const MgLevel<T> &Lc = mg.lv[1];
    if (!Y0) {   // y = D r into the scratch block
        mg_scale<T>(ctx, d, mg, gy, R0, T0, flag);
        Y0 = T0;
    }
    // r1 = -F^T y
    const int gyd = std::max(1, std::min(gy, (Lc.n + TY - 1) / TY));
    launch_sspmm<T, MG_DOWN>(ctx, d, KC_MG_FINE, Lc.n, 1, Lc.n, L.fd_ptr, L.fd_col, L.f_ab + L.fu_nnz * L.R,
                             L.fd_nnz, L.n, gyd, sig, L.dinv, Y0, nullptr, Lc.r, flag, nullptr);
    cplx<T> *e = cycle<T>(ctx, d, mg, 1, gy, sig, flag);
    // z = D (2 r - M y - F e), r^T z
    launch_sspmm<T, MG_UP>(ctx, d, KC_MG_FINE, L.n, L.R, L.ngroups, L.gptr, L.gcol, L.ab, L.nnz_union, L.n, gy, sig,
                           L.dinv, Y0, R0, Z0, flag, part, L.fu_ptr, L.fu_col, L.f_ab, L.fu_nnz, e, Lc.n);
}

template <typename T>
void mg_rz(Ctx &ctx, const KrylovDims &d, int gy, const cplx<T> *R, const cplx<T> *Z, const int32_t *flag, T *part) {
    launch_rz<T>(ctx, d, gy, R, Z, flag, part);
}

#define INST(T)                                                                                                  \
    template void mg_dinv<T>(Ctx &, MgSolve<T> &, const PoleSet<T> &);                                           \
    template void mg_apply<T>(Ctx &, const KrylovDims &, MgSolve<T> &, const cplx<T> *, const int32_t *, T *,  \
                              int, const cplx<T> *, cplx<T> *, cplx<T> *, const cplx<T> *);                     \
    template void mg_rz<T>(Ctx &, const KrylovDims &, int, const cplx<T> *, const cplx<T> *, const int32_t *, T *);
INST(float)
INST(double)
#undef INST

}  // namespace slrf
