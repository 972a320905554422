// Multigrid V/W-cycle preconditioner for the block COCG of krylov.cu.
//
// One cycle is applied to all (pole, column) systems at once: every level
// keeps the column-block layout of the Krylov state (complex n_l x W, row
// stride W, pole j in columns [j*Lp, j*Lp + Lp)), the level operator of pole
// j is A_l - sigma_j B_l with the Galerkin pencil of mg_setup.cpp, and the
// smoother is damped Jacobi, D_lj = omega_l / (a_ii - sigma_j b_ii) with
// omega_l = omega / rho(D_l^{-1} A_l) (4/3 by default: the high-frequency
// modes are damped whatever the level's diagonal dominance).  With
// R_l = P_l^T, equal pre- and post-smoothing and the exact coarsest solve
// V (Lambda - sigma_j)^{-1} V^T, the cycle is a complex symmetric linear
// operator, as COCG requires of its preconditioner.
//
// Finest level (one sweep each side, the pre-smoothing from zero folded in):
//   t  = r - M (D r)                  k_mg_sspmm<RESID0>
//   r1 = P^T t                        k_mg_xfer<RESTRICT>
//   e  = cycle(1, r1)
//   z1 = D r + P e                    k_mg_xfer<PROLONG0>
//   z  = z1 + D (r - M z1), r^T z     k_mg_sspmm<SMOOTH>  (+ partial dots)
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

enum { MG_RESID0 = 0, MG_RESID = 1, MG_SMOOTH = 2 };
enum { MG_RESTRICT = 0, MG_PROLONG0 = 1, MG_PROLONG_ADD = 2 };

// Column group of a thread: VC consecutive columns of one pole (Lp is even).
template <int VC>
__device__ __forceinline__ bool col_active(const int32_t *flag, int c0) {
    bool a = false;
#pragma unroll
    for (int v = 0; v < VC; ++v) a |= flag[c0 + v] == 1;
    return a;
}

// ---------------------------------------------------------------------------
// Shifted level product in row-group form (R rows per group share one union
// column list with R (a, b) pairs per entry; R = 1 is plain CSR):
//   RESID0: out = r - M (D r)   (gathers r and D of the neighbour rows)
//   RESID : out = r - M x
//   SMOOTH: out = x + D (r - M x), optional partial r^T out per column
// ---------------------------------------------------------------------------
template <typename T, int VC, int R, int MODE>
__global__ void __launch_bounds__(32 * TY, 6)
k_mg_sspmm(int n, int W, int Lp, int N, int ngroups, const int32_t *__restrict__ gptr,
           const int32_t *__restrict__ ucol, const cplx<T> *__restrict__ uab, const cplx<T> *__restrict__ sig,
           const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ X, const cplx<T> *__restrict__ Rv,
           cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag, T *__restrict__ part) {
    using C = cplx<T>;
    // measured on the 2D bench: 2-deep gathers at 6 CTAs per SM beat 4-deep at 4
    // (125 vs 134 ms per solve) and 8-deep (155 ms)
    constexpr int UNR = 2;
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
            const int e0 = __ldg(gptr + g), e1 = __ldg(gptr + g + 1);
            C sa[R][VC], sb[R][VC];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < VC; ++v) sa[r][v] = sb[r][v] = mk((T)0, (T)0);
            for (int e = e0; e < e1; e += UNR) {
                int cc[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) cc[u] = (e + u < e1) ? __ldg(ucol + e + u) : -1;
                CV<T, VC> x[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (cc[u] >= 0) {
                        x[u] = ldcv(X + (int64_t)cc[u] * W + c0);
                        if (MODE == MG_RESID0) {
                            const C dk = dinv[(int64_t)cc[u] * N + j];
#pragma unroll
                            for (int v = 0; v < VC; ++v) x[u].v[v] = cmul(dk, x[u].v[v]);
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < VC; ++v) x[u].v[v] = mk((T)0, (T)0);
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (cc[u] < 0) break;
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
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = g * R + r;
                if (row >= n) break;
                const int64_t base = (int64_t)row * W + c0;
                const CV<T, VC> rr = ldcv(Rv + base);
                CV<T, VC> o;
                if (MODE == MG_SMOOTH) {
                    const CV<T, VC> xr = ldcv(X + base);
                    const C d = dinv[(int64_t)row * N + j];
#pragma unroll
                    for (int v = 0; v < VC; ++v) {
                        const C y = csub(sa[r][v], cmul(s, sb[r][v]));
                        o.v[v] = cfma(d, csub(rr.v[v], y), xr.v[v]);
                        rz[v] = cfma(rr.v[v], o.v[v], rz[v]);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < VC; ++v) o.v[v] = csub(rr.v[v], csub(sa[r][v], cmul(s, sb[r][v])));
                }
                stcv(Out + base, o);
            }
        }
    }
    if constexpr (MODE == MG_SMOOTH) {
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
// Grid transfers with a real CSR matrix (P or P^T), all W columns:
//   RESTRICT   : out = M x
//   PROLONG0   : out = D r + M x
//   PROLONG_ADD: out += M x           (out is the level iterate, updated in place)
// ---------------------------------------------------------------------------
template <typename T, int VC, int MODE>
__global__ void __launch_bounds__(32 * TY)
k_mg_xfer(int n_out, int W, int Lp, int N, int rows_per_block, const int32_t *__restrict__ ptr,
          const int32_t *__restrict__ col, const T *__restrict__ val, const cplx<T> *__restrict__ X,
          const cplx<T> *__restrict__ Rv, const cplx<T> *__restrict__ dinv, cplx<T> *Out,
          const int32_t *__restrict__ flag) {
    using C = cplx<T>;
    constexpr int UNR = 4;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    if (cg >= ng) return;
    const int c0 = cg * VC;
    if (!col_active<VC>(flag, c0)) return;
    const int j = c0 / Lp;
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
        } else if (MODE == MG_PROLONG0) {
            const CV<T, VC> rr = ldcv(Rv + base);
            const C d = dinv[(int64_t)row * N + j];
#pragma unroll
            for (int v = 0; v < VC; ++v) o.v[v] = cfma(d, rr.v[v], acc[v]);
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
double vec_bytes(const KrylovDims &d, int n) {
    return (double)n * d.W() * d.frac * sizeof(cplx<T>);
}

template <typename T, int MODE>
void launch_sspmm(Ctx &ctx, const KrylovDims &d, const MgLevel<T> &L, int gy, const cplx<T> *sig,
                  const cplx<T> *X, const cplx<T> *Rv, cplx<T> *Out, const int32_t *flag, T *part) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    const double vb = vec_bytes<T>(d, L.n);
    const double bytes = 4.0 * (L.ngroups + 1) + (double)L.nnz_union * (4 + L.R * sizeof(cplx<T>)) +
                         (MODE == MG_SMOOTH ? 4 : 3) * vb + (double)L.n * d.N * sizeof(cplx<T>);
    ctx.before(L.n == d.n ? KC_MG_FINE : KC_MG_COARSE, bytes, 8.0 * (double)L.nnz_union * L.R * W * d.frac);
#define SSP(RR)                                                                                                   \
    k_mg_sspmm<T, VC, RR, MODE><<<grid, block, 0, ctx.stream>>>(L.n, W, d.Lp, d.N, L.ngroups, L.gptr, L.gcol,      \
                                                               L.ab, sig, L.dinv, X, Rv, Out, flag, part)
    switch (L.R) {
        case 1: SSP(1); break;
        case 2: SSP(2); break;
        case 3: SSP(3); break;
        default: SSP(4); break;
    }
#undef SSP
    ctx.after();
}

template <typename T, int MODE>
void launch_xfer(Ctx &ctx, const KrylovDims &d, int n_out, int n_in, int64_t nnz, const int32_t *ptr,
                 const int32_t *col, const T *val, int gy, const cplx<T> *X, const cplx<T> *Rv, const cplx<T> *dinv,
                 cplx<T> *Out, const int32_t *flag) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    int gyy = std::min(gy, (n_out + TY - 1) / TY);
    if (gyy < 1) gyy = 1;
    dim3 grid((W / VC + 31) / 32, gyy), block(32, TY);
    const int rpb = (n_out + gyy - 1) / gyy;
    const double bytes = 4.0 * (n_out + 1) + (double)nnz * (4 + sizeof(T)) + vec_bytes<T>(d, n_in) +
                         (MODE == MG_RESTRICT ? 1 : 2) * vec_bytes<T>(d, n_out) +
                         (MODE == MG_PROLONG0 ? (double)n_out * d.N * sizeof(cplx<T>) : 0.0);
    ctx.before(KC_MG_TRANSFER, bytes, 4.0 * (double)nnz * W * d.frac);
    k_mg_xfer<T, VC, MODE><<<grid, block, 0, ctx.stream>>>(n_out, W, d.Lp, d.N, rpb, ptr, col, val, X, Rv, dinv, Out,
                                                          flag);
    ctx.after();
}

template <typename T>
void coarse_solve(Ctx &ctx, const KrylovDims &d, const MgSolve<T> &mg, const cplx<T> *Rv, cplx<T> *Y, cplx<T> *Z,
                  const int32_t *flag) {
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
        ctx.before(KC_MG_TRANSFER, 2 * vec_bytes<T>(d, L.n), 0);
        k_mg_jacobi0<T, VC><<<grid, block, 0, ctx.stream>>>(L.n, W, d.Lp, d.N, L.dinv, L.r, z, flag);
        ctx.after();
    }
    for (int s = 1; s < mg.nu; ++s) {
        launch_sspmm<T, MG_SMOOTH>(ctx, d, L, gyl, sig, z, L.r, t, flag, nullptr);
        std::swap(z, t);
    }
    const MgLevel<T> &Lc = mg.lv[l + 1];
    for (int v = 0; v < mg.gamma; ++v) {
        launch_sspmm<T, MG_RESID>(ctx, d, L, gyl, sig, z, L.r, t, flag, nullptr);
        launch_xfer<T, MG_RESTRICT>(ctx, d, Lc.n, L.n, L.r_nnz, L.rptr, L.rcol, L.rval, gy, t, nullptr, nullptr,
                                    Lc.r, flag);
        cplx<T> *e = cycle<T>(ctx, d, mg, l + 1, gy, sig, flag);
        launch_xfer<T, MG_PROLONG_ADD>(ctx, d, L.n, Lc.n, L.p_nnz, L.pptr, L.pcol, L.pval, gy, e, nullptr, nullptr,
                                       z, flag);
    }
    for (int s = 0; s < mg.nu; ++s) {
        launch_sspmm<T, MG_SMOOTH>(ctx, d, L, gyl, sig, z, L.r, t, flag, nullptr);
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
}

template <typename T>
void mg_apply(Ctx &ctx, const KrylovDims &d, MgSolve<T> &mg, const cplx<T> *sig, const int32_t *flag, T *part,
              int gy, const cplx<T> *R0, cplx<T> *Z0, cplx<T> *T0) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    if (mg.nlev == 1) {
        coarse_solve<T>(ctx, d, mg, R0, T0, Z0, flag);
        dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
        ctx.before(KC_MG_TRANSFER, 2 * vec_bytes<T>(d, d.n), 0);
        k_mg_rz<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, R0, Z0, flag, part);
        ctx.after();
        return;
    }
    MgLevel<T> &L = mg.lv[0];
    const MgLevel<T> &Lc = mg.lv[1];
    launch_sspmm<T, MG_RESID0>(ctx, d, L, gy, sig, R0, R0, T0, flag, nullptr);
    launch_xfer<T, MG_RESTRICT>(ctx, d, Lc.n, L.n, L.r_nnz, L.rptr, L.rcol, L.rval, gy, T0, nullptr, nullptr, Lc.r,
                                flag);
    cplx<T> *e = cycle<T>(ctx, d, mg, 1, gy, sig, flag);
    launch_xfer<T, MG_PROLONG0>(ctx, d, L.n, Lc.n, L.p_nnz, L.pptr, L.pcol, L.pval, gy, e, R0, L.dinv, T0, flag);
    launch_sspmm<T, MG_SMOOTH>(ctx, d, L, gy, sig, T0, R0, Z0, flag, part);
}

#define INST(T)                                                                                                  \
    template void mg_dinv<T>(Ctx &, MgSolve<T> &, const PoleSet<T> &);                                           \
    template void mg_apply<T>(Ctx &, const KrylovDims &, MgSolve<T> &, const cplx<T> *, const int32_t *, T *,  \
                              int, const cplx<T> *, cplx<T> *, cplx<T> *);
INST(float)
INST(double)
#undef INST

}  // namespace slrf
