// Block BiCGStab over all (pole, column) shifted systems: the Krylov method
// the paper uses for the shifted solves (Section 4.2.1), as the alternative
// to COCG.  Right-preconditioned (y = M^{-1} p, z = M^{-1} s), Hermitian
// inner products, shadow residual r^ = r_0 (van der Vorst 1992; Saad,
// Iterative Methods, Algorithm 9.5):
//
//   y = M^{-1} p ; v = A_sigma y ; alpha = rho / (r^, v) ; s = r - alpha v
//   z = M^{-1} s ; t = A_sigma z ; omega = (t, s) / (t, t)
//   x += alpha y + omega z ; r = s - omega t ; rho' = (r^, r)
//   p = r + (rho'/rho)(alpha/omega)(p - omega v)
//
// Same column-block layout and per-column flags as krylov.cu; the iterate is
// never stored: the filter sum is accumulated in U (pole sum in registers).
// s overwrites r in place (s = r - alpha v, then r = s - omega t).
#include <cuda_runtime.h>

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

// conj(a) b
template <typename C> __device__ __forceinline__ C cdotc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}

// Write per-CTA partial sums acc[v][0..2] of VC columns to part[blockIdx.y][c][0..2].
template <typename T, int VC>
__device__ __forceinline__ void store_partials(T acc[VC][3], int W, int c0, bool live, T *part) {
    __shared__ T red[TY][32][VC * 3];
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int v = 0; v < VC; ++v)
#pragma unroll
        for (int s = 0; s < 3; ++s) red[ty][tx][v * 3 + s] = acc[v][s];
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
            T *o = part + ((int64_t)blockIdx.y * W + c0 + v) * 4;
            o[0] = s0;
            o[1] = s1;
            o[2] = s2;
        }
    }
}

template <int VC>
__device__ __forceinline__ bool any_active(const int32_t *flag, int c0) {
    bool a = false;
#pragma unroll
    for (int v = 0; v < VC; ++v) a |= flag[c0 + v] == 1;
    return a;
}

// r^ = r, p = r; partials (r^, r) = |r|^2 (slots 0, 1) and |r|^2 (slot 2)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_bcg_init(int n, int W, const cplx<T> *__restrict__ R, cplx<T> *__restrict__ Rh, cplx<T> *__restrict__ P,
           const int32_t *__restrict__ flag, T *__restrict__ part) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cg = blockIdx.x * 32 + tx, c0 = cg * VC;
    const bool live = cg < W / VC;
    T acc[VC][3];
#pragma unroll
    for (int v = 0; v < VC; ++v) acc[v][0] = acc[v][1] = acc[v][2] = (T)0;
    if (live && any_active<VC>(flag, c0)) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            const int64_t base = (int64_t)row * W + c0;
            const CV<T, VC> r = ldcv(R + base);
            stcv(Rh + base, r);
            stcv(P + base, r);
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                acc[v][0] += cabs2(r.v[v]);
                acc[v][2] += cabs2(r.v[v]);
            }
        }
    }
    store_partials<T, VC>(acc, W, c0, live, part);
}

// out = D in (Jacobi); D = dinv[row][pole]
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_bcg_jacobi(int n, int W, int Lp, int N, const cplx<T> *__restrict__ dinv, const cplx<T> *__restrict__ In,
             cplx<T> *__restrict__ Out, const int32_t *__restrict__ flag) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cg = blockIdx.x * 32 + tx, c0 = cg * VC;
    if (cg >= W / VC || !any_active<VC>(flag, c0)) return;
    const int j = c0 / Lp;
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        const cplx<T> d = dinv[(int64_t)row * N + j];
        CV<T, VC> o = ldcv(In + base);
#pragma unroll
        for (int v = 0; v < VC; ++v) o.v[v] = cmul(d, o.v[v]);
        stcv(Out + base, o);
    }
}

// partials: conj(a) b (slots 0, 1) and, if c != nullptr, |c|^2 (slot 2)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_bcg_dot(int n, int W, const cplx<T> *__restrict__ A, const cplx<T> *__restrict__ B, const cplx<T> *__restrict__ Cn,
          const int32_t *__restrict__ flag, T *__restrict__ part) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cg = blockIdx.x * 32 + tx, c0 = cg * VC;
    const bool live = cg < W / VC;
    T acc[VC][3];
#pragma unroll
    for (int v = 0; v < VC; ++v) acc[v][0] = acc[v][1] = acc[v][2] = (T)0;
    if (live && any_active<VC>(flag, c0)) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            const int64_t base = (int64_t)row * W + c0;
            const CV<T, VC> a = ldcv(A + base), b = ldcv(B + base);
#pragma unroll
            for (int v = 0; v < VC; ++v) {
                const cplx<T> d = cdotc(a.v[v], b.v[v]);
                acc[v][0] += d.x;
                acc[v][1] += d.y;
            }
            if (Cn) {
                const CV<T, VC> c = ldcv(Cn + base);
#pragma unroll
                for (int v = 0; v < VC; ++v) acc[v][2] += cabs2(c.v[v]);
            }
        }
    }
    store_partials<T, VC>(acc, W, c0, live, part);
}

// s = r - alpha v (in place in R); with a Jacobi diagonal also z = D s
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_bcg_s(int n, int W, int Lp, int N, cplx<T> *__restrict__ R, const cplx<T> *__restrict__ V,
        const cplx<T> *__restrict__ alpha, const cplx<T> *__restrict__ dinv, cplx<T> *__restrict__ Z,
        const int32_t *__restrict__ flag) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cg = blockIdx.x * 32 + tx, c0 = cg * VC;
    if (cg >= W / VC || !any_active<VC>(flag, c0)) return;
    const int j = c0 / Lp;
    cplx<T> a[VC];
    bool act[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        act[v] = flag[c0 + v] == 1;
        a[v] = alpha[c0 + v];
    }
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        CV<T, VC> r = ldcv(R + base);
        const CV<T, VC> vv = ldcv(V + base);
#pragma unroll
        for (int v = 0; v < VC; ++v)
            if (act[v]) r.v[v] = csub(r.v[v], cmul(a[v], vv.v[v]));
        stcv(R + base, r);
        if (dinv) {
            const cplx<T> d = dinv[(int64_t)row * N + j];
#pragma unroll
            for (int v = 0; v < VC; ++v) r.v[v] = cmul(d, r.v[v]);
            stcv(Z + base, r);
        }
    }
}

// U += Re(ua_alpha y + ua_omega z) (pole sum), r = s - omega t; partials
// (r^, r) (slots 0, 1) and |r|^2 (slot 2).  One thread owns VC columns of a
// pole slot and walks the N poles.
template <typename T, int VC, int NP>
__global__ void __launch_bounds__(32 * TY)
k_bcg_update(int n, int W, int Lp, int N, cplx<T> *__restrict__ R, const cplx<T> *__restrict__ Rh,
             const cplx<T> *__restrict__ Y, const cplx<T> *__restrict__ Z, const cplx<T> *__restrict__ Tt,
             const cplx<T> *__restrict__ omega, const cplx<T> *__restrict__ ua, const cplx<T> *__restrict__ ua2,
             const int32_t *__restrict__ flag, T *__restrict__ U, T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cgl = blockIdx.x * 32 + tx, c0 = cgl * VC;
    const bool live = cgl < Lp / VC;
    unsigned actmask = 0;
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
                const CV<T, VC> rh = ldcv(Rh + base), y = ldcv(Y + base), z = ldcv(Z + base), t = ldcv(Tt + base);
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    if (!(mj & (1u << v))) continue;
                    const int col = j * Lp + c0 + v;
                    const C w1 = ua[col], w2 = ua2[col], om = omega[col];
                    u[v] += w1.x * y.v[v].x - w1.y * y.v[v].y + w2.x * z.v[v].x - w2.y * z.v[v].y;
                    r.v[v] = csub(r.v[v], cmul(om, t.v[v]));
                    const C d = cdotc(rh.v[v], r.v[v]);
                    acc[j][v][0] += d.x;
                    acc[j][v][1] += d.y;
                    acc[j][v][2] += cabs2(r.v[v]);
                }
                stcv(R + base, r);
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
                o[0] = s0;
                o[1] = s1;
                o[2] = s2;
            }
        }
        __syncthreads();
    }
}

// p = r + (beta alpha / omega)(p - omega v)  (beta = rho'/rho from the reduction)
template <typename T, int VC>
__global__ void __launch_bounds__(32 * TY)
k_bcg_p(int n, int W, const cplx<T> *__restrict__ R, const cplx<T> *__restrict__ V, cplx<T> *__restrict__ P,
        const cplx<T> *__restrict__ alpha, const cplx<T> *__restrict__ beta, const cplx<T> *__restrict__ omega,
        const int32_t *__restrict__ flag) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cg = blockIdx.x * 32 + tx, c0 = cg * VC;
    if (cg >= W / VC || !any_active<VC>(flag, c0)) return;
    cplx<T> f[VC], om[VC];
    bool act[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
        act[v] = flag[c0 + v] == 1;
        om[v] = omega[c0 + v];
        // beta alpha / omega (omega != 0 for an active column: checked by the reduction)
        const cplx<T> ba = cmul(beta[c0 + v], alpha[c0 + v]);
        const T den = cabs2(om[v]);
        f[v].x = (ba.x * om[v].x + ba.y * om[v].y) / den;
        f[v].y = (ba.y * om[v].x - ba.x * om[v].y) / den;
    }
    for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
        const int64_t base = (int64_t)row * W + c0;
        const CV<T, VC> r = ldcv(R + base), vv = ldcv(V + base);
        CV<T, VC> p = ldcv(P + base);
#pragma unroll
        for (int v = 0; v < VC; ++v)
            if (act[v]) p.v[v] = cfma(f[v], csub(p.v[v], cmul(om[v], vv.v[v])), r.v[v]);
        stcv(P + base, p);
    }
}

// per-column scalar reductions (one warp per column, FP64 sums of the partials)
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

// alpha = rho / (r^, v); ua = 2 coef alpha
template <typename T>
__global__ void k_bcg_alpha(int W, int gy, const T *__restrict__ part, KrylovScalars<T> s) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    if ((threadIdx.x & 31) == 0 && s.flag[col] == 1) {
        const double den = s0 * s0 + s1 * s1;
        if (!(den > 0.0) || !isfinite(den)) {
            s.flag[col] = 2;
            return;
        }
        const double rr = (double)s.rho[col].x, ri = (double)s.rho[col].y;
        const double ar = (rr * s0 + ri * s1) / den, ai = (ri * s0 - rr * s1) / den;
        s.alpha[col] = mk((T)ar, (T)ai);
        const double2 c = s.coef[col];
        s.ua[col] = mk((T)(2.0 * (c.x * ar - c.y * ai)), (T)(2.0 * (c.x * ai + c.y * ar)));
    }
}

// omega = (t, s) / (t, t); ua2 = 2 coef omega.  t = 0 means s = 0 (A_sigma
// nonsingular): omega = 0 keeps x += alpha y and leaves r = s = 0.
template <typename T>
__global__ void k_bcg_omega(int W, int gy, const T *__restrict__ part, KrylovScalars<T> s, cplx<T> *__restrict__ omega,
                            cplx<T> *__restrict__ ua2) {
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= W) return;
    double s0, s1, s2;
    warp_sum3(part, gy, W, col, s0, s1, s2);
    if ((threadIdx.x & 31) == 0 && s.flag[col] == 1) {
        double orr = 0.0, oi = 0.0;
        if (s2 > 0.0 && isfinite(s2)) {
            orr = s0 / s2;
            oi = s1 / s2;
        } else if (!isfinite(s2)) {
            s.flag[col] = 2;
            return;
        }
        omega[col] = mk((T)orr, (T)oi);
        const double2 c = s.coef[col];
        ua2[col] = mk((T)(2.0 * (c.x * orr - c.y * oi)), (T)(2.0 * (c.x * oi + c.y * orr)));
    }
}

// After the convergence test: an active column with omega = 0 cannot continue
// (the direction update divides by omega): breakdown.
template <typename T>
__global__ void k_bcg_check_omega(int W, const cplx<T> *__restrict__ omega, int32_t *__restrict__ flag) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= W || flag[col] != 1) return;
    if (!(cabs2(omega[col]) > (T)0)) flag[col] = 2;
}

}  // namespace

template <typename T>
void bicgstab_init(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_INIT, 3 * vb, 0);
    k_bcg_init<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, kb.R, bb.Rh, kb.P, kb.s.flag, kb.s.part);
    ctx.after();
}

template <typename T>
void bicgstab_precond_jacobi(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, const cplx<T> *In, cplx<T> *Out) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_DIR, 2 * vb, 6.0 * d.n * W * d.frac);
    k_bcg_jacobi<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.dinv, In, Out, kb.s.flag);
    ctx.after();
}

template <typename T>
void bicgstab_alpha(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_REDUCE, 2 * vb, 8.0 * d.n * W * d.frac);
    k_bcg_dot<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, bb.Rh, bb.V, nullptr, kb.s.flag, kb.s.part);
    ctx.after();
    ctx.before(KC_KRYLOV_REDUCE, (double)kb.gy * W * 4 * sizeof(T), 0);
    k_bcg_alpha<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, kb.gy, kb.s.part, kb.s);
    ctx.after();
}

template <typename T>
void bicgstab_s(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb, bool jacobi) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_UPDATE, (jacobi ? 4 : 3) * vb, 8.0 * d.n * W * d.frac);
    k_bcg_s<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, bb.V, kb.s.alpha,
                                                    jacobi ? kb.dinv : nullptr, bb.Z, kb.s.flag);
    ctx.after();
}

template <typename T>
void bicgstab_omega(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_REDUCE, 2 * vb, 12.0 * d.n * W * d.frac);
    k_bcg_dot<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, bb.Tt, kb.R, bb.Tt, kb.s.flag, kb.s.part);
    ctx.after();
    ctx.before(KC_KRYLOV_REDUCE, (double)kb.gy * W * 4 * sizeof(T), 0);
    k_bcg_omega<T><<<(W * 32 + 255) / 256, 256, 0, ctx.stream>>>(W, kb.gy, kb.s.part, kb.s, bb.omega, bb.ua2);
    ctx.after();
}

template <typename T, int NP>
static void launch_bcg_update(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    dim3 grid((d.Lp / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_UPDATE, 6 * vb + 2.0 * d.n * d.Lp * sizeof(T), 24.0 * d.n * W * d.frac);
    k_bcg_update<T, VC, NP><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, kb.R, bb.Rh, bb.Y, bb.Z, bb.Tt, bb.omega,
                                                             kb.s.ua, bb.ua2, kb.s.flag, kb.Uacc, kb.s.part);
    ctx.after();
}

template <typename T>
void bicgstab_update(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    if (d.N <= 2)
        launch_bcg_update<T, 2>(ctx, d, kb, bb);
    else if (d.N <= 4)
        launch_bcg_update<T, 4>(ctx, d, kb, bb);
    else if (d.N <= 8)
        launch_bcg_update<T, 8>(ctx, d, kb, bb);
    else
        launch_bcg_update<T, 16>(ctx, d, kb, bb);
}

template <typename T>
void bicgstab_direction(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, BcgBuffers<T> &bb) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W();
    ctx.before(KC_KRYLOV_REDUCE, 4.0 * W, 0);
    k_bcg_check_omega<T><<<(W + 255) / 256, 256, 0, ctx.stream>>>(W, bb.omega, kb.s.flag);
    ctx.after();
    dim3 grid((W / VC + 31) / 32, kb.gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    ctx.before(KC_KRYLOV_DIR, 4 * vb, 14.0 * d.n * W * d.frac);
    k_bcg_p<T, VC><<<grid, block, 0, ctx.stream>>>(d.n, W, kb.R, bb.V, kb.P, kb.s.alpha, kb.s.beta, bb.omega,
                                                    kb.s.flag);
    ctx.after();
}

#define INST(T)                                                                                                  \
    template void bicgstab_init<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);            \
    template void bicgstab_precond_jacobi<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, const cplx<T> *,     \
                                             cplx<T> *);                                                         \
    template void bicgstab_alpha<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);           \
    template void bicgstab_s<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &, bool);         \
    template void bicgstab_omega<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);           \
    template void bicgstab_update<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);          \
    template void bicgstab_direction<T>(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);
INST(float)
INST(double)
#undef INST

}  // namespace slrf
