// No-fill incomplete factorisation of the shifted matrices, GPU-native.
//
// The paper preconditions its BiCGStab solves with ILU (drop tolerance 1e-4
// after a reverse Cuthill-McKee ordering; Section 4.2.1, Table 1).  Its
// classical form is sequential twice over: the factorisation eliminates row
// after row, and each application runs two triangular solves whose
// wavefronts follow the matrix bandwidth.  The form built here keeps the
// factor's pattern to the pencil's own (no fill) and replaces both
// sequential parts by fixed-point sweeps that run over all entries, all
// poles and all columns at once:
//
//  * factor: M_j = A - sigma_j B ~ L D L^T (L unit lower triangular,
//    unconjugated transpose: M_j is complex symmetric).  The entries satisfy
//        l_ik = (m_ik - sum_{q<k} l_iq d_q l_kq) / d_k      (k < i)
//        d_i  =  m_ii - sum_{q<i} l_iq^2 d_q
//    on the pattern; starting from l_ik = m_ik / m_kk, d_i = m_ii, every
//    sweep evaluates all right-hand sides from the previous iterate
//    (Chow and Patel's fine-grained ILU, symmetric form), in FP64;
//  * application: z = L^{-T} D^{-1} L^{-1} r with each triangular solve
//    replaced by s Jacobi sweeps y <- r - (L - I) y from y = r, that is by
//    P = I - N + N^2 - ... (N = L - I, s + 1 terms), so z = P^T D^{-1} P r:
//    a fixed, complex symmetric operator, as COCG requires of its
//    preconditioner (BiCGStab accepts it too).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace slrf {

std::vector<int32_t> ilu_pattern_host(int n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                                      int64_t *nnzl_out) {
    std::vector<int32_t> lptr(n + 1, 0), lcol, lrow, lsrc;
    for (int i = 0; i < n; ++i) {
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] < i) {
                lcol.push_back(ci[k]);
                lrow.push_back(i);
                lsrc.push_back(k);
            }
        lptr[i + 1] = (int32_t)lcol.size();
    }
    const int64_t nnzl = (int64_t)lcol.size();
    // by columns: the rows of L^T, rows ascending within each column
    std::vector<int32_t> tptr(n + 1, 0), trow(nnzl), tidx(nnzl);
    for (int64_t e = 0; e < nnzl; ++e) ++tptr[lcol[e] + 1];
    for (int c = 0; c < n; ++c) tptr[c + 1] += tptr[c];
    std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
    for (int64_t e = 0; e < nnzl; ++e) {
        const int32_t pos = fill[lcol[e]]++;
        trow[pos] = lrow[e];
        tidx[pos] = (int32_t)e;
    }
    std::vector<int32_t> out;
    out.reserve(2 * (size_t)(n + 1) + 6 * (size_t)nnzl);
    out.insert(out.end(), lptr.begin(), lptr.end());
    out.insert(out.end(), lcol.begin(), lcol.end());
    out.insert(out.end(), lrow.begin(), lrow.end());
    out.insert(out.end(), lsrc.begin(), lsrc.end());
    out.insert(out.end(), tptr.begin(), tptr.end());
    out.insert(out.end(), trow.begin(), trow.end());
    out.insert(out.end(), tidx.begin(), tidx.end());
    *nnzl_out = nnzl;
    return out;
}

void ilu_pattern_views(const int32_t *dev, int n, int64_t nnzl, IluPattern &pat) {
    pat.n = n;
    pat.nnzl = nnzl;
    pat.lptr = dev;
    pat.lcol = pat.lptr + (n + 1);
    pat.lrow = pat.lcol + nnzl;
    pat.lsrc = pat.lrow + nnzl;
    pat.tptr = pat.lsrc + nnzl;
    pat.trow = pat.tptr + (n + 1);
    pat.tidx = pat.trow + nnzl;
}

namespace {

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// m = a - sigma b for pencil entry k
__device__ __forceinline__ double2 shifted(const double *a, const double *b, int64_t k, double sr, double si) {
    return make_double2(a[k] - sr * b[k], -si * b[k]);
}

// start: l_ik = m_ik / m_kk, d_i = m_ii (all poles)
__global__ void k_ilu_init(int n, int64_t nnzl, PoleSet<double> ps, const int32_t *__restrict__ lcol,
                           const int32_t *__restrict__ lsrc, const double *__restrict__ a, const double *__restrict__ b,
                           const double *__restrict__ da, const double *__restrict__ db, double2 *__restrict__ L,
                           double2 *__restrict__ D) {
    const int j = blockIdx.y;
    const double sr = ps.re[j], si = ps.im[j];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzl; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = lcol[e];
        L[(int64_t)j * nnzl + e] = cdiv(shifted(a, b, lsrc[e], sr, si), make_double2(da[c] - sr * db[c], -si * db[c]));
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        D[i * ps.N + j] = make_double2(da[i] - sr * db[i], -si * db[i]);
}

// One fixed-point sweep: (Lold, Dold) -> (Lnew, Dnew), every entry from the
// previous iterate (deterministic for any thread order).
__global__ void k_ilu_sweep(int n, int64_t nnzl, PoleSet<double> ps, const int32_t *__restrict__ lptr,
                            const int32_t *__restrict__ lcol, const int32_t *__restrict__ lrow,
                            const int32_t *__restrict__ lsrc, const double *__restrict__ a,
                            const double *__restrict__ b, const double *__restrict__ da, const double *__restrict__ db,
                            const double2 *__restrict__ Lold, const double2 *__restrict__ Dold,
                            double2 *__restrict__ Lnew, double2 *__restrict__ Dnew) {
    const int j = blockIdx.y, N = ps.N;
    const double sr = ps.re[j], si = ps.im[j];
    const double2 *Lj = Lold + (int64_t)j * nnzl;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzl; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = lrow[e], c = lcol[e];
        // s = sum over q < c in both lower rows i and c of l_iq d_q l_cq
        double2 s = make_double2(0.0, 0.0);
        int p = lptr[i], pe = (int)e;   // row i's entries with column < c precede e
        int q = lptr[c], qe = lptr[c + 1];
        while (p < pe && q < qe) {
            const int cp = lcol[p], cq = lcol[q];
            if (cp == cq) {
                s = cfma(cmul(Lj[p], Dold[(int64_t)cp * N + j]), Lj[q], s);
                ++p;
                ++q;
            } else if (cp < cq) {
                ++p;
            } else {
                ++q;
            }
        }
        Lnew[(int64_t)j * nnzl + e] = cdiv(csub(shifted(a, b, lsrc[e], sr, si), s), Dold[(int64_t)c * N + j]);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int p = lptr[i]; p < lptr[i + 1]; ++p) s = cfma(cmul(Lj[p], Lj[p]), Dold[(int64_t)lcol[p] * N + j], s);
        Dnew[i * N + j] = csub(make_double2(da[i] - sr * db[i], -si * db[i]), s);
    }
}

// FP64 factor -> the apply's precision: L as is, D inverted
template <typename T>
__global__ void k_ilu_store(int n, int64_t nnzl, int N, const double2 *__restrict__ L, const double2 *__restrict__ D,
                            cplx<T> *__restrict__ Lo, cplx<T> *__restrict__ Dinv) {
    const int64_t tl = (int64_t)N * nnzl, td = (int64_t)n * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tl + td; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < tl) {
            Lo[e] = mk((T)L[e].x, (T)L[e].y);
        } else {
            const double2 v = cdiv(make_double2(1.0, 0.0), D[e - tl]);
            Dinv[e - tl] = mk((T)v.x, (T)v.y);
        }
    }
}

}  // namespace

size_t ilu_factor_work_bytes(const IluPattern &pat, int N) {
    return 2 * ((size_t)N * pat.nnzl + (size_t)pat.n * N) * sizeof(double2) + 1024;
}

template <typename T>
void ilu_factor(Ctx &ctx, const DevPencil &A, const IluPattern &pat, const PoleSet<double> &ps, int sweeps,
                void *work, cplx<T> *out, IluFactor<T> &fac) {
    const int N = ps.N, n = pat.n;
    const int64_t nnzl = pat.nnzl;
    double2 *L0 = reinterpret_cast<double2 *>(work);
    double2 *D0 = L0 + (size_t)N * nnzl;
    double2 *L1 = D0 + (size_t)n * N;
    double2 *D1 = L1 + (size_t)N * nnzl;
    const int64_t items = std::max<int64_t>(nnzl, n);
    const dim3 grid((unsigned)std::min<int64_t>((items + 255) / 256, 4096), N);
    ctx.before(KC_KRYLOV_INIT, (double)N * (nnzl * 40.0 + n * 32.0), 0);
    k_ilu_init<<<grid, 256, 0, ctx.stream>>>(n, nnzl, ps, pat.lcol, pat.lsrc, A.a, A.b, A.diag_a, A.diag_b, L0, D0);
    ctx.after();
    for (int s = 0; s < sweeps; ++s) {
        ctx.before(KC_KRYLOV_INIT, (double)N * (nnzl * 64.0 + n * 48.0), 0);
        k_ilu_sweep<<<grid, 256, 0, ctx.stream>>>(n, nnzl, ps, pat.lptr, pat.lcol, pat.lrow, pat.lsrc, A.a, A.b,
                                                  A.diag_a, A.diag_b, L0, D0, L1, D1);
        ctx.after();
        std::swap(L0, L1);
        std::swap(D0, D1);
    }
    cplx<T> *Lo = out;
    cplx<T> *Dinv = out + (size_t)N * nnzl;
    const int64_t tot = (int64_t)N * nnzl + (int64_t)n * N;
    ctx.before(KC_KRYLOV_INIT, (double)tot * (16 + sizeof(cplx<T>)), 0);
    k_ilu_store<T><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, ctx.stream>>>(n, nnzl, N, L0, D0, Lo,
                                                                                              Dinv);
    ctx.after();
    fac.N = N;
    fac.L = Lo;
    fac.Dinv = Dinv;
}

// ---------------------------------------------------------------------------
// application: Jacobi sweeps of the two triangular solves over all
// (pole, column) systems, in the state's column-block layout
// ---------------------------------------------------------------------------
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

// LOWER:  Out_i = In_i - sum_{k<i} l_ik G_k                      (rows of L)
// UPPER:  Out_i = w_i - sum_{k>i} l_ki G'_k,  w = D^{-1} Ys       (rows of L^T)
//         with G' = D^{-1} Ys on the first sweep (FIRST), else G;
//         DOTS: partial sums of Rdot^T Out per column (slots 0, 1)
template <typename T, int VC, bool UPPER, bool FIRST, bool DOTS>
__global__ void __launch_bounds__(32 * TY)
k_ilu_tri(int n, int W, int Lp, int N, int64_t nnzl, const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
          const int32_t *__restrict__ map, const cplx<T> *__restrict__ Lv, const cplx<T> *__restrict__ Dinv,
          const cplx<T> *__restrict__ In, const cplx<T> *__restrict__ G, cplx<T> *__restrict__ Out,
          const cplx<T> *__restrict__ Rdot, const int32_t *__restrict__ flag, T *__restrict__ part) {
    using C = cplx<T>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ng = W / VC;
    const int cg = blockIdx.x * 32 + tx;
    const int c0 = cg * VC;
    bool act = false;
    int j = 0;
    if (cg < ng) {
#pragma unroll
        for (int v = 0; v < VC; ++v) act |= flag[c0 + v] == 1;
        j = c0 / Lp;
    }
    const C *Lj = Lv + (int64_t)j * nnzl;
    C rz[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) rz[v] = mk((T)0, (T)0);
    if (act) {
        for (int row = blockIdx.y * TY + ty; row < n; row += gridDim.y * TY) {
            C acc[VC];
#pragma unroll
            for (int v = 0; v < VC; ++v) acc[v] = mk((T)0, (T)0);
            for (int p = __ldg(ptr + row); p < __ldg(ptr + row + 1); ++p) {
                const int k = __ldg(idx + p);
                const C l = Lj[UPPER ? __ldg(map + p) : p];
                CV<T, VC> g = ldcv(G + (int64_t)k * W + c0);
                if (FIRST) {
                    const C dk = Dinv[(int64_t)k * N + j];
#pragma unroll
                    for (int v = 0; v < VC; ++v) g.v[v] = cmul(dk, g.v[v]);
                }
#pragma unroll
                for (int v = 0; v < VC; ++v) acc[v] = cfma(l, g.v[v], acc[v]);
            }
            const int64_t base = (int64_t)row * W + c0;
            CV<T, VC> o = ldcv(In + base);
            if (UPPER) {
                const C di = Dinv[(int64_t)row * N + j];
#pragma unroll
                for (int v = 0; v < VC; ++v) o.v[v] = cmul(di, o.v[v]);
            }
#pragma unroll
            for (int v = 0; v < VC; ++v) o.v[v] = csub(o.v[v], acc[v]);
            stcv(Out + base, o);
            if (DOTS) {
                const CV<T, VC> r = ldcv(Rdot + base);
#pragma unroll
                for (int v = 0; v < VC; ++v) rz[v] = cfma(r.v[v], o.v[v], rz[v]);
            }
        }
    }
    if (DOTS) {
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

}  // namespace

template <typename T>
void ilu_apply(Ctx &ctx, const KrylovDims &d, const IluPattern &pat, const IluFactor<T> &fac, int tri_sweeps,
               int gy, const int32_t *flag, const cplx<T> *In, cplx<T> *Out, cplx<T> *F, cplx<T> *Ys, T *part) {
    constexpr int VC = VecN<T>::VC;
    const int W = d.W(), s = std::max(1, tri_sweeps);
    dim3 grid((W / VC + 31) / 32, gy), block(32, TY);
    const double vb = (double)d.n * W * d.frac * sizeof(cplx<T>);
    const double lb = (double)pat.nnzl * (8 + d.N * sizeof(cplx<T>));
    // lower sweeps y_t = In - N y_{t-1} (y_0 = In), ending in Ys
    const cplx<T> *prev = In;
    for (int t = 1; t <= s; ++t) {
        cplx<T> *dst = ((s - t) % 2 == 0) ? Ys : F;
        ctx.before(KC_KRYLOV_DIR, 3 * vb + lb, 8.0 * pat.nnzl * W * d.frac);
        k_ilu_tri<T, VC, false, false, false><<<grid, block, 0, ctx.stream>>>(
            d.n, W, d.Lp, d.N, pat.nnzl, pat.lptr, pat.lcol, nullptr, fac.L, fac.Dinv, In, prev, dst, nullptr, flag,
            nullptr);
        ctx.after();
        prev = dst;
    }
    // upper sweeps z_t = w - N^T z_{t-1} (z_0 = w = D^{-1} Ys), ending in Out
    for (int t = 1; t <= s; ++t) {
        cplx<T> *dst = ((s - t) % 2 == 0) ? Out : F;
        const bool last = t == s;
        ctx.before(KC_KRYLOV_DIR, (last && part ? 4 : 3) * vb + lb + (double)d.n * d.N * sizeof(cplx<T>),
                   8.0 * pat.nnzl * W * d.frac);
#define TRI(FIRST, DOTS)                                                                                        \
    k_ilu_tri<T, VC, true, FIRST, DOTS><<<grid, block, 0, ctx.stream>>>(d.n, W, d.Lp, d.N, pat.nnzl, pat.tptr,  \
                                                                         pat.trow, pat.tidx, fac.L, fac.Dinv, Ys, \
                                                                         t == 1 ? Ys : prev, dst, In, flag, part)
        if (t == 1 && last && part) TRI(true, true);
        else if (t == 1) TRI(true, false);
        else if (last && part) TRI(false, true);
        else TRI(false, false);
#undef TRI
        ctx.after();
        prev = dst;
    }
}

#define INST(T)                                                                                                     \
    template void ilu_factor<T>(Ctx &, const DevPencil &, const IluPattern &, const PoleSet<double> &, int, void *,  \
                                cplx<T> *, IluFactor<T> &);                                                        \
    template void ilu_apply<T>(Ctx &, const KrylovDims &, const IluPattern &, const IluFactor<T> &, int, int,       \
                               const int32_t *, const cplx<T> *, cplx<T> *, cplx<T> *, cplx<T> *, T *);
INST(float)
INST(double)
#undef INST

}  // namespace slrf
