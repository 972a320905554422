// Host construction of the smoothed-aggregation hierarchy (see mg.h).
//
// Per level: strength graph on nodes (blocks of `block` dofs), greedy
// aggregation, tentative prolongator T (piecewise constant per dof
// component), one damped-Jacobi smoothing step P = (I - w D^{-1} A) T with
// w = 4 / (3 rho(D^{-1} A)), Galerkin pencil (P^T A P, P^T B P).  The
// coarsest pencil is reduced to a standard eigenproblem through the Cholesky
// factor of B_c and diagonalised by Householder tridiagonalisation and the
// implicit symmetric QR iteration with Wilkinson shifts (Golub & Van Loan,
// Matrix Computations, Sections 8.3.1 and 8.3.3).  Everything is FP64 and
// deterministic: the row products are computed in parallel, but every row
// is formed by one thread in a fixed order and sorted by column.
#include "mg.h"
#include "host_pool.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <atomic>
#include <iterator>
#include <mutex>
#include <numeric>
#include <thread>

namespace slrf {
namespace {

int n_threads(int64_t work) { return host_threads(work); }

template <class Fn>
void parallel_for_rows(int nrows, int nt, Fn fn) {
    host_parallel_rows(nrows, nt, fn);
}

// Sparse rows produced by a per-row accumulator (sparse accumulator with a
// marker array), one or two value arrays.  `row_fn(i, add)` calls
// add(col, va, vb) for every contribution to row i.
struct RowsOut {
    std::vector<int32_t> ptr, col;
    std::vector<double> a, b;
};

template <class RowFn>
void build_rows(int nrows, int ncols, bool pair, int64_t work, RowFn row_fn, RowsOut &out) {
    const int nt = n_threads(work);
    struct Part {
        std::vector<int32_t> len, col;
        std::vector<double> a, b;
    };
    std::vector<Part> parts(nt);
    parallel_for_rows(nrows, nt, [&](int r0, int r1, int t) {
        Part &p = parts[t];
        p.len.reserve(r1 - r0);
        std::vector<int32_t> mark(ncols, -1), cols;
        std::vector<double> acc_a(ncols, 0.0), acc_b(pair ? ncols : 0, 0.0);
        for (int i = r0; i < r1; ++i) {
            cols.clear();
            auto add = [&](int c, double va, double vb) {
                if (mark[c] != i) {
                    mark[c] = i;
                    acc_a[c] = 0.0;
                    if (pair) acc_b[c] = 0.0;
                    cols.push_back(c);
                }
                acc_a[c] += va;
                if (pair) acc_b[c] += vb;
            };
            row_fn(i, add);
            std::sort(cols.begin(), cols.end());
            p.len.push_back((int32_t)cols.size());
            for (int c : cols) {
                p.col.push_back(c);
                p.a.push_back(acc_a[c]);
                if (pair) p.b.push_back(acc_b[c]);
            }
        }
    });
    out.ptr.assign(nrows + 1, 0);
    {
        int row = 0;
        for (auto &p : parts)
            for (int32_t l : p.len) {
                out.ptr[row + 1] = out.ptr[row] + l;
                ++row;
            }
    }
    const int64_t tot = out.ptr[nrows];
    out.col.resize(tot);
    out.a.resize(tot);
    if (pair) out.b.resize(tot);
    std::vector<int64_t> off(nt + 1, 0);
    for (int t = 0; t < nt; ++t) off[t + 1] = off[t] + (int64_t)parts[t].col.size();
    host_team(nt, [&](int t) {   // each part to its place
        const Part &p = parts[t];
        std::copy(p.col.begin(), p.col.end(), out.col.begin() + off[t]);
        std::copy(p.a.begin(), p.a.end(), out.a.begin() + off[t]);
        if (pair) std::copy(p.b.begin(), p.b.end(), out.b.begin() + off[t]);
    });
}

// Transpose of an nrows x ncols CSR pattern: tptr (ncols + 1) and, per entry
// of the transpose, its source row trow and source position tsrc; every row
// of the transpose lists its source rows ascending.  Row ranges in parallel:
// counts per (range, column), offsets in (column, range) order, then each
// range writes its entries; the result is that of one serial pass.
void transpose_pattern(int nrows, int ncols, const int32_t *ptr, const int32_t *col, std::vector<int32_t> &tptr,
                       int32_t *trow, int32_t *tsrc) {
    const int nt = n_threads(ptr[nrows]);
    std::vector<int32_t> cnt((size_t)nt * ncols, 0);
    parallel_for_rows(nrows, nt, [&](int r0, int r1, int t) {
        int32_t *c = &cnt[(size_t)t * ncols];
        for (int32_t k = ptr[r0]; k < ptr[r1]; ++k) c[col[k]]++;
    });
    tptr.assign(ncols + 1, 0);
    int32_t run = 0;
    for (int c = 0; c < ncols; ++c) {
        tptr[c] = run;
        for (int t = 0; t < nt; ++t) {
            const int32_t v = cnt[(size_t)t * ncols + c];
            cnt[(size_t)t * ncols + c] = run;
            run += v;
        }
    }
    tptr[ncols] = run;
    parallel_for_rows(nrows, nt, [&](int r0, int r1, int t) {
        int32_t *o = &cnt[(size_t)t * ncols];
        for (int i = r0; i < r1; ++i)
            for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
                const int32_t d = o[col[k]]++;
                trow[d] = i;
                tsrc[d] = k;
            }
    });
}

HostCsr transpose(const HostCsr &M) {
    HostCsr T;
    T.n_rows = M.n_cols;
    T.n_cols = M.n_rows;
    const size_t nz = M.col.size();
    T.col.resize(nz);
    T.val.resize(nz);
    std::vector<int32_t> src(nz);
    transpose_pattern(M.n_rows, M.n_cols, M.ptr.data(), M.col.data(), T.ptr, T.col.data(), src.data());
    parallel_for_rows((int)nz, n_threads((int64_t)nz), [&](int d0, int d1, int) {
        for (int d = d0; d < d1; ++d) T.val[d] = M.val[src[d]];
    });
    return T;
}

// Strong node neighbours: ||A_IJ||_F >= theta * sqrt(||A_II||_F ||A_JJ||_F).
// Node ranges in parallel; each node's list is formed by one thread, sorted.
void strength(int n, const int32_t *ptr, const int32_t *col, const double *a, int bs, double theta,
              std::vector<int32_t> &sptr, std::vector<int32_t> &scol) {
    const int nn = n / bs;
    std::vector<double> dnorm(nn, 0.0);   // ||A_II||_F^2
    const int nt = n_threads(ptr[n]);
    parallel_for_rows(nn, nt, [&](int I0, int I1, int) {
        for (int I = I0; I < I1; ++I) {
            const int lo = I * bs, hi = lo + bs;
            double t = 0.0;
            for (int i = lo; i < hi; ++i)
                for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k)
                    if (col[k] >= lo && col[k] < hi) t += a[k] * a[k];
            dnorm[I] = t;
        }
    });
    std::vector<std::vector<int32_t>> len(nt), out(nt);
    const double th2 = theta * theta;
    parallel_for_rows(nn, nt, [&](int I0, int I1, int t) {
        if (bs == 1) {   // rows hold each column once, ascending: no accumulation
            for (int I = I0; I < I1; ++I) {
                int32_t cnt = 0;
                for (int32_t k = ptr[I]; k < ptr[I + 1]; ++k) {
                    const int J = col[k];
                    if (J != I && a[k] * a[k] >= th2 * std::sqrt(dnorm[I] * dnorm[J])) {
                        out[t].push_back(J);
                        ++cnt;
                    }
                }
                len[t].push_back(cnt);
            }
            return;
        }
        std::vector<int32_t> mark(nn, -1), nb;
        std::vector<double> acc(nn, 0.0);
        for (int I = I0; I < I1; ++I) {
            nb.clear();
            for (int i = I * bs; i < I * bs + bs; ++i)
                for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
                    const int J = bs == 1 ? col[k] : col[k] / bs;
                    if (J == I) continue;
                    if (mark[J] != I) {
                        mark[J] = I;
                        acc[J] = 0.0;
                        nb.push_back(J);
                    }
                    acc[J] += a[k] * a[k];
                }
            std::sort(nb.begin(), nb.end());
            int32_t cnt = 0;
            for (int J : nb)
                if (acc[J] >= th2 * std::sqrt(dnorm[I] * dnorm[J])) {
                    out[t].push_back(J);
                    ++cnt;
                }
            len[t].push_back(cnt);
        }
    });
    sptr.assign(nn + 1, 0);
    int I = 0;
    std::vector<int64_t> off(nt + 1, 0);
    for (int t = 0; t < nt; ++t) {
        for (int32_t l : len[t]) {
            sptr[I + 1] = sptr[I] + l;
            ++I;
        }
        off[t + 1] = off[t] + (int64_t)out[t].size();
    }
    scol.resize(off[nt]);
    host_team(nt, [&](int t) { std::copy(out[t].begin(), out[t].end(), scol.begin() + off[t]); });
}

// Greedy aggregation in node order: (1) a node whose strong neighbours are
// all free starts an aggregate with them; (2) a free node joins the
// aggregate of a strong neighbour assigned in (1); (3) what is left forms
// aggregates with its free strong neighbours.
int aggregate(int nn, const std::vector<int32_t> &sptr, const std::vector<int32_t> &scol, std::vector<int32_t> &agg) {
    agg.assign(nn, -1);
    int na = 0;
    for (int i = 0; i < nn; ++i) {
        if (agg[i] >= 0) continue;
        bool free_all = true;
        for (int32_t k = sptr[i]; k < sptr[i + 1] && free_all; ++k) free_all = agg[scol[k]] < 0;
        if (!free_all) continue;
        agg[i] = na;
        for (int32_t k = sptr[i]; k < sptr[i + 1]; ++k) agg[scol[k]] = na;
        ++na;
    }
    std::vector<int32_t> first(agg);
    for (int i = 0; i < nn; ++i) {
        if (agg[i] >= 0) continue;
        for (int32_t k = sptr[i]; k < sptr[i + 1]; ++k)
            if (first[scol[k]] >= 0) {
                agg[i] = first[scol[k]];
                break;
            }
    }
    for (int i = 0; i < nn; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = na;
        for (int32_t k = sptr[i]; k < sptr[i + 1]; ++k)
            if (agg[scol[k]] < 0) agg[scol[k]] = na;
        ++na;
    }
    return na;
}

// Reusable barrier for a fixed team of threads.
class Barrier {
  public:
    explicit Barrier(int n) : n_(n), left_(n) {}
    // The last thread to arrive opens the next generation; the others spin
    // briefly on it (the teams here pass one barrier every few microseconds)
    // and then sleep on the condition variable.
    void wait() {
        const int64_t g = gen_.load(std::memory_order_acquire);
        if (left_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
            left_.store(n_, std::memory_order_relaxed);
            {
                std::lock_guard<std::mutex> lk(m_);
                gen_.store(g + 1, std::memory_order_release);
            }
            cv_.notify_all();
            return;
        }
        for (int i = 0; i < 20000; ++i)
            if (gen_.load(std::memory_order_acquire) != g) return;
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != g; });
    }

  private:
    std::mutex m_;
    std::condition_variable cv_;
    const int n_;
    std::atomic<int> left_;
    std::atomic<int64_t> gen_{0};
};

// Aggregates of fewer than min_nodes nodes join the aggregate of a neighbour
// node in the matrix graph: for each small aggregate in turn (ascending), the
// first neighbour, in node then column order, that lies in another
// aggregate.  The aggregates are then renumbered by their first node.
// Returns the new count.
int merge_small_aggregates(int nn, int bs, const int32_t *ptr, const int32_t *col, int min_nodes,
                           std::vector<int32_t> &agg, int na) {
    if (min_nodes <= 1) return na;
    std::vector<int32_t> parent(na), size(na, 0), first(na, -1);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int a) {
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        return a;
    };
    for (int I = 0; I < nn; ++I) {
        size[agg[I]]++;
        if (first[agg[I]] < 0) first[agg[I]] = I;
    }
    // nodes of each aggregate, ascending (counting sort)
    std::vector<int32_t> aptr(na + 1, 0), anode(nn);
    for (int I = 0; I < nn; ++I) aptr[agg[I] + 1]++;
    for (int a = 0; a < na; ++a) aptr[a + 1] += aptr[a];
    {
        std::vector<int32_t> fill(aptr.begin(), aptr.end() - 1);
        for (int I = 0; I < nn; ++I) anode[fill[agg[I]]++] = I;
    }
    for (int a = 0; a < na; ++a) {
        const int ra = find(a);
        if (ra != a || size[ra] >= min_nodes) continue;
        int target = -1;
        for (int32_t t = aptr[a]; t < aptr[a + 1] && target < 0; ++t)
            for (int i = anode[t] * bs; i < anode[t] * bs + bs && target < 0; ++i)
                for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
                    const int rb = find(agg[col[k] / bs]);
                    if (rb != ra) {
                        target = rb;
                        break;
                    }
                }
        if (target < 0) continue;   // isolated: left as it is
        parent[ra] = target;
        size[target] += size[ra];
    }
    std::vector<int32_t> id(na, -1);
    int cnt = 0;
    for (int I = 0; I < nn; ++I) {
        const int r = find(agg[I]);
        if (id[r] < 0) id[r] = cnt++;
        agg[I] = id[r];
    }
    return cnt;
}

// Tentative prolongator from a near-null space Bn (cn x kn, row-major): per
// aggregate the thin QR of its rows (dofs of its nodes in ascending order),
// by modified Gram-Schmidt with a second pass; a column whose remainder is
// below 1e-10 of its norm is replaced by the unit vector with the largest
// component outside the columns so far (R keeps zero on its diagonal).
// tval (cn x kn): row i of T holds Q's row of dof i in columns agg*kn ..
// agg*kn + kn - 1; Bc (na*kn x kn): the R factors, stacked.  Returns false if
// an aggregate has fewer dofs than kn.
bool tentative_qr(int cn, int bs, int kn, const std::vector<int32_t> &agg, int na, const std::vector<double> &Bn,
                  std::vector<double> &tval, std::vector<double> &Bc) {
    const int nn = cn / bs;
    std::vector<int32_t> aptr(na + 1, 0), anode(nn);
    for (int I = 0; I < nn; ++I) aptr[agg[I] + 1]++;
    for (int a = 0; a < na; ++a) aptr[a + 1] += aptr[a];
    {
        std::vector<int32_t> fill(aptr.begin(), aptr.end() - 1);
        for (int I = 0; I < nn; ++I) anode[fill[agg[I]]++] = I;
    }
    for (int a = 0; a < na; ++a)
        if ((aptr[a + 1] - aptr[a]) * bs < kn) return false;
    tval.assign((size_t)cn * kn, 0.0);
    Bc.assign((size_t)na * kn * kn, 0.0);
    parallel_for_rows(na, n_threads((int64_t)cn * kn * kn), [&](int a0, int a1, int) {
        std::vector<double> Q, v;
        for (int a = a0; a < a1; ++a) {
            const int m = (aptr[a + 1] - aptr[a]) * bs;
            auto dof = [&](int l) { return anode[aptr[a] + l / bs] * bs + l % bs; };
            Q.assign((size_t)m * kn, 0.0);   // column-major m x kn
            double *R = &Bc[(size_t)a * kn * kn];
            for (int j = 0; j < kn; ++j) {
                v.resize(m);
                double n0 = 0.0;
                for (int l = 0; l < m; ++l) {
                    v[l] = Bn[(size_t)dof(l) * kn + j];
                    n0 += v[l] * v[l];
                }
                n0 = std::sqrt(n0);
                for (int pass = 0; pass < 2; ++pass)
                    for (int i = 0; i < j; ++i) {
                        const double *qi = &Q[(size_t)i * m];
                        double r = 0.0;
                        for (int l = 0; l < m; ++l) r += qi[l] * v[l];
                        for (int l = 0; l < m; ++l) v[l] -= r * qi[l];
                        R[(size_t)i * kn + j] += r;
                    }
                double nv = 0.0;
                for (int l = 0; l < m; ++l) nv += v[l] * v[l];
                nv = std::sqrt(nv);
                if (nv > 1e-10 * n0 && nv > 0.0) {
                    R[(size_t)j * kn + j] = nv;
                } else {   // deficient: complete with the unit vector least inside span(Q)
                    int best = 0;
                    double bestr = -1.0;
                    for (int l = 0; l < m; ++l) {
                        double in = 0.0;
                        for (int i = 0; i < j; ++i) in += Q[(size_t)i * m + l] * Q[(size_t)i * m + l];
                        if (1.0 - in > bestr) {
                            bestr = 1.0 - in;
                            best = l;
                        }
                    }
                    std::fill(v.begin(), v.end(), 0.0);
                    v[best] = 1.0;
                    for (int pass = 0; pass < 2; ++pass)
                        for (int i = 0; i < j; ++i) {
                            const double *qi = &Q[(size_t)i * m];
                            double r = 0.0;
                            for (int l = 0; l < m; ++l) r += qi[l] * v[l];
                            for (int l = 0; l < m; ++l) v[l] -= r * qi[l];
                        }
                    nv = 0.0;
                    for (int l = 0; l < m; ++l) nv += v[l] * v[l];
                    nv = std::sqrt(nv);
                }
                double *qj = &Q[(size_t)j * m];
                for (int l = 0; l < m; ++l) qj[l] = v[l] / nv;
            }
            for (int l = 0; l < m; ++l)
                for (int j = 0; j < kn; ++j) tval[(size_t)dof(l) * kn + j] = Q[(size_t)j * m + l];
        }
    });
    return true;
}

// Largest |eigenvalue| of D^{-1} A by power iteration (deterministic start).
// One team of threads runs all the steps on fixed row chunks; the squared
// norms are summed per chunk and the chunks added in order by every thread,
// so the estimate does not depend on the thread count.
double rho_dinv_a(int n, const int32_t *ptr, const int32_t *col, const double *a, const std::vector<double> &d) {
    constexpr int NIT = 30, NCH = 64;
    std::vector<double> buf[2] = {std::vector<double>(n), std::vector<double>(n)};
    uint64_t s = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < n; ++i) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        buf[0][i] = 0.5 + (double)(s >> 11) * (1.0 / 9007199254740992.0);
    }
    // step it: y = (D^{-1} A x) * scale with x = buf[it & 1] the previous,
    // unnormalised iterate and scale = 1 / ||x_prev||; the normalised x has
    // squared norm sum (scale x_i)^2 over its rows
    std::vector<double> part[2] = {std::vector<double>(2 * NCH), std::vector<double>(2 * NCH)};
    auto chunk = [&](int c) { return (int)((int64_t)n * c / NCH); };
    // 30 sweeps over the pattern: threads pay off from ~50 k stored entries
    const int nt = n_threads((int64_t)ptr[n] * 4);
    Barrier bar(nt);
    double lam_out = 0.0;
    auto team = [&](int c0, int c1, int tid) {
        double scale = 1.0, lam = 0.0;
        for (int it = 0; it < NIT; ++it) {
            const std::vector<double> &x = buf[it & 1];
            std::vector<double> &y = buf[(it + 1) & 1];
            std::vector<double> &pp = part[it & 1];
            for (int c = c0; c < c1; ++c) {
                double sx = 0.0, sy = 0.0;
                for (int i = chunk(c); i < chunk(c + 1); ++i) {
                    double t = 0.0;
                    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) t += a[k] * x[col[k]];
                    const double yi = t / d[i] * scale, xi = x[i] * scale;
                    y[i] = yi;
                    sx += xi * xi;
                    sy += yi * yi;
                }
                pp[2 * c] = sx;
                pp[2 * c + 1] = sy;
            }
            bar.wait();
            double nx = 0.0, ny = 0.0;
            for (int c = 0; c < NCH; ++c) {
                nx += pp[2 * c];
                ny += pp[2 * c + 1];
            }
            lam = std::sqrt(ny / nx);
            scale = 1.0 / std::sqrt(ny);
        }
        if (tid == 0) lam_out = lam;
    };
    host_team(nt, [&](int t) { team(NCH * t / nt, NCH * (t + 1) / nt, t); });
    return lam_out;
}

// In-place dense Cholesky S = L L^T (lower, row-major); false if not SPD.
bool cholesky_lower(int n, std::vector<double> &S) {
    for (int j = 0; j < n; ++j) {
        double djj = S[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) djj -= S[(size_t)j * n + k] * S[(size_t)j * n + k];
        if (!(djj > 0.0) || !std::isfinite(djj)) return false;
        const double ljj = std::sqrt(djj);
        S[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = S[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= S[(size_t)i * n + k] * S[(size_t)j * n + k];
            S[(size_t)i * n + j] = t / ljj;
        }
        for (int k = j + 1; k < n; ++k) S[(size_t)j * n + k] = 0.0;
    }
    return true;
}

// Threads for the O(n^3) steps of an n x n dense problem (one below n = 320,
// where the per-step barriers of the reduction would cost more than they save).
int dense_threads(int n) { return n >= 320 ? n_threads((int64_t)n * n * n) : 1; }

}  // namespace

// V^T A_l V = diag(lam), V^T B_l V = I.
std::string mg_level_eig(const HostLevel &L, std::vector<double> &V, std::vector<double> &lam) {
    const int n = L.n;
    std::vector<double> Ad((size_t)n * n, 0.0), Bd((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int32_t k = L.ptr[i]; k < L.ptr[i + 1]; ++k) {
            Ad[(size_t)i * n + L.col[k]] = L.a[k];
            Bd[(size_t)i * n + L.col[k]] = L.b[k];
        }
    // symmetrise (Galerkin products are symmetric up to rounding)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            const double sa = 0.5 * (Ad[(size_t)i * n + j] + Ad[(size_t)j * n + i]);
            const double sb = 0.5 * (Bd[(size_t)i * n + j] + Bd[(size_t)j * n + i]);
            Ad[(size_t)i * n + j] = Ad[(size_t)j * n + i] = sa;
            Bd[(size_t)i * n + j] = Bd[(size_t)j * n + i] = sb;
        }
    if (!cholesky_lower(n, Bd)) return "multigrid setup: coarse mass matrix is not positive definite";
    // Y <- L^{-1} Y by forward substitution, one row of Y at a time (the
    // inner loops run along rows of the row-major arrays); the columns of Y
    // are independent, so threads take column ranges
    const int nt = dense_threads(n);
    auto forward = [&](std::vector<double> &Y) {
        parallel_for_rows(n, nt, [&](int c0, int c1, int) {
            for (int i = 0; i < n; ++i) {
                double *__restrict yi = &Y[(size_t)i * n];
                for (int k = 0; k < i; ++k) {
                    const double l = Bd[(size_t)i * n + k];
                    const double *__restrict yk = &Y[(size_t)k * n];
                    for (int c = c0; c < c1; ++c) yi[c] -= l * yk[c];
                }
                const double inv = 1.0 / Bd[(size_t)i * n + i];
                for (int c = c0; c < c1; ++c) yi[c] *= inv;
            }
        });
    };
    // X = L^{-1} A_c, then C = L^{-1} X^T (= L^{-1} A_c L^{-T})
    std::vector<double> X(Ad);
    forward(X);
    std::vector<double> C((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < n; ++c) C[(size_t)i * n + c] = X[(size_t)c * n + i];
    forward(C);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            const double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
            C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
        }
    std::vector<double> Q;
    host_syev(n, C, lam, Q);
    // V = L^{-T} Q (back substitution, one row of V at a time, column ranges
    // in parallel)
    V = Q;
    parallel_for_rows(n, nt, [&](int c0, int c1, int) {
        for (int i = n - 1; i >= 0; --i) {
            double *__restrict vi = &V[(size_t)i * n];
            for (int k = i + 1; k < n; ++k) {
                const double l = Bd[(size_t)k * n + i];
                const double *__restrict vk = &V[(size_t)k * n];
                for (int c = c0; c < c1; ++c) vi[c] -= l * vk[c];
            }
            const double inv = 1.0 / Bd[(size_t)i * n + i];
            for (int c = c0; c < c1; ++c) vi[c] *= inv;
        }
    });
    return "";
}

void host_syev(int n, std::vector<double> &S, std::vector<double> &w, std::vector<double> &Q) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    std::vector<double> v(n), p(n), q(n);
    // Householder reduction to tridiagonal form: S <- H S H on the trailing
    // block, Q <- Q H, for each column k.  One team of threads: thread 0 forms
    // the reflector, all threads update row ranges between barriers; every
    // entry is computed by one thread in the same order whatever the team size.
    struct Refl {
        bool skip = true;
        double alpha = 0.0, beta = 0.0, vv = 0.0;
    } rf[2];
    const int nt = dense_threads(n);
    Barrier bar(nt);
    auto range = [&](int m, int t, int &r0, int &r1) {
        r0 = (int)((int64_t)m * t / nt);
        r1 = (int)((int64_t)m * (t + 1) / nt);
    };
    auto reduce = [&](int, int, int tid) {
        for (int k = 0; k + 2 < n; ++k) {
            const int m = n - k - 1;   // length of the sub-column
            Refl &R = rf[k & 1];
            if (tid == 0) {
                double xn = 0.0;
                for (int i = 0; i < m; ++i) {
                    v[i] = S[(size_t)(k + 1 + i) * n + k];
                    xn += v[i] * v[i];
                }
                xn = std::sqrt(xn);
                R.skip = xn == 0.0;
                if (!R.skip) {
                    R.alpha = v[0] > 0 ? -xn : xn;
                    v[0] -= R.alpha;
                    R.vv = 0.0;
                    for (int i = 0; i < m; ++i) R.vv += v[i] * v[i];
                    R.skip = !(R.vv > 0.0);
                    R.beta = R.skip ? 0.0 : 2.0 / R.vv;
                }
            }
            bar.wait();
            if (R.skip) continue;
            int r0, r1;
            range(m, tid, r0, r1);
            // p = beta * S22 v
            for (int i = r0; i < r1; ++i) {
                double t = 0.0;
                const double *row = &S[(size_t)(k + 1 + i) * n + k + 1];
                for (int j = 0; j < m; ++j) t += row[j] * v[j];
                p[i] = R.beta * t;
            }
            bar.wait();
            if (tid == 0) {
                double vp = 0.0;
                for (int i = 0; i < m; ++i) vp += v[i] * p[i];
                const double K = vp / R.vv;
                for (int i = 0; i < m; ++i) q[i] = p[i] - K * v[i];
            }
            bar.wait();
            {
                const double *__restrict vp_ = v.data();
                const double *__restrict qp_ = q.data();
                for (int i = r0; i < r1; ++i) {
                    double *__restrict row = &S[(size_t)(k + 1 + i) * n + k + 1];
                    const double vi = vp_[i], qi = qp_[i];
                    for (int j = 0; j < m; ++j) row[j] -= vi * qp_[j] + qi * vp_[j];
                }
            }
            // Q[:, k+1:] -= beta (Q[:, k+1:] v) v^T
            int q0, q1;
            range(n, tid, q0, q1);
            for (int r = q0; r < q1; ++r) {
                double t = 0.0;
                double *__restrict row = &Q[(size_t)r * n + k + 1];
                const double *__restrict vp_ = v.data();
                for (int j = 0; j < m; ++j) t += row[j] * vp_[j];
                const double f = R.beta * t;
                for (int j = 0; j < m; ++j) row[j] -= f * vp_[j];
            }
            if (tid == 0) {
                S[(size_t)(k + 1) * n + k] = S[(size_t)k * n + k + 1] = R.alpha;
                for (int i = 1; i < m; ++i) S[(size_t)(k + 1 + i) * n + k] = S[(size_t)k * n + k + 1 + i] = 0.0;
            }
            bar.wait();
        }
    };
    host_team(nt, [&](int t) { reduce(0, 0, t); });
    // the QR phase rotates pairs of eigenvector columns: keep them as rows of Q^T
    std::vector<double> Qt((size_t)n * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Qt[(size_t)c * n + r] = Q[(size_t)r * n + c];
    std::vector<double> d(n), e(n > 0 ? n : 1, 0.0);
    for (int i = 0; i < n; ++i) d[i] = S[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = S[(size_t)(i + 1) * n + i];
    // Implicit symmetric QR steps with Wilkinson shifts on the unreduced
    // trailing block; each Givens rotation R on (k, k+1) maps T -> R T R^T
    // and Q -> Q R^T.  The rotations are recorded and applied to Q^T at the
    // end, each thread to its own range of components (in the same order).
    std::vector<int32_t> rot_k;
    std::vector<double> rot_c, rot_s;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1;
    int64_t guard = 0;
    const int64_t guard_max = 60LL * n + 100;
    while (hi > 0 && guard < guard_max) {
        for (int i = 0; i < hi; ++i)
            if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
        while (hi > 0 && e[hi - 1] == 0.0) --hi;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) --lo;
        ++guard;
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double mu = d[hi] - eh * eh / (dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, eh));
        double x = d[lo] - mu, z = e[lo], bulge = 0.0;
        for (int k = lo; k < hi; ++k) {
            if (k > lo) {
                x = e[k - 1];
                z = bulge;
            }
            const double r = std::hypot(x, z);
            double c = 1.0, s = 0.0;
            if (r > 0.0) {
                c = x / r;
                s = z / r;
            }
            if (k > lo) e[k - 1] = r;
            const double a0 = d[k], b0 = e[k], a1 = d[k + 1];
            d[k] = c * c * a0 + 2.0 * c * s * b0 + s * s * a1;
            d[k + 1] = s * s * a0 - 2.0 * c * s * b0 + c * c * a1;
            e[k] = c * s * (a1 - a0) + (c * c - s * s) * b0;
            if (k + 1 < hi) {
                bulge = s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            rot_k.push_back(k);
            rot_c.push_back(c);
            rot_s.push_back(s);
        }
    }
    // one parallel region without barriers: worth threads well below the
    // size at which the reduction's per-step barriers pay
    parallel_for_rows(n, n >= 64 ? n_threads((int64_t)rot_k.size() * n) : 1, [&](int c0, int c1, int) {
        for (size_t t = 0; t < rot_k.size(); ++t) {
            const double c = rot_c[t], s = rot_s[t];
            double *__restrict qk = &Qt[(size_t)rot_k[t] * n];
            double *__restrict qk1 = qk + n;
            for (int row = c0; row < c1; ++row) {
                const double zk = qk[row], zk1 = qk1[row];
                qk[row] = c * zk + s * zk1;
                qk1[row] = -s * zk + c * zk1;
            }
        }
    });
    // ascending order
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] < d[j]; });
    w.resize(n);
    std::vector<double> Qs((size_t)n * n);
    for (int c = 0; c < n; ++c) {
        w[c] = d[idx[c]];
        for (int r = 0; r < n; ++r) Qs[(size_t)r * n + c] = Qt[(size_t)idx[c] * n + r];
    }
    Q.swap(Qs);
}

void mg_fused_pattern(const HostLevel &L0, int n_coarse, int R, FusedLayout &out) {
    out = FusedLayout();
    out.R = R;
    const int64_t n0 = L0.n, ng = (n0 + R - 1) / R;
    // up: groups of R fine rows, sorted union of their coarse columns.  Group
    // ranges in parallel: unions per thread, then one prefix sum; the layout
    // does not depend on the thread count.
    const int nt = n_threads((int64_t)L0.fcol.size() * 4);
    std::vector<std::vector<int32_t>> ucat(nt);
    std::vector<int32_t> glen(ng);
    parallel_for_rows((int)ng, nt, [&](int g0, int g1, int t) {
        std::vector<int32_t> u, w;
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t r0 = g * R, r1 = std::min<int64_t>(n0, r0 + R);
            u.clear();
            for (int64_t r = r0; r < r1; ++r) {   // rows are ascending without repeats: set unions
                w.clear();
                std::set_union(u.begin(), u.end(), L0.fcol.begin() + L0.fptr[r], L0.fcol.begin() + L0.fptr[r + 1],
                               std::back_inserter(w));
                u.swap(w);
            }
            glen[g] = (int32_t)u.size();
            ucat[t].insert(ucat[t].end(), u.begin(), u.end());
        }
    });
    out.up_ptr.assign(ng + 1, 0);
    for (int64_t g = 0; g < ng; ++g) out.up_ptr[g + 1] = out.up_ptr[g] + glen[g];
    out.up_col.resize(out.up_ptr[ng]);
    host_team(nt, [&](int t) {
        const int64_t g0 = ng * t / nt;   // the first group of range t
        std::copy(ucat[t].begin(), ucat[t].end(), out.up_col.begin() + out.up_ptr[g0]);
    });
    // down: F^T, coarse row c lists the fine rows i with an entry (i, c),
    // ascending, and their positions in the pattern of A P
    const int64_t nz = (int64_t)L0.fcol.size();
    out.down_col.resize(nz);
    out.down_src.resize(nz);
    transpose_pattern((int)n0, n_coarse, L0.fptr.data(), L0.fcol.data(), out.down_ptr, out.down_col.data(),
                      out.down_src.data());
}

void mg_fused_values(const HostLevel &L0, const FusedLayout &FL, double *q_out) {
    const int R = FL.R;
    const int64_t n0 = L0.n, ng = (int64_t)FL.up_ptr.size() - 1, nz = (int64_t)FL.down_col.size();
    // the four values of one stored pair (fine row i, entry k of A P's
    // pattern), or zeros for a padding slot
    auto slot = [&](double *q, int64_t i, int32_t k, bool hit) {
        if (!hit) {
            q[0] = q[1] = q[2] = q[3] = 0.0;
            return;
        }
        q[0] = L0.fap[k];
        q[1] = L0.fbp[k];
        q[2] = L0.fp[k] * L0.diag_a[i];
        q[3] = L0.fp[k] * L0.diag_b[i];
    };
    const int nt = n_threads((int64_t)L0.fcol.size() * 4);
    double *q_up = q_out, *q_dn = q_out + FL.up_col.size() * (size_t)R * 4;
    parallel_for_rows((int)ng, nt, [&](int g0, int g1, int) {
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t r0 = g * R;
            // the group's union list and each row's list are both ascending:
            // one cursor per row walks its list along the union
            for (int r = 0; r < R; ++r) {
                const int64_t row = r0 + r;
                int32_t k = row < n0 ? L0.fptr[row] : 0;
                const int32_t k1 = row < n0 ? L0.fptr[row + 1] : 0;
                for (int32_t e = FL.up_ptr[g]; e < FL.up_ptr[g + 1]; ++e) {
                    double *q = q_up + ((size_t)e * R + r) * 4;
                    const bool hit = k < k1 && L0.fcol[k] == FL.up_col[e];
                    slot(q, hit ? row : 0, hit ? k : 0, hit);
                    if (hit) ++k;
                }
            }
        }
    });
    parallel_for_rows((int)nz, nt, [&](int d0, int d1, int) {
        for (int64_t d = d0; d < d1; ++d) slot(q_dn + (size_t)d * 4, FL.down_col[d], FL.down_src[d], true);
    });
}

std::string mg_build(int n, const int32_t *ptr, const int32_t *col, const double *a, const double *b,
                     const MgParams &prm, HostHierarchy &H) {
    const auto t0 = std::chrono::steady_clock::now();
    H = HostHierarchy();
    int bs = (prm.block > 1 && n % prm.block == 0) ? prm.block : 1;
    // near-null space of the current level (cn x kn); kn = 0: the constant
    // per dof component
    int kn = prm.near_null && prm.n_null > 0 ? prm.n_null : 0;
    std::vector<double> Bn;
    if (kn) Bn.assign(prm.near_null, prm.near_null + (size_t)n * kn);
    // current level as raw arrays (level 0 borrows the caller's pencil)
    const int32_t *cp = ptr, *cc = col;
    const double *ca = a, *cb = b;
    int cn = n;
    H.lv.emplace_back();
    H.lv[0].n = n;
    for (;;) {
        HostLevel &L = H.lv.back();
        L.diag_a.assign(cn, 0.0);
        L.diag_b.assign(cn, 0.0);
        parallel_for_rows(cn, n_threads(cp[cn]), [&](int r0, int r1, int) {
            for (int i = r0; i < r1; ++i)
                for (int32_t k = cp[i]; k < cp[i + 1]; ++k)
                    if (cc[k] == i) {
                        L.diag_a[i] += ca[k];
                        L.diag_b[i] += cb[k];
                    }
        });
        for (int i = 0; i < cn; ++i)
            if (!(L.diag_a[i] > 0.0) || !(L.diag_b[i] > 0.0))
                return "multigrid setup: non-positive diagonal entry in row " + std::to_string(i);
        for (int i = 0; i < cn; ++i) L.maxba = std::max(L.maxba, L.diag_b[i] / L.diag_a[i]);
        if (cn <= prm.coarse_target || (int)H.lv.size() >= prm.max_levels) break;
        // aggregation on the node graph
        std::vector<int32_t> sptr, scol, agg;
        strength(cn, cp, cc, ca, bs, prm.theta, sptr, scol);
        const int nn = cn / bs;
        int na = aggregate(nn, sptr, scol, agg);
        if (kn) na = merge_small_aggregates(nn, bs, cp, cc, (kn + bs - 1) / bs, agg, na);
        const int nc = na * (kn ? kn : bs);
        if (nc >= cn || nc > 0.85 * cn) break;   // coarsening stalled
        std::vector<int32_t> tcol;
        std::vector<double> tval, Bc;
        if (kn) {   // T from the near-null space: kn entries per row
            if (!tentative_qr(cn, bs, kn, agg, na, Bn, tval, Bc))
                return "multigrid setup: an aggregate has fewer unknowns than the near-null space";
        } else {   // T: the constant per dof component, one entry per row
            std::vector<int32_t> asz(na, 0);
            for (int I = 0; I < nn; ++I) asz[agg[I]]++;
            tcol.resize(cn);
            tval.resize(cn);
            for (int i = 0; i < cn; ++i) {
                const int I = i / bs, c = i % bs;
                tcol[i] = agg[I] * bs + c;
                tval[i] = 1.0 / std::sqrt((double)asz[agg[I]]);
            }
        }
        // P = T - w D^{-1} A T
        L.rho = rho_dinv_a(cn, cp, cc, ca, L.diag_a);
        const double w = 4.0 / (3.0 * L.rho);
        RowsOut Pr;
        if (kn) {
            build_rows(cn, nc, false, (int64_t)cp[cn] * kn, [&](int i, auto &add) {
                const double f = -w / L.diag_a[i];
                for (int32_t k = cp[i]; k < cp[i + 1]; ++k) {
                    const int j = cc[k], c0 = agg[j / bs] * kn;
                    for (int t = 0; t < kn; ++t) add(c0 + t, f * ca[k] * tval[(size_t)j * kn + t], 0.0);
                }
                const int c0 = agg[i / bs] * kn;
                for (int t = 0; t < kn; ++t) add(c0 + t, tval[(size_t)i * kn + t], 0.0);
            }, Pr);
        } else {
            build_rows(cn, nc, false, (int64_t)cp[cn], [&](int i, auto &add) {
                const double f = -w / L.diag_a[i];
                for (int32_t k = cp[i]; k < cp[i + 1]; ++k) add(tcol[cc[k]], f * ca[k] * tval[cc[k]], 0.0);
                add(tcol[i], tval[i], 0.0);
            }, Pr);
        }
        L.P.n_rows = cn;
        L.P.n_cols = nc;
        L.P.ptr = std::move(Pr.ptr);
        L.P.col = std::move(Pr.col);
        L.P.val = std::move(Pr.a);
        L.Rt = transpose(L.P);
        // (A P, B P), then P^T (A P, B P)
        RowsOut APr;
        const HostCsr &P = L.P;
        build_rows(cn, nc, true, (int64_t)cp[cn] * 8, [&](int i, auto &add) {
            for (int32_t k = cp[i]; k < cp[i + 1]; ++k) {
                const int j = cc[k];
                for (int32_t t = P.ptr[j]; t < P.ptr[j + 1]; ++t) add(P.col[t], ca[k] * P.val[t], cb[k] * P.val[t]);
            }
        }, APr);
        HostLevel next;
        next.n = nc;
        RowsOut Cr;
        const HostCsr &Rt = L.Rt;
        build_rows(nc, nc, true, (int64_t)APr.ptr[cn] * 4, [&](int I, auto &add) {
            for (int32_t t = Rt.ptr[I]; t < Rt.ptr[I + 1]; ++t) {
                const int i = Rt.col[t];
                const double r = Rt.val[t];
                for (int32_t k = APr.ptr[i]; k < APr.ptr[i + 1]; ++k) add(APr.col[k], r * APr.a[k], r * APr.b[k]);
            }
        }, Cr);
        if (H.lv.size() == 1) {   // finest level: keep (P, A P, B P) on the pattern of A P
            L.fptr = std::move(APr.ptr);
            L.fcol = std::move(APr.col);
            L.fap = std::move(APr.a);
            L.fbp = std::move(APr.b);
            L.fp.assign(L.fcol.size(), 0.0);
            std::atomic<bool> outside{false};
            parallel_for_rows(cn, n_threads((int64_t)L.fcol.size()), [&](int r0, int r1, int) {
                for (int i = r0; i < r1; ++i) {
                    int32_t k = L.fptr[i];
                    for (int32_t t = P.ptr[i]; t < P.ptr[i + 1]; ++t) {
                        while (k < L.fptr[i + 1] && L.fcol[k] < P.col[t]) ++k;
                        if (k < L.fptr[i + 1] && L.fcol[k] == P.col[t]) L.fp[k] = P.val[t];
                        else outside.store(true, std::memory_order_relaxed);
                    }
                }
            });
            if (outside.load()) return "multigrid setup: prolongator entry outside the pattern of A P";
        }
        next.ptr = std::move(Cr.ptr);
        next.col = std::move(Cr.col);
        next.a = std::move(Cr.a);
        next.b = std::move(Cr.b);
        H.lv.push_back(std::move(next));
        HostLevel &N2 = H.lv.back();
        cp = N2.ptr.data();
        cc = N2.col.data();
        ca = N2.a.data();
        cb = N2.b.data();
        cn = nc;
        if (kn) {   // the next level: kn dofs per node, near-null space from the R factors
            bs = kn;
            Bn.swap(Bc);
            N2.nullspace = Bn;
            N2.n_null = kn;
        }
    }
    HostLevel &Lc = H.lv.back();
    if (H.lv.size() == 1) {   // no coarsening: the coarsest level is the pencil itself
        Lc.ptr.assign(ptr, ptr + n + 1);
        Lc.col.assign(col, col + ptr[n]);
        Lc.a.assign(a, a + ptr[n]);
        Lc.b.assign(b, b + ptr[n]);
    }
    if (Lc.n > 4096) return "multigrid setup: coarsening stalled at " + std::to_string(Lc.n) + " unknowns";
    if (!prm.defer_coarse_eig) {
        std::string err = mg_coarse_eig(H);
        if (!err.empty()) return err;
    }
    H.ms_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return "";
}

std::string mg_coarse_eig(HostHierarchy &H) {
    HostLevel &Lc = H.lv.back();
    std::string err = mg_level_eig(Lc, H.V, H.lam);
    if (!err.empty()) return err;
    if (H.lv.size() == 1) {   // level 0 keeps no pencil copy
        Lc.ptr.clear();
        Lc.col.clear();
        Lc.a.clear();
        Lc.b.clear();
    }
    return "";
}

}  // namespace slrf
