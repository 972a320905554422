// Host-side pole/weight sets of the rational filter (not timed; FP64).
//
// Phi(x) = sum_j 2 Re(w_j / (x - sigma_j)) on the real axis (Section 3, filter
// of the conjugate-pair reduction).
//
// * Quadrature rules on the circle with centre c = gamma/2, radius r = gamma/2
//   (Section 3.2).  With z(t) = c + r e^{it}, the projector's contour integral
//   (1/2 pi i) \oint dz/(z - x) equals (1/2 pi) \int r e^{it}/(z(t) - x) dt, so
//   an angle rule (t_k, omega_k) on (0, pi) gives sigma_k = z(t_k) and
//   w_k = -r e^{i t_k} omega_k / (2 pi); the lower half plane is the mirror.
//     midpoint:        t_k = (2k-1) pi / (2N), omega_k = pi / N
//     Gauss-Legendre:  nodes s_k of P_N, t_k = pi (1 - s_k)/2, omega_k = (pi/2) g_k
//     Gauss-Chebyshev: s_k = cos((2k-1) pi/(2N)), t_k = pi (1 - s_k)/2,
//                      omega_k = (pi/2)(pi/N) sqrt(1 - s_k^2)
// * SLRF (Section 3.1): sigma_j = x_j (1 + i alpha), x_j in (0, gamma];
//   minimise ||Phi - h||_delta^2 with delta = beta on [0, gamma], 1 on
//   (gamma, 10 gamma], trapezoidal rule on each piece.  For fixed x the weights
//   solve a weighted linear least-squares problem (Householder QR here); the
//   abscissae are optimised by a projected Levenberg-Marquardt iteration on
//   their increments (kept >= 1/(4N) apart) from six deterministic starts.
//   The design is done at gamma = 1 and scaled: sigma -> gamma sigma,
//   w -> gamma w, because Phi_gamma(x) = Phi_1(x / gamma).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "slrf.h"

namespace {

using cd = std::complex<double>;
const double PI = 3.14159265358979323846;

void order_by_real(int N, std::vector<cd> &s, std::vector<cd> &w) {
    std::vector<int> idx(N);
    for (int i = 0; i < N; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return s[a].real() < s[b].real(); });
    std::vector<cd> s2(N), w2(N);
    for (int i = 0; i < N; ++i) {
        s2[i] = s[idx[i]];
        w2[i] = w[idx[i]];
    }
    s = s2;
    w = w2;
}

// Gauss-Legendre nodes/weights on [-1, 1]: Newton's method on P_N from the
// asymptotic guesses cos(pi (i + 3/4)/(N + 1/2)); weight 2/((1 - z^2) P_N'(z)^2).
void gauss_legendre(int N, std::vector<double> &x, std::vector<double> &g) {
    x.assign(N, 0.0);
    g.assign(N, 0.0);
    for (int i = 0; i < N; ++i) {
        double z = cos(PI * (i + 0.75) / (N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p = 1.0, pm = 0.0;   // P_j(z), P_{j-1}(z)
            for (int j = 1; j <= N; ++j) {
                const double pn = ((2.0 * j - 1.0) * z * p - (j - 1.0) * pm) / j;
                pm = p;
                p = pn;
            }
            dp = N * (z * p - pm) / (z * z - 1.0);
            const double dz = p / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        g[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void quadrature(int rule, int N, double gamma, std::vector<cd> &s, std::vector<cd> &w) {
    const double c = 0.5 * gamma, r = 0.5 * gamma;
    std::vector<double> t(N), om(N);
    if (rule == SLRF_RULE_MIDPOINT) {
        for (int k = 0; k < N; ++k) {
            t[k] = (2.0 * (k + 1) - 1.0) * PI / (2.0 * N);
            om[k] = PI / N;
        }
    } else if (rule == SLRF_RULE_GAUSS_LEGENDRE) {
        std::vector<double> x, g;
        gauss_legendre(N, x, g);
        for (int k = 0; k < N; ++k) {
            t[k] = PI * (1.0 - x[k]) / 2.0;
            om[k] = 0.5 * PI * g[k];
        }
    } else {
        for (int k = 0; k < N; ++k) {
            const double sk = cos((2.0 * (k + 1) - 1.0) * PI / (2.0 * N));
            t[k] = PI * (1.0 - sk) / 2.0;
            om[k] = 0.5 * PI * (PI / N) * sqrt(std::max(0.0, 1.0 - sk * sk));
        }
    }
    s.resize(N);
    w.resize(N);
    for (int k = 0; k < N; ++k) {
        const cd e = std::polar(1.0, t[k]);
        s[k] = c + r * e;
        w[k] = -r * e * om[k] / (2.0 * PI);
    }
    order_by_real(N, s, w);
}

// ---------------------------------------------------------------- SLRF
struct Grid {
    std::vector<double> t, sw, h;   // nodes, sqrt(trapezoid weight * delta), target
};

Grid make_grid(double beta, double kappa) {
    const int m1 = 401, m2 = 1801;
    Grid g;
    for (int i = 0; i < m1; ++i) {
        double wt = 1.0 / (m1 - 1);
        if (i == 0 || i == m1 - 1) wt *= 0.5;
        g.t.push_back((double)i / (m1 - 1));
        g.sw.push_back(sqrt(beta * wt));
        g.h.push_back(1.0);
    }
    for (int i = 0; i < m2; ++i) {
        double wt = (kappa - 1.0) / (m2 - 1);
        if (i == 0 || i == m2 - 1) wt *= 0.5;
        g.t.push_back(1.0 + (kappa - 1.0) * i / (m2 - 1));
        g.sw.push_back(sqrt(wt));
        g.h.push_back(0.0);
    }
    return g;
}

// Weighted least squares min ||G c - h||_W by Householder QR; returns residual
// vector (weighted) and the coefficients.
void lsq(const Grid &g, const std::vector<double> &x, double alpha, std::vector<double> &coef,
         std::vector<double> &res) {
    const int M = (int)g.t.size(), N = (int)x.size(), K = 2 * N;
    std::vector<double> G((size_t)M * K), b(M);
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < N; ++j) {
            const cd sig(x[j], x[j] * alpha);
            const cd inv = 1.0 / (g.t[i] - sig);
            G[(size_t)i * K + j] = 2.0 * inv.real() * g.sw[i];
            G[(size_t)i * K + N + j] = -2.0 * inv.imag() * g.sw[i];
        }
        b[i] = g.h[i] * g.sw[i];
    }
    std::vector<double> Gorig = G, borig = b;
    // Householder QR, columns 0..K-1
    std::vector<double> diag(K);
    for (int k = 0; k < K; ++k) {
        double nrm = 0;
        for (int i = k; i < M; ++i) nrm += G[(size_t)i * K + k] * G[(size_t)i * K + k];
        nrm = sqrt(nrm);
        const double a = G[(size_t)k * K + k] > 0 ? -nrm : nrm;
        diag[k] = a;
        if (nrm == 0) continue;
        G[(size_t)k * K + k] -= a;
        double vnorm2 = 0;
        for (int i = k; i < M; ++i) vnorm2 += G[(size_t)i * K + k] * G[(size_t)i * K + k];
        if (vnorm2 == 0) continue;
        for (int j = k + 1; j < K; ++j) {
            double d = 0;
            for (int i = k; i < M; ++i) d += G[(size_t)i * K + k] * G[(size_t)i * K + j];
            const double f = 2 * d / vnorm2;
            for (int i = k; i < M; ++i) G[(size_t)i * K + j] -= f * G[(size_t)i * K + k];
        }
        double d = 0;
        for (int i = k; i < M; ++i) d += G[(size_t)i * K + k] * b[i];
        const double f = 2 * d / vnorm2;
        for (int i = k; i < M; ++i) b[i] -= f * G[(size_t)i * K + k];
    }
    coef.assign(K, 0.0);
    for (int k = K - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < K; ++j) s -= G[(size_t)k * K + j] * coef[j];
        coef[k] = diag[k] != 0 ? s / diag[k] : 0.0;
    }
    res.assign(M, 0.0);
    for (int i = 0; i < M; ++i) {
        double s = -borig[i];
        for (int k = 0; k < K; ++k) s += Gorig[(size_t)i * K + k] * coef[k];
        res[i] = s;
    }
}

// residual vector of the outer problem at increments a (cumulative x)
void outer_res(const Grid &g, const std::vector<double> &a, double alpha, std::vector<double> &r) {
    const int N = (int)a.size();
    std::vector<double> x(N);
    double acc = 0;
    for (int i = 0; i < N; ++i) {
        acc += a[i];
        x[i] = std::min(1.0, std::max(1e-3, acc));
    }
    std::vector<double> coef;
    lsq(g, x, alpha, coef, r);
    r.push_back(std::max(0.0, acc - 1.0) * 1e3);
}

double sumsq(const std::vector<double> &r) {
    double s = 0;
    for (double v : r) s += v * v;
    return s;
}

// small dense solve (K x K) with partial pivoting
bool solve_small(int K, std::vector<double> M, std::vector<double> &b) {
    for (int k = 0; k < K; ++k) {
        int p = k;
        for (int i = k + 1; i < K; ++i)
            if (fabs(M[i * K + k]) > fabs(M[p * K + k])) p = i;
        if (M[p * K + k] == 0) return false;
        if (p != k) {
            for (int j = 0; j < K; ++j) std::swap(M[k * K + j], M[p * K + j]);
            std::swap(b[k], b[p]);
        }
        for (int i = k + 1; i < K; ++i) {
            const double f = M[i * K + k] / M[k * K + k];
            for (int j = k; j < K; ++j) M[i * K + j] -= f * M[k * K + j];
            b[i] -= f * b[k];
        }
    }
    for (int k = K - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < K; ++j) s -= M[k * K + j] * b[j];
        b[k] = s / M[k * K + k];
    }
    return true;
}

void slrf_design(int N, double alpha, double beta, std::vector<double> &xbest) {
    const Grid g = make_grid(beta, 10.0);
    const double gap = 1.0 / (4.0 * N);
    std::vector<double> lb(N, gap), ub(N, 1.0);
    lb[0] = 1e-3;
    double fbest = INFINITY;
    for (int start = 0; start < 6; ++start) {
        std::vector<double> a(N);
        double prev = 0;
        for (int i = 0; i < N; ++i) {
            const double x0 = (i + 0.5) / N * (0.5 + 0.1 * start);
            a[i] = std::max(x0 - prev, lb[i] * 1.01);
            prev = x0;
        }
        std::vector<double> r;
        outer_res(g, a, alpha, r);
        double f = sumsq(r);
        double mu = 1e-3;
        for (int it = 0; it < 300; ++it) {
            // forward-difference Jacobian
            const int M = (int)r.size();
            std::vector<double> J((size_t)M * N);
            for (int k = 0; k < N; ++k) {
                std::vector<double> a2 = a, r2;
                const double hstep = 1e-7 * std::max(1.0, fabs(a[k]));
                a2[k] += hstep;
                outer_res(g, a2, alpha, r2);
                for (int i = 0; i < M; ++i) J[(size_t)i * N + k] = (r2[i] - r[i]) / hstep;
            }
            std::vector<double> JtJ((size_t)N * N, 0.0), Jtr(N, 0.0);
            for (int i = 0; i < M; ++i)
                for (int p = 0; p < N; ++p) {
                    Jtr[p] += J[(size_t)i * N + p] * r[i];
                    for (int q = 0; q < N; ++q) JtJ[p * N + q] += J[(size_t)i * N + p] * J[(size_t)i * N + q];
                }
            bool improved = false;
            for (int tries = 0; tries < 20; ++tries) {
                std::vector<double> Mx = JtJ, step(N);
                for (int p = 0; p < N; ++p) {
                    Mx[p * N + p] += mu * std::max(JtJ[p * N + p], 1e-12);
                    step[p] = -Jtr[p];
                }
                if (!solve_small(N, Mx, step)) {
                    mu *= 4;
                    continue;
                }
                std::vector<double> a2(N);
                for (int p = 0; p < N; ++p) a2[p] = std::min(ub[p], std::max(lb[p], a[p] + step[p]));
                std::vector<double> r2;
                outer_res(g, a2, alpha, r2);
                const double f2 = sumsq(r2);
                if (f2 < f) {
                    const double rel = (f - f2) / std::max(f, 1e-300);
                    a = a2;
                    r = r2;
                    f = f2;
                    mu = std::max(mu / 3.0, 1e-12);
                    improved = rel > 1e-15;
                    break;
                }
                mu *= 4;
            }
            if (!improved) break;
        }
        if (f < fbest) {
            fbest = f;
            xbest.assign(N, 0.0);
            double acc = 0;
            for (int i = 0; i < N; ++i) {
                acc += a[i];
                xbest[i] = std::min(1.0, std::max(1e-3, acc));
            }
        }
    }
}

}  // namespace

extern "C" slrf_status slrf_design_poles(int32_t rule, int32_t N, double alpha, double beta, double gamma,
                                         double *sigma_re, double *sigma_im, double *w_re, double *w_im) {
    if (N < 1 || N > SLRF_MAX_POLES || !(gamma > 0) || !sigma_re || !sigma_im || !w_re || !w_im)
        return SLRF_EINVAL;
    std::vector<cd> s, w;
    if (rule == SLRF_RULE_MIDPOINT || rule == SLRF_RULE_GAUSS_LEGENDRE || rule == SLRF_RULE_GAUSS_CHEBYSHEV) {
        quadrature(rule, N, gamma, s, w);
    } else if (rule == SLRF_RULE_SLRF) {
        if (!(alpha > 0) || !(beta > 0)) return SLRF_EINVAL;
        std::vector<double> x;
        slrf_design(N, alpha, beta, x);
        const Grid g = make_grid(beta, 10.0);
        std::vector<double> coef, res;
        lsq(g, x, alpha, coef, res);
        s.resize(N);
        w.resize(N);
        for (int j = 0; j < N; ++j) {
            s[j] = gamma * cd(x[j], x[j] * alpha);
            w[j] = gamma * cd(coef[j], coef[N + j]);
        }
        order_by_real(N, s, w);
    } else {
        return SLRF_EINVAL;
    }
    for (int j = 0; j < N; ++j) {
        sigma_re[j] = s[j].real();
        sigma_im[j] = s[j].imag();
        w_re[j] = w[j].real();
        w_im[j] = w[j].imag();
    }
    return SLRF_OK;
}

extern "C" slrf_status slrf_filter_eval(const slrf_filter *f, const double *x, int64_t count, double *phi) {
    if (!f || !x || !phi || count < 0 || f->n_poles < 1 || f->n_poles > SLRF_MAX_POLES) return SLRF_EINVAL;
    for (int64_t k = 0; k < count; ++k) {
        double s = 0;
        for (int j = 0; j < f->n_poles; ++j) {
            const cd w(f->w_re[j], f->w_im[j]);
            const cd sg(f->sigma_re[j], f->sigma_im[j]);
            s += 2.0 * (w / (x[k] - sg)).real();
        }
        phi[k] = s;
    }
    return SLRF_OK;
}
