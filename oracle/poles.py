"""Pole/weight sets and the scalar rational filter (oracle; test infrastructure).

Conventions (Section 3, Eq. for the rational function filter and the
conjugate-pair reduction that follows it): a filter is given by N poles
sigma_j in the upper half plane and weights w_j; the lower-half poles are the
conjugates, so on the real axis

    Phi(x) = sum_j w_j/(x - sigma_j) + conj(w_j)/(x - conj(sigma_j))
           = sum_j 2 Re(w_j / (x - sigma_j)).

The 1/(2 pi i) factor of the contour form is absorbed into w_j.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize as so


def phi(x, sigma, w):
    """Phi at real or complex points x (Section 3, Eq. of Phi(lambda))."""
    x = np.asarray(x, dtype=complex)
    sigma = np.asarray(sigma, dtype=complex)
    w = np.asarray(w, dtype=complex)
    terms = w[None, :] / (x.reshape(-1, 1) - sigma[None, :]) \
        + np.conj(w)[None, :] / (x.reshape(-1, 1) - np.conj(sigma)[None, :])
    out = terms.sum(axis=1).reshape(np.shape(x))
    return out


def phi_real(x, sigma, w):
    """Phi on the real axis, where it is real by conjugate symmetry."""
    return np.real(phi(np.asarray(x, dtype=float), sigma, w))


def dphi(x, sigma, w):
    """Derivative Phi'(x) of the filter."""
    x = np.asarray(x, dtype=complex)
    sigma = np.asarray(sigma, dtype=complex)
    w = np.asarray(w, dtype=complex)
    terms = -w[None, :] / (x.reshape(-1, 1) - sigma[None, :]) ** 2 \
        - np.conj(w)[None, :] / (x.reshape(-1, 1) - np.conj(sigma)[None, :]) ** 2
    return terms.sum(axis=1).reshape(np.shape(x))


def separation_factor(sigma, w, gamma):
    """|Phi'(gamma)| (Definition 3.1)."""
    return float(abs(dphi(np.array([gamma]), sigma, w)[0]))


# ---------------------------------------------------------------------------
# Quadrature rules on the circle through 0 and gamma (Section 3.2)
# ---------------------------------------------------------------------------
def quadrature_poles(rule: str, N: int, gamma: float):
    """Upper-half poles and weights of a quadrature rule on a circle.

    The contour is the circle with centre c = gamma/2 and radius r = gamma/2.
    With z(theta) = c + r e^{i theta}, the spectral projector's contour
    integral (1/2 pi i) \\oint dz/(z - x) becomes (1/2 pi) \\int r e^{i theta}
    /(z(theta) - x) d theta; a rule with angles theta_k in (0, pi) and angle
    weights omega_k then gives, in the convention Phi(x) = sum w/(x - sigma),

        sigma_k = c + r e^{i theta_k},  w_k = -r e^{i theta_k} omega_k / (2 pi).

    rule:
      * "midpoint": theta_k = (2k-1) pi/(2N), omega_k = pi/N.
      * "gauss_legendre": Gauss-Legendre nodes t_k on [-1, 1] mapped to
        theta_k = pi (1 - t_k)/2, omega_k = (pi/2) g_k.
      * "gauss_chebyshev": first-kind Chebyshev nodes t_k = cos((2k-1) pi/(2N)),
        theta_k = pi (1 - t_k)/2, omega_k = (pi/2)(pi/N) sqrt(1 - t_k^2).
        (The paper names the rule but gives no formula; this is the reading
        used throughout.)
    Poles are returned ordered by increasing real part.
    """
    c = r = 0.5 * gamma
    k = np.arange(1, N + 1)
    if rule == "midpoint":
        theta = (2 * k - 1) * np.pi / (2 * N)
        omega = np.full(N, np.pi / N)
    elif rule == "gauss_legendre":
        t, g = np.polynomial.legendre.leggauss(N)
        theta = np.pi * (1 - t) / 2
        omega = (np.pi / 2) * g
    elif rule == "gauss_chebyshev":
        t = np.cos((2 * k - 1) * np.pi / (2 * N))
        theta = np.pi * (1 - t) / 2
        omega = (np.pi / 2) * (np.pi / N) * np.sqrt(1 - t ** 2)
    else:
        raise ValueError(rule)
    e = np.exp(1j * theta)
    sigma = c + r * e
    w = -r * e * omega / (2 * np.pi)
    order = np.argsort(sigma.real)
    return sigma[order], w[order]


# ---------------------------------------------------------------------------
# Shifted Laplace rational filter design (Section 3.1)
# ---------------------------------------------------------------------------
def slrf_grid(beta: float, kappa: float = 10.0, m_in: int = 401, m_out: int = 1801):
    """Trapezoidal nodes/weights for the delta-inner product at gamma = 1.

    delta(t) = beta on [0, 1], 1 on (1, kappa], 0 elsewhere, so
    ||Phi - h||_delta^2 = beta int_0^1 (Phi-1)^2 + int_1^kappa Phi^2 (Phi is
    real on the real axis).  Each piece uses its own composite trapezoidal rule
    so that the jump of delta and of h at t = 1 falls on a grid point.
    """
    t1 = np.linspace(0.0, 1.0, m_in)
    w1 = np.full(m_in, 1.0 / (m_in - 1))
    w1[[0, -1]] *= 0.5
    t2 = np.linspace(1.0, kappa, m_out)
    w2 = np.full(m_out, (kappa - 1.0) / (m_out - 1))
    w2[[0, -1]] *= 0.5
    t = np.concatenate([t1, t2])
    wt = np.concatenate([beta * w1, w2])
    h = np.concatenate([np.ones(m_in), np.zeros(m_out)])
    return t, wt, h


def slrf_weights(x, alpha, t, wt, h):
    """Optimal weights for fixed pole abscissae x_j (linear least squares).

    Phi(t) = sum_j 2 [Re w_j Re(1/(t - s_j)) - Im w_j Im(1/(t - s_j))],
    s_j = x_j (1 + i alpha), is linear in (Re w, Im w); minimise
    sum_m wt_m (Phi(t_m) - h_m)^2.  Returns (sigma, w, weighted residual).
    """
    x = np.asarray(x, dtype=float)
    s = x * (1 + 1j * alpha)
    g = 1.0 / (t[:, None] - s[None, :])
    G = np.concatenate([2 * g.real, -2 * g.imag], axis=1)
    sw = np.sqrt(wt)
    coef, *_ = np.linalg.lstsq(G * sw[:, None], h * sw, rcond=None)
    res = (G @ coef - h) * sw
    N = x.size
    return s, coef[:N] + 1j * coef[N:], res


def slrf_poles(N: int, alpha: float, beta: float, gamma: float = 1.0, kappa: float = 10.0,
               min_gap: float | None = None):
    """SLRF poles sigma_j = gamma x_j (1 + i alpha) and weights (Section 3.1).

    Minimises ||Phi - h||_delta^2 over x_j in (0, 1] and w_j at gamma = 1 by
    variable projection (weights eliminated by linear least squares), then
    scales: Phi_gamma(x) = Phi_1(x/gamma) gives sigma -> gamma sigma,
    w -> gamma w.  Readings where the paper is silent: the abscissae are kept
    ordered with a minimum gap ``min_gap`` (default 1/(4N)) so that poles stay
    distinct, and the best of six deterministic starts is taken.
    """
    t, wt, h = slrf_grid(beta, kappa)
    gap = 1.0 / (4 * N) if min_gap is None else min_gap

    def resid(a):
        x = np.cumsum(a)
        pen = max(0.0, x[-1] - 1.0) * 1e3
        return np.concatenate([slrf_weights(np.clip(x, 1e-3, 1.0), alpha, t, wt, h)[2], [pen]])

    best = None
    lb = np.full(N, gap)
    lb[0] = 1e-3
    for k in range(6):
        x0 = (np.arange(1, N + 1) - 0.5) / N * (0.5 + 0.1 * k)
        a0 = np.diff(np.concatenate([[0.0], x0]))
        a0 = np.maximum(a0, lb * 1.01)
        sol = so.least_squares(resid, a0, bounds=(lb, 1.0), xtol=1e-15, ftol=1e-15,
                               gtol=1e-15, max_nfev=2000)
        if best is None or sol.cost < best.cost:
            best = sol
    x = np.clip(np.cumsum(best.x), 1e-3, 1.0)
    s, w, _ = slrf_weights(x, alpha, t, wt, h)
    return gamma * s, gamma * w
