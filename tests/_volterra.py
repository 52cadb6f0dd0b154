"""Reference solutions of the retarded single layer on the unit sphere for
zonal data (test infrastructure).

Sec. 4.3 (experiment 3) solves V w = g on the unit sphere for
g = g0(t) Re Y_1^0(x), whose exact solution w = w0(t) Re Y_1^0(x) it takes
from a reference outside the paper. Here w0 comes from its own equation: for
w(t, x) = w0(t) P_n(x3) the single layer (eq. slp) on the unit sphere, where
the surface element at chord distance r = |x - y| is 2 pi r dr and
<x, y> = 1 - r^2/2, gives by the Funk-Hecke formula

    V w (t, x) = P_n(x3) * (1/2) int_0^{min(t,2)} w0(t - r) P_n(1 - r^2/2) dr,

so w0 solves the first-kind Volterra equation

    (1/2) int_0^{min(t,2)} w0(t - r) P_n(1 - r^2/2) dr = g0(t).        (V1)

With F(t) = int_{max(0,t-2)}^t w0(s) k(t - s) ds, k(r) = P_n(1 - r^2/2) / 2,
differentiating (V1) gives the second-kind equation

    w0(t) k(0) - 1[t > 2] w0(t - 2) k(2) + int_{max(0,t-2)}^t w0(s) k'(t - s) ds = g0'(t),

with k(0) = 1/2, k(2) = (-1)^n / 2 and k'(r) = -r P_n'(1 - r^2/2) / 2, which
vanishes at r = 0: the trapezoidal rule on a grid of step h = 2 / M is then
explicit (O(h^2)). For n = 0 and g0 = sin^2(pi t / 2) 1[t < 2] it reproduces
w0 = pi sin(pi t), the closed form of the sphere.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(n, x):
    """P_n(x)."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return npleg.legval(x, c)


def dlegendre(n, x):
    """P_n'(x)."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return npleg.legval(x, npleg.legder(c))


def solve_zonal(n, dg0, T, M=2000):
    """w0 on the grid t_i = i h, h = 2 / M, 0 <= t_i <= T, from the derivative
    dg0 of the data (vectorised callable; g0(0) = 0 assumed)."""
    h = 2.0 / M
    N = int(round(T / h))
    t = np.arange(N + 1) * h
    w = np.zeros(N + 1)
    r = np.arange(M + 1) * h                      # kernel lags 0 .. 2
    kp = -0.5 * r * dlegendre(n, 1.0 - 0.5 * r * r)
    k2 = 0.5 * (-1.0) ** n
    g1 = dg0(t)
    for i in range(N + 1):
        j0 = max(0, i - M)
        # trapezoid over s = t_j, j0 .. i (the j = i term has k'(0) = 0)
        lags = i - np.arange(j0, i + 1)
        vals = w[j0:i + 1] * kp[lags]
        integral = h * (vals.sum() - 0.5 * (vals[0] + vals[-1])) if i > j0 else 0.0
        tail = k2 * w[i - M] if i > M else 0.0
        w[i] = 2.0 * (g1[i] + tail - integral)
    return t, w


def apply_zonal(n, t_grid, w_grid, t, nodes=64):
    """(1/2) int_0^{min(t,2)} w0(t - r) P_n(1 - r^2/2) dr for each t, with a
    Gauss-Legendre rule in r on [0, min(t, 2)] and w0 interpolated linearly
    from the grid: the left side of (V1), evaluated independently of the
    solver's rule."""
    x, wq = npleg.leggauss(nodes)
    out = np.zeros(len(t))
    for k, tk in enumerate(t):
        b = min(tk, 2.0)
        if b <= 0:
            continue
        r = 0.5 * b * (x + 1.0)
        out[k] = 0.5 * 0.5 * b * np.sum(wq * np.interp(tk - r, t_grid, w_grid) * legendre(n, 1.0 - 0.5 * r * r))
    return out
