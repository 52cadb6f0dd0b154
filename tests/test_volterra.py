"""Pins of the zonal reference solutions of the unit sphere (tests/_volterra.py),
the reference of the spherical-harmonic convergence study (Sec. 4.3,
experiment 3)."""
import math

import numpy as np
import pytest

from _volterra import apply_zonal, legendre, solve_zonal


def g0(t):
    """Data of experiment 3: t^4 exp(-2t) for t > 0."""
    t = np.asarray(t, dtype=float)
    return np.where(t > 0, t ** 4 * np.exp(-2 * t), 0.0)


def dg0(t):
    t = np.asarray(t, dtype=float)
    return np.where(t > 0, (4 * t ** 3 - 2 * t ** 4) * np.exp(-2 * t), 0.0)


def test_uniform_data_gives_the_sphere_closed_form():
    """n = 0, g = sin^2(pi t/2) 1[t < 2]: w0 = pi sin(pi t) for all t (for
    t > 2 the equation reads w0(t) = w0(t - 2)). With k' = 0 the recursion
    w0(t) = 2 g0'(t) + w0(t - 2) has no quadrature error: exact to rounding."""
    dg = lambda t: np.where(t < 2, 0.5 * math.pi * np.sin(math.pi * t), 0.0)
    for M, tol in [(500, 1e-12), (2000, 1e-12)]:
        t, w = solve_zonal(0, dg, 6.0, M=M)
        err = np.abs(w - math.pi * np.sin(math.pi * t)).max()
        assert err <= tol, (M, err)


def test_zonal_solution_satisfies_the_first_kind_equation():
    """n = 1, 2: the solver's w0 put back into (V1) with an independent rule
    (Gauss-Legendre in r, linear interpolation of w0) gives g0."""
    ts = np.linspace(0.05, 7.9, 40)
    for n in (1, 2):
        t, w = solve_zonal(n, dg0, 8.0, M=4000)
        lhs = apply_zonal(n, t, w, ts, nodes=200)
        err = np.abs(lhs - g0(ts)).max() / g0(ts).max()
        assert err <= 2e-5, (n, err)


@pytest.mark.parametrize("n", [1, 2])
def test_funk_hecke_reduction_by_surface_quadrature(n):
    """V(w0 P_n(x3))(t, x) computed as a surface integral over the unit sphere
    (polar coordinates about x: |x - y| = 2 sin(theta/2), dA = sin(theta)
    dtheta dphi, so the 1/r of the kernel cancels) equals P_n(x3) times the
    left side of (V1): the reduction behind the reference, checked by brute
    force at a few (t, x)."""
    t_grid, w = solve_zonal(n, dg0, 6.0, M=4000)
    th, wt = np.polynomial.legendre.leggauss(400)
    th = 0.5 * math.pi * (th + 1.0)
    wt = 0.5 * math.pi * wt
    ph = np.linspace(0.0, 2 * math.pi, 96, endpoint=False)
    for alpha, t in [(0.3, 1.2), (1.1, 2.7), (2.4, 4.5), (math.pi / 2, 3.3)]:
        x = np.array([math.sin(alpha), 0.0, math.cos(alpha)])
        u = np.array([math.cos(alpha), 0.0, -math.sin(alpha)])
        v = np.array([0.0, 1.0, 0.0])
        T, P = np.meshgrid(th, ph, indexing="ij")
        y3 = x[2] * np.cos(T) + np.sin(T) * (np.cos(P) * u[2] + np.sin(P) * v[2])
        r = 2.0 * np.sin(0.5 * T)
        wv = np.interp(t - r, t_grid, w, left=0.0)
        integrand = wv * legendre(n, y3) * np.cos(0.5 * T) / (4 * math.pi)
        surf = np.sum(wt[:, None] * integrand) * (2 * math.pi / len(ph))
        red = legendre(n, x[2]) * apply_zonal(n, t_grid, w, [t], nodes=400)[0]
        assert abs(surf - red) <= 1e-6 * max(1.0, abs(red)), (alpha, t, surf, red)
