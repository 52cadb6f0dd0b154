"""Brute-force reference for the single-layer inner integral (tests only).

V 1_sigma (t, x) = 1/(4 pi) * int_K 1[(t - |x - y|, y) in sigma] / |x - y| dA(y)

which is the retarded single layer potential of eq. slp after integrating the
delta over tau on the flat panel hyperplane Gamma_K x R. It is evaluated
without any of the oracle's machinery: polar coordinates (r = |x - y|, phi)
around the foot point of x in the plane of K turn dA/|x-y| into dr dphi;
membership is decided by the four barycentric coordinates of the 4D point;
along each ray the sign changes of every barycentric coordinate are found by
dense sampling plus bisection, and the pieces between them are tested at
their midpoints; the
phi-integral is adaptive Gauss-Kronrod quadrature from scipy, started on
many equal pieces of the circle.
"""
import numpy as np
from scipy import integrate


def _frame(tet):
    Y = tet[:, 1:]
    # spatial triangle: the three distinct spatial points
    pts = []
    for y in Y:
        if not any(np.array_equal(y, p) for p in pts):
            pts.append(y)
    a, b, c = pts[:3]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    e1 = (b - a) / np.linalg.norm(b - a)
    e2 = np.cross(n, e1)
    return a, n, e1, e2


def _bary_solver(tet, a, e1, e2):
    # local coordinates (tau, u, v) of the vertices, barycentric by 3x3 inverse
    L = np.stack([tet[:, 0], (tet[:, 1:] - a) @ e1, (tet[:, 1:] - a) @ e2], axis=1)
    M = (L[1:] - L[0]).T
    Minv = np.linalg.inv(M)
    return L[0], Minv


def brute_V(x, tet, rtol=1e-11, nsamp=1500, npieces=96):
    x = np.asarray(x, float)
    tet = np.asarray(tet, float)
    t = x[0]
    a, n, e1, e2 = _frame(tet)
    d = float(np.dot(x[1:] - a, n))
    xb = x[1:] - d * n
    ub = np.array([np.dot(xb - a, e1), np.dot(xb - a, e2)])
    L0, Minv = _bary_solver(tet, a, e1, e2)
    rmax = t - tet[:, 0].min()
    rmin = abs(d)
    if rmax <= rmin:
        return 0.0

    def bary(r, cphi, sphi):
        r = np.asarray(r, float)
        s = np.sqrt(np.maximum(r * r - d * d, 0.0))
        loc = np.stack([t - r, ub[0] + s * cphi, ub[1] + s * sphi], axis=-1)
        lam = (loc - L0) @ Minv.T
        return np.concatenate([lam, (1.0 - lam.sum(axis=-1))[..., None]], axis=-1)

    rs = np.linspace(rmin, rmax, nsamp)

    def measure(phi):
        cphi, sphi = np.cos(phi), np.sin(phi)
        lam = bary(rs, cphi, sphi)               # [nsamp, 4]
        pos = lam > 0
        roots = [rmin, rmax]
        for k in range(4):
            idx = np.nonzero(pos[1:, k] != pos[:-1, k])[0]
            if idx.size == 0:
                continue
            lo, hi = rs[idx].copy(), rs[idx + 1].copy()
            vlo = pos[idx, k]
            for _ in range(56):
                mid = 0.5 * (lo + hi)
                same = (bary(mid, cphi, sphi)[:, k] > 0) == vlo
                lo = np.where(same, mid, lo)
                hi = np.where(same, hi, mid)
            roots += list(0.5 * (lo + hi))
        roots = np.sort(np.array(roots))
        a, b = roots[:-1], roots[1:]
        keep = b > a
        a, b = a[keep], b[keep]
        if a.size == 0:
            return 0.0
        inside = (bary(0.5 * (a + b), cphi, sphi) > 0).all(axis=-1)
        return float(np.sum((b - a)[inside]))

    # many starting pieces: a single adaptive pass over the full circle can
    # miss narrow features and report false convergence
    grid = np.linspace(0.0, 2.0 * np.pi, npieces + 1)
    val = 0.0
    for a0, b0 in zip(grid[:-1], grid[1:]):
        v, _ = integrate.quad(measure, a0, b0, limit=200, epsabs=1e-14, epsrel=rtol)
        val += v
    return val / (4.0 * np.pi)


def laplace_triangle(x, tri):
    """(1/4pi) int_K dA/|x-y| for a flat triangle K (textbook polar form).

    Around the foot point xb of x, int_K dA/|x-y| = int dphi [sqrt(s(phi)^2+d^2)
    - |d|] with s(phi) the distance to the boundary, for xb inside K; a point
    outside is handled by the signed sum over the three sub-triangles
    (xb, P_k, P_{k+1}). Each sub-triangle is integrated in phi by adaptive
    quadrature between its two vertex directions.
    """
    x = np.asarray(x, float)
    P = np.asarray(tri, float)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = float(np.dot(x - P[0], n))
    xb = x - d * n
    total = 0.0
    for k in range(3):
        A, B = P[k] - xb, P[(k + 1) % 3] - xb
        orient = np.dot(np.cross(A, B), n)
        if abs(orient) < 1e-300:
            continue
        sgn = np.sign(orient)
        e = B - A
        # foot of the perpendicular on the edge line
        lam0 = -np.dot(A, e) / np.dot(e, e)
        F = A + lam0 * e
        p = np.linalg.norm(F)
        if p < 1e-300:
            continue
        eu = e / np.linalg.norm(e)
        wa, wb = np.dot(A, eu), np.dot(B, eu)
        # angle psi from the foot direction: w = p tan(psi)
        pa, pb = np.arctan2(wa, p), np.arctan2(wb, p)

        def f(psi):
            s = p / np.cos(psi)
            return np.sqrt(s * s + d * d) - abs(d)

        v, _ = integrate.quad(f, min(pa, pb), max(pa, pb), epsabs=1e-15, epsrel=1e-14, limit=200)
        total += sgn * v
    return total / (4.0 * np.pi)


def laplace_triangle_ball(x, tri, rho):
    """(1/4pi) int_{K cap B(x, rho)} dA/|x-y|: the Laplace single layer of a flat
    triangle K restricted to the ball of radius rho around x (textbook polar
    form as in laplace_triangle). Around the foot point xb, with d the height
    of x over the plane and s the in-plane distance,
    int dA/|x-y| over the disk part = int dphi [min(sqrt(s(phi)^2 + d^2), rho) - |d|];
    the signed sum over the sub-triangles (xb, P_k, P_{k+1}) covers K. Each
    phi-integral is split where the edge line leaves the ball (the kink of
    the min)."""
    x = np.asarray(x, float)
    P = np.asarray(tri, float)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    d = float(np.dot(x - P[0], n))
    if rho <= abs(d):
        return 0.0
    xb = x - d * n
    total = 0.0
    for k in range(3):
        A, B = P[k] - xb, P[(k + 1) % 3] - xb
        orient = np.dot(np.cross(A, B), n)
        if abs(orient) < 1e-300:
            continue
        sgn = np.sign(orient)
        e = B - A
        lam0 = -np.dot(A, e) / np.dot(e, e)
        F = A + lam0 * e
        p = np.linalg.norm(F)
        if p < 1e-300:
            continue
        eu = e / np.linalg.norm(e)
        wa, wb = np.dot(A, eu), np.dot(B, eu)
        pa, pb = np.arctan2(wa, p), np.arctan2(wb, p)
        lo, hi = min(pa, pb), max(pa, pb)

        def f(psi):
            s = p / np.cos(psi)
            return min(np.sqrt(s * s + d * d), rho) - abs(d)

        cuts = [lo, hi]
        sr2 = rho * rho - d * d
        if sr2 > p * p:
            c = np.arccos(p / np.sqrt(sr2))      # s(psi) = s_rho at psi = +-c
            cuts += [v for v in (-c, c) if lo < v < hi]
        cuts = sorted(cuts)
        v = 0.0
        for a, b in zip(cuts[:-1], cuts[1:]):
            vv, _ = integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-14, limit=200)
            v += vv
        total += sgn * v
    return total / (4.0 * np.pi)
