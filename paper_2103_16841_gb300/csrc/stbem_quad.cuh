// Device math of the light-cone-clipped single-layer quadrature.
//
// For an apex x = (t, x_s) and a flat spatial triangle K, the retarded single
// layer potential (eq. slp) of a panel sigma that lies between the graphs
// tau = P_lo(y) and tau = P_hi(y) over K is, after the delta is integrated
// over tau on the panel hyperplane Gamma_K x R,
//
//     V 1_sigma (x) = W_{P_lo}(x) - W_{P_hi}(x),
//     W_P(x) = 1/(4 pi) int_K 1[P(y) + |x_s - y| < t] / |x_s - y| dA(y).
//
// W_P is the potential of the half-infinite column above the face tau = P(y);
// its lit set R = K cap E, E = {y : P(y) + |x_s - y| < t}, is convex. In polar
// coordinates (r = |x_s - y|, phi) around the foot point xb of x_s,
// dA / r = dr dphi (the regularisation that the Lemma kernel_para expresses
// as k_{psi,1} J = r0 on the chart l_2), so by Green's theorem, with the
// winding number oint dphi = 2 pi 1[xb in R] folded in,
//
//     4 pi W_P = oint_{dR} (r - |d|) dphi,
//
// d the signed height of x_s over the plane of K. The boundary of R consists
// of pieces of the triangle edges (closed form below) and arcs of the conic
// dE (the light cone cut by the face plane). The conic arcs are integrated on
// the circle of cone directions n(theta) that hit the face plane,
// <n, c n_K + d grad P> = d, where the integrand (r - |d|) dphi/dtheta is a
// rational trigonometric function; the Gauss-Legendre order follows from its
// nearest pole, and near poles get a sinh map (Johnston & Elliott 2005).
// For d = 0 the conic has its focus at xb and the arc integral is closed form.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#ifndef STBEM_PI
#define STBEM_PI 3.14159265358979323846
#endif

namespace stbem {

constexpr int MAX_NTHETA = 32;

// Gauss-Legendre nodes/weights on [-1,1] for n = 1..MAX_NTHETA, packed:
// rule n starts at offset n*(n-1)/2 (filled by upload_gauss_tables in the
// translation unit that launches the quadrature kernels).
static __constant__ double c_gl_x[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
static __constant__ double c_gl_w[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
// host copies (the same functions also compile for the host, for checks)
static double h_gl_x[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
static double h_gl_w[MAX_NTHETA * (MAX_NTHETA + 1) / 2];

#define STBEM_HD __host__ __device__

STBEM_HD inline const double* gl_x() {
#ifdef __CUDA_ARCH__
  return c_gl_x;
#else
  return h_gl_x;
#endif
}
STBEM_HD inline const double* gl_w() {
#ifdef __CUDA_ARCH__
  return c_gl_w;
#else
  return h_gl_w;
#endif
}

// the same tables rounded to FP32 for the FP32 rules (no conversion per node)
static __constant__ float c_gl_xf[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
static __constant__ float c_gl_wf[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
static float h_gl_xf[MAX_NTHETA * (MAX_NTHETA + 1) / 2];
static float h_gl_wf[MAX_NTHETA * (MAX_NTHETA + 1) / 2];

// nodes / weights of rule n in precision R
template <typename R>
STBEM_HD inline const R* gl_nodes(int n);
template <typename R>
STBEM_HD inline const R* gl_weights(int n);
template <>
STBEM_HD inline const double* gl_nodes<double>(int n) { return gl_x() + n * (n - 1) / 2; }
template <>
STBEM_HD inline const double* gl_weights<double>(int n) { return gl_w() + n * (n - 1) / 2; }
template <>
STBEM_HD inline const float* gl_nodes<float>(int n) {
#ifdef __CUDA_ARCH__
  return c_gl_xf + n * (n - 1) / 2;
#else
  return h_gl_xf + n * (n - 1) / 2;
#endif
}
template <>
STBEM_HD inline const float* gl_weights<float>(int n) {
#ifdef __CUDA_ARCH__
  return c_gl_wf + n * (n - 1) / 2;
#else
  return h_gl_wf + n * (n - 1) / 2;
#endif
}

struct ColGeom {         // per spatial triangle ("column"), column frame
  double X[3][3];        // corners (input coordinates), ascending spatial-vertex id
  double c0[3];          // corner 0
  double e1[3], e2[3], n[3];
  double Q[3][2];        // corners in the frame (Q[0] = 0); counter-clockwise
  double U[3][2];        // unit edge directions, edge k: Q[k] -> Q[k+1]
  double L[3];           // edge lengths
  double area, diam;
  double ctr[3], rad;    // centroid ball (pruning only)
};

struct FaceGeom {
  double p[3];   // face times at the three corners
  double g[2];   // gradient of P in the column frame
};

template <typename R>
struct PtR {             // apex-against-column quantities in precision R (column frame)
  R d;                   // signed height over the plane of K (0 if |d| < 1e-13 diam)
  R xb[2];               // foot point
  R q[3][2];             // corners relative to xb
  R ps[3];               // signed distance of xb to edge line k (> 0 inside)
  R ws[3];               // coordinate of Q[k] along edge k, origin at the foot of xb
  R rs[3];               // |x_s - corner_k| in precision R
  R Efull[3];            // int (r - |d|) dphi along the whole edge k (far field: int (r - C) dphi)
  // far field of the mixed path (see edge_far): the contour integrand is
  // r - C with C = |x_s - corner 0|; far_rho: lower bound of the in-plane
  // distance from xb to K
  int far;
  R C, far_rho;
};

struct PointCol {        // apex x against one column
  double t;
  double r[3];           // |x_s - corner_k| (FP64: the cone-function values need it)
  double rlo;            // lower bound of dist(x_s, K)
  double Wst;            // 4 pi * potential of the whole triangle
  float Wst_f;
  int inK;
  PtR<double> D;
  PtR<float> F;          // filled for the mixed-precision path
  float rho_hi[3], rho_lo[3];   // r_k - t as an FP32 pair (mixed path)
  float nt_hi, nt_lo;           // -t as an FP32 pair
  float rlot_hi, rlot_lo;       // rlo - t as an FP32 pair
};

// per face, FP32 view for the mixed path: corner times as FP32 pairs
struct FaceF {
  float p_hi[3], p_lo[3];
  float g[2];
  float pmin_hi, pmin_lo;
};

STBEM_HD inline void split2(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// a + b for FP32 pairs (TwoSum on the high parts), rounded to one float
STBEM_HD inline float add2(float ahi, float alo, float bhi, float blo) {
  float s = ahi + bhi;
  float bb = s - ahi;
  float e = (ahi - (s - bb)) + (bhi - bb);
  return s + (e + (alo + blo));
}

STBEM_HD inline void make_facef(const FaceGeom& F, FaceF& o) {
  int km = 0;
  for (int k = 0; k < 3; ++k) {
    split2(F.p[k], o.p_hi[k], o.p_lo[k]);
    if (F.p[k] < F.p[km]) km = k;
  }
  o.pmin_hi = o.p_hi[km]; o.pmin_lo = o.p_lo[km];
  o.g[0] = (float)F.g[0]; o.g[1] = (float)F.g[1];
}

template <typename R>
struct ColR {            // edge data of a column in precision R
  R Q[3][2], U[3][2], L[3], diam;
};

STBEM_HD inline void sc(float x, float* s, float* c) { sincosf(x, s, c); }
STBEM_HD inline void sc(double x, double* s, double* c) { sincos(x, s, c); }

template <typename R>
STBEM_HD inline const PtR<R>& pt(const PointCol& P);
template <>
STBEM_HD inline const PtR<double>& pt<double>(const PointCol& P) { return P.D; }
template <>
STBEM_HD inline const PtR<float>& pt<float>(const PointCol& P) { return P.F; }

struct ArcRule {
  int nmin, nmax;    // Gauss node bounds per piece
  double tol;        // target relative accuracy of a piece
  float ltol_f;      // log(1 / tol), kept so that no rule choice divides or
  double ltol_d;     // takes a logarithm in FP64 at run time
  int fp32_short;    // FP32 shortcut of arc_piece allowed (nmin >= 4, tol >= 1 / 1.6e7)
};

STBEM_HD inline void rule_finish(ArcRule& r) {
  r.ltol_d = log(1.0 / r.tol);
  r.ltol_f = (float)r.ltol_d;
  r.fp32_short = r.nmin >= 4 && r.tol >= 1.0 / 1.6e7;
}

// log(1 / tol) of a rule in precision R
template <typename R>
STBEM_HD inline R rule_ltol(const ArcRule& r);
template <>
STBEM_HD inline float rule_ltol<float>(const ArcRule& r) { return r.ltol_f; }
template <>
STBEM_HD inline double rule_ltol<double>(const ArcRule& r) { return r.ltol_d; }

// n_max = 0 selects the default cap (32 nodes FP64, 16 nodes MIXED).
// (log(1e7) and log(1e15) written out: this is called per point and column)
STBEM_HD inline ArcRule make_rule(int precision_mixed, int n_max) {
  ArcRule r;
  if (precision_mixed) {
    r.nmin = 4; r.nmax = n_max ? n_max : 16; r.tol = 1e-7; r.ltol_d = 16.11809565095832;
  } else {
    r.nmin = 6; r.nmax = n_max ? n_max : 32; r.tol = 1e-15; r.ltol_d = 34.538776394910684;
  }
  if (r.nmin > r.nmax) r.nmin = r.nmax;
  r.ltol_f = (float)r.ltol_d;
  r.fp32_short = r.nmin >= 4 && precision_mixed;
  return r;
}

// ---------------------------------------------------------------------------
// Green's theorem with the winding number removed: since oint dphi equals
// 2 pi 1[xb in R],  4 pi W = oint_{dR} (r - |d|) dphi.
// Along the line of edge k (signed distance p_s of xb, edge coordinate w
// with the foot of the perpendicular at 0, r = sqrt(A^2 + w^2),
// A^2 = p_s^2 + d^2):  (r - |d|) dphi = (r - |d|) p_s / (p^2 + w^2) dw, with
// antiderivative
//   E(w) = p_s asinh(w / A) - sgn(p_s) |d| atan(w p (p^2 + w^2) / ((r + |d|)(p^2 r + w^2 |d|)))
// (the atan is the difference of atan(w |d| / (p r)) and the plain angle
// atan(w / p)). Differences E(w_b) - E(w_a) are formed without cancellation:
// asinh(w_b/A) - asinh(w_a/A) = asinh((w_b r_a - w_a r_b) / A^2) and
// w_b r_a - w_a r_b = A^2 (w_b - w_a)(w_b + w_a) / (w_b r_a + w_a r_b) when
// w_a w_b >= 0.
// ---------------------------------------------------------------------------
template <typename R>
STBEM_HD inline R edge_T(R w, R r, R p, R ad) {
  return atan(w * p * (p * p + w * w) / ((r + ad) * (p * p * r + w * w * ad)));
}

template <typename R>
STBEM_HD inline R edge_dE(R wa, R dw, R p_s, R d) {
  R p = fabs(p_s), ad = fabs(d);
  R A2 = p_s * p_s + d * d;
  if (A2 == R(0) || dw == R(0)) return R(0);
  R wb = wa + dw;
  R ra = sqrt(A2 + wa * wa), rb = sqrt(A2 + wb * wb);
  R dasinh;
  if (wa * wb >= R(0)) dasinh = asinh(dw * (wb + wa) / (wb * ra + wa * rb));
  else dasinh = asinh((wb * ra - wa * rb) / A2);
  R val = p_s * dasinh;
  if (p > R(0) && ad > R(0)) {
    R dt = edge_T<R>(wb, rb, p, ad) - edge_T<R>(wa, ra, p, ad);
    val -= (p_s > R(0) ? ad : -ad) * dt;
  }
  return val;
}

// The same edge integral on [wa, wa + dw] by Gauss-Legendre, for edges that
// are short against their distance from the apex. Since r^2 - d^2 = p^2 + w^2,
// the integrand (r - |d|) p_s / (p^2 + w^2) equals p_s / (r + |d|): positive,
// free of cancellation, and analytic up to the branch points w = +-iA. In
// FP32 the closed form above loses the relative accuracy of such an edge:
// its asinh and atan terms are O(1) with a difference of O(dw / A). Returns
// false when the branch points are close (Bernstein parameter below 4, or
// more than six nodes needed): there the edge is not far from the apex, the
// closed form keeps its accuracy, and the caller takes it.
template <typename R>
STBEM_HD inline bool edge_gauss(R wa, R dw, R p_s, R d, const ArcRule& rule, R& out) {
  R A2 = p_s * p_s + d * d;
  if (A2 == R(0) || dw == R(0) || p_s == R(0)) { out = R(0); return true; }
  R hl = R(0.5) * dw, m = wa + hl;
  R a = -m / hl, b = sqrt(A2) / fabs(hl);
  R s = R(0.5) * (sqrt((a - R(1)) * (a - R(1)) + b * b) + sqrt((a + R(1)) * (a + R(1)) + b * b));
  R rho = s + sqrt(fmax(s * s - R(1), R(0)));
  if (!(rho >= R(4))) return false;
  int n = (int)ceil(rule_ltol<R>(rule) / (R(2) * log(rho))) + 1;
  if (n > 6) return false;   // the closed form costs about as much as six nodes
  n = n < 2 ? 2 : n;
  const R* X = gl_nodes<R>(n);
  const R* Wt = gl_weights<R>(n);
  R ad = fabs(d), acc = R(0);
  for (int k = 0; k < n; ++k) {
    R w = m + hl * (R)X[k];
    acc += (R)Wt[k] / (sqrt(A2 + w * w) + ad);
  }
  out = acc * p_s * hl;
  return true;
}

// int (r - |d|) dphi along edge coordinates [wa, wa + dw]: the closed form in
// FP64; in FP32 the Gauss form wherever it applies
template <typename R>
STBEM_HD inline R edge_int(R wa, R dw, R p_s, R d, const ArcRule& rule) {
  if (sizeof(R) == 4) {
    R v;
    if (edge_gauss<R>(wa, dw, p_s, d, rule, v)) return v;
  }
  return edge_dE<R>(wa, dw, p_s, d);
}

// ---------------------------------------------------------------------------
// Far field of the mixed path. When the foot point xb lies far outside K
// (in-plane distance rho_K >= FAR_RHO diam K), every piece of
// oint (r - |d|) dphi is O(diam K) while their sum, 4 pi W, is
// O(diam K^2 / dist): the FP32 terms would keep only eps rho_K / diam K of
// relative accuracy. Since xb then lies outside the lit set R, oint C dphi = 0
// around dR for any constant C, so
//     4 pi W = oint_{dR} (r - C) dphi,   C = |x_s - corner 0|,
// and with u the point in column coordinates (origin at corner 0) and
// q0 = corner 0 - xb,
//     r - C = (|q|^2 - |q0|^2) / (r + C) = <u, 2 q0 + u> / (r + C),
// formed from O(diam K) coordinates, so every piece is O(diam K^2 / dist)
// with relative accuracy eps. Edge pieces are integrated in the edge
// parameter, conic arcs over their chord (arc_far); both rules are
// Gauss-Legendre with the order taken from the nearest complex zero of |q|^2.
// ---------------------------------------------------------------------------
constexpr float FAR_RHO = 1.5f;

// Gauss-Legendre order reaching relative accuracy tol on [-1, 1] for an
// integrand analytic except at z = a +- i b (Bernstein ellipse parameter)
template <typename R>
STBEM_HD inline int gauss_order(R a, R b, R ltol, int nmin, int nmax) {
  const R s = R(0.5) * (sqrt((a - R(1)) * (a - R(1)) + b * b) + sqrt((a + R(1)) * (a + R(1)) + b * b));
  const R rho = s + sqrt(fmax(s * s - R(1), R(0)));
  if (!(rho > R(1.0001))) return nmax;
  const int n = (int)ceil(ltol / (R(2) * log(rho))) + 1;
  return n < nmin ? nmin : (n > nmax ? nmax : n);
}

// int (r - C) dphi along edge k for u = Q_k + lambda L_k U_k, lambda in
// [la, lb]: dphi = p_s L_k dlambda / |q|^2 (p_s the signed distance of xb to
// the edge line, constant along it)
template <typename R>
STBEM_HD inline R edge_far(const PtR<R>& P, const ColR<R>& G, int k, R la, R lb, const ArcRule& rule) {
  const R h = R(0.5) * (lb - la);
  if (!(h > R(0))) return R(0);
  const R mid = R(0.5) * (la + lb), L = G.L[k];
  const R q0x = -P.xb[0], q0y = -P.xb[1];
  // |q|^2 = 0 at lambda = lambda_foot +- i |p_s| / L
  const int n = gauss_order<R>((-P.ws[k] / L - mid) / h, fabs(P.ps[k]) / (L * h), rule_ltol<R>(rule), 3, 10);
  const R* X = gl_nodes<R>(n);
  const R* Wt = gl_weights<R>(n);
  const R ex = G.U[k][0] * L, ey = G.U[k][1] * L, d2 = P.d * P.d;
  R acc = R(0);
  for (int i = 0; i < n; ++i) {
    const R lam = mid + h * (R)X[i];
    const R ux = G.Q[k][0] + lam * ex, uy = G.Q[k][1] + lam * ey;
    const R qx = q0x + ux, qy = q0y + uy, q2 = qx * qx + qy * qy;
    const R r = sqrt(q2 + d2);
    const R del = (ux * (R(2) * q0x + ux) + uy * (R(2) * q0y + uy)) / (r + P.C);
    acc += (R)Wt[i] * del / q2;
  }
  return acc * P.ps[k] * L * h;
}

// int (r - C) dphi along the conic dE from event uA to event uB (column
// coordinates), E on the left. With u = y - uA the conic is
//     2 <m, u> + Q(u) = 0,   m = q_A + r_A g,   Q(u) = |u|^2 - <g, u>^2,
// (square of |x - y| = r_A - <g, u>, which holds on the cone since
// tau = P(y) is linear). Over the chord, u = s D + h(s) nu (D = uB - uA, nu
// its left unit normal): a h^2 + b(s) h + c(s) = 0 with a = Q(nu),
// b = 2 <m, nu> + 2 s B(D, nu), c = s (s - 1) Q(D) (B on the conic), h the
// small root (h(0) = h(1) = 0). On the arc r - C = (r_A - C) - <g, u>. Applies
// to arcs that are nearly straight with E on the left (b < 0 on [0, 1],
// sagitta <= |D| / 16); returns false otherwise (the caller takes conic_arc).
template <typename R>
STBEM_HD inline bool arc_far(const R* xb, R d, R C, R far_rho, const R* g, const R* uA, const R* D, const ArcRule& rule,
                             R& out) {
  const R Dx = D[0], Dy = D[1];
  const R l2 = Dx * Dx + Dy * Dy;
  if (!(l2 > R(0))) { out = R(0); return true; }
  const R l = sqrt(l2), nx = -Dy / l, ny = Dx / l;
  const R q0x = -xb[0], q0y = -xb[1];
  const R qAx = q0x + uA[0], qAy = q0y + uA[1];
  const R rA = sqrt(qAx * qAx + qAy * qAy + d * d);
  const R mx = qAx + rA * g[0], my = qAy + rA * g[1];
  // m cancels where the conic bends sharply at A (|grad P| near 1, or the cone
  // just reaching the plane); its FP32 rounding then sets the arc's shape
  if (!(mx * mx + my * my >= R(0.0025) * (qAx * qAx + qAy * qAy))) return false;
  const R gD = g[0] * Dx + g[1] * Dy, gn = g[0] * nx + g[1] * ny;
  const R QD = l2 - gD * gD, a = R(1) - gn * gn, BDn = -gD * gn;
  const R b0 = R(2) * (mx * nx + my * ny), b1 = b0 + R(2) * BDn;
  if (!(b0 < R(0) && b1 < R(0))) return false;
  {
    const R bh = R(0.5) * (b0 + b1), ch = R(-0.25) * QD;
    const R disc = bh * bh - R(4) * a * ch;
    if (!(disc > R(0))) return false;
    const R hh = R(-2) * ch / (bh - sqrt(disc));
    if (!(fabs(hh) <= R(0.0625) * l)) return false;
  }
  const R delA = (uA[0] * (R(2) * q0x + uA[0]) + uA[1] * (R(2) * q0y + uA[1])) / (rA + C);
  // |q|^2 has no zero within far_rho of the chord (it lies in K)
  const int n = gauss_order<R>(R(0), R(2) * far_rho / l, rule_ltol<R>(rule), 4, 10);
  const R* X = gl_nodes<R>(n);
  const R* Wt = gl_weights<R>(n);
  R acc = R(0);
  for (int i = 0; i < n; ++i) {
    const R sv = R(0.5) * (R(1) + (R)X[i]);
    const R c = sv * (sv - R(1)) * QD, b = b0 + R(2) * sv * BDn;
    const R disc = fmax(b * b - R(4) * a * c, R(0));
    const R h = R(-2) * c / (b - sqrt(disc));
    const R dh = -((R(2) * sv - R(1)) * QD + R(2) * BDn * h) / (R(2) * a * h + b);
    const R wx = sv * Dx + h * nx, wy = sv * Dy + h * ny;   // u - uA
    const R tx = Dx + dh * nx, ty = Dy + dh * ny;
    const R qx = qAx + wx, qy = qAy + wy, q2 = qx * qx + qy * qy;
    const R del = delA - (g[0] * wx + g[1] * wy);
    acc += (R)Wt[i] * del * (qx * ty - qy * tx) / q2;
  }
  out = R(0.5) * acc;
  return true;
}

template <typename R>
STBEM_HD inline void make_colr(const ColGeom& G, ColR<R>& C) {
  for (int k = 0; k < 3; ++k) {
    C.Q[k][0] = (R)G.Q[k][0]; C.Q[k][1] = (R)G.Q[k][1];
    C.U[k][0] = (R)G.U[k][0]; C.U[k][1] = (R)G.U[k][1]; C.L[k] = (R)G.L[k];
  }
  C.diam = (R)G.diam;
}

// whole-edge integral k of the mixed path (the fully lit triangle is the sum
// over the three edges): the far-field form when P.far, else edge_int
STBEM_HD inline float edge_full_mixed(const PointCol& P, const ColR<float>& CR, int k) {
  const PtR<float>& T = P.F;
  const ArcRule er = make_rule(1, 0);
  if (T.far) return edge_far<float>(T, CR, k, 0.f, 1.f, er);
  return edge_int<float>(T.ws[k], CR.L[k], T.ps[k], T.d, er);
}

// Geometry of apex x against column G and the whole-triangle potential (the
// fully lit case). FP64 path: everything in FP64. Mixed path: the relative
// position, the height d, the foot point and the corner distances in FP64
// (they carry the cancellation between |x - y| and t - tau), the rest in FP32.
// With defer_edges (mixed path only)
// the whole-edge integrals Efull and the whole-triangle value Wst are left to
// the caller (edge_full_mixed per edge, then point_col_finish), so that a warp
// can spread the three edges of its points over its lanes.
STBEM_HD inline void point_col(const double* x, const ColGeom& G, PointCol& P, bool prec_fp32,
                               bool defer_edges = false, const ColR<float>* CRf = nullptr) {
  P.t = x[0];
  double rel[3] = {x[1] - G.c0[0], x[2] - G.c0[1], x[3] - G.c0[2]};
  double d = rel[0] * G.n[0] + rel[1] * G.n[1] + rel[2] * G.n[2];
  if (fabs(d) < 1e-13 * G.diam) d = 0.0;
  double xb0 = rel[0] * G.e1[0] + rel[1] * G.e1[1] + rel[2] * G.e1[2];
  double xb1 = rel[0] * G.e2[0] + rel[1] * G.e2[1] + rel[2] * G.e2[2];
  for (int k = 0; k < 3; ++k) {
    double dx = x[1] - G.X[k][0], dy = x[2] - G.X[k][1], dz = x[3] - G.X[k][2];
    P.r[k] = sqrt(dx * dx + dy * dy + dz * dz);
  }
  if (prec_fp32) {
    PtR<float>& T = P.F;
    T.d = (float)d;
    T.xb[0] = (float)xb0;
    T.xb[1] = (float)xb1;
    int in = 1;
    float out = 0.f, W = 0.f;
    // (the column's FP32 frame from CRf when given: no conversions per point)
    for (int k = 0; k < 3; ++k) {
      T.q[k][0] = (CRf ? CRf->Q[k][0] : (float)G.Q[k][0]) - T.xb[0];
      T.q[k][1] = (CRf ? CRf->Q[k][1] : (float)G.Q[k][1]) - T.xb[1];
      T.rs[k] = (float)P.r[k];
    }
    for (int k = 0; k < 3; ++k) {
      float ux = CRf ? CRf->U[k][0] : (float)G.U[k][0], uy = CRf ? CRf->U[k][1] : (float)G.U[k][1];
      T.ps[k] = T.q[k][0] * uy - T.q[k][1] * ux;
      T.ws[k] = T.q[k][0] * ux + T.q[k][1] * uy;
      if (!(T.ps[k] > 0.f)) in = 0;
      out = fmaxf(out, -T.ps[k]);
      split2(P.r[k] - P.t, P.rho_hi[k], P.rho_lo[k]);
    }
    T.far = out >= FAR_RHO * (CRf ? CRf->diam : (float)G.diam);
    T.C = T.rs[0];
    T.far_rho = out;
    if (!defer_edges) {
      ColR<float> CR;
      make_colr<float>(G, CR);
      for (int k = 0; k < 3; ++k) {
        T.Efull[k] = edge_full_mixed(P, CR, k);
        W += T.Efull[k];
      }
    }
    P.inK = in;
    P.rlo = sqrt(d * d + (double)out * (double)out);
    P.Wst = (double)W;
    P.Wst_f = W;
    P.D.d = d;
    P.D.xb[0] = xb0;
    P.D.xb[1] = xb1;
    split2(-P.t, P.nt_hi, P.nt_lo);
    split2(P.rlo - P.t, P.rlot_hi, P.rlot_lo);
    return;
  }
  PtR<double>& D = P.D;
  D.far = 0;
  D.C = 0.0;
  D.far_rho = 0.0;
  D.d = d;
  D.xb[0] = xb0;
  D.xb[1] = xb1;
  int in = 1;
  double out = 0.0, W = 0.0;
  for (int k = 0; k < 3; ++k) {
    D.q[k][0] = G.Q[k][0] - D.xb[0];
    D.q[k][1] = G.Q[k][1] - D.xb[1];
    D.rs[k] = P.r[k];
  }
  for (int k = 0; k < 3; ++k) {
    D.ps[k] = D.q[k][0] * G.U[k][1] - D.q[k][1] * G.U[k][0];
    D.ws[k] = D.q[k][0] * G.U[k][0] + D.q[k][1] * G.U[k][1];
    if (!(D.ps[k] > 0.0)) in = 0;
    out = fmax(out, -D.ps[k]);
    D.Efull[k] = edge_dE<double>(D.ws[k], G.L[k], D.ps[k], d);
    W += D.Efull[k];
  }
  P.inK = in;
  P.rlo = sqrt(d * d + out * out);
  P.Wst = W;
  P.Wst_f = (float)W;
}

// the whole-triangle value of the mixed path from its three edge integrals
STBEM_HD inline void point_col_finish(PointCol& P) {
  const float W = (P.F.Efull[0] + P.F.Efull[1]) + P.F.Efull[2];
  P.Wst = (double)W;
  P.Wst_f = W;
}

// ---------------------------------------------------------------------------
// Conic arcs (all in precision R)
// ---------------------------------------------------------------------------
template <typename R>
struct ArcFrame {
  R wh[3], ea[3], eb[3];  // circle of directions: n = ca wh + sa (cos th ea + sin th eb)
  R ca, sa;
  R c, d, g[2];
};

// D0 = c^2 - d^2 (1 - |g|^2) is passed in: it sets the conic's size and
// cancels when the cone only just reaches the face plane, so callers form it
// with more care than c and d allow (see cut_in_mixed).
template <typename R>
STBEM_HD inline bool arc_frame(R c, R d, const R* g, R D0, ArcFrame<R>& F) {
  R w[3] = {d * g[0], d * g[1], c};
  R wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  if (!(wn > R(0))) return false;
  if (!(D0 > R(0))) return false;
  for (int i = 0; i < 3; ++i) F.wh[i] = w[i] / wn;
  F.ca = d / wn;
  F.sa = sqrt(D0) / wn;
  R a[3] = {R(1), R(0), R(0)};
  if (fabs(F.wh[0]) >= R(0.8)) { a[0] = R(0); a[1] = R(1); }
  R pa = a[0] * F.wh[0] + a[1] * F.wh[1] + a[2] * F.wh[2];
  R ea[3] = {a[0] - pa * F.wh[0], a[1] - pa * F.wh[1], a[2] - pa * F.wh[2]};
  R la = sqrt(ea[0] * ea[0] + ea[1] * ea[1] + ea[2] * ea[2]);
  for (int i = 0; i < 3; ++i) F.ea[i] = ea[i] / la;
  F.eb[0] = F.wh[1] * F.ea[2] - F.wh[2] * F.ea[1];
  F.eb[1] = F.wh[2] * F.ea[0] - F.wh[0] * F.ea[2];
  F.eb[2] = F.wh[0] * F.ea[1] - F.wh[1] * F.ea[0];
  F.c = c; F.d = d; F.g[0] = g[0]; F.g[1] = g[1];
  return true;
}

template <typename R>
STBEM_HD inline R arc_theta(const ArcFrame<R>& F, const R* y) {
  R r = sqrt(y[0] * y[0] + y[1] * y[1] + F.d * F.d);
  R nh[3] = {-y[0] / r, -y[1] / r, F.d / r};
  R cb = nh[0] * F.eb[0] + nh[1] * F.eb[1] + nh[2] * F.eb[2];
  R cA = nh[0] * F.ea[0] + nh[1] * F.ea[1] + nh[2] * F.ea[2];
  return atan2(cb, cA);
}

// theta(y + dy) - theta(y) in (-pi, pi] for a short step dy: the change of
// the direction nh = (-y, d) / r is formed as ((-dy, 0) - nh (r' - r)) / r'
// with r' - r = <dy, 2y + dy> / (r + r'), so the result keeps its relative
// accuracy when |dy| is much smaller than |y|.
template <typename R>
STBEM_HD inline R arc_dtheta(const ArcFrame<R>& F, const R* y, const R* dy) {
  R r = sqrt(y[0] * y[0] + y[1] * y[1] + F.d * F.d);
  R y1[2] = {y[0] + dy[0], y[1] + dy[1]};
  R r1 = sqrt(y1[0] * y1[0] + y1[1] * y1[1] + F.d * F.d);
  R dr = (dy[0] * (y[0] + y1[0]) + dy[1] * (y[1] + y1[1])) / (r + r1);
  R nh[3] = {-y[0] / r, -y[1] / r, F.d / r};
  R dn[3] = {(-dy[0] - nh[0] * dr) / r1, (-dy[1] - nh[1] * dr) / r1, -nh[2] * dr / r1};
  R a0 = nh[0] * F.ea[0] + nh[1] * F.ea[1] + nh[2] * F.ea[2];
  R a1 = nh[0] * F.eb[0] + nh[1] * F.eb[1] + nh[2] * F.eb[2];
  R b0 = dn[0] * F.ea[0] + dn[1] * F.ea[1] + dn[2] * F.ea[2];
  R b1 = dn[0] * F.eb[0] + dn[1] * F.eb[1] + dn[2] * F.eb[2];
  return atan2(a0 * b1 - a1 * b0, (a0 * a0 + a1 * a1) + (a0 * b0 + a1 * b1));
}

// direction of the conic point y(theta) = -r n_par; returns r, n_par, n_par', n_n, n_n'
template <typename R>
STBEM_HD inline void arc_point(const ArcFrame<R>& F, R th, R& r, R* np, R* dp, R& nn, R& dn) {
  R s, co;
  sc(th, &s, &co);
  R n3[3], d3[3];
  for (int i = 0; i < 3; ++i) {
    n3[i] = F.ca * F.wh[i] + F.sa * (co * F.ea[i] + s * F.eb[i]);
    d3[i] = F.sa * (-s * F.ea[i] + co * F.eb[i]);
  }
  np[0] = n3[0]; np[1] = n3[1]; dp[0] = d3[0]; dp[1] = d3[1]; nn = n3[2]; dn = d3[2];
  if (fabs(F.c) >= fabs(F.d)) r = F.c / (R(1) - (F.g[0] * np[0] + F.g[1] * np[1]));
  else r = F.d / nn;
}

// Arc integrand of (r - |d|) dphi: with r - |d| = r^2 |n_par|^2 / (r + |d|) and
// dphi/dth = cross(n_par, n_par') / |n_par|^2,
//   I(th) = r(th)^2 cross(n_par, n_par') / (r(th) + |d|),
// the direction basis rotated so that th is measured from the interval midpoint.
template <typename R>
struct ArcEval {
  R ca, sa;
  R wh[3], ea[3], eb[3];
  R c, d, g0, g1;
  bool use_c;
  STBEM_HD inline R operator()(R th) const {
    R s, co;
    sc(th, &s, &co);
    R n0 = ca * wh[0] + sa * (co * ea[0] + s * eb[0]);
    R n1 = ca * wh[1] + sa * (co * ea[1] + s * eb[1]);
    R n2 = ca * wh[2] + sa * (co * ea[2] + s * eb[2]);
    R d0 = sa * (-s * ea[0] + co * eb[0]);
    R d1 = sa * (-s * ea[1] + co * eb[1]);
    R r = use_c ? c / (R(1) - (g0 * n0 + g1 * n1)) : d / n2;
    R cr = n0 * d1 - n1 * d0;
    return r * r * cr / (r + fabs(d));
  }
};

// Nearest pole of A0 - A1 cos(theta - th1), in the coordinate u of the
// interval [mid - half, mid + half] -> [-1, 1]: keeps the pole with the
// smallest Bernstein-ellipse parameter rho = s + sqrt(s^2 - 1),
// s = (|u - 1| + |u + 1|) / 2. Complex zeros th1 +- i acosh(A0/A1) when
// A0 > A1; real zeros th1 +- acos(A0/A1) otherwise (the asymptote directions
// of a hyperbolic conic: outside the arc, but possibly close to its ends).
template <typename R>
STBEM_HD inline void pole_at(R th, R eta, R mid, R half, R& best_rho, R& best_a, R& best_b) {
  const R twopi = (R)(2.0 * STBEM_PI);
  R k = rint((mid - th) / twopi);
  R a = (th + twopi * k - mid) / half;
  R b = eta / half;
  R s = R(0.5) * (sqrt((a - R(1)) * (a - R(1)) + b * b) + sqrt((a + R(1)) * (a + R(1)) + b * b));
  R rho = s + sqrt(fmax(s * s - R(1), R(0)));
  if (rho < best_rho) { best_rho = rho; best_a = a; best_b = b; }
}
template <typename R>
STBEM_HD inline void consider_pole(R A0, R Aa, R Ab, R mid, R half, R& best_rho, R& best_a, R& best_b) {
  R A1 = sqrt(Aa * Aa + Ab * Ab);
  if (!(A1 > R(0))) return;
  R th1 = atan2(Ab, Aa);
  if (A0 > A1) {
    pole_at<R>(th1, acosh(A0 / A1), mid, half, best_rho, best_a, best_b);
  } else {
    R ac = acos(fmax(R(-1), A0 / A1));
    pole_at<R>(th1 + ac, R(0), mid, half, best_rho, best_a, best_b);
    pole_at<R>(th1 - ac, R(0), mid, half, best_rho, best_a, best_b);
  }
}

// int_lo^hi I(theta) dtheta. The integrand is a rational trigonometric
// function; its nearest pole sets the Gauss-Legendre order needed
// (error ~ rho^(-2n)). Poles closer than 0.3 half-lengths to the interval
// get a sinh map towards them (Johnston & Elliott 2005) instead.
template <typename R>
STBEM_HD __noinline__ R arc_piece(const ArcFrame<R>& F, R lo, R hi, const ArcRule& rule) {
  R mid = R(0.5) * (lo + hi), half = R(0.5) * (hi - lo);
  if (!(half > R(0))) return R(0);
  R best_rho = R(1e30), best_a = R(0), best_b = R(1e30);
  R sm, cm;
  sc(mid, &sm, &cm);
  {
    // poles of I: L1 = 1 - <g, n_par> = 0 (r -> infinity) and
    // r + |d| = 0, i.e. L1 = -c / |d| (complex for the valid arc). Both are
    // zeros of f = A0 - A1 cos(theta - theta1); since |f(z) - f(mid)| <=
    // A1 sinh|z - mid|, f has no zero within asinh(|f(mid)| / A1) of mid.
    // In FP32, when that disk holds a Bernstein ellipse of the piece with
    // parameter >= 16 (the minimum order already reaches the tolerance there),
    // the exact pole location cannot change the rule and is skipped.
    R gw = F.g[0] * F.wh[0] + F.g[1] * F.wh[1];
    R ga = F.g[0] * F.ea[0] + F.g[1] * F.ea[1];
    R gb = F.g[0] * F.eb[0] + F.g[1] * F.eb[1];
    bool far_poles = false;
    if (sizeof(R) == 4) {
      const R Aa = F.sa * ga, Ab = F.sa * gb;
      const R A1 = sqrt(Aa * Aa + Ab * Ab);
      const R f1 = (R(1) - F.ca * gw) - (Aa * cm + Ab * sm);
      const R f2 = f1 + F.c / fabs(F.d);
      const R fm = fmin(fabs(f1), fabs(f2));
      far_poles = !(A1 > R(0)) || R(2) * asinh(fm / A1) >= R(16) * half;
      // Gauss error ~ R^(-2n): R >= 15.9 and n_min >= 4 reach 15.9^-6 < 1/1.6e7
      far_poles = far_poles && rule.fp32_short;
    }
    if (!far_poles) {
      consider_pole<R>(R(1) - F.ca * gw, F.sa * ga, F.sa * gb, mid, half, best_rho, best_a, best_b);
      consider_pole<R>(R(1) + F.c / fabs(F.d) - F.ca * gw, F.sa * ga, F.sa * gb, mid, half, best_rho, best_a,
                       best_b);
    }
  }
  ArcEval<R> E;
  E.ca = F.ca; E.sa = F.sa;
  for (int i = 0; i < 3; ++i) {
    E.wh[i] = F.wh[i];
    E.ea[i] = cm * F.ea[i] + sm * F.eb[i];
    E.eb[i] = -sm * F.ea[i] + cm * F.eb[i];
  }
  E.c = F.c; E.d = F.d; E.g0 = F.g[0]; E.g1 = F.g[1];
  E.use_c = fabs(F.c) >= fabs(F.d);
  R acc = R(0);
  if (best_b < R(0.3)) {
    const int n = rule.nmax;
    const R* X = gl_nodes<R>(n);
    const R* Wt = gl_weights<R>(n);
    R a = best_a, b = best_b;
    if (a > R(1)) { b = sqrt((a - R(1)) * (a - R(1)) + b * b); a = R(1); }
    else if (a < R(-1)) { b = sqrt((a + R(1)) * (a + R(1)) + b * b); a = R(-1); }
    // a pole computed on the interval itself (rounding of a real pole that
    // lies just outside): keep the map finite
    b = fmax(b, R(sizeof(R) == 4 ? 1e-5 : 1e-12));
    R s1 = asinh((R(1) + a) / b), s2 = asinh((R(1) - a) / b);
    R mu = R(0.5) * (s1 + s2), et = R(0.5) * (s1 - s2);
    for (int k = 0; k < n; ++k) {
      R v = mu * (R)X[k] - et;
      R u = a + b * sinh(v);
      acc += (R)Wt[k] * b * mu * cosh(v) * E(half * u);
    }
  } else {
    int n = rule.nmin;
    if (best_rho < R(1e29)) {
      int need = (int)ceil(rule_ltol<R>(rule) / (R(2) * log(best_rho))) + 1;
      n = need < rule.nmin ? rule.nmin : (need > rule.nmax ? rule.nmax : need);
    }
    const R* X = gl_nodes<R>(n);
    const R* Wt = gl_weights<R>(n);
    for (int k = 0; k < n; ++k) acc += (R)Wt[k] * E(half * (R)X[k]);
  }
  return acc * half;
}

// d = 0: the conic r = c / (1 + G0 cos(psi)), psi = phi - phi_g, has its
// focus at xb; exact antiderivatives of dpsi / (1 + e cos psi).
template <typename R>
STBEM_HD inline R arc_d0_U(R psi, R e) {
  const R pi = (R)STBEM_PI;
  if (e < R(1)) {
    R k = sqrt((R(1) - e) / (R(1) + e));
    return R(2) / sqrt(R(1) - e * e) * (atan(k * tan(R(0.5) * psi)) + pi * floor((psi + pi) / (R(2) * pi)));
  } else if (e > R(1)) {
    // ln|(a + b tan(psi/2)) / (a - b tan(psi/2))| / sqrt(e^2-1), a = sqrt(e+1), b = sqrt(e-1):
    // continuous through psi = pi, singular only on the asymptote directions
    R a = sqrt(e + R(1)), b = sqrt(e - R(1));
    R s, co;
    sc(R(0.5) * psi, &s, &co);
    return log(fabs((a * co + b * s) / (a * co - b * s))) / sqrt(e * e - R(1));
  }
  return tan(R(0.5) * psi);
}

template <typename R>
STBEM_HD __noinline__ R arc_d0(const R* A, const R* dAB, bool full, R c, const R* g) {
  if (c == R(0)) return R(0);
  const R pi = (R)STBEM_PI, twopi = (R)(2.0 * STBEM_PI);
  R G0 = sqrt(g[0] * g[0] + g[1] * g[1]);
  if (full) return twopi * c / sqrt(R(1) - G0 * G0);
  R phg = G0 > R(0) ? atan2(g[1], g[0]) : R(0);
  R pa = atan2(A[1], A[0]);
  // polar angle from A to B = A + dAB around xb, in (-pi, pi]
  R dp = atan2(A[0] * dAB[1] - A[1] * dAB[0], (A[0] * A[0] + A[1] * A[1]) + (A[0] * dAB[0] + A[1] * dAB[1]));
  R span;
  if (c > R(0)) { span = dp; if (span < R(0)) span += twopi; }
  else { span = -dp; if (span < R(0)) span += twopi; span = -span; }
  R psa = pa - phg;
  psa = fmod(psa + pi, twopi);
  if (psa < R(0)) psa += twopi;
  psa -= pi;
  return c * (arc_d0_U<R>(psa + span, G0) - arc_d0_U<R>(psa, G0));
}

// Arc from point A (relative to xb) to B = A + dAB along dE with E on the
// left; full = closed ellipse (A, dAB ignored). dAB is passed on its own so
// that short arcs far from xb keep their relative accuracy.
template <typename R>
STBEM_HD __noinline__ R conic_arc(const R* A, const R* dAB, bool full, R c, R d, const R* g, R D0,
                                  const ArcRule& rule, double c64, const double* g64, bool tiny_is_short = false) {
  if (d == R(0)) {
    // closed form in FP64 in every precision: it is a difference of
    // antiderivative values, and it only arises for coplanar pairs
    double A64[2] = {A ? (double)A[0] : 0.0, A ? (double)A[1] : 0.0};
    double D64[2] = {dAB ? (double)dAB[0] : 0.0, dAB ? (double)dAB[1] : 0.0};
    return (R)arc_d0<double>(A64, D64, full, c64, g64);
  }
  ArcFrame<R> F;
  if (!arc_frame<R>(c, d, g, D0, F)) return R(0);
  if (F.sa < R(sizeof(R) == 4 ? 1e-6 : 1e-14)) return R(0);
  const R pi = (R)STBEM_PI, twopi = (R)(2.0 * STBEM_PI);
  R thA = full ? R(0) : arc_theta<R>(F, A);
  // orientation: tangent dy/dtheta against grad F = g + y/r at the start point
  R r, np[2], dp[2], nn, dn;
  arc_point<R>(F, thA, r, np, dp, nn, dn);
  R dr;
  if (fabs(F.c) >= fabs(F.d)) {
    R L1 = R(1) - (g[0] * np[0] + g[1] * np[1]);
    dr = r * (g[0] * dp[0] + g[1] * dp[1]) / L1;
  } else {
    dr = -r * dn / nn;
  }
  R T[2] = {-dr * np[0] - r * dp[0], -dr * np[1] - r * dp[1]};
  R y[2] = {-r * np[0], -r * np[1]};
  R ry = sqrt(y[0] * y[0] + y[1] * y[1] + d * d);
  R gF[2] = {g[0] + y[0] / ry, g[1] + y[1] / ry};
  R s = (T[0] * gF[1] - T[1] * gF[0]) < R(0) ? R(1) : R(-1);
  R span;
  if (full) span = twopi;
  else {
    R dth = arc_dtheta<R>(F, A, dAB);
    if (sizeof(R) == 4 && !(fabs(dth) >= R(1e-5))) {
      // FP32: the two events are as close as their rounding (the cone grazing
      // a corner), so the sign of the span cannot tell a vanishing arc from a
      // full turn. Where the lit set cannot be a whole ellipse inside the
      // triangle (tiny_is_short) the arc is the short one; otherwise NaN asks
      // the caller to recompute the face in FP64.
      if (!tiny_is_short) return (R)nan("");
      span = fabs(dth);
    } else {
      span = s > R(0) ? dth : -dth;
      if (span < R(0)) span += twopi;
    }
  }
  R lo = s > R(0) ? thA : thA - span;
  R hi = s > R(0) ? thA + span : thA;
  R val;
  if (span > pi) {
    R m = R(0.5) * (lo + hi);
    val = arc_piece<R>(F, lo, m, rule) + arc_piece<R>(F, m, hi, rule);
  } else {
    val = arc_piece<R>(F, lo, hi, rule);
  }
  return s * val;
}

// Column frame of a spatial triangle with corners X0, X1, X2 (counter-clockwise
// in the frame by construction: n = (X1-X0) x (X2-X0)).
STBEM_HD inline void make_colgeom(const double* X0, const double* X1, const double* X2, ColGeom& G) {
  for (int i = 0; i < 3; ++i) {
    G.X[0][i] = X0[i]; G.X[1][i] = X1[i]; G.X[2][i] = X2[i];
    G.c0[i] = X0[i];
  }
  double a[3] = {X1[0] - X0[0], X1[1] - X0[1], X1[2] - X0[2]};
  double b[3] = {X2[0] - X0[0], X2[1] - X0[1], X2[2] - X0[2]};
  double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double al = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  for (int i = 0; i < 3; ++i) { G.n[i] = n[i] / nl; G.e1[i] = a[i] / al; }
  G.e2[0] = G.n[1] * G.e1[2] - G.n[2] * G.e1[1];
  G.e2[1] = G.n[2] * G.e1[0] - G.n[0] * G.e1[2];
  G.e2[2] = G.n[0] * G.e1[1] - G.n[1] * G.e1[0];
  G.Q[0][0] = 0.0; G.Q[0][1] = 0.0;
  G.Q[1][0] = al;  G.Q[1][1] = 0.0;
  G.Q[2][0] = b[0] * G.e1[0] + b[1] * G.e1[1] + b[2] * G.e1[2];
  G.Q[2][1] = b[0] * G.e2[0] + b[1] * G.e2[1] + b[2] * G.e2[2];
  G.diam = 0.0;
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    double ex = G.Q[k1][0] - G.Q[k][0], ey = G.Q[k1][1] - G.Q[k][1];
    double l = sqrt(ex * ex + ey * ey);
    G.L[k] = l; G.U[k][0] = ex / l; G.U[k][1] = ey / l;
    G.diam = fmax(G.diam, l);
  }
  G.area = 0.5 * nl;
  for (int i = 0; i < 3; ++i) G.ctr[i] = (X0[i] + X1[i] + X2[i]) / 3.0;
  G.rad = 0.0;
  for (int k = 0; k < 3; ++k) {
    double dx = G.X[k][0] - G.ctr[0], dy = G.X[k][1] - G.ctr[1], dz = G.X[k][2] - G.ctr[2];
    G.rad = fmax(G.rad, sqrt(dx * dx + dy * dy + dz * dz));
  }
}

STBEM_HD inline void face_gradient(const ColGeom& G, FaceGeom& F) {
  F.g[0] = (F.p[1] - F.p[0]) / G.Q[1][0];
  F.g[1] = ((F.p[2] - F.p[0]) - F.g[0] * G.Q[2][0]) / G.Q[2][1];
}

// ---------------------------------------------------------------------------
// 4 pi W_P(x) for a face with corner times p[3] and in-frame gradient g.
// Step 1 (FP64): cone-function values F_k = P(corner_k) + |x_s - corner_k| - t
// at the corners decide the fully lit (all < 0: the whole-triangle value)
// and certainly dark cases; c = t - P(xb).
// Step 2 (precision R): the cut case, by Green's theorem on dR.
// ---------------------------------------------------------------------------
enum { FACE_DARK = 0, FACE_LIT = 1, FACE_CUT = 2 };

STBEM_HD inline int face_class(const ColGeom& G, const PointCol& P, const FaceGeom& Fc, double* F, double& c) {
  const double t = P.t;
  int nlit = 0;
  double pmin = Fc.p[0];
  for (int k = 0; k < 3; ++k) {
    F[k] = (Fc.p[k] - t) + P.r[k];
    if (F[k] < 0.0) ++nlit;
    pmin = fmin(pmin, Fc.p[k]);
  }
  if (nlit == 3) return FACE_LIT;
  // P + r - t >= min p + dist(x_s, K) - t >= 0: no lit point
  if ((pmin - t) + P.rlo >= 0.0) return FACE_DARK;
  // c = t - P(xb), P(xb) = p0 + <g, xb - Q0>, Q0 = 0
  c = t - (Fc.p[0] + Fc.g[0] * P.D.xb[0] + Fc.g[1] * P.D.xb[1]);
  if (fabs(c) < 1e-13 * G.diam) c = 0.0;
  return FACE_CUT;
}

// Step 1 for the mixed path in FP32 pairs: F_k = p_k + (r_k - t) and
// c = -((p_0 - t) + <g, xb>) keep their absolute accuracy although p_k, r_k
// and t are O(T) and F_k, c are O(diam K) near the cone.
STBEM_HD inline int face_class_mixed(const PointCol& P, const FaceF& Fc, float* F, float& c, float diam) {
  int nlit = 0;
  for (int k = 0; k < 3; ++k) {
    F[k] = add2(Fc.p_hi[k], Fc.p_lo[k], P.rho_hi[k], P.rho_lo[k]);
    if (F[k] < 0.f) ++nlit;
  }
  if (nlit == 3) return FACE_LIT;
  if (add2(Fc.pmin_hi, Fc.pmin_lo, P.rlot_hi, P.rlot_lo) >= 0.f) return FACE_DARK;
  {
    // F = P + |x_s - y| - t is convex on K: its tangent plane at the corner m
    // of smallest F, F_m + (P(y) - P(Q_m)) + <Q_m - xb, y - Q_m> / r_m, bounds
    // it from below and is linear, so no point of K is lit when the bound is
    // positive at the three corners (margin: the FP32 error of the linear term)
    const int m = F[0] <= F[1] ? (F[0] <= F[2] ? 0 : 2) : (F[1] <= F[2] ? 1 : 2);
    const float qx = P.F.q[m][0], qy = P.F.q[m][1], rm = P.F.rs[m];
    float lo = F[m];
    for (int k = 0; k < 3; ++k) {
      if (k == m) continue;
      const float dp = add2(Fc.p_hi[k], Fc.p_lo[k], -Fc.p_hi[m], -Fc.p_lo[m]);
      const float lin = (qx * (P.F.q[k][0] - qx) + qy * (P.F.q[k][1] - qy)) / rm;
      lo = fminf(lo, F[m] + dp + lin);
    }
    if (lo > 4e-7f * rm) return FACE_DARK;
  }
  float p0t = add2(Fc.p_hi[0], Fc.p_lo[0], P.nt_hi, P.nt_lo);
  c = -(p0t + (Fc.g[0] * P.F.xb[0] + Fc.g[1] * P.F.xb[1]));
  if (fabsf(c) < 1e-6f * diam) c = 0.f;
  return FACE_CUT;
}

// Near-singular faces of the mixed path, computed in FP64: the apex lies
// nearly in the plane of K (|d| < 0.01 diam K: the cone's directions to the
// plane are nearly tangent to it), or nearly in it with the cone's vertex
// near the plane as well (|c|, |d| < 0.05 diam K: the conic passes close to
// its focus). FP32 arcs lose up to 1e-4 of W on both.
STBEM_HD inline bool near_singular_mixed(float c, float d, float diam) {
  return fabsf(d) < 0.01f * diam || fmaxf(fabsf(c), fabsf(d)) < 0.05f * diam;
}

// Inputs of the cut case in precision R: cone-function values F_k at the
// corners, a0_k = t - p_k, a1_k = p_{k+1} - p_k, the in-frame gradient g,
// c = t - P(xb); c64 / g64 feed the FP64 closed form of coplanar (d = 0) arcs.
template <typename R>
struct FaceCutIn {
  R F[3], a0[3], a1[3], g[2], c;
  R D0;                // c^2 - d^2 (1 - |g|^2), the conic's size (see cut_in_mixed)
  double c64, g64[2];
};

STBEM_HD inline void cut_in_fp64(const PointCol& P, const FaceGeom& Fc, const double* F, double c,
                                 FaceCutIn<double>& o) {
  for (int k = 0; k < 3; ++k) {
    o.F[k] = F[k];
    o.a0[k] = P.t - Fc.p[k];
    o.a1[k] = Fc.p[(k + 1) % 3] - Fc.p[k];
  }
  o.g[0] = o.g64[0] = Fc.g[0];
  o.g[1] = o.g64[1] = Fc.g[1];
  o.c = o.c64 = c;
  o.D0 = c * c - P.D.d * P.D.d * (1.0 - (Fc.g[0] * Fc.g[0] + Fc.g[1] * Fc.g[1]));
}

STBEM_HD inline void cut_in_mixed(const PointCol& P, const FaceF& Fc, const float* F, float c, const FaceGeom& F64,
                                  FaceCutIn<float>& o) {
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    o.F[k] = F[k];
    o.a0[k] = -add2(Fc.p_hi[k], Fc.p_lo[k], P.nt_hi, P.nt_lo);
    o.a1[k] = add2(Fc.p_hi[k1], Fc.p_lo[k1], -Fc.p_hi[k], -Fc.p_lo[k]);
  }
  o.g[0] = Fc.g[0]; o.g[1] = Fc.g[1];
  o.g64[0] = F64.g[0]; o.g64[1] = F64.g[1];
  o.c = c;
  o.c64 = (double)c;
  // the conic's size D0 = c^2 - d^2 (1 - |g|^2): where the cone only just
  // reaches the face plane (|D0| < c^2 / 20) its two terms cancel, and c (an
  // O(1) difference formed in FP32 pairs, but with <g, xb> in FP32) loses the
  // relative accuracy D0 needs; there it is formed in FP64 from the apex's
  // FP64 geometry (about 3 % of the cut faces)
  const float d = P.F.d;
  float D0 = c * c - d * d * (1.f - (Fc.g[0] * Fc.g[0] + Fc.g[1] * Fc.g[1]));
  if (fabsf(D0) < 0.05f * c * c) {
    const double c64 = P.t - (F64.p[0] + (F64.g[0] * P.D.xb[0] + F64.g[1] * P.D.xb[1]));
    const double d64 = P.D.d;
    D0 = (float)(c64 * c64 - d64 * d64 * (1.0 - (F64.g[0] * F64.g[0] + F64.g[1] * F64.g[1])));
  }
  o.D0 = D0;
}

// A conic arc of a cut face (d != 0) recorded for evaluation later: the
// quadrature kernel collects the arcs of all cut pairs of a warp and then
// integrates them one per lane over the compacted list.
// Far-field arcs (far != 0) keep A in column coordinates and the apex data
// of the far-field form (foot point xb, C, far_rho).
template <typename R>
struct ArcRec {
  R A[2], dAB[2], c, d, g[2], D0;
  R xb[2], C, far_rho;
  int full, tiny_is_short, far;
};

// A far-field arc over its chord (arc_far), or conic_arc shifted from the
// integrand r - |d| to r - C by (|d| - C) times the angle the arc spans at xb
// (strongly curved arcs, or the long way round). A: start in column
// coordinates.
template <typename R>
STBEM_HD inline R far_arc_value(const R* xb, R d, R C, R far_rho, R c, const R* g, R D0, const R* A, const R* dAB,
                                bool tiny_short, const ArcRule& rule, double c64, const double* g64) {
  R v;
  if (arc_far<R>(xb, d, C, far_rho, g, A, dAB, rule, v)) return v;
  const R ya[2] = {A[0] - xb[0], A[1] - xb[1]};
  v = conic_arc<R>(ya, dAB, false, c, d, g, D0, rule, c64, g64, tiny_short);
  const R bx = ya[0] + dAB[0], by = ya[1] + dAB[1];
  const R dphi = atan2(ya[0] * by - ya[1] * bx, ya[0] * bx + ya[1] * by);
  return v - (xb[0] * xb[0] + xb[1] * xb[1]) / (C + fabs(d)) * dphi;
}

template <typename R>
STBEM_HD inline R arc_value(const ArcRec<R>& a, const ArcRule& rule) {
  if (a.far)
    return far_arc_value<R>(a.xb, a.d, a.C, a.far_rho, a.c, a.g, a.D0, a.A, a.dAB, a.tiny_is_short != 0, rule, 0.0,
                            nullptr);
  return conic_arc<R>(a.full ? nullptr : a.A, a.full ? nullptr : a.dAB, a.full != 0, a.c, a.d, a.g, a.D0, rule, 0.0,
                      nullptr, a.tiny_is_short != 0);
}

// 4 pi W_P(x) of a cut face. With `defer` given, arcs with d != 0 (at most
// three) are appended to defer[*ndefer] instead of integrated, and the
// return value holds the edge pieces (and any coplanar arc) only.
template <typename R>
STBEM_HD __noinline__ double face_cut(const ColR<R>& G, const PointCol& P64, const FaceCutIn<R>& in,
                                      const ArcRule& rule, ArcRec<R>* defer = nullptr, int* ndefer = nullptr) {
  const PtR<R>& P = pt<R>(P64);
  const R d = P.d, c = in.c;
  const R* g = in.g;
  const R* F = in.F;
  R total = R(0);
  R ev_y[6][2], ev_l[6][2];
  int ev_in[6];
  int nev = 0;
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    R la = R(0), lb = R(1);
    bool has = false, la_root = false, lb_root = false;
    if (F[k] < R(0) && F[k1] < R(0)) {
      has = true;
    } else {
      R a0 = in.a0[k], a1 = in.a1[k];
      R Ex = G.U[k][0] * G.L[k], Ey = G.U[k][1] * G.L[k];
      R A2 = G.L[k] * G.L[k] - a1 * a1;
      R B2 = R(2) * ((P.q[k][0] * Ex + P.q[k][1] * Ey) + a0 * a1);
      R C2 = F[k] * (P.rs[k] + a0);   // |q_k|^2 + d^2 - a0^2 without cancellation
      R rt[2];
      int nr = 0;
      if (fabs(A2) <= R(sizeof(R) == 4 ? 1e-6 : 1e-14) * (G.L[k] * G.L[k] + a1 * a1)) {
        if (B2 != R(0)) rt[nr++] = -C2 / B2;
      } else {
        R disc = B2 * B2 - R(4) * A2 * C2;
        if (disc >= R(0)) {
          R sq = sqrt(disc);
          R qq = R(-0.5) * (B2 + (B2 >= R(0) ? sq : -sq));
          if (qq != R(0)) { rt[nr++] = qq / A2; rt[nr++] = C2 / qq; }
          else rt[nr++] = R(0);
        }
      }
      // keep roots of r = a (a = t - P >= 0), not of r = -a
      R v[2];
      int nv = 0;
      const R slack = R(sizeof(R) == 4 ? 1e-5 : 1e-12);
      for (int i = 0; i < nr; ++i)
        if (a0 - a1 * rt[i] > R(0) && rt[i] >= -slack && rt[i] <= R(1) + slack) v[nv++] = fmin(R(1), fmax(R(0), rt[i]));
      if (nv == 2 && v[0] > v[1]) { R tmp = v[0]; v[0] = v[1]; v[1] = tmp; }
      // F is convex along the edge: with F(0) < 0 <= F(1) its root in [0, 1] is
      // the larger one (the other lies before the edge start); with
      // F(0) >= 0 > F(1) it is the smaller one
      if (F[k] < R(0)) {           // exit on this edge
        lb = nv ? v[nv - 1] : R(1); lb_root = nv > 0; has = true;
      } else if (F[k1] < R(0)) {   // entry on this edge
        la = nv ? v[0] : R(0); la_root = nv > 0; has = true;
      } else if (nv == 2 && v[1] > v[0]) {
        la = v[0]; lb = v[1]; la_root = lb_root = true; has = true;
      }
    }
    if (!has) continue;
    if (!la_root && !lb_root) total += P.Efull[k];
    else if (P.far) total += edge_far<R>(P, G, k, la, lb, rule);
    else total += edge_int<R>(P.ws[k] + la * G.L[k], (lb - la) * G.L[k], P.ps[k], d, rule);
    // events relative to xb (O(distance)) and in column coordinates (O(diam K));
    // differences of the latter give arc spans without cancellation
    for (int e = 0; e < 2; ++e) {
      if (!(e == 0 ? la_root : lb_root)) continue;
      R lam = e == 0 ? la : lb;
      ev_in[nev] = e == 0;
      ev_y[nev][0] = P.q[k][0] + lam * G.U[k][0] * G.L[k];
      ev_y[nev][1] = P.q[k][1] + lam * G.U[k][1] * G.L[k];
      ev_l[nev][0] = G.Q[k][0] + lam * G.U[k][0] * G.L[k];
      ev_l[nev][1] = G.Q[k][1] + lam * G.U[k][1] * G.L[k];
      ++nev;
    }
  }
  // the lit set is a whole ellipse inside K only if the conic is bounded and
  // narrower than K (its width across g is at least 2 sqrt(c^2 - d^2))
  const bool tiny_short = (g[0] * g[0] + g[1] * g[1] >= R(1)) || (c * c - d * d > R(0.25) * G.diam * G.diam);
  if (nev > 0) {
    // events are in perimeter order; each exit connects to the next entry
    for (int i = 0; i < nev; ++i) {
      if (ev_in[i]) continue;
      for (int s = 1; s <= nev; ++s) {
        int j = (i + s) % nev;
        if (ev_in[j]) {
          R dAB[2] = {ev_l[j][0] - ev_l[i][0], ev_l[j][1] - ev_l[i][1]};
          if (P.far && !(defer && d != R(0))) {
            total += far_arc_value<R>(P.xb, d, P.C, P.far_rho, c, g, in.D0, ev_l[i], dAB, tiny_short, rule, in.c64,
                                      in.g64);
            break;
          }
          if (defer && d != R(0)) {
            ArcRec<R>& a = defer[(*ndefer)++];
            a.far = P.far;
            if (P.far) {
              a.A[0] = ev_l[i][0]; a.A[1] = ev_l[i][1];
              a.xb[0] = P.xb[0]; a.xb[1] = P.xb[1]; a.C = P.C; a.far_rho = P.far_rho;
            } else {
              a.A[0] = ev_y[i][0]; a.A[1] = ev_y[i][1];
            }
            a.dAB[0] = dAB[0]; a.dAB[1] = dAB[1];
            a.c = c; a.d = d; a.g[0] = g[0]; a.g[1] = g[1]; a.D0 = in.D0; a.full = 0; a.tiny_is_short = tiny_short;
          } else {
            total += conic_arc<R>(ev_y[i], dAB, false, c, d, g, in.D0, rule, in.c64, in.g64, tiny_short);
          }
          break;
        }
      }
    }
  } else {
    // no crossing: E inside K (closed ellipse) or E cap K empty
    R G2 = g[0] * g[0] + g[1] * g[1];
    if (!(G2 < R(1) && c > R(0) && in.D0 > R(0))) return 0.0;   // c > |d| sqrt(1 - |g|^2)
    R G0 = sqrt(G2);
    R sst = G0 > R(0) ? fabs(d) * G0 / sqrt(R(1) - G2) : R(0);
    R yst[2] = {G0 > R(0) ? -sst * g[0] / G0 : R(0), G0 > R(0) ? -sst * g[1] / G0 : R(0)};
    for (int k = 0; k < 3; ++k) {
      R rel[2] = {yst[0] - P.q[k][0], yst[1] - P.q[k][1]};
      if (!(G.U[k][0] * rel[1] - G.U[k][1] * rel[0] > R(0))) return 0.0;
    }
    if (defer && d != R(0)) {
      ArcRec<R>& a = defer[(*ndefer)++];
      a.A[0] = a.A[1] = a.dAB[0] = a.dAB[1] = R(0);
      a.c = c; a.d = d; a.g[0] = g[0]; a.g[1] = g[1]; a.D0 = in.D0; a.full = 1; a.tiny_is_short = 0; a.far = 0;
    } else {
      total += conic_arc<R>(nullptr, nullptr, true, c, d, g, in.D0, rule, in.c64, in.g64);
    }
  }
  return (double)total;
}

// 4 pi W_P(x) in one call (used by the kernel-level entry point and checks)
template <bool FP32>
STBEM_HD inline double face_W(const ColGeom& G, const PointCol& P, const FaceGeom& Fc, const ArcRule& rule) {
  if (FP32) {
    FaceF Ff;
    make_facef(Fc, Ff);
    float F[3], c = 0.f;
    int cls = face_class_mixed(P, Ff, F, c, (float)G.diam);
    if (cls == FACE_LIT) return P.Wst;
    if (cls == FACE_DARK) return 0.0;
    if (near_singular_mixed(c, P.F.d, (float)G.diam)) return nan("");   // the caller recomputes it in FP64
    ColR<float> CR;
    make_colr<float>(G, CR);
    FaceCutIn<float> in;
    cut_in_mixed(P, Ff, F, c, Fc, in);
    return face_cut<float>(CR, P, in, rule);
  }
  double F[3], c = 0.0;
  int cls = face_class(G, P, Fc, F, c);
  if (cls == FACE_LIT) return P.Wst;
  if (cls == FACE_DARK) return 0.0;
  ColR<double> CR;
  make_colr<double>(G, CR);
  FaceCutIn<double> in;
  cut_in_fp64(P, Fc, F, c, in);
  return face_cut<double>(CR, P, in, rule);
}

// 4 pi W_P(x) entirely in FP64 from the apex coordinates: the fallback of the
// mixed path for near-singular faces and for faces whose FP32 evaluation is
// not finite (see conic_arc). The arc rule aims at 1e-10 (the mixed operator's
// target is 1e-7): pieces away from a pole take fewer nodes than the FP64
// operator's 1e-15 rule needs.
STBEM_HD __noinline__ inline double face_W_fp64(const double* x, const ColGeom& G, const FaceGeom& Fc, int n_theta) {
  PointCol P;
  point_col(x, G, P, false);
  ArcRule r;
  r.nmin = 4;
  r.nmax = n_theta ? n_theta : 32;   // pieces next to a pole (sinh map) take nmax
  r.tol = 1e-10;
  rule_finish(r);
  return face_W<false>(G, P, Fc, r);
}

}  // namespace stbem
