/*
 * Plain FP64 CPU oracle for the energetic retarded single-layer Galerkin
 * matrix of Poelz & Schanz, "On the space-time discretization of variational
 * retarded potential boundary integral equations".
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file. The product path never calls it and
 * shares no code with it.
 *
 * What it computes, each step citing the paper:
 *   - panels as intersections of half-spaces with outward conormals
 *     (Sec. 3.1, eq. pnl_ilf; face distance eq. dist_faces);
 *   - the inner integral I = T_k 1_sigma (x) of Def. int_inner for the single
 *     layer kernel k_1 (eq. kfunc), through the light-cone parametrization of
 *     Def. lc_para with the choices of Def. choice_r (rotation R, scale r0,
 *     causality r0 <= 0 => 0) and the hyperplane condition eq. para_hypl
 *     (rho0 = <x - x_sigma, nu>/r0).  On the chart l_2 of Sec. 3.1 the
 *     integrand k_{psi,1}(l_2) J_{l_2} of eq. kernel_para_full equals r0
 *     (the chart Jacobian is not printed in the paper; it is derived from the
 *     map l_2 and the product is exactly r0, and the same holds on l_1), so
 *     I = r0 * area{(rho, phi): rho in [|rho0|, 1], phi_sigma(psi(l_2)) < 0}
 *     (eq. int_inner_param). The paper integrates this region with a quadtree
 *     of exactly parametrised cells; here the rho-measure along every phi is
 *     taken exactly from the roots of the four face functions, and the
 *     phi-integral is taken by adaptive Gauss-Legendre pairs on the pieces
 *     between the phi where the rho-structure changes;
 *   - V 1_sigma = I / (4 pi) (the Lemma drops the 4 pi of k_1);
 *   - the outer integral of eq. int_bform for P0 test functions,
 *     A_ij = -sum_{F in faces(sigma_i)} nu_{F,t} int_F V 1_{sigma_j} dS,
 *     with the composite midpoint rule of Fig. int_tri_mid (m_Q^2 congruent
 *     sub-triangles, one centroid each);
 *   - the right-hand side b_I(g, v_h) = -sum_F nu_{F,t} int_F g dS of
 *     eq. int_bform with A = Id, by a composite Duffy-collapsed Gauss rule
 *     fine enough to resolve the data;
 *   - the sparsity predicate (causality, strong Huygens principle, spatial
 *     reach) in a fixed FP64 operation order;
 *   - dense LU with partial pivoting.
 * Compile with -ffp-contract=off so every product and sum rounds on its own.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n            */
/* ------------------------------------------------------------------ */
#define GMAX 40
typedef struct { int n; double x[GMAX]; double w[GMAX]; } gauss_rule;

static void gauss_legendre(int n, gauss_rule* g) {
  g->n = n;
  for (int i = 0; i < n; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    g->x[i] = z;
    g->w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static gauss_rule G_LO, G_HI, G_FACE;
static pthread_once_t rules_once = PTHREAD_ONCE_INIT;
static void init_rules(void) {
  gauss_legendre(10, &G_LO);
  gauss_legendre(16, &G_HI);
  gauss_legendre(12, &G_FACE);
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot4(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double det3(const double a[3], const double b[3], const double c[3]) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
         a[2] * (b[0] * c[1] - b[1] * c[0]);
}

/* ------------------------------------------------------------------ */
/* Tetrahedron in R^4: hyperplane normal, outward face conormals        */
/* (eq. pnl_ilf), face areas                                           */
/* ------------------------------------------------------------------ */
typedef struct {
  double X[4][4];      /* vertices (t, x, y, z) */
  double nu[4];        /* unit normal of the panel's tangent hyperplane */
  double cn[4][4];     /* cn[i]: outward unit conormal of the face opposite vertex i */
  double area[4];      /* area of the face opposite vertex i */
  double vol;          /* 3-volume of the panel */
} tet_geom;

static void tet_geometry(const double X[4][4], tet_geom* g) {
  memcpy(g->X, X, sizeof(g->X));
  double E[3][4];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 4; ++c) E[k][c] = X[k + 1][c] - X[0][c];
  /* generalized cross product: component c is (-1)^c times the minor without column c */
  for (int c = 0; c < 4; ++c) {
    double m[3][3];
    for (int r = 0; r < 3; ++r) {
      int cc = 0;
      for (int q = 0; q < 4; ++q)
        if (q != c) m[r][cc++] = E[r][q];
    }
    double d = det3(m[0], m[1], m[2]);
    g->nu[c] = (c % 2 == 0) ? d : -d;
  }
  double nn = sqrt(dot4(g->nu, g->nu));
  g->vol = nn / 6.0;
  for (int c = 0; c < 4; ++c) g->nu[c] /= nn;
  for (int i = 0; i < 4; ++i) {
    int a = (i + 1) % 4, b = (i + 2) % 4, cidx = (i + 3) % 4;
    double u1[4], u2[4], w[4], q1[4], q2[4];
    for (int c = 0; c < 4; ++c) {
      u1[c] = X[b][c] - X[a][c];
      u2[c] = X[cidx][c] - X[a][c];
      w[c] = X[i][c] - X[a][c];
    }
    double l1 = sqrt(dot4(u1, u1));
    for (int c = 0; c < 4; ++c) q1[c] = u1[c] / l1;
    double p = dot4(u2, q1);
    for (int c = 0; c < 4; ++c) q2[c] = u2[c] - p * q1[c];
    double l2 = sqrt(dot4(q2, q2));
    for (int c = 0; c < 4; ++c) q2[c] /= l2;
    double w1 = dot4(w, q1), w2 = dot4(w, q2);
    double wp[4];
    for (int c = 0; c < 4; ++c) wp[c] = w[c] - w1 * q1[c] - w2 * q2[c];
    double lw = sqrt(dot4(wp, wp));
    for (int c = 0; c < 4; ++c) g->cn[i][c] = -wp[c] / lw;
    double uu = dot4(u1, u1) * dot4(u2, u2) - dot4(u1, u2) * dot4(u1, u2);
    g->area[i] = 0.5 * sqrt(uu > 0 ? uu : 0.0);
  }
}

/* ------------------------------------------------------------------ */
/* Inner integral (Sec. 3.1)                                           */
/* ------------------------------------------------------------------ */
typedef struct {
  double r0, rho0, rhoa, rho0sq;
  double gam[4], alp[4], bx[4], by[4];
} inner_ctx;

/* f_i(rho) = <psi(l_2(rho,phi)) - X_i, nu_i>/1 with
 *   psi = x - r0 rho (1, R e(phi, theta)), rho cos(theta) = rho0:
 *   f_i = gam_i - alp_i rho - beta_i(phi) sqrt(rho^2 - rho0^2),
 *   gam_i = <x - X_face_i, nu_i>, alp_i = r0 nu_{i,t},
 *   beta_i(phi) = r0 <cos(phi) e1 + sin(phi) e2, nu_{i,x}>.        */
static double face_fn(const inner_ctx* c, int i, double beta, double rho) {
  double q2 = rho * rho - c->rho0sq;
  double q = q2 > 0 ? sqrt(q2) : 0.0;
  return c->gam[i] - c->alp[i] * rho - beta * q;
}

static int face_roots(const inner_ctx* c, int i, double beta, double lo, double hi, double* out) {
  double al = c->alp[i], ga = c->gam[i];
  double a = al * al - beta * beta;
  double b = -2.0 * al * ga;
  double cc = ga * ga + beta * beta * c->rho0sq;
  double cand[2];
  int nc = 0;
  double scale = fabs(al) + fabs(beta) + fabs(ga);
  if (scale == 0.0) return 0;
  if (fabs(beta) <= 1e-15 * (fabs(al) + fabs(ga))) {
    /* face with a purely temporal conormal: f_i is linear in rho */
    if (al != 0.0) cand[nc++] = ga / al;
  } else if (fabs(a) <= 1e-15 * (al * al + beta * beta)) {
    if (b != 0.0) cand[nc++] = -cc / b;
  } else {
    double disc = b * b - 4.0 * a * cc;
    /* a double root may round to a slightly negative discriminant */
    if (disc < 0.0 && disc > -1e-13 * b * b) disc = 0.0;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double q = -0.5 * (b + (b >= 0 ? sq : -sq));
    if (q != 0.0) {
      cand[nc++] = q / a;
      cand[nc++] = cc / q;
    } else {
      cand[nc++] = 0.0;
    }
  }
  int n = 0;
  for (int k = 0; k < nc; ++k) {
    double r = cand[k];
    if (!(r > lo && r < hi)) continue;
    /* one guarded Newton step on the unsquared function */
    double f = face_fn(c, i, beta, r);
    double q2 = r * r - c->rho0sq;
    if (q2 > 1e-24) {
      double df = -al - beta * r / sqrt(q2);
      if (df != 0.0) {
        double rn = r - f / df;
        if (rn > lo && rn < hi) {
          double fn = face_fn(c, i, beta, rn);
          if (fabs(fn) < fabs(f)) { r = rn; f = fn; }
        }
      }
    }
    /* reject roots of the squared equation that belong to the other branch */
    if (fabs(f) > 1e-9 * scale) continue;
    out[n++] = r;
  }
  return n;
}

static void sort_small(double* v, int n) {
  for (int i = 1; i < n; ++i) {
    double x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
    v[j + 1] = x;
  }
}

/* exact measure of {rho in [|rho0|, 1] : max_i f_i(rho) < 0} along phi */
static double rho_measure(const inner_ctx* c, double phi) {
  double cp = cos(phi), sp = sin(phi);
  double beta[4];
  double br[12];
  int nb = 0;
  br[nb++] = c->rhoa;
  br[nb++] = 1.0;
  for (int i = 0; i < 4; ++i) {
    beta[i] = c->bx[i] * cp + c->by[i] * sp;
    nb += face_roots(c, i, beta[i], c->rhoa, 1.0, br + nb);
  }
  sort_small(br, nb);
  double L = 0.0;
  for (int k = 0; k + 1 < nb; ++k) {
    double a = br[k], b = br[k + 1];
    if (!(b > a)) continue;
    double m = 0.5 * (a + b);
    int inside = 1;
    for (int i = 0; i < 4 && inside; ++i)
      if (!(face_fn(c, i, beta[i], m) < 0.0)) inside = 0;
    if (inside) L += b - a;
  }
  return L;
}

/* smoothstep map u in [0,1] -> phi in [a,b]; both ends get a vanishing
 * derivative so that square-root end behaviour at tangency is regular */
static double piece_gauss(const inner_ctx* c, double a, double b, const gauss_rule* g) {
  double s = 0.0, h = b - a;
  for (int k = 0; k < g->n; ++k) {
    double u = 0.5 * (g->x[k] + 1.0);
    double phi = a + h * u * u * (3.0 - 2.0 * u);
    double dphi = h * 6.0 * u * (1.0 - u);
    s += 0.5 * g->w[k] * dphi * rho_measure(c, phi);
  }
  return s;
}

static double piece_adaptive(const inner_ctx* c, double a, double b, int depth) {
  double lo = piece_gauss(c, a, b, &G_LO);
  double hi = piece_gauss(c, a, b, &G_HI);
  double tol = 1e-15 * (b - a) + 1e-17;
  if (fabs(hi - lo) <= tol || depth >= 40) return hi;
  double m = 0.5 * (a + b);
  return piece_adaptive(c, a, m, depth + 1) + piece_adaptive(c, m, b, depth + 1);
}

static double wrap2pi(double p) {
  double t = fmod(p, 2.0 * ORC_PI);
  if (t < 0) t += 2.0 * ORC_PI;
  return t;
}

/* I (without 1/(4 pi)) for apex x and panel g */
static double inner_I(const double x[4], const tet_geom* g) {
  double t = x[0];
  /* Def. choice_r: r0 = sup_{y in sigma} (t - tau) = max over vertices */
  double r0 = -INFINITY;
  for (int k = 0; k < 4; ++k) {
    double v = t - g->X[k][0];
    if (v > r0) r0 = v;
  }
  if (!(r0 > 0.0)) return 0.0;
  /* R with R^T nu_x = e3: columns e1, e2, nK */
  double nK[3] = {g->nu[1], g->nu[2], g->nu[3]};
  double nl = sqrt(dot3(nK, nK));
  for (int k = 0; k < 3; ++k) nK[k] /= nl;
  double e1[3], e2[3];
  {
    double ax[3] = {1, 0, 0};
    if (fabs(nK[0]) > 0.6) { ax[0] = 0; ax[1] = 1; }
    double p = dot3(ax, nK);
    for (int k = 0; k < 3; ++k) e1[k] = ax[k] - p * nK[k];
    double l = sqrt(dot3(e1, e1));
    for (int k = 0; k < 3; ++k) e1[k] /= l;
    e2[0] = nK[1] * e1[2] - nK[2] * e1[1];
    e2[1] = nK[2] * e1[0] - nK[0] * e1[2];
    e2[2] = nK[0] * e1[1] - nK[1] * e1[0];
  }
  double xm0[4];
  for (int c = 0; c < 4; ++c) xm0[c] = x[c] - g->X[0][c];
  double dist = dot4(xm0, g->nu); /* <x - x_sigma, nu> */
  inner_ctx C;
  C.r0 = r0;
  C.rho0 = dist / r0; /* eq. para_hypl */
  C.rhoa = fabs(C.rho0);
  C.rho0sq = C.rho0 * C.rho0;
  if (C.rhoa >= 1.0) return 0.0;
  for (int i = 0; i < 4; ++i) {
    int a = (i + 1) % 4;
    double xm[4];
    for (int c = 0; c < 4; ++c) xm[c] = x[c] - g->X[a][c];
    C.gam[i] = dot4(xm, g->cn[i]);
    C.alp[i] = r0 * g->cn[i][0];
    double cx[3] = {g->cn[i][1], g->cn[i][2], g->cn[i][3]};
    C.bx[i] = r0 * dot3(e1, cx);
    C.by[i] = r0 * dot3(e2, cx);
  }
  /* phi at which the rho-structure can change */
  double br[96];
  int nb = 0;
  double xb[3]; /* foot point of x on the panel plane */
  for (int k = 0; k < 3; ++k) xb[k] = x[k + 1] - dist * nK[k];
  /* (a) directions of the vertices' spatial positions; the lit point is
   *     y = xb - s (cos phi e1 + sin phi e2) */
  for (int v = 0; v < 4; ++v) {
    double d3[3] = {xb[0] - g->X[v][1], xb[1] - g->X[v][2], xb[2] - g->X[v][3]};
    double u = dot3(d3, e1), w = dot3(d3, e2);
    if (u * u + w * w > 1e-30) br[nb++] = wrap2pi(atan2(w, u));
  }
  /* (b) the cone meets one of the six edges */
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) {
      double dx0[3] = {x[1] - g->X[a][1], x[2] - g->X[a][2], x[3] - g->X[a][3]};
      double de[3] = {g->X[b][1] - g->X[a][1], g->X[b][2] - g->X[a][2], g->X[b][3] - g->X[a][3]};
      double dt0 = t - g->X[a][0], dte = g->X[b][0] - g->X[a][0];
      double qa = dot3(de, de) - dte * dte;
      double qb = -2.0 * (dot3(dx0, de) - dt0 * dte);
      double qc = dot3(dx0, dx0) - dt0 * dt0;
      double lam[2];
      int nl2 = 0;
      if (fabs(qa) < 1e-14 * (dot3(de, de) + dte * dte)) {
        if (qb != 0.0) lam[nl2++] = -qc / qb;
      } else {
        double disc = qb * qb - 4 * qa * qc;
        if (disc >= 0) {
          double sq = sqrt(disc);
          double q = -0.5 * (qb + (qb >= 0 ? sq : -sq));
          if (q != 0.0) { lam[nl2++] = q / qa; lam[nl2++] = qc / q; }
        }
      }
      for (int k = 0; k < nl2; ++k) {
        double l = lam[k];
        if (l < -1e-12 || l > 1 + 1e-12) continue;
        if (dt0 - l * dte < 0) continue;
        double z[3] = {g->X[a][1] + l * de[0], g->X[a][2] + l * de[1], g->X[a][3] + l * de[2]};
        double d3[3] = {xb[0] - z[0], xb[1] - z[1], xb[2] - z[2]};
        double u = dot3(d3, e1), w = dot3(d3, e2);
        if (u * u + w * w > 1e-30) br[nb++] = wrap2pi(atan2(w, u));
      }
    }
  /* (c) tangency of a face function (double root), and (d) directions where
   *     its squared equation loses its quadratic term */
  for (int i = 0; i < 4; ++i) {
    double B = sqrt(C.bx[i] * C.bx[i] + C.by[i] * C.by[i]);
    if (B <= 0.0) continue;
    double ph = atan2(C.by[i], C.bx[i]);
    double targ[2];
    int nt = 0;
    targ[nt++] = fabs(C.alp[i]);
    if (C.rho0sq > 0.0) {
      double v = C.alp[i] * C.alp[i] - C.gam[i] * C.gam[i] / C.rho0sq;
      if (v >= 0.0) targ[nt++] = sqrt(v);
    }
    for (int k = 0; k < nt; ++k) {
      double cv = targ[k] / B;
      if (cv > 1.0) continue;
      double ac = acos(cv), ac2 = acos(-cv);
      br[nb++] = wrap2pi(ph + ac);
      br[nb++] = wrap2pi(ph - ac);
      br[nb++] = wrap2pi(ph + ac2);
      br[nb++] = wrap2pi(ph - ac2);
    }
  }
  br[nb++] = 0.0;
  br[nb++] = 2.0 * ORC_PI;
  sort_small(br, nb);
  double total = 0.0;
  for (int k = 0; k + 1 < nb; ++k) {
    double a = br[k], b = br[k + 1];
    if (b - a < 1e-14) continue;
    total += piece_adaptive(&C, a, b, 0);
  }
  return r0 * total;
}

/* ------------------------------------------------------------------ */
/* Public oracle API                                                   */
/* ------------------------------------------------------------------ */

/* V 1_sigma (x), including the 1/(4 pi) of k_1. tet: [4][4] (t,x,y,z). */
double orc_inner(const double* x4, const double* tet16) {
  pthread_once(&rules_once, init_rules);
  double X[4][4];
  memcpy(X, tet16, sizeof(X));
  tet_geom g;
  tet_geometry(X, &g);
  return inner_I(x4, &g) / (4.0 * ORC_PI);
}

/* Geometry dump for tests: nu[4], cn[16], area[4], vol */
void orc_tet_geometry(const double* tet16, double* nu, double* cn, double* area, double* vol) {
  double X[4][4];
  memcpy(X, tet16, sizeof(X));
  tet_geom g;
  tet_geometry(X, &g);
  memcpy(nu, g.nu, sizeof(g.nu));
  memcpy(cn, g.cn, sizeof(g.cn));
  memcpy(area, g.area, sizeof(g.area));
  *vol = g.vol;
}

/* Reference points of the composite midpoint rule (Fig. int_tri_mid):
 * barycentric (xi1, xi2) of the m^2 sub-triangle centroids. */
int orc_midpoint_rule(int m, double* xi) {
  int n = 0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; i + j <= m - 1; ++j) {
      xi[2 * n] = (i + 1.0 / 3.0) / m;
      xi[2 * n + 1] = (j + 1.0 / 3.0) / m;
      ++n;
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; i + j <= m - 2; ++j) {
      xi[2 * n] = (i + 2.0 / 3.0) / m;
      xi[2 * n + 1] = (j + 2.0 / 3.0) / m;
      ++n;
    }
  return n;
}

typedef struct {
  int n_stv;
  const double* X;  /* [n_stv][4] */
  const int* sv;    /* [n_stv] */
  int n_tet;
  const int* tets;  /* [n_tet][4] */
} orc_mesh;

static void tet_vertices(const orc_mesh* m, int i, double X[4][4]) {
  for (int k = 0; k < 4; ++k) memcpy(X[k], m->X + 4 * m->tets[4 * i + k], 4 * sizeof(double));
}

/* The face opposite vertex k has nu_t = 0 exactly when it holds two nodes of
 * the same spatial vertex (a vertical edge); decided on ids, never on floats. */
static int face_is_vertical(const orc_mesh* m, int i, int k) {
  int ids[3], n = 0;
  for (int q = 0; q < 4; ++q)
    if (q != k) ids[n++] = m->sv[m->tets[4 * i + q]];
  return ids[0] == ids[1] || ids[0] == ids[2] || ids[1] == ids[2];
}

static double entry(const orc_mesh* m, int i, int j, int mq) {
  double Xi[4][4], Xj[4][4];
  tet_vertices(m, i, Xi);
  tet_vertices(m, j, Xj);
  tet_geom gi, gj;
  tet_geometry(Xi, &gi);
  tet_geometry(Xj, &gj);
  double xi[2 * 64];
  int nq = orc_midpoint_rule(mq, xi);
  double sum = 0.0;
  for (int k = 0; k < 4; ++k) {
    if (face_is_vertical(m, i, k)) continue;
    int a = (k + 1) % 4, b = (k + 2) % 4, c = (k + 3) % 4;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
      double x[4];
      for (int d = 0; d < 4; ++d)
        x[d] = Xi[a][d] + xi[2 * q] * (Xi[b][d] - Xi[a][d]) + xi[2 * q + 1] * (Xi[c][d] - Xi[a][d]);
      s += inner_I(x, &gj);
    }
    sum += -gi.cn[k][0] * (gi.area[k] / nq) * s;
  }
  return sum / (4.0 * ORC_PI);
}

/* Sparsity predicate; the operation order below is the contract.
 *
 * P(i,j) holds when some outer quadrature point x_q of panel i (the m_Q^2
 * sub-triangle centroids of its two faces with nu_t != 0) may see panel j on
 * its backward light cone. For one x_q the panel j is skipped when
 *   C1: tau_min(j) >= t_q                       (causality, Def. choice_r),
 *   C2: max over the vertices y_b of |x_q - y_b| - (t_q - tau_b) < 0
 *       (panel strictly inside the backward cone: the delta of the
 *        fundamental solution never meets it; the map is convex, so its
 *        maximum over the panel sits at a vertex),
 *   C3: phi_Xi(x_q - c_j) - d_r(|x_q - c_j|) > 0 for the 4D ball B_r(c_j)
 *       around the panel's vertex mean (Theorem phi_xi_sphere: the cone
 *       cannot reach the ball, as in Algorithm ApproximateLitLeaves).
 * The outer points are formed from the face vertices taken in ascending
 * spatial-vertex id, xi = (3k+1)/(3m) or (3k+2)/(3m), as
 * x = (X_a + xi1 (X_b - X_a)) + xi2 (X_c - X_a), with no fused operations. */
static double tmin4(const double X[4][4]) {
  double m = X[0][0];
  if (X[1][0] < m) m = X[1][0];
  if (X[2][0] < m) m = X[2][0];
  if (X[3][0] < m) m = X[3][0];
  return m;
}
static double dist3(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return sqrt((dx * dx + dy * dy) + dz * dz);
}

/* outer points of the nu_t != 0 faces of tet i, canonical order; returns count */
static int outer_points(const orc_mesh* m, int i, int mq, double (*xo)[4]) {
  double xi[2 * 64];
  int nq = orc_midpoint_rule(mq, xi);
  int n = 0;
  for (int k = 0; k < 4; ++k) {
    if (face_is_vertical(m, i, k)) continue;
    int v[3], s[3], c = 0;
    for (int q = 0; q < 4; ++q)
      if (q != k) { v[c] = m->tets[4 * i + q]; s[c] = m->sv[v[c]]; ++c; }
    for (int a = 1; a < 3; ++a)
      for (int b = a; b > 0 && s[b - 1] > s[b]; --b) {
        int t = s[b]; s[b] = s[b - 1]; s[b - 1] = t;
        t = v[b]; v[b] = v[b - 1]; v[b - 1] = t;
      }
    const double* A = m->X + 4 * v[0];
    const double* B = m->X + 4 * v[1];
    const double* C = m->X + 4 * v[2];
    for (int q = 0; q < nq; ++q) {
      for (int d = 0; d < 4; ++d) {
        double p = A[d] + xi[2 * q] * (B[d] - A[d]);
        xo[n][d] = p + xi[2 * q + 1] * (C[d] - A[d]);
      }
      ++n;
    }
  }
  return n;
}

static void ball4(const double X[4][4], double c[4], double* r) {
  for (int d = 0; d < 4; ++d) c[d] = (((X[0][d] + X[1][d]) + X[2][d]) + X[3][d]) / 4.0;
  double mx = 0.0;
  for (int v = 0; v < 4; ++v) {
    double a = X[v][0] - c[0], b = X[v][1] - c[1], e = X[v][2] - c[2], f = X[v][3] - c[3];
    double l = sqrt(((a * a + b * b) + e * e) + f * f);
    if (l > mx) mx = l;
  }
  *r = mx;
}

static int point_sees(const double* x, const double Xj[4][4], double tnj, const double* cj, double rj) {
  if (!(tnj < x[0])) return 0;                                   /* C1 */
  double mx = -INFINITY;
  for (int b = 0; b < 4; ++b) {
    double v = dist3(x + 1, Xj[b] + 1) - (x[0] - Xj[b][0]);
    if (v > mx) mx = v;
  }
  if (!(mx >= 0.0)) return 0;                                    /* C2 */
  double al = dist3(x + 1, cj + 1);
  double phi = al - (x[0] - cj[0]);
  double dr = (al < rj / sqrt(2.0)) ? al + sqrt(rj * rj - al * al) : rj * sqrt(2.0);
  if ((phi - dr) > 0.0) return 0;                                /* C3 */
  return 1;
}

static int pattern_mq(const orc_mesh* m, int i, int j, int mq) {
  double xo[128][4];
  int n = outer_points(m, i, mq, xo);
  double Xj[4][4], cj[4], rj;
  tet_vertices(m, j, Xj);
  ball4(Xj, cj, &rj);
  double tnj = tmin4(Xj);
  for (int q = 0; q < n; ++q)
    if (point_sees(xo[q], Xj, tnj, cj, rj)) return 1;
  return 0;
}

static int pattern(const orc_mesh* m, int i, int j) { return pattern_mq(m, i, j, 3); }

int orc_pattern_pair(int n_stv, const double* X, const int* sv, int n_tet, const int* tets, int mq, int i, int j) {
  orc_mesh m = {n_stv, X, sv, n_tet, tets};
  return pattern_mq(&m, i, j, mq);
}

/* ---------------- threaded drivers ---------------- */
typedef struct {
  const orc_mesh* m;
  int mq, npairs, use_pattern;
  const int* pairs; /* [npairs][2] */
  double* out;
  int next;
  pthread_mutex_t mu;
} entry_job;

static void* entry_worker(void* arg) {
  entry_job* J = (entry_job*)arg;
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int k = J->next;
    J->next += 8;
    pthread_mutex_unlock(&J->mu);
    if (k >= J->npairs) break;
    int e = k + 8 < J->npairs ? k + 8 : J->npairs;
    for (; k < e; ++k) {
      int i = J->pairs[2 * k], j = J->pairs[2 * k + 1];
      if (J->use_pattern && !pattern_mq(J->m, i, j, J->mq)) J->out[k] = 0.0;
      else J->out[k] = entry(J->m, i, j, J->mq);
    }
  }
  return NULL;
}

/* A_ij for a list of (i, j); use_pattern=0 evaluates every pair by the
 * definition (exact zeros must come out on their own). */
int orc_entries(int n_stv, const double* X, const int* sv, int n_tet, const int* tets, int mq,
                int npairs, const int* pairs, double* out, int use_pattern, int nthreads) {
  pthread_once(&rules_once, init_rules);
  orc_mesh m = {n_stv, X, sv, n_tet, tets};
  entry_job J;
  J.m = &m; J.mq = mq; J.npairs = npairs; J.pairs = pairs; J.out = out;
  J.use_pattern = use_pattern; J.next = 0;
  pthread_mutex_init(&J.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, entry_worker, &J);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&J.mu);
  return 0;
}

/* Dense pattern [n_tet][n_tet] as bytes */
int orc_pattern_dense(int n_stv, const double* X, const int* sv, int n_tet, const int* tets, int mq,
                      unsigned char* P) {
  orc_mesh m = {n_stv, X, sv, n_tet, tets};
  for (int i = 0; i < n_tet; ++i)
    for (int j = 0; j < n_tet; ++j) P[(size_t)i * n_tet + j] = (unsigned char)pattern_mq(&m, i, j, mq);
  return 0;
}

/* Pattern rows for a subset of test panels: for each listed row i, writes the
 * count and the admissible j (ascending) into cols (capacity cap per row). */
int orc_pattern_rows(int n_stv, const double* X, const int* sv, int n_tet, const int* tets, int mq,
                     int nrows, const int* rows, int cap, int* counts, int* cols) {
  orc_mesh m = {n_stv, X, sv, n_tet, tets};
  for (int r = 0; r < nrows; ++r) {
    int n = 0;
    for (int j = 0; j < n_tet; ++j)
      if (pattern_mq(&m, rows[r], j, mq)) {
        if (n < cap) cols[(size_t)r * cap + n] = j;
        ++n;
      }
    counts[r] = n;
  }
  return 0;
}

/* ---------------- right-hand side ---------------- */
static double data_g(int kind, const double* prm, const double* x) {
  if (kind == 0) {
    double t = x[0];
    if (!(t > 0.0 && t < 2.0)) return 0.0;
    double s = sin(0.5 * ORC_PI * t);
    return s * s;
  }
  double a = (x[0] - (x[1] * prm[0] + x[2] * prm[1] + x[3] * prm[2]) - prm[3]) / prm[4];
  return exp(-a * a);
}

/* int over the 4D face triangle (A, B, C) of g: the face is split into m^2
 * congruent sub-triangles (the same subdivision as Fig. int_tri_mid), each
 * integrated by a Duffy-collapsed 12 x 12 Gauss-Legendre rule. */
static double face_integral(const double* A, const double* B, const double* C, double area, int m, int kind,
                            const double* prm) {
  const gauss_rule* G = &G_FACE;
  double tot = 0.0;
  for (int p = 0; p < m; ++p)
    for (int q = 0; p + q < m; ++q)
      for (int down = 0; down < 2; ++down) {
        double b0[2], b1[2], b2[2]; /* (xi1, xi2) of the sub-triangle corners */
        if (!down) {
          b0[0] = (double)p / m; b0[1] = (double)q / m;
          b1[0] = (double)(p + 1) / m; b1[1] = (double)q / m;
          b2[0] = (double)p / m; b2[1] = (double)(q + 1) / m;
        } else {
          if (p + q + 2 > m) continue;
          b0[0] = (double)(p + 1) / m; b0[1] = (double)q / m;
          b1[0] = (double)(p + 1) / m; b1[1] = (double)(q + 1) / m;
          b2[0] = (double)p / m; b2[1] = (double)(q + 1) / m;
        }
        for (int a = 0; a < G->n; ++a) {
          double u = 0.5 * (G->x[a] + 1.0), wu = 0.5 * G->w[a];
          for (int c = 0; c < G->n; ++c) {
            double v = 0.5 * (G->x[c] + 1.0), wv = 0.5 * G->w[c];
            double x1 = (1.0 - u) * b0[0] + u * (1.0 - v) * b1[0] + u * v * b2[0];
            double x2 = (1.0 - u) * b0[1] + u * (1.0 - v) * b1[1] + u * v * b2[1];
            double x[4];
            for (int d = 0; d < 4; ++d) x[d] = A[d] + x1 * (B[d] - A[d]) + x2 * (C[d] - A[d]);
            tot += wu * wv * u * data_g(kind, prm, x);
          }
        }
      }
  return 2.0 * area / ((double)m * m) * tot;
}

/* b[i + n_tet*r] = -sum_F nu_{F,t} int_F g_r dS. The subdivision level makes
 * a sub-triangle span at most a quarter of the data's length scale (pulse
 * width w; 0.5 for the sin^2 data). */
int orc_rhs(int n_stv, const double* X, const int* sv, int n_tet, const int* tets, int kind,
            int nrhs, const double* params, double* b) {
  pthread_once(&rules_once, init_rules);
  orc_mesh m = {n_stv, X, sv, n_tet, tets};
  for (int i = 0; i < n_tet; ++i) {
    double Xi[4][4];
    tet_vertices(&m, i, Xi);
    tet_geom g;
    tet_geometry(Xi, &g);
    double diam = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int c = a + 1; c < 4; ++c) {
        double dd = dist3(Xi[a] + 1, Xi[c] + 1);
        if (dd > diam) diam = dd;
      }
    for (int r = 0; r < nrhs; ++r) {
      const double* prm = params ? params + 5 * r : NULL;
      double scale = kind == 1 ? 0.25 * prm[4] : 0.25;
      int msub = 1;
      while (msub < 64 && diam / msub > scale) msub *= 2;
      double sum = 0.0;
      for (int k = 0; k < 4; ++k) {
        if (face_is_vertical(&m, i, k)) continue;
        int a = (k + 1) % 4, bb = (k + 2) % 4, c = (k + 3) % 4;
        sum += -g.cn[k][0] * face_integral(Xi[a], Xi[bb], Xi[c], g.area[k], msub, kind, prm);
      }
      b[(size_t)i + (size_t)n_tet * r] = sum;
    }
  }
  return 0;
}

/* ---------------- dense LU with partial pivoting ---------------- */
/* A row-major n x n (overwritten), B [n][nrhs] row-major (overwritten by X) */
int orc_lu_solve(int n, double* A, int nrhs, double* B) {
  int* piv = (int*)malloc(sizeof(int) * n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double mx = fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; ++r)
      if (fabs(A[(size_t)r * n + k]) > mx) { mx = fabs(A[(size_t)r * n + k]); p = r; }
    piv[k] = p;
    if (mx == 0.0) { free(piv); return 1; }
    if (p != k) {
      for (int c = 0; c < n; ++c) {
        double t = A[(size_t)k * n + c]; A[(size_t)k * n + c] = A[(size_t)p * n + c]; A[(size_t)p * n + c] = t;
      }
      for (int c = 0; c < nrhs; ++c) {
        double t = B[(size_t)k * nrhs + c]; B[(size_t)k * nrhs + c] = B[(size_t)p * nrhs + c]; B[(size_t)p * nrhs + c] = t;
      }
    }
    double d = A[(size_t)k * n + k];
    for (int r = k + 1; r < n; ++r) {
      double f = A[(size_t)r * n + k] / d;
      if (f == 0.0) continue;
      A[(size_t)r * n + k] = f;
      for (int c = k + 1; c < n; ++c) A[(size_t)r * n + c] -= f * A[(size_t)k * n + c];
      for (int c = 0; c < nrhs; ++c) B[(size_t)r * nrhs + c] -= f * B[(size_t)k * nrhs + c];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int c = 0; c < nrhs; ++c) {
      double s = B[(size_t)k * nrhs + c];
      for (int q = k + 1; q < n; ++q) s -= A[(size_t)k * n + q] * B[(size_t)q * nrhs + c];
      B[(size_t)k * nrhs + c] = s / A[(size_t)k * n + k];
    }
  }
  free(piv);
  return 0;
}
