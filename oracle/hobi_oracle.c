/*
 * hobi_oracle.c -- plain, slow FP64 CPU oracle for the HOBI-PB method of
 * W. Geng, "Parallel Higher-order Boundary Integral Electrostatics
 * Computation on Molecular Surfaces with Curved Triangulation".
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path (the
 * CUDA library) never calls it, and the two share no code, headers, tables
 * or constant generators.
 *
 * Everything is IEEE double. The code follows the paper's steps in order:
 *   Sec. 2.1  well-posed equations Eqs. (8)/(9), kernels K1..K4 and
 *             sources S1,S2 (Eq. (10), Eq. (11));
 *   Sec. 2.2  cubic edge arcs, the (r,s)->(u,v) map (Eq. (14)), the 10-point
 *             cubic interpolant (Eq. (15)), the curved-element
 *             quadrature with Jacobian, the 4-point regular rule and the
 *             regular matvec terms (Eqs. (17)/(18));
 *   Sec. 2.3  the Duffy map r=(1-y)x, s=yx with 4x4 Gauss-Legendre on
 *             singular triangles (Eqs. (19)/(20));
 *   Sec. 2.5  the solvation energy (Eq. (23));
 *   GMRES     (Sec. 1 abstract; the iteration loop of the Table 1 pseudocode, Sec. 2.6).
 *
 * Readings where the paper is silent or inconsistent: eps = eps2/eps1; S1,S2
 * carry 1/eps1; the diagonal term is counted once; the regular rule is the degree-3 collapsed Gauss-Jacobi x
 * Gauss-Legendre product; the edge arc is a cubic Hermite curve whose end
 * tangents are the chord projected onto each end's tangent plane, scaled to
 * the chord length; curve normals are the normalised linear blend of the end
 * normals made orthogonal to the curve tangent; densities are interpolated
 * linearly from the three vertices (the n=1..3 sum); the target normal is
 * the input vertex normal; GMRES runs by default on the unknowns scaled by
 * the inverse diagonal coefficients (1/2)(1+eps) and (1/2)(1+1/eps) (right
 * preconditioning by that constant diagonal; the paper states none).
 *
 * Parity: pinned by the tests (quadrature exactness, shape functions,
 * kernels vs finite differences, Born/Kirkwood spheres, the kappa=0
 * double-layer identity, convergence order, brute-force quadrature, LU).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void unit3(double* a) {
  double n = norm3(a);
  a[0] /= n; a[1] /= n; a[2] /= n;
}

/* ------------------------------------------------------------------ */
/* Quadrature rules                                                    */
/* ------------------------------------------------------------------ */

/* Regular rule on the unit right triangle (Sec. 2.2, N_GR = 4).
 * The paper names a 4-point "Gauss-Radau" rule without printing it. Reading:
 * the collapsed product rule (r,s) = ((1-eta) xi, eta xi), with 2-point
 * Gauss-Jacobi in xi (weight xi on [0,1]) and 2-point Gauss-Legendre in eta.
 * Exact for all polynomials of total degree <= 3; weights sum to 1/2. */
void or_regular_rule(double r[4], double s[4], double w[4]) {
  double xi[2], wx[2], eta[2], we[2];
  xi[0] = (6.0 - sqrt(6.0)) / 10.0;
  xi[1] = (6.0 + sqrt(6.0)) / 10.0;
  wx[0] = (9.0 - sqrt(6.0)) / 36.0;
  wx[1] = (9.0 + sqrt(6.0)) / 36.0;
  eta[0] = 0.5 - 0.5 / sqrt(3.0);
  eta[1] = 0.5 + 0.5 / sqrt(3.0);
  we[0] = 0.5;
  we[1] = 0.5;
  int m = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      r[m] = (1.0 - eta[b]) * xi[a];
      s[m] = eta[b] * xi[a];
      w[m] = wx[a] * we[b];
      ++m;
    }
}

/* 4-point Gauss-Legendre rule on [0,1] (Sec. 2.3, N_GL = 4). */
void or_gauss_legendre4(double x[4], double w[4]) {
  double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)); /* inner node on [-1,1] */
  double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0)); /* outer node */
  double wa = (18.0 + sqrt(30.0)) / 36.0;
  double wb = (18.0 - sqrt(30.0)) / 36.0;
  double t[4] = {-b, -a, a, b};
  double v[4] = {wb, wa, wa, wb};
  for (int k = 0; k < 4; ++k) {
    x[k] = 0.5 * (1.0 + t[k]);
    w[k] = 0.5 * v[k];
  }
}

/* Singular rule: the 16 points of the 4x4 Gauss-Legendre tensor rule on the
 * unit square mapped by r = (1-y) x, s = y x (Sec. 2.3); the weight includes
 * the Duffy Jacobian x. The singular vertex sits at (r,s) = (0,0). */
void or_singular_rule(double r[16], double s[16], double w[16]) {
  double g[4], gw[4];
  or_gauss_legendre4(g, gw);
  int m = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double x = g[a], y = g[b];
      r[m] = (1.0 - y) * x;
      s[m] = y * x;
      w[m] = gw[a] * gw[b] * x;
      ++m;
    }
}

/* ------------------------------------------------------------------ */
/* Cubic (P3) Lagrange basis on the 10-point triangle (Eq. (15)) */
/* ------------------------------------------------------------------ */
/* Node order used throughout the oracle, by (r,s):
 *  0:(0,0)=X1  1:(1,0)=X2  2:(0,1)=X3
 *  3:(1/3,0)   4:(2/3,0)          on edge X1X2
 *  5:(0,1/3)   6:(0,2/3)          on edge X1X3
 *  7:(2/3,1/3) 8:(1/3,2/3)        on edge X2X3
 *  9:(1/3,1/3)                    interior
 * Barycentrics L1 = 1-r-s, L2 = r, L3 = s. */
void or_p3_basis(double r, double s, double N[10], double Nr[10], double Ns[10]) {
  double L[3] = {1.0 - r - s, r, s};
  double dLr[3] = {-1.0, 1.0, 0.0};
  double dLs[3] = {-1.0, 0.0, 1.0};
  /* vertex k: (1/2) L (3L-1)(3L-2) */
  for (int k = 0; k < 3; ++k) {
    double l = L[k];
    double f = 0.5 * l * (3.0 * l - 1.0) * (3.0 * l - 2.0);
    double df = 0.5 * ((3.0 * l - 1.0) * (3.0 * l - 2.0) + 3.0 * l * (3.0 * l - 2.0) + 3.0 * l * (3.0 * l - 1.0));
    N[k] = f;
    Nr[k] = df * dLr[k];
    Ns[k] = df * dLs[k];
  }
  /* edge node nearer vertex i on edge (i,j): (9/2) Li Lj (3 Li - 1) */
  int ei[6] = {0, 1, 0, 2, 1, 2};
  int ej[6] = {1, 0, 2, 0, 2, 1};
  for (int e = 0; e < 6; ++e) {
    int i = ei[e], j = ej[e];
    double li = L[i], lj = L[j];
    double f = 4.5 * li * lj * (3.0 * li - 1.0);
    double dfi = 4.5 * lj * (6.0 * li - 1.0); /* d/dLi */
    double dfj = 4.5 * li * (3.0 * li - 1.0); /* d/dLj */
    N[3 + e] = f;
    Nr[3 + e] = dfi * dLr[i] + dfj * dLr[j];
    Ns[3 + e] = dfi * dLs[i] + dfj * dLs[j];
  }
  /* interior: 27 L1 L2 L3 */
  N[9] = 27.0 * L[0] * L[1] * L[2];
  Nr[9] = 27.0 * (dLr[0] * L[1] * L[2] + L[0] * dLr[1] * L[2] + L[0] * L[1] * dLr[2]);
  Ns[9] = 27.0 * (dLs[0] * L[1] * L[2] + L[0] * dLs[1] * L[2] + L[0] * L[1] * dLs[2]);
}

/* ------------------------------------------------------------------ */
/* Curved edge arc between two nodes with normals (Sec. 2.2)          */
/* ------------------------------------------------------------------ */
/* x(t) = c0 + c1 t + c2 t^2 + c3 t^3 fixed by 12 conditions: the two end
 * positions (6) and the two end tangents (6). Reading: each end tangent is
 * the chord projected onto that end's tangent plane, normalised and scaled
 * by the chord length (cubic Hermite form). The normal along the arc is the
 * linear blend of the end normals made orthogonal to the arc tangent and
 * normalised (the paper's curvature rule is undefined on straight arcs). */
void or_edge_arc(const double* P, const double* nP, const double* Q, const double* nQ, double t,
                 double* x, double* n) {
  double e[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
  double L = norm3(e);
  double tp[3], tq[3];
  double ep = dot3(e, nP), eq = dot3(e, nQ);
  for (int k = 0; k < 3; ++k) {
    tp[k] = e[k] - ep * nP[k];
    tq[k] = e[k] - eq * nQ[k];
  }
  unit3(tp);
  unit3(tq);
  /* Hermite coefficients c0..c3 from x(0)=P, x(1)=Q, x'(0)=L tp, x'(1)=L tq */
  double c0[3], c1[3], c2[3], c3[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = P[k];
    c1[k] = L * tp[k];
    c2[k] = 3.0 * (Q[k] - P[k]) - 2.0 * L * tp[k] - L * tq[k];
    c3[k] = 2.0 * (P[k] - Q[k]) + L * tp[k] + L * tq[k];
  }
  double dx[3];
  for (int k = 0; k < 3; ++k) {
    x[k] = c0[k] + t * (c1[k] + t * (c2[k] + t * c3[k]));
    dx[k] = c1[k] + t * (2.0 * c2[k] + 3.0 * t * c3[k]);
  }
  unit3(dx);
  double w[3];
  for (int k = 0; k < 3; ++k) w[k] = (1.0 - t) * nP[k] + t * nQ[k];
  double wt = dot3(w, dx);
  for (int k = 0; k < 3; ++k) n[k] = w[k] - wt * dx[k];
  unit3(n);
}

/* The 10 interpolation points of one curved element (Sec. 2.2, the 10-point construction):
 * vertices, two points on each edge arc at t = 1/3, 2/3, and the interior
 * point (r,s) = (1/3,1/3), i.e. (u,v) = (2/3,1/2) by Eq. (14): the arc from
 * Y1 = arc X1X2 at u to Y2 = arc X1X3 at u, evaluated at v. */
void or_element_points(const double* X1, const double* n1, const double* X2, const double* n2,
                       const double* X3, const double* n3, double pts[10][3]) {
  double nn[3];
  memcpy(pts[0], X1, 3 * sizeof(double));
  memcpy(pts[1], X2, 3 * sizeof(double));
  memcpy(pts[2], X3, 3 * sizeof(double));
  or_edge_arc(X1, n1, X2, n2, 1.0 / 3.0, pts[3], nn);
  or_edge_arc(X1, n1, X2, n2, 2.0 / 3.0, pts[4], nn);
  or_edge_arc(X1, n1, X3, n3, 1.0 / 3.0, pts[5], nn);
  or_edge_arc(X1, n1, X3, n3, 2.0 / 3.0, pts[6], nn);
  or_edge_arc(X2, n2, X3, n3, 1.0 / 3.0, pts[7], nn);
  or_edge_arc(X2, n2, X3, n3, 2.0 / 3.0, pts[8], nn);
  double u = 2.0 / 3.0, v = 0.5;
  double Y1[3], m1[3], Y2[3], m2[3];
  or_edge_arc(X1, n1, X2, n2, u, Y1, m1);
  or_edge_arc(X1, n1, X3, n3, u, Y2, m2);
  or_edge_arc(Y1, m1, Y2, m2, v, pts[9], nn);
}

/* Point, unit normal and area Jacobian |x_r x x_s| of the interpolated curved
 * element at (r,s) (Eq. (15) and the curved-element quadrature rule). */
void or_element_eval(const double pts[10][3], double r, double s, double* x, double* nu, double* J) {
  double N[10], Nr[10], Ns[10];
  or_p3_basis(r, s, N, Nr, Ns);
  double xr[3] = {0, 0, 0}, xs[3] = {0, 0, 0};
  x[0] = x[1] = x[2] = 0.0;
  for (int k = 0; k < 10; ++k)
    for (int c = 0; c < 3; ++c) {
      x[c] += N[k] * pts[k][c];
      xr[c] += Nr[k] * pts[k][c];
      xs[c] += Ns[k] * pts[k][c];
    }
  cross3(xr, xs, nu);
  *J = norm3(nu);
  nu[0] /= *J; nu[1] /= *J; nu[2] /= *J;
}

/* ------------------------------------------------------------------ */
/* Kernels (Eq. (10))                                                     */
/* ------------------------------------------------------------------ */
/* K1..K4 at target x (normal nx) and source y (normal ny):
 *   K1 = G0 - Gk,                 K2 = eps dGk/dny - dG0/dny,
 *   K3 = dG0/dnx - dGk/dnx / eps,  K4 = d2Gk/dnxdny - d2G0/dnxdny,
 * with G0 = 1/(4 pi r), Gk = exp(-kappa r)/(4 pi r), written out through the
 * derivatives of G(r) (d = x - y, r = |d|):
 *   dG/dny = -G'(r) (d.ny)/r ... in closed form below. */
void or_kernels(const double* x, const double* nx, const double* y, const double* ny, double eps,
                double kappa, double K[4]) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r = norm3(d);
  double ax = dot3(d, nx), ay = dot3(d, ny), c = dot3(nx, ny);
  double E = exp(-kappa * r);
  double G0 = 1.0 / (4.0 * OR_PI * r);
  double Gk = E / (4.0 * OR_PI * r);
  /* first derivatives: dG0/dny = ay/(4 pi r^3), dG0/dnx = -ax/(4 pi r^3),
   * dGk/dny = E(1+kr) ay/(4 pi r^3), dGk/dnx = -E(1+kr) ax/(4 pi r^3) */
  double r3 = r * r * r, r5 = r3 * r * r;
  double dG0_dny = ay / (4.0 * OR_PI * r3);
  double dG0_dnx = -ax / (4.0 * OR_PI * r3);
  double dGk_dny = E * (1.0 + kappa * r) * ay / (4.0 * OR_PI * r3);
  double dGk_dnx = -E * (1.0 + kappa * r) * ax / (4.0 * OR_PI * r3);
  /* second mixed derivatives:
   * d2G0 = [c/r^3 - 3 ax ay/r^5]/(4 pi),
   * d2Gk = [E(1+kr) c/r^3 - E(3+3kr+k^2 r^2) ax ay/r^5]/(4 pi) */
  double d2G0 = (c / r3 - 3.0 * ax * ay / r5) / (4.0 * OR_PI);
  double d2Gk = (E * (1.0 + kappa * r) * c / r3 -
                 E * (3.0 + 3.0 * kappa * r + kappa * kappa * r * r) * ax * ay / r5) /
                (4.0 * OR_PI);
  K[0] = G0 - Gk;
  K[1] = eps * dGk_dny - dG0_dny;
  K[2] = dG0_dnx - dGk_dnx / eps;
  K[3] = d2Gk - d2G0;
}

/* Free-space Green's functions, exported so the tests can difference them. */
double or_G(double x0, double x1, double x2, double y0, double y1, double y2, double kappa) {
  double d[3] = {x0 - y0, x1 - y1, x2 - y2};
  double r = norm3(d);
  return exp(-kappa * r) / (4.0 * OR_PI * r);
}

/* ------------------------------------------------------------------ */
/* Problem context                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t nv, nf, nc;
  double* V;   /* nv*3 */
  double* Nv;  /* nv*3 unit vertex normals */
  int32_t* F;  /* nf*3 */
  double* Qc;  /* nc*4 */
  double eps1, eps2, kappa, eps;
  double* pts; /* nf*10*3 element interpolation points */
  /* regular rule tables: node y, unit normal, W_{j,m,n} = w_m J_m L_n(r_m,s_m) */
  double* gy;  /* nf*4*3 */
  double* gn;  /* nf*4*3 */
  double* gW;  /* nf*4*3 */
} or_ctx;

/* Build the curved elements and the regular-rule tables (routines (2), (3) of
 * Sec. 2.6). Input normals are normalised here (reading: the target normal is
 * the input vertex normal). */
or_ctx* or_create(const double* V, int64_t nv, const int32_t* F, int64_t nf, const double* Nrm,
                  const double* Qc, int64_t nc, double eps1, double eps2, double kappa) {
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->nv = nv; c->nf = nf; c->nc = nc;
  c->eps1 = eps1; c->eps2 = eps2; c->kappa = kappa;
  c->eps = eps2 / eps1; /* reading: eps = eps2/eps1 makes Eqs. (8)/(9) consistent */
  c->V = (double*)malloc(sizeof(double) * 3 * nv);
  c->Nv = (double*)malloc(sizeof(double) * 3 * nv);
  c->F = (int32_t*)malloc(sizeof(int32_t) * 3 * nf);
  c->Qc = (double*)malloc(sizeof(double) * 4 * (nc > 0 ? nc : 1));
  memcpy(c->V, V, sizeof(double) * 3 * nv);
  memcpy(c->F, F, sizeof(int32_t) * 3 * nf);
  if (nc > 0) memcpy(c->Qc, Qc, sizeof(double) * 4 * nc);
  for (int64_t i = 0; i < nv; ++i) {
    double n[3] = {Nrm[3 * i], Nrm[3 * i + 1], Nrm[3 * i + 2]};
    unit3(n);
    memcpy(&c->Nv[3 * i], n, sizeof n);
  }
  c->pts = (double*)malloc(sizeof(double) * 30 * nf);
  c->gy = (double*)malloc(sizeof(double) * 12 * nf);
  c->gn = (double*)malloc(sizeof(double) * 12 * nf);
  c->gW = (double*)malloc(sizeof(double) * 12 * nf);
  double rr[4], ss[4], ww[4];
  or_regular_rule(rr, ss, ww);
  for (int64_t j = 0; j < nf; ++j) {
    int a = F[3 * j], b = F[3 * j + 1], d = F[3 * j + 2];
    double(*P)[3] = (double(*)[3])(c->pts + 30 * j);
    or_element_points(&c->V[3 * a], &c->Nv[3 * a], &c->V[3 * b], &c->Nv[3 * b], &c->V[3 * d],
                      &c->Nv[3 * d], P);
    for (int m = 0; m < 4; ++m) {
      double x[3], nu[3], J;
      or_element_eval((const double(*)[3])P, rr[m], ss[m], x, nu, &J);
      double L[3] = {1.0 - rr[m] - ss[m], rr[m], ss[m]};
      for (int k = 0; k < 3; ++k) {
        c->gy[12 * j + 3 * m + k] = x[k];
        c->gn[12 * j + 3 * m + k] = nu[k];
        c->gW[12 * j + 3 * m + k] = ww[m] * J * L[k];
      }
    }
  }
  return c;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->V); free(c->Nv); free(c->F); free(c->Qc);
  free(c->pts); free(c->gy); free(c->gn); free(c->gW);
  free(c);
}

/* Export the regular-rule node table: y[nf*4*3], nu[nf*4*3], W[nf*4*3]. */
void or_get_nodes(const or_ctx* c, double* y, double* nu, double* W) {
  memcpy(y, c->gy, sizeof(double) * 12 * c->nf);
  memcpy(nu, c->gn, sizeof(double) * 12 * c->nf);
  memcpy(W, c->gW, sizeof(double) * 12 * c->nf);
}

void or_get_element_points(const or_ctx* c, double* pts) { memcpy(pts, c->pts, sizeof(double) * 30 * c->nf); }

/* Singular-triangle contribution to rows i and i+N_v from face j, of which
 * vertex i is a corner (Sec. 2.3, Eqs. (19)/(20)). The element keeps its
 * geometry in stored vertex order; the singular rule's (r',s') frame puts
 * vertex i at the origin through a cyclic relabelling of the barycentrics.
 * Returns the 2x2 coefficient blocks acting on (u_{N_v+v}, u_v) for the
 * three corners v = F[j][0..2]:
 *   out[n][0] = sum W K1, out[n][1] = sum W K2, out[n][2] = sum W K3, out[n][3] = sum W K4. */
static void singular_face_coeffs(const or_ctx* c, int64_t i, int64_t j, const double* rs_r,
                                 const double* rs_s, const double* rs_w, int nq, double out[3][4]) {
  const int32_t* f = &c->F[3 * j];
  int k = (f[0] == i) ? 0 : (f[1] == i) ? 1 : 2;
  const double(*P)[3] = (const double(*)[3])(c->pts + 30 * j);
  memset(out, 0, sizeof(double) * 12);
  for (int m = 0; m < nq; ++m) {
    double Lp[3] = {1.0 - rs_r[m] - rs_s[m], rs_r[m], rs_s[m]}; /* vertex i first */
    double L[3];
    L[k] = Lp[0];
    L[(k + 1) % 3] = Lp[1];
    L[(k + 2) % 3] = Lp[2];
    double x[3], nu[3], J, K[4];
    or_element_eval(P, L[1], L[2], x, nu, &J);
    or_kernels(&c->V[3 * i], &c->Nv[3 * i], x, nu, c->eps, c->kappa, K);
    for (int n = 0; n < 3; ++n)
      for (int q = 0; q < 4; ++q) out[n][q] += rs_w[m] * J * L[n] * K[q];
  }
}

/* Exported: singular coefficients of one (vertex, incident face) pair with the
 * paper's 16-point rule (used by the brute-force tests). */
int or_singular_coeffs(const or_ctx* c, int64_t i, int64_t j, double* out12) {
  const int32_t* f = &c->F[3 * j];
  if (f[0] != i && f[1] != i && f[2] != i) return -1;
  double r[16], s[16], w[16];
  or_singular_rule(r, s, w);
  singular_face_coeffs(c, i, j, r, s, w, 16, (double(*)[4])out12);
  return 0;
}

/* Same with an n x n Gauss-Legendre product rule under the Duffy map (n<=64),
 * for brute-force convergence checks of the singular integrals. */
int or_singular_coeffs_n(const or_ctx* c, int64_t i, int64_t j, int ngl, const double* gx,
                         const double* gw, double* out12) {
  const int32_t* f = &c->F[3 * j];
  if (f[0] != i && f[1] != i && f[2] != i) return -1;
  int nq = ngl * ngl;
  double* r = (double*)malloc(sizeof(double) * nq * 3);
  double *s = r + nq, *w = r + 2 * nq;
  int m = 0;
  for (int a = 0; a < ngl; ++a)
    for (int b = 0; b < ngl; ++b) {
      r[m] = (1.0 - gx[b]) * gx[a];
      s[m] = gx[b] * gx[a];
      w[m] = gw[a] * gw[b] * gx[a];
      ++m;
    }
  singular_face_coeffs(c, i, j, r, s, w, nq, (double(*)[4])out12);
  free(r);
  return 0;
}

/* One row pair of the matvec {Au}_i, {Au}_{i+N_v} (Eqs. (17)-(20), the
 * diagonal term counted once): regular faces with the 4-point rule, the
 * faces having vertex i as a corner with the 16-point singular rule. */
static void matvec_row(const or_ctx* c, const double* u, int64_t i, const double* sr, const double* ss,
                       const double* sw, double* out1, double* out2) {
  const int64_t nv = c->nv;
  double s1 = 0.0, s2 = 0.0;
  const double* x = &c->V[3 * i];
  const double* nx = &c->Nv[3 * i];
  for (int64_t j = 0; j < c->nf; ++j) {
    const int32_t* f = &c->F[3 * j];
    if (f[0] == i || f[1] == i || f[2] == i) {
      double cf[3][4];
      singular_face_coeffs(c, i, j, sr, ss, sw, 16, cf);
      for (int n = 0; n < 3; ++n) {
        double dphi = u[nv + f[n]], phi = u[f[n]];
        s1 += cf[n][0] * dphi + cf[n][1] * phi;
        s2 += cf[n][2] * dphi + cf[n][3] * phi;
      }
    } else {
      for (int m = 0; m < 4; ++m) {
        double K[4];
        or_kernels(x, nx, &c->gy[12 * j + 3 * m], &c->gn[12 * j + 3 * m], c->eps, c->kappa, K);
        for (int n = 0; n < 3; ++n) {
          double W = c->gW[12 * j + 3 * m + n];
          double dphi = u[nv + f[n]], phi = u[f[n]];
          s1 += W * (K[0] * dphi + K[1] * phi);
          s2 += W * (K[2] * dphi + K[3] * phi);
        }
      }
    }
  }
  *out1 = 0.5 * (1.0 + c->eps) * u[i] - s1;
  *out2 = 0.5 * (1.0 + 1.0 / c->eps) * u[nv + i] - s2;
}

/* Full matvec Au (length 2 N_v), rows computed independently (routine (5)). */
void or_matvec(const or_ctx* c, const double* u, double* Au) {
  double sr[16], ss[16], sw[16];
  or_singular_rule(sr, ss, sw);
  const int64_t nv = c->nv;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nv; ++i) matvec_row(c, u, i, sr, ss, sw, &Au[i], &Au[nv + i]);
}

/* Selected rows only: out[2k] = {Au}_{rows[k]}, out[2k+1] = {Au}_{rows[k]+N_v}. */
void or_matvec_rows(const or_ctx* c, const double* u, const int64_t* rows, int64_t nrows, double* out) {
  double sr[16], ss[16], sw[16];
  or_singular_rule(sr, ss, sw);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nrows; ++k) matvec_row(c, u, rows[k], sr, ss, sw, &out[2 * k], &out[2 * k + 1]);
}

/* Right-hand side b = [S1; S2] at the vertices (Eq. (11), routine (1)), with the
 * 1/eps1 factor of the charge potential in Omega_1 (reading). */
void or_rhs(const or_ctx* c, double* b) {
  const int64_t nv = c->nv;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nv; ++i) {
    const double* x = &c->V[3 * i];
    const double* nx = &c->Nv[3 * i];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < c->nc; ++k) {
      const double* q = &c->Qc[4 * k];
      double d[3] = {x[0] - q[0], x[1] - q[1], x[2] - q[2]};
      double r = norm3(d);
      s1 += q[3] / (4.0 * OR_PI * c->eps1 * r);
      s2 += -q[3] * dot3(d, nx) / (4.0 * OR_PI * c->eps1 * r * r * r);
    }
    b[i] = s1;
    b[nv + i] = s2;
  }
}

/* Reaction potential at the charge sites, phi_reac(x_k) = integral of
 * K1 dphi/dnu + K2 phi with the regular rule over every face
 * (Eq. (23), routine (6)). */
void or_reaction_potential(const or_ctx* c, const double* u, const double* pts, int64_t np, double* phi) {
  const int64_t nv = c->nv;
  double unused_nx[3] = {0.0, 0.0, 1.0}; /* K1, K2 do not use the target normal */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < np; ++k) {
    double s = 0.0;
    for (int64_t j = 0; j < c->nf; ++j) {
      const int32_t* f = &c->F[3 * j];
      for (int m = 0; m < 4; ++m) {
        double K[4];
        or_kernels(&pts[3 * k], unused_nx, &c->gy[12 * j + 3 * m], &c->gn[12 * j + 3 * m], c->eps, c->kappa, K);
        for (int n = 0; n < 3; ++n)
          s += c->gW[12 * j + 3 * m + n] * (K[0] * u[nv + f[n]] + K[1] * u[f[n]]);
      }
    }
    phi[k] = s;
  }
}

/* Reaction field -grad_x phi_reac at points x (the gradient of the Sec. 2.5 reaction potential
 * with respect to the point, same regular rule): with d = x - y, r = |d|, a = d.ny,
 *   grad G0 = -d/(4 pi r^3),  grad Gk = -E(1 + kr) d/(4 pi r^3),
 *   grad dG0/dny = [ny - 3 a d/r^2]/(4 pi r^3),
 *   grad dGk/dny = [E(1 + kr) ny - kappa^2 E a d - 3 E(1 + kr) a d/r^2]/(4 pi r^3)
 * (d/dr of E(1 + kr) is -kappa^2 r E), so grad K1 = grad G0 - grad Gk and
 * grad K2 = eps grad dGk/dny - grad dG0/dny. field[3k + c] for point k, component c. */
static void or_kernel_grads(const double* x, const double* y, const double* ny, double eps, double kappa,
                            double g1[3], double g2[3]) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r = norm3(d);
  double a = dot3(d, ny);
  double E = exp(-kappa * r);
  double P = E * (1.0 + kappa * r);
  double r3 = r * r * r;
  for (int c = 0; c < 3; ++c) {
    double gG0 = -d[c] / (4.0 * OR_PI * r3);
    double gGk = -P * d[c] / (4.0 * OR_PI * r3);
    double gdG0 = (ny[c] - 3.0 * a * d[c] / (r * r)) / (4.0 * OR_PI * r3);
    double gdGk = (P * ny[c] - kappa * kappa * E * a * d[c] - 3.0 * P * a * d[c] / (r * r)) / (4.0 * OR_PI * r3);
    g1[c] = gG0 - gGk;
    g2[c] = eps * gdGk - gdG0;
  }
}

void or_reaction_field(const or_ctx* c, const double* u, const double* pts, int64_t np, double* field) {
  const int64_t nv = c->nv;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < np; ++k) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < c->nf; ++j) {
      const int32_t* f = &c->F[3 * j];
      for (int m = 0; m < 4; ++m) {
        double g1[3], g2[3];
        or_kernel_grads(&pts[3 * k], &c->gy[12 * j + 3 * m], &c->gn[12 * j + 3 * m], c->eps, c->kappa, g1, g2);
        for (int n = 0; n < 3; ++n) {
          const double w = c->gW[12 * j + 3 * m + n];
          for (int q = 0; q < 3; ++q) s[q] += w * (g1[q] * u[nv + f[n]] + g2[q] * u[f[n]]);
        }
      }
    }
    for (int q = 0; q < 3; ++q) field[3 * k + q] = -s[q];
  }
}

/* E_sol in kcal/mol: (1/2) sum_k q_k phi_reac(x_k), with phi in the G-units
 * of the formulation converted by 4 pi C, C = 332.0716 kcal A/(mol e^2). */
double or_energy(const or_ctx* c, const double* u) {
  if (c->nc == 0) return 0.0;
  double* pts = (double*)malloc(sizeof(double) * 3 * c->nc);
  double* phi = (double*)malloc(sizeof(double) * c->nc);
  for (int64_t k = 0; k < c->nc; ++k)
    for (int d = 0; d < 3; ++d) pts[3 * k + d] = c->Qc[4 * k + d];
  or_reaction_potential(c, u, pts, c->nc, phi);
  double e = 0.0;
  for (int64_t k = 0; k < c->nc; ++k) e += c->Qc[4 * k + 3] * phi[k];
  free(pts);
  free(phi);
  return 0.5 * 4.0 * OR_PI * 332.0716 * e;
}

/* ------------------------------------------------------------------ */
/* GMRES (restarted, modified Gram-Schmidt, Givens rotations)          */
/* ------------------------------------------------------------------ */
/* Solves A x = b (n unknowns, A applied by op) from x0 = 0; stops when
 * ||b - A x||_2 / ||b||_2 <= tol (the Givens residual estimate) or after max_it
 * matvecs. Returns the iteration count; resid[k] (if non-NULL, length max_it+1)
 * holds the relative residual estimate after k iterations.
 * dscale (NULL: none): GMRES runs on A D x' = b with x = D x', D = diag(dscale), i.e.
 * each Arnoldi step applies A to D v and the update is x += D (V y); the residual and the
 * stopping test stay those of A x = b (reading: the unknowns scaled by the inverse of the
 * diagonal coefficients of Eqs. (17)-(20)). */
typedef void (*or_operator)(const or_ctx* c, const double* u, double* Au);

static int gmres_core(const or_ctx* c, or_operator op, int64_t n, const double* b, double tol, int max_it,
                      int restart, const double* dscale, double* x, double* resid, int* converged) {
  int m = restart;
  double* Vb = (double*)malloc(sizeof(double) * n * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* w = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * m);
  double* z = (double*)malloc(sizeof(double) * n);
  double bnorm = 0.0;
  for (int64_t i = 0; i < n; ++i) bnorm += b[i] * b[i];
  bnorm = sqrt(bnorm);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  int it = 0;
  *converged = 0;
  if (resid) resid[0] = 1.0;
  if (bnorm == 0.0) { *converged = 1; goto done; }
  while (it < max_it) {
    /* r = b - A x */
    op(c, x, w);
    double beta = 0.0;
    for (int64_t i = 0; i < n; ++i) { w[i] = b[i] - w[i]; beta += w[i] * w[i]; }
    beta = sqrt(beta);
    if (beta / bnorm <= tol) { *converged = 1; break; }
    for (int64_t i = 0; i < n; ++i) Vb[i] = w[i] / beta;
    memset(g, 0, sizeof(double) * (m + 1));
    g[0] = beta;
    int k;
    for (k = 0; k < m && it < max_it; ++k) {
      if (dscale) {
        for (int64_t i = 0; i < n; ++i) z[i] = dscale[i] * Vb[n * k + i];
        op(c, z, w);
      } else {
        op(c, &Vb[n * k], w);
      }
      ++it;
      for (int jj = 0; jj <= k; ++jj) {
        double h = 0.0;
        for (int64_t i = 0; i < n; ++i) h += Vb[n * jj + i] * w[i];
        H[jj * m + k] = h;
        for (int64_t i = 0; i < n; ++i) w[i] -= h * Vb[n * jj + i];
      }
      double hn = 0.0;
      for (int64_t i = 0; i < n; ++i) hn += w[i] * w[i];
      hn = sqrt(hn);
      H[(k + 1) * m + k] = hn;
      for (int jj = 0; jj < k; ++jj) {
        double t0 = cs[jj] * H[jj * m + k] + sn[jj] * H[(jj + 1) * m + k];
        double t1 = -sn[jj] * H[jj * m + k] + cs[jj] * H[(jj + 1) * m + k];
        H[jj * m + k] = t0;
        H[(jj + 1) * m + k] = t1;
      }
      double a = H[k * m + k], bb = H[(k + 1) * m + k];
      double den = sqrt(a * a + bb * bb);
      cs[k] = a / den;
      sn[k] = bb / den;
      H[k * m + k] = den;
      H[(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      double rel = fabs(g[k + 1]) / bnorm;
      if (resid) resid[it] = rel;
      if (hn != 0.0)
        for (int64_t i = 0; i < n; ++i) Vb[n * (k + 1) + i] = w[i] / hn;
      if (rel <= tol || hn == 0.0) { ++k; *converged = (rel <= tol); break; }
    }
    /* back-substitution and update x += V y */
    for (int ii = k - 1; ii >= 0; --ii) {
      double t = g[ii];
      for (int jj = ii + 1; jj < k; ++jj) t -= H[ii * m + jj] * y[jj];
      y[ii] = t / H[ii * m + ii];
    }
    if (dscale) {
      for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int jj = 0; jj < k; ++jj) t += y[jj] * Vb[n * jj + i];
        x[i] += dscale[i] * t;
      }
    } else {
      for (int jj = 0; jj < k; ++jj)
        for (int64_t i = 0; i < n; ++i) x[i] += y[jj] * Vb[n * jj + i];
    }
    if (*converged) break;
  }
done:
  free(Vb); free(H); free(cs); free(sn); free(g); free(w); free(y); free(z);
  return it;
}

/* The inverse diagonal coefficients of the two row blocks of Eqs. (17)-(20) (and (21)-(22)):
 * 1 / ((1/2)(1 + eps)) for the first half of the unknowns, 1 / ((1/2)(1 + 1/eps)) for the second. */
static double* diag_scale(const or_ctx* c, int64_t n) {
  double* d = (double*)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) d[i] = i < n / 2 ? 1.0 / (0.5 * (1.0 + c->eps)) : 1.0 / (0.5 * (1.0 + 1.0 / c->eps));
  return d;
}

int or_gmres(const or_ctx* c, const double* b, double tol, int max_it, int restart, int scaled, double* x,
             double* resid, int* converged) {
  const int64_t n = 2 * c->nv;
  double* d = scaled ? diag_scale(c, n) : NULL;
  int it = gmres_core(c, or_matvec, n, b, tol, max_it, restart, d, x, resid, converged);
  free(d);
  return it;
}

/* ------------------------------------------------------------------ */
/* Low-order scheme, LOBI-PB (Sec. 2.4, Eqs. (21)/(22))               */
/* ------------------------------------------------------------------ */
/* Flat triangles with centroid collocation: unknowns are phi and dphi/dnu at the
 * N_f centroids, each triangle contributes W_j = its area times the kernels at its
 * centroid, and the singular (self) triangle j = i is dropped. Normals are the flat
 * face normals. */
static void lobi_face(const or_ctx* c, int64_t j, double* x, double* n, double* A) {
  const int32_t* f = &c->F[3 * j];
  const double *a = &c->V[3 * f[0]], *b = &c->V[3 * f[1]], *d = &c->V[3 * f[2]];
  double e1[3], e2[3];
  for (int k = 0; k < 3; ++k) {
    x[k] = (a[k] + b[k] + d[k]) / 3.0;
    e1[k] = b[k] - a[k];
    e2[k] = d[k] - a[k];
  }
  cross3(e1, e2, n);
  double len = norm3(n);
  *A = 0.5 * len;
  n[0] /= len; n[1] /= len; n[2] /= len;
}

void or_lobi_geometry(const or_ctx* c, double* x, double* n, double* A) {
  for (int64_t j = 0; j < c->nf; ++j) lobi_face(c, j, &x[3 * j], &n[3 * j], &A[j]);
}

static void lobi_row(const or_ctx* c, const double* u, int64_t i, double* out1, double* out2) {
  const int64_t nf = c->nf;
  double xi[3], ni[3], Ai;
  lobi_face(c, i, xi, ni, &Ai);
  double s1 = 0.0, s2 = 0.0;
  for (int64_t j = 0; j < nf; ++j) {
    if (j == i) continue; /* the singular triangle is removed */
    double xj[3], nj[3], Aj, K[4];
    lobi_face(c, j, xj, nj, &Aj);
    or_kernels(xi, ni, xj, nj, c->eps, c->kappa, K);
    s1 += Aj * (K[0] * u[nf + j] + K[1] * u[j]);
    s2 += Aj * (K[2] * u[nf + j] + K[3] * u[j]);
  }
  *out1 = 0.5 * (1.0 + c->eps) * u[i] - s1;
  *out2 = 0.5 * (1.0 + 1.0 / c->eps) * u[nf + i] - s2;
}

void or_lobi_matvec(const or_ctx* c, const double* u, double* Au) {
  const int64_t nf = c->nf;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nf; ++i) lobi_row(c, u, i, &Au[i], &Au[nf + i]);
}

void or_lobi_matvec_rows(const or_ctx* c, const double* u, const int64_t* rows, int64_t nrows, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nrows; ++k) lobi_row(c, u, rows[k], &out[2 * k], &out[2 * k + 1]);
}

/* Sources S1, S2 (Eq. (11), with 1/eps1) at the centroids, face normals. */
void or_lobi_rhs(const or_ctx* c, double* b) {
  const int64_t nf = c->nf;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nf; ++i) {
    double x[3], nx[3], A;
    lobi_face(c, i, x, nx, &A);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < c->nc; ++k) {
      const double* q = &c->Qc[4 * k];
      double d[3] = {x[0] - q[0], x[1] - q[1], x[2] - q[2]};
      double r = norm3(d);
      s1 += q[3] / (4.0 * OR_PI * c->eps1 * r);
      s2 += -q[3] * dot3(d, nx) / (4.0 * OR_PI * c->eps1 * r * r * r);
    }
    b[i] = s1;
    b[nf + i] = s2;
  }
}

/* E_sol (kcal/mol) with the centroid rule for the reaction potential (Eq. (23)). */
double or_lobi_energy(const or_ctx* c, const double* u) {
  const int64_t nf = c->nf;
  double unused_nx[3] = {0.0, 0.0, 1.0}; /* K1, K2 do not use the target normal */
  double e = 0.0;
  for (int64_t k = 0; k < c->nc; ++k) {
    const double* q = &c->Qc[4 * k];
    double phi = 0.0;
    for (int64_t j = 0; j < nf; ++j) {
      double xj[3], nj[3], Aj, K[4];
      lobi_face(c, j, xj, nj, &Aj);
      or_kernels(q, unused_nx, xj, nj, c->eps, c->kappa, K);
      phi += Aj * (K[0] * u[nf + j] + K[1] * u[j]);
    }
    e += q[3] * phi;
  }
  return 0.5 * 4.0 * OR_PI * 332.0716 * e;
}

int or_lobi_gmres(const or_ctx* c, const double* b, double tol, int max_it, int restart, int scaled, double* x,
                  double* resid, int* converged) {
  const int64_t n = 2 * c->nf;
  double* d = scaled ? diag_scale(c, n) : NULL;
  int it = gmres_core(c, or_lobi_matvec, n, b, tol, max_it, restart, d, x, resid, converged);
  free(d);
  return it;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
