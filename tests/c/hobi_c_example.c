/* A C program using the library through include/hobi.h only: plain host pointers, no Python.
 * Builds a sphere (octahedron refined `level` times, vertices projected to radius R, exact radial
 * normals), puts a +1 e charge at the centre, solves in both precisions and prints the
 * solvation energy next to the Born value -C/2 (1/eps1 - 1/eps2) q^2 / R (Sec. 3.2, Table 2).
 * Usage: hobi_c_example [level] [radius]; exit status 0 when both solves converge. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "hobi.h"

typedef struct {
  double* v;
  int nv, cap;
  int* e; /* edge (a, b, midpoint) triples, a < b */
  int ne, ecap;
} mesh_t;

static int add_vertex(mesh_t* m, double x, double y, double z) {
  if (m->nv == m->cap) {
    m->cap = 2 * m->cap + 16;
    m->v = (double*)realloc(m->v, sizeof(double) * 3 * m->cap);
  }
  double r = sqrt(x * x + y * y + z * z);
  m->v[3 * m->nv] = x / r;
  m->v[3 * m->nv + 1] = y / r;
  m->v[3 * m->nv + 2] = z / r;
  return m->nv++;
}

static int midpoint(mesh_t* m, int a, int b) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  for (int k = 0; k < m->ne; ++k)
    if (m->e[3 * k] == lo && m->e[3 * k + 1] == hi) return m->e[3 * k + 2];
  int c = add_vertex(m, 0.5 * (m->v[3 * a] + m->v[3 * b]), 0.5 * (m->v[3 * a + 1] + m->v[3 * b + 1]),
                     0.5 * (m->v[3 * a + 2] + m->v[3 * b + 2]));
  if (m->ne == m->ecap) {
    m->ecap = 2 * m->ecap + 16;
    m->e = (int*)realloc(m->e, sizeof(int) * 3 * m->ecap);
  }
  m->e[3 * m->ne] = lo;
  m->e[3 * m->ne + 1] = hi;
  m->e[3 * m->ne + 2] = c;
  m->ne++;
  return c;
}

int main(int argc, char** argv) {
  const int level = argc > 1 ? atoi(argv[1]) : 3;
  const double R = argc > 2 ? atof(argv[2]) : 2.0;
  mesh_t m = {0};
  const double p[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  for (int i = 0; i < 6; ++i) add_vertex(&m, p[i][0], p[i][1], p[i][2]);
  /* counter-clockwise seen from outside */
  int nf = 8;
  int* f = (int*)malloc(sizeof(int) * 3 * nf);
  const int f0[8][3] = {{0, 2, 4}, {2, 1, 4}, {1, 3, 4}, {3, 0, 4}, {2, 0, 5}, {1, 2, 5}, {3, 1, 5}, {0, 3, 5}};
  for (int i = 0; i < 8; ++i)
    for (int k = 0; k < 3; ++k) f[3 * i + k] = f0[i][k];
  for (int l = 0; l < level; ++l) {
    int* g = (int*)malloc(sizeof(int) * 12 * nf);
    m.ne = 0;
    for (int i = 0; i < nf; ++i) {
      int a = f[3 * i], b = f[3 * i + 1], c = f[3 * i + 2];
      int ab = midpoint(&m, a, b), bc = midpoint(&m, b, c), ca = midpoint(&m, c, a);
      int t[4][3] = {{a, ab, ca}, {ab, b, bc}, {ca, bc, c}, {ab, bc, ca}};
      for (int q = 0; q < 4; ++q)
        for (int k = 0; k < 3; ++k) g[12 * i + 3 * q + k] = t[q][k];
    }
    free(f);
    f = g;
    nf *= 4;
  }
  double* V = (double*)malloc(sizeof(double) * 3 * m.nv);
  for (int i = 0; i < 3 * m.nv; ++i) V[i] = R * m.v[i];
  int32_t* F = (int32_t*)malloc(sizeof(int32_t) * 3 * nf);
  for (int i = 0; i < 3 * nf; ++i) F[i] = f[i];
  const double Q[4] = {0.0, 0.0, 0.0, 1.0};
  const double eps1 = 1.0, eps2 = 80.0;
  const double born = -0.5 * 332.0716 * (1.0 / eps1 - 1.0 / eps2) / R;
  int status = 0;
  for (int prec = 0; prec < 2; ++prec) {
    hobi_options opt;
    hobi_default_options(&opt);
    opt.precision = prec == 0 ? HOBI_FP64 : HOBI_FP32_BULK;
    hobi_t h = NULL;
    if (hobi_setup(V, m.nv, F, nf, m.v, Q, 1, eps1, eps2, 0.0, &opt, &h) != HOBI_OK) {
      fprintf(stderr, "hobi_setup: %s\n", hobi_last_error());
      return 2;
    }
    double* phi = (double*)malloc(sizeof(double) * m.nv);
    double* dphi = (double*)malloc(sizeof(double) * m.nv);
    hobi_solve_info info = {0};
    int r = hobi_solve(h, 1e-8, 200, phi, dphi, &info);
    double e = 0.0;
    if (r == HOBI_OK) r = hobi_energy(h, &e);
    /* reaction potential and field at the centre and at an interior point */
    const double pts[6] = {0.0, 0.0, 0.0, 0.3 * R, 0.2 * R, -0.1 * R};
    double pr[2] = {0.0, 0.0}, fr[6] = {0.0};
    if (r == HOBI_OK) r = hobi_reaction_potential(h, pts, 2, pr);
    if (r == HOBI_OK) r = hobi_reaction_field(h, pts, 2, fr);
    if (r != HOBI_OK) {
      fprintf(stderr, "solve/energy/potential/field: %s\n", hobi_last_error());
      status = 3;
    }
    printf("%s vertices %d faces %d iterations %d E_sol %.8f born %.8f\n", prec == 0 ? "fp64" : "fp32", m.nv, nf,
           info.iterations, e, born);
    printf("%s phi_reac %.10e %.10e field %.6e %.6e %.6e %.6e %.6e %.6e\n", prec == 0 ? "fp64" : "fp32", pr[0], pr[1],
           fr[0], fr[1], fr[2], fr[3], fr[4], fr[5]);
    free(phi);
    free(dphi);
    hobi_destroy(h);
  }
  free(V);
  free(F);
  free(f);
  free(m.v);
  free(m.e);
  return status;
}
