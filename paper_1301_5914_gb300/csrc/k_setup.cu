// k_setup.cu -- one-time setup kernels of the HOBI-PB solver (FP64).
//
//  * vertex -> incident-face adjacency (sorted rows, deterministic)
//  * mesh validation: index range, closed and consistently oriented (every directed edge has
//    exactly one opposite edge), referenced vertices, finite non-zero normals, positive volume
//  * curved-element node generator (Sec. 2.2): cubic edge arcs through the vertices with the
//    vertex normals, the 10 interpolation points, the cubic (10-point) interpolant
//    (Eq. (15)), and the 4 regular-rule nodes per element with position, unit normal and
//    W_{j,m,n} = w_m J L_n (Eq. (17))
//  * singular correction (Sec. 2.3, Eqs. (19)/(20)): for each vertex i and each face j having i
//    as a corner, the 16-point Duffy/Gauss-Legendre sum minus the 4-point regular sum that the
//    far-field kernel adds for the same face
//  * right-hand side S1, S2 (Eq. (11)) with the charges' 1/eps1
#include <math.h>

#include <cmath>

#include "ff_body.cuh"

namespace hobi {
namespace {

// ------------------------------------------------------------------ vector helpers (FP64)
__device__ __forceinline__ double3 mk(double x, double y, double z) { return make_double3(x, y, z); }
__device__ __forceinline__ double3 operator+(double3 a, double3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ double3 operator-(double3 a, double3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 operator*(double s, double3 a) { return mk(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross(double3 a, double3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double3 normalized(double3 a) { return (1.0 / sqrt(dot(a, a))) * a; }
__device__ __forceinline__ double3 ld3(const double* p) { return mk(p[0], p[1], p[2]); }
__device__ __forceinline__ void st3(double* p, double3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

// deterministic block sum (blockDim.x a power of two <= 1024)
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ adjacency
__global__ void k_count_degree(int n3, const int* F, int nv, int* deg) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  int v = F[t];
  if (v >= 0 && v < nv) atomicAdd(&deg[v], 1);
}

// Exclusive prefix sum of n ints by one block of 1024 threads; out has n+1 entries.
__global__ void k_scan_1block(int n, const int* in, int* out) {
  __shared__ int sums[1024];
  const int tid = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int b = min(n, tid * chunk), e = min(n, b + chunk);
  int s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  sums[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int v = tid >= off ? sums[tid - off] : 0;
    __syncthreads();
    sums[tid] += v;
    __syncthreads();
  }
  int run = tid ? sums[tid - 1] : 0;
  for (int i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (tid == 1023) out[n] = sums[1023];
}

__global__ void k_fill_incidence(int n3, const int* F, int nv, const int* ptr, int* cursor, int* face) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  int v = F[t];
  if (v < 0 || v >= nv) return;
  int pos = atomicAdd(&cursor[v], 1);
  face[ptr[v] + pos] = t / 3;
}

// Sort each row by face index (rows are short) so every later pass is deterministic.
__global__ void k_sort_rows(int nv, const int* ptr, int* face) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  int b = ptr[v], e = ptr[v + 1];
  for (int i = b + 1; i < e; ++i) {
    int key = face[i];
    int j = i - 1;
    while (j >= b && face[j] > key) {
      face[j + 1] = face[j];
      --j;
    }
    face[j + 1] = key;
  }
}

// ------------------------------------------------------------------ validation
__device__ __forceinline__ bool has_directed_edge(const int* f, int p, int q) {
  return (f[0] == p && f[1] == q) || (f[1] == p && f[2] == q) || (f[2] == p && f[0] == q);
}

constexpr int kValThreads = 256;

__global__ void k_validate_faces(int nv, int nf, const double* V, const int* F, const int* ptr,
                                 const int* inc, double* vol_part, int* flags) {
  __shared__ double sh[kValThreads];
  double vol = 0.0;
  int fl = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
    const int* f = F + 3 * j;
    int a = f[0], b = f[1], c = f[2];
    if (a < 0 || a >= nv || b < 0 || b >= nv || c < 0 || c >= nv || a == b || b == c || a == c) {
      fl |= kBadIndex;
      continue;
    }
    double3 A = ld3(V + 3 * a), B = ld3(V + 3 * b), C = ld3(V + 3 * c);
    double3 cr = cross(B - A, C - A);
    double ar = sqrt(dot(cr, cr));
    if (!(ar > 0.0) || !isfinite(ar)) fl |= kDegenerateFace;
    vol += dot(A, cross(B, C)) / 6.0;
    int ed[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int k = 0; k < 3; ++k) {
      int p = ed[k][0], q = ed[k][1];
      int same = 0, opp = 0;
      for (int e = ptr[p]; e < ptr[p + 1]; ++e) same += has_directed_edge(F + 3 * inc[e], p, q);
      for (int e = ptr[q]; e < ptr[q + 1]; ++e) opp += has_directed_edge(F + 3 * inc[e], q, p);
      if (same != 1 || opp != 1) fl |= kOpenOrInconsistent;
    }
  }
  if (fl) atomicOr(flags, fl);
  double s = block_sum(vol, sh);
  if (threadIdx.x == 0) vol_part[blockIdx.x] = s;
}

__global__ void k_validate_vertices(int nv, const double* V, const double* Nin, const int* ptr, double* Nout,
                                    double* center_part, int* flags) {
  __shared__ double sh[kValThreads];
  double sx = 0.0, sy = 0.0, sz = 0.0;
  int fl = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    double3 x = ld3(V + 3 * i);
    if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z)) fl |= kNonFinite;
    if (ptr[i + 1] == ptr[i]) fl |= kUnreferencedVertex;
    double3 n = ld3(Nin + 3 * i);
    double len = sqrt(dot(n, n));
    if (!(len > 0.0) || !isfinite(len)) {
      fl |= kBadNormal;
      len = 1.0;
    }
    st3(Nout + 3 * i, (1.0 / len) * n);
    sx += x.x;
    sy += x.y;
    sz += x.z;
  }
  if (fl) atomicOr(flags, fl);
  double a = block_sum(sx, sh), b = block_sum(sy, sh), c = block_sum(sz, sh);
  if (threadIdx.x == 0) {
    center_part[3 * blockIdx.x + 0] = a;
    center_part[3 * blockIdx.x + 1] = b;
    center_part[3 * blockIdx.x + 2] = c;
  }
}

__global__ void k_validate_charges(int nc, const double* Q, int* flags) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  const double* q = Q + 4 * k;
  if (!isfinite(q[0]) || !isfinite(q[1]) || !isfinite(q[2]) || !isfinite(q[3])) atomicOr(flags, kBadCharge);
}

__global__ void k_finish_validate(int nv, const double* vol_part, int nb, const double* center_part,
                                  double* center, int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double vol = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
  for (int b = 0; b < nb; ++b) {
    vol += vol_part[b];
    cx += center_part[3 * b];
    cy += center_part[3 * b + 1];
    cz += center_part[3 * b + 2];
  }
  if (!(vol > 0.0)) atomicOr(flags, kNegativeVolume);
  center[0] = cx / nv;
  center[1] = cy / nv;
  center[2] = cz / nv;
}

// ------------------------------------------------------------------ curved elements (Sec. 2.2)
// Arc between nodes P, Q with unit normals nP, nQ: cubic Hermite curve through P (t=0) and Q (t=1)
// whose end tangents are the chord projected on each end's tangent plane, unit length times the
// chord length |Q-P|. Normal along the arc: the blend (1-t) nP + t nQ with its component along
// the arc tangent removed, normalised.
__device__ void arc_point(double3 P, double3 nP, double3 Q, double3 nQ, double t, double3* x, double3* n) {
  double3 e = Q - P;
  double L = sqrt(dot(e, e));
  double3 TP = L * normalized(e - dot(e, nP) * nP);
  double3 TQ = L * normalized(e - dot(e, nQ) * nQ);
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2.0 * t3 - 3.0 * t2 + 1.0, h10 = t3 - 2.0 * t2 + t;
  double h01 = 3.0 * t2 - 2.0 * t3, h11 = t3 - t2;
  double d00 = 6.0 * t2 - 6.0 * t, d10 = 3.0 * t2 - 4.0 * t + 1.0;
  double d01 = 6.0 * t - 6.0 * t2, d11 = 3.0 * t2 - 2.0 * t;
  *x = h00 * P + h10 * TP + h01 * Q + h11 * TQ;
  double3 tau = normalized(d00 * P + d10 * TP + d01 * Q + d11 * TQ);
  double3 w = (1.0 - t) * nP + t * nQ;
  *n = normalized(w - dot(w, tau) * tau);
}

// Element point order used on the device:
//   0,1,2: X1 (r,s)=(0,0), X2 (1,0), X3 (0,1)
//   3,4  : arc X1->X2 at 1/3, 2/3      (1/3,0), (2/3,0)
//   5,6  : arc X2->X3 at 1/3, 2/3      (2/3,1/3), (1/3,2/3)
//   7,8  : arc X3->X1 at 1/3, 2/3      (0,2/3), (0,1/3)
//   9    : (1/3,1/3) = (u,v) = (2/3,1/2) of Eq. (14): arc Y1->Y2 at 1/2 with Y1 = arc X1->X2 at 2/3,
//          Y2 = arc X1->X3 at 2/3 (= arc X3->X1 at 1/3 by the arc's symmetry)
__device__ void element_points(double3 X1, double3 n1, double3 X2, double3 n2, double3 X3, double3 n3,
                               double3 p[10]) {
  double3 m4, m7, dummy;
  p[0] = X1;
  p[1] = X2;
  p[2] = X3;
  arc_point(X1, n1, X2, n2, 1.0 / 3.0, &p[3], &dummy);
  arc_point(X1, n1, X2, n2, 2.0 / 3.0, &p[4], &m4);
  arc_point(X2, n2, X3, n3, 1.0 / 3.0, &p[5], &dummy);
  arc_point(X2, n2, X3, n3, 2.0 / 3.0, &p[6], &dummy);
  arc_point(X3, n3, X1, n1, 1.0 / 3.0, &p[7], &m7);
  arc_point(X3, n3, X1, n1, 2.0 / 3.0, &p[8], &dummy);
  arc_point(p[4], m4, p[7], m7, 0.5, &p[9], &dummy);
}

// Cubic Lagrange basis on the 10 points above and its (r,s) derivatives at (r,s), in point order.
// Barycentrics l1 = 1-r-s, l2 = r, l3 = s. Vertex functions l(3l-1)(3l-2)/2, edge functions
// 9/2 la lb (3 la - 1) for the point nearer corner a, centre 27 l1 l2 l3.
__device__ void basis(double r, double s, double* N, double* Nr, double* Ns) {
  const double l[3] = {1.0 - r - s, r, s};
  const double dlr[3] = {-1.0, 1.0, 0.0}, dls[3] = {-1.0, 0.0, 1.0};
  for (int a = 0; a < 3; ++a) {
    double la = l[a];
    double df = 0.5 * (27.0 * la * la - 18.0 * la + 2.0);
    N[a] = 0.5 * la * (3.0 * la - 1.0) * (3.0 * la - 2.0);
    Nr[a] = df * dlr[a];
    Ns[a] = df * dls[a];
  }
  // (near corner, far corner, point index)
  const int ep[6][3] = {{0, 1, 3}, {1, 0, 4}, {1, 2, 5}, {2, 1, 6}, {2, 0, 7}, {0, 2, 8}};
  for (int e = 0; e < 6; ++e) {
    double la = l[ep[e][0]], lb = l[ep[e][1]];
    double fa = 4.5 * lb * (6.0 * la - 1.0), fb = 4.5 * la * (3.0 * la - 1.0);
    N[ep[e][2]] = 4.5 * la * lb * (3.0 * la - 1.0);
    Nr[ep[e][2]] = fa * dlr[ep[e][0]] + fb * dlr[ep[e][1]];
    Ns[ep[e][2]] = fa * dls[ep[e][0]] + fb * dls[ep[e][1]];
  }
  N[9] = 27.0 * l[0] * l[1] * l[2];
  Nr[9] = 27.0 * (l[1] * l[2] * dlr[0] + l[0] * l[2] * dlr[1] + l[0] * l[1] * dlr[2]);
  Ns[9] = 27.0 * (l[1] * l[2] * dls[0] + l[0] * l[2] * dls[1] + l[0] * l[1] * dls[2]);
}

// Interpolant value and (r,s) derivatives from basis values B = {N[10], Nr[10], Ns[10]}.
__device__ __forceinline__ void combine_points(const double3 p[10], const double* B, double3* x, double3* xr,
                                               double3* xs) {
  double3 X = mk(0, 0, 0), R = mk(0, 0, 0), S = mk(0, 0, 0);
  for (int q = 0; q < 10; ++q) {
    X = X + B[q] * p[q];
    R = R + B[10 + q] * p[q];
    S = S + B[20 + q] * p[q];
  }
  *x = X;
  *xr = R;
  *xs = S;
}

// Cubic Lagrange interpolant on the 10 points: value and (r,s) derivatives at (r,s).
__device__ void interpolate(const double3 p[10], double r, double s, double3* x, double3* xr, double3* xs) {
  double B[30];
  basis(r, s, B, B + 10, B + 20);
  combine_points(p, B, x, xr, xs);
}

// The 4-point regular rule: collapsed coordinates r = xi (1 - eta), s = xi eta; xi from the
// 2-point Gauss-Jacobi rule for the weight xi on [0,1], eta from 2-point Gauss-Legendre.
__device__ void regular_point(int m, double* r, double* s, double* w) {
  const double r6 = sqrt(6.0), r3 = sqrt(3.0);
  int a = m >> 1, b = m & 1;
  double xi = a ? (6.0 + r6) / 10.0 : (6.0 - r6) / 10.0;
  double wx = a ? (9.0 + r6) / 36.0 : (9.0 - r6) / 36.0;
  double eta = b ? 0.5 + 0.5 / r3 : 0.5 - 0.5 / r3;
  *r = xi * (1.0 - eta);
  *s = xi * eta;
  *w = 0.5 * wx;
}

__global__ void k_node_gen(int nf, const int* F, const double* V, const double* Nv, double* elem, double* ny,
                           double* nnu, double* nW, int* flags) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nf) return;
  int a = F[3 * j], b = F[3 * j + 1], c = F[3 * j + 2];
  double3 p[10];
  element_points(ld3(V + 3 * a), ld3(Nv + 3 * a), ld3(V + 3 * b), ld3(Nv + 3 * b), ld3(V + 3 * c),
                 ld3(Nv + 3 * c), p);
  for (int k = 0; k < 10; ++k) st3(elem + 30 * (size_t)j + 3 * k, p[k]);
  for (int m = 0; m < 4; ++m) {
    double r, s, w;
    regular_point(m, &r, &s, &w);
    double3 x, xr, xs;
    interpolate(p, r, s, &x, &xr, &xs);
    double3 cr = cross(xr, xs);
    double J = sqrt(dot(cr, cr));
    if (!(J > 0.0) || !isfinite(J) || !isfinite(x.x + x.y + x.z)) atomicOr(flags, kDegenerateElement);
    size_t node = 4 * (size_t)j + m;
    st3(ny + 3 * node, x);
    st3(nnu + 3 * node, (1.0 / J) * cr);
    nW[3 * node + 0] = w * J * (1.0 - r - s);
    nW[3 * node + 1] = w * J * r;
    nW[3 * node + 2] = w * J * s;
  }
}

// ------------------------------------------------------------------ kernels K1..K4 (Eq. (10))
// With d = x - y, r = |d|, E = exp(-kappa r), P = E (1 + kappa r), Q = E (3 + 3 kappa r + kappa^2 r^2):
//   4 pi K1 = (1 - E)/r,  4 pi K2 = (eps P - 1) (d.ny)/r^3,  4 pi K3 = (P/eps - 1) (d.nx)/r^3,
//   4 pi K4 = (P - 1)(nx.ny)/r^3 - (Q - 3)(d.nx)(d.ny)/r^5.
// 1/r and E come from the FP64 far field's own routines (ff_body.cuh: MUFU rsqrt seed + Newton
// step, table-driven exponential with the 256-entry table `tab` in shared memory), within a few
// units in the last place of sqrt, division and exp.
struct KernelConsts {
  double eps, ieps, kappa, c256;  // c256 = -256 log2(e) kappa: E = 2^(c256 r / 256)
};
__device__ void kernels_fp64(double3 x, double3 nx, double3 y, double3 ny, const KernelConsts& kc,
                             const double* tab, double K[4]) {
  double3 d = x - y;
  double r2 = dot(d, d);
  double ir = ff::rsqrt_f64(r2);
  double r = r2 * ir;
  double ir2 = ir * ir, ir3 = ir2 * ir;
  double kr = kc.kappa * r;
  double E = ff::exp2_256th(r * kc.c256, tab);
  double P = E * (1.0 + kr);
  double Q = E * (3.0 + kr * (3.0 + kr));
  double ax = dot(d, nx), ay = dot(d, ny), c = dot(nx, ny);
  K[0] = kInv4Pi * (1.0 - E) * ir;
  K[1] = kInv4Pi * (kc.eps * P - 1.0) * ay * ir3;
  K[2] = kInv4Pi * (P * kc.ieps - 1.0) * ax * ir3;
  K[3] = kInv4Pi * ((P - 1.0) * c - (Q - 3.0) * ax * ay * ir2) * ir3;
}

// The 16-point singular rule in the (r', s') frame with the target vertex at the origin: the
// 4 x 4 Gauss-Legendre tensor rule on [0,1]^2 under the Duffy map r' = (1 - y) x, s' = y x, with
// the map's Jacobian x folded into the weights. Computed once on the host.
struct SingularRule {
  double r[16], s[16], w[16];
};

__global__ void k_vertex_of_entry(int nv, const int* ptr, int* vert) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) vert[e] = i;
}

// One thread per (vertex i, incident face j) entry.
__global__ void k_correction(int n_entries, const int* vert, const int* F, const double* V, const double* Nv,
                             const int* inc_face, const double* elem, const double* ny, const double* nnu,
                             const double* nW, KernelConsts kc, SingularRule rule, double* corr) {
  __shared__ double tab[ff::kExpTable];
  // basis values at the 16 rule points for each of the 3 corners the target vertex can be
  __shared__ double bt[3 * 16][30];
  ff::exp_table_init(tab);
  for (int t = threadIdx.x; t < 3 * 16; t += blockDim.x) {
    const int kk = t / 16, m = t % 16;
    double l[3];
    l[kk] = 1.0 - rule.r[m] - rule.s[m];
    l[(kk + 1) % 3] = rule.r[m];
    l[(kk + 2) % 3] = rule.s[m];
    basis(l[1], l[2], bt[t], bt[t] + 10, bt[t] + 20);
  }
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += gridDim.x * blockDim.x) {
    int i = vert[e], j = inc_face[e];
    const int* f = F + 3 * j;
    int k = (f[0] == i) ? 0 : ((f[1] == i) ? 1 : 2);
    double3 x = ld3(V + 3 * i), nx = ld3(Nv + 3 * i);
    double3 p[10];
    for (int q = 0; q < 10; ++q) p[q] = ld3(elem + 30 * (size_t)j + 3 * q);
    double acc[3][4] = {};
    // 16-point singular rule: Duffy map with vertex i at the origin of the (r',s') frame
    for (int m = 0; m < 16; ++m) {
      const double rp = rule.r[m], sp = rule.s[m];
      double l[3];
      l[k] = 1.0 - rp - sp;
      l[(k + 1) % 3] = rp;
      l[(k + 2) % 3] = sp;
      double3 y, yr, ys;
      combine_points(p, bt[16 * k + m], &y, &yr, &ys);
      double3 cr = cross(yr, ys);
      double J2 = dot(cr, cr);
      double iJ = ff::rsqrt_f64(J2);
      double K[4];
      kernels_fp64(x, nx, y, iJ * cr, kc, tab, K);
      double w = rule.w[m] * (J2 * iJ);
      for (int n = 0; n < 3; ++n)
        for (int q = 0; q < 4; ++q) acc[n][q] += w * l[n] * K[q];
    }
    // minus the regular-rule terms of the same face that the far field includes
    for (int m = 0; m < 4; ++m) {
      size_t node = 4 * (size_t)j + m;
      double K[4];
      kernels_fp64(x, nx, ld3(ny + 3 * node), ld3(nnu + 3 * node), kc, tab, K);
      for (int n = 0; n < 3; ++n)
        for (int q = 0; q < 4; ++q) acc[n][q] -= nW[3 * node + n] * K[q];
    }
    for (int n = 0; n < 3; ++n)
      for (int q = 0; q < 4; ++q) corr[12 * (size_t)e + 4 * n + q] = acc[n][q];
  }
}

// ------------------------------------------------------------------ right-hand side (Eq. (11))
// One thread per vertex sums G0 and its normal derivative over all charges (staged 256 at a time
// in shared memory). 1/r comes from the far field's FP64 reciprocal square root (a MUFU seed and
// one second-order Newton step), not from sqrt and a division: 19 FP64 operations per pair.
__global__ void k_rhs(int nv, int nc, const double* V, const double* Nv, const double* Q, double eps1,
                      double* b) {
  __shared__ double sq[256 * 4];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double3 x = mk(0, 0, 0), n = mk(0, 0, 1);
  if (i < nv) {
    x = ld3(V + 3 * i);
    n = ld3(Nv + 3 * i);
  }
  double s1 = 0.0, s2 = 0.0;
  for (int base = 0; base < nc; base += 256) {
    int cnt = min(256, nc - base);
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * cnt; t += blockDim.x) sq[t] = Q[4 * (size_t)base + t];
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      const double3 d = x - mk(sq[4 * k], sq[4 * k + 1], sq[4 * k + 2]);
      const double ir = ff::rsqrt_f64(dot(d, d));
      const double qir = sq[4 * k + 3] * ir;
      s1 += qir;
      s2 = fma(-qir * (ir * ir), dot(d, n), s2);
    }
  }
  if (i < nv) {
    b[i] = s1 * kInv4Pi / eps1;
    b[nv + i] = s2 * kInv4Pi / eps1;
  }
}

// ------------------------------------------------------------------ targets
__global__ void k_targets(int nv, const double* V, const double* Nv, const double* center, double xs, float4* t32,
                          double* t64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double3 x = ld3(V + 3 * i) - ld3(center), n = ld3(Nv + 3 * i);
  t32[2 * i] = make_float4((float)(xs * x.x), (float)(xs * x.y), (float)(xs * x.z), 0.f);
  t32[2 * i + 1] = make_float4((float)n.x, (float)n.y, (float)n.z, 0.f);
  double* o = t64 + 8 * (size_t)i;
  o[0] = xs * x.x; o[1] = xs * x.y; o[2] = xs * x.z; o[3] = 0.0;
  o[4] = n.x; o[5] = n.y; o[6] = n.z; o[7] = 0.0;
}

__global__ void k_points(int np, const double* P, int stride, const double* center, double xs, float4* t32,
                         double* t64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double3 x = ld3(P + (size_t)stride * i) - ld3(center);
  t32[2 * i] = make_float4((float)(xs * x.x), (float)(xs * x.y), (float)(xs * x.z), 0.f);
  t32[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  double* o = t64 + 8 * (size_t)i;
  o[0] = xs * x.x; o[1] = xs * x.y; o[2] = xs * x.z; o[3] = 0.0;
  o[4] = 0.0; o[5] = 0.0; o[6] = 0.0; o[7] = 0.0;
}

// LOBI-PB (Sec. 2.4): per flat face its centroid, unit normal and area (weight (A, 0, 0)).
__global__ void k_lobi_geometry(int nf, const int* F, const double* V, double* ny, double* nnu, double* nW,
                                int* flags) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nf) return;
  double3 a = ld3(V + 3 * F[3 * j]), b = ld3(V + 3 * F[3 * j + 1]), c = ld3(V + 3 * F[3 * j + 2]);
  double3 cr = cross(b - a, c - a);
  double len = sqrt(dot(cr, cr));
  if (!(len > 0.0) || !isfinite(len)) atomicOr(flags, kDegenerateElement);
  st3(ny + 3 * (size_t)j, (1.0 / 3.0) * (a + b + c));
  st3(nnu + 3 * (size_t)j, (1.0 / len) * cr);
  nW[3 * (size_t)j] = 0.5 * len;
  nW[3 * (size_t)j + 1] = 0.0;
  nW[3 * (size_t)j + 2] = 0.0;
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_lobi_geometry(int nf, const int* F, const double* V, double* ny, double* nnu, double* nW,
                                 int* flags, cudaStream_t s) {
  k_lobi_geometry<<<nblk(nf, 128), 128, 0, s>>>(nf, F, V, ny, nnu, nW, flags);
  return cudaGetLastError();
}

cudaError_t launch_adjacency(int nv, int nf, const int* F, int* deg, int* inc_ptr, int* inc_face,
                             int* entry_vertex, cudaStream_t s) {
  cudaMemsetAsync(deg, 0, sizeof(int) * nv, s);
  int n3 = 3 * nf;
  k_count_degree<<<nblk(n3, 256), 256, 0, s>>>(n3, F, nv, deg);
  k_scan_1block<<<1, 1024, 0, s>>>(nv, deg, inc_ptr);
  cudaMemsetAsync(deg, 0, sizeof(int) * nv, s);  // reused as the per-row fill cursor
  k_fill_incidence<<<nblk(n3, 256), 256, 0, s>>>(n3, F, nv, inc_ptr, deg, inc_face);
  k_sort_rows<<<nblk(nv, 128), 128, 0, s>>>(nv, inc_ptr, inc_face);
  k_vertex_of_entry<<<nblk(nv, 128), 128, 0, s>>>(nv, inc_ptr, entry_vertex);
  return cudaGetLastError();
}

cudaError_t launch_validate(int nv, int nf, int nc, const double* V, const double* Nv_in, const int* F,
                            const int* inc_ptr, const int* inc_face, const double* Q, double* Nv_unit,
                            double* vol_part, double* center_part, int* flags, cudaStream_t s) {
  k_validate_faces<<<kValidateBlocks, kValThreads, 0, s>>>(nv, nf, V, F, inc_ptr, inc_face, vol_part, flags);
  k_validate_vertices<<<kValidateBlocks, kValThreads, 0, s>>>(nv, V, Nv_in, inc_ptr, Nv_unit, center_part, flags);
  if (nc > 0) k_validate_charges<<<nblk(nc, 256), 256, 0, s>>>(nc, Q, flags);
  return cudaGetLastError();
}

cudaError_t launch_finish_validate(int nv, const double* vol_part, const double* center_part, double* center,
                                   int* flags, cudaStream_t s) {
  k_finish_validate<<<1, 32, 0, s>>>(nv, vol_part, kValidateBlocks, center_part, center, flags);
  return cudaGetLastError();
}

cudaError_t launch_node_gen(int nf, const int* F, const double* V, const double* Nv, double* elem, double* ny,
                            double* nnu, double* nW, int* flags, cudaStream_t s) {
  k_node_gen<<<nblk(nf, 128), 128, 0, s>>>(nf, F, V, Nv, elem, ny, nnu, nW, flags);
  return cudaGetLastError();
}

cudaError_t launch_correction_entries(int n_entries, const int* vert, const int* F, const double* V,
                                      const double* Nv, const int* inc_face, const double* elem, const double* ny,
                                      const double* nnu, const double* nW, double eps, double kappa, double* corr,
                                      cudaStream_t s) {
  // 4-point Gauss-Legendre on [0, 1]: nodes 1/2 (1 -+ sqrt(3/7 +- (2/7) sqrt(6/5))), weights
  // (18 -+ sqrt(30))/72 for the outer / inner pair
  const double t = 2.0 / 7.0 * std::sqrt(1.2);
  const double inner = std::sqrt(3.0 / 7.0 - t), outer = std::sqrt(3.0 / 7.0 + t);
  const double win = (18.0 + std::sqrt(30.0)) / 72.0, wout = (18.0 - std::sqrt(30.0)) / 72.0;
  const double gx[4] = {0.5 - 0.5 * outer, 0.5 - 0.5 * inner, 0.5 + 0.5 * inner, 0.5 + 0.5 * outer};
  const double gw[4] = {wout, win, win, wout};
  SingularRule rule;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      rule.r[4 * a + b] = (1.0 - gx[b]) * gx[a];
      rule.s[4 * a + b] = gx[b] * gx[a];
      rule.w[4 * a + b] = gw[a] * gw[b] * gx[a];
    }
  KernelConsts kc;
  kc.eps = eps;
  kc.ieps = 1.0 / eps;
  kc.kappa = kappa;
  kc.c256 = -ff::kExpTable * 1.44269504088896340735992468100 * kappa;
  if (n_entries <= 0) return cudaSuccess;
  k_correction<<<nblk(n_entries, 64), 64, 0, s>>>(n_entries, vert, F, V, Nv, inc_face, elem, ny, nnu, nW, kc, rule,
                                                    corr);
  return cudaGetLastError();
}

cudaError_t launch_rhs(int nv, int nc, const double* V, const double* Nv, const double* Q, double eps1, double* b,
                       cudaStream_t s) {
  // one-warp blocks: a large molecule spreads over all SMs in one wave (the FP64 pipe needs only a
  // warp or two per SM sub-partition), instead of 1-2 blocks of 256 per SM with a ragged second wave
  k_rhs<<<nblk(nv, 32), 32, 0, s>>>(nv, nc, V, Nv, Q, eps1, b);
  return cudaGetLastError();
}

cudaError_t launch_targets(int nv, const double* V, const double* Nv, const double* center, double xs,
                           float4* tgt32, double* tgt64, cudaStream_t s) {
  k_targets<<<nblk(nv, 256), 256, 0, s>>>(nv, V, Nv, center, xs, tgt32, tgt64);
  return cudaGetLastError();
}

cudaError_t launch_points(int np, const double* P, int stride, const double* center, double xs, float4* tgt32,
                          double* tgt64, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_points<<<nblk(np, 256), 256, 0, s>>>(np, P, stride, center, xs, tgt32, tgt64);
  return cudaGetLastError();
}
}  // namespace hobi
