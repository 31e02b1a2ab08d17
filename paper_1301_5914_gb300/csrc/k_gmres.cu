// k_gmres.cu -- device-resident restarted GMRES in FP64 (the Krylov solver of the paper's
// abstract and of the iteration loop in the Table 1 pseudocode), written so that one iteration is a fixed
// sequence of kernels whose iteration index lives in device memory (GmresState.k): the host can
// capture the sequence once as a CUDA graph and replay it.
//
// Orthogonalisation: classical Gram-Schmidt applied twice (CGS2), which is as stable as modified
// Gram-Schmidt and needs a fixed number of launches per iteration; all dot products are
// deterministic two-stage block reductions. Givens rotations and the residual estimate run in a
// single thread.
#include <math.h>

#include "hobi_internal.cuh"

namespace hobi {
namespace {

constexpr int kThreads = 256;

__device__ double block_reduce(double v) {
  __shared__ double warp_sums[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_sums[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < kThreads / 32 ? warp_sums[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// part[j * kDotBlocks + b] = sum over block b's slice of V_j . w, for j = 0..k (self: w . w only)
__global__ void k_dots(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ w, int64_t n,
                       const GmresState* st, int self, double* __restrict__ part) {
  const int kmax = self ? 0 : st->k;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per;
  const int64_t b1 = b0 + per < n ? b0 + per : n;
  for (int j = 0; j <= kmax; ++j) {
    const double* v = self ? w : Vb + (int64_t)j * ld;
    double s = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += v[i] * w[i];
    s = block_reduce(s);
    if (threadIdx.x == 0) part[j * kDotBlocks + blockIdx.x] = s;
  }
}

// c[j] = sum_b part[j][b]; hcol[j] = (accumulate ? hcol[j] : 0) + c[j]
__global__ void k_reduce_dots(const double* __restrict__ part, const GmresState* st, int self, double* c,
                              double* hcol, int accumulate) {
  const int j = blockIdx.x;
  const int kmax = self ? 0 : st->k;
  if (j > kmax) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < kDotBlocks; b += blockDim.x) s += part[j * kDotBlocks + b];
  s = block_reduce(s);
  if (threadIdx.x == 0) {
    c[j] = s;
    if (hcol) hcol[j] = accumulate ? hcol[j] + s : s;
  }
}

// w -= sum_{j<=k} c_j V_j
__global__ void k_axpy_basis(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ c,
                             const GmresState* st, double* __restrict__ w, int64_t n) {
  const int k = st->k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j <= k; ++j) s -= c[j] * Vb[(int64_t)j * ld + i];
    w[i] = s;
  }
}

// Column k of the Hessenberg matrix: apply the previous rotations, form the new one, update g.
__global__ void k_givens(GmresState* st, int m, double* H, double* cs, double* sn, double* g,
                         const double* hcol, const double* hn2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->k;
  const double hn = sqrt(hn2[0]);
  for (int j = 0; j <= k; ++j) H[j * m + k] = hcol[j];
  H[(k + 1) * m + k] = hn;
  for (int j = 0; j < k; ++j) {
    double a = H[j * m + k], b = H[(j + 1) * m + k];
    H[j * m + k] = cs[j] * a + sn[j] * b;
    H[(j + 1) * m + k] = -sn[j] * a + cs[j] * b;
  }
  double a = H[k * m + k], b = H[(k + 1) * m + k];
  double den = sqrt(a * a + b * b);
  double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  cs[k] = c;
  sn[k] = s;
  H[k * m + k] = den;
  H[(k + 1) * m + k] = 0.0;
  g[k + 1] = -s * g[k];
  g[k] = c * g[k];
  st->hn = hn;
  st->rel = fabs(g[k + 1]) / st->bnorm;
  st->it += 1;
  if (st->rel <= st->tol) st->converged = 1;
  if (!isfinite(hn) || !isfinite(st->rel) || (!(hn > 0.0) && !st->converged)) st->breakdown = 1;
}

// V_{k+1} = w / h_{k+1,k}
__global__ void k_next_basis(double* __restrict__ Vb, int64_t ld, const double* __restrict__ w, int64_t n,
                             const GmresState* st) {
  const int k = st->k;
  const double hn = st->hn;
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double* v = Vb + (int64_t)(k + 1) * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

__global__ void k_advance(GmresState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->k += 1;
}

// V_0 = r / ||r|| (r already in V_0), g = (||r||, 0, ...), k = 0
__global__ void k_cycle_start(double* __restrict__ Vb, int64_t n, const double* nrm2, GmresState* st, double* g,
                              int m, int first) {
  const double beta = sqrt(nrm2[0]);
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Vb[i] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int j = 0; j <= m; ++j) g[j] = 0.0;
    g[0] = beta;
    st->k = 0;
    if (first) {
      st->bnorm = beta;
      st->it = 0;
      st->converged = 0;
      st->breakdown = 0;
    }
    st->rel = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
    if (!(beta > 0.0) || st->rel <= st->tol) st->converged = 1;
  }
}

// y = H(0:k,0:k)^{-1} g(0:k)   (k = number of columns built in this cycle)
__global__ void k_backsolve(const double* H, int m, const double* g, const GmresState* st, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int j = i + 1; j < k; ++j) t -= H[i * m + j] * y[j];
    y[i] = t / H[i * m + i];
  }
}

// x += sum_{j<k} y_j V_j, or with scaled unknowns x += dscale * sum_{j<k} y_j V_j
__global__ void k_update_x(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ y,
                           const GmresState* st, double* __restrict__ x, int64_t n, const double* __restrict__ dscale) {
  const int k = st->k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (dscale) {
      double t = 0.0;
      for (int j = 0; j < k; ++j) t += y[j] * Vb[(int64_t)j * ld + i];
      x[i] += dscale[i] * t;
    } else {
      double s = x[i];
      for (int j = 0; j < k; ++j) s += y[j] * Vb[(int64_t)j * ld + i];
      x[i] = s;
    }
  }
}

// z = dscale * V_k (k from device memory)
__global__ void k_scale_column(const double* __restrict__ Vb, int64_t ld, const int* kptr,
                               const double* __restrict__ dscale, double* __restrict__ z, int64_t n) {
  const double* v = Vb + (int64_t)(*kptr) * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = dscale[i] * v[i];
}

__global__ void k_fill_scale(double* __restrict__ d, int64_t half, double lo, double hi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * half; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = i < half ? lo : hi;
}

__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Ax[i];
}

// x += d (mixed-precision refinement)
__global__ void k_add_in_place(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// out[0] = ||v||_2, one block, fixed summation order
__global__ void k_norm2(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * v[i];
  s = block_reduce(s);
  if (threadIdx.x == 0) out[0] = sqrt(s);
}

inline int grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_dots(const double* Vb, int64_t ld, const double* w, int64_t n, const GmresState* st, int self,
                        double* part, cudaStream_t s) {
  k_dots<<<kDotBlocks, kThreads, 0, s>>>(Vb, ld, w, n, st, self, part);
  return cudaGetLastError();
}

cudaError_t launch_reduce_dots(const double* part, int m, const GmresState* st, int self, double* c, double* hcol,
                               int accumulate, cudaStream_t s) {
  k_reduce_dots<<<self ? 1 : m + 1, kThreads, 0, s>>>(part, st, self, c, hcol, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_axpy_basis(const double* Vb, int64_t ld, const double* c, const GmresState* st, double* w,
                              int64_t n, cudaStream_t s) {
  k_axpy_basis<<<grid_for(n), kThreads, 0, s>>>(Vb, ld, c, st, w, n);
  return cudaGetLastError();
}

cudaError_t launch_givens(GmresState* st, int m, double* H, double* cs, double* sn, double* g, const double* hcol,
                          const double* hn2, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(st, m, H, cs, sn, g, hcol, hn2);
  return cudaGetLastError();
}

cudaError_t launch_next_basis(double* Vb, int64_t ld, const double* w, int64_t n, GmresState* st, cudaStream_t s) {
  k_next_basis<<<grid_for(n), kThreads, 0, s>>>(Vb, ld, w, n, st);
  return cudaGetLastError();
}

cudaError_t launch_advance(GmresState* st, cudaStream_t s) {
  k_advance<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_cycle_start(double* Vb, int64_t n, const double* nrm2, GmresState* st, double* g, int m,
                               int first, cudaStream_t s) {
  k_cycle_start<<<grid_for(n), kThreads, 0, s>>>(Vb, n, nrm2, st, g, m, first);
  return cudaGetLastError();
}

cudaError_t launch_finish_cycle(const double* H, int m, const double* g, const GmresState* st, double* y,
                                const double* Vb, int64_t ld, double* x, int64_t n, const double* dscale,
                                cudaStream_t s) {
  k_backsolve<<<1, 32, 0, s>>>(H, m, g, st, y);
  k_update_x<<<grid_for(n), kThreads, 0, s>>>(Vb, ld, y, st, x, n, dscale);
  return cudaGetLastError();
}

cudaError_t launch_scale_column(const double* Vb, int64_t ld, const int* kptr, const double* dscale, double* z,
                                int64_t n, cudaStream_t s) {
  k_scale_column<<<grid_for(n), kThreads, 0, s>>>(Vb, ld, kptr, dscale, z, n);
  return cudaGetLastError();
}

cudaError_t launch_fill_scale(double* d, int64_t half, double lo, double hi, cudaStream_t s) {
  k_fill_scale<<<grid_for(2 * half), kThreads, 0, s>>>(d, half, lo, hi);
  return cudaGetLastError();
}

cudaError_t launch_add_in_place(double* x, const double* d, int64_t n, cudaStream_t s) {
  k_add_in_place<<<grid_for(n), kThreads, 0, s>>>(x, d, n);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const double* v, int64_t n, double* out, cudaStream_t s) {
  k_norm2<<<1, kThreads, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_residual_start(const double* b, const double* Ax, double* r, int64_t n, cudaStream_t s) {
  k_residual<<<grid_for(n), kThreads, 0, s>>>(b, Ax, r, n);
  return cudaGetLastError();
}

}  // namespace hobi
