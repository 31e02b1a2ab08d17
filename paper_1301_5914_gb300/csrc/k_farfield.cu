// k_farfield.cu -- the per-iteration hot path of the HOBI-PB matvec (Sec. 2.2-2.3, Eqs. (17)-(20)).
//
// For every target vertex x_i (unit normal nu_i) and every regular-rule node y (normal nu_y) of
// every element, the far-field kernel accumulates (d = x_i - y, r = |d|, E = exp(-kappa r),
// P = E (1 + kappa r), Q = E (3 + 3 kappa r + kappa^2 r^2)):
//
//   row 1:  (1 - E)/r sigma + (eps P - 1)/r^3 (d . m)
//   row 2:  nu_i . [ (P - 1)/r^3 m + ((P/eps - 1)/r^3 sigma - (Q - 3)/r^5 (d . m)) d ]
//
// with sigma = sum_n W_{j,m,n} u_{N_v + v_n} / (4 pi) and m = nu_y sum_n W_{j,m,n} u_{v_n} / (4 pi).
// Row 1 is the K1/K2 sum of Eq. (17) and row 2 the K3/K4 sum of Eq. (18) (Eq. (10) written out), with
// the target normal pulled out of the source sum so that each pair needs one vector
// accumulation instead of two dot products. Faces incident to x_i are included here and
// replaced by the singular rule through the precomputed correction (combine kernel).
//
// FP32-bulk kernel: each thread keeps 8 targets in registers as four packed pairs and evaluates
// every pair formula with Blackwell's paired FP32 instructions (__ffma2_rn / __fmul2_rn /
// __fadd2_rn: one instruction = the same operation on two targets), which halves the issue
// slots of the FMA-pipe work so that the FMA pipe itself becomes the limit. Source tiles (128
// nodes in the default one-warp shape) are staged in shared memory by bulk asynchronous copies,
// each source value stored twice ({v, v}) so one LDS.128
// feeds two packed operands; rsqrt and exp2 go to the MUFU pipe (rsqrt.approx / ex2.approx).
// Each tile's FP32 sum is folded into a compensated (two-float) accumulator, and the result is
// written as FP64 per (source chunk, target); the combine kernel adds the chunks in a fixed order.
//
// FP32 evaluation order (30 FMA-pipe operations per pair). With kappa > 0 the FP32 tables hold
// kappa x, kappa y and kappa m, so that kappa r is the scaled r; with v = (d . m)/r^2,
// P - 1 = E (1 + kappa r) - 1 and Q - 3 = 3 (P - 1) + E (kappa r)^2 (and r^2 v = d . m):
//   row 1 / eps = [ (1 - E) sigma/eps + (P - 1 + 1 - 1/eps) v ] / r
//   S = (P - 1)(sigma/eps - 3 v) + (sigma/eps - sigma) - E kappa^2 (d . m)
//   row 2 vector += (P - 1)/r^3 m + S/r^3 d
// which is the pair formula above multiplied out; the scale factors (eps kappa for row 1,
// kappa^2 for row 2) are applied once per target to the FP64 result.
#include <math.h>

#include "ff_body.cuh"

namespace hobi {
namespace {

// ------------------------------------------------------------------ gather (per matvec)
__global__ void k_gather32(int n_nodes, int nv, const int* __restrict__ F, const double* __restrict__ ny,
                           const double* __restrict__ nnu, const double* __restrict__ nW,
                           const double* __restrict__ center, const double* __restrict__ u, const int* kptr,
                           int64_t ld, double inv_eps, double xs, float4* __restrict__ src,
                           const int* __restrict__ pos) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_nodes) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  ff::gather32_node(node, nv, F, ny, nnu, nW, center, u, inv_eps, xs, src, pos ? pos[node] : node);
}

__global__ void k_gather64(int n_nodes, int nv, const int* __restrict__ F, const double* __restrict__ ny,
                           const double* __restrict__ nnu, const double* __restrict__ nW,
                           const double* __restrict__ center, const double* __restrict__ u, const int* kptr,
                           int64_t ld, double inv_eps, double xs, double* __restrict__ src) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_nodes) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  ff::gather64_node(node, nv, F, ny, nnu, nW, center, u, inv_eps, xs, src);
}

__global__ void k_gather_lobi(bool fp32, int nf, const double* __restrict__ ny, const double* __restrict__ nnu,
                              const double* __restrict__ nW, const double* __restrict__ center,
                              const double* __restrict__ u, const int* kptr, int64_t ld, double inv_eps,
                              double xs, float4* __restrict__ src32, double* __restrict__ src64) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nf) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  if (fp32)
    ff::gather32_lobi(j, nf, ny, nnu, nW, center, u, inv_eps, xs, src32);
  else
    ff::gather64_lobi(j, nf, ny, nnu, nW, center, u, inv_eps, xs, src64);
}

// Padding nodes: far away with zero densities, so every term they add is exactly zero.
__global__ void k_pad(int n_nodes, int n_pad, float4* src32, double* src64) {
  int node = n_nodes + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_pad) return;
  src32[4 * (size_t)node] = make_float4(-1.0e4f, -1.0e4f, -1.0e4f, -1.0e4f);
  src32[4 * (size_t)node + 1] = make_float4(-1.0e4f, -1.0e4f, 0.f, 0.f);
  src32[4 * (size_t)node + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
  src32[4 * (size_t)node + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
  double* o = src64 + 8 * (size_t)node;
  o[0] = o[1] = o[2] = 1.0e4;
  o[3] = o[4] = o[5] = o[6] = o[7] = 0.0;
}

// ------------------------------------------------------------------ far field kernels
// resident blocks per SM the register budget is sized for: 512 threads, or 256 with 8 targets each
template <int NT, int TP>
constexpr int ff32_min_blocks() {
  return (TP >= 4 ? 256 : 512) / NT;
}

template <bool ROW2, bool KS, bool SKIP_SELF, int NT, int TP, int TILE>
__global__ void __launch_bounds__(NT, ff32_min_blocks<NT, TP>())
    k_farfield32(const float4* __restrict__ tgt, int nt, const float4* __restrict__ src, int n_tiles, int tpc,
                 FF32Consts cs, double* __restrict__ part, int64_t ldp, int* err) {
  __shared__ __align__(128) float4 sh[2 * 4 * TILE];
  __shared__ __align__(8) unsigned long long bars[2];
  if (threadIdx.x == 0) ff::tile_barriers_init(bars);
  __syncthreads();
  uint32_t phases = 0;
  const int t0 = blockIdx.y * tpc;
  ff::ff32_block<ROW2, KS, SKIP_SELF, NT, TP, TILE>(tgt, nt, src, t0, min(n_tiles, t0 + tpc), cs,
                                                    part + (size_t)blockIdx.y * ldp, blockIdx.x, sh, bars, phases,
                                                    err);
}

template <bool ROW2, bool KS, bool SKIP_SELF>
__global__ void __launch_bounds__(kFF64Threads)
    k_farfield64(const double* __restrict__ tgt, int nt, const double* __restrict__ src, int n_tiles, int tpc,
                 ff::FF64Consts cs, double* __restrict__ part, int64_t ldp) {
  __shared__ double2 sh[4 * kTile];
  __shared__ double tab[ff::kExpTable];
  ff::exp_table_init(tab);  // read only after the tile loop's first __syncthreads()
  const int t0 = blockIdx.y * tpc;
  ff::ff64_block<ROW2, KS, SKIP_SELF>(tgt, nt, src, t0, min(n_tiles, t0 + tpc), cs, part + (size_t)blockIdx.y * ldp,
                                      blockIdx.x, sh, tab);
}

// The FP64 far field's 1/sqrt(x) and exp(-x), element by element (accuracy tests).
__global__ void k_fp64_pair_functions(const double* __restrict__ x, int64_t n, double* __restrict__ rs,
                                      double* __restrict__ ex) {
  __shared__ double tab[ff::kExpTable];
  ff::exp_table_init(tab);
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  constexpr double kNegLog2eT = -ff::kExpTable * 1.44269504088896340735992468100;
  rs[k] = x[k] > 0.0 ? ff::rsqrt_f64(x[k]) : 1.0 / 0.0;
  ex[k] = ff::exp2_256th(x[k] * kNegLog2eT, tab);
}

// Failure-path check of the source-tile pipeline: one warp initialises the two tile barriers
// exactly as the far-field kernels do and waits, through the same bounded wait, on a phase that no
// copy will complete. The wait gives up after its spin bound and the kernel sets *err like a far-
// field block whose bulk copy never arrived (no copy is in flight, so nothing is left to drain).
__global__ void k_tile_wait_check(int* err) {
  __shared__ __align__(8) unsigned long long bars[2];
  if (threadIdx.x == 0) ff::tile_barriers_init(bars);
  __syncthreads();
  const bool ok = ff::tile_wait(&bars[0], 0u);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, 1);
}

// ------------------------------------------------------------------ combine
// Au_i = (1/2)(1+eps) u_i - [sum_c part_c,i + sum over incident entries of corr . (u_{N_v+v}, u_v)]
// Au_{N_v+i} = (1/2)(1+1/eps) u_{N_v+i} - [...] with the K3/K4 coefficients. Diagonal once.
__global__ void k_combine(int nv, int chunks, const double* __restrict__ part, const int* __restrict__ F,
                          const int* __restrict__ ptr, const int* __restrict__ inc, const double* __restrict__ corr,
                          double eps, const double* __restrict__ u, const int* kptr, int64_t ld,
                          double* __restrict__ Au) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  ff::combine_vertex(i, nv, chunks, part, F, ptr, inc, corr, eps, u, Au);
}

__global__ void k_reduce_points(int np, int chunks, const double* __restrict__ part, double* __restrict__ phi) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[(size_t)c * np + k];
  phi[k] = s;
}

__global__ void k_energy_sum(int nc, const double* __restrict__ Q, const double* __restrict__ phi, double* e) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) s += Q[4 * (size_t)k + 3] * phi[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) e[0] = 0.5 * 4.0 * kPi * kCoulomb * sh[0];
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_gather(bool fp32, int n_nodes, int nv, const int* F, const double* ny,
                          const double* nnu, const double* nW, const double* center, const double* u,
                          const int* kptr, int64_t ld, double inv_eps, double xs, float4* src32, double* src64,
                          cudaStream_t s, const int* pos) {
  if (fp32)
    k_gather32<<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, nv, F, ny, nnu, nW, center, u, kptr, ld, inv_eps, xs,
                                                  src32, pos);
  else
    k_gather64<<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, nv, F, ny, nnu, nW, center, u, kptr, ld, inv_eps, xs,
                                                  src64);
  return cudaGetLastError();
}

cudaError_t launch_gather_lobi(bool fp32, int nf, const double* ny, const double* nnu, const double* nW,
                               const double* center, const double* u, const int* kptr, int64_t ld, double inv_eps,
                               double xs, float4* src32, double* src64, cudaStream_t s) {
  k_gather_lobi<<<nblk(nf, 256), 256, 0, s>>>(fp32, nf, ny, nnu, nW, center, u, kptr, ld, inv_eps, xs, src32,
                                              src64);
  return cudaGetLastError();
}

cudaError_t launch_pad_sources(int n_nodes, int n_pad, float4* src32, double* src64, cudaStream_t s) {
  if (n_pad > n_nodes) k_pad<<<nblk(n_pad - n_nodes, 256), 256, 0, s>>>(n_nodes, n_pad, src32, src64);
  return cudaGetLastError();
}

// FP32 block shapes the planner and the autotuner choose from: threads, target pairs per thread,
// source nodes per shared-memory tile. Shape 0 is the default for large problems; the smaller
// blocks (down to one warp, each with its own tile pipeline) keep 8 targets per thread where
// they can and give more blocks for problems with few targets.
struct FF32Shape {
  int nt, tp, tile;
};
constexpr FF32Shape kShapes[kNumFF32Shapes] = {{32, 4, 128}, {64, 4, 128}, {32, 4, 64}, {32, 2, 64}};

template <bool ROW2, bool KS, bool SKIP>
cudaError_t launch32_shape(int shape, dim3 grid, const float4* tgt, int nt, const float4* src, int n_tiles, int tpc,
                           const FF32Consts& cs, double* part, int64_t ldp, int* err, cudaStream_t s) {
  switch (shape) {
    case 1:
      k_farfield32<ROW2, KS, SKIP, 64, 4, 128><<<grid, 64, 0, s>>>(tgt, nt, src, n_tiles, tpc, cs, part, ldp, err);
      break;
    case 2:
      k_farfield32<ROW2, KS, SKIP, 32, 4, 64><<<grid, 32, 0, s>>>(tgt, nt, src, n_tiles, tpc, cs, part, ldp, err);
      break;
    case 3:
      k_farfield32<ROW2, KS, SKIP, 32, 2, 64><<<grid, 32, 0, s>>>(tgt, nt, src, n_tiles, tpc, cs, part, ldp, err);
      break;
    default:
      k_farfield32<ROW2, KS, SKIP, 32, 4, 128><<<grid, 32, 0, s>>>(tgt, nt, src, n_tiles, tpc, cs, part, ldp, err);
  }
  return cudaGetLastError();
}

template <bool ROW2, bool SKIP>
int occupancy32(int shape) {
  int n = 1;
  switch (shape) {
    case 1:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<ROW2, true, SKIP, 64, 4, 128>, 64, 0);
      break;
    case 2:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<ROW2, true, SKIP, 32, 4, 64>, 32, 0);
      break;
    case 3:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<ROW2, true, SKIP, 32, 2, 64>, 32, 0);
      break;
    default:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<ROW2, true, SKIP, 32, 4, 128>, 32, 0);
  }
  return n > 0 ? n : 1;
}

int farfield_blocks_per_sm(bool fp32, bool row2, int shape) {
  int n = 1;
  if (fp32) return row2 ? occupancy32<true, false>(shape) : occupancy32<false, false>(shape);
  if (row2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield64<true, true, false>, kFF64Threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield64<false, true, false>, kFF64Threads, 0);
  return n > 0 ? n : 1;
}

// Number of source chunks for a shape: (target blocks x chunks) equal-sized blocks filling the
// machine's block slots with the least idle time in the last wave. Tiles are `tile` nodes.
FarFieldPlan plan_farfield(bool fp32, int n_targets, int n_nodes_pad, bool row2, int num_sms, int blocks_per_sm,
                           int shape) {
  FarFieldPlan p;
  p.n_targets = n_targets;
  p.row2 = row2;
  p.shape = fp32 ? shape : 0;
  const int tile = fp32 ? kShapes[p.shape].tile : kTile;
  p.n_tiles = n_nodes_pad / tile;
  const int per_block = fp32 ? kShapes[p.shape].nt * 2 * kShapes[p.shape].tp : kFF64Threads * kFF64Targets;
  const int tt = (n_targets + per_block - 1) / per_block;
  const long slots = (long)num_sms * blocks_per_sm;
  const int cmax = p.n_tiles < 512 ? p.n_tiles : 512;
  double best = -1.0;
  int best_c = 1, best_tpc = p.n_tiles;
  for (int c = 1; c <= cmax; ++c) {
    int tpc = (p.n_tiles + c - 1) / c;
    int chunks = (p.n_tiles + tpc - 1) / tpc;
    long blocks = (long)tt * chunks;
    long waves = (blocks + slots - 1) / slots;
    double eff = (double)tt * p.n_tiles / ((double)waves * slots * tpc);
    if (eff > best * 1.002) {
      best = eff;
      best_c = chunks;
      best_tpc = tpc;
    }
  }
  p.chunks = best_c;
  p.tiles_per_chunk = best_tpc;
  return p;
}

cudaError_t launch_farfield(bool fp32, const FarFieldPlan& p, const float4* tgt32, const double* tgt64,
                            const float4* src32, const double* src64, double eps, double kappa, double* part,
                            int* err, cudaStream_t s, bool skip_self) {
  const int64_t ldp = p.row2 ? 2 * (int64_t)p.n_targets : (int64_t)p.n_targets;
  if (fp32) {
    const FF32Shape& sh = kShapes[p.shape];
    const int per_block = sh.nt * 2 * sh.tp;
    dim3 grid((p.n_targets + per_block - 1) / per_block, p.chunks);
    const FF32Consts cs = ff32_consts(eps, kappa);
    const bool ks = ff32_kappa_scaled(kappa);
    const int nt = p.n_targets, nti = p.n_tiles, tpc = p.tiles_per_chunk;
    if (p.row2 && skip_self)
      return ks ? launch32_shape<true, true, true>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s)
                : launch32_shape<true, false, true>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s);
    if (p.row2)
      return ks ? launch32_shape<true, true, false>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s)
                : launch32_shape<true, false, false>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s);
    return ks ? launch32_shape<false, true, false>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s)
              : launch32_shape<false, false, false>(p.shape, grid, tgt32, nt, src32, nti, tpc, cs, part, ldp, err, s);
  }
  dim3 grid((p.n_targets + kFF64Threads * kFF64Targets - 1) / (kFF64Threads * kFF64Targets), p.chunks);
  const ff::FF64Consts cs = ff::ff64_consts(eps, kappa);
  const bool ks = ff32_kappa_scaled(kappa);
  const int nt = p.n_targets, nti = p.n_tiles, tpc = p.tiles_per_chunk;
  if (p.row2 && skip_self) {
    if (ks) k_farfield64<true, true, true><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
    else k_farfield64<true, false, true><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
  } else if (p.row2) {
    if (ks) k_farfield64<true, true, false><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
    else k_farfield64<true, false, false><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
  } else {
    if (ks) k_farfield64<false, true, false><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
    else k_farfield64<false, false, false><<<grid, kFF64Threads, 0, s>>>(tgt64, nt, src64, nti, tpc, cs, part, ldp);
  }
  return cudaGetLastError();
}

cudaError_t launch_fp64_pair_functions(const double* x, int64_t n, double* rsqrt_x, double* exp_neg_x,
                                       cudaStream_t s) {
  if (n > 0) k_fp64_pair_functions<<<nblk(n, 256), 256, 0, s>>>(x, n, rsqrt_x, exp_neg_x);
  return cudaGetLastError();
}

cudaError_t launch_tile_wait_check(int* err, cudaStream_t s) {
  k_tile_wait_check<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

cudaError_t launch_combine(int nv, int chunks, const double* part, const int* F, const int* inc_ptr,
                           const int* inc_face, const double* corr, double eps, const double* u, const int* kptr,
                           int64_t ld, double* Au, cudaStream_t s) {
  k_combine<<<nblk(nv, 256), 256, 0, s>>>(nv, chunks, part, F, inc_ptr, inc_face, corr, eps, u, kptr, ld, Au);
  return cudaGetLastError();
}

cudaError_t launch_reduce_points(int np, int chunks, const double* part, double* phi, cudaStream_t s) {
  if (np > 0) k_reduce_points<<<nblk(np, 256), 256, 0, s>>>(np, chunks, part, phi);
  return cudaGetLastError();
}

cudaError_t launch_energy_sum(int nc, const double* Q, const double* phi, double* e, cudaStream_t s) {
  k_energy_sum<<<1, 256, 0, s>>>(nc, Q, phi, e);
  return cudaGetLastError();
}

}  // namespace hobi
