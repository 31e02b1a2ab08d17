// k_batch.cu -- many molecules solved together: every GMRES step runs one far-field launch over a
// task list covering all unconverged molecules (FP32: one one-warp block per task; FP64: persistent
// blocks pulling tasks from a counter), plus batched gather, combine and
// FP64 Arnoldi/Givens kernels on the concatenation of the molecules' vectors.
//
// The per-pair arithmetic, the node densities and the combine step are the single-molecule
// device functions (ff_body.cuh), so a batched solve reproduces the single solves.
//
// Concatenated vectors: molecule m owns [u_off_m, u_off_m + 2 N_v,m). The vector is cut into
// segments of at most kSegLen entries that never straddle two molecules; dot products reduce
// per segment and then per molecule over its contiguous segment range, in a fixed order.
#include <math.h>

#include "ff_body.cuh"

namespace hobi {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int find_segment(const int64_t* off, int n, int64_t g) {
  // largest m with off[m] <= g (off has n+1 entries, off[0] = 0)
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool mol_done(const MolState* ms, int m) {
  return ms && (ms[m].converged || ms[m].breakdown);
}

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
  return r;
}

// ---------------------------------------------------------------- matvec pieces
__global__ void k_gather_batch(bool fp32, const MolDesc* __restrict__ mols, int nmol, const int64_t* node_off,
                               int64_t total_nodes, const double* __restrict__ u, const int* kptr, int64_t ld,
                               const MolState* ms) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= total_nodes) return;
  int m = find_segment(node_off, nmol, g);
  if (mol_done(ms, m)) return;
  const MolDesc& d = mols[m];
  const double* um = u + (kptr ? (int64_t)(*kptr) * ld : 0) + d.u_off;
  int node = (int)(g - node_off[m]);
  if (fp32)
    ff::gather32_node(node, d.nv, d.F, d.ny, d.nnu, d.nW, d.center, um, 1.0 / d.eps, d.xs, d.fast ? d.fsrc : d.src32,
                      d.fast ? d.fpos[node] : node);
  else
    ff::gather64_node(node, d.nv, d.F, d.ny, d.nnu, d.nW, d.center, um, 1.0 / d.eps, d.xs, d.src64);
}

// Batched FP32 far field: one one-warp block per task (molecule, target block, source tiles
// [t0, t1) or treecode piece, chunk); blocks of converged molecules return at once. The task list
// is sorted longest first and blocks are dispatched in index order, so the long tasks start first.
// Each task writes its own partial slot, so the result does not depend on the schedule. (A
// persistent form, blocks pulling tasks from an atomic counter, measured 4.5 % slower.)
template <bool KS>
__global__ void __launch_bounds__(kBatchFF32Threads, 8)
    k_farfield_batch32(const MolDesc* __restrict__ mols, const FFTask* __restrict__ tasks, const MolState* ms,
                       FF32Consts cs, int* err) {
  constexpr int kStage = kFastSeg > kBatchFF32Tile ? kFastSeg : kBatchFF32Tile;  // entries per stage
  __shared__ __align__(128) float4 sh[2 * 4 * kStage];
  __shared__ __align__(8) unsigned long long bars[2];
  if (threadIdx.x == 0) ff::tile_barriers_init(bars);
  __syncthreads();
  uint32_t phases = 0;
  const FFTask tk = tasks[blockIdx.x];
  if (mol_done(ms, tk.mol)) return;
  const MolDesc& d = mols[tk.mol];
  double* out = d.part + (size_t)tk.chunk * 2 * d.nv;
  // a timed-out tile pipeline is reported through err
  if (tk.fast) {  // treecode task: a piece of a batch's segment list (direct leaves and proxies)
    const int2 b = d.fbatch[tk.bx];
    const ff::SegmentTiles tiles{d.fsrc, d.fseg + tk.t0};
    ff::ff32_core<true, KS, false, kBatchFF32Threads, kFF32Targets / 2, kFastSeg>(
        d.ftgt, b.x, b.x + b.y, d.ftmap, d.nv, tiles, tk.t1 - tk.t0, cs, out, sh, bars, phases, err);
  } else {
    ff::ff32_block<true, KS, false, kBatchFF32Threads, kFF32Targets / 2, kBatchFF32Tile>(
        d.tgt32, d.nv, d.src32, tk.t0, tk.t1, cs, out, tk.bx, sh, bars, phases, err);
  }
}

// Batched FP64 far field: persistent blocks pull tasks from an atomic counter (reset to 0 before
// each launch) until the list is exhausted; tasks of converged molecules are skipped.
template <bool KS>
__global__ void __launch_bounds__(kFF64Threads)
    k_farfield_batch64(const MolDesc* __restrict__ mols, const FFTask* __restrict__ tasks, int ntasks, int* counter,
                       const MolState* ms, ff::FF64Consts cs) {
  __shared__ double2 sh[4 * kTile];
  __shared__ double tab[ff::kExpTable];
  __shared__ int s_task;
  ff::exp_table_init(tab);  // read only after the barriers below
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntasks) break;
    const FFTask tk = tasks[t];
    if (mol_done(ms, tk.mol)) continue;
    const MolDesc& d = mols[tk.mol];
    ff::ff64_block<true, KS>(d.tgt64, d.nv, d.src64, tk.t0, tk.t1, cs, d.part + (size_t)tk.chunk * 2 * d.nv, tk.bx,
                             sh, tab);
  }
}

__global__ void k_combine_batch(const MolDesc* __restrict__ mols, int nmol, const int64_t* vert_off,
                                int64_t total_verts, const double* __restrict__ u, const int* kptr, int64_t ld,
                                double* __restrict__ Au, const MolState* ms, bool fp32) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= total_verts) return;
  int m = find_segment(vert_off, nmol, g);
  if (mol_done(ms, m)) return;
  const MolDesc& d = mols[m];
  const double* um = u + (kptr ? (int64_t)(*kptr) * ld : 0) + d.u_off;
  ff::combine_vertex((int)(g - vert_off[m]), d.nv, fp32 && d.fast ? d.fchunks : d.chunks, d.part, d.F, d.inc_ptr,
                     d.inc_face, d.corr, d.eps, um, Au + d.u_off);
}

// ---------------------------------------------------------------- GMRES on the concatenation
// part[j * nseg + s] = (V_j . w) over segment s, j = 0..k (self: w . w)
__global__ void k_bdots(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ w,
                        const Segment* __restrict__ seg, int nseg, const BatchState* gs, const MolState* ms,
                        int self, double* __restrict__ part) {
  const int kmax = self ? 0 : gs->k;
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    if (mol_done(ms, sg.mol)) continue;
    for (int j = 0; j <= kmax; ++j) {
      const double* v = self ? w : Vb + (int64_t)j * ld;
      double acc = 0.0;
      for (int i = threadIdx.x; i < sg.len; i += blockDim.x) acc += v[sg.start + i] * w[sg.start + i];
      acc = block_reduce(acc);
      if (threadIdx.x == 0) part[(int64_t)j * nseg + s] = acc;
    }
  }
}

// c[m * ldc + j] = sum over molecule m's segments; hcol[m * ldc + j] = (accumulate ? hcol : 0) + c
__global__ void k_breduce(const double* __restrict__ part, int nseg, const int* __restrict__ mol_seg, int nmol,
                          const BatchState* gs, const MolState* ms, int self, int ldc, double* c, double* hcol,
                          int accumulate) {
  const int m = blockIdx.x, j = blockIdx.y;
  if (m >= nmol || j > (self ? 0 : gs->k) || mol_done(ms, m)) return;
  double acc = 0.0;
  for (int s = mol_seg[m] + threadIdx.x; s < mol_seg[m + 1]; s += blockDim.x) acc += part[(int64_t)j * nseg + s];
  acc = block_reduce(acc);
  if (threadIdx.x == 0) {
    c[m * ldc + j] = acc;
    if (hcol) hcol[m * ldc + j] = accumulate ? hcol[m * ldc + j] + acc : acc;
  }
}

// w -= sum_{j<=k} c[mol][j] V_j over every unconverged molecule's segments
__global__ void k_baxpy(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ c, int ldc,
                        const Segment* __restrict__ seg, int nseg, const BatchState* gs, const MolState* ms,
                        double* __restrict__ w) {
  const int k = gs->k;
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    if (mol_done(ms, sg.mol)) continue;
    const double* cm = c + sg.mol * ldc;
    for (int i = threadIdx.x; i < sg.len; i += blockDim.x) {
      const int64_t gi = sg.start + i;
      double acc = w[gi];
      for (int j = 0; j <= k; ++j) acc -= cm[j] * Vb[(int64_t)j * ld + gi];
      w[gi] = acc;
    }
  }
}

// One thread per molecule: Hessenberg column k, previous rotations, new rotation, residual.
__global__ void k_bgivens(BatchState* gs, MolState* ms, int nmol, int m, double* H, double* cs, double* sn,
                          double* g, const double* hcol, const double* nrm, int ldc) {
  const int mol = blockIdx.x * blockDim.x + threadIdx.x;
  if (mol >= nmol) return;
  MolState& st = ms[mol];
  if (st.converged || st.breakdown) return;
  const int k = gs->k;
  double* Hm = H + (size_t)mol * (m + 1) * m;
  double* csm = cs + (size_t)mol * m;
  double* snm = sn + (size_t)mol * m;
  double* gm = g + (size_t)mol * (m + 1);
  const double* hc = hcol + (size_t)mol * ldc;
  const double hn = sqrt(nrm[(size_t)mol * ldc]);
  for (int j = 0; j <= k; ++j) Hm[j * m + k] = hc[j];
  Hm[(k + 1) * m + k] = hn;
  for (int j = 0; j < k; ++j) {
    double a = Hm[j * m + k], b = Hm[(j + 1) * m + k];
    Hm[j * m + k] = csm[j] * a + snm[j] * b;
    Hm[(j + 1) * m + k] = -snm[j] * a + csm[j] * b;
  }
  double a = Hm[k * m + k], b = Hm[(k + 1) * m + k];
  double den = sqrt(a * a + b * b);
  double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  csm[k] = c;
  snm[k] = s;
  Hm[k * m + k] = den;
  Hm[(k + 1) * m + k] = 0.0;
  gm[k + 1] = -s * gm[k];
  gm[k] = c * gm[k];
  st.hn = hn;
  st.rel = fabs(gm[k + 1]) / st.bnorm;
  st.it += 1;
  st.cols = k + 1;
  if (st.rel <= st.tol) st.converged = 1;
  if (!isfinite(hn) || !isfinite(st.rel) || (!(hn > 0.0) && !st.converged)) st.breakdown = 1;
}

// V_{k+1} = w / h_{k+1,k} for molecules still iterating
__global__ void k_bnext(double* __restrict__ Vb, int64_t ld, const double* __restrict__ w,
                        const Segment* __restrict__ seg, int nseg, const BatchState* gs, const MolState* ms) {
  const int k = gs->k;
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    if (mol_done(ms, sg.mol)) continue;
    const double hn = ms[sg.mol].hn;
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    double* v = Vb + (int64_t)(k + 1) * ld;
    for (int i = threadIdx.x; i < sg.len; i += blockDim.x) v[sg.start + i] = w[sg.start + i] * inv;
  }
}

__global__ void k_badvance(BatchState* gs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    gs->k += 1;
    gs->it += 1;
  }
}

// V_0 = r / ||r|| per molecule, g = (||r||, 0, ...), k = 0, per-molecule cycle column count 0
__global__ void k_bcycle_scale(double* __restrict__ Vb, const Segment* __restrict__ seg, int nseg,
                               const double* nrm, int ldc, const MolState* ms) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    if (mol_done(ms, sg.mol)) continue;
    const double beta = sqrt(nrm[(size_t)sg.mol * ldc]);
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int i = threadIdx.x; i < sg.len; i += blockDim.x) Vb[sg.start + i] *= inv;
  }
}

__global__ void k_bcycle_state(BatchState* gs, MolState* ms, int nmol, const double* nrm, int ldc, double* g, int m,
                               int first) {
  const int mol = blockIdx.x * blockDim.x + threadIdx.x;
  if (mol == 0) gs->k = 0;
  if (mol >= nmol) return;
  MolState& st = ms[mol];
  st.cols = 0;
  if (st.converged || st.breakdown) return;
  const double beta = sqrt(nrm[(size_t)mol * ldc]);
  double* gm = g + (size_t)mol * (m + 1);
  for (int j = 0; j <= m; ++j) gm[j] = 0.0;
  gm[0] = beta;
  if (first) st.bnorm = beta;
  st.rel = st.bnorm > 0.0 ? beta / st.bnorm : 0.0;
  if (!(beta > 0.0) || st.rel <= st.tol) st.converged = 1;
}

// y_m = H_m(0:c,0:c)^{-1} g_m(0:c), c = columns the molecule built in this cycle
__global__ void k_bbacksolve(const double* H, int m, const double* g, const MolState* ms, int nmol, double* y) {
  const int mol = blockIdx.x * blockDim.x + threadIdx.x;
  if (mol >= nmol) return;
  const int k = ms[mol].cols;
  const double* Hm = H + (size_t)mol * (m + 1) * m;
  const double* gm = g + (size_t)mol * (m + 1);
  double* ym = y + (size_t)mol * m;
  for (int i = k - 1; i >= 0; --i) {
    double t = gm[i];
    for (int j = i + 1; j < k; ++j) t -= Hm[i * m + j] * ym[j];
    ym[i] = t / Hm[i * m + i];
  }
}

__global__ void k_bupdate_x(const double* __restrict__ Vb, int64_t ld, const double* __restrict__ y, int m,
                            const Segment* __restrict__ seg, int nseg, const MolState* ms, double* __restrict__ x,
                            const double* __restrict__ dscale) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    const int k = ms[sg.mol].cols;
    if (k == 0) continue;
    const double* ym = y + (size_t)sg.mol * m;
    for (int i = threadIdx.x; i < sg.len; i += blockDim.x) {
      const int64_t gi = sg.start + i;
      if (dscale) {  // scaled unknowns: x += D (V y)
        double t = 0.0;
        for (int j = 0; j < k; ++j) t += ym[j] * Vb[(int64_t)j * ld + gi];
        x[gi] += dscale[gi] * t;
      } else {
        double acc = x[gi];
        for (int j = 0; j < k; ++j) acc += ym[j] * Vb[(int64_t)j * ld + gi];
        x[gi] = acc;
      }
    }
  }
}

__global__ void k_bresidual(const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
                            const Segment* __restrict__ seg, int nseg, const MolState* ms) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment sg = seg[s];
    if (mol_done(ms, sg.mol)) continue;
    for (int i = threadIdx.x; i < sg.len; i += blockDim.x) r[sg.start + i] = b[sg.start + i] - Ax[sg.start + i];
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }
inline int seg_grid(int nseg) { return nseg < 4096 ? (nseg > 0 ? nseg : 1) : 4096; }

}  // namespace

cudaError_t launch_gather_batch(bool fp32, const MolDesc* mols, int nmol, const int64_t* node_off, int64_t total_nodes,
                                const double* u, const int* kptr, int64_t ld, const MolState* ms, cudaStream_t s) {
  k_gather_batch<<<nblk(total_nodes, 256), 256, 0, s>>>(fp32, mols, nmol, node_off, total_nodes, u, kptr, ld, ms);
  return cudaGetLastError();
}

cudaError_t launch_farfield_batch(bool fp32, const MolDesc* mols, const FFTask* tasks, int ntasks, int* counter,
                                  const MolState* ms, double eps, double kappa, int grid, int* err, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (fp32 && ff32_kappa_scaled(kappa)) {
    k_farfield_batch32<true><<<ntasks, kBatchFF32Threads, 0, s>>>(mols, tasks, ms, ff32_consts(eps, kappa), err);
  } else if (fp32) {
    k_farfield_batch32<false><<<ntasks, kBatchFF32Threads, 0, s>>>(mols, tasks, ms, ff32_consts(eps, kappa), err);
  } else {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (ff32_kappa_scaled(kappa))
      k_farfield_batch64<true><<<grid, kFF64Threads, 0, s>>>(mols, tasks, ntasks, counter, ms, ff::ff64_consts(eps, kappa));
    else
      k_farfield_batch64<false><<<grid, kFF64Threads, 0, s>>>(mols, tasks, ntasks, counter, ms, ff::ff64_consts(eps, kappa));
  }
  return cudaGetLastError();
}

int farfield_batch_blocks_per_sm(bool fp32, double kappa) {
  int n = 1;
  if (fp32 && ff32_kappa_scaled(kappa))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield_batch32<true>, kBatchFF32Threads, 0);
  else if (fp32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield_batch32<false>, kBatchFF32Threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield_batch64<true>, kFF64Threads, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_combine_batch(const MolDesc* mols, int nmol, const int64_t* vert_off, int64_t total_verts,
                                 const double* u, const int* kptr, int64_t ld, double* Au, const MolState* ms,
                                 bool fp32, cudaStream_t s) {
  k_combine_batch<<<nblk(total_verts, 256), 256, 0, s>>>(mols, nmol, vert_off, total_verts, u, kptr, ld, Au, ms,
                                                         fp32);
  return cudaGetLastError();
}

cudaError_t launch_bdots(const double* Vb, int64_t ld, const double* w, const Segment* seg, int nseg,
                         const BatchState* gs, const MolState* ms, int self, double* part, cudaStream_t s) {
  k_bdots<<<seg_grid(nseg), kThreads, 0, s>>>(Vb, ld, w, seg, nseg, gs, ms, self, part);
  return cudaGetLastError();
}

cudaError_t launch_breduce(const double* part, int nseg, const int* mol_seg, int nmol, int m, const BatchState* gs,
                           const MolState* ms, int self, int ldc, double* c, double* hcol, int accumulate,
                           cudaStream_t s) {
  dim3 grid(nmol, self ? 1 : m + 1);
  k_breduce<<<grid, kThreads, 0, s>>>(part, nseg, mol_seg, nmol, gs, ms, self, ldc, c, hcol, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_baxpy(const double* Vb, int64_t ld, const double* c, int ldc, const Segment* seg, int nseg,
                         const BatchState* gs, const MolState* ms, double* w, cudaStream_t s) {
  k_baxpy<<<seg_grid(nseg), kThreads, 0, s>>>(Vb, ld, c, ldc, seg, nseg, gs, ms, w);
  return cudaGetLastError();
}

cudaError_t launch_bgivens(BatchState* gs, MolState* ms, int nmol, int m, double* H, double* cs, double* sn, double* g,
                           const double* hcol, const double* nrm, int ldc, cudaStream_t s) {
  k_bgivens<<<nblk(nmol, 64), 64, 0, s>>>(gs, ms, nmol, m, H, cs, sn, g, hcol, nrm, ldc);
  return cudaGetLastError();
}

cudaError_t launch_bnext(double* Vb, int64_t ld, const double* w, const Segment* seg, int nseg, const BatchState* gs,
                         const MolState* ms, cudaStream_t s) {
  k_bnext<<<seg_grid(nseg), kThreads, 0, s>>>(Vb, ld, w, seg, nseg, gs, ms);
  return cudaGetLastError();
}

cudaError_t launch_badvance(BatchState* gs, cudaStream_t s) {
  k_badvance<<<1, 32, 0, s>>>(gs);
  return cudaGetLastError();
}

cudaError_t launch_bcycle_start(double* Vb, const Segment* seg, int nseg, BatchState* gs, MolState* ms, int nmol,
                                const double* nrm, int ldc, double* g, int m, int first, cudaStream_t s) {
  k_bcycle_scale<<<seg_grid(nseg), kThreads, 0, s>>>(Vb, seg, nseg, nrm, ldc, ms);
  k_bcycle_state<<<nblk(nmol, 64), 64, 0, s>>>(gs, ms, nmol, nrm, ldc, g, m, first);
  return cudaGetLastError();
}

cudaError_t launch_bfinish(const double* H, int m, const double* g, const MolState* ms, int nmol, double* y,
                           const double* Vb, int64_t ld, const Segment* seg, int nseg, double* x,
                           const double* dscale, cudaStream_t s) {
  k_bbacksolve<<<nblk(nmol, 64), 64, 0, s>>>(H, m, g, ms, nmol, y);
  k_bupdate_x<<<seg_grid(nseg), kThreads, 0, s>>>(Vb, ld, y, m, seg, nseg, ms, x, dscale);
  return cudaGetLastError();
}

cudaError_t launch_bresidual(const double* b, const double* Ax, double* r, const Segment* seg, int nseg,
                             const MolState* ms, cudaStream_t s) {
  k_bresidual<<<seg_grid(nseg), kThreads, 0, s>>>(b, Ax, r, seg, nseg, ms);
  return cudaGetLastError();
}

}  // namespace hobi
