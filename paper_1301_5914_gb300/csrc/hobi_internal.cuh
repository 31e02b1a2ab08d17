// hobi_internal.cuh -- declarations shared by the CUDA translation units of libhobi.
//
// Data layout in device memory (per handle):
//   V[n_v][3], Nv[n_v][3] (unit), F[n_f][3], Q[n_c][4]        FP64 / int32 inputs
//   elem[n_f][10][3]          the 10 interpolation points of each curved element (FP64)
//   ny[n_n][3], nnu[n_n][3], nW[n_n][3]                        regular-rule nodes, n_n = 4 n_f,
//                                                              node index = 4 j + m (FP64)
//   inc_ptr[n_v+1], inc_face[3 n_f]                            vertex -> incident faces (sorted)
//   corr[3 n_f][3][4]         singular correction per (vertex, incident face) entry (FP64)
//   tgt32[n_v][2] float4      target xs (x - c) and unit normal (FP32 path)
//   tgt64[n_v][8] double      {xs (x - c), 0, unit normal, 0} (FP64 path)
//   src32[n_pad][4] float4    per node, each value twice for paired FP32 math, rebuilt per matvec:
//                             {-xs y}, {sigma/eps}, {m = xs mu nu_y}, {sigma/eps - sigma}
//                             (y relative to c; sigma, mu / 4pi; xs = ff32_coord_scale(kappa))
//   src64[n_pad][8] double    per node, rebuilt per matvec: -xs y, sigma/eps, m = xs mu nu_y,
//                             sigma/eps - sigma (FP64 path; the FP32 quantities, once each)
//   part[chunks][2 n_v]       FP64 far-field partial sums per source chunk
// c is the vertex centroid: both precisions work in coordinates relative to it, scaled by xs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hobi {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * 3.14159265358979323846);
constexpr double kCoulomb = 332.0716;  // kcal A / (mol e^2)

// Far-field tiling (FP32): targets per thread and the FP64 / padding tile. 8 targets per thread
// (4 packed pairs) with 8 warps per SM: fewer warps than 2 targets per thread would allow, but
// more independent pair chains per warp, which hides the MUFU and FMA latencies better. The
// block shapes of the single-molecule kernel are listed below (kNumFF32Shapes).
constexpr int kFF32Threads = 32;
constexpr int kFF32Targets = 8;
constexpr int kTile = 256;
// FP64 path
constexpr int kFF64Threads = 128;
constexpr int kFF64Targets = 2;

// Mesh validation flag bits (setup).
enum MeshFlag : int {
  kBadIndex = 1,
  kOpenOrInconsistent = 2,
  kUnreferencedVertex = 4,
  kBadNormal = 8,
  kNonFinite = 16,
  kNegativeVolume = 32,
  kDegenerateFace = 64,
  kBadCharge = 128,
  kDegenerateElement = 256,
};

// ---- setup kernels (k_setup.cu) ----
// builds inc_ptr/inc_face (rows sorted by face) and entry_vertex[3 nf] (entry -> vertex)
cudaError_t launch_adjacency(int nv, int nf, const int* F, int* deg, int* inc_ptr, int* inc_face,
                             int* entry_vertex, cudaStream_t s);
// validation runs kValidateBlocks blocks; vol_part[kValidateBlocks], center_part[3 kValidateBlocks]
constexpr int kValidateBlocks = 256;
cudaError_t launch_validate(int nv, int nf, int nc, const double* V, const double* Nv_in, const int* F,
                            const int* inc_ptr, const int* inc_face, const double* Q, double* Nv_unit,
                            double* vol_part, double* center_part, int* flags, cudaStream_t s);
cudaError_t launch_finish_validate(int nv, const double* vol_part, const double* center_part, double* center,
                                   int* flags, cudaStream_t s);
// sets kDegenerateElement in *flags if a quadrature node's Jacobian is zero or not finite
cudaError_t launch_node_gen(int nf, const int* F, const double* V, const double* Nv, double* elem, double* ny,
                            double* nnu, double* nW, int* flags, cudaStream_t s);
// one thread per (vertex, incident face) entry; vert[e] is the entry's vertex
cudaError_t launch_correction_entries(int n_entries, const int* vert, const int* F, const double* V,
                                      const double* Nv, const int* inc_face, const double* elem, const double* ny,
                                      const double* nnu, const double* nW, double eps, double kappa, double* corr,
                                      cudaStream_t s);
// LOBI-PB flat-face centroids, unit normals and areas
cudaError_t launch_lobi_geometry(int nf, const int* F, const double* V, double* ny, double* nnu, double* nW,
                                 int* flags, cudaStream_t s);
cudaError_t launch_rhs(int nv, int nc, const double* V, const double* Nv, const double* Q, double eps1,
                       double* b, cudaStream_t s);
// FP32 far-field coordinate scale. For kappa >= kKappaScaledMin the FP32 tables hold coordinates
// (and m) multiplied by kappa, so the kernel's kappa r is the scaled distance itself and the row
// sums are rescaled once per target; below it (kappa = 0 included) they are stored unscaled. The
// bound keeps kappa r far inside the FP32 range for any distance above 1e-6 A.
constexpr double kKappaScaledMin = 1e-6;
inline bool ff32_kappa_scaled(double kappa) { return kappa >= kKappaScaledMin; }
inline double ff32_coord_scale(double kappa) { return ff32_kappa_scaled(kappa) ? kappa : 1.0; }
// Per-launch constants of the FP32 pair arithmetic (row 1 is summed divided by eps).
struct FF32Consts {
  float kap, neg_kl2e, kap_sq;  // unscaled mode: kappa, -kappa log2(e), kappa^2
  float one_minus_inv_eps;      // 1 - 1/eps
  double row1_scale;            // eps xs
  double row2_scale;            // xs^2
};
inline FF32Consts ff32_consts(double eps, double kappa) {
  const double xs = ff32_coord_scale(kappa);
  FF32Consts c;
  c.kap = (float)kappa;
  c.neg_kl2e = (float)(-kappa * 1.4426950408889634074);
  c.kap_sq = (float)(kappa * kappa);
  c.one_minus_inv_eps = (float)(1.0 - 1.0 / eps);
  c.row1_scale = eps * xs;
  c.row2_scale = xs * xs;
  return c;
}
// xs: ff32_coord_scale(kappa), applied to the coordinates of both the FP32 and the FP64 tables.
cudaError_t launch_targets(int nv, const double* V, const double* Nv, const double* center, double xs,
                           float4* tgt32, double* tgt64, cudaStream_t s);
cudaError_t launch_points(int np, const double* P, int stride, const double* center, double xs, float4* tgt32,
                          double* tgt64, cudaStream_t s);

// ---- far field (k_farfield.cu) ----
// Source densities of the current iterate u (2 n_v) for every node; padded nodes stay inert.
// If kptr != nullptr the vector is u + (*kptr) * ld (GMRES basis column).
cudaError_t launch_gather(bool fp32, int n_nodes, int nv, const int* F, const double* ny,
                          const double* nnu, const double* nW, const double* center, const double* u,
                          const int* kptr, int64_t ld, double inv_eps, double xs, float4* src32, double* src64,
                          cudaStream_t s, const int* pos = nullptr);
cudaError_t launch_pad_sources(int n_nodes, int n_pad, float4* src32, double* src64, cudaStream_t s);

// FP32 far-field block shapes (threads, targets per thread, source tile): 0 = 32 x 8, tile 128
// (one warp, 8 blocks per SM); 1 = 64 x 8, tile 128; 2 = 32 x 8, tile 64; 3 = 32 x 4, tile 64
// (small problems). Targets per block: 256, 512, 256, 128.
constexpr int kNumFF32Shapes = 4;
struct FarFieldPlan {
  int n_targets;
  int n_tiles;          // source tiles (of the shape's tile size; kTile for FP64)
  int tiles_per_chunk;
  int chunks;
  bool row2;            // compute the second row (K3, K4) too
  int shape;            // FP32 block shape
};
FarFieldPlan plan_farfield(bool fp32, int n_targets, int n_nodes_pad, bool row2, int num_sms,
                           int blocks_per_sm, int shape = 0);
int farfield_blocks_per_sm(bool fp32, bool row2, int shape = 0);
// skip_self: pairs at zero distance contribute nothing (LOBI-PB, where targets are source nodes).
// err: device flag set to nonzero if the FP32 kernel's tile pipeline timed out (then the partial
// sums are incomplete and the call must be reported as failed).
cudaError_t launch_farfield(bool fp32, const FarFieldPlan& p, const float4* tgt32, const double* tgt64,
                            const float4* src32, const double* src64, double eps, double kappa,
                            double* part, int* err, cudaStream_t s, bool skip_self = false);
// The FP64 far field's own 1/sqrt(x) and exp(-x) on n points (device arrays).
cudaError_t launch_fp64_pair_functions(const double* x, int64_t n, double* rsqrt_x, double* exp_neg_x,
                                       cudaStream_t s);
// One warp waits, with the far-field kernels' bounded wait, on a tile barrier nothing completes,
// and sets *err when the wait gives up (failure-path check).
cudaError_t launch_tile_wait_check(int* err, cudaStream_t s);
// LOBI-PB node densities (one node per face)
cudaError_t launch_gather_lobi(bool fp32, int nf, const double* ny, const double* nnu, const double* nW,
                               const double* center, const double* u, const int* kptr, int64_t ld, double inv_eps,
                               double xs, float4* src32, double* src64, cudaStream_t s);
// Au = diag u - (sum of chunk partials + singular correction)  (rows i and n_v + i)
cudaError_t launch_combine(int nv, int chunks, const double* part, const int* F, const int* inc_ptr,
                           const int* inc_face, const double* corr, double eps, const double* u,
                           const int* kptr, int64_t ld, double* Au, cudaStream_t s);
// phi[k] = sum over chunks of part[c][k]; then e = 0.5 * 4 pi C * sum_k q_k phi[k]
cudaError_t launch_reduce_points(int np, int chunks, const double* part, double* phi, cudaStream_t s);
cudaError_t launch_energy_sum(int nc, const double* Q, const double* phi, double* e, cudaStream_t s);

// Reaction field -grad phi_reac at p.n_targets points (k_field.cu): per chunk of source tiles the
// three components to part[chunk][3][n]; the FP32 plan is shape 0's (32 threads x 8 targets,
// 128-node tiles), the FP64 plan the FP64 far field's. field[3 i + c] = sum over chunks.
int field_blocks_per_sm(bool fp32, double kappa);
cudaError_t launch_field(bool fp32, const FarFieldPlan& p, const float4* t32, const double* t64, const float4* src32,
                         const double* src64, double eps, double kappa, double* part, int* err, cudaStream_t s);
cudaError_t launch_reduce_field(int np, int chunks, const double* part, double* field, cudaStream_t s);
// f[3 k + c] = 4 pi C q_k field[3 k + c], charges Q[n_c][4] (x, y, z, q)
cudaError_t launch_charge_forces(int nc, const double* Q, const double* field, double* f, cudaStream_t s);

// ---- GMRES (k_gmres.cu) ----
struct GmresState {
  int k;          // column being built in the current cycle
  int it;         // total Krylov iterations
  int converged;
  int breakdown;
  double bnorm;
  double rel;     // |g_{k+1}| / ||b||
  double tol;
  double hn;      // last h_{k+1,k}
};
constexpr int kDotBlocks = 296;
cudaError_t launch_dots(const double* Vb, int64_t ld, const double* w, int64_t n, const GmresState* st,
                        int self, double* part, cudaStream_t s);
cudaError_t launch_reduce_dots(const double* part, int m, const GmresState* st, int self, double* c,
                               double* hcol, int accumulate, cudaStream_t s);
cudaError_t launch_axpy_basis(const double* Vb, int64_t ld, const double* c, const GmresState* st, double* w,
                              int64_t n, cudaStream_t s);
cudaError_t launch_givens(GmresState* st, int m, double* H, double* cs, double* sn, double* g,
                          const double* hcol, const double* hn2, cudaStream_t s);
cudaError_t launch_next_basis(double* Vb, int64_t ld, const double* w, int64_t n, GmresState* st,
                              cudaStream_t s);
cudaError_t launch_advance(GmresState* st, cudaStream_t s);
cudaError_t launch_cycle_start(double* Vb, int64_t n, const double* nrm2, GmresState* st, double* g, int m,
                               int first, cudaStream_t s);
// x += D (V y) with D = diag(dscale), or x += V y when dscale is null
cudaError_t launch_finish_cycle(const double* H, int m, const double* g, const GmresState* st, double* y,
                                const double* Vb, int64_t ld, double* x, int64_t n, const double* dscale,
                                cudaStream_t s);
// z = diag(dscale) V_(*kptr) (the Arnoldi vector on the scaled unknowns)
cudaError_t launch_scale_column(const double* Vb, int64_t ld, const int* kptr, const double* dscale, double* z,
                                int64_t n, cudaStream_t s);
// d[i] = lo for i < half, hi for half <= i < 2 half
cudaError_t launch_fill_scale(double* d, int64_t half, double lo, double hi, cudaStream_t s);
cudaError_t launch_residual_start(const double* b, const double* Ax, double* r, int64_t n, cudaStream_t s);
// mixed-precision refinement: x += d; out[0] = ||v||_2 (device scalar)
cudaError_t launch_add_in_place(double* x, const double* d, int64_t n, cudaStream_t s);
cudaError_t launch_norm2(const double* v, int64_t n, double* out, cudaStream_t s);


// ---- batched solve (k_batch.cu) ----
struct MolDesc {          // one molecule's device tables (owned by its single-molecule handle)
  const int* F;
  const double *ny, *nnu, *nW, *center;
  const int *inc_ptr, *inc_face;
  const double* corr;
  const float4* tgt32;
  const double* tgt64;
  float4* src32;
  double* src64;
  double* part;           // [chunks][2 nv] partials of the batched far field
  int nv, n_nodes, chunks;
  double eps;
  double xs;              // coordinate scale of the far-field tables (ff32_coord_scale)
  int64_t u_off;          // offset of the molecule's 2 nv block in the concatenated vectors
  // fast summation of the FP32 far field (fast = 1): tree-ordered node and proxy entries,
  // batch-ordered targets, segments, and the upward tables; fchunks partial rows
  int fast, fchunks;
  const int* fpos;
  float4* fsrc;
  const float4* ftgt;
  const int* ftmap;
  const int2* fseg;
  const int2* fbatch;
  const float* faxes;
  const float* fhalf;
  float4* fpartial;
  const int2* fpcitems;
  const int* fpcoff;
};
struct FFTask {           // one batched far-field work item: targets of block bx, tiles [t0, t1)
  int mol, bx, t0, t1, chunk;
  int fast;               // 1: treecode task, bx = batch, [t0, t1) = segments of the molecule's list
};
struct Segment {          // piece of the concatenated vector inside one molecule
  int64_t start;
  int len, mol;
};
struct BatchState {
  int k;                  // column being built in the current cycle (shared by all molecules)
  int it;                 // batched iterations run
};
struct MolState {
  int converged, breakdown;
  int cols;               // columns this molecule built in the current cycle
  int it;                 // this molecule's Krylov iterations
  double bnorm, rel, tol, hn;
};
constexpr int kSegLen = 4096;
constexpr int kTilesPerTask = 16;  // kTile-node tiles per task (FP64), i.e. 4096 source nodes
// Batched FP32 far field: one one-warp block per task, 8 targets per thread (256 targets per
// task, so a molecule wastes at most 255 target slots) and 128-node tiles, 32 of them per task
// (the same 4096 source nodes per chunk as the FP64 tasks).
constexpr int kBatchFF32Threads = 32;
constexpr int kBatchFF32Tile = 128;
constexpr int kBatchFF32TilesPerTask = kTilesPerTask * kTile / kBatchFF32Tile;
// ---- fast summation of the far field (k_fast.cu): barycentric Lagrange treecode ----
constexpr int kFastLeaf = 256;      // source-tree leaf size (nodes)
constexpr int kFastBatch = 256;     // targets per batch = per evaluation block
constexpr int kFastThreads = 32;    // evaluation block: one warp, 8 targets per thread
constexpr int kFastSeg = 128;       // source entries per segment (one shared-memory stage)
constexpr int kFastUpSpan = 2048;   // nodes per upward work item
constexpr int kFastMaxDegree = 10;
// batches: a molecule uses the treecode when it has at least kFastMinTargets targets and its plan
// needs at most kFastMaxFraction of the direct pair evaluations; pieces of ~kFastPieceSources
constexpr int kFastMinTargets = 4096;
constexpr double kFastMaxFraction = 0.6;
constexpr int kFastPieceSources = 4096;
struct FastTask {                   // one evaluation task: segments [s0, s1) of a batch
  int batch, s0, s1, chunk;
};
struct FastUpItem {                 // nodes [n0, n1) (tree order) of proxy cluster pc
  int pc, n0, n1;
};
struct FastPlanHost {
  int degree = 0, chunks = 1, n_entries = 0;
  int64_t direct_pairs = 0, approx_pairs = 0;
  std::vector<int> node_pos;        // node -> tree position
  std::vector<int> tmap;            // batch order position -> target
  std::vector<int2> batch;          // (first position, count)
  std::vector<int2> seg;            // (source entry, count <= kFastSeg)
  std::vector<FastTask> tasks;      // longest first
  std::vector<FastUpItem> up;
  std::vector<int2> pc_items;       // per proxy cluster: (first item, items)
  std::vector<int> pc_offset;       // per proxy cluster: first proxy entry
  std::vector<int> pc_cluster;      // per proxy cluster: source-tree cluster
  std::vector<float> axes;          // per proxy cluster: 3 x (n+1) scaled Chebyshev coordinates
  std::vector<float> half;          // per proxy cluster: 3 scaled half-extents
};
// y: nodes (n_nodes x 3), x: targets (nv x 3), FP64 absolute coordinates; center and xs as for
// the FP32 tables. Each batch's segment list is cut into `chunks` pieces: enough for about 8
// tasks per resident block (piece_sources = 0), or pieces of about piece_sources source entries.
void build_fast_plan(const double* y, int n_nodes, const double* x, int nv, const double* center, double xs,
                     int degree, double theta, int resident_blocks, int piece_sources, FastPlanHost* out);
cudaError_t launch_fast_targets(int nv, const int* tmap, const float4* tgt32, float4* tgtf, cudaStream_t s);
cudaError_t launch_fast_upward(int nup, const FastUpItem* items, const float* axes, const float* half,
                               float4* srcf, int degree, float4* partial, int npc, const int2* pc_items,
                               const int* pc_off, double eps, cudaStream_t s);
cudaError_t launch_fast_eval(const FastTask* tasks, int ntasks, const int2* batch, const int2* seg, const float4* srcf,
                             const float4* tgtf, const int* tmap, int nv, double eps, double kappa, double* part,
                             int* err, cudaStream_t s);
int fast_eval_blocks_per_sm(double kappa);
// batched treecode upward pass: work items and proxy clusters of every fast molecule
struct FastUpItemB {
  int mol, pc, n0, n1, local;  // local: the item's index among its molecule's items
};
struct FastPCB {
  int mol, pc;
};
cudaError_t launch_fast_upward_batch(int nitems, const FastUpItemB* items, int npcs, const FastPCB* pcs,
                                     const MolDesc* mols, const MolState* ms, int degree, double eps,
                                     cudaStream_t s);

cudaError_t launch_gather_batch(bool fp32, const MolDesc* mols, int nmol, const int64_t* node_off, int64_t total_nodes,
                                const double* u, const int* kptr, int64_t ld, const MolState* ms, cudaStream_t s);
// FP32: one block per task; FP64: `grid` persistent blocks sharing the task counter `counter`
cudaError_t launch_farfield_batch(bool fp32, const MolDesc* mols, const FFTask* tasks, int ntasks, int* counter,
                                  const MolState* ms, double eps, double kappa, int grid, int* err, cudaStream_t s);
int farfield_batch_blocks_per_sm(bool fp32, double kappa);
cudaError_t launch_combine_batch(const MolDesc* mols, int nmol, const int64_t* vert_off, int64_t total_verts,
                                 const double* u, const int* kptr, int64_t ld, double* Au, const MolState* ms,
                                 bool fp32, cudaStream_t s);
cudaError_t launch_bdots(const double* Vb, int64_t ld, const double* w, const Segment* seg, int nseg,
                         const BatchState* gs, const MolState* ms, int self, double* part, cudaStream_t s);
cudaError_t launch_breduce(const double* part, int nseg, const int* mol_seg, int nmol, int m, const BatchState* gs,
                           const MolState* ms, int self, int ldc, double* c, double* hcol, int accumulate,
                           cudaStream_t s);
cudaError_t launch_baxpy(const double* Vb, int64_t ld, const double* c, int ldc, const Segment* seg, int nseg,
                         const BatchState* gs, const MolState* ms, double* w, cudaStream_t s);
cudaError_t launch_bgivens(BatchState* gs, MolState* ms, int nmol, int m, double* H, double* cs, double* sn, double* g,
                           const double* hcol, const double* nrm, int ldc, cudaStream_t s);
cudaError_t launch_bnext(double* Vb, int64_t ld, const double* w, const Segment* seg, int nseg, const BatchState* gs,
                         const MolState* ms, cudaStream_t s);
cudaError_t launch_badvance(BatchState* gs, cudaStream_t s);
cudaError_t launch_bcycle_start(double* Vb, const Segment* seg, int nseg, BatchState* gs, MolState* ms, int nmol,
                                const double* nrm, int ldc, double* g, int m, int first, cudaStream_t s);
cudaError_t launch_bfinish(const double* H, int m, const double* g, const MolState* ms, int nmol, double* y,
                           const double* Vb, int64_t ld, const Segment* seg, int nseg, double* x,
                           const double* dscale, cudaStream_t s);
cudaError_t launch_bresidual(const double* b, const double* Ax, double* r, const Segment* seg, int nseg,
                             const MolState* ms, cudaStream_t s);

}  // namespace hobi
