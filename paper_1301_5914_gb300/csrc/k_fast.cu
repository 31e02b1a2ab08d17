// k_fast.cu -- fast summation of the far field: a barycentric Lagrange treecode (beyond the
// paper, which evaluates the far field directly and names fast summation as future work; the
// method is Wang, Tlupova and Krasny's kernel-independent treecode, 2020).
//
// The far-field sum of a matvec (the regular-rule part of Eqs. (17)-(18)) is linear in
// the node densities sigma and m with coefficients that are smooth functions of the source
// position away from the target. For a target batch B and a source cluster C that are well
// separated, the sum over C's nodes is replaced by a sum over C's (n+1)^3 tensor Chebyshev
// points (second kind, in C's bounding box) whose densities are the nodes' densities
// interpolated onto them with the barycentric Lagrange basis. Because the pair formula is the
// same, the proxies are simply more source entries in the FP32 source layout, and the
// evaluation kernel is the far-field block of ff_body.cuh run over a list of source segments.
//
// Setup (host): an octree over the nodes (tight boxes, midpoint octants, leaves of at most
// kFastLeaf nodes, depth-first order), target batches by recursive longest-axis splits into sets
// of kFastBatch targets, and per batch the traversal: a cluster of more than (n+1)^3 nodes with
// r_B + r_C < theta |c_B - c_C| is approximated, a leaf otherwise summed directly, an inner
// cluster opened. Each batch's segment list is cut into `chunks` pieces of equal work.
// Per matvec: the gather writes the node densities in tree order, the upward kernels form the
// proxy densities, and one block per (batch, piece) task evaluates it into the piece's partial
// rows, which the usual combine kernel adds up with the singular correction.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ff_body.cuh"

namespace hobi {

// ------------------------------------------------------------------ host: plan construction
namespace {

struct Cluster {
  int begin, end;
  double lo[3], hi[3];
  std::vector<int> children;
};

void tight_box(const double* P, const int* idx, int n, double* lo, double* hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = P[3 * (size_t)idx[0] + d];
    hi[d] = lo[d];
  }
  for (int t = 1; t < n; ++t)
    for (int d = 0; d < 3; ++d) {
      const double v = P[3 * (size_t)idx[t] + d];
      lo[d] = std::min(lo[d], v);
      hi[d] = std::max(hi[d], v);
    }
}

// Octree over the points: tight boxes, a cluster of more than `leaf` points whose box is not a
// point splits into the octants of its box midpoint (coordinate > midpoint is the upper half,
// octant index x + 2y + 4z, empty octants dropped); points listed depth first.
int build_octree(const double* P, std::vector<int>& idx, int leaf, std::vector<Cluster>& cl, std::vector<int>& order) {
  const int ci = (int)cl.size();
  cl.push_back(Cluster());
  cl[ci].begin = (int)order.size();
  double lo[3], hi[3];
  tight_box(P, idx.data(), (int)idx.size(), lo, hi);
  std::memcpy(cl[ci].lo, lo, sizeof lo);
  std::memcpy(cl[ci].hi, hi, sizeof hi);
  const bool flat = !(hi[0] > lo[0] || hi[1] > lo[1] || hi[2] > lo[2]);
  if ((int)idx.size() > leaf && !flat) {
    const double mid[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
    std::vector<int> oct[8];
    for (int t : idx) {
      const double* p = P + 3 * (size_t)t;
      oct[(p[0] > mid[0] ? 1 : 0) + (p[1] > mid[1] ? 2 : 0) + (p[2] > mid[2] ? 4 : 0)].push_back(t);
    }
    std::vector<int>().swap(idx);
    for (int o = 0; o < 8; ++o)
      if (!oct[o].empty()) {
        const int ch = build_octree(P, oct[o], leaf, cl, order);
        cl[ci].children.push_back(ch);
      }
  } else {
    order.insert(order.end(), idx.begin(), idx.end());
  }
  cl[ci].end = (int)order.size();
  return ci;
}

// Target batches: a set of c > batch targets is ordered along the longest axis of its tight box
// (ties by index) and split after floor(ceil(c / batch) / 2) * batch targets.
void build_batches(const double* X, std::vector<int>& idx, int batch, std::vector<Cluster>& out,
                   std::vector<int>& order) {
  double lo[3], hi[3];
  tight_box(X, idx.data(), (int)idx.size(), lo, hi);
  const int c = (int)idx.size();
  if (c <= batch) {
    Cluster b;
    b.begin = (int)order.size();
    b.end = b.begin + c;
    std::memcpy(b.lo, lo, sizeof lo);
    std::memcpy(b.hi, hi, sizeof hi);
    out.push_back(b);
    order.insert(order.end(), idx.begin(), idx.end());
    return;
  }
  int a = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[a] - lo[a]) a = d;
  std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
    const double vp = X[3 * (size_t)p + a], vq = X[3 * (size_t)q + a];
    return vp < vq || (vp == vq && p < q);
  });
  const int cut = (c + batch - 1) / batch / 2 * batch;
  std::vector<int> left(idx.begin(), idx.begin() + cut), right(idx.begin() + cut, idx.end());
  std::vector<int>().swap(idx);
  build_batches(X, left, batch, out, order);
  build_batches(X, right, batch, out, order);
}

void center_radius(const Cluster& c, double* ctr, double* r) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    ctr[d] = 0.5 * (c.lo[d] + c.hi[d]);
    const double e = c.hi[d] - c.lo[d];
    s += e * e;
  }
  *r = 0.5 * std::sqrt(s);
}

void traverse(const std::vector<Cluster>& cl, int ci, const double* cb, double rb, double theta, int n3,
              std::vector<int>& direct, std::vector<int>& approx) {
  const Cluster& c = cl[ci];
  double cc[3], rc;
  center_radius(c, cc, &rc);
  const double dx = cc[0] - cb[0], dy = cc[1] - cb[1], dz = cc[2] - cb[2];
  if (c.end - c.begin > n3 && rb + rc < theta * std::sqrt(dx * dx + dy * dy + dz * dz)) {
    approx.push_back(ci);
  } else if (c.children.empty()) {
    direct.push_back(ci);
  } else {
    for (int ch : c.children) traverse(cl, ch, cb, rb, theta, n3, direct, approx);
  }
}

}  // namespace

void build_fast_plan(const double* y, int n_nodes, const double* x, int nv, const double* center, double xs,
                     int degree, double theta, int resident_blocks, int piece_sources, FastPlanHost* out) {
  FastPlanHost& F = *out;
  F = FastPlanHost();
  const int n1 = degree + 1, n3 = n1 * n1 * n1;
  F.degree = degree;
  // source tree
  std::vector<Cluster> cl;
  std::vector<int> order, idx(n_nodes);
  for (int t = 0; t < n_nodes; ++t) idx[t] = t;
  build_octree(y, idx, kFastLeaf, cl, order);
  F.node_pos.assign(n_nodes, 0);
  for (int p = 0; p < n_nodes; ++p) F.node_pos[order[p]] = p;
  // target batches
  std::vector<Cluster> bt;
  std::vector<int> torder, tidx(nv);
  for (int t = 0; t < nv; ++t) tidx[t] = t;
  build_batches(x, tidx, kFastBatch, bt, torder);
  F.tmap = torder;
  // interaction lists and segments
  std::vector<int> pc_of(cl.size(), -1);
  std::vector<std::vector<int2>> segs(bt.size());
  F.direct_pairs = F.approx_pairs = 0;
  for (size_t b = 0; b < bt.size(); ++b) {
    double cb[3], rb;
    center_radius(bt[b], cb, &rb);
    std::vector<int> direct, approx;
    traverse(cl, 0, cb, rb, theta, n3, direct, approx);
    const int64_t nb = bt[b].end - bt[b].begin;
    for (int ci : direct) {
      // leaves adjacent in tree order are adjacent in memory: fill the previous segment first
      int s = cl[ci].begin;
      if (!segs[b].empty()) {
        int2& last = segs[b].back();
        if (last.x + last.y == s && last.y < kFastSeg) {
          const int add = std::min(kFastSeg - last.y, cl[ci].end - s);
          last.y += add;
          s += add;
        }
      }
      for (; s < cl[ci].end; s += kFastSeg) segs[b].push_back({s, std::min(kFastSeg, cl[ci].end - s)});
      F.direct_pairs += nb * (cl[ci].end - cl[ci].begin);
    }
    for (int ci : approx) {
      if (pc_of[ci] < 0) {
        pc_of[ci] = (int)F.pc_offset.size();
        F.pc_offset.push_back(n_nodes + n3 * (int)(F.pc_offset.size()));
        F.pc_cluster.push_back(ci);
      }
      const int off = F.pc_offset[pc_of[ci]];
      for (int s = 0; s < n3; s += kFastSeg) segs[b].push_back({off + s, std::min(kFastSeg, n3 - s)});
      F.approx_pairs += nb * n3;
    }
  }
  const int npc = (int)F.pc_offset.size();
  F.n_entries = n_nodes + npc * n3;
  // proxy clusters: Chebyshev axes (scaled, relative to the centroid) and upward work items
  F.axes.assign((size_t)npc * 3 * n1, 0.f);
  F.half.assign((size_t)npc * 3, 0.f);
  for (int pc = 0; pc < npc; ++pc) {
    const Cluster& c = cl[F.pc_cluster[pc]];
    double half[3], hmax = 0.0;
    for (int d = 0; d < 3; ++d) {
      half[d] = 0.5 * (c.hi[d] - c.lo[d]);
      hmax = std::max(hmax, half[d]);
    }
    for (int d = 0; d < 3; ++d) {
      half[d] = std::max(half[d], 1e-3 * hmax);
      const double mid = 0.5 * (c.lo[d] + c.hi[d]);
      for (int k = 0; k < n1; ++k)
        F.axes[((size_t)pc * 3 + d) * n1 + k] =
            (float)(xs * (mid + half[d] * std::cos(3.14159265358979323846 * k / degree) - center[d]));
      F.half[(size_t)pc * 3 + d] = (float)(xs * half[d]);
    }
    const int first = (int)F.up.size();
    for (int s = c.begin; s < c.end; s += kFastUpSpan) F.up.push_back({pc, s, std::min(c.end, s + kFastUpSpan)});
    F.pc_items.push_back({first, (int)F.up.size() - first});
  }
  // batches and tasks: every batch's segment list cut into `chunks` pieces of equal work
  const int nb = (int)bt.size();
  int chunks;
  if (piece_sources > 0) {
    int64_t total = 0;
    for (const auto& sg : segs)
      for (const int2& e : sg) total += e.y;
    chunks = (int)((total / std::max(nb, 1) + piece_sources - 1) / piece_sources);
  } else {
    chunks = (8 * resident_blocks + nb - 1) / nb;
  }
  chunks = std::max(1, std::min(chunks, 256));
  F.chunks = chunks;
  std::vector<std::pair<int64_t, FastTask>> tl;
  for (int b = 0; b < nb; ++b) {
    F.batch.push_back({bt[b].begin, bt[b].end - bt[b].begin});
    const int s_first = (int)F.seg.size();
    int64_t total = 0;
    for (const int2& sg : segs[b]) total += sg.y;
    F.seg.insert(F.seg.end(), segs[b].begin(), segs[b].end());
    int64_t acc = 0;
    int s = 0;
    const int ns = (int)segs[b].size();
    for (int c = 0; c < chunks; ++c) {
      const int s0 = s;
      const int64_t goal = total * (c + 1) / chunks;
      while (s < ns && (acc < goal || c == chunks - 1)) acc += segs[b][s++].y;
      int64_t cost = 0;
      for (int q = s0; q < s; ++q) cost += segs[b][q].y;
      tl.push_back({cost, FastTask{b, s_first + s0, s_first + s, c}});
    }
  }
  std::stable_sort(tl.begin(), tl.end(), [](const std::pair<int64_t, FastTask>& a,
                                             const std::pair<int64_t, FastTask>& b2) { return a.first > b2.first; });
  for (auto& t : tl) F.tasks.push_back(t.second);
}

// ------------------------------------------------------------------ device
namespace {

// Barycentric Lagrange basis of the Chebyshev points s[0..n1) (weights (-1)^k, halved at both
// ends) at x; a coordinate within 1e-6 half-extents of a point takes the Kronecker value.
__device__ __forceinline__ void lagrange_row(float x, const float* s, float h, int n1, float* L) {
  int hit = -1;
  for (int k = 0; k < n1; ++k)
    if (hit < 0 && fabsf(x - s[k]) < 1e-6f * h) hit = k;
  if (hit >= 0) {
    for (int k = 0; k < n1; ++k) L[k] = k == hit ? 1.f : 0.f;
    return;
  }
  float den = 0.f;
  for (int k = 0; k < n1; ++k) {
    float w = (k & 1) ? -1.f : 1.f;
    if (k == 0 || k == n1 - 1) w *= 0.5f;
    const float t = w / (x - s[k]);
    L[k] = t;
    den += t;
  }
  const float inv = 1.f / den;
  for (int k = 0; k < n1; ++k) L[k] *= inv;
}

__global__ void k_fast_targets(int nv, const int* __restrict__ tmap, const float4* __restrict__ tgt32,
                               float4* __restrict__ tgtf) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  const int i = tmap[p];
  tgtf[2 * (size_t)p] = tgt32[2 * (size_t)i];
  tgtf[2 * (size_t)p + 1] = tgt32[2 * (size_t)i + 1];
}

constexpr int kUpThreads = 128;
constexpr int kUpNodes = 64;  // nodes whose basis values are staged per pass

// Partial proxy densities (sigma/eps, m) of one work item: nodes [n0, n_end) (tree order) of a
// proxy cluster with Chebyshev axes ax and half-extents hf, to out[p], p = (i N1 + j) N1 + k.
// Nodes go in passes of kUpNodes: the first kUpNodes threads stage each node's L_i(x) L_j(y)
// products, its L_k(z) row and its densities in shared memory. Thread t then owns the pair
// ij = t mod N1^2 and the node group g = t / N1^2 (G groups): it accumulates the N1 proxies
// (ij, k) over the nodes of its group, one shared load of L_i L_j per node and the L_k row
// reused for all k; the groups are added in shared memory at the end.
template <int N1>
struct UpwardShape {
  static constexpr int N2 = N1 * N1, N3 = N2 * N1;
  static constexpr int G = kUpThreads / N2;  // node groups (N2 <= 121 < kUpThreads)
  static constexpr size_t stage_bytes = sizeof(float4) * kUpNodes + sizeof(float) * kUpNodes * (N2 + N1);
  static constexpr size_t bytes = stage_bytes + (G > 1 ? sizeof(float4) * G * N3 : 0);
};

template <int N1>
__device__ __forceinline__ void upward_block(int n0, int n_end, const float* __restrict__ ax,
                                             const float* __restrict__ hf, const float4* __restrict__ srcf,
                                             float4* __restrict__ out, float* dyn) {
  using S = UpwardShape<N1>;
  constexpr int N2 = S::N2, N3 = S::N3, G = S::G;
  float4* sq = reinterpret_cast<float4*>(dyn);
  float* sLxy = dyn + 4 * kUpNodes;      // [kUpNodes][N2]
  float* sLz = sLxy + kUpNodes * N2;     // [kUpNodes][N1]
  const int ij = threadIdx.x % N2, g = threadIdx.x / N2;
  const bool active = g < G;
  float2 a01[N1], a23[N1];  // (sigma/eps, m_x), (m_y, m_z) of proxies (ij, k)
#pragma unroll
  for (int k = 0; k < N1; ++k) a01[k] = a23[k] = make_float2(0.f, 0.f);
  for (int c0 = n0; c0 < n_end; c0 += kUpNodes) {
    const int node = c0 + threadIdx.x;
    if (threadIdx.x < kUpNodes && node < n_end) {
      const float4 A = srcf[4 * (size_t)node], B = srcf[4 * (size_t)node + 1];
      const float4 C = srcf[4 * (size_t)node + 2], D = srcf[4 * (size_t)node + 3];
      float Lx[N1], Ly[N1];
      lagrange_row(-A.x, ax, hf[0], N1, Lx);
      lagrange_row(-A.z, ax + N1, hf[1], N1, Ly);
      lagrange_row(-B.x, ax + 2 * N1, hf[2], N1, sLz + threadIdx.x * N1);
      float* row = sLxy + threadIdx.x * N2;
#pragma unroll
      for (int a = 0; a < N1; ++a)
#pragma unroll
        for (int b = 0; b < N1; ++b) row[a * N1 + b] = Lx[a] * Ly[b];
      sq[threadIdx.x] = make_float4(B.z, C.x, C.z, D.x);  // sigma/eps, m
    }
    __syncthreads();
    if (active) {
      const int cnt = min(kUpNodes, n_end - c0);
      for (int t = g; t < cnt; t += G) {
        const float4 q4 = sq[t];
        const float2 q01 = make_float2(q4.x, q4.y), q23 = make_float2(q4.z, q4.w);
        const float wij = sLxy[t * N2 + ij];
        const float* lz = sLz + t * N1;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          const float w = wij * lz[k];
          const float2 ww = make_float2(w, w);
          a01[k] = __ffma2_rn(ww, q01, a01[k]);
          a23[k] = __ffma2_rn(ww, q23, a23[k]);
        }
      }
    }
    __syncthreads();
  }
  if (G == 1) {
    if (active)
#pragma unroll
      for (int k = 0; k < N1; ++k) out[ij * N1 + k] = make_float4(a01[k].x, a01[k].y, a23[k].x, a23[k].y);
    return;
  }
  float4* red = reinterpret_cast<float4*>(reinterpret_cast<char*>(dyn) + S::stage_bytes);  // [G][N3]
  if (active)
#pragma unroll
    for (int k = 0; k < N1; ++k) red[g * N3 + ij * N1 + k] = make_float4(a01[k].x, a01[k].y, a23[k].x, a23[k].y);
  __syncthreads();
  for (int p = threadIdx.x; p < N3; p += kUpThreads) {
    float4 s = red[p];
    for (int q = 1; q < G; ++q) {  // groups added in a fixed order
      const float4 v = red[q * N3 + p];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    out[p] = s;
  }
}

template <int N1>
__global__ void __launch_bounds__(kUpThreads) k_fast_upward(const FastUpItem* __restrict__ items,
                                                            const float* __restrict__ axes,
                                                            const float* __restrict__ half,
                                                            const float4* __restrict__ srcf,
                                                            float4* __restrict__ partial) {
  extern __shared__ __align__(16) float dyn[];
  const FastUpItem it = items[blockIdx.x];
  upward_block<N1>(it.n0, it.n1, axes + (size_t)it.pc * 3 * N1, half + (size_t)it.pc * 3, srcf,
                   partial + (size_t)blockIdx.x * UpwardShape<N1>::N3, dyn);
}

// The same over the work items of every molecule of a batch that uses fast summation.
template <int N1>
__global__ void __launch_bounds__(kUpThreads) k_fast_upward_batch(const FastUpItemB* __restrict__ items,
                                                                  const MolDesc* __restrict__ mols,
                                                                  const MolState* ms) {
  extern __shared__ __align__(16) float dyn[];
  const FastUpItemB it = items[blockIdx.x];
  if (ms && (ms[it.mol].converged || ms[it.mol].breakdown)) return;
  const MolDesc& d = mols[it.mol];
  upward_block<N1>(it.n0, it.n1, d.faxes + (size_t)it.pc * 3 * N1, d.fhalf + (size_t)it.pc * 3, d.fsrc,
                   d.fpartial + (size_t)it.local * UpwardShape<N1>::N3, dyn);
}

// Proxy source entries: partial densities of each cluster's items added in order, written in
// the FP32 source layout {-s, sigma/eps, m, sigma/eps - sigma} after the tree-ordered nodes.
__device__ __forceinline__ void finish_entry(int pc, int p, const int2* __restrict__ pc_items,
                                             const int* __restrict__ pc_off, const float* __restrict__ axes,
                                             const float4* __restrict__ partial, int n1, float one_minus_eps,
                                             float4* __restrict__ srcf) {
  const int n3 = n1 * n1 * n1;
  const int2 r = pc_items[pc];
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = 0; q < r.y; ++q) {
    const float4 v = partial[(size_t)(r.x + q) * n3 + p];
    s.x += v.x;
    s.y += v.y;
    s.z += v.z;
    s.w += v.w;
  }
  const float* ax = axes + (size_t)pc * 3 * n1;
  const float x = ax[p / (n1 * n1)], y = ax[n1 + (p / n1) % n1], z = ax[2 * n1 + p % n1];
  const float sd = s.x * one_minus_eps;
  float4* o = srcf + 4 * ((size_t)pc_off[pc] + p);
  o[0] = make_float4(-x, -x, -y, -y);
  o[1] = make_float4(-z, -z, s.x, s.x);
  o[2] = make_float4(s.y, s.y, s.z, s.z);
  o[3] = make_float4(s.w, s.w, sd, sd);
}

__global__ void k_fast_finish(int npc, const int2* __restrict__ pc_items, const int* __restrict__ pc_off,
                              const float* __restrict__ axes, const float4* __restrict__ partial, int n1,
                              float one_minus_eps, float4* __restrict__ srcf) {
  const int n3 = n1 * n1 * n1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)npc * n3) return;
  finish_entry((int)(g / n3), (int)(g % n3), pc_items, pc_off, axes, partial, n1, one_minus_eps, srcf);
}

__global__ void k_fast_finish_batch(int npcs, const FastPCB* __restrict__ pcs, const MolDesc* __restrict__ mols,
                                    const MolState* ms, int n1, float one_minus_eps) {
  const int n3 = n1 * n1 * n1;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)npcs * n3) return;
  const FastPCB e = pcs[g / n3];
  if (ms && (ms[e.mol].converged || ms[e.mol].breakdown)) return;
  const MolDesc& d = mols[e.mol];
  finish_entry(e.pc, (int)(g % n3), d.fpcitems, d.fpcoff, d.faxes, d.fpartial, n1, one_minus_eps, d.fsrc);
}

// Evaluation: one one-warp block per (batch, piece) task, running the far-field block over the
// piece's segments into the piece's partial rows. The plan lists tasks longest first and blocks
// are dispatched in index order, so the long tasks start first. (A persistent form, blocks pulling
// tasks from an atomic counter, measured 7 % slower with the same arithmetic.)
template <bool KS>
__global__ void __launch_bounds__(kFastThreads, 8)
    k_fast_eval(const FastTask* __restrict__ tasks, const int2* __restrict__ batch, const int2* __restrict__ seg,
                const float4* __restrict__ srcf, const float4* __restrict__ tgtf, const int* __restrict__ tmap,
                int nv, FF32Consts cs, double* __restrict__ part, int* err) {
  __shared__ __align__(128) float4 sh[2 * 4 * kFastSeg];
  __shared__ __align__(8) unsigned long long bars[2];
  if (threadIdx.x == 0) ff::tile_barriers_init(bars);
  __syncthreads();
  uint32_t phases = 0;
  const FastTask tk = tasks[blockIdx.x];
  const int2 b = batch[tk.batch];
  const ff::SegmentTiles tiles{srcf, seg + tk.s0};
  ff::ff32_core<true, KS, false, kFastThreads, kFF32Targets / 2, kFastSeg>(
      tgtf, b.x, b.x + b.y, tmap, nv, tiles, tk.s1 - tk.s0, cs, part + (size_t)tk.chunk * 2 * nv, sh, bars, phases,
      err);  // a timed-out tile pipeline is reported through err
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_fast_targets(int nv, const int* tmap, const float4* tgt32, float4* tgtf, cudaStream_t s) {
  k_fast_targets<<<nblk(nv, 256), 256, 0, s>>>(nv, tmap, tgt32, tgtf);
  return cudaGetLastError();
}

cudaError_t launch_fast_upward(int nup, const FastUpItem* items, const float* axes, const float* half,
                               float4* srcf, int degree, float4* partial, int npc, const int2* pc_items,
                               const int* pc_off, double eps, cudaStream_t s) {
  const int n1 = degree + 1;
  if (nup > 0) {
    switch (n1) {
#define HOBI_UPWARD_CASE(N) \
  case N:                   \
    k_fast_upward<N><<<nup, kUpThreads, UpwardShape<N>::bytes, s>>>(items, axes, half, srcf, partial); \
    break;
      HOBI_UPWARD_CASE(3)
      HOBI_UPWARD_CASE(4)
      HOBI_UPWARD_CASE(5)
      HOBI_UPWARD_CASE(6)
      HOBI_UPWARD_CASE(7)
      HOBI_UPWARD_CASE(8)
      HOBI_UPWARD_CASE(9)
      HOBI_UPWARD_CASE(10)
      HOBI_UPWARD_CASE(11)
#undef HOBI_UPWARD_CASE
      default:
        return cudaErrorInvalidValue;
    }
  }
  const int64_t n = (int64_t)npc * n1 * n1 * n1;
  if (n > 0)
    k_fast_finish<<<nblk(n, 256), 256, 0, s>>>(npc, pc_items, pc_off, axes, partial, n1, (float)(1.0 - eps), srcf);
  return cudaGetLastError();
}

cudaError_t launch_fast_eval(const FastTask* tasks, int ntasks, const int2* batch, const int2* seg, const float4* srcf,
                             const float4* tgtf, const int* tmap, int nv, double eps, double kappa, double* part,
                             int* err, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const FF32Consts cs = ff32_consts(eps, kappa);
  if (ff32_kappa_scaled(kappa))
    k_fast_eval<true><<<ntasks, kFastThreads, 0, s>>>(tasks, batch, seg, srcf, tgtf, tmap, nv, cs, part, err);
  else
    k_fast_eval<false><<<ntasks, kFastThreads, 0, s>>>(tasks, batch, seg, srcf, tgtf, tmap, nv, cs, part, err);
  return cudaGetLastError();
}

cudaError_t launch_fast_upward_batch(int nitems, const FastUpItemB* items, int npcs, const FastPCB* pcs,
                                     const MolDesc* mols, const MolState* ms, int degree, double eps,
                                     cudaStream_t s) {
  const int n1 = degree + 1;
  if (nitems > 0) {
    switch (n1) {
#define HOBI_UPWARD_CASE(N) \
  case N:                   \
    k_fast_upward_batch<N><<<nitems, kUpThreads, UpwardShape<N>::bytes, s>>>(items, mols, ms); \
    break;
      HOBI_UPWARD_CASE(3)
      HOBI_UPWARD_CASE(4)
      HOBI_UPWARD_CASE(5)
      HOBI_UPWARD_CASE(6)
      HOBI_UPWARD_CASE(7)
      HOBI_UPWARD_CASE(8)
      HOBI_UPWARD_CASE(9)
      HOBI_UPWARD_CASE(10)
      HOBI_UPWARD_CASE(11)
#undef HOBI_UPWARD_CASE
      default:
        return cudaErrorInvalidValue;
    }
  }
  const int64_t n = (int64_t)npcs * n1 * n1 * n1;
  if (n > 0) k_fast_finish_batch<<<nblk(n, 256), 256, 0, s>>>(npcs, pcs, mols, ms, n1, (float)(1.0 - eps));
  return cudaGetLastError();
}

int fast_eval_blocks_per_sm(double kappa) {
  int n = 1;
  if (ff32_kappa_scaled(kappa))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_eval<true>, kFastThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_eval<false>, kFastThreads, 0);
  return n > 0 ? n : 1;
}

}  // namespace hobi
