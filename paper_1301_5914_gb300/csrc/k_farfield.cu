// k_farfield.cu -- the per-iteration hot path of the HOBI-PB matvec (Sec. 2.2-2.3, Eqs. eqdbef3-6).
//
// For every target vertex x_i (unit normal nu_i) and every regular-rule node y (normal nu_y) of
// every element, the far-field kernel accumulates (d = x_i - y, r = |d|, E = exp(-kappa r),
// P = E (1 + kappa r), Q = E (3 + 3 kappa r + kappa^2 r^2)):
//
//   row 1:  (1 - E)/r sigma + (eps P - 1)/r^3 (d . m)
//   row 2:  nu_i . [ (P - 1)/r^3 m + ((P/eps - 1)/r^3 sigma - (Q - 3)/r^5 (d . m)) d ]
//
// with sigma = sum_n W_{j,m,n} u_{N_v + v_n} / (4 pi) and m = nu_y sum_n W_{j,m,n} u_{v_n} / (4 pi).
// Row 1 is the K1/K2 sum of eqdbef3 and row 2 the K3/K4 sum of eqdbef4 (Eq_Ls written out), with
// the target normal pulled out of the source sum so that each pair needs one vector
// accumulation instead of two dot products. Faces incident to x_i are included here and
// replaced by the singular rule through the precomputed correction (combine kernel).
//
// FP32-bulk kernel: each thread keeps 4 targets in registers as two packed pairs and evaluates
// every pair formula with Blackwell's paired FP32 instructions (__ffma2_rn / __fmul2_rn /
// __fadd2_rn: one instruction = the same operation on two targets), which halves the issue
// slots of the FMA-pipe work so that the FMA pipe itself becomes the limit. 256-node source
// tiles are staged in shared memory, each source value stored twice ({v, v}) so one LDS.128
// feeds two packed operands; rsqrt and exp2 go to the MUFU pipe (rsqrt.approx / ex2.approx).
// Each tile's FP32 sum is folded into a compensated (two-float) accumulator, and the result is
// written as FP64 per (source chunk, target); the combine kernel adds the chunks in a fixed order.
#include <math.h>

#include "hobi_internal.cuh"

namespace hobi {
namespace {

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// hi + lo += v, error-free transformation of the addition (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  float s = __fadd_rn(hi, v);
  float bp = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ------------------------------------------------------------------ gather (per matvec)
__global__ void k_gather32(int n_nodes, int nv, const int* __restrict__ F, const double* __restrict__ ny,
                           const double* __restrict__ nnu, const double* __restrict__ nW,
                           const double* __restrict__ center, const double* __restrict__ u, const int* kptr,
                           int64_t ld, double inv_eps, float4* __restrict__ src) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_nodes) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  int j = node >> 2;
  int a = F[3 * j], b = F[3 * j + 1], c = F[3 * j + 2];
  const double* W = nW + 3 * (size_t)node;
  double sig = (W[0] * u[nv + a] + W[1] * u[nv + b] + W[2] * u[nv + c]) * kInv4Pi;
  double mu = (W[0] * u[a] + W[1] * u[b] + W[2] * u[c]) * kInv4Pi;
  const double* y = ny + 3 * (size_t)node;
  const double* n = nnu + 3 * (size_t)node;
  // {-y_x, -y_x, -y_y, -y_y}, {-y_z, -y_z, sigma, sigma}, {m_x, m_x, m_y, m_y}, {m_z, m_z, sigma/eps, sigma/eps}
  const float yx = (float)(center[0] - y[0]), yy = (float)(center[1] - y[1]), yz = (float)(center[2] - y[2]);
  const float sg = (float)sig, se = (float)(sig * inv_eps);
  const float mx = (float)(mu * n[0]), my = (float)(mu * n[1]), mz = (float)(mu * n[2]);
  float4* o = src + 4 * (size_t)node;
  o[0] = make_float4(yx, yx, yy, yy);
  o[1] = make_float4(yz, yz, sg, sg);
  o[2] = make_float4(mx, mx, my, my);
  o[3] = make_float4(mz, mz, se, se);
}

__global__ void k_gather64(int n_nodes, int nv, const int* __restrict__ F, const double* __restrict__ ny,
                           const double* __restrict__ nnu, const double* __restrict__ nW,
                           const double* __restrict__ center, const double* __restrict__ u, const int* kptr,
                           int64_t ld, double* __restrict__ src) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= n_nodes) return;
  if (kptr) u += (int64_t)(*kptr) * ld;
  int j = node >> 2;
  int a = F[3 * j], b = F[3 * j + 1], c = F[3 * j + 2];
  const double* W = nW + 3 * (size_t)node;
  double sig = (W[0] * u[nv + a] + W[1] * u[nv + b] + W[2] * u[nv + c]) * kInv4Pi;
  double mu = (W[0] * u[a] + W[1] * u[b] + W[2] * u[c]) * kInv4Pi;
  const double* y = ny + 3 * (size_t)node;
  const double* n = nnu + 3 * (size_t)node;
  double* o = src + 8 * (size_t)node;
  o[0] = y[0] - center[0];
  o[1] = y[1] - center[1];
  o[2] = y[2] - center[2];
  o[3] = sig;
  o[4] = mu * n[0];
  o[5] = mu * n[1];
  o[6] = mu * n[2];
  o[7] = 0.0;
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

// ------------------------------------------------------------------ far field, FP32 bulk
__device__ __forceinline__ float2 pair_of(float a) { return make_float2(a, a); }

template <bool ROW2>
__global__ void __launch_bounds__(kFF32Threads, 2)
    k_farfield32(const float4* __restrict__ tgt, int nt, const float4* __restrict__ src, int n_tiles, int tpc,
                 float neg_kl2e, float kap, float eps, double* __restrict__ part, int64_t ldp) {
  constexpr int T = kFF32Targets, TP = kFF32Targets / 2, NT = kFF32Threads;
  __shared__ float4 sh[4 * kTile];
  float2 px[TP], py[TP], pz[TP];  // target k = 2p + lane
  float qx[T], qy[T], qz[T];
  float h1[T], l1[T], h2[T], l2[T];
  const int base = blockIdx.x * (NT * T) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = min(base + k * NT, nt - 1);
    float4 a = tgt[2 * (size_t)i], b = tgt[2 * (size_t)i + 1];
    if (k & 1) {
      px[k >> 1].y = a.x; py[k >> 1].y = a.y; pz[k >> 1].y = a.z;
    } else {
      px[k >> 1].x = a.x; py[k >> 1].x = a.y; pz[k >> 1].x = a.z;
    }
    qx[k] = b.x; qy[k] = b.y; qz[k] = b.z;
    h1[k] = l1[k] = h2[k] = l2[k] = 0.f;
  }
  const float2 nk2 = pair_of(neg_kl2e), kap2 = pair_of(kap), eps2 = pair_of(eps);
  const float2 m1 = pair_of(-1.f), three = pair_of(3.f), m3 = pair_of(-3.f);
  const int t0 = blockIdx.y * tpc;
  const int t1 = min(n_tiles, t0 + tpc);
  for (int tile = t0; tile < t1; ++tile) {
    __syncthreads();
    const float4* g = src + (size_t)tile * (4 * kTile);
    for (int q = threadIdx.x; q < 4 * kTile; q += NT) sh[q] = g[q];
    __syncthreads();
    float2 a1[TP], wx[TP], wy[TP], wz[TP];
#pragma unroll
    for (int k = 0; k < TP; ++k) a1[k] = wx[k] = wy[k] = wz[k] = pair_of(0.f);
#pragma unroll 2
    for (int s = 0; s < kTile; ++s) {
      const float4 A = sh[4 * s], B = sh[4 * s + 1], C = sh[4 * s + 2], D = sh[4 * s + 3];
      const float2 nyx = make_float2(A.x, A.y), nyy = make_float2(A.z, A.w), nyz = make_float2(B.x, B.y);
      const float2 sg = make_float2(B.z, B.w), mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w);
      const float2 mz = make_float2(D.x, D.y), se = make_float2(D.z, D.w);
#pragma unroll
      for (int k = 0; k < TP; ++k) {
        const float2 dx = __fadd2_rn(px[k], nyx), dy = __fadd2_rn(py[k], nyy), dz = __fadd2_rn(pz[k], nyz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 r = __fmul2_rn(r2, ir);
        const float2 ea = __fmul2_rn(nk2, r);
        const float2 E = make_float2(exp2_approx(ea.x), exp2_approx(ea.y));
        const float2 aym = __ffma2_rn(dz, mz, __ffma2_rn(dy, my, __fmul2_rn(dx, mx)));  // d . m
        const float2 ir2 = __fmul2_rn(ir, ir);
        const float2 ir3 = __fmul2_rn(ir2, ir);
        const float2 u3 = __fmul2_rn(aym, ir3);                                       // (d . m)/r^3
        const float2 kr = __fmul2_rn(kap2, r);
        const float2 P = __ffma2_rn(E, kr, E);
        // row 1: (1 - E)/r sigma + (eps P - 1)(d . m)/r^3
        a1[k] = __ffma2_rn(__ffma2_rn(make_float2(-E.x, -E.y), ir, ir), sg, a1[k]);
        a1[k] = __ffma2_rn(__ffma2_rn(eps2, P, m1), u3, a1[k]);
        if (ROW2) {
          const float2 Q3 = __ffma2_rn(E, __ffma2_rn(kr, __fadd2_rn(kr, three), three), m3);  // Q - 3
          const float2 w = __ffma2_rn(P, ir3, make_float2(-ir3.x, -ir3.y));                  // (P - 1)/r^3
          const float2 q2 = __fmul2_rn(Q3, ir2);
          // (P/eps - 1) sigma / r^3 - (Q - 3)(d . m)/r^5
          const float2 sv = __ffma2_rn(make_float2(-q2.x, -q2.y), u3,
                                       __fmul2_rn(__ffma2_rn(P, se, make_float2(-sg.x, -sg.y)), ir3));
          wx[k] = __ffma2_rn(w, mx, __ffma2_rn(sv, dx, wx[k]));
          wy[k] = __ffma2_rn(w, my, __ffma2_rn(sv, dy, wy[k]));
          wz[k] = __ffma2_rn(w, mz, __ffma2_rn(sv, dz, wz[k]));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < TP; ++k) {
      two_sum_acc(h1[2 * k], l1[2 * k], a1[k].x);
      two_sum_acc(h1[2 * k + 1], l1[2 * k + 1], a1[k].y);
      if (ROW2) {
        two_sum_acc(h2[2 * k], l2[2 * k], fmaf(qx[2 * k], wx[k].x, fmaf(qy[2 * k], wy[k].x, qz[2 * k] * wz[k].x)));
        two_sum_acc(h2[2 * k + 1], l2[2 * k + 1],
                    fmaf(qx[2 * k + 1], wx[k].y, fmaf(qy[2 * k + 1], wy[k].y, qz[2 * k + 1] * wz[k].y)));
      }
    }
  }
  double* out = part + (size_t)blockIdx.y * ldp;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = base + k * NT;
    if (i < nt) {
      out[i] = (double)h1[k] + (double)l1[k];
      if (ROW2) out[nt + i] = (double)h2[k] + (double)l2[k];
    }
  }
}

// ------------------------------------------------------------------ far field, plain FP64
template <bool ROW2>
__global__ void __launch_bounds__(kFF64Threads)
    k_farfield64(const double* __restrict__ tgt, int nt, const double* __restrict__ src, int n_tiles, int tpc,
                 double kap, double eps, double ieps, double* __restrict__ part, int64_t ldp) {
  constexpr int T = kFF64Targets, NT = kFF64Threads;
  __shared__ double2 sh[4 * kTile];
  double px[T], py[T], pz[T], qx[T], qy[T], qz[T], a1[T], a2[T];
  const int base = blockIdx.x * (NT * T) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = min(base + k * NT, nt - 1);
    const double* t = tgt + 8 * (size_t)i;
    px[k] = t[0]; py[k] = t[1]; pz[k] = t[2];
    qx[k] = t[4]; qy[k] = t[5]; qz[k] = t[6];
    a1[k] = a2[k] = 0.0;
  }
  const int t0 = blockIdx.y * tpc;
  const int t1 = min(n_tiles, t0 + tpc);
  for (int tile = t0; tile < t1; ++tile) {
    __syncthreads();
    const double2* g = reinterpret_cast<const double2*>(src) + (size_t)tile * (4 * kTile);
    for (int q = threadIdx.x; q < 4 * kTile; q += NT) sh[q] = g[q];
    __syncthreads();
    for (int s = 0; s < kTile; ++s) {
      const double2 y01 = sh[4 * s], y2s = sh[4 * s + 1], m01 = sh[4 * s + 2], m2 = sh[4 * s + 3];
#pragma unroll
      for (int k = 0; k < T; ++k) {
        double dx = px[k] - y01.x, dy = py[k] - y01.y, dz = pz[k] - y2s.x;
        double r2 = dx * dx + dy * dy + dz * dz;
        double r = sqrt(r2);
        double ir = 1.0 / r;
        double kr = kap * r;
        double E = exp(-kr);
        double P = E * (1.0 + kr);
        double aym = dx * m01.x + dy * m01.y + dz * m2.x;
        double ir3 = ir * ir * ir;
        a1[k] += (1.0 - E) * ir * y2s.y + (eps * P - 1.0) * ir3 * aym;
        if (ROW2) {
          double Q3 = E * (3.0 + kr * (3.0 + kr)) - 3.0;
          double ir5 = ir3 * ir * ir;
          double w = (P - 1.0) * ir3;
          double sv = (P * ieps - 1.0) * ir3 * y2s.y - Q3 * ir5 * aym;
          a2[k] += qx[k] * (w * m01.x + sv * dx) + qy[k] * (w * m01.y + sv * dy) + qz[k] * (w * m2.x + sv * dz);
        }
      }
    }
  }
  double* out = part + (size_t)blockIdx.y * ldp;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = base + k * NT;
    if (i < nt) {
      out[i] = a1[k];
      if (ROW2) out[nt + i] = a2[k];
    }
  }
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
  double s1 = 0.0, s2 = 0.0;
  const size_t ldp = 2 * (size_t)nv;
  for (int c = 0; c < chunks; ++c) {
    s1 += part[c * ldp + i];
    s2 += part[c * ldp + nv + i];
  }
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
    const int* f = F + 3 * inc[e];
    const double* C = corr + 12 * (size_t)e;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      double dphi = u[nv + f[n]], phi = u[f[n]];
      s1 += C[4 * n] * dphi + C[4 * n + 1] * phi;
      s2 += C[4 * n + 2] * dphi + C[4 * n + 3] * phi;
    }
  }
  Au[i] = 0.5 * (1.0 + eps) * u[i] - s1;
  Au[nv + i] = 0.5 * (1.0 + 1.0 / eps) * u[nv + i] - s2;
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

cudaError_t launch_gather(bool fp32, int n_nodes, int n_pad, int nv, const int* F, const double* ny,
                          const double* nnu, const double* nW, const double* center, const double* u,
                          const int* kptr, int64_t ld, double inv_eps, float4* src32, double* src64,
                          cudaStream_t s) {
  (void)n_pad;
  if (fp32)
    k_gather32<<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, nv, F, ny, nnu, nW, center, u, kptr, ld, inv_eps, src32);
  else
    k_gather64<<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, nv, F, ny, nnu, nW, center, u, kptr, ld, src64);
  return cudaGetLastError();
}

cudaError_t launch_pad_sources(int n_nodes, int n_pad, float4* src32, double* src64, cudaStream_t s) {
  if (n_pad > n_nodes) k_pad<<<nblk(n_pad - n_nodes, 256), 256, 0, s>>>(n_nodes, n_pad, src32, src64);
  return cudaGetLastError();
}

int farfield_blocks_per_sm(bool fp32, bool row2) {
  int n = 1;
  if (fp32) {
    if (row2)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<true>, kFF32Threads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield32<false>, kFF32Threads, 0);
  } else {
    if (row2)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield64<true>, kFF64Threads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_farfield64<false>, kFF64Threads, 0);
  }
  return n > 0 ? n : 1;
}

// Choose the number of source chunks so that (target tiles x chunks) equal-sized blocks fill the
// machine's block slots with the least idle time in the last wave.
FarFieldPlan plan_farfield(bool fp32, int n_targets, int n_nodes_pad, bool row2, int num_sms, int blocks_per_sm) {
  FarFieldPlan p;
  p.n_targets = n_targets;
  p.row2 = row2;
  p.n_tiles = n_nodes_pad / kTile;
  const int per_block = fp32 ? kFF32Threads * kFF32Targets : kFF64Threads * kFF64Targets;
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
                            cudaStream_t s) {
  const int64_t ldp = p.row2 ? 2 * (int64_t)p.n_targets : (int64_t)p.n_targets;
  if (fp32) {
    dim3 grid((p.n_targets + kFF32Threads * kFF32Targets - 1) / (kFF32Threads * kFF32Targets), p.chunks);
    const float neg_kl2e = (float)(-kappa * 1.4426950408889634074);
    if (p.row2)
      k_farfield32<true><<<grid, kFF32Threads, 0, s>>>(tgt32, p.n_targets, src32, p.n_tiles, p.tiles_per_chunk,
                                                       neg_kl2e, (float)kappa, (float)eps, part, ldp);
    else
      k_farfield32<false><<<grid, kFF32Threads, 0, s>>>(tgt32, p.n_targets, src32, p.n_tiles, p.tiles_per_chunk,
                                                        neg_kl2e, (float)kappa, (float)eps, part, ldp);
  } else {
    dim3 grid((p.n_targets + kFF64Threads * kFF64Targets - 1) / (kFF64Threads * kFF64Targets), p.chunks);
    if (p.row2)
      k_farfield64<true><<<grid, kFF64Threads, 0, s>>>(tgt64, p.n_targets, src64, p.n_tiles, p.tiles_per_chunk,
                                                       kappa, eps, 1.0 / eps, part, ldp);
    else
      k_farfield64<false><<<grid, kFF64Threads, 0, s>>>(tgt64, p.n_targets, src64, p.n_tiles, p.tiles_per_chunk,
                                                        kappa, eps, 1.0 / eps, part, ldp);
  }
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
