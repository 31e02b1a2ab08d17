// k_field.cu -- the reaction field -grad phi_reac at points off the surface.
//
// phi_reac is the reaction potential of Sec. 2.5 (the K1/K2 sum of Eq. (23) with the regular rule
// on every element, as for the energy). With d = x - y, r = |d|, E = exp(-kappa r),
// P = E (1 + kappa r) and the far field's node densities sigma, m (k_farfield.cu):
//   phi_reac(x) = sum_nodes (1 - E)/r sigma + (eps P - 1)(d . m)/r^3
// and, since the gradient of E (1 + kappa r) with respect to x is -kappa^2 E d,
//   -grad phi_reac(x) = -eps sum_nodes [ beta d + (P - 1/eps) m ] / r^3,
//   beta = (P - 1) sigma/eps - kappa^2 E (d . m) - 3 (P - 1/eps) (d . m)/r^2.
// The FP32 kernel evaluates it like the far field's row 2 (paired FP32 instructions on
// kappa-scaled coordinates, 128-node source tiles bulk-copied into two shared-memory stages,
// a compensated sum per tile, 28 FMA-pipe operations + 2 MUFU per pair); the FP64 kernel with
// the FP64 far field's 1/sqrt and exp routines. Each writes, per chunk of source tiles, the
// three components of its targets; k_reduce_field adds the chunks in a fixed order.
#include "ff_body.cuh"

namespace hobi {
namespace {

constexpr int kFieldThreads = 32, kFieldPairs = 4, kFieldTile = 128;  // 8 targets per thread

template <bool KS>
__global__ void __launch_bounds__(kFieldThreads, 8)
    k_field32(const float4* __restrict__ tgt, int nt, const float4* __restrict__ src, int n_tiles, int tpc,
              FF32Consts cs, double scale, double* __restrict__ part, int* err) {
  constexpr int NT = kFieldThreads, TP = kFieldPairs, T = 2 * TP, TILE = kFieldTile;
  __shared__ __align__(128) float4 sh[2 * 4 * TILE];
  __shared__ __align__(8) unsigned long long bars[2];
  if (threadIdx.x == 0) ff::tile_barriers_init(bars);
  __syncthreads();
  const int t0 = blockIdx.y * tpc, ntile = min(n_tiles, t0 + tpc) - t0;
  const int base = blockIdx.x * (NT * T) + threadIdx.x;
  float2 px[TP], py[TP], pz[TP];  // target k = 2p + lane
  float hx[T], lx[T], hy[T], ly[T], hz[T], lz[T];
#pragma unroll
  for (int k = 0; k < T; ++k) {
    const float4 a = tgt[2 * (size_t)min(base + k * NT, nt - 1)];
    if (k & 1) {
      px[k >> 1].y = a.x; py[k >> 1].y = a.y; pz[k >> 1].y = a.z;
    } else {
      px[k >> 1].x = a.x; py[k >> 1].x = a.y; pz[k >> 1].x = a.z;
    }
    hx[k] = lx[k] = hy[k] = ly[k] = hz[k] = lz[k] = 0.f;
  }
  constexpr float kLog2e = 1.4426950408889634f;
  const float2 one = ff::pair_of(1.f), m1 = ff::pair_of(-1.f), m3 = ff::pair_of(-3.f);
  const float2 l2e = ff::pair_of(kLog2e), nl2e = ff::pair_of(-kLog2e);
  const float2 kap2 = ff::pair_of(cs.kap), nk2 = ff::pair_of(cs.neg_kl2e), kk2 = ff::pair_of(cs.kap_sq);
  const float2 omie = ff::pair_of(cs.one_minus_inv_eps);
  if (threadIdx.x == 0)
    for (int k = 0; k < 2 && k < ntile; ++k)
      ff::tile_copy(sh + k * 4 * TILE, src + (size_t)(t0 + k) * 4 * TILE, TILE * 4 * sizeof(float4), &bars[k]);
  uint32_t phases = 0;
  for (int kt = 0; kt < ntile; ++kt) {
    const int stage = kt & 1;
    const bool ok = ff::tile_wait(&bars[stage], (phases >> stage) & 1u);
    if (__syncthreads_or(!ok)) {  // a copy never completed: report, drain, stop without writing
      if (threadIdx.x == 0) {
        atomicOr(err, 1);
        for (int j = kt; j < ntile && j < kt + 2; ++j) ff::tile_wait(&bars[j & 1], (phases >> (j & 1)) & 1u);
      }
      return;
    }
    phases ^= 1u << stage;
    const float4* cur = sh + stage * 4 * TILE;
    float2 fx[TP], fy[TP], fz[TP];
#pragma unroll
    for (int k = 0; k < TP; ++k) fx[k] = fy[k] = fz[k] = ff::pair_of(0.f);
    for (int s = 0; s < TILE; ++s) {
      const float4 A = cur[4 * s], B = cur[4 * s + 1], C = cur[4 * s + 2], D = cur[4 * s + 3];
      const float2 nyx = make_float2(A.x, A.y), nyy = make_float2(A.z, A.w), nyz = make_float2(B.x, B.y);
      const float2 se = make_float2(B.z, B.w), mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w);
      const float2 mz = make_float2(D.x, D.y);
#pragma unroll
      for (int k = 0; k < TP; ++k) {
        const float2 dx = __fadd2_rn(px[k], nyx), dy = __fadd2_rn(py[k], nyy), dz = __fadd2_rn(pz[k], nyz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 ir = make_float2(ff::rsqrt_approx(r2.x), ff::rsqrt_approx(r2.y));
        const float2 aym = __ffma2_rn(dz, mz, __ffma2_rn(dy, my, __fmul2_rn(dx, mx)));  // d . m
        const float2 ir2 = __fmul2_rn(ir, ir);
        const float2 v = __fmul2_rn(aym, ir2);
        float2 r1, ea;  // 1 + kappa r, -kappa r log2(e)
        if (KS) {
          r1 = __ffma2_rn(r2, ir, one);
          ea = __ffma2_rn(nl2e, r1, l2e);
        } else {
          const float2 r = __fmul2_rn(r2, ir);
          r1 = __ffma2_rn(kap2, r, one);
          ea = __fmul2_rn(nk2, r);
        }
        const float2 E = make_float2(ff::exp2_approx(ea.x), ff::exp2_approx(ea.y));
        const float2 nE = make_float2(-E.x, -E.y);
        const float2 Pm1 = __ffma2_rn(E, r1, m1);  // P - 1
        const float2 Pe = __fadd2_rn(Pm1, omie);   // P - 1/eps
        const float2 ir3 = __fmul2_rn(ir2, ir);
        // beta = (P - 1) sigma/eps - 3 (P - 1/eps) v - E kappa^2 (d . m)
        const float2 t = __ffma2_rn(m3, __fmul2_rn(Pe, v), __fmul2_rn(KS ? nE : __fmul2_rn(nE, kk2), aym));
        const float2 bs = __fmul2_rn(__ffma2_rn(Pm1, se, t), ir3);
        const float2 as = __fmul2_rn(Pe, ir3);
        fx[k] = __ffma2_rn(as, mx, __ffma2_rn(bs, dx, fx[k]));
        fy[k] = __ffma2_rn(as, my, __ffma2_rn(bs, dy, fy[k]));
        fz[k] = __ffma2_rn(as, mz, __ffma2_rn(bs, dz, fz[k]));
      }
    }
#pragma unroll
    for (int k = 0; k < TP; ++k) {
      ff::two_sum_acc(hx[2 * k], lx[2 * k], fx[k].x);
      ff::two_sum_acc(hx[2 * k + 1], lx[2 * k + 1], fx[k].y);
      ff::two_sum_acc(hy[2 * k], ly[2 * k], fy[k].x);
      ff::two_sum_acc(hy[2 * k + 1], ly[2 * k + 1], fy[k].y);
      ff::two_sum_acc(hz[2 * k], lz[2 * k], fz[k].x);
      ff::two_sum_acc(hz[2 * k + 1], lz[2 * k + 1], fz[k].y);
    }
    __syncthreads();  // every thread has finished reading this stage
    if (threadIdx.x == 0 && kt + 2 < ntile)
      ff::tile_copy(sh + stage * 4 * TILE, src + (size_t)(t0 + kt + 2) * 4 * TILE, TILE * 4 * sizeof(float4),
                    &bars[stage]);
  }
  double* out = part + (size_t)blockIdx.y * 3 * nt;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    const int i = base + k * NT;
    if (i < nt) {
      out[i] = ((double)hx[k] + (double)lx[k]) * scale;
      out[nt + i] = ((double)hy[k] + (double)ly[k]) * scale;
      out[2 * (size_t)nt + i] = ((double)hz[k] + (double)lz[k]) * scale;
    }
  }
}

// FP64: kFF64Threads threads x kFF64Targets targets, kTile-node tiles staged by plain loads.
template <bool KS>
__global__ void __launch_bounds__(kFF64Threads)
    k_field64(const double* __restrict__ tgt, int nt, const double* __restrict__ src, int n_tiles, int tpc,
              ff::FF64Consts cs, double scale, double* __restrict__ part) {
  constexpr int T = kFF64Targets, NT = kFF64Threads;
  __shared__ double2 sh[4 * kTile];
  __shared__ double tab[ff::kExpTable];
  ff::exp_table_init(tab);  // read only after the tile loop's first __syncthreads()
  const int t0 = blockIdx.y * tpc, t1 = min(n_tiles, t0 + tpc);
  const int base = blockIdx.x * (NT * T) + threadIdx.x;
  double px[T], py[T], pz[T], fx[T], fy[T], fz[T];
#pragma unroll
  for (int k = 0; k < T; ++k) {
    const double* t = tgt + 8 * (size_t)min(base + k * NT, nt - 1);
    px[k] = t[0]; py[k] = t[1]; pz[k] = t[2];
    fx[k] = fy[k] = fz[k] = 0.0;
  }
  for (int tile = t0; tile < t1; ++tile) {
    __syncthreads();
    const double2* g = reinterpret_cast<const double2*>(src) + (size_t)tile * (4 * kTile);
    for (int q = threadIdx.x; q < 4 * kTile; q += NT) sh[q] = g[q];
    __syncthreads();
    for (int s = 0; s < kTile; ++s) {
      const double2 A = sh[4 * s], B = sh[4 * s + 1], C = sh[4 * s + 2], D = sh[4 * s + 3];
#pragma unroll
      for (int k = 0; k < T; ++k) {
        const double dx = px[k] + A.x, dy = py[k] + A.y, dz = pz[k] + B.x;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double ir = ff::rsqrt_f64(r2);
        const double r = r2 * ir;
        const double E = ff::exp2_256th(r * cs.c256, tab);
        const double Pm1 = fma(E, KS ? r + 1.0 : fma(cs.kap, r, 1.0), -1.0);  // P - 1
        const double Pe = Pm1 + cs.omie;                                      // P - 1/eps
        const double aym = fma(dz, D.x, fma(dy, C.y, dx * C.x));             // d . m
        const double ir2 = ir * ir, ir3 = ir2 * ir;
        const double v = aym * ir2;
        const double beta = fma(Pm1, B.y, fma(KS ? -E : -E * cs.kap_sq, aym, -3.0 * Pe * v));
        const double bs = beta * ir3, as = Pe * ir3;
        fx[k] = fma(as, C.x, fma(bs, dx, fx[k]));
        fy[k] = fma(as, C.y, fma(bs, dy, fy[k]));
        fz[k] = fma(as, D.x, fma(bs, dz, fz[k]));
      }
    }
  }
  double* out = part + (size_t)blockIdx.y * 3 * nt;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    const int i = base + k * NT;
    if (i < nt) {
      out[i] = fx[k] * scale;
      out[nt + i] = fy[k] * scale;
      out[2 * (size_t)nt + i] = fz[k] * scale;
    }
  }
}

// field[3 i + c] = sum over chunks of part[chunk][c][i], chunks in order
__global__ void k_reduce_field(int np, int chunks, const double* __restrict__ part, double* __restrict__ field) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[((size_t)k * 3 + c) * np + i];
    field[3 * (size_t)i + c] = s;
  }
}

// Reaction-field force on each charge: f[3 k + c] = 4 pi C q_k field[3 k + c] (kcal/(mol A));
// f may be field itself (each thread reads and writes only its own three entries)
__global__ void k_charge_forces(int nc, const double* __restrict__ Q, const double* field, double* f) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  const double s = 4.0 * kPi * kCoulomb * Q[4 * (size_t)k + 3];
  for (int c = 0; c < 3; ++c) f[3 * (size_t)k + c] = s * field[3 * (size_t)k + c];
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int field_blocks_per_sm(bool fp32, double kappa) {
  int n = 1;
  if (fp32 && ff32_kappa_scaled(kappa))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_field32<true>, kFieldThreads, 0);
  else if (fp32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_field32<false>, kFieldThreads, 0);
  else if (ff32_kappa_scaled(kappa))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_field64<true>, kFF64Threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_field64<false>, kFF64Threads, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_field(bool fp32, const FarFieldPlan& p, const float4* t32, const double* t64, const float4* src32,
                         const double* src64, double eps, double kappa, double* part, int* err, cudaStream_t s) {
  if (p.n_targets <= 0) return cudaSuccess;
  const bool ks = ff32_kappa_scaled(kappa);
  const double xs = ff32_coord_scale(kappa);
  const double scale = -eps * xs * xs;
  if (fp32) {
    const dim3 grid(nblk(p.n_targets, kFieldThreads * 2 * kFieldPairs), p.chunks);
    const FF32Consts cs = ff32_consts(eps, kappa);
    if (ks)
      k_field32<true><<<grid, kFieldThreads, 0, s>>>(t32, p.n_targets, src32, p.n_tiles, p.tiles_per_chunk, cs, scale,
                                                      part, err);
    else
      k_field32<false><<<grid, kFieldThreads, 0, s>>>(t32, p.n_targets, src32, p.n_tiles, p.tiles_per_chunk, cs,
                                                       scale, part, err);
  } else {
    const dim3 grid(nblk(p.n_targets, kFF64Threads * kFF64Targets), p.chunks);
    const ff::FF64Consts cs = ff::ff64_consts(eps, kappa);
    if (ks)
      k_field64<true><<<grid, kFF64Threads, 0, s>>>(t64, p.n_targets, src64, p.n_tiles, p.tiles_per_chunk, cs, scale,
                                                     part);
    else
      k_field64<false><<<grid, kFF64Threads, 0, s>>>(t64, p.n_targets, src64, p.n_tiles, p.tiles_per_chunk, cs,
                                                      scale, part);
  }
  return cudaGetLastError();
}

cudaError_t launch_charge_forces(int nc, const double* Q, const double* field, double* f, cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  k_charge_forces<<<nblk(nc, 256), 256, 0, s>>>(nc, Q, field, f);
  return cudaGetLastError();
}

cudaError_t launch_reduce_field(int np, int chunks, const double* part, double* field, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_reduce_field<<<nblk(np, 256), 256, 0, s>>>(np, chunks, part, field);
  return cudaGetLastError();
}

}  // namespace hobi
