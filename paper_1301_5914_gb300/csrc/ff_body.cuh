// ff_body.cuh -- the far-field pair sum of one thread block, shared by the single-molecule
// kernels (k_farfield.cu) and the batched kernels (k_batch.cu) so both evaluate
// exactly the same arithmetic. The formulas are documented in k_farfield.cu.
#pragma once

#include <type_traits>

#include "hobi_internal.cuh"

namespace hobi {
namespace ff {

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

__device__ __forceinline__ float2 pair_of(float a) { return make_float2(a, a); }

// ---- source-tile pipeline: 1D bulk asynchronous copies (TMA) completing on mbarriers
// Bounded waits: each mbarrier.try_wait poll suspends for about 4 us when the phase is incomplete
// (measured on GB300), so 2^18 polls give up after about a second; then report and stop.
constexpr int kMaxBarrierSpins = 1 << 18;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Called by one thread, then __syncthreads(): two single-arrival barriers for the two tile stages.
__device__ __forceinline__ void tile_barriers_init(unsigned long long* bars) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])) : "memory");
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global to
// shared memory; completion is signalled on `bar` together with the expected byte count.
__device__ __forceinline__ void tile_copy(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic reads of dst come first
  asm volatile(
      "{\n\t.reg .b64 state;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 state, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait until the barrier's phase with the given parity has completed; false after the spin bound.
__device__ __forceinline__ bool tile_wait(unsigned long long* bar, uint32_t parity) {
  for (int i = 0; i < kMaxBarrierSpins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Source tiles of the FP32 far field. ContigTiles: tiles [t0, t0 + n) of TILE nodes of one
// array. SegmentTiles: a list of (first entry, count <= stage capacity) pieces of one array.
template <int TILE>
struct ContigTiles {
  const float4* src;
  int t0;
  __device__ __forceinline__ const float4* ptr(int k) const { return src + (size_t)(t0 + k) * (4 * TILE); }
  __device__ __forceinline__ int count(int) const { return TILE; }
  __device__ __forceinline__ int first_node(int k) const { return (t0 + k) * TILE; }
};
struct SegmentTiles {
  const float4* src;
  const int2* seg;
  __device__ __forceinline__ const float4* ptr(int k) const { return src + 4 * (size_t)seg[k].x; }
  __device__ __forceinline__ int count(int k) const { return seg[k].y; }
  __device__ __forceinline__ int first_node(int k) const { return seg[k].x; }
};

// One block's FP32 far field: NT threads with 2 TP targets each (targets first + threadIdx.x +
// k NT, below lim) against `ntile` source tiles of at most TILE nodes; results (FP64) to
// out[o] (row 1) and out[ld2 + o] (row 2), o = map[i] (or i without a map). SKIP_SELF: a pair at
// zero distance (a collocation point that is also a source node, LOBI-PB, where target i is
// source node i) contributes nothing; only the tiles that hold some of the block's own targets
// run the pair body with the zero-distance test, the others the plain body.
// KS: coordinates and m are stored multiplied by kappa (FF32Consts), so kappa r is the scaled
// distance itself.
// Tiles stream through two shared-memory stages (sh: 2 x 4 TILE float4) by bulk asynchronous
// copies issued by thread 0, each stage with its mbarrier (bars, initialised by
// tile_barriers_init); `phases` carries the two barriers' parities across calls of one block.
// If a barrier wait exceeds its bound, *err is set, in-flight copies are awaited (bounded) and
// false is returned without writing outputs.
template <bool ROW2, bool KS, bool SKIP_SELF, int NT, int TP, int TILE, class Tiles>
__device__ __forceinline__ bool ff32_core(const float4* __restrict__ tgt, int first, int lim,
                                          const int* __restrict__ map, int ld2, const Tiles& tiles, int ntile,
                                          const FF32Consts& cs, double* __restrict__ out, float4* sh,
                                          unsigned long long* bars, uint32_t& phases, int* err) {
  constexpr int T = 2 * TP;
  constexpr int kUnroll = TP >= 4 ? 1 : 2;  // 4 packed pairs already give enough independent chains
  float2 px[TP], py[TP], pz[TP];  // target k = 2p + lane
  float qx[T], qy[T], qz[T];
  float h1[T], l1[T], h2[T], l2[T];
  const int base = first + threadIdx.x;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = min(base + k * NT, lim - 1);
    float4 a = tgt[2 * (size_t)i], b = tgt[2 * (size_t)i + 1];
    if (k & 1) {
      px[k >> 1].y = a.x; py[k >> 1].y = a.y; pz[k >> 1].y = a.z;
    } else {
      px[k >> 1].x = a.x; py[k >> 1].x = a.y; pz[k >> 1].x = a.z;
    }
    qx[k] = b.x; qy[k] = b.y; qz[k] = b.z;
    h1[k] = l1[k] = h2[k] = l2[k] = 0.f;
  }
  constexpr float kLog2e = 1.4426950408889634f;
  const float2 one = pair_of(1.f), m1 = pair_of(-1.f), m3 = pair_of(-3.f);
  const float2 l2e = pair_of(kLog2e), nl2e = pair_of(-kLog2e);
  const float2 kap2 = pair_of(cs.kap), nk2 = pair_of(cs.neg_kl2e), kk2 = pair_of(cs.kap_sq);
  const float2 omie = pair_of(cs.one_minus_inv_eps);
  __syncthreads();  // the stages are free (a previous call of this block has consumed them)
  if (threadIdx.x == 0)
    for (int k = 0; k < 2 && k < ntile; ++k)
      tile_copy(sh + k * 4 * TILE, tiles.ptr(k), (uint32_t)tiles.count(k) * 4 * sizeof(float4), &bars[k]);
  for (int kt = 0; kt < ntile; ++kt) {  // kt: tile of this call
    const int stage = kt & 1;
    const bool ok = tile_wait(&bars[stage], (phases >> stage) & 1u);
    if (__syncthreads_or(!ok)) {  // a copy never completed: report, drain, stop
      if (threadIdx.x == 0) {
        atomicOr(err, 1);
        for (int j = kt; j < ntile && j < kt + 2; ++j) tile_wait(&bars[j & 1], (phases >> (j & 1)) & 1u);
      }
      return false;
    }
    phases ^= 1u << stage;
    const float4* cur = sh + stage * 4 * TILE;
    const int cnt = tiles.count(kt);
    float2 a1[TP], wx[TP], wy[TP], wz[TP];
#pragma unroll
    for (int k = 0; k < TP; ++k) a1[k] = wx[k] = wy[k] = wz[k] = pair_of(0.f);
    // the tile's pair sums; SELF: with the zero-distance test (a uniform choice per tile)
    auto tile_sum = [&](auto self_tag) {
      constexpr bool SELF = decltype(self_tag)::value;
#pragma unroll kUnroll
    for (int s = 0; s < cnt; ++s) {
      const float4 A = cur[4 * s], B = cur[4 * s + 1], C = cur[4 * s + 2], D = cur[4 * s + 3];
      const float2 nyx = make_float2(A.x, A.y), nyy = make_float2(A.z, A.w), nyz = make_float2(B.x, B.y);
      const float2 se = make_float2(B.z, B.w), mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w);
      const float2 mz = make_float2(D.x, D.y), sd = make_float2(D.z, D.w);
#pragma unroll
      for (int k = 0; k < TP; ++k) {
        const float2 dx = __fadd2_rn(px[k], nyx), dy = __fadd2_rn(py[k], nyy), dz = __fadd2_rn(pz[k], nyz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        if (SELF) {  // 1/r -> 0 before anything else: every term of the pair then vanishes
          ir.x = r2.x > 0.f ? ir.x : 0.f;
          ir.y = r2.y > 0.f ? ir.y : 0.f;
        }
        const float2 aym = __ffma2_rn(dz, mz, __ffma2_rn(dy, my, __fmul2_rn(dx, mx)));  // d . m
        const float2 ir2 = __fmul2_rn(ir, ir);
        const float2 v = __fmul2_rn(aym, ir2);  // (d . m)/r^2
        float2 r1, ea;                          // 1 + kappa r, -kappa r log2(e)
        if (KS) {
          r1 = __ffma2_rn(r2, ir, one);
          ea = __ffma2_rn(nl2e, r1, l2e);
        } else {
          const float2 r = __fmul2_rn(r2, ir);
          r1 = __ffma2_rn(kap2, r, one);
          ea = __fmul2_rn(nk2, r);
        }
        const float2 E = make_float2(exp2_approx(ea.x), exp2_approx(ea.y));
        const float2 nE = make_float2(-E.x, -E.y);
        const float2 Pm1 = __ffma2_rn(E, r1, m1);  // P - 1
        // row 1 / eps = [ (1 - E) sigma/eps + (P - 1/eps)(d . m)/r^2 ] / r
        const float2 g = __ffma2_rn(nE, se, se);
        a1[k] = __ffma2_rn(__ffma2_rn(__fadd2_rn(Pm1, omie), v, g), ir, a1[k]);
        if (ROW2) {
          const float2 ir3 = __fmul2_rn(ir2, ir);
          // S = (P/eps - 1) sigma - (Q - 3)(d . m)/r^2, with Q - 3 = 3 (P - 1) + E (kappa r)^2 and
          // r^2 (d . m)/r^2 = d . m:  S = (P - 1)(sigma/eps - 3 v) + (sigma/eps - sigma) - E kappa^2 (d . m)
          const float2 t = __ffma2_rn(Pm1, __ffma2_rn(m3, v, se), sd);
          const float2 S = __ffma2_rn(KS ? nE : __fmul2_rn(nE, kk2), aym, t);
          const float2 w = __fmul2_rn(Pm1, ir3);  // (P - 1)/r^3
          const float2 sv = __fmul2_rn(S, ir3);
          wx[k] = __ffma2_rn(w, mx, __ffma2_rn(sv, dx, wx[k]));
          wy[k] = __ffma2_rn(w, my, __ffma2_rn(sv, dy, wy[k]));
          wz[k] = __ffma2_rn(w, mz, __ffma2_rn(sv, dz, wz[k]));
        }
      }
    }
    };
    if constexpr (SKIP_SELF) {
      const int n0 = tiles.first_node(kt);
      if (n0 < first + NT * T && n0 + cnt > first)
        tile_sum(std::true_type{});
      else
        tile_sum(std::false_type{});
    } else {
      tile_sum(std::false_type{});
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
    __syncthreads();  // every thread has finished reading this stage
    if (threadIdx.x == 0 && kt + 2 < ntile)
      tile_copy(sh + stage * 4 * TILE, tiles.ptr(kt + 2), (uint32_t)tiles.count(kt + 2) * 4 * sizeof(float4),
                &bars[stage]);
  }
#pragma unroll
  for (int k = 0; k < T; ++k) {
    const int i = base + k * NT;
    if (i < lim) {
      const int o = map ? map[i] : i;
      out[o] = ((double)h1[k] + (double)l1[k]) * cs.row1_scale;
      if (ROW2) out[ld2 + o] = ((double)h2[k] + (double)l2[k]) * cs.row2_scale;
    }
  }
  return true;
}

// One block's share of the FP32 far field over contiguous tiles: targets bx*NT*2TP ... of nt,
// source tiles [t0, t1) of TILE nodes, rows to out[i] and out[nt + i] (see ff32_core).
template <bool ROW2, bool KS, bool SKIP_SELF = false, int NT = kFF32Threads, int TP = kFF32Targets / 2,
          int TILE = kTile>
__device__ __forceinline__ bool ff32_block(const float4* __restrict__ tgt, int nt, const float4* __restrict__ src,
                                           int t0, int t1, const FF32Consts& cs, double* __restrict__ out, int bx,
                                           float4* sh, unsigned long long* bars, uint32_t& phases, int* err) {
  const ContigTiles<TILE> tiles{src, t0};
  return ff32_core<ROW2, KS, SKIP_SELF, NT, TP, TILE>(tgt, bx * (NT * 2 * TP), nt, nullptr, nt, tiles, t1 - t0, cs,
                                                       out, sh, bars, phases, err);
}

// ---- FP64 pair primitives. GB300 runs double-precision FMA/add/multiply at about 1/64 of the
// FP32 rate, but its MUFU pipe returns 1/sqrt and 1/x seeds for doubles (rsqrt.approx.f64) at the
// FP32 MUFU rate, and integer work runs beside both. So the FP64 far field takes 1/r from the MUFU
// seed plus one Newton step, and exp(-kappa r) from a table plus a short polynomial, instead of the
// library's full-range sqrt, division and exp: 44 FP64-pipe operations per pair instead of ~70.

// 1/sqrt(x), x > 0 normal: seed y0 = rsqrt.approx.f64(x), then with e = 1 - x y0^2 (so that
// x y0^2 = 1 - e), 1/sqrt(x) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + O(e^3)). With the seed's
// relative error below 2^-20 the truncation is below 2^-58; the result is within a few units in
// the last place (checked against numpy in the tests). 5 FP64 operations (+1 MUFU).
__device__ __forceinline__ double rsqrt_f64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double p = fma(e, 0.375, 0.5);
  return fma(y * e, p, y);
}

// 2^(j/256), j = 0..255, in shared memory: each FP64 far-field block fills it once (exp2 from the
// CUDA math library; one evaluation per thread).
constexpr int kExpTable = 256;
__device__ __forceinline__ void exp_table_init(double* tab) {
  for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) tab[j] = exp2((double)j / kExpTable);
}

// 2^(t/256) for -2^51 < t <= 0 by Tang's table-driven method (ACM TOMS 15(2), 1989) with a 256-entry
// table: t = n + f with n = round(t) (the 1.5 * 2^52 shift puts n in the low word) and |f| <= 1/2
// exact, 2^(t/256) = 2^floor(n/256) * 2^((n mod 256)/256) * exp(f ln2/256), the last factor by its
// Taylor polynomial of degree 4 (|f ln2/256| <= 0.00136, truncation below 4e-17). The power of two
// is added to the exponent field; n is clamped at -256 * 1021 (the result stays a normal double,
// at most 2^-1020), so t below that (e^-707.7 and smaller: padding nodes, distant pairs) gives a
// value within 5e-308 of the true one. 3 + 4 + 1 FP64 operations; the rest is integer work.
__device__ __forceinline__ double exp2_256th(double t, const double* __restrict__ tab) {
  constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52
  constexpr double c = 0.693147180559945309417232121458 / kExpTable;  // ln(2) / 256
  constexpr double k2 = c * c / 2.0, k3 = k2 * c / 3.0, k4 = k3 * c / 4.0;
  const double nd = t + kShift;
  const double f = t - (nd - kShift);
  // n = nd - kShift as integers (exact for |t| < 2^51), clamped before it is narrowed to 32 bits
  const long long n64 = __double_as_longlong(nd) - __double_as_longlong(kShift);
  const int n = (int)max(n64, (long long)(-kExpTable * 1021));
  const double p = fma(fma(fma(fma(k4, f, k3), f, k2), f, c), f, 1.0);
  const double v = tab[n & (kExpTable - 1)] * p;
  return __hiloint2double(__double2hiint(v) + (n >> 8) * (1 << 20), __double2loint(v));
}

// Per-launch constants of the FP64 pair arithmetic (row 1 is summed divided by eps).
struct FF64Consts {
  double c256;        // -256 log2(e) (kappa-scaled tables) or -256 kappa log2(e): 2^(c256 r / 256) = E
  double kap, kap_sq; // unscaled mode: kappa, kappa^2
  double omie;        // 1 - 1/eps
  double row1_scale;  // eps xs
  double row2_scale;  // xs^2
};
inline FF64Consts ff64_consts(double eps, double kappa) {
  const double xs = ff32_coord_scale(kappa);
  constexpr double kLog2e = 1.44269504088896340735992468100;
  FF64Consts c;
  c.c256 = -kExpTable * kLog2e * (ff32_kappa_scaled(kappa) ? 1.0 : kappa);
  c.kap = kappa;
  c.kap_sq = kappa * kappa;
  c.omie = 1.0 - 1.0 / eps;
  c.row1_scale = eps * xs;
  c.row2_scale = xs * xs;
  return c;
}

// One block's share of the FP64 far field (2 targets per thread): targets bx*NT*T ... of nt,
// source tiles [t0, t1) of kTile nodes; sh: 4 kTile double2, tab: the exp table (initialised,
// with a __syncthreads() between, before the first call). The FP32 kernel's multiplied-out pair
// formula in double precision, with the same table layout:
//   targets: {xs (x - c), 0, nu_x, 0}; sources: {-xs (y - c), sigma/eps, xs m, sigma/eps - sigma}
// where xs = kappa for kappa-scaled tables (KS), else 1; then kappa r is the scaled r (KS).
template <bool ROW2, bool KS, bool SKIP_SELF = false>
__device__ __forceinline__ void ff64_block(const double* __restrict__ tgt, int nt, const double* __restrict__ src,
                                           int t0, int t1, const FF64Consts& cs, double* __restrict__ out, int bx,
                                           double2* sh, const double* __restrict__ tab) {
  constexpr int T = kFF64Targets, NT = kFF64Threads;
  double px[T], py[T], pz[T], qx[T], qy[T], qz[T], a1[T], wx[T], wy[T], wz[T];
  const int base = bx * (NT * T) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = min(base + k * NT, nt - 1);
    const double* t = tgt + 8 * (size_t)i;
    px[k] = t[0]; py[k] = t[1]; pz[k] = t[2];
    qx[k] = t[4]; qy[k] = t[5]; qz[k] = t[6];
    a1[k] = wx[k] = wy[k] = wz[k] = 0.0;
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
        double ir = rsqrt_f64(r2);
        if (SKIP_SELF) ir = r2 > 0.0 ? ir : 0.0;  // every term of a zero-distance pair then vanishes
        const double r = r2 * ir;
        const double E = exp2_256th(r * cs.c256, tab);
        const double Pm1 = fma(E, KS ? r + 1.0 : fma(cs.kap, r, 1.0), -1.0);  // P - 1
        const double aym = fma(dz, D.x, fma(dy, C.y, dx * C.x));             // d . m
        const double ir2 = ir * ir;
        const double v = aym * ir2;
        // row 1 / eps = [ (1 - E) sigma/eps + (P - 1 + 1 - 1/eps) v ] / r
        a1[k] = fma(fma(Pm1 + cs.omie, v, fma(-E, B.y, B.y)), ir, a1[k]);
        if (ROW2) {
          // S = (P - 1)(sigma/eps - 3 v) + (sigma/eps - sigma) - E kappa^2 (d . m)
          const double S = fma(KS ? -E : -E * cs.kap_sq, aym, fma(Pm1, fma(-3.0, v, B.y), D.y));
          const double ir3 = ir2 * ir;
          const double w = Pm1 * ir3, sv = S * ir3;
          wx[k] = fma(w, C.x, fma(sv, dx, wx[k]));
          wy[k] = fma(w, C.y, fma(sv, dy, wy[k]));
          wz[k] = fma(w, D.x, fma(sv, dz, wz[k]));
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < T; ++k) {
    int i = base + k * NT;
    if (i < nt) {
      out[i] = a1[k] * cs.row1_scale;
      if (ROW2) out[nt + i] = fma(qx[k], wx[k], fma(qy[k], wy[k], qz[k] * wz[k])) * cs.row2_scale;
    }
  }
}

// Node densities of the iterate u for one node (Sec. 2.2, W_{j,m,n} with linear density
// interpolation): sigma = sum_n W u_{N_v+v_n}/4pi, mu = sum_n W u_{v_n}/4pi; the FP32 layout
// stores each value twice for the paired arithmetic: {-xs y}, {sigma/eps}, {m = xs mu nu_y},
// {sigma/eps - sigma}, where xs is the far field's coordinate scale (ff32_coord_scale).
__device__ __forceinline__ void gather32_node(int node, int nv, const int* __restrict__ F,
                                              const double* __restrict__ ny, const double* __restrict__ nnu,
                                              const double* __restrict__ nW, const double* __restrict__ center,
                                              const double* __restrict__ u, double inv_eps, double xs,
                                              float4* __restrict__ src, int slot) {
  int j = node >> 2;
  int a = F[3 * j], b = F[3 * j + 1], c = F[3 * j + 2];
  const double* W = nW + 3 * (size_t)node;
  double sig = (W[0] * u[nv + a] + W[1] * u[nv + b] + W[2] * u[nv + c]) * kInv4Pi;
  double mu = (W[0] * u[a] + W[1] * u[b] + W[2] * u[c]) * kInv4Pi;
  const double* y = ny + 3 * (size_t)node;
  const double* n = nnu + 3 * (size_t)node;
  const float yx = (float)(xs * (center[0] - y[0])), yy = (float)(xs * (center[1] - y[1])),
              yz = (float)(xs * (center[2] - y[2]));
  const float se = (float)(sig * inv_eps), sd = (float)(sig * inv_eps - sig);
  const double xm = xs * mu;
  const float mx = (float)(xm * n[0]), my = (float)(xm * n[1]), mz = (float)(xm * n[2]);
  float4* o = src + 4 * (size_t)slot;
  o[0] = make_float4(yx, yx, yy, yy);
  o[1] = make_float4(yz, yz, se, se);
  o[2] = make_float4(mx, mx, my, my);
  o[3] = make_float4(mz, mz, sd, sd);
}

// FP64 layout of the same node: {-xs y}, sigma/eps, {m = xs mu nu_y}, sigma/eps - sigma (y
// relative to the centroid c), one double each.
__device__ __forceinline__ void gather64_node(int node, int nv, const int* __restrict__ F,
                                              const double* __restrict__ ny, const double* __restrict__ nnu,
                                              const double* __restrict__ nW, const double* __restrict__ center,
                                              const double* __restrict__ u, double inv_eps, double xs,
                                              double* __restrict__ src) {
  int j = node >> 2;
  int a = F[3 * j], b = F[3 * j + 1], c = F[3 * j + 2];
  const double* W = nW + 3 * (size_t)node;
  double sig = (W[0] * u[nv + a] + W[1] * u[nv + b] + W[2] * u[nv + c]) * kInv4Pi;
  double mu = (W[0] * u[a] + W[1] * u[b] + W[2] * u[c]) * kInv4Pi;
  const double* y = ny + 3 * (size_t)node;
  const double* n = nnu + 3 * (size_t)node;
  const double xm = xs * mu;
  double* o = src + 8 * (size_t)node;
  o[0] = xs * (center[0] - y[0]);
  o[1] = xs * (center[1] - y[1]);
  o[2] = xs * (center[2] - y[2]);
  o[3] = sig * inv_eps;
  o[4] = xm * n[0];
  o[5] = xm * n[1];
  o[6] = xm * n[2];
  o[7] = sig * inv_eps - sig;
}

// LOBI-PB node = face j: centroid y_j, face normal nu_j, weight A_j (area), densities from the
// centroid unknowns u_j, u_{N_f+j} (Sec. 2.4, Eqs. (21)/(22)).
__device__ __forceinline__ void gather32_lobi(int j, int nf, const double* __restrict__ ny,
                                              const double* __restrict__ nnu, const double* __restrict__ nW,
                                              const double* __restrict__ center, const double* __restrict__ u,
                                              double inv_eps, double xs, float4* __restrict__ src) {
  const double A = nW[3 * (size_t)j];
  const double sig = A * u[nf + j] * kInv4Pi, mu = A * u[j] * kInv4Pi;
  const double* y = ny + 3 * (size_t)j;
  const double* n = nnu + 3 * (size_t)j;
  const float yx = (float)(xs * (center[0] - y[0])), yy = (float)(xs * (center[1] - y[1])),
              yz = (float)(xs * (center[2] - y[2]));
  const float se = (float)(sig * inv_eps), sd = (float)(sig * inv_eps - sig);
  const double xm = xs * mu;
  const float mx = (float)(xm * n[0]), my = (float)(xm * n[1]), mz = (float)(xm * n[2]);
  float4* o = src + 4 * (size_t)j;
  o[0] = make_float4(yx, yx, yy, yy);
  o[1] = make_float4(yz, yz, se, se);
  o[2] = make_float4(mx, mx, my, my);
  o[3] = make_float4(mz, mz, sd, sd);
}

__device__ __forceinline__ void gather64_lobi(int j, int nf, const double* __restrict__ ny,
                                              const double* __restrict__ nnu, const double* __restrict__ nW,
                                              const double* __restrict__ center, const double* __restrict__ u,
                                              double inv_eps, double xs, double* __restrict__ src) {
  const double A = nW[3 * (size_t)j];
  const double sig = A * u[nf + j] * kInv4Pi, mu = A * u[j] * kInv4Pi;
  const double* y = ny + 3 * (size_t)j;
  const double* n = nnu + 3 * (size_t)j;
  const double xm = xs * mu;
  double* o = src + 8 * (size_t)j;
  o[0] = xs * (center[0] - y[0]);
  o[1] = xs * (center[1] - y[1]);
  o[2] = xs * (center[2] - y[2]);
  o[3] = sig * inv_eps;
  o[4] = xm * n[0];
  o[5] = xm * n[1];
  o[6] = xm * n[2];
  o[7] = sig * inv_eps - sig;
}

// Au_i = (1/2)(1+eps) u_i - [sum_c part_c,i + sum over incident entries of corr . (u_{N_v+v}, u_v)]
// Au_{N_v+i} = (1/2)(1+1/eps) u_{N_v+i} - [...] with the K3/K4 coefficients. Diagonal once.
__device__ __forceinline__ void combine_vertex(int i, int nv, int chunks, const double* __restrict__ part,
                                               const int* __restrict__ F, const int* __restrict__ ptr,
                                               const int* __restrict__ inc, const double* __restrict__ corr,
                                               double eps, const double* __restrict__ u, double* __restrict__ Au) {
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

}  // namespace ff
}  // namespace hobi
